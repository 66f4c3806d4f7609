"""lbmd_particle_sums_static: the particle momentum / kinetic-energy sums of
lbmd_observables for callers that cannot allocate device memory (for example
code running while a framework captures its stream into a CUDA graph, or code
inside a framework whose caching allocator owns the device memory).  It keeps
its scratch in a fixed __device__ array instead of calling cudaMalloc.

Checked through the C ABI against the existing entry point on two calls in a
row (the second sees different velocities and reuses the scratch).  This file
is collected last on purpose."""
import numpy as np
import pytest

pytestmark = pytest.mark.gpu


def test_particle_sums_static_matches_observables_twice():
    torch = pytest.importorskip("torch")
    from paper_1610_02733_gb300 import inputs, lbmd

    assert torch.cuda.is_available()
    shape, n, kT = (16, 16, 16), 20000, 1e-3
    g = lbmd.LBMD(*shape, variant="B", n_sub=5, kT=kT, zeta=1.0, seed=3, max_particles=n)
    # masses 1, 2 or 4: their reciprocals are exact in the FP32 particle
    # storage, so both entry points sum exactly the same values
    mass = 2.0 ** np.floor(inputs.uniform(n, 0.0, 3.0, 3))
    g.add_particles(inputs.uniform_positions(n, shape, 3), inputs.maxwell_velocities(n, kT, 3, mass), mass)
    # device buffers are the caller's: allocated here by the test, not by the entry point
    vel = torch.empty(3 * n, dtype=torch.float64, device="cuda")
    m = torch.tensor(mass, dtype=torch.float64, device="cuda")
    out = torch.empty(4, dtype=torch.float64, device="cuda")
    for call in range(2):
        g.cycle(1)
        g.particles_device(None, vel)
        lbmd.lbmd_particle_sums_static(vel.data_ptr(), m.data_ptr(), n, out.data_ptr(), g.stream)
        torch.cuda.synchronize()
        got = out.cpu().numpy()
        ob = g.observables()
        want = np.concatenate([ob["p_particles"], [2.0 * ob["e_kin"]]])
        scale = np.abs(want).max()
        assert np.abs(got - want).max() <= 1e-12 * scale, (call, got, want)


def test_particle_sums_static_edge_cases_and_no_allocation():
    torch = pytest.importorskip("torch")
    from paper_1610_02733_gb300 import inputs, lbmd

    shape, n, kT = (12, 12, 12), 5000, 1e-3
    g = lbmd.LBMD(*shape, variant="B", n_sub=2, kT=kT, zeta=1.0, seed=4, max_particles=n)
    g.add_particles(inputs.uniform_positions(n, shape, 4), inputs.maxwell_velocities(n, kT, 4))
    g.cycle(1)
    vel = torch.empty(3 * n, dtype=torch.float64, device="cuda")
    out = torch.full((4,), float("nan"), dtype=torch.float64, device="cuda")
    g.particles_device(None, vel)
    # n = 0: no partial-sum block runs, the sums are zero
    lbmd.lbmd_particle_sums_static(vel.data_ptr(), 0, 0, out.data_ptr(), g.stream)
    torch.cuda.synchronize()
    assert np.array_equal(out.cpu().numpy(), np.zeros(4))
    # mass NULL: unit masses, as in the context
    lbmd.lbmd_particle_sums_static(vel.data_ptr(), 0, n, out.data_ptr(), g.stream)
    torch.cuda.synchronize()
    ob = g.observables()
    want = np.concatenate([ob["p_particles"], [2.0 * ob["e_kin"]]])
    assert np.abs(out.cpu().numpy() - want).max() <= 1e-12 * np.abs(want).max()
    # no device memory taken by a call (after the first one, which has loaded
    # the kernels' module)
    torch.cuda.synchronize()
    free0 = torch.cuda.mem_get_info()[0]
    lbmd.lbmd_particle_sums_static(vel.data_ptr(), 0, n, out.data_ptr(), g.stream)
    torch.cuda.synchronize()
    assert torch.cuda.mem_get_info()[0] == free0
    g.close()


def test_particle_sums_static_rejects_oversize():
    from paper_1610_02733_gb300 import lbmd
    with pytest.raises(lbmd.LbmdError) as ei:
        lbmd.lbmd_particle_sums_static(0x1000, 0, 4194305, 0x2000)
    assert ei.value.status == lbmd.LBMD_ERR_CAPACITY
