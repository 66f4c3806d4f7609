"""The asynchronous host accessors (uploads and downloads on streams of the
context's own, observables completed by synchronize) give bit for bit what the
synchronising accessors give at the same points of the stream order: in a
pipelined loop that uploads particles, runs a cycle and downloads the
particles and observables every step, with more queued observables than the
two slots (a slot reused before synchronize), mixed with synchronising calls,
with pageable numpy and pinned torch arrays; the checks of queued observables
(the fixed-point range flag) are reported by synchronize."""
import numpy as np
import pytest

from paper_1610_02733_gb300 import inputs, lbmd

pytestmark = pytest.mark.gpu

SHAPE = (20, 16, 12)


def _obs_equal(a, b):
    for k in ("mass", "kT_particles", "e_kin", "lb_step", "md_step"):
        assert a[k] == b[k], k
    for k in ("p_fluid", "p_particles"):
        np.testing.assert_array_equal(a[k], b[k])


def _make(variant, precision, n):
    g = lbmd.LBMD(*SHAPE, variant=variant, precision=precision, n_sub=5, kT=1e-4, zeta=1.0, seed=71, max_particles=n)
    g.add_particles(inputs.uniform_positions(n, SHAPE, 71), inputs.maxwell_velocities(n, 1e-4, 71))
    return g


@pytest.mark.parametrize("variant,precision", [("B", "fp32"), ("A", "fp32"), ("B", "fp64"), ("B", "bf16dev")])
@pytest.mark.parametrize("pinned", [False, True])
def test_pipelined_loop_equals_synchronous_calls(variant, precision, pinned):
    torch = pytest.importorskip("torch")
    n, steps = 300, 5
    uploads = [(np.ascontiguousarray(inputs.uniform_positions(n, SHAPE, 80 + k).reshape(-1)),
                np.ascontiguousarray(inputs.maxwell_velocities(n, 1e-4, 80 + k).reshape(-1))) for k in range(steps)]

    def host(a):
        return torch.from_numpy(a.copy()).pin_memory() if pinned else a.copy()

    def empty():
        return torch.empty(3 * n, dtype=torch.float64).pin_memory() if pinned else np.empty(3 * n)

    # synchronous twin
    s = _make(variant, precision, n)
    want = []
    for k in range(steps):
        s.set_particles(*uploads[k])
        s.run_cycles(1)
        o = s.observables()
        want.append((o, *s.particles()))
    f_want = s.populations()
    s.close()

    a = _make(variant, precision, n)
    up = [(host(p), host(v)) for p, v in uploads]
    outs = [(empty(), empty()) for _ in range(steps)]
    obs = []
    a.set_particles_async(*up[0])
    for k in range(steps):
        a.run_cycles(1)
        obs.append(a.observables_async())  # five queued: slots reused before synchronize
        a.particles_async(*outs[k])
        if k + 1 < steps:
            a.set_particles_async(*up[k + 1])
    a.synchronize()
    for k in range(steps):
        _obs_equal(lbmd.observables_dict(obs[k]), want[k][0])
        for got, w in zip(outs[k], want[k][1:]):
            got = got.numpy() if hasattr(got, "numpy") else got
            np.testing.assert_array_equal(got.reshape(n, 3), w)
    np.testing.assert_array_equal(a.populations(), f_want)
    a.close()


def test_mixed_with_synchronous_calls():
    n = 200
    s, a = _make("B", "fp32", n), _make("B", "fp32", n)
    for g in (s, a):
        g.run_cycles(1)
    o_async = a.observables_async()
    o_sync = a.observables()  # must not overwrite the queued sums before they are read
    pos, vel = np.empty(3 * n), np.empty(3 * n)
    a.particles_async(pos, vel)
    a.run_cycles(1)
    p_sync, v_sync = a.particles()  # after the cycle: the queued download holds the state before it
    a.synchronize()
    w0 = s.observables()
    wp, wv = s.particles()
    s.run_cycles(1)
    _obs_equal(lbmd.observables_dict(o_async), w0)
    _obs_equal(o_sync, w0)
    np.testing.assert_array_equal(pos.reshape(n, 3), wp)
    np.testing.assert_array_equal(vel.reshape(n, 3), wv)
    wp1, wv1 = s.particles()
    np.testing.assert_array_equal(p_sync, wp1)
    np.testing.assert_array_equal(v_sync, wv1)
    a.synchronize()  # nothing queued
    s.close()
    a.close()


def test_synchronize_reports_the_range_flag():
    g = lbmd.LBMD(6, 5, 4, variant="B", kT=0.0)
    rest = g.populations()
    f = rest.copy()
    f[1, 7] += 0.6
    f[2, 7] -= 0.6  # |j| = 1.2: beyond half the FP32 range
    g.observables_async()
    g.set_populations(f)
    g.observables_async()
    with pytest.raises(lbmd.LbmdError) as e:
        g.synchronize()
    assert e.value.status == lbmd.LBMD_ERR_RANGE
    g.set_populations(rest)
    o = g.observables_async()
    g.synchronize()
    _obs_equal(lbmd.observables_dict(o), g.observables())
    g.close()
