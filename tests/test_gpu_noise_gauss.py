"""The Gaussian noise option on the GPU against the oracle: normal variates by
the Box-Muller transform of pairs of Philox words (device log and sincospi
against the oracle's C library, hence a tolerance rather than bits) for the
fluid modes (Sec. 2) and the particles' random force (Eq. (4))."""
import numpy as np
import pytest

from gpu_common import TOL, assert_pops_close, assert_vec_close, pair
from paper_1610_02733_gb300 import inputs, lbmd

pytestmark = pytest.mark.gpu


@pytest.mark.parametrize("precision", ["fp32", "fp64"])
def test_one_lb_step(precision):
    shape = (11, 7, 9)
    o, g = pair(shape, precision=precision, kT=1e-3, nu=0.11, nu_bulk=0.3, gamma_ghost=0.2,
                body_force=(1e-5, 0.0, -2e-5), seed=77, noise="gauss")
    f0 = inputs.perturbed(o.populations(), 0.05, 3)
    for obj in (o, g):
        obj.set_populations(f0)
        obj.md_substep()
        obj.lb_step()
    assert_pops_close(g.populations(), o.populations(), precision)
    o.close()
    g.close()


@pytest.mark.parametrize("precision", ["fp32", "fp64"])
@pytest.mark.parametrize("variant,integrator", [("A", "start"), ("B", "start"), ("B", "half_step"), ("C", "start")])
def test_coupled_cycles(precision, variant, integrator):
    shape, n = (12, 10, 8), 300
    o, g = pair(shape, precision=precision, variant=variant, n_sub=4, kT=1e-3, zeta=1.5, seed=21,
                max_particles=n, integrator=integrator, noise="gauss")
    pos, vel = inputs.uniform_positions(n, shape, 21), inputs.maxwell_velocities(n, 1e-3, 21)
    for obj in (o, g):
        obj.add_particles(pos, vel)
    o.cycle(3)
    g.run_cycles(3)
    assert_pops_close(g.populations(), o.populations(), precision)
    po, vo = o.particles()
    pg, vg = g.particles()
    d = pg - po
    d -= np.array(shape) * np.round(d / np.array(shape))
    assert np.abs(d).max() <= TOL[precision] * max(shape)
    assert_vec_close(vg, vo, precision, "velocities")
    o.close()
    g.close()


def test_spread_paths_and_replay_agree_bitwise():
    shape, n = (24, 20, 18), 4000
    runs = {}
    for spread, graph in (("rows", False), ("atomic", False), ("tiles", False), ("rows", True)):
        g = lbmd.LBMD(*shape, variant="B", n_sub=5, kT=1e-4, zeta=1.5, seed=3, max_particles=n, spread=spread,
                      noise="gauss")
        g.add_particles(inputs.uniform_positions(n, shape, 3), inputs.maxwell_velocities(n, 1e-4, 3))
        if graph:
            g.run_cycles(2)
        else:
            g.cycle(2)
        runs[spread, graph] = (g.populations(), *g.particles())
        g.close()
    for key in runs:
        for a, b in zip(runs[key], runs["rows", False]):
            np.testing.assert_array_equal(a, b)


def test_noise_option_arguments():
    for precision in ("fp16dev", "bf16dev_sr"):
        with pytest.raises(lbmd.LbmdError) as e:
            lbmd.LBMD(6, 6, 6, precision=precision, noise="gauss")
        assert e.value.status == lbmd.LBMD_ERR_ARG
    with pytest.raises(lbmd.LbmdError):
        lbmd.LBMD(6, 6, 6, noise=2)
