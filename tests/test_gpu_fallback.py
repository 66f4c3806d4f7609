"""The fused post-stream moments and their fallback.

The LB step's collide kernel computes the moments rho*, j* (Eqs. (1), (2)) of a
node row once the 27 collide blocks around that row have pushed; a block that
waits longer than its poll limit leaves the row to a follow-up kernel.  These
tests force that fallback -- for every row (poll limit 0) and for whichever
rows time out (poll limit 1) -- and require the results to be bitwise those
of the normal run and, through it, within the parity tolerances of the
oracle (Sec. 2 collision and streaming, Sec. 3 coupling, Sec. 4 variant C).
"""
import numpy as np
import pytest

from gpu_common import assert_pops_close, assert_vec_close, pair
from paper_1610_02733_gb300 import inputs, lbmd

pytestmark = pytest.mark.gpu

FUSE_LAG = 2  # the fused moments trail the push front by two planes


def _fused_rows(shape):
    """Collide blocks (rows of up to 256 nodes) whose moments the collide
    kernel itself computes: planes FUSE_LAG + 1 .. nz - 1 push the rows of
    planes 1 .. nz - 1 - FUSE_LAG."""
    nx, ny, nz = shape
    bx = 256 if nx >= 256 else (128 if nx >= 128 else (64 if nx >= 64 else 32))
    return ((nx + bx - 1) // bx) * ny * max(0, nz - 1 - FUSE_LAG)


def _state(g):
    pos, vel = g.particles()
    return g.populations(), g.node_field(), pos, vel


@pytest.mark.parametrize("precision", ["fp32", "fp64"])
@pytest.mark.parametrize("variant", ["A", "B", "C"])
def test_fallback_rows_give_the_fused_bits(precision, variant):
    shape, n, n_sub, cycles = (64, 64, 64), 4096, 2, 2
    pos = inputs.uniform_positions(n, shape, 21)
    vel = inputs.maxwell_velocities(n, 1e-4, 21)
    runs = {}
    for polls in (-1, 0, 1):
        o, g = pair(shape, precision=precision, variant=variant, n_sub=n_sub, kT=1e-4, zeta=1.0, seed=13,
                    max_particles=n)
        g.set_moments_wait(polls)
        g.add_particles(pos, vel)
        # one cycle call by call, the other replayed from the captured graph
        g.cycle(1)
        g.run_cycles(cycles - 1)
        runs[polls] = _state(g) + (g.moments_fallback_rows(),)
        if polls == -1:
            o.add_particles(pos, vel)
            o.cycle(cycles)
            assert_pops_close(runs[polls][0], o.populations(), precision)
            assert_vec_close(runs[polls][3], o.particles()[1], precision, "velocities")
        o.close()
        g.close()
    for polls in (0, 1):
        for a, b, what in zip(runs[polls][:4], runs[-1][:4], ("populations", "node field", "positions",
                                                              "velocities")):
            assert np.array_equal(a, b), "%s differ with poll limit %d" % (what, polls)
    # with no wait every fused row went to the follow-up kernel
    assert runs[0][4] == cycles * _fused_rows(shape)
    assert 0 <= runs[1][4] <= cycles * _fused_rows(shape)


@pytest.mark.parametrize("precision", ["fp32", "fp64"])
def test_fallback_one_lb_step_against_the_oracle(precision):
    # every row through the fallback, one LB step from a perturbed state,
    # element by element against the oracle
    shape = (70, 9, 11)  # ragged: one 64-node block plus a 6-node block per row
    o, g = pair(shape, precision=precision, variant="B", kT=1e-3, nu=0.11, body_force=(1e-5, 0.0, -2e-5), seed=5)
    g.set_moments_wait(0)
    f0 = inputs.perturbed(o.populations(), 0.05, 9)
    for obj in (o, g):
        obj.set_populations(f0)
        obj.md_substep()
        obj.lb_step()
    assert_pops_close(g.populations(), o.populations(), precision)
    nf_g, nf_o = g.node_field(), o.node_field()
    assert_vec_close(nf_g[:, 0], nf_o[:, 0], precision, "rho")
    assert_vec_close(nf_g[:, 1:], nf_o[:, 1:], precision, "j")
    assert g.moments_fallback_rows() == _fused_rows(shape)
    g.close()
    o.close()


def test_moments_wait_arguments():
    g = lbmd.LBMD(8, 8, 8, max_particles=0)
    with pytest.raises(lbmd.LbmdError):
        g.set_moments_wait(-2)
    g.set_moments_wait(5)
    g.set_moments_wait(-1)
    assert g.moments_fallback_rows() == 0
    g.close()
