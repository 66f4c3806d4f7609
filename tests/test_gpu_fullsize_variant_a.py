"""Variant A at the benchmark's full size: 256^3 periodic D3Q19, 10^6 ideal
particles, m = 10, kT = 1e-4, zeta = 1, FP32.

At this size the node field does not fit in L2, so the MD steps interpolate
from a frozen copy of the active nodes' compact records (refreshed by the
post-stream moments of each LB step) and hand their transfers to a second,
accumulating copy.  The oracle runs every step of two cycles on the same
inputs: the first MD phase (fluid at rest), the whole LB step, and the second
MD phase, whose node velocities are the frozen post-stream ones.  After each
MD phase every particle and every node's pending transfer is compared.
"""
import numpy as np
import pytest

from paper_1610_02733_gb300 import inputs

pytestmark = pytest.mark.gpu

SHAPE = (256, 256, 256)
NP = 1_000_000
N_SUB = 10


@pytest.fixture(scope="module")
def states():
    from gpu_common import pair
    o, g = pair(SHAPE, precision="fp32", variant="A", n_sub=N_SUB, kT=1e-4, zeta=1.0, seed=1, max_particles=NP)
    pos = inputs.uniform_positions(NP, SHAPE, 1)
    vel = inputs.maxwell_velocities(NP, 1e-4, 1)
    o.add_particles(pos, vel)
    g.add_particles(pos, vel)
    yield o, g
    o.close()
    g.close()


def _md_phase(o, g):
    for _ in range(N_SUB):
        o.md_substep()
        g.md_substep()


def _compare(o, g):
    po, vo = o.particles()
    pg, vg = g.particles()
    d = pg - po
    d -= 256.0 * np.round(d / 256.0)
    assert np.abs(d).max() < 1e-4
    assert np.abs(vg - vo).max() <= 1e-5 * np.abs(vo).max()
    Jg, Jo = g.transfer(), o.jacc()
    assert np.abs(Jg - Jo).max() <= 1e-5 * np.abs(Jo).max()
    assert np.count_nonzero(np.abs(Jo).sum(axis=1)) > 0.3 * Jo.shape[0]


def test_variant_a_first_md_phase_full_size(states):
    o, g = states
    _md_phase(o, g)
    _compare(o, g)


def test_variant_a_second_cycle_full_size(states):
    # the LB step, then MD steps that read the frozen post-stream velocities
    o, g = states
    o.lb_step()
    g.lb_step()
    assert g.counts()["lb_step"] == 1
    _md_phase(o, g)
    _compare(o, g)
    ob = g.observables()
    assert abs(ob["mass"] / 256 ** 3 - 1.0) < 1e-6
