"""The bead-spring configuration of the A-versus-B cost comparison at its own
size: a 64^3 periodic D3Q19 fluid (rho = 1, nu = 1/6, kT = 1e-4) with 64
random-walk chains of 64 beads (harmonic bonds k = 30, r0 = 1, mass 1,
zeta = 2), n = tau_LB / dt = 10 MD steps per LB step, variants A and B (Sec.
3), against the FP64 oracle on the same seeded inputs.

Three cycles: populations within 1e-5 (FP32) / 1e-12 (FP64) of w_i rho per
value after the first cycle, and positions and velocities within the
tolerances of the several-cycle bonded runs (the chains' dynamics is chaotic,
FP32 rounding grows): 1e-3 (FP32) / 1e-9 (FP64).
"""
import numpy as np
import pytest

from gpu_common import W, assert_pops_close, pair
from paper_1610_02733_gb300 import inputs

pytestmark = pytest.mark.gpu

SHAPE = (64, 64, 64)
N_CHAINS, N_BEADS = 64, 64


def _periodic_diff(a, b, shape):
    d = a - b
    L = np.array(shape, dtype=float)
    return d - L * np.round(d / L)


@pytest.mark.parametrize("precision", ["fp32", "fp64"])
@pytest.mark.parametrize("variant", ["A", "B"])
def test_bead_spring_64_cubed(precision, variant):
    pos, bonds = inputs.bead_spring_chains(N_CHAINS, N_BEADS, SHAPE, 2)
    n = pos.shape[0]
    vel = inputs.maxwell_velocities(n, 1e-4, 2)
    o, g = pair(SHAPE, precision=precision, variant=variant, n_sub=10, kT=1e-4, zeta=2.0, seed=12,
                max_particles=n, max_bonds=bonds.shape[0])
    for obj in (o, g):
        obj.add_particles(pos, vel)
        obj.add_bonds(bonds, 30.0, 1.0)
        obj.cycle(1)
    assert_pops_close(g.populations(), o.populations(), precision)
    for obj in (o, g):
        obj.cycle(2)
    tol = {"fp32": 1e-3, "fp64": 1e-9}[precision]
    po, vo = o.particles()
    pg, vg = g.particles()
    assert np.abs(_periodic_diff(pg, po, SHAPE)).max() < tol
    assert np.abs(vg - vo).max() < tol * np.abs(vo).max()
    err = np.abs(g.populations() - o.populations()) / W[:, None]
    assert err.max() < {"fp32": 1e-5, "fp64": 1e-11}[precision]
    ob_o, ob_g = o.observables(), g.observables()
    assert abs(ob_g["mass"] / ob_o["mass"] - 1) < {"fp32": 1e-6, "fp64": 1e-13}[precision]
    o.close()
    g.close()
