"""BASELINE's first configuration at its own size and length: 8^3 periodic
D3Q19, rho = 1, nu = 1/6, kT = 1e-4, fluid at rest, 10 ideal particles (mass
1, zeta = 1) at uniform random positions with Maxwellian velocities, m = 5,
1000 MD steps, Philox seed 1, FP64, variants A and B (Sec. 3) -- the whole
run against the oracle, element by element."""
import numpy as np
import pytest

from gpu_common import assert_pops_close, assert_vec_close, pair
from paper_1610_02733_gb300 import inputs

pytestmark = pytest.mark.gpu


@pytest.mark.parametrize("variant", ["A", "B"])
def test_config1_full_run(variant):
    shape, n, n_sub, kT = (8, 8, 8), 10, 5, 1e-4
    o, g = pair(shape, precision="fp64", variant=variant, n_sub=n_sub, kT=kT, zeta=1.0, seed=1, max_particles=n)
    pos, vel = inputs.uniform_positions(n, shape, 1), inputs.maxwell_velocities(n, kT, 1)
    for obj in (o, g):
        obj.add_particles(pos, vel)
    cycles = 1000 // n_sub
    o.cycle(cycles)
    g.run_cycles(cycles)
    assert g.observables()["md_step"] == 1000
    assert_pops_close(g.populations(), o.populations(), "fp64")
    po, vo = o.particles()
    pg, vg = g.particles()
    d = pg - po
    d -= 8.0 * np.round(d / 8.0)
    assert np.abs(d).max() < 1e-10
    assert_vec_close(vg, vo, "fp64", "velocities")
    ob_g, ob_o = g.observables(), o.observables()
    assert abs(ob_g["kT_particles"] / ob_o["kT_particles"] - 1.0) < 1e-10
    o.close()
    g.close()
