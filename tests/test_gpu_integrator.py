"""The HALF_STEP integrator (coupling force from the half-step velocity after
the drift, transfer around the new position) on the GPU against the FP64
oracle's integrator 1: ideal particles and Kremer-Grest chains, variants A, B
and C, FP32 and FP64, over several LB cycles (the last coupling force is
carried across the re-ordering of the particles at every LB step)."""
import numpy as np
import pytest

from gpu_common import TOL, W, assert_pops_close, assert_vec_close, pair
from paper_1610_02733_gb300 import inputs, lj_units

pytestmark = pytest.mark.gpu


def _periodic_diff(a, b, shape):
    d = a - b
    L = np.asarray(shape, dtype=float)
    return d - L * np.round(d / L)


@pytest.mark.parametrize("precision", ["fp32", "fp64"])
@pytest.mark.parametrize("variant", ["A", "B", "C"])
def test_ideal_particles_several_cycles(precision, variant):
    shape, n = (13, 10, 9), 300
    o, g = pair(shape, precision=precision, variant=variant, n_sub=5, kT=1e-4, zeta=2.0, seed=31, max_particles=n,
                integrator="half_step")
    pos, vel = inputs.uniform_positions(n, shape, 31), inputs.maxwell_velocities(n, 1e-4, 31)
    for obj in (o, g):
        obj.add_particles(pos, vel)
    for _ in range(3):
        o.cycle(1)
        g.cycle(1)
        assert_pops_close(g.populations(), o.populations(), precision)
        pg, vg = g.particles()
        po, vo = o.particles()
        assert np.abs(_periodic_diff(pg, po, shape)).max() <= TOL[precision] * max(shape)
        assert_vec_close(vg, vo, precision, "velocities")


@pytest.mark.parametrize("precision", ["fp32", "fp64"])
@pytest.mark.parametrize("variant", ["A", "B", "C"])
def test_kremer_grest_chains(precision, variant):
    shape, m, dt, zeta = (16, 12, 10), 5, 0.005, 5.0
    lp = lj_units.lattice_params(m, dt, zeta)
    pos, bonds = inputs.self_avoiding_chains(4, 32, shape, 32)
    n = pos.shape[0]
    o, g = pair(shape, precision=precision, variant=variant, n_sub=m, kT=lp["kT"], zeta=lp["zeta"], nu=lp["nu"],
                seed=32, max_particles=n, max_bonds=bonds.shape[0], integrator="half_step")
    vel = inputs.maxwell_velocities(n, lp["kT"], 32)
    for obj in (o, g):
        obj.add_particles(pos, vel)
        obj.set_lj(lp["lj_eps"], lp["lj_sigma"], lp["lj_rc"])
        obj.add_fene_bonds(bonds, lp["fene_k"], lp["fene_R0"])
    o.cycle(3)
    g.run_cycles(3)
    po, vo = o.particles()
    pg, vg = g.particles()
    tol = {"fp32": 1e-3, "fp64": 1e-9}[precision]
    assert np.abs(_periodic_diff(pg, po, shape)).max() < tol
    assert np.abs(vg - vo).max() < tol * np.abs(vo).max()
    err = np.abs(g.populations() - o.populations()) / W[:, None]
    assert float(err.max()) <= TOL[precision]


@pytest.mark.parametrize("precision", ["fp32", "fp64"])
def test_variants_a_and_b_coincide_bitwise_at_m_equal_one(precision):
    shape, n = (12, 10, 8), 50
    runs = {}
    for variant in ("A", "B"):
        _, g = pair(shape, precision=precision, variant=variant, n_sub=1, kT=1e-3, zeta=1.5, seed=9,
                    max_particles=n, integrator="half_step")
        g.add_particles(inputs.uniform_positions(n, shape, 2), inputs.maxwell_velocities(n, 1e-3, 2))
        g.cycle(5)
        runs[variant] = (g.populations(), *g.particles())
    for a, b in zip(runs["A"], runs["B"]):
        np.testing.assert_array_equal(a, b)


def test_graph_replay_equals_separate_calls():
    shape, n = (16, 12, 10), 200
    runs = []
    for graph in (False, True):
        _, g = pair(shape, precision="fp32", variant="B", n_sub=4, kT=1e-4, zeta=1.5, seed=33, max_particles=n,
                    integrator="half_step")
        g.add_particles(inputs.uniform_positions(n, shape, 33), inputs.maxwell_velocities(n, 1e-4, 33))
        if graph:
            g.run_cycles(4)
        else:
            g.cycle(4)
        runs.append((g.populations(), *g.particles()))
    for a, b in zip(*runs):
        np.testing.assert_array_equal(a, b)
