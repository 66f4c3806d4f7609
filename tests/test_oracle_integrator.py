"""Pins of the oracle's second reading of the MD integrator (integrator 1):
velocity Verlet that evaluates the coupling force of Eq. (4) where an MD code
evaluates its forces, after the drift, from the half-step velocity and the
node velocities interpolated at the new position; the momentum transfer of
Eqs. (7), (8) goes to the nodes around that position.

Pinned against: the exact stationary temperature of the discretised
Ornstein-Uhlenbeck process in a bath at rest (kT for the full-step velocity,
where integrator 0 gives kT / (1 - zeta dt / 2m)); a single particle's first
two steps in closed form; momentum conservation at every MD step once the
half of the last coupling impulse that the particle has not yet received is
counted; and A = B at m = 1."""
import numpy as np
import pytest

from oracle import oracle as orc
from paper_1610_02733_gb300 import inputs


def _mean_T(o, burn, cycles):
    o.cycle(burn)
    T = []
    for _ in range(cycles):
        o.cycle(1)
        T.append(o.observables()["kT_particles"])
    return float(np.mean(T))


def test_dense_bath_temperature_is_exact():
    # rho0 = 1e6: a bath at rest.  With u = 0 the half-step velocity obeys
    # w' = w (1 - zeta dt / m) + dt xi / m, stationary variance
    # kT / m / (1 - zeta dt / 2m); the full-step velocity v = w (1 - zeta dt / 2m)
    # + (dt / 2m) xi then has variance kT / m exactly.  Integrator 0 (the
    # explicit step from the start-of-step velocity) gives kT / (1 - zeta dt / 2m).
    kT, zeta, n_sub = 1e-3, 2.0, 5  # zeta dt = 0.4
    T = {}
    for integ in (0, 1):
        o = orc.Oracle(4, 4, 4, n_sub=n_sub, variant=1, kT=kT, zeta=zeta, rho0=1e6, seed=8, integrator=integ)
        n = 200
        o.add_particles(inputs.uniform_positions(n, (4, 4, 4), 8), inputs.maxwell_velocities(n, kT, 8))
        T[integ] = _mean_T(o, 20, 600) / kT
    assert abs(T[1] - 1.0) < 0.02
    assert abs(T[0] * (1.0 - 0.5 * zeta / n_sub) - 1.0) < 0.02


@pytest.mark.parametrize("variant", [0, 1, 2])
def test_single_particle_first_two_steps(variant):
    zeta, n_sub, m = 0.7, 4, 2.5
    dt = 1.0 / n_sub
    o = orc.Oracle(6, 6, 6, n_sub=n_sub, variant=variant, kT=0.0, zeta=zeta, integrator=1)
    v0 = np.array([0.01, -0.02, 0.005])
    R0 = np.array([2.3, 4.9, 0.1])
    o.add_particles(R0[None], v0[None], np.array([m]))
    # step 1: no previous force, drift with v0, friction from v0 at R1
    o.md_substep()
    R1 = R0 + dt * v0
    pos, vel = o.particles()
    np.testing.assert_allclose(pos[0], R1, rtol=1e-14)
    F1 = -zeta * v0
    np.testing.assert_allclose(o.coupling_forces()[0], F1, rtol=1e-14)
    np.testing.assert_allclose(vel[0], v0 + 0.5 * dt * F1 / m, rtol=1e-14)
    if variant != 2:  # C moves the transfer into the populations at once
        corner, delta = o.trilinear(R1)
        J = o.jacc()
        for k in range(8):
            np.testing.assert_allclose(J[corner[k]], -delta[k] * dt * F1, rtol=1e-12, atol=1e-20)
    # step 2: half kick with F1, drift; in variant A the fluid still looks at
    # rest (u = 0), so F2 = -zeta w2 with w2 the half-step velocity
    o.md_substep()
    w2 = vel[0] + 0.5 * dt * F1 / m
    R2 = R1 + dt * w2
    pos, vel = o.particles()
    np.testing.assert_allclose(pos[0], R2, rtol=1e-13)
    if variant == 0:
        F2 = -zeta * w2
        np.testing.assert_allclose(o.coupling_forces()[0], F2, rtol=1e-13)
        np.testing.assert_allclose(vel[0], w2 + 0.5 * dt * F2 / m, rtol=1e-13)


@pytest.mark.parametrize("variant", [0, 1, 2])
def test_momentum_with_pending_half_impulse(variant):
    # fluid + particles + dt/2 sum F_c (the half impulse each particle gets at
    # the start of its next step) is conserved at every MD step, bonds included
    n_sub = 4
    o = orc.Oracle(8, 7, 6, n_sub=n_sub, variant=variant, kT=1e-4, zeta=1.5, seed=5, integrator=1)
    pos, bonds = inputs.bead_spring_chains(3, 6, (8, 7, 6), 5)
    o.add_particles(pos, inputs.maxwell_velocities(pos.shape[0], 1e-3, 5))
    o.add_bonds(bonds, 2.0, 1.0)
    total = None
    for _ in range(3):
        for _ in range(n_sub):
            o.md_substep()
            ob = o.observables()
            p = ob["p_fluid"] + ob["p_particles"] + 0.5 / n_sub * o.coupling_forces().sum(axis=0)
            total = p if total is None else total
            assert np.abs(p - total).max() < 1e-14
        o.lb_step()


def test_variants_coincide_at_m_equal_one():
    runs = []
    for variant in (0, 1):
        o = orc.Oracle(6, 5, 4, n_sub=1, variant=variant, kT=1e-3, zeta=2.0, seed=3, integrator=1)
        o.add_particles(inputs.uniform_positions(12, (6, 5, 4), 3), inputs.maxwell_velocities(12, 1e-3, 3))
        o.cycle(4)
        runs.append((o.populations(), *o.particles()))
    for a, b in zip(*runs):
        np.testing.assert_array_equal(a, b)


def test_integrators_differ_only_at_order_dt():
    # same physics, different discretisation: after a fixed time the two
    # readings differ by O(dt) (halving dt halves the difference)
    d = []
    for n_sub in (4, 8):
        res = []
        for integ in (0, 1):
            o = orc.Oracle(6, 6, 6, n_sub=n_sub, variant=1, kT=0.0, zeta=1.0, seed=2, integrator=integ)
            o.add_particles(inputs.uniform_positions(10, (6, 6, 6), 2), inputs.maxwell_velocities(10, 1e-3, 2))
            o.cycle(3)
            res.append(o.particles()[1])
        d.append(float(np.abs(res[0] - res[1]).max()))
    assert 1.6 < d[0] / d[1] < 2.5
