"""Pins of the oracle's full LB/MD update against closed forms and invariants.

* Shear-wave decay.  At nu = 1/6 every non-conserved mode relaxes fully, so a
  linear shear wave u_x = U sin(k y) decays per LB step by exactly
  (2 + cos k) / 3 (worked out by hand from streaming the linear equilibrium);
  at other viscosities the decay approaches the continuum exp(-nu k^2).
* A uniform body force g adds exactly g per node per LB step (Eq. (3) with
  Delta'_i).
* Mass is conserved exactly, total (fluid + pending transfer + particle)
  momentum at every MD step, for both variants (Sec. 3).
* Variant B keeps the momentum the particles see conserved at every MD step;
  variant A does not (Sec. 3).
* At m = 1 variants A and B coincide (Sec. 3).
* Trilinear weights (Eq. (5)) sum to one and reproduce linear fields.
* One ideal particle in a fluid at rest, kT = 0: v' = v (1 - zeta dt / m)
  after one MD step, and the fluid gains exactly -Delta P (Eqs. (6)-(8)).
"""
import numpy as np
import pytest

from paper_1610_02733_gb300 import inputs


def _feq(c, w, rho, u):
    cu = u @ c.T  # (n, 19)
    uu = (u * u).sum(axis=1)
    return (w[None, :] * rho[:, None] * (1 + 3 * cu + 4.5 * cu ** 2 - 1.5 * uu[:, None])).T


def _shear_wave_state(orc, L, U):
    c, w = orc.d3q19()
    c = c.astype(float)
    n = L ** 3
    idx = np.arange(n)
    y = (idx // L) % L
    k = 2 * np.pi / L
    u = np.zeros((n, 3))
    u[:, 0] = U * np.sin(k * y)
    return _feq(c, w, np.ones(n), u), np.sin(k * y), k


def _jx_amplitude(o, profile):
    nf = o.node_field()
    return (nf[:, 1] * profile).sum() / (profile * profile).sum()


@pytest.mark.parametrize("L", [16, 32])
def test_shear_wave_exact_decay_at_nu_one_sixth(orc, L):
    f0, prof, k = _shear_wave_state(orc, L, 1e-6)
    o = orc.Oracle(L, L, L, n_sub=1, nu=1.0 / 6.0, kT=0.0)
    o.set_populations(f0)
    a0 = _jx_amplitude(o, prof)
    lam = (2.0 + np.cos(k)) / 3.0
    for step in range(3):
        o.md_substep()
        o.lb_step()
        a1 = _jx_amplitude(o, prof)
        assert abs(a1 / a0 - lam) < 1e-9
        a0 = a1


@pytest.mark.parametrize("nu", [0.05, 0.5])
def test_shear_wave_continuum_viscosity(orc, nu):
    # Away from nu = 1/6 the lattice decay rate equals nu k^2 up to a
    # second-order lattice correction: the relative error must shrink four-fold
    # when k halves, and the Richardson-extrapolated rate must match nu k^2.
    errs = {}
    for L in (16, 32):
        f0, prof, k = _shear_wave_state(orc, L, 1e-6)
        o = orc.Oracle(L, L, L, n_sub=1, nu=nu, kT=0.0)
        o.set_populations(f0)
        amps = []
        for step in range(60):
            o.md_substep()
            o.lb_step()
            amps.append(_jx_amplitude(o, prof))
        rate = np.log(amps[20] / amps[59]) / 39.0
        errs[L] = rate / (nu * k * k) - 1.0
    assert abs(errs[32]) < 0.02
    assert 3.5 < errs[16] / errs[32] < 4.6
    assert abs((4.0 * errs[32] - errs[16]) / 3.0) < 0.006


def test_body_force_momentum_and_uniform_flow(orc):
    g = np.array([1e-5, -2e-5, 3e-6])
    o = orc.Oracle(6, 5, 4, n_sub=3, body_force=g, kT=0.0)
    n = 6 * 5 * 4
    for step in range(1, 6):
        o.cycle(1)
        ob = o.observables()
        np.testing.assert_allclose(ob["p_fluid"], step * g * n, rtol=0, atol=1e-14 * n * step)
        nf = o.node_field()
        np.testing.assert_allclose(nf[:, 1:], np.broadcast_to(step * g, (n, 3)), rtol=1e-11)
        np.testing.assert_allclose(nf[:, 0], 1.0, rtol=0, atol=1e-14)


def _system(orc, variant, n_sub, kT=1e-4, zeta=1.0, shape=(8, 8, 8), n=10, seed=1):
    o = orc.Oracle(*shape, n_sub=n_sub, variant=variant, kT=kT, zeta=zeta, seed=seed)
    pos = inputs.uniform_positions(n, shape, seed)
    vel = inputs.maxwell_velocities(n, max(kT, 1e-4), seed)
    o.add_particles(pos, vel)
    return o


@pytest.mark.parametrize("variant", [0, 1])
def test_conservation_every_md_step(orc, variant):
    o = _system(orc, variant, 5, kT=1e-3, zeta=2.0, n=30)
    ob0 = o.observables()
    p0 = ob0["p_fluid"] + ob0["p_particles"]
    scale = np.abs(o.particles()[1]).sum() + 1.0
    for cyc in range(4):
        for s in range(5):
            assert o.md_substep() == 0
            ob = o.observables()
            assert abs(ob["mass"] - ob0["mass"]) <= 1e-13 * ob0["mass"]
            np.testing.assert_allclose(ob["p_fluid"] + ob["p_particles"], p0, rtol=0, atol=1e-14 * scale)
        assert o.lb_step() == 0
        ob = o.observables()
        assert abs(ob["mass"] - ob0["mass"]) <= 1e-13 * ob0["mass"]
        np.testing.assert_allclose(ob["p_fluid"] + ob["p_particles"], p0, rtol=0, atol=1e-14 * scale)


def test_seen_momentum_conserved_per_md_step_only_in_b(orc):
    # momentum the particles see (node field) + particle momentum
    res = {}
    for variant in (0, 1):
        o = _system(orc, variant, 5, kT=1e-3, zeta=2.0, n=30)
        o.cycle(2)
        def seen():
            return o.node_field()[:, 1:].sum(axis=0) + o.observables()["p_particles"]
        p0 = seen()
        drift = 0.0
        for s in range(5):
            o.md_substep()
            drift = max(drift, np.abs(seen() - p0).max())
        res[variant] = drift
    assert res[1] < 1e-14
    assert res[0] > 1e-6


def test_variants_coincide_at_m_equal_one(orc):
    oa = _system(orc, 0, 1, kT=1e-3, zeta=3.0, n=25)
    ob = _system(orc, 1, 1, kT=1e-3, zeta=3.0, n=25)
    oa.cycle(6)
    ob.cycle(6)
    np.testing.assert_array_equal(oa.populations(), ob.populations())
    pa, va = oa.particles()
    pb, vb = ob.particles()
    np.testing.assert_array_equal(pa, pb)
    np.testing.assert_array_equal(va, vb)


def test_variants_differ_at_m_above_one(orc):
    oa = _system(orc, 0, 5, kT=1e-3, zeta=3.0, n=25)
    ob = _system(orc, 1, 5, kT=1e-3, zeta=3.0, n=25)
    oa.cycle(2)
    ob.cycle(2)
    assert np.abs(oa.particles()[1] - ob.particles()[1]).max() > 1e-8


def test_trilinear_weights(orc):
    L = (7, 6, 5)
    o = orc.Oracle(*L)
    pts = inputs.uniform_positions(200, L, 3)
    pts = np.vstack([pts, [[0, 0, 0], [6.999999, 5.5, 0.0], [3.0, 2.0, 1.0]]])
    for R in pts:
        corner, delta = o.trilinear(R)
        assert abs(delta.sum() - 1.0) < 1e-15
        assert np.all(delta >= 0)
        # linear reproduction on the unwrapped cube: sum delta_k r_k = R
        base = np.floor(R)
        offs = np.array([[k & 1, (k >> 1) & 1, (k >> 2) & 1] for k in range(8)], dtype=float)
        np.testing.assert_allclose(delta @ (base + offs), R, rtol=0, atol=1e-13)
        # corner indices are the wrapped cube corners
        cc = (base[None, :] + offs).astype(int) % np.array(L)
        want = cc[:, 0] + L[0] * (cc[:, 1] + L[1] * cc[:, 2])
        np.testing.assert_array_equal(corner, want)
    # a particle exactly on a node puts weight 1 on that node
    corner, delta = o.trilinear(np.array([3.0, 2.0, 1.0]))
    assert delta[0] == 1.0 and corner[0] == 3 + 7 * (2 + 6 * 1)


@pytest.mark.parametrize("variant", [0, 1])
def test_single_particle_one_step_closed_form(orc, variant):
    zeta, n_sub, m = 0.7, 4, 2.5
    o = orc.Oracle(6, 6, 6, n_sub=n_sub, variant=variant, kT=0.0, zeta=zeta)
    v0 = np.array([0.01, -0.02, 0.005])
    R0 = np.array([2.3, 4.9, 0.1])
    o.add_particles(R0[None], v0[None], np.array([m]))
    o.md_substep()
    dt = 1.0 / n_sub
    pos, vel = o.particles()
    np.testing.assert_allclose(vel[0], v0 * (1 - zeta * dt / m), rtol=1e-14)
    # drift with the half-kicked velocity
    np.testing.assert_allclose(pos[0], R0 + dt * v0 * (1 - 0.5 * zeta * dt / m), rtol=1e-14)
    dP = -zeta * dt * v0
    np.testing.assert_allclose(o.jacc().sum(axis=0), -dP, rtol=1e-13)
    corner, delta = o.trilinear(R0)
    J = o.jacc()
    for k in range(8):
        np.testing.assert_allclose(J[corner[k]], -delta[k] * dP, rtol=1e-12, atol=1e-20)


def test_momentum_exchange_reaches_common_velocity(orc):
    # kT = 0: a particle moving through a fluid at rest; total momentum is
    # conserved, and both relax towards the common velocity P / (M + m).
    o = orc.Oracle(4, 4, 4, n_sub=2, variant=1, kT=0.0, zeta=1.0)
    v0 = np.array([0.05, 0.0, -0.03])
    o.add_particles(np.array([[1.5, 1.5, 1.5]]), v0[None])
    o.cycle(400)
    M = 64.0 + 1.0
    pos, vel = o.particles()
    np.testing.assert_allclose(vel[0], v0 / M, rtol=1e-3, atol=1e-8)
    ob = o.observables()
    np.testing.assert_allclose(ob["p_fluid"] + ob["p_particles"], v0, rtol=0, atol=1e-13)


def _oscillator_energy_error(orc, n_sub):
    o = orc.Oracle(8, 8, 8, n_sub=n_sub, variant=1, kT=0.0, zeta=0.0)
    o.add_particles(np.array([[7.6, 1.0, 1.0], [0.8, 1.0, 1.0]]), np.zeros((2, 3)))
    o.add_bonds(np.array([[0, 1]]), 30.0, 1.0)
    e0 = 0.5 * 30.0 * 0.2 ** 2
    emax = 0.0
    for cyc in range(2):
        for s in range(n_sub):
            o.md_substep()
            pos, vel = o.particles()
            np.testing.assert_allclose(vel[0] + vel[1], 0.0, atol=1e-15)
            d = pos[1] - pos[0]
            d -= 8 * np.round(d / 8)
            r = np.linalg.norm(d)
            e = 0.5 * (vel ** 2).sum() + 0.5 * 30.0 * (r - 1.0) ** 2
            emax = max(emax, abs(e / e0 - 1.0))
            if cyc == 0 and s == 0:
                assert vel[0, 0] > 0 and vel[1, 0] < 0  # the stretched spring pulls
        o.lb_step()
    return emax


def test_bond_forces_conserve_momentum_and_energy(orc):
    # Two beads on a harmonic bond (k = 30, r0 = 1) across the periodic
    # boundary, no friction: momentum stays zero, and velocity Verlet keeps
    # the oscillator energy within O((omega dt)^2) of its initial value, the
    # error shrinking four-fold when dt halves.
    e20 = _oscillator_energy_error(orc, 20)
    e40 = _oscillator_energy_error(orc, 40)
    assert e20 < 0.06
    assert 3.3 < e20 / e40 < 4.7


def test_sequence_errors(orc):
    o = orc.Oracle(4, 4, 4, n_sub=2)
    assert o.lb_step() == orc.ORC_ERR_SEQUENCE
    assert o.md_substep() == 0
    assert o.lb_step() == orc.ORC_ERR_SEQUENCE
    assert o.md_substep() == 0
    assert o.md_substep() == orc.ORC_ERR_SEQUENCE
    assert o.lb_step() == 0


def test_fluid_equipartition(orc):
    # particle-free fluid at kT: <j_x^2> = rho kT (1 - 1/N) and the stress
    # modes of the post-stream populations have variance mu rho b_k.
    L, kT = 6, 1e-3
    o = orc.Oracle(L, L, L, n_sub=1, kT=kT, seed=11)
    e, b = orc.modes()
    o.cycle(150)
    j2, m2 = [], []
    for t in range(400):
        o.cycle(1)
        nf = o.node_field()
        j2.append((nf[:, 1:] ** 2).mean(axis=0))
        if t % 4 == 0:
            f = o.populations()
            m2.append(((e[4:10] @ f) ** 2).mean(axis=1))
    n = L ** 3
    jv = np.mean(j2) / (kT * (1 - 1.0 / n))
    assert abs(jv - 1.0) < 0.04
    mv = np.mean(m2, axis=0) / (3 * kT * b[4:10])
    np.testing.assert_allclose(mv, 1.0, atol=0.05)


def _mean_particle_temperature(o, burn, cycles):
    o.cycle(burn)
    T = []
    for t in range(cycles):
        o.cycle(1)
        T.append(o.observables()["kT_particles"])
    return np.mean(T)


def test_particle_noise_is_discrete_ornstein_uhlenbeck(orc):
    # A very dense fluid (rho0 = 1e6) is a bath at rest: each MD step is then
    # v' = v (1 - zeta dt / m) + dt sqrt(2 zeta kT / dt) xi / m, whose
    # stationary variance is kT / m / (1 - zeta dt / (2 m)) exactly.  This pins
    # the random-force amplitude of Eq. (4) and the explicit friction step.
    kT, zeta, n_sub, m = 1e-3, 2.0, 5, 1.0
    o = orc.Oracle(4, 4, 4, n_sub=n_sub, variant=1, kT=kT, zeta=zeta, rho0=1e6, seed=8)
    n = 200
    o.add_particles(inputs.uniform_positions(n, (4, 4, 4), 8), inputs.maxwell_velocities(n, kT, 8))
    ratio = _mean_particle_temperature(o, 20, 600) / kT
    want = 1.0 / (1.0 - zeta * (1.0 / n_sub) / (2.0 * m))
    assert abs(ratio / want - 1.0) < 0.02


def test_particle_temperature_variant_b_small_zeta_dt(orc):
    # ideal particles at small zeta dt: <m v^2>/3 -> kT (fluctuation-
    # dissipation of the coupling, Sec. 1 and Sec. 3)
    kT = 1e-3
    o = _system(orc, 1, 5, kT=kT, zeta=0.1, shape=(8, 8, 8), n=60, seed=4)
    ratio = _mean_particle_temperature(o, 200, 2500) / kT
    assert abs(ratio - 1.0) < 0.04


def test_variant_a_heats_up_more_than_b(orc):
    # Sec. 3: at large friction and time-scale ratio the lagging node
    # velocities of variant A heat the particles up; variant B much less.
    kT = 1e-3
    T = {}
    for variant in (0, 1):
        o = _system(orc, variant, 10, kT=kT, zeta=2.0, shape=(8, 8, 8), n=60, seed=4)
        T[variant] = _mean_particle_temperature(o, 100, 800) / kT
    assert T[0] - 1.0 > 2.0 * (T[1] - 1.0)
    assert T[0] - T[1] > 0.1
