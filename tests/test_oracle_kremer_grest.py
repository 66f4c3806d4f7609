"""Pins of the oracle's Kremer-Grest interactions (Sec. 4): Lennard-Jones
between all beads, cut off at 2^(7/6) sigma and shifted to zero there, FENE
springs along the chains, and the LJ-unit conversion of the paper's test.

They fix the potentials by textbook values (the LJ minimum -epsilon at
2^(1/6) sigma, the force 24 epsilon / sigma at r = sigma, FENE's harmonic
limit against the separately pinned harmonic bond, the Kremer-Grest bond
length), tie the forces to finite differences of the energies, and check
momentum and (without the fluid coupling) energy conservation of the
integrator with these forces."""
import numpy as np
import pytest

from oracle import oracle as orc
from paper_1610_02733_gb300 import inputs, lj_units

RC = 2.0 ** (7.0 / 6.0)
BOX = (9, 8, 10)


def _pair(r, direction=(0.3, -0.5, 0.8), centre=(4.1, 3.7, 5.2), eps=1.0, sigma=1.0, rc=RC, fene=None):
    o = orc.Oracle(*BOX)
    u = np.asarray(direction) / np.linalg.norm(direction)
    c = np.asarray(centre)
    o.add_particles(np.stack([c - 0.5 * r * u, c + 0.5 * r * u]), np.zeros((2, 3)))
    o.set_lj(eps, sigma, rc)
    if fene is not None:
        o.add_fene_bonds(np.array([[0, 1]]), *fene)
    return o, u


def test_lj_textbook_points():
    eps, sigma = 0.7, 1.1
    rmin = 2.0 ** (1.0 / 6.0) * sigma
    o, u = _pair(rmin, eps=eps, sigma=sigma, rc=RC * sigma)
    F, E = o.conservative_forces()
    assert np.abs(F).max() < 1e-13  # force-free at the minimum
    e_min = E["lj"]
    o, u = _pair(sigma, eps=eps, sigma=sigma, rc=RC * sigma)
    F, E = o.conservative_forces()
    # U(sigma) = 0 before the shift, U(r_min) = -eps: the shift cancels
    assert e_min - E["lj"] == pytest.approx(-eps, rel=1e-13)
    # |F(sigma)| = 24 eps / sigma, repulsive: particle 0 pushed along -u
    assert F[0] @ u == pytest.approx(-24.0 * eps / sigma, rel=1e-13)
    assert np.allclose(F[0], -F[1], rtol=0, atol=1e-15)
    # continuous energy at the cut-off (the shift), nothing beyond it
    o, _ = _pair(RC * sigma * (1 - 1e-9), eps=eps, sigma=sigma, rc=RC * sigma)
    assert abs(o.conservative_forces()[1]["lj"]) < 1e-8
    o, _ = _pair(RC * sigma * (1 + 1e-9), eps=eps, sigma=sigma, rc=RC * sigma)
    F, E = o.conservative_forces()
    assert E["lj"] == 0.0 and not F.any()


def test_minimum_image_across_the_boundary():
    # the same pair, once in the middle of the box and once split by the
    # periodic face x = 0 / x = 9
    o1, _ = _pair(1.05, direction=(1, 0.2, 0.1), centre=(4.5, 4.0, 5.0))
    o2, _ = _pair(1.05, direction=(1, 0.2, 0.1), centre=(0.1, 4.0, 5.0))
    F1, E1 = o1.conservative_forces()
    F2, E2 = o2.conservative_forces()
    assert np.allclose(F1, F2, rtol=1e-12, atol=0) and E1["lj"] == pytest.approx(E2["lj"], rel=1e-12)


def test_fene_harmonic_limit_and_divergence():
    k, R0 = 30.0, 1.5
    for r in (1e-2, 2e-2):
        of, u = _pair(r, eps=0.0, fene=(k, R0))
        oh = orc.Oracle(*BOX)
        oh.add_particles(of.particles()[0], np.zeros((2, 3)))
        oh.add_bonds(np.array([[0, 1]]), k, 0.0)  # harmonic, rest length 0
        Ff, Ef = of.conservative_forces()
        Fh, Eh = oh.conservative_forces()
        # FENE = harmonic (k, r0 = 0) to relative order (r / R0)^2
        x = (r / R0) ** 2
        assert np.abs(Ff - Fh).max() <= 1.01 * x * np.abs(Fh).max()
        assert abs(Ef["fene"] - Eh["harmonic"]) <= 0.6 * x * Eh["harmonic"]
    # energy grows without bound towards R0, force undefined beyond it
    e = [_pair(R0 * (1 - d), eps=0.0, fene=(k, R0))[0].conservative_forces()[1]["fene"] for d in (1e-2, 1e-4, 1e-6)]
    assert e[0] < e[1] < e[2] and e[2] - e[1] == pytest.approx(0.5 * k * R0 ** 2 * np.log(100.0), rel=1e-3)
    F, _ = _pair(R0 * 1.01, eps=0.0, fene=(k, R0))[0].conservative_forces()
    assert np.isnan(F).all()


def test_kremer_grest_bond_length():
    # FENE (k = 30, R0 = 1.5) + LJ: the bond rests at about 0.96-0.97 sigma
    # (Kremer & Grest), where the FENE pull balances the LJ repulsion
    def pull(r):
        o, u = _pair(r, fene=(lj_units.K_FENE, lj_units.R0_FENE))
        return o.conservative_forces()[0][0] @ u  # > 0: particle 0 pulled towards 1
    lo, hi = 0.9, 1.05
    assert pull(lo) < 0 < pull(hi)
    for _ in range(60):
        mid = 0.5 * (lo + hi)
        lo, hi = (mid, hi) if pull(mid) < 0 else (lo, mid)
    assert 0.95 < lo < 0.98


def _chain_system(n_sub=1, zeta=0.0, kT=0.0, seed=4, eps=1.0, v_kT=0.05):
    pos, bonds = inputs.self_avoiding_chains(3, 10, BOX, seed)
    o = orc.Oracle(*BOX, n_sub=n_sub, zeta=zeta, kT=kT, seed=seed)
    o.add_particles(pos, inputs.maxwell_velocities(pos.shape[0], v_kT, seed))
    o.set_lj(eps, 1.0, RC)
    o.add_fene_bonds(bonds, 30.0 * eps, 1.5)
    o.add_bonds(bonds[:3], 5.0, 1.0)  # a few harmonic bonds on top
    return o


def test_forces_are_minus_energy_gradient():
    o = _chain_system()
    pos0, vel0 = o.particles()
    F, _ = o.conservative_forces()
    h = 1e-6

    def energy(p):
        o.set_particles(p, None)
        return sum(o.conservative_forces()[1].values())
    for i, a in ((0, 0), (4, 1), (17, 2), (29, 0)):
        pp, pm = pos0.copy(), pos0.copy()
        pp[i, a] += h
        pm[i, a] -= h
        fd = -(energy(pp) - energy(pm)) / (2 * h)
        assert F[i, a] == pytest.approx(fd, rel=1e-6, abs=1e-7 * np.abs(F).max())


def test_newtons_third_law():
    o = _chain_system()
    F, E = o.conservative_forces()
    assert E["lj"] != 0.0 and E["fene"] > 0.0 and E["harmonic"] > 0.0
    assert np.abs(F.sum(axis=0)).max() <= 1e-12 * np.abs(F).max()


def test_energy_conservation_is_second_order_in_dt():
    # no coupling (zeta = 0, kT = 0): velocity Verlet with the conservative
    # forces alone; the energy error scales as dt^2 (epsilon = 0.01 makes the
    # LJ time 10 lattice units: dt = 0.04 and 0.02 are 0.004 and 0.002 tau)
    err = []
    for m in (25, 50):
        o = _chain_system(n_sub=m, eps=0.01, v_kT=0.005)
        pos, vel = o.particles()

        def total():
            p, v = o.particles()
            return 0.5 * float((v ** 2).sum()) + sum(o.conservative_forces()[1].values())
        e0, worst = total(), 0.0
        for _ in range(2):
            for _ in range(m):
                o.md_substep()
                worst = max(worst, abs(total() - e0))
            o.lb_step()
        err.append(worst)
    assert err[1] > 0 and 3.0 < err[0] / err[1] < 5.0


def test_lj_unit_conversion_invariants():
    for m, dt, zeta in ((1, 0.001, 1.0), (5, 0.005, 5.0), (10, 0.01, 20.0)):
        p = lj_units.lattice_params(m, dt, zeta)
        assert p["n_sub"] == m
        # friction per MD step, zeta dt / mu, is the same in both unit systems
        assert p["zeta"] * (1.0 / m) == pytest.approx(zeta * dt, rel=1e-14)
        # k_B T = epsilon, thermal speed (kT/mu)^(1/2) = 1 sigma/tau
        assert p["kT"] / p["lj_eps"] == pytest.approx(1.0, rel=1e-14)
        assert np.sqrt(p["kT"]) / p["velocity_scale"] == pytest.approx(1.0, rel=1e-14)
        # momentum diffusion time across sigma: sigma^2 / nu = tau / 3
        assert (1.0 / p["nu"]) * p["tau_lb"] == pytest.approx(1.0 / 3.0, rel=1e-14)
        assert lj_units.temperature_in_lj(p["kT"], p) == pytest.approx(1.0, rel=1e-14)
