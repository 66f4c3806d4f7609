"""Pins of the oracle's LB collision (Sec. 2 and the forcing term of Sec. 3).

* With every relaxation factor equal, the moment-space MRT collision with
  forcing must reduce to the textbook single-relaxation-time (BGK) collision
  with Guo's forcing term, written here directly in population space.
* The collision conserves mass and changes momentum by exactly F tau_LB,
  with or without thermal noise.
* A fluid in local equilibrium with no force is a fixed point of the
  deterministic collision, for any relaxation factors.
* The noise is a zero-mean perturbation of the non-conserved modes whose
  variance is mu rho b_k (1 - gamma_k^2), mu = 3 kT.
"""
import numpy as np
import pytest

from paper_1610_02733_gb300 import inputs


def _lattice(orc):
    c, w = orc.d3q19()
    return c.astype(float), w


def _feq(c, w, rho, u):
    """Textbook second-order equilibrium w_i rho (1 + 3 c.u + 9/2 (c.u)^2 - 3/2 u^2)."""
    cu = c @ u
    return w * rho * (1.0 + 3.0 * cu + 4.5 * cu ** 2 - 1.5 * (u @ u))


def _bgk_guo(c, w, f, F, tau):
    """Single-relaxation-time collision with Guo et al.'s forcing term:
    f' = f - (f - feq(rho, u)) / tau + (1 - 1/(2 tau)) w_i [3 (c_i - u) + 9 (c_i.u) c_i] . F,
    u = (j + F/2) / rho."""
    rho = f.sum()
    j = c.T @ f
    u = (j + 0.5 * F) / rho
    feq = _feq(c, w, rho, u)
    src = (1.0 - 0.5 / tau) * w * ((3.0 * (c - u) + 9.0 * (c @ u)[:, None] * c) @ F)
    return f - (f - feq) / tau + src


@pytest.mark.parametrize("nu", [1.0 / 6.0, 0.05, 0.5, 1.3])
def test_mrt_with_equal_rates_is_bgk_guo(orc, nu):
    c, w = _lattice(orc)
    g = (6 * nu - 1) / (6 * nu + 1)
    tau = 1.0 / (1.0 - g)
    # bulk viscosity 2 nu / 3 and ghost factor g give every mode the same rate
    o = orc.Oracle(4, 4, 4, nu=nu, nu_bulk=2.0 * nu / 3.0, gamma_ghost=g, kT=0.0)
    for seed in range(5):
        f = inputs.perturbed(w, 0.3, seed)
        F = inputs.uniform(3, -1e-2, 1e-2, seed)
        got = o.collide_node(f, F)
        want = _bgk_guo(c, w, f, F, tau)
        np.testing.assert_allclose(got, want, rtol=0, atol=1e-15)


def test_collision_invariants_with_noise(orc):
    c, w = _lattice(orc)
    o = orc.Oracle(4, 4, 4, nu=0.3, nu_bulk=0.2, gamma_ghost=0.4, kT=1e-3, seed=99)
    for node in range(20):
        f = inputs.perturbed(w * 1.1, 0.2, node)
        F = inputs.uniform(3, -1e-2, 1e-2, node)
        fp = o.collide_node(f, F, node=node, lb_step=3)
        assert abs(fp.sum() - f.sum()) < 1e-15
        np.testing.assert_allclose(c.T @ fp, c.T @ f + F, rtol=0, atol=1e-16)


def test_equilibrium_is_fixed_point(orc):
    c, w = _lattice(orc)
    for nu, nub, gg in [(1 / 6, -1, 0.0), (0.02, 0.7, 0.3), (0.9, 0.01, -0.5)]:
        o = orc.Oracle(4, 4, 4, nu=nu, nu_bulk=nub, gamma_ghost=gg, kT=0.0)
        u = np.array([0.03, -0.02, 0.01])
        feq = _feq(c, w, 1.05, u)
        # second-order feq is a fixed point of the relaxation of every mode
        np.testing.assert_allclose(o.collide_node(feq, np.zeros(3)), feq, rtol=0, atol=2e-16)


def test_noise_moments(orc):
    # Post-collision modes: m'_k - m'_k(kT=0) = sqrt(mu rho b_k (1 - g_k^2)) xi_k,
    # xi_k zero-mean unit-variance; conserved modes untouched.
    c, w = _lattice(orc)
    e, b = orc.modes()
    kT, nu, nub, gg = 2e-3, 0.25, 0.3, 0.2
    gs = (6 * nu - 1) / (6 * nu + 1)
    gb = (9 * nub - 1) / (9 * nub + 1)
    gam = np.array([0, 0, 0, 0, gb] + [gs] * 5 + [gg] * 9)
    o_hot = orc.Oracle(4, 4, 4, nu=nu, nu_bulk=nub, gamma_ghost=gg, kT=kT, seed=5)
    o_cold = orc.Oracle(4, 4, 4, nu=nu, nu_bulk=nub, gamma_ghost=gg, kT=0.0, seed=5)
    rho = 1.2
    f = w * rho
    samples = []
    for node in range(4000):
        d = e @ (o_hot.collide_node(f, np.zeros(3), node=node) - o_cold.collide_node(f, np.zeros(3), node=node))
        samples.append(d)
    s = np.array(samples)
    np.testing.assert_allclose(s[:, :4], 0.0, atol=1e-15)
    var = s[:, 4:].var(axis=0)
    want = 3 * kT * rho * b[4:] * (1 - gam[4:] ** 2)
    # 4000 samples of a uniform variable: relative sd of the variance ~ 1.4 %
    np.testing.assert_allclose(var / want, 1.0, atol=0.07)
    assert np.all(np.abs(s[:, 4:].mean(axis=0)) < 4 * np.sqrt(want / 4000))
