"""Pins of the oracle's Gaussian noise option (normal variates by the
Box-Muller transform of pairs of Philox words, instead of unit-variance
uniform ones; the amplitudes of Sec. 2 and Eq. (4) are the same).

The transform is pinned by distribution-level checks that a wrong radius,
angle, word or bit choice fails: the variates pass a Kolmogorov-Smirnov test
against the standard normal, the squared radius of a pair against the
exponential law of mean 2 and its angle against the uniform law, with the
normal's moments and no correlation inside a pair.  The fluid noise of the
collision then has the documented variance per mode, normal kurtosis, and
exactly the variates of the documented Philox words; the particles' random
force gives the discrete Ornstein-Uhlenbeck temperature of a bath at rest.
"""
import numpy as np
import pytest

from paper_1610_02733_gb300 import inputs

stats = pytest.importorskip("scipy.stats")


def _pairs(orc, n_calls, seed=(7, 3)):
    words = np.array([orc.philox4x32_10([i, 11, 5, 0], list(seed)) for i in range(n_calls)], dtype=np.uint64)
    w = words.reshape(-1, 2)
    return np.array([orc.box_muller(int(a), int(b)) for a, b in w])


def test_box_muller_is_standard_normal(orc):
    g = _pairs(orc, 20000)  # 40,000 pairs
    x = g.ravel()
    assert stats.kstest(x, "norm").pvalue > 1e-3
    assert abs(x.mean()) < 4 / np.sqrt(x.size)
    assert abs(x.var() - 1.0) < 4 * np.sqrt(2.0 / x.size)
    assert abs(stats.kurtosis(x, fisher=False) - 3.0) < 0.1
    assert abs(np.corrcoef(g[:, 0], g[:, 1])[0, 1]) < 4 / np.sqrt(g.shape[0])
    r2 = (g ** 2).sum(axis=1)
    assert stats.kstest(r2, "expon", args=(0, 2.0)).pvalue > 1e-3
    theta = np.arctan2(g[:, 1], g[:, 0])
    assert stats.kstest(theta, "uniform", args=(-np.pi, 2 * np.pi)).pvalue > 1e-3


def test_box_muller_special_words(orc):
    # top 24 bits h2 = 2^22 give u2 = 1/4 + 2^-25: the pair points along +y;
    # u1 -> 1 gives a radius -> 0, the smallest u1 a radius of ~5.7; u1 = 1/2
    # and u2 -> 0 the radius sqrt(2 ln 2) along +x
    a = orc.box_muller(0xFFFFFF00, (2 ** 22) << 8)
    assert np.hypot(*a) < 1e-3
    b = orc.box_muller(1 << 8, (2 ** 22) << 8)
    assert abs(b[0]) < 1e-5 * abs(b[1]) and b[1] > 5.0
    c = orc.box_muller(1 << 31, 0)  # u1 ~ 1/2, u2 ~ 0: along +x, radius sqrt(2 ln 2)
    assert abs(c[0] - np.sqrt(2 * np.log(2))) < 1e-6 and abs(c[1]) < 1e-6


def _mode_noise(orc, noise, n_nodes, kT=2e-3, rho=1.2):
    e, b = orc.modes()
    nu, nub, gg = 0.25, 0.3, 0.2
    gs = (6 * nu - 1) / (6 * nu + 1)
    gb = (9 * nub - 1) / (9 * nub + 1)
    gam = np.array([0, 0, 0, 0, gb] + [gs] * 5 + [gg] * 9)
    hot = orc.Oracle(4, 4, 4, nu=nu, nu_bulk=nub, gamma_ghost=gg, kT=kT, seed=5, noise=noise)
    cold = orc.Oracle(4, 4, 4, nu=nu, nu_bulk=nub, gamma_ghost=gg, kT=0.0, seed=5, noise=noise)
    _, w = orc.d3q19()
    f = w * rho
    d = np.array([e @ (hot.collide_node(f, np.zeros(3), node=k) - cold.collide_node(f, np.zeros(3), node=k))
                  for k in range(n_nodes)])
    amp = np.sqrt(3 * kT * rho * b * (1 - gam ** 2))
    return d, amp


def test_fluid_noise_modes_gauss(orc):
    d, amp = _mode_noise(orc, "gauss", 4000)
    np.testing.assert_allclose(d[:, :4], 0.0, atol=1e-15)
    xi = d[:, 4:] / amp[4:]
    np.testing.assert_allclose(xi.var(axis=0), 1.0, atol=0.1)
    assert np.all(np.abs(xi.mean(axis=0)) < 4 / np.sqrt(xi.shape[0]))
    kurt = stats.kurtosis(xi, axis=0, fisher=False)
    assert np.all(np.abs(kurt - 3.0) < 0.4), kurt  # uniform variates: 1.8
    # the uniform option keeps its flat distribution
    du, ampu = _mode_noise(orc, "uniform", 4000)
    assert np.all(np.abs(stats.kurtosis(du[:, 4:] / ampu[4:], axis=0, fisher=False) - 1.8) < 0.2)


def test_fluid_noise_words_gauss(orc):
    # node k's variates are Box-Muller pairs of the words of Philox calls
    # (k, lb_step, 0, q), q = 0..3, in mode order
    d, amp = _mode_noise(orc, "gauss", 6)
    for k in range(6):
        want = []
        for q in range(4):
            wds = orc.philox4x32_10([k, 0, 0, q], [5, 0])
            want += list(orc.box_muller(int(wds[0]), int(wds[1]))) + list(orc.box_muller(int(wds[2]), int(wds[3])))
        np.testing.assert_allclose(d[k, 4:] / amp[4:], want[:15], rtol=1e-12, atol=1e-12)


def test_particle_noise_gauss_is_discrete_ornstein_uhlenbeck(orc):
    # a bath at rest (rho0 = 1e6): v' = v (1 - zeta dt / m) + dt sqrt(2 zeta kT / dt) xi / m
    # has the stationary temperature kT / (1 - zeta dt / 2m) for any
    # unit-variance xi; and the velocity increments are normal
    kT, zeta, n_sub = 1e-3, 2.0, 5
    o = orc.Oracle(4, 4, 4, n_sub=n_sub, variant=1, kT=kT, zeta=zeta, rho0=1e6, seed=8, noise="gauss")
    n = 200
    o.add_particles(inputs.uniform_positions(n, (4, 4, 4), 8), inputs.maxwell_velocities(n, kT, 8))
    for _ in range(20):
        o.cycle(1)
    T, steps = [], []
    for _ in range(600):
        v0 = o.particles()[1].copy()
        o.md_substep()
        steps.append(o.particles()[1] - v0 * (1 - zeta / n_sub))
        for _ in range(n_sub - 1):
            o.md_substep()
        o.lb_step()
        T.append(o.observables()["kT_particles"])
    want = kT / (1.0 - zeta * (1.0 / n_sub) / 2.0)
    assert abs(np.mean(T) / want - 1.0) < 0.02
    xi = np.array(steps).ravel()
    xi /= xi.std()
    assert abs(stats.kurtosis(xi, fisher=False) - 3.0) < 0.15
