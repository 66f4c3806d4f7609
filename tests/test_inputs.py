"""The seeded input generators: reproducible, inside the box, with the
distributions and geometric constraints they promise (they hold none of the
method's arithmetic; these checks keep the parity cases meaningful)."""
import numpy as np

from paper_1610_02733_gb300 import inputs


def _min_image(d, L):
    return d - L * np.round(d / L)


def test_reproducible_and_in_the_box():
    shape = (7, 9, 11)
    a = inputs.uniform_positions(1000, shape, 3)
    assert np.array_equal(a, inputs.uniform_positions(1000, shape, 3))
    assert not np.array_equal(a, inputs.uniform_positions(1000, shape, 4))
    assert (a >= 0).all() and (a < np.asarray(shape)).all()


def test_maxwell_variance_per_mass():
    mass = np.where(np.arange(60000) % 2 == 0, 1.0, 4.0)
    v = inputs.maxwell_velocities(60000, 2e-3, 5, mass)
    for m in (1.0, 4.0):
        var = v[mass == m].var(axis=0)
        assert np.allclose(var, 2e-3 / m, rtol=0.03)


def test_self_avoiding_chains():
    shape = (12, 10, 9)
    pos, bonds = inputs.self_avoiding_chains(4, 40, shape, 7, bond=0.97, d_min=0.9)
    L = np.asarray(shape, dtype=float)
    assert pos.shape == (160, 3) and bonds.shape == (156, 2)
    assert (pos >= 0).all() and (pos < L).all()
    d = _min_image(pos[:, None, :] - pos[None, :, :], L)
    r = np.sqrt((d ** 2).sum(-1))
    np.fill_diagonal(r, np.inf)
    assert r.min() >= 0.9 - 1e-12
    bl = np.linalg.norm(_min_image(pos[bonds[:, 1]] - pos[bonds[:, 0]], L), axis=1)
    assert np.allclose(bl, 0.97, atol=1e-12)
    # bonds join consecutive beads of each chain only
    assert ((bonds[:, 1] - bonds[:, 0]) == 1).all() and not (bonds[:, 1] % 40 == 0).any()
    p2, _ = inputs.self_avoiding_chains(4, 40, shape, 7, bond=0.97, d_min=0.9)
    assert np.array_equal(pos, p2)


def test_replica_configs():
    c = inputs.replica_configs(64, 9)
    assert set(np.unique(c["dims"][:, 0])) <= {12, 16, 24, 32}
    assert (c["dims"][:, 0] == c["dims"][:, 1]).all() and (c["dims"][:, 0] == c["dims"][:, 2]).all()
    assert c["n_particles"].min() >= 1 and c["n_particles"].max() <= 400
    assert (c["zeta"] >= 0.5).all() and (c["zeta"] <= 5.0).all()
    assert set(np.unique(c["n_sub"])) <= {1, 5, 10}
    assert c["variant"][:4] == ["A", "B", "A", "B"]
