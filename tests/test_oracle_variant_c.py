"""Pins of the oracle's variant C (Sec. 4): after every MD step the
populations take that step's momentum transfer through the forcing part
Delta'_i of the collision alone (no relaxation, noise or streaming), with the
local streaming velocity u = (j + F/2)/rho."""
import numpy as np

from oracle import oracle as orc
from paper_1610_02733_gb300 import inputs

SHAPE = (6, 5, 4)


def _lattice():
    c, w = orc.d3q19()
    return np.asarray(c, dtype=float).reshape(19, 3), np.asarray(w)


def test_forcing_update_moments():
    # a random state and a random transfer field, no particles: one MD step
    # applies exactly the forcing update
    nu = 0.11
    o = orc.Oracle(*SHAPE, variant=2, n_sub=2, nu=nu)
    f0 = inputs.perturbed(o.populations(), 0.05, 1)
    o.set_populations(f0)
    F = inputs.uniform((o.n_nodes, 3), -1e-3, 1e-3, 2)
    o.set_jacc(F)
    o.md_substep()
    df = o.populations() - f0
    c, w = _lattice()
    rho = f0.sum(axis=0)
    j = c.T @ f0
    u = (j + 0.5 * F.T) / rho
    gs = (6 * nu - 1) / (6 * nu + 1)
    # mass unchanged, momentum + F exactly
    assert np.abs(df.sum(axis=0)).max() < 1e-15
    assert np.abs(c.T @ df - F.T).max() < 1e-15
    # second moment: (1 + gamma_s) / 2 (u F + F u) for the traceless part
    # (Guo's forcing term with the prefactor 1 - 1/(2 tau) = (1 + gamma)/2)
    for a in range(3):
        for b in range(3):
            got = (c[:, a, None] * c[:, b, None] * df).sum(axis=0)
            want = 0.5 * (1 + gs) * (u[a] * F[:, b] + u[b] * F[:, a])
            if a == b:  # trace part relaxes with gamma_bulk = 0: (u.F) (1 + 0) / 3 each
                trace_got = sum((c[:, d, None] ** 2 * df).sum(axis=0) for d in range(3))
                trace_want = (u * F.T).sum(axis=0) * 2 * 0.5  # (1 + gamma_b) u.F with gamma_b = 0
                assert np.abs(trace_got - trace_want).max() < 1e-15
                continue
            assert np.abs(got - want).max() < 1e-15
    # ghost modes untouched
    e, b = orc.modes()
    assert np.abs(e[10:] @ df).max() < 1e-15
    # and the transfer is consumed
    assert np.abs(o.jacc()).max() == 0.0


def _run(variant, n_sub, scale, cycles=2):
    o = orc.Oracle(*SHAPE, variant=variant, n_sub=n_sub, zeta=1.0, kT=0.0, nu=0.13, seed=3)
    pos = inputs.uniform_positions(6, SHAPE, 4)
    vel = scale * inputs.maxwell_velocities(6, 1.0, 4)
    o.add_particles(pos, vel)
    return o


def test_momentum_conserved_at_every_md_step():
    o = _run(2, 4, 0.05)
    p0 = None
    for _ in range(3):
        for _ in range(4):
            o.md_substep()
            ob = o.observables()
            p = ob["p_fluid"] + ob["p_particles"]
            if p0 is None:
                p0 = p
            assert np.abs(p - p0).max() < 1e-14
        o.lb_step()


def test_node_momentum_equals_variant_b():
    # the particles see j* + J_acc in B and the updated populations' j in C:
    # the same momentum (mass and density unchanged by the update)
    ob, oc = _run(1, 5, 0.05), _run(2, 5, 0.05)
    for _ in range(3):
        ob.md_substep()
        oc.md_substep()
        nb, nc = ob.node_field(), oc.node_field()
        assert np.abs(nb - nc).max() < 1e-14


def test_differs_from_b_only_at_second_order():
    # one MD step per LB step: C applies the forcing before the collision, B
    # inside it; the populations after the LB step differ by O(F^2)
    d = []
    for scale in (0.04, 0.02):
        ob, oc = _run(1, 1, scale), _run(2, 1, scale)
        for o in (ob, oc):
            o.md_substep()
            o.lb_step()
        d.append(np.abs(ob.populations() - oc.populations()).max())
    assert d[0] > 0 and 3.0 < d[0] / d[1] < 5.0
