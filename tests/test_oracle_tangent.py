"""Pins of the oracle's tangent (lbmd_tangent.c), the reference for the GPU
adjoint: its values are the plain oracle's results bit for bit (same
algorithm in dual numbers, same operation order), and its derivatives of the
drag sum S = sum over MD steps and particles of F_x (Eq. (4)) agree with
central finite differences of the plain oracle, which shares no derivative
code with it."""
import numpy as np
import pytest

from oracle import oracle as orc
from paper_1610_02733_gb300 import inputs

SHAPE = (6, 5, 4)
KW = dict(n_sub=3, nu=0.11, body_force=(2e-3, -1e-3, 5e-4), seed=7)


def _particles(n=5, seed=3):
    # away from cell faces, so that finite differences see a smooth map
    g = np.random.default_rng(seed)
    base = g.integers(0, min(SHAPE), size=(n, 3)).astype(float)
    return base + 0.3 + 0.4 * g.random((n, 3)), 0.02 * (g.random((n, 3)) - 0.5)


def _oracle_drag(zeta, pos, vel, cycles, variant, kT):
    o = orc.Oracle(*SHAPE, variant=variant, kT=kT, zeta=zeta, **KW)
    o.add_particles(pos, vel)
    S = 0.0
    for _ in range(cycles):
        for _ in range(KW["n_sub"]):
            o.md_substep()
            S += float(o.coupling_forces()[:, 0].sum())
        o.lb_step()
    return S, o


def _tangent(zeta, pos, vel, cycles, variant, kT, dpos=None, dzeta=0.0):
    t = orc.Tangent(*SHAPE, variant=variant, kT=kT, zeta=zeta, **KW)
    t.set_particles(pos, vel, dpos, dzeta)
    t.cycle(cycles)
    return t


@pytest.mark.parametrize("variant", [0, 1])
@pytest.mark.parametrize("kT", [0.0, 1e-4])
def test_values_equal_the_oracle(variant, kT):
    pos, vel = _particles()
    S, o = _oracle_drag(1.3, pos, vel, 2, variant, kT)
    t = _tangent(1.3, pos, vel, 2, variant, kT, dzeta=1.0)
    fv, _ = t.populations()
    assert np.array_equal(fv, o.populations())
    pv, vv, _, _ = t.particles()
    po, vo = o.particles()
    assert np.array_equal(pv, po) and np.array_equal(vv, vo)
    assert t.drag()[0] == pytest.approx(S, rel=1e-13, abs=1e-18)


@pytest.mark.parametrize("variant", [0, 1])
@pytest.mark.parametrize("kT", [0.0, 1e-4])
def test_zeta_derivative_matches_finite_differences(variant, kT):
    pos, vel = _particles()
    z, h = 1.3, 1e-5
    fd = (_oracle_drag(z + h, pos, vel, 2, variant, kT)[0] - _oracle_drag(z - h, pos, vel, 2, variant, kT)[0]) / (2 * h)
    d = _tangent(z, pos, vel, 2, variant, kT, dzeta=1.0).drag()[1]
    assert d == pytest.approx(fd, rel=1e-6, abs=1e-12)


@pytest.mark.parametrize("variant", [0, 1])
@pytest.mark.parametrize("kT", [0.0, 1e-4])
def test_position_derivative_matches_finite_differences(variant, kT):
    pos, vel = _particles()
    e = inputs.uniform(pos.shape, -1.0, 1.0, 11)
    h = 1e-6
    fd = (_oracle_drag(1.3, pos + h * e, vel, 2, variant, kT)[0]
          - _oracle_drag(1.3, pos - h * e, vel, 2, variant, kT)[0]) / (2 * h)
    d = _tangent(1.3, pos, vel, 2, variant, kT, dpos=e).drag()[1]
    assert d == pytest.approx(fd, rel=1e-5, abs=1e-10)


def test_population_derivative_matches_finite_differences():
    # the tangent of the fluid state itself (used by nothing but this pin):
    # d f / d zeta after two cycles
    pos, vel = _particles()
    h = 1e-5
    fp = _oracle_drag(1.3 + h, pos, vel, 2, 1, 1e-4)[1].populations()
    fm = _oracle_drag(1.3 - h, pos, vel, 2, 1, 1e-4)[1].populations()
    _, df = _tangent(1.3, pos, vel, 2, 1, 1e-4, dzeta=1.0).populations()
    fd = (fp - fm) / (2 * h)
    scale = float(np.abs(fd).max())
    assert scale > 0
    assert float(np.abs(df - fd).max()) <= 1e-5 * scale
