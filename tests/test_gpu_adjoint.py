"""Hand-written adjoint of the coupled step (lbmd_adjoint_*) against the
oracle's tangent (lbmd_tangent.c, itself pinned to finite differences of the
plain oracle) and against central finite differences of the GPU's own FP64
forward pass.

L(zeta, R0) = mean coupling force F_x over all MD steps and particles
(variant B, fluid at rest initially, uniform body force along x).  Particle
positions start well inside their cells and move little, so that no
particle crosses a cell face (where the piecewise-smooth map has kinks)
within the finite-difference steps."""
import numpy as np
import pytest

from oracle import oracle as orc
from paper_1610_02733_gb300 import inputs, lbmd

pytestmark = pytest.mark.gpu

BODY = (1e-5, 0.0, 0.0)


def _particles(n, shape, seed, vscale):
    g = np.random.default_rng(seed)
    base = np.stack([g.integers(0, L, n) for L in shape], axis=1).astype(float)
    return base + 0.3 + 0.4 * g.random((n, 3)), vscale * (g.random((n, 3)) - 0.5)


def _tangent(shape, n_sub, cycles, zeta, kT, pos, vel, dpos=None, dzeta=0.0, seed=5):
    t = orc.Tangent(*shape, n_sub=n_sub, variant=1, kT=kT, zeta=zeta, body_force=BODY, seed=seed)
    t.set_particles(pos, vel, dpos, dzeta)
    t.cycle(cycles)
    S, dS = t.drag()
    norm = 1.0 / (cycles * n_sub * pos.shape[0])
    return S * norm, dS * norm


@pytest.mark.parametrize("precision,tol", [("fp64", 1e-9), ("fp32", 1e-3)])
@pytest.mark.parametrize("kT", [0.0, 1e-4])
def test_adjoint_matches_oracle_tangent(precision, tol, kT):
    shape, n_sub, cycles, zeta, n = (12, 10, 8), 5, 4, 1.5, 16
    pos, vel = _particles(n, shape, 3, 2e-3)
    ad = lbmd.Adjoint(*shape, n_particles=n, n_cycles=cycles, n_sub=n_sub, precision=precision, kT=kT,
                      body_force=BODY, seed=5)
    L = ad.forward(zeta, pos, vel)
    dz, dpos = ad.backward()
    Lo, dzo = _tangent(shape, n_sub, cycles, zeta, kT, pos, vel, dzeta=1.0)
    # L is a mean of drags of both signs (random initial velocities against
    # the accelerating fluid): FP32 rounding of the terms leaves ~1e-4 of it
    assert L == pytest.approx(Lo, rel=1e-12 if precision == "fp64" else tol)
    assert dz == pytest.approx(dzo, rel=tol)
    for s in (1, 2):
        e = inputs.uniform(pos.shape, -1.0, 1.0, 20 + s)
        _, de = _tangent(shape, n_sub, cycles, zeta, kT, pos, vel, dpos=e)
        got = float((dpos * e).sum())
        # relative to the size of the terms of the directional derivative
        # (it sums contributions of both signs)
        assert abs(got - de) <= tol * float(np.abs(dpos * e).sum()), (got, de)


@pytest.mark.parametrize("kT", [0.0, 1e-4])
def test_adjoint_matches_gpu_finite_differences_full_size(kT):
    # the batched configuration of the adjoint: 32^3, 64 particles, zeta 1.5,
    # m = 10, 200 MD steps, body force 1e-5
    shape, n_sub, cycles, zeta, n = (32, 32, 32), 10, 20, 1.5, 64
    pos, vel = _particles(n, shape, 4, 1e-3)
    ad = lbmd.Adjoint(*shape, n_particles=n, n_cycles=cycles, n_sub=n_sub, precision="fp64", kT=kT,
                      body_force=BODY, seed=9)
    ad.forward(zeta, pos, vel)
    dz, dpos = ad.backward()
    h = 1e-6 * zeta
    fd = (ad.forward(zeta + h, pos, vel) - ad.forward(zeta - h, pos, vel)) / (2 * h)
    assert dz == pytest.approx(fd, rel=1e-6)
    hp = 1e-6
    for p, a in ((0, 0), (7, 1), (33, 2)):
        pp, pm = pos.copy(), pos.copy()
        pp[p, a] += hp
        pm[p, a] -= hp
        fdp = (ad.forward(zeta, pp, vel) - ad.forward(zeta, pm, vel)) / (2 * hp)
        # finite differences of positions resolve the fixed-point rounding
        # of the transfers (2^-56 per transfer) at ~1e-10 here
        scale = float(np.abs(dpos).max())
        assert abs(dpos[p, a] - fdp) <= 1e-4 * scale + 1e-10, (p, a, dpos[p, a], fdp, scale)


def test_torch_autograd_function():
    torch = pytest.importorskip("torch")
    shape, n = (12, 10, 8), 8
    pos, vel = _particles(n, shape, 5, 1e-3)
    ad = lbmd.Adjoint(*shape, n_particles=n, n_cycles=3, n_sub=5, precision="fp64", body_force=BODY, seed=2)
    drag = lbmd.drag_function(ad, vel)
    zeta = torch.tensor(1.5, dtype=torch.float64, requires_grad=True)
    R0 = torch.tensor(pos, dtype=torch.float64, requires_grad=True)
    loss = drag(zeta, R0)
    (2.0 * loss).backward()
    L = ad.forward(1.5, pos, vel)
    dz, dpos = ad.backward()
    assert float(loss.detach()) == L
    assert float(zeta.grad) == pytest.approx(2.0 * dz, rel=1e-14)
    assert np.allclose(R0.grad.numpy(), 2.0 * dpos, rtol=1e-14, atol=0)
