"""The host accessors' FP32 <-> FP64 conversions and the observables' sums of
the FP32 forms, which run on the integer and FP32 pipes (bit-field
arithmetic, fixed-point and two-sum accumulation) instead of FP64
arithmetic.

Conversions are compared bit for bit with numpy's IEEE arithmetic: a
position x becomes the cell floor(x) and the FP32 offset x - floor(x)
rounded to nearest even (moved to the next node, periodically, when it
rounds to 1; wrapped into the box first), and reads back as cell + offset
rounded to nearest even in FP64; a velocity reads back as its FP32 rounding.
The cases cover ties, offsets that round up to the next node, subnormal and
zero offsets, signed zeros, positions outside the box and far from it, and
velocities outside FP32's normal range.  The observables are compared with
exact (math.fsum) sums of the stored FP32 values.
"""
import math

import numpy as np
import pytest

from paper_1610_02733_gb300 import inputs, lbmd

pytestmark = pytest.mark.gpu

SHAPE = (48, 20, 12)


def _expected_position(x, L):
    x = np.float64(x)
    if not (0.0 <= x < L):
        x = x - L * np.floor(x / L)
        if x >= L:
            x = x - L
    fl = np.floor(x)
    f = np.float32(x - fl)
    if f >= np.float32(1.0):
        f = np.float32(0.0)
        fl = fl + 1.0
        if fl >= L:
            fl = 0.0
    return np.float64(fl) + np.float64(f)


def _edge_coordinates(L):
    t = 2.0 ** -24
    vals = [0.0, -0.0, 1e-300, 5e-324, 2.0 ** -126, 2.0 ** -127, 2.0 ** -149, 1e-45, 0.5, 1.0 - 2.0 ** -60,
            1.0 - t / 4, 1.0 - t / 2, 1.0 - t, 1.0, 1.0 + 2.0 ** -40, L - 1e-12, L - 2.0 ** -40, L - 1.0, L - 0.5,
            L, L + 0.25, -0.25, -1e-12, -L, 3.5 * L, -7.25 * L, 1e6 * L + 0.3, 17.0, 17.0 + t / 2 * 17,
            17.0 + 2.0 ** -25, 17.0 + 3 * 2.0 ** -26, 1.0 + 2.0 ** -24 * 3, 2.5 + 2.0 ** -30]
    # fractions exactly half-way between FP32 values in [1/2, 1) and [1/4, 1/2)
    for k in range(8):
        vals += [9.0 + 0.5 + (2 * k + 1) * 2.0 ** -25, 3.0 + 0.25 + (2 * k + 1) * 2.0 ** -26]
    return [v for v in vals if abs(v) < 2.0 ** 40]


def _edge_velocities():
    t = 2.0 ** -24
    vals = [0.0, -0.0, 1e-300, -1e-300, 2.0 ** -126, 2.0 ** -127, 1e-39, -1e-42, 1.0 + t, 1.0 + 3 * t,
            -(1.0 + t), 1.0 + t + 2.0 ** -50, 0.1, -0.3, 3.4e38, 3.5e38, -1e39, 65504.0, 1.0 - t / 2, 1.0 - t / 4]
    return vals


@pytest.mark.parametrize("variant", ["B", "A"])
def test_positions_and_velocities_round_trip_bitwise(variant):
    rng = np.random.default_rng(7)
    L = np.array(SHAPE, dtype=np.float64)
    edges_x = _edge_coordinates(L[0])
    edges_v = _edge_velocities()
    n = 4000
    pos = inputs.uniform_positions(n, SHAPE, 7)
    vel = inputs.maxwell_velocities(n, 1e-3, 7)
    # random doubles with full 52-bit fractions, some far outside the box
    pos[:500] = rng.uniform(-3, 4, (500, 3)) * L
    pos[500:500 + len(edges_x), 0] = edges_x
    pos[1000:1000 + len(edges_x), 1] = [e * L[1] / L[0] for e in edges_x]
    pos[2000:2000 + len(edges_x), 2] = [min(e, 1e6 * L[2]) for e in edges_x]
    vel[:len(edges_v), 0] = edges_v
    vel[100:100 + len(edges_v), 2] = edges_v[::-1]
    vel[200:400] = rng.standard_normal((200, 3)) * 10.0 ** rng.uniform(-30, 30, (200, 1))
    g = lbmd.LBMD(*SHAPE, variant=variant, kT=0.0, max_particles=n)
    g.add_particles(inputs.uniform_positions(n, SHAPE, 8), np.zeros((n, 3)))
    with np.errstate(over="ignore"):
        g.set_particles(np.ascontiguousarray(pos.reshape(-1)), np.ascontiguousarray(vel.reshape(-1)))
        got_p, got_v = g.particles()
        want_v = vel.astype(np.float32).astype(np.float64)
    want_p = np.array([[_expected_position(pos[i, d], L[d]) for d in range(3)] for i in range(n)])
    bad = np.nonzero(got_p.view(np.int64) != want_p.view(np.int64))
    assert bad[0].size == 0, (pos[bad][:5], got_p[bad][:5], want_p[bad][:5])
    badv = np.nonzero(got_v.view(np.int64) != want_v.view(np.int64))
    assert badv[0].size == 0, (vel[badv][:5], got_v[badv][:5], want_v[badv][:5])
    g.close()


def _fsum(a):
    return math.fsum(np.asarray(a, dtype=np.float64).ravel())


@pytest.mark.parametrize("masses", [False, True])
def test_observables_equal_exact_sums_of_the_stored_values(masses):
    shape, n = (40, 24, 16), 3000
    g = lbmd.LBMD(*shape, variant="B", kT=1e-3, zeta=1.0, n_sub=5, seed=4, max_particles=n)
    m = np.random.default_rng(4).uniform(0.5, 3.0, n) if masses else None
    g.add_particles(inputs.uniform_positions(n, shape, 4), inputs.maxwell_velocities(n, 1e-3, 4), m)
    g.run_cycles(3)
    o = g.observables()
    _, v = g.particles()
    # the stored inverse mass is the FP32 rounding of 1/m
    w = np.ones(n) if m is None else (1.0 / m).astype(np.float32).astype(np.float64)
    mv = v / w[:, None]
    np.testing.assert_allclose(o["p_particles"], [_fsum(mv[:, d]) for d in range(3)],
                               rtol=0, atol=1e-12 * _fsum(np.abs(mv)))
    e2 = _fsum((v * v).sum(axis=1) / w)
    assert abs(2 * o["e_kin"] - e2) <= 1e-12 * e2
    nf = g.node_field()
    assert abs(o["mass"] - _fsum(nf[:, 0])) <= 1e-13 * o["mass"]
    pf = [_fsum(nf[:, 1 + d]) for d in range(3)]
    np.testing.assert_allclose(o["p_fluid"], pf, rtol=0, atol=1e-14 * _fsum(np.abs(nf[:, 1:])))
    g.close()


@pytest.mark.parametrize("precision", ["fp32", "fp64"])
def test_mass_sum_far_from_rho0_and_non_finite_fluid(precision):
    # densities beyond the FP32 form's fixed-point mass range (>= 2^(e + 4))
    # are added beside it in double precision; a NaN density makes the
    # observables non-finite, reported by both the synchronising and the
    # queued observables
    shape = (24, 10, 8)
    g = lbmd.LBMD(*shape, variant="B", precision=precision, kT=0.0)
    rest = g.populations()
    f = rest.copy()
    f[:, 17] *= 5000.0  # a node at rest with 5000 rho0
    f[:, 400] *= 40.0
    g.set_populations(f)
    o = g.observables()
    nf = g.node_field()
    assert abs(o["mass"] - _fsum(nf[:, 0])) <= 1e-13 * o["mass"]
    assert abs(o["mass"] / _fsum(f) - 1.0) <= (1e-6 if precision == "fp32" else 1e-13)
    f[3, 55] = np.nan
    g.set_populations(f)
    with pytest.raises(lbmd.LbmdError) as e:
        g.observables()
    assert e.value.status == lbmd.LBMD_ERR_NONFINITE
    g.observables_async()
    with pytest.raises(lbmd.LbmdError) as e:
        g.synchronize()
    assert e.value.status == lbmd.LBMD_ERR_NONFINITE
    g.set_populations(rest)
    g.observables()
    g.close()
