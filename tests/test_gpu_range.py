"""Range of the fixed-point momentum density.

The node field holds j (Eq. (2)) and the particles' transfers (Eqs. (7), (8))
as integers in units of 2^(e - 30) (FP32) / 2^(e - 56) (FP64), e = ceil(log2
rho0).  These tests check that the unit follows rho0 -- a dense fluid
(rho0 = 1e6, where j of an ordinary flow is far beyond the range of the
rho0 = 1 unit) matches the oracle and gives the discrete Ornstein-Uhlenbeck
temperature of a bath at rest -- and that a node whose momentum reaches half
the range raises the flag lbmd_observables reports.
"""
import numpy as np
import pytest

from gpu_common import W, assert_vec_close, pair
from paper_1610_02733_gb300 import inputs, lbmd

pytestmark = pytest.mark.gpu


@pytest.mark.parametrize("precision", ["fp32", "fp64"])
def test_dense_fluid_against_the_oracle(precision):
    shape, n, n_sub, rho0, kT = (8, 6, 10), 24, 5, 1.0e6, 1e-3
    o, g = pair(shape, precision=precision, variant="B", n_sub=n_sub, rho0=rho0, kT=kT, zeta=2.0, seed=8,
                max_particles=n)
    # a flow of u ~ 0.02: j ~ 2e4, beyond |j| < 2 of the unit 2^-30
    f0 = inputs.perturbed(o.populations(), 0.05, 4)
    pos, vel = inputs.uniform_positions(n, shape, 8), inputs.maxwell_velocities(n, kT, 8)
    for obj in (o, g):
        obj.set_populations(f0)
        obj.add_particles(pos, vel)
        obj.cycle(2)
    err = np.abs(g.populations() - o.populations()) / (W[:, None] * rho0)
    assert err.max() <= {"fp32": 1e-5, "fp64": 1e-12}[precision], err.max()
    # j is a small difference of populations of size rho0: compare it on the
    # scale of rho0 (FP32 populations of 5e4 carry absolute errors ~1e-2)
    nf_g, nf_o = g.node_field(), o.node_field()
    assert np.abs(nf_g[:, 1:] - nf_o[:, 1:]).max() / rho0 <= {"fp32": 1e-6, "fp64": 1e-13}[precision]
    assert np.abs(nf_g[:, 1:]).max() > 100.0  # the flow really is beyond the rho0 = 1 range
    assert_vec_close(g.particles()[1], o.particles()[1], precision, "velocities")
    g.observables()  # no range error
    o.close()
    g.close()


def test_dense_fluid_bath_gives_the_ornstein_uhlenbeck_temperature():
    # rho0 = 1e6: the fluid is a bath at rest, and every MD step is
    # v' = v (1 - zeta dt / m) + dt sqrt(2 zeta kT / dt) xi / m, whose
    # stationary <m v^2> / 3 is kT / (1 - zeta dt / 2m) exactly (the oracle
    # pins the same value)
    shape, n, n_sub, kT, zeta = (8, 8, 8), 6000, 5, 1e-3, 2.0
    g = lbmd.LBMD(*shape, variant="B", n_sub=n_sub, rho0=1e6, kT=kT, zeta=zeta, seed=3, max_particles=n)
    g.add_particles(inputs.uniform_positions(n, shape, 3), inputs.maxwell_velocities(n, kT, 3))
    g.run_cycles(20)
    T = []
    for _ in range(200):
        g.run_cycles(1)
        T.append(g.observables()["kT_particles"])
    want = kT / (1.0 - zeta * (1.0 / n_sub) / 2.0)
    assert abs(np.mean(T) / want - 1.0) < 0.01, (np.mean(T), want)
    g.close()


@pytest.mark.parametrize("precision,beyond,inside", [("fp32", 1.2, 0.9), ("fp64", 70.0, 60.0)])
def test_range_flag(precision, beyond, inside):
    # a node carrying |j| beyond half the range (1 in FP32, 64 in FP64 at
    # rho0 = 1) raises the flag; a new fluid state clears it
    shape = (6, 5, 4)
    g = lbmd.LBMD(*shape, variant="B", precision=precision, kT=0.0)
    rest = g.populations()

    def with_jx(j):
        f = rest.copy()
        f[1, 7] += 0.5 * j  # c = +x
        f[2, 7] -= 0.5 * j  # c = -x
        return f

    g.set_populations(with_jx(beyond))
    with pytest.raises(lbmd.LbmdError) as e:
        g.observables()
    assert e.value.status == lbmd.LBMD_ERR_RANGE
    g.set_populations(rest)
    g.observables()
    g.set_populations(with_jx(inside))
    g.observables()
    g.close()


def test_rho0_outside_the_supported_range_is_rejected():
    for rho0 in (2.0 ** 61, 2.0 ** -62):
        with pytest.raises(lbmd.LbmdError):
            lbmd.LBMD(4, 4, 4, rho0=rho0)
