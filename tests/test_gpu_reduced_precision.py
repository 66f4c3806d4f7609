"""Reduced-precision population storage (FP16 / BF16 deviations from the
rest state w_i rho0, FP32 arithmetic) against the FP64 oracle.

The initial state is rounded to the storage format here in the test (numpy
float16, torch bfloat16 on the CPU, both round to nearest), so that the
oracle and the GPU start from exactly the same populations; the remaining
difference after one LB step is the rounding of the stored result plus FP32
arithmetic: at most about half a unit in the last place of the stored
deviation.  Per-observable errors over a longer coupled run are checked
against the FP32 GPU path and the oracle."""
import numpy as np
import pytest

from gpu_common import D3Q19_C, W, assert_rounded_like_oracle, expected_readback, pair, storage_base32
from paper_1610_02733_gb300 import inputs

pytestmark = pytest.mark.gpu

# one LB step, relative to w_i rho0: round to nearest is off by at most half a
# grid step of the stored deviation, stochastic rounding by at most one
TOL = {"fp16dev": 1e-4, "bf16dev": 1e-3, "fp16dev_sr": 2e-4, "bf16dev_sr": 2e-3}


def _round_deviation(f, rho0, precision):
    # deviations from the FP32 rest value, rounded to the storage format: the
    # sum is (for all but the tiniest deviations) an FP32 number whose stored
    # deviation is exactly the rounded one
    base = storage_base32(rho0).astype(np.float64)[:, None]
    dev = f - base
    if precision.startswith("fp16"):
        dev = dev.astype(np.float16).astype(np.float64)
    else:
        torch = pytest.importorskip("torch")
        dev = torch.from_numpy(dev).to(torch.bfloat16).to(torch.float64).numpy()
    return base + dev


def _sources(shape):
    """Source node r - c_i of every (i, r) of the post-stream populations."""
    nx, ny, nz = shape
    r = np.arange(nx * ny * nz)
    xyz = np.stack([r % nx, (r // nx) % ny, r // (nx * ny)], axis=1)
    s = (xyz[None, :, :] - D3Q19_C[:, None, :]) % np.array(shape)
    return s[..., 0] + nx * (s[..., 1] + ny * s[..., 2])


@pytest.mark.parametrize("precision", ["fp16dev", "bf16dev", "fp16dev_sr", "bf16dev_sr"])
@pytest.mark.parametrize("kT", [0.0, 1e-4])
def test_one_lb_step(precision, kT):
    shape = (10, 6, 14)
    o, g = pair(shape, precision=precision, kT=kT, nu=0.11, nu_bulk=0.3, gamma_ghost=0.2,
                body_force=(1e-5, -2e-5, 3e-5), seed=1234)
    f0 = _round_deviation(inputs.perturbed(o.populations(), 0.02, 7), 1.0, precision)
    o.set_populations(f0)
    g.set_populations(f0)
    # the stored deviations are exact; the read-back adds w_i rho0 in FP32
    assert float((np.abs(g.populations() - f0) / W[:, None]).max()) < 1e-7
    for obj in (o, g):
        obj.md_substep()
        obj.lb_step()
    fg, fo = g.populations(), o.populations()
    err = float((np.abs(fg - fo) / W[:, None]).max())
    assert err <= TOL[precision], err
    # every stored value is the oracle's value rounded onto the storage grid
    # (to nearest, or stochastically with the same Philox bits)
    i = np.repeat(np.arange(19), fo.shape[1])
    want, step, dist = expected_readback(fo.ravel(), i, _sources(shape).ravel(), precision, seed=1234, lb_step=0)
    exact = assert_rounded_like_oracle(fg.ravel(), want, step, dist)
    assert exact > 0.8, exact


# stated errors of 20 variant-B cycles at kT = 1e-4 (256 particles, 16^3),
# relative to the FP64 oracle on the same Philox streams: (mass, total
# momentum relative to the particle momentum scale, particle temperature)
BOUNDS = {"fp32": (2e-6, 1e-3, 0.01), "fp16dev": (2e-5, 0.05, 0.02), "bf16dev": (1e-4, 0.3, 0.05),
          "fp16dev_sr": (2e-5, 0.05, 0.02), "bf16dev_sr": (1e-4, 0.3, 0.05)}


@pytest.mark.parametrize("precision", ["fp32", "fp16dev", "bf16dev", "fp16dev_sr", "bf16dev_sr"])
def test_coupled_run_observables(precision):
    shape, n, kT = (16, 16, 16), 256, 1e-4
    o, g = pair(shape, precision=precision, variant="B", n_sub=10, kT=kT, zeta=1.0, seed=2, max_particles=n)
    pos, vel = inputs.uniform_positions(n, shape, 2), inputs.maxwell_velocities(n, kT, 2)
    for obj in (o, g):
        obj.add_particles(pos, vel)
    o.cycle(20)
    g.run_cycles(20)
    ob_o, ob = o.observables(), g.observables()
    mass_err = abs(ob["mass"] / ob_o["mass"] - 1.0)
    p_scale = np.abs(ob_o["p_particles"]).max() + 1e-12
    p_err = np.abs((ob["p_fluid"] + ob["p_particles"]) - (ob_o["p_fluid"] + ob_o["p_particles"])).max() / p_scale
    t_err = abs(ob["kT_particles"] / ob_o["kT_particles"] - 1.0)
    print("%s: mass %.2e  momentum %.2e  temperature %.2e" % (precision, mass_err, p_err, t_err))
    bm, bp, bt = BOUNDS[precision]
    assert mass_err < bm and p_err < bp and t_err < bt, (mass_err, p_err, t_err)


# The reduced-precision workload at its own size: 256^3, 10^6 ideal particles
# (zeta = 1, uniform positions), variant B, m = 10, kT = 1e-4, 1000 MD steps.
# Mass and total (fluid + particle) momentum are conserved in exact arithmetic
# (Sec. 2); what is left is rounding.  FP32: the FP32 sum of 19 populations
# near w_i rho0 rounds alike at every node of the near-uniform fluid, and the
# collision writes it back -- a systematic mass drift of ~1.4e-8 per LB step.
# The deviation forms sum small deviations instead, so their mass moves only
# by the random walk of the stored roundings, and so does their momentum
# (a random walk of the 16-bit roundings of the stored deviations, which
# stochastic rounding cannot remove: its per-store variance is twice that of
# rounding to nearest).  The particle temperature is compared with the FP32
# run on the same Philox streams.
C5_SHAPE, C5_NP, C5_CYCLES = (256, 256, 256), 1_000_000, 100
C5_BOUNDS = {  # (mass rel., momentum / sqrt(N_p m kT), temperature rel. to FP32)
    "fp32": (3e-6, 1e-3, 0.0),
    "fp16dev": (1e-7, 0.1, 1e-5), "fp16dev_sr": (1e-7, 0.1, 1e-5),
    "bf16dev": (1e-7, 0.4, 1e-4), "bf16dev_sr": (1e-7, 0.4, 1e-4),
}


def _c5_run(precision):
    from paper_1610_02733_gb300 import lbmd
    g = lbmd.LBMD(*C5_SHAPE, variant="B", precision=precision, n_sub=10, kT=1e-4, zeta=1.0, seed=11,
                  max_particles=C5_NP)
    vel = inputs.maxwell_velocities(C5_NP, 1e-4, 11)
    g.add_particles(inputs.uniform_positions(C5_NP, C5_SHAPE, 11), vel)
    g.run_cycles(C5_CYCLES)
    ob = g.observables()
    g.close()
    return ob, vel.sum(axis=0)


@pytest.fixture(scope="module")
def c5_fp32():
    return _c5_run("fp32")


@pytest.mark.parametrize("precision", ["fp32", "fp16dev", "fp16dev_sr", "bf16dev", "bf16dev_sr"])
def test_config5_conservation_and_temperature(c5_fp32, precision):
    ob, p0 = c5_fp32 if precision == "fp32" else _c5_run(precision)
    n_nodes = np.prod(C5_SHAPE)
    mass_err = abs(ob["mass"] / n_nodes - 1.0)
    p_scale = np.sqrt(C5_NP * 1e-4)
    p_err = float(np.linalg.norm(np.array(ob["p_fluid"]) + np.array(ob["p_particles"]) - p0)) / p_scale
    t_err = abs(ob["kT_particles"] / c5_fp32[0]["kT_particles"] - 1.0)
    print("%s: mass %.2e  momentum %.2e  temperature vs FP32 %.2e  kT %.4e" %
          (precision, mass_err, p_err, t_err, ob["kT_particles"]))
    bm, bp, bt = C5_BOUNDS[precision]
    assert mass_err < bm and p_err < bp and t_err <= bt, (mass_err, p_err, t_err)
    assert abs(ob["kT_particles"] / 1e-4 - 1.0) < 0.1  # the bath's temperature (within START's zeta dt / 2m)
