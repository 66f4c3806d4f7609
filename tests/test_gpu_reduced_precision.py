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

from gpu_common import W, pair
from paper_1610_02733_gb300 import inputs

pytestmark = pytest.mark.gpu

TOL = {"fp16dev": 1e-4, "bf16dev": 1e-3}


def _round_deviation(f, rho0, precision):
    base = W[:, None] * rho0
    dev = f - base
    if precision == "fp16dev":
        dev = dev.astype(np.float16).astype(np.float64)
    else:
        torch = pytest.importorskip("torch")
        dev = torch.from_numpy(dev).to(torch.bfloat16).to(torch.float64).numpy()
    return base + dev


@pytest.mark.parametrize("precision", ["fp16dev", "bf16dev"])
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
    err = float((np.abs(g.populations() - o.populations()) / W[:, None]).max())
    assert err <= TOL[precision], err


# stated errors of 20 variant-B cycles at kT = 1e-4 (256 particles, 16^3),
# relative to the FP64 oracle on the same Philox streams: (mass, total
# momentum relative to the particle momentum scale, particle temperature)
BOUNDS = {"fp32": (2e-6, 1e-3, 0.01), "fp16dev": (2e-5, 0.05, 0.02), "bf16dev": (1e-4, 0.3, 0.05)}


@pytest.mark.parametrize("precision", ["fp32", "fp16dev", "bf16dev"])
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
