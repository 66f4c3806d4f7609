"""Shared set-up of the GPU parity tests: one oracle state and one GPU context
built from the same parameters and the same seeded inputs."""
import numpy as np

from oracle import oracle as orc
from paper_1610_02733_gb300 import inputs, lbmd

# Tolerances per population after one LB step, relative to the population
# scale w_i rho: FP32 storage and arithmetic 1e-5, FP64 1e-12.
TOL = {"fp32": 1e-5, "fp64": 1e-12}


def pair(shape, *, precision="fp32", variant="B", n_sub=1, kT=0.0, zeta=1.0, nu=1.0 / 6.0, nu_bulk=-1.0,
         gamma_ghost=0.0, body_force=(0.0, 0.0, 0.0), seed=1, rho0=1.0, max_particles=0, max_bonds=0,
         integrator="start", spread="auto"):
    o = orc.Oracle(*shape, n_sub=n_sub, variant={"A": 0, "B": 1, "C": 2}[variant], rho0=rho0, nu=nu, nu_bulk=nu_bulk,
                   gamma_ghost=gamma_ghost, kT=kT, zeta=zeta, body_force=body_force, seed=seed,
                   integrator={"start": 0, "half_step": 1}[integrator])
    g = lbmd.LBMD(*shape, variant=variant, precision=precision, n_sub=n_sub, rho0=rho0, nu=nu, nu_bulk=nu_bulk,
                  gamma_ghost=gamma_ghost, kT=kT, zeta=zeta, body_force=body_force, seed=seed,
                  max_particles=max_particles, max_bonds=max_bonds, integrator=integrator, spread=spread)
    return o, g


def random_state(o, seed, amplitude=0.05):
    """Populations near the fluid at rest (the oracle's initial state)."""
    return inputs.perturbed(o.populations(), amplitude, seed)


W = np.array([1 / 3] + [1 / 18] * 6 + [1 / 36] * 12)


def assert_pops_close(got, want, precision, rho0=1.0):
    """Element-by-element check, relative to each population's own scale
    w_i rho0.  (Thermal noise moves a single population by up to ~30 % of
    that scale per step at kT = 1e-3, so the value itself can come close to
    zero; the scale is what FP32 rounding is proportional to.)"""
    err = np.abs(got - want) / (W[:, None] * rho0)
    worst = float(err.max())
    assert worst <= TOL[precision], "max relative population error %.3e > %.0e" % (worst, TOL[precision])
    return worst


def assert_vec_close(got, want, precision, what):
    """Particle or node vectors: relative to the largest magnitude present."""
    scale = max(float(np.abs(want).max()), 1e-300)
    err = float(np.abs(got - want).max()) / scale
    tol = {"fp32": 1e-5, "fp64": 1e-12}[precision]
    assert err <= tol, "%s: max error %.3e of scale %.3e > %.0e" % (what, err, scale, tol)
    return err
