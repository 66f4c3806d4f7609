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
         integrator="start", spread="auto", noise="uniform"):
    o = orc.Oracle(*shape, n_sub=n_sub, variant={"A": 0, "B": 1, "C": 2}[variant], rho0=rho0, nu=nu, nu_bulk=nu_bulk,
                   gamma_ghost=gamma_ghost, kT=kT, zeta=zeta, body_force=body_force, seed=seed,
                   integrator={"start": 0, "half_step": 1}[integrator], noise=noise)
    g = lbmd.LBMD(*shape, variant=variant, precision=precision, n_sub=n_sub, rho0=rho0, nu=nu, nu_bulk=nu_bulk,
                  gamma_ghost=gamma_ghost, kT=kT, zeta=zeta, body_force=body_force, seed=seed,
                  max_particles=max_particles, max_bonds=max_bonds, integrator=integrator, spread=spread,
                  noise=noise)
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


def assert_pops_close_per_value(got, want, precision):
    """Element by element, relative to each value itself: the check the
    parity tolerance states, used where no population comes near zero (kT
    up to 1e-4, moderate flows)."""
    err = np.abs(got - want) / np.abs(want)
    worst = float(err.max())
    assert worst <= TOL[precision], "max per-value relative population error %.3e > %.0e" % (worst, TOL[precision])
    return worst


def assert_vec_close(got, want, precision, what):
    """Particle or node vectors: relative to the largest magnitude present."""
    scale = max(float(np.abs(want).max()), 1e-300)
    err = float(np.abs(got - want).max()) / scale
    tol = {"fp32": 1e-5, "fp64": 1e-12}[precision]
    assert err <= tol, "%s: max error %.3e of scale %.3e > %.0e" % (what, err, scale, tol)
    return err


# Reduced-precision storage: grid of the stored deviation and whether the
# collision rounds it stochastically.
STORAGE = {"fp16dev": ("fp16", False), "bf16dev": ("bf16", False), "fp16dev_sr": ("fp16", True),
           "bf16dev_sr": ("bf16", True)}

D3Q19_C = np.array([[0, 0, 0], [1, 0, 0], [-1, 0, 0], [0, 1, 0], [0, -1, 0], [0, 0, 1], [0, 0, -1], [1, 1, 0],
                    [-1, -1, 0], [1, -1, 0], [-1, 1, 0], [1, 0, 1], [-1, 0, -1], [1, 0, -1], [-1, 0, 1], [0, 1, 1],
                    [0, -1, -1], [0, 1, -1], [0, -1, 1]])


def storage_base32(rho0=1.0):
    """The FP32 rest value w_i rho0 the deviations are taken from."""
    return (W.astype(np.float32) * np.float32(rho0)).astype(np.float32)


def expected_readback(post, i, src, precision, seed, lb_step, rho0=1.0):
    """What the GPU reads back for population i whose exact (oracle)
    post-collision value at source node src is `post`: the deviation from
    the FP32 rest value rounded by the oracle onto the storage grid (to
    nearest, or stochastically with the Philox bits of (src, lb_step)), then
    added back to the rest value in FP32.  Returns (value, grid step of the
    exact deviation, distance of the exact deviation from the nearest point
    where the rounding decision changes: the rounding threshold, or a grid
    value)."""
    fmt, sr = STORAGE[precision]
    post, i, src = np.asarray(post, dtype=np.float64), np.asarray(i), np.asarray(src, dtype=np.uint32)
    base = storage_base32(rho0)[i]
    dev = post - base.astype(np.float64)
    r16 = orc.sr_bits(seed, src, lb_step)[np.arange(src.size), i] if sr else None
    stored = orc.round_storage(dev, fmt, r16)
    value = (base + stored.astype(np.float32)).astype(np.float64)
    p, emin = orc.STORAGE_FORMATS[fmt]
    a = np.abs(dev)
    expo = np.maximum(np.floor(np.log2(np.maximum(a, 1e-300))), emin)
    step = np.exp2(expo - (p - 1))
    frac = a / step - np.floor(a / step)
    thr = r16 / 65536.0 if sr else 0.5
    dist = np.minimum(np.abs(frac - thr), np.minimum(frac, 1.0 - frac)) * step
    return value, step, dist


def assert_rounded_like_oracle(got, want, step, dist, ulps=16):
    """The GPU value equals the oracle's rounded value except where the FP32
    collision's error (below `ulps` units in the last place of the FP32
    population) can put the deviation on the other side of a rounding
    decision: there they differ by one grid step (two across a binade), or,
    for a deviation so small that its grid is finer than the FP32 error, by
    that error.  Returns the fraction of bit-identical values."""
    eps = ulps * np.spacing(np.abs(want).astype(np.float32)).astype(np.float64)
    diff = np.abs(got - want)
    assert (diff <= 2.0 * step + eps).all(), float((diff / (2.0 * step + eps)).max())
    off = diff > 0.0
    near = dist <= eps
    assert np.all(near[off]), "%d values rounded the other way far from a threshold" % int(np.sum(off & ~near))
    return float(np.mean(~off))
