"""Thin ctypes binding of the C ABI in ``include/lbmd.h`` (argument
marshalling only: every step of the LB/MD path runs in the CUDA library).

The functions keep the ABI's names (``lbmd_create``, ``lbmd_md_substep``,
...).  ``LBMD`` is a small convenience wrapper around one context.  The
library is loaded from ``_build/liblbmd.so``; if it is missing the import of
the library fails loudly -- there is no CPU fallback.
"""
from __future__ import annotations

import ctypes as ct
import os

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "_build", "liblbmd.so")

LBMD_OK = 0
LBMD_ERR_ARG = -1
LBMD_ERR_CUDA = -2
LBMD_ERR_OOM = -3
LBMD_ERR_SEQUENCE = -4
LBMD_ERR_NONFINITE = -5
LBMD_ERR_CAPACITY = -6
LBMD_ERR_RANGE = -7
LBMD_BATCH_PERIOD_GRAPH = 0
LBMD_BATCH_PERSISTENT = 1
BATCH_SCHEDULES = {"period_graph": LBMD_BATCH_PERIOD_GRAPH, "persistent": LBMD_BATCH_PERSISTENT}
VARIANT_A, VARIANT_B, VARIANT_C = 0, 1, 2
FP32, FP64, FP16_DEV, BF16_DEV, FP16_DEV_SR, BF16_DEV_SR = 0, 1, 2, 3, 4, 5
PRECISIONS = {"fp32": FP32, "fp64": FP64, "fp16dev": FP16_DEV, "bf16dev": BF16_DEV, "fp16dev_sr": FP16_DEV_SR,
              "bf16dev_sr": BF16_DEV_SR}
INTEGRATOR_START, INTEGRATOR_HALF_STEP = 0, 1
INTEGRATORS = {"start": INTEGRATOR_START, "half_step": INTEGRATOR_HALF_STEP}
SPREAD_AUTO, SPREAD_ROWS, SPREAD_ATOMIC, SPREAD_TILES = 0, 1, 2, 3
SPREADS = {"auto": SPREAD_AUTO, "rows": SPREAD_ROWS, "atomic": SPREAD_ATOMIC, "tiles": SPREAD_TILES}
NOISE_UNIFORM, NOISE_GAUSS = 0, 1
NOISES = {"uniform": NOISE_UNIFORM, "gauss": NOISE_GAUSS}

# every symbol include/lbmd.h declares
EXPORTS = (
    "lbmd_create", "lbmd_destroy", "lbmd_add_particles", "lbmd_add_bonds", "lbmd_add_fene_bonds", "lbmd_set_lj",
    "lbmd_set_particles", "lbmd_state_size", "lbmd_save_state", "lbmd_load_state",
    "lbmd_md_substep", "lbmd_lb_step", "lbmd_run_cycles", "lbmd_observables", "lbmd_get_populations",
    "lbmd_set_populations", "lbmd_get_node_field", "lbmd_get_transfer", "lbmd_get_particles",
    "lbmd_get_particles_device", "lbmd_get_counts", "lbmd_stream", "lbmd_last_error", "lbmd_status_string",
    "lbmd_set_particles_async", "lbmd_get_particles_async", "lbmd_observables_async", "lbmd_synchronize",
    "lbmd_particle_sums_static", "lbmd_set_moments_wait", "lbmd_moments_fallback_rows", "lbmd_set_frozen_copy",
    "lbmd_batch_create", "lbmd_batch_destroy", "lbmd_batch_add_particles", "lbmd_batch_run", "lbmd_batch_kinetic",
    "lbmd_batch_kinetic_device",
    "lbmd_batch_unstable", "lbmd_batch_get_populations", "lbmd_batch_set_populations", "lbmd_batch_get_particles",
    "lbmd_batch_get_counts", "lbmd_batch_tuning", "lbmd_batch_set_lb_grid", "lbmd_batch_stream",
    "lbmd_batch_last_error", "lbmd_batch_set_schedule", "lbmd_batch_persistent_tuning",
    "lbmd_adjoint_create", "lbmd_adjoint_destroy", "lbmd_adjoint_forward", "lbmd_adjoint_backward",
    "lbmd_adjoint_last_error",
)


class LbmdParams(ct.Structure):
    _fields_ = [
        ("nx", ct.c_int32), ("ny", ct.c_int32), ("nz", ct.c_int32),
        ("n_sub", ct.c_int32), ("variant", ct.c_int32), ("precision", ct.c_int32),
        ("rho0", ct.c_double), ("nu", ct.c_double), ("nu_bulk", ct.c_double),
        ("gamma_ghost", ct.c_double), ("kT", ct.c_double), ("zeta", ct.c_double),
        ("body_force", ct.c_double * 3), ("seed", ct.c_uint64),
        ("max_particles", ct.c_int64), ("max_bonds", ct.c_int64), ("stream", ct.c_void_p),
        ("integrator", ct.c_int32), ("spread", ct.c_int32), ("noise", ct.c_int32),
    ]


class LbmdBatchParams(ct.Structure):
    _fields_ = [
        ("n_replicas", ct.c_int32), ("dims", ct.c_void_p), ("n_sub", ct.c_void_p), ("variant", ct.c_void_p),
        ("zeta", ct.c_void_p), ("seed", ct.c_void_p), ("max_particles", ct.c_void_p), ("precision", ct.c_int32),
        ("rho0", ct.c_double), ("nu", ct.c_double), ("nu_bulk", ct.c_double), ("gamma_ghost", ct.c_double),
        ("kT", ct.c_double), ("stream", ct.c_void_p),
    ]


class LbmdAdjointParams(ct.Structure):
    _fields_ = [
        ("nx", ct.c_int32), ("ny", ct.c_int32), ("nz", ct.c_int32), ("n_sub", ct.c_int32),
        ("n_particles", ct.c_int32), ("n_cycles", ct.c_int32), ("precision", ct.c_int32), ("pad_", ct.c_int32),
        ("rho0", ct.c_double), ("nu", ct.c_double), ("nu_bulk", ct.c_double), ("gamma_ghost", ct.c_double),
        ("kT", ct.c_double), ("body_force", ct.c_double * 3), ("seed", ct.c_uint64), ("stream", ct.c_void_p),
    ]


class LbmdObservables(ct.Structure):
    _fields_ = [
        ("mass", ct.c_double), ("p_fluid", ct.c_double * 3), ("p_particles", ct.c_double * 3),
        ("kT_particles", ct.c_double), ("e_kin", ct.c_double), ("lb_step", ct.c_int64), ("md_step", ct.c_int64),
    ]


class LbmdError(RuntimeError):
    def __init__(self, status, msg):
        super().__init__("%s (status %d): %s" % (msg, status, ""))
        self.status = status


_lib = None


def load():
    """Load liblbmd.so (raises if it has not been built)."""
    global _lib
    if _lib is not None:
        return _lib
    if not os.path.exists(LIB_PATH):
        raise ImportError("liblbmd.so not built (%s): run __graft_entry__.build()" % LIB_PATH)
    L = ct.CDLL(LIB_PATH)
    P = ct.c_void_p
    dp = ct.POINTER(ct.c_double)
    i64p = ct.POINTER(ct.c_int64)
    for name in EXPORTS:
        getattr(L, name)  # every declared symbol must resolve
    L.lbmd_create.argtypes = [ct.POINTER(LbmdParams), ct.POINTER(ct.c_void_p)]
    L.lbmd_destroy.argtypes = [P]
    L.lbmd_add_particles.argtypes = [P, ct.c_int64, dp, dp, dp, i64p]
    L.lbmd_add_bonds.argtypes = [P, ct.c_int64, i64p, ct.c_double, ct.c_double]
    L.lbmd_add_fene_bonds.argtypes = [P, ct.c_int64, i64p, ct.c_double, ct.c_double]
    L.lbmd_set_lj.argtypes = [P, ct.c_double, ct.c_double, ct.c_double]
    L.lbmd_state_size.argtypes = [P, i64p]
    L.lbmd_save_state.argtypes = [P, ct.c_void_p, ct.c_int64]
    L.lbmd_load_state.argtypes = [P, ct.c_void_p, ct.c_int64]
    L.lbmd_set_particles.argtypes = [P, ct.c_void_p, ct.c_void_p]
    L.lbmd_md_substep.argtypes = [P]
    L.lbmd_lb_step.argtypes = [P]
    L.lbmd_run_cycles.argtypes = [P, ct.c_int64]
    L.lbmd_observables.argtypes = [P, ct.POINTER(LbmdObservables)]
    for name in ("lbmd_get_populations", "lbmd_set_populations", "lbmd_get_node_field", "lbmd_get_transfer"):
        getattr(L, name).argtypes = [P, ct.c_void_p]
    L.lbmd_get_particles.argtypes = [P, ct.c_void_p, ct.c_void_p]
    L.lbmd_get_particles_device.argtypes = [P, ct.c_void_p, ct.c_void_p]
    L.lbmd_set_particles_async.argtypes = [P, ct.c_void_p, ct.c_void_p]
    L.lbmd_get_particles_async.argtypes = [P, ct.c_void_p, ct.c_void_p]
    L.lbmd_observables_async.argtypes = [P, ct.POINTER(LbmdObservables)]
    L.lbmd_synchronize.argtypes = [P]
    L.lbmd_get_counts.argtypes = [P, i64p, i64p, i64p, i64p, ct.POINTER(ct.c_int32)]
    L.lbmd_particle_sums_static.argtypes = [ct.c_void_p, ct.c_void_p, ct.c_int64, ct.c_void_p, ct.c_void_p]
    L.lbmd_set_moments_wait.argtypes = [P, ct.c_int32]
    L.lbmd_moments_fallback_rows.argtypes = [P, i64p]
    L.lbmd_set_frozen_copy.argtypes = [P, ct.c_int32]
    L.lbmd_stream.restype = ct.c_void_p
    L.lbmd_stream.argtypes = [P]
    L.lbmd_last_error.restype = ct.c_char_p
    L.lbmd_last_error.argtypes = [P]
    L.lbmd_status_string.restype = ct.c_char_p
    L.lbmd_status_string.argtypes = [ct.c_int]
    i32 = ct.c_int32
    L.lbmd_batch_create.argtypes = [ct.POINTER(LbmdBatchParams), ct.POINTER(ct.c_void_p)]
    L.lbmd_batch_destroy.argtypes = [P]
    L.lbmd_batch_add_particles.argtypes = [P, i32, ct.c_int64, P, P, P]
    L.lbmd_batch_run.argtypes = [P, ct.c_int64]
    L.lbmd_batch_kinetic.argtypes = [P, P]
    L.lbmd_batch_kinetic_device.argtypes = [P, P]
    L.lbmd_batch_unstable.argtypes = [P, P]
    L.lbmd_batch_get_populations.argtypes = [P, i32, P]
    L.lbmd_batch_set_populations.argtypes = [P, i32, P]
    L.lbmd_batch_get_particles.argtypes = [P, i32, P, P]
    L.lbmd_batch_get_counts.argtypes = [P, i32, i64p, i64p, i64p]
    L.lbmd_batch_tuning.argtypes = [P, ct.POINTER(i32), ct.POINTER(i32), P, P]
    L.lbmd_batch_set_lb_grid.argtypes = [P, i32]
    L.lbmd_batch_set_schedule.argtypes = [P, i32, i32]
    L.lbmd_batch_persistent_tuning.argtypes = [P, ct.POINTER(i32), P]
    L.lbmd_batch_stream.restype = ct.c_void_p
    L.lbmd_batch_stream.argtypes = [P]
    L.lbmd_batch_last_error.restype = ct.c_char_p
    L.lbmd_batch_last_error.argtypes = [P]
    L.lbmd_adjoint_create.argtypes = [ct.POINTER(LbmdAdjointParams), ct.POINTER(ct.c_void_p)]
    L.lbmd_adjoint_destroy.argtypes = [P]
    L.lbmd_adjoint_forward.argtypes = [P, ct.c_double, P, P, dp]
    L.lbmd_adjoint_backward.argtypes = [P, dp, P]
    L.lbmd_adjoint_last_error.restype = ct.c_char_p
    L.lbmd_adjoint_last_error.argtypes = [P]
    for name in EXPORTS:
        if name not in ("lbmd_stream", "lbmd_last_error", "lbmd_status_string", "lbmd_batch_stream",
                        "lbmd_batch_last_error", "lbmd_adjoint_last_error"):
            getattr(L, name).restype = ct.c_int
    _lib = L
    return L


def _ptr(a: np.ndarray):
    return a.ctypes.data_as(ct.c_void_p)


def _host_addr(a):
    """Address of a host array: numpy array or (pinned) torch CPU tensor."""
    if a is None:
        return None
    if hasattr(a, "data_ptr"):
        return ct.c_void_p(a.data_ptr())
    return _ptr(a)


def _f64(a, n=None) -> np.ndarray:
    a = np.ascontiguousarray(a, dtype=np.float64)
    if n is not None:
        a = a.reshape(n)
    return a


# ---------------------------------------------------------------------------
# ABI-named functions (handle = ct.c_void_p)
# ---------------------------------------------------------------------------
def _check(h, rc, what):
    if rc != LBMD_OK:
        L = load()
        msg = L.lbmd_last_error(h).decode(errors="replace")
        err = LbmdError(rc, what)
        err.args = ("%s failed: %s (status %d: %s)" % (what, msg, rc,
                                                      L.lbmd_status_string(rc).decode()),)
        raise err
    return rc


def lbmd_create(params: LbmdParams):
    L = load()
    h = ct.c_void_p()
    _check(None, L.lbmd_create(ct.byref(params), ct.byref(h)), "lbmd_create")
    return h


def lbmd_destroy(h):
    return load().lbmd_destroy(h)


def lbmd_md_substep(h):
    return _check(h, load().lbmd_md_substep(h), "lbmd_md_substep")


def lbmd_lb_step(h):
    return _check(h, load().lbmd_lb_step(h), "lbmd_lb_step")


def lbmd_run_cycles(h, n: int):
    return _check(h, load().lbmd_run_cycles(h, int(n)), "lbmd_run_cycles")


def observables_dict(o: LbmdObservables) -> dict:
    return {"mass": o.mass, "p_fluid": np.array(list(o.p_fluid)), "p_particles": np.array(list(o.p_particles)),
            "kT_particles": o.kT_particles, "e_kin": o.e_kin, "lb_step": o.lb_step, "md_step": o.md_step}


def lbmd_observables(h) -> dict:
    o = LbmdObservables()
    _check(h, load().lbmd_observables(h, ct.byref(o)), "lbmd_observables")
    return observables_dict(o)


def lbmd_particle_sums_static(vel_ptr: int, mass_ptr, n: int, out_ptr: int, stream=None):
    """Device pointers in, 4 device doubles out; allocates nothing (see the
    header comment of the C function)."""
    return _check(None, load().lbmd_particle_sums_static(
        ct.c_void_p(vel_ptr), None if not mass_ptr else ct.c_void_p(mass_ptr), int(n), ct.c_void_p(out_ptr),
        None if stream is None else ct.c_void_p(stream)), "lbmd_particle_sums_static")


def make_params(nx, ny, nz, *, n_sub=1, variant=VARIANT_B, precision=FP32, rho0=1.0, nu=1.0 / 6.0, nu_bulk=-1.0,
                gamma_ghost=0.0, kT=0.0, zeta=1.0, body_force=(0.0, 0.0, 0.0), seed=1, max_particles=0,
                max_bonds=0, stream=None, integrator="start", spread="auto", noise="uniform") -> LbmdParams:
    p = LbmdParams()
    p.nx, p.ny, p.nz = int(nx), int(ny), int(nz)
    p.n_sub, p.variant, p.precision = int(n_sub), int(variant), int(precision)
    p.rho0, p.nu, p.nu_bulk, p.gamma_ghost = float(rho0), float(nu), float(nu_bulk), float(gamma_ghost)
    p.kT, p.zeta = float(kT), float(zeta)
    for a in range(3):
        p.body_force[a] = float(body_force[a])
    p.seed = int(seed)
    p.max_particles, p.max_bonds = int(max_particles), int(max_bonds)
    p.stream = stream
    p.integrator = INTEGRATORS[integrator] if isinstance(integrator, str) else int(integrator)
    p.spread = SPREADS[spread] if isinstance(spread, str) else int(spread)
    p.noise = NOISES[noise] if isinstance(noise, str) else int(noise)
    return p


class LBMD:
    """One simulation context on the current CUDA device.

    Keyword arguments are the fields of ``lbmd_params`` (lattice units,
    a = tau_LB = 1).  ``precision`` is ``"fp32"``, ``"fp64"``, ``"fp16dev"`` or
    ``"bf16dev"`` (populations stored as FP16 / BF16 deviations from the rest
    state, FP32 arithmetic), or ``"fp16dev_sr"`` / ``"bf16dev_sr"`` (the same,
    the collision rounding the stored deviations stochastically); ``variant``
    is ``"A"``, ``"B"`` or ``"C"``;
    ``integrator`` is ``"start"`` (coupling force from the start of the MD
    step, Eq. (6)) or ``"half_step"`` (from the half-step velocity after the
    drift); ``noise`` is ``"uniform"`` (default) or ``"gauss"`` (normal
    variates by Box-Muller); ``spread`` (variant B) is ``"auto"``, ``"tiles"``, ``"rows"`` or ``"atomic"``
    (the path that hands the transfers to the nodes; bitwise the same
    results).
    """

    def __init__(self, nx, ny, nz, *, variant="B", precision="fp32", **kw):
        v = {"A": VARIANT_A, "B": VARIANT_B, "C": VARIANT_C, 0: VARIANT_A, 1: VARIANT_B, 2: VARIANT_C}[variant]
        pr = PRECISIONS[precision] if isinstance(precision, str) else int(precision)
        self.params = make_params(nx, ny, nz, variant=v, precision=pr, **kw)
        self.shape = (int(nx), int(ny), int(nz))
        self.n_nodes = int(nx) * int(ny) * int(nz)
        self.n_sub = self.params.n_sub
        self._pending = []  # host objects the asynchronous accessors still use
        self._h = lbmd_create(self.params)

    @property
    def handle(self):
        return self._h

    def close(self):
        if getattr(self, "_h", None) is not None and self._h.value:
            lbmd_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()

    # sequence ---------------------------------------------------------------
    def add_particles(self, pos, vel, mass=None) -> int:
        pos = _f64(pos).reshape(-1, 3)
        vel = _f64(vel).reshape(-1, 3)
        n = pos.shape[0]
        m = None if mass is None else _f64(mass, n)
        first = ct.c_int64(0)
        dp = ct.POINTER(ct.c_double)
        _check(self._h, load().lbmd_add_particles(
            self._h, n, pos.ctypes.data_as(dp), vel.ctypes.data_as(dp),
            None if m is None else m.ctypes.data_as(dp), ct.byref(first)), "lbmd_add_particles")
        return first.value

    def add_bonds(self, pairs, k, r0):
        pairs = np.ascontiguousarray(pairs, dtype=np.int64).reshape(-1, 2)
        _check(self._h, load().lbmd_add_bonds(self._h, pairs.shape[0], pairs.ctypes.data_as(ct.POINTER(ct.c_int64)),
                                              float(k), float(r0)), "lbmd_add_bonds")

    def add_fene_bonds(self, pairs, k, R0):
        """FENE springs U = -(k/2) R0^2 ln(1 - (r/R0)^2) (Kremer-Grest chains, Sec. 4)."""
        pairs = np.ascontiguousarray(pairs, dtype=np.int64).reshape(-1, 2)
        _check(self._h, load().lbmd_add_fene_bonds(self._h, pairs.shape[0],
                                                   pairs.ctypes.data_as(ct.POINTER(ct.c_int64)), float(k), float(R0)),
               "lbmd_add_fene_bonds")

    def save_state(self) -> bytes:
        """The context's state at a cycle boundary (populations, particles,
        bonds, LJ parameters, step counters) as bytes; load_state restores it."""
        size = ct.c_int64(0)
        _check(self._h, load().lbmd_state_size(self._h, ct.byref(size)), "lbmd_state_size")
        buf = ct.create_string_buffer(size.value)
        _check(self._h, load().lbmd_save_state(self._h, buf, size.value), "lbmd_save_state")
        return buf.raw

    def load_state(self, state: bytes):
        """Restore a saved state into this context (same parameters, no particles yet)."""
        buf = ct.create_string_buffer(bytes(state), len(state))
        _check(self._h, load().lbmd_load_state(self._h, buf, len(state)), "lbmd_load_state")

    def set_lj(self, eps, sigma, r_cut):
        """Lennard-Jones between all particles, cut off (and shifted) at r_cut; r_cut = 0: off (Sec. 4)."""
        _check(self._h, load().lbmd_set_lj(self._h, float(eps), float(sigma), float(r_cut)), "lbmd_set_lj")

    def set_particles(self, pos=None, vel=None):
        """Host arrays (numpy or pinned torch tensors, float64, 3 N each)."""
        self._keep = (pos, vel)
        _check(self._h, load().lbmd_set_particles(self._h, _host_addr(pos), _host_addr(vel)), "lbmd_set_particles")

    def md_substep(self):
        return lbmd_md_substep(self._h)

    def lb_step(self):
        return lbmd_lb_step(self._h)

    def cycle(self, k: int = 1):
        for _ in range(int(k)):
            for _ in range(self.n_sub):
                lbmd_md_substep(self._h)
            lbmd_lb_step(self._h)

    def run_cycles(self, k: int):
        return lbmd_run_cycles(self._h, k)

    # accessors ----------------------------------------------------------------
    def observables(self) -> dict:
        return lbmd_observables(self._h)

    def populations(self) -> np.ndarray:
        out = np.empty(19 * self.n_nodes)
        _check(self._h, load().lbmd_get_populations(self._h, _ptr(out)), "lbmd_get_populations")
        return out.reshape(19, self.n_nodes)

    def set_populations(self, f):
        f = _f64(f, 19 * self.n_nodes)
        _check(self._h, load().lbmd_set_populations(self._h, _ptr(f)), "lbmd_set_populations")

    def node_field(self) -> np.ndarray:
        out = np.empty(4 * self.n_nodes)
        _check(self._h, load().lbmd_get_node_field(self._h, _ptr(out)), "lbmd_get_node_field")
        return out.reshape(self.n_nodes, 4)

    def transfer(self) -> np.ndarray:
        out = np.empty(3 * self.n_nodes)
        _check(self._h, load().lbmd_get_transfer(self._h, _ptr(out)), "lbmd_get_transfer")
        return out.reshape(self.n_nodes, 3)

    def counts(self):
        a, b, c, d = (ct.c_int64() for _ in range(4))
        e = ct.c_int32()
        load().lbmd_get_counts(self._h, ct.byref(a), ct.byref(b), ct.byref(c), ct.byref(d), ct.byref(e))
        return {"n_particles": a.value, "n_bonds": b.value, "lb_step": c.value, "md_step": d.value,
                "substeps_done": e.value}

    @property
    def n_particles(self) -> int:
        return self.counts()["n_particles"]

    def particles(self, out=None):
        """Positions and velocities in id order as (n, 3) arrays; with out =
        (pos, vel), caller host arrays of 3 N float64 (numpy or pinned torch
        tensors) are filled and returned instead."""
        if out is not None:
            _check(self._h, load().lbmd_get_particles(self._h, _host_addr(out[0]), _host_addr(out[1])),
                   "lbmd_get_particles")
            return out
        n = self.n_particles
        pos = np.empty(3 * max(n, 1))
        vel = np.empty(3 * max(n, 1))
        _check(self._h, load().lbmd_get_particles(self._h, _ptr(pos), _ptr(vel)), "lbmd_get_particles")
        return pos[:3 * n].reshape(n, 3), vel[:3 * n].reshape(n, 3)

    # asynchronous accessors: enqueue only; host arrays stay in use until synchronize()
    def set_particles_async(self, pos=None, vel=None):
        """Enqueue an upload of host arrays (pinned torch tensors or numpy,
        float64, 3 N each), which must stay unchanged until synchronize()."""
        self._pending.append((pos, vel))
        _check(self._h, load().lbmd_set_particles_async(self._h, _host_addr(pos), _host_addr(vel)),
               "lbmd_set_particles_async")

    def particles_async(self, pos, vel):
        """Enqueue a download of the positions and velocities at this point of
        the stream order into host arrays of 3 N float64 (either may be None),
        filled once synchronize() returns."""
        self._pending.append((pos, vel))
        _check(self._h, load().lbmd_get_particles_async(self._h, _host_addr(pos), _host_addr(vel)),
               "lbmd_get_particles_async")

    def observables_async(self) -> LbmdObservables:
        """Enqueue the observables at this point of the stream order; the
        returned structure is filled (observables_dict() reads it) once
        synchronize() returns, which also reports its checks."""
        o = LbmdObservables()
        self._pending.append(o)
        _check(self._h, load().lbmd_observables_async(self._h, ct.byref(o)), "lbmd_observables_async")
        return o

    def synchronize(self):
        """Wait for all enqueued work and complete the queued observables."""
        st = load().lbmd_synchronize(self._h)
        self._pending = []
        _check(self._h, st, "lbmd_synchronize")

    def set_moments_wait(self, polls: int):
        """Poll limit of the fused post-stream moments' wait (-1: default, 0:
        every row to the follow-up kernel); results do not depend on it."""
        _check(self._h, load().lbmd_set_moments_wait(self._h, int(polls)), "lbmd_set_moments_wait")

    def set_frozen_copy(self, on: bool):
        """Variant A: read the frozen node velocities from a copy of the
        compact records (True) or the node field (False); same results.  Only
        at a cycle boundary."""
        _check(self._h, load().lbmd_set_frozen_copy(self._h, 1 if on else 0), "lbmd_set_frozen_copy")

    def moments_fallback_rows(self) -> int:
        """Rows whose fused moments the follow-up kernel computed, since creation."""
        v = ct.c_int64(0)
        _check(self._h, load().lbmd_moments_fallback_rows(self._h, ct.byref(v)), "lbmd_moments_fallback_rows")
        return v.value

    def particles_device(self, pos, vel):
        """Stream-ordered copy into caller-owned device tensors (float64, 3 N)."""
        _check(self._h, load().lbmd_get_particles_device(
            self._h, None if pos is None else ct.c_void_p(pos.data_ptr()),
            None if vel is None else ct.c_void_p(vel.data_ptr())), "lbmd_get_particles_device")

    @property
    def stream(self) -> int:
        return load().lbmd_stream(self._h) or 0


# ---------------------------------------------------------------------------
# Batched replicas
# ---------------------------------------------------------------------------
def _bcheck(h, rc, what):
    if rc != LBMD_OK:
        L = load()
        msg = L.lbmd_batch_last_error(h).decode(errors="replace")
        err = LbmdError(rc, what)
        err.args = ("%s failed: %s (status %d: %s)" % (what, msg, rc, L.lbmd_status_string(rc).decode()),)
        raise err
    return rc


class Batch:
    """Many independent replica boxes advanced together (``lbmd_batch_*``).

    ``dims``: R x 3 lattice sizes; ``n_sub``, ``variant`` ("A"/"B" or 0/1),
    ``zeta``, ``seed``, ``max_particles``: one per replica (scalars are
    broadcast).  ``rho0``, ``nu``, ``nu_bulk``, ``gamma_ghost``, ``kT`` are
    shared.  Replica r evolves as ``LBMD(*dims[r], n_sub=n_sub[r], ...,
    seed=seed[r])`` would.
    """

    def __init__(self, dims, *, n_sub=1, variant="B", zeta=1.0, seed=1, max_particles=0, precision="fp32",
                 rho0=1.0, nu=1.0 / 6.0, nu_bulk=-1.0, gamma_ghost=0.0, kT=0.0, stream=None):
        dims = np.ascontiguousarray(dims, dtype=np.int32).reshape(-1, 3)
        R = dims.shape[0]

        def per(x, dtype):
            a = np.asarray(x)
            if a.ndim == 0:
                a = np.full(R, a)
            return np.ascontiguousarray(a, dtype=dtype).reshape(R)

        vmap = {"A": VARIANT_A, "B": VARIANT_B, 0: VARIANT_A, 1: VARIANT_B}
        if isinstance(variant, str) or np.asarray(variant).ndim == 0:
            variant = [variant] * R
        self.dims = dims
        self.n_sub = per(n_sub, np.int32)
        self.variant = np.array([vmap[v] for v in variant], dtype=np.int32)
        self.zeta = per(zeta, np.float64)
        self.seed = per(seed, np.uint64)
        self.max_particles = per(max_particles, np.int32)
        self.R = R
        p = LbmdBatchParams()
        p.n_replicas = R
        p.dims, p.n_sub, p.variant = _ptr(self.dims), _ptr(self.n_sub), _ptr(self.variant)
        p.zeta, p.seed, p.max_particles = _ptr(self.zeta), _ptr(self.seed), _ptr(self.max_particles)
        p.precision = PRECISIONS[precision] if isinstance(precision, str) else int(precision)
        p.rho0, p.nu, p.nu_bulk, p.gamma_ghost, p.kT = float(rho0), float(nu), float(nu_bulk), float(gamma_ghost), \
            float(kT)
        p.stream = stream
        self._h = ct.c_void_p()
        _bcheck(None, load().lbmd_batch_create(ct.byref(p), ct.byref(self._h)), "lbmd_batch_create")

    def close(self):
        if getattr(self, "_h", None) is not None and self._h.value:
            load().lbmd_batch_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def n_nodes(self, r: int) -> int:
        return int(np.prod(self.dims[r]))

    def add_particles(self, r: int, pos, vel, mass=None):
        pos = _f64(pos).reshape(-1, 3)
        vel = _f64(vel).reshape(-1, 3)
        m = None if mass is None else _f64(mass, pos.shape[0])
        _bcheck(self._h, load().lbmd_batch_add_particles(self._h, int(r), pos.shape[0], _ptr(pos), _ptr(vel),
                                                         None if m is None else _ptr(m)), "lbmd_batch_add_particles")

    def run(self, md_steps: int):
        _bcheck(self._h, load().lbmd_batch_run(self._h, int(md_steps)), "lbmd_batch_run")

    def kinetic(self) -> np.ndarray:
        """R x 5: sum m v^2, sum m v (3), particle count."""
        out = np.empty(5 * self.R)
        _bcheck(self._h, load().lbmd_batch_kinetic(self._h, _ptr(out)), "lbmd_batch_kinetic")
        return out.reshape(self.R, 5)

    def kinetic_device(self, out_ptr: int):
        """Stream-ordered: 5 R doubles into caller-owned device memory."""
        _bcheck(self._h, load().lbmd_batch_kinetic_device(self._h, ct.c_void_p(out_ptr)),
                "lbmd_batch_kinetic_device")

    def unstable(self) -> np.ndarray:
        out = np.empty(self.R, dtype=np.int32)
        _bcheck(self._h, load().lbmd_batch_unstable(self._h, _ptr(out)), "lbmd_batch_unstable")
        return out

    def populations(self, r: int) -> np.ndarray:
        out = np.empty(19 * self.n_nodes(r))
        _bcheck(self._h, load().lbmd_batch_get_populations(self._h, int(r), _ptr(out)), "lbmd_batch_get_populations")
        return out.reshape(19, -1)

    def set_populations(self, r: int, f):
        f = _f64(f, 19 * self.n_nodes(r))
        _bcheck(self._h, load().lbmd_batch_set_populations(self._h, int(r), _ptr(f)), "lbmd_batch_set_populations")

    def counts(self, r: int) -> dict:
        a, b, c = ct.c_int64(), ct.c_int64(), ct.c_int64()
        _bcheck(self._h, load().lbmd_batch_get_counts(self._h, int(r), ct.byref(a), ct.byref(b), ct.byref(c)),
                "lbmd_batch_get_counts")
        return {"n_particles": a.value, "lb_step": b.value, "md_step": c.value}

    def particles(self, r: int):
        n = self.counts(r)["n_particles"]
        pos, vel = np.empty(3 * max(n, 1)), np.empty(3 * max(n, 1))
        if n:
            _bcheck(self._h, load().lbmd_batch_get_particles(self._h, int(r), _ptr(pos), _ptr(vel)),
                    "lbmd_batch_get_particles")
        return pos[:3 * n].reshape(n, 3), vel[:3 * n].reshape(n, 3)

    def tuning(self) -> dict:
        nb, pb = ct.c_int32(), ct.c_int32()
        lb, pt = np.zeros(3), np.zeros(3)
        _bcheck(self._h, load().lbmd_batch_tuning(self._h, ct.byref(nb), ct.byref(pb), _ptr(lb), _ptr(pt)),
                "lbmd_batch_tuning")
        return {"nodes_per_block": nb.value, "particle_block": pb.value, "candidates": [64, 128, 256],
                "lb_ms": lb.tolist(), "particle_ms": pt.tolist()}

    def set_lb_grid(self, max_blocks: int):
        """Cap on the blocks of the persistent LB kernels (0: as many as fit)."""
        _bcheck(self._h, load().lbmd_batch_set_lb_grid(self._h, int(max_blocks)), "lbmd_batch_set_lb_grid")

    def set_schedule(self, schedule: str, cluster_blocks: int = 0):
        """Schedule of run(): "period_graph" (per-tick kernels, a period
        replayed from a CUDA graph) or "persistent" (one launch per call,
        thread-block clusters of cluster_blocks blocks each running whole
        replicas; 0 = the tuned size)."""
        _bcheck(self._h, load().lbmd_batch_set_schedule(self._h, BATCH_SCHEDULES[schedule], int(cluster_blocks)),
                "lbmd_batch_set_schedule")

    def persistent_tuning(self) -> dict:
        c = ct.c_int32()
        ms = np.zeros(5)
        _bcheck(self._h, load().lbmd_batch_persistent_tuning(self._h, ct.byref(c), _ptr(ms)),
                "lbmd_batch_persistent_tuning")
        return {"cluster_blocks": c.value, "candidates": [1, 2, 4, 8, 16], "period_ms": ms.tolist()}

    @property
    def stream(self) -> int:
        return load().lbmd_batch_stream(self._h) or 0


# ---------------------------------------------------------------------------
# Adjoint of the coupled step (mean particle drag along x)
# ---------------------------------------------------------------------------
def _acheck(h, rc, what):
    if rc != LBMD_OK:
        L = load()
        msg = L.lbmd_adjoint_last_error(h).decode(errors="replace")
        err = LbmdError(rc, what)
        err.args = ("%s failed: %s (status %d: %s)" % (what, msg, rc, L.lbmd_status_string(rc).decode()),)
        raise err
    return rc


class Adjoint:
    """``lbmd_adjoint_*``: L(zeta, R0) = mean particle drag F_x over K cycles
    of m MD steps (variant B, fluid starting at rest, ideal particles of mass
    1), its value (``forward``) and its gradient (``backward``) from the
    hand-written adjoint kernels."""

    def __init__(self, nx, ny, nz, *, n_particles, n_cycles, n_sub=10, precision="fp64", rho0=1.0, nu=1.0 / 6.0,
                 nu_bulk=-1.0, gamma_ghost=0.0, kT=0.0, body_force=(0.0, 0.0, 0.0), seed=1, stream=None):
        p = LbmdAdjointParams()
        p.nx, p.ny, p.nz, p.n_sub = int(nx), int(ny), int(nz), int(n_sub)
        p.n_particles, p.n_cycles = int(n_particles), int(n_cycles)
        p.precision = PRECISIONS[precision] if isinstance(precision, str) else int(precision)
        p.rho0, p.nu, p.nu_bulk, p.gamma_ghost, p.kT = float(rho0), float(nu), float(nu_bulk), float(gamma_ghost), \
            float(kT)
        for a in range(3):
            p.body_force[a] = float(body_force[a])
        p.seed = int(seed)
        p.stream = stream
        self.n_particles = int(n_particles)
        self._h = ct.c_void_p()
        _acheck(None, load().lbmd_adjoint_create(ct.byref(p), ct.byref(self._h)), "lbmd_adjoint_create")

    def close(self):
        if getattr(self, "_h", None) is not None and self._h.value:
            load().lbmd_adjoint_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def forward(self, zeta: float, pos0, vel0) -> float:
        pos0 = _f64(pos0, 3 * self.n_particles)
        vel0 = _f64(vel0, 3 * self.n_particles)
        out = ct.c_double()
        _acheck(self._h, load().lbmd_adjoint_forward(self._h, float(zeta), _ptr(pos0), _ptr(vel0), ct.byref(out)),
                "lbmd_adjoint_forward")
        return out.value

    def backward(self):
        """(dL/dzeta, dL/dR0 as an N_p x 3 array) of the last forward pass."""
        dz = ct.c_double()
        dpos = np.zeros(3 * max(self.n_particles, 1))
        _acheck(self._h, load().lbmd_adjoint_backward(self._h, ct.byref(dz), _ptr(dpos)), "lbmd_adjoint_backward")
        return dz.value, dpos[:3 * self.n_particles].reshape(-1, 3)


def drag_function(adjoint: Adjoint, vel0):
    """A ``torch.autograd.Function`` L(zeta, R0) backed by ``adjoint``: its
    forward runs the forward pass, its backward the adjoint kernels.  zeta is
    a 0-d tensor, R0 an N_p x 3 tensor (float64, CPU); vel0 is fixed."""
    import torch

    vel0 = np.ascontiguousarray(vel0, dtype=np.float64)

    class _Drag(torch.autograd.Function):
        @staticmethod
        def forward(ctx, zeta, pos0):
            loss = adjoint.forward(float(zeta), pos0.detach().cpu().numpy(), vel0)
            return torch.tensor(loss, dtype=torch.float64)

        @staticmethod
        def backward(ctx, grad):
            dz, dpos = adjoint.backward()
            g = float(grad)
            return torch.tensor(g * dz, dtype=torch.float64), torch.from_numpy(g * dpos)

    return _Drag.apply
