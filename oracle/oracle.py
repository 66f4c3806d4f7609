"""ctypes front end of the FP64 CPU oracle (``lbmd_oracle.c``).

TEST INFRASTRUCTURE: only ``tests/``, ``__graft_entry__.smoke()`` and the
CPU-baseline leg of ``bench.py`` import this module.  The product library
(``paper_1610_02733_gb300``) never does.

``build()`` compiles the C oracle with gcc into ``oracle/_build``.  The
``Oracle`` class mirrors the state machine of the paper's coupled LB/MD
scheme (Sec. 3): ``md_substep`` m times, then ``lb_step``.
"""
from __future__ import annotations

import ctypes as ct
import os
import subprocess

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_BUILD = os.path.join(_HERE, "_build")
_LIB_PATH = os.path.join(_BUILD, "liblbmd_oracle.so")
# timing build for the all-cores CPU baseline: the same sources with OpenMP
# (the LB node loops run over threads; the particle loop stays serial)
_OMP_PATH = os.path.join(_BUILD, "liblbmd_oracle_omp.so")
_SRC = os.path.join(_HERE, "lbmd_oracle.c")
_SRCS = [_SRC, os.path.join(_HERE, "lbmd_tangent.c")]

ORC_OK = 0
ORC_ERR_SEQUENCE = -4


def _compile(path: str, extra, force: bool) -> str:
    os.makedirs(_BUILD, exist_ok=True)
    hdr = os.path.join(_HERE, "lbmd_oracle.h")
    if (not force and os.path.exists(path)
            and os.path.getmtime(path) >= max([os.path.getmtime(f) for f in _SRCS] + [os.path.getmtime(hdr)])):
        return path
    tmp = path + ".tmp%d" % os.getpid()
    cmd = ["gcc", "-std=c99", "-O2", "-fno-fast-math", "-ffp-contract=off", "-fPIC", "-shared"] + list(extra) + \
          ["-o", tmp] + _SRCS + ["-lm"]
    subprocess.check_call(cmd)
    os.replace(tmp, path)
    return path


def build(force: bool = False) -> str:
    """Compile the oracle (plain C99, -O2, no fast-math, single thread) and
    return the path; also the OpenMP timing build where gcc supports it."""
    path = _compile(_LIB_PATH, [], force)
    try:
        build_openmp(force)
    except (subprocess.CalledProcessError, OSError):
        pass  # no OpenMP runtime: the all-cores baseline reports itself unavailable
    return path


def build_openmp(force: bool = False) -> str:
    """The timing build: the same sources with -fopenmp (identical results)."""
    return _compile(_OMP_PATH, ["-fopenmp"], force)


class OrcParams(ct.Structure):
    _fields_ = [
        ("nx", ct.c_int32), ("ny", ct.c_int32), ("nz", ct.c_int32),
        ("n_sub", ct.c_int32), ("variant", ct.c_int32), ("integrator", ct.c_int32),
        ("rho0", ct.c_double), ("nu", ct.c_double), ("nu_bulk", ct.c_double),
        ("gamma_ghost", ct.c_double), ("kT", ct.c_double), ("zeta", ct.c_double),
        ("body_force", ct.c_double * 3), ("seed", ct.c_uint64), ("noise", ct.c_int32),
    ]


_libs = {}


def lib(openmp: bool = False):
    """The oracle library (openmp: the timing build)."""
    key = bool(openmp)
    if key not in _libs:
        L = ct.CDLL(build_openmp() if openmp else build())
        _libs[key] = L
        P = ct.c_void_p
        dp = ct.POINTER(ct.c_double)
        L.orc_create.restype = P
        L.orc_create.argtypes = [ct.POINTER(OrcParams)]
        L.orc_destroy.argtypes = [P]
        L.orc_add_particles.argtypes = [P, ct.c_int64, dp, dp, dp]
        L.orc_add_bonds.argtypes = [P, ct.c_int64, ct.POINTER(ct.c_int64), ct.c_double, ct.c_double]
        L.orc_add_fene_bonds.argtypes = [P, ct.c_int64, ct.POINTER(ct.c_int64), ct.c_double, ct.c_double]
        L.orc_set_lj.argtypes = [P, ct.c_double, ct.c_double, ct.c_double]
        L.orc_conservative_forces.argtypes = [P, dp, dp]
        L.orc_md_substep.argtypes = [P]
        L.orc_lb_step.argtypes = [P]
        L.orc_observables.argtypes = [P, dp]
        for name in ("orc_get_populations", "orc_set_populations", "orc_get_jacc", "orc_set_jacc",
                     "orc_get_node_field", "orc_get_coupling_forces"):
            getattr(L, name).argtypes = [P, dp]
        L.orc_get_particles.argtypes = [P, dp, dp]
        L.orc_set_particles.argtypes = [P, dp, dp]
        L.orc_counters.argtypes = [P, ct.POINTER(ct.c_int64)]
        L.orc_set_counters.argtypes = [P, ct.c_int64, ct.c_int64]
        L.orc_num_particles.restype = ct.c_int64
        L.orc_num_particles.argtypes = [P]
        u32p = ct.POINTER(ct.c_uint32)
        L.orc_philox4x32_10.argtypes = [u32p, u32p, u32p]
        L.orc_uniform_unit.restype = ct.c_double
        L.orc_uniform_unit.argtypes = [ct.c_uint32]
        L.orc_uniform_unit16.restype = ct.c_double
        L.orc_uniform_unit16.argtypes = [ct.c_uint32]
        L.orc_box_muller.argtypes = [ct.c_uint32, ct.c_uint32, dp]
        L.orc_d3q19.argtypes = [ct.POINTER(ct.c_int32), dp]
        L.orc_modes.argtypes = [dp, dp]
        L.orc_collide_node.argtypes = [P, dp, dp, ct.c_uint32, ct.c_uint32, dp]
        L.orc_trilinear.argtypes = [P, dp, ct.POINTER(ct.c_int64), dp]
        L.orc_round_storage.restype = ct.c_double
        L.orc_round_storage.argtypes = [ct.c_double, ct.c_int, ct.c_int, ct.c_uint32, ct.c_int]
        L.orc_round_storage_n.argtypes = [ct.c_int64, dp, ct.c_int, ct.c_int, u32p, ct.c_int, dp]
        L.orc_sr_bits_n.argtypes = [ct.c_uint64, ct.c_int64, u32p, ct.c_uint32, u32p]
        L.tan_create.restype = P
        L.tan_create.argtypes = [ct.POINTER(OrcParams)]
        L.tan_destroy.argtypes = [P]
        L.tan_set_particles.argtypes = [P, ct.c_int64, dp, dp, dp, ct.c_double]
        L.tan_md_substep.argtypes = [P]
        L.tan_lb_step.argtypes = [P]
        L.tan_drag.argtypes = [P, dp]
        L.tan_get_populations.argtypes = [P, dp, dp]
        L.tan_get_particles.argtypes = [P, dp, dp, dp, dp]
    return _libs[key]


def _dp(a: np.ndarray):
    return a.ctypes.data_as(ct.POINTER(ct.c_double))


def _f64(a) -> np.ndarray:
    return np.ascontiguousarray(a, dtype=np.float64)


def philox4x32_10(ctr, key) -> np.ndarray:
    c = (ct.c_uint32 * 4)(*[int(x) & 0xFFFFFFFF for x in ctr])
    k = (ct.c_uint32 * 2)(*[int(x) & 0xFFFFFFFF for x in key])
    o = (ct.c_uint32 * 4)()
    lib().orc_philox4x32_10(c, k, o)
    return np.array(list(o), dtype=np.uint32)


def uniform_unit(x: int) -> float:
    return lib().orc_uniform_unit(int(x) & 0xFFFFFFFF)


def box_muller(w1: int, w2: int):
    """The two standard normal variates of the Gaussian noise option from two
    32-bit Philox words."""
    out = np.zeros(2)
    lib().orc_box_muller(int(w1) & 0xFFFFFFFF, int(w2) & 0xFFFFFFFF, _dp(out))
    return out


def uniform_unit16(h: int) -> float:
    return lib().orc_uniform_unit16(int(h) & 0xFFFFFFFF)


# Binary grids of the reduced-precision population storage: (significand
# bits p, minimum normal exponent emin).
STORAGE_FORMATS = {"fp16": (11, -14), "bf16": (8, -126)}


def round_storage(x, fmt, r=None):
    """x rounded onto the FP16 / BF16 grid: to nearest (ties to even) when r
    is None, else stochastically with the 16-bit random numbers r (one per
    element)."""
    x = _f64(x)
    p, emin = STORAGE_FORMATS[fmt]
    out = np.empty_like(x)
    rp = None
    if r is not None:
        r = np.ascontiguousarray(np.broadcast_to(r, x.shape), dtype=np.uint32)
        rp = r.ctypes.data_as(ct.POINTER(ct.c_uint32))
    lib().orc_round_storage_n(x.size, _dp(x), p, emin, rp, 0 if r is None else 1, _dp(out))
    return out


def sr_bits(seed, nodes, lb_step):
    """The 16-bit random numbers of the stochastic rounding: array (len(nodes),
    19), population i of node nodes[k]'s post-collision state in LB step
    lb_step."""
    nodes = np.ascontiguousarray(nodes, dtype=np.uint32)
    out = np.empty((nodes.size, 19), dtype=np.uint32)
    u32p = ct.POINTER(ct.c_uint32)
    lib().orc_sr_bits_n(int(seed), nodes.size, nodes.ctypes.data_as(u32p), int(lb_step) & 0xFFFFFFFF,
                        out.ctypes.data_as(u32p))
    return out


def d3q19():
    c = np.zeros(57, dtype=np.int32)
    w = np.zeros(19)
    lib().orc_d3q19(c.ctypes.data_as(ct.POINTER(ct.c_int32)), _dp(w))
    return c.reshape(19, 3), w


def modes():
    e = np.zeros(19 * 19)
    b = np.zeros(19)
    lib().orc_modes(_dp(e), _dp(b))
    return e.reshape(19, 19), b


class Oracle:
    """The oracle's state: populations, pending momentum transfer, particles.

    Parameters follow the C-ABI of the GPU library: lattice units (a = 1,
    tau_LB = 1), ``n_sub`` = m MD steps per LB step, ``variant`` 0 = A, 1 = B, 2 = C,
    ``integrator`` 0 = coupling force from the start of the MD step (Eq. (6)),
    1 = from the half-step velocity after the drift (see orc_md_substep).
    ``noise``: 0 / "uniform" (unit-variance uniform variates), 1 / "gauss"
    (standard normal variates by Box-Muller).
    """

    def __init__(self, nx, ny, nz, *, n_sub=1, variant=1, rho0=1.0, nu=1.0 / 6.0, nu_bulk=-1.0,
                 gamma_ghost=0.0, kT=0.0, zeta=1.0, body_force=(0.0, 0.0, 0.0), seed=1, integrator=0,
                 noise=0, openmp=False):
        p = OrcParams()
        p.noise = {"uniform": 0, "gauss": 1}.get(noise, noise)
        p.nx, p.ny, p.nz = int(nx), int(ny), int(nz)
        p.n_sub, p.variant, p.integrator = int(n_sub), int(variant), int(integrator)
        p.rho0, p.nu, p.nu_bulk, p.gamma_ghost = float(rho0), float(nu), float(nu_bulk), float(gamma_ghost)
        p.kT, p.zeta = float(kT), float(zeta)
        for a in range(3):
            p.body_force[a] = float(body_force[a])
        p.seed = int(seed)
        self.params = p
        self.shape = (int(nx), int(ny), int(nz))
        self.n_nodes = int(nx) * int(ny) * int(nz)
        self.n_sub = int(n_sub)
        self._lib = lib(openmp)
        h = self._lib.orc_create(ct.byref(p))
        if not h:
            raise ValueError("orc_create rejected the parameters")
        self._h = ct.c_void_p(h)

    def close(self):
        if getattr(self, "_h", None) is not None and self._h.value:
            self._lib.orc_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    # state machine ---------------------------------------------------------
    def add_particles(self, pos, vel, mass=None):
        pos = _f64(pos).reshape(-1, 3)
        vel = _f64(vel).reshape(-1, 3)
        m = None if mass is None else _f64(mass).reshape(-1)
        rc = self._lib.orc_add_particles(self._h, pos.shape[0], _dp(pos), _dp(vel),
                                     None if m is None else _dp(m))
        if rc != ORC_OK:
            raise RuntimeError("orc_add_particles: %d" % rc)

    def add_bonds(self, pairs, k, r0):
        pairs = np.ascontiguousarray(pairs, dtype=np.int64).reshape(-1, 2)
        rc = self._lib.orc_add_bonds(self._h, pairs.shape[0], pairs.ctypes.data_as(ct.POINTER(ct.c_int64)),
                                 float(k), float(r0))
        if rc != ORC_OK:
            raise RuntimeError("orc_add_bonds: %d" % rc)

    def add_fene_bonds(self, pairs, k, R0):
        """FENE springs U = -(k/2) R0^2 ln(1 - (r/R0)^2) (Sec. 4)."""
        pairs = np.ascontiguousarray(pairs, dtype=np.int64).reshape(-1, 2)
        rc = self._lib.orc_add_fene_bonds(self._h, pairs.shape[0], pairs.ctypes.data_as(ct.POINTER(ct.c_int64)),
                                      float(k), float(R0))
        if rc != ORC_OK:
            raise RuntimeError("orc_add_fene_bonds: %d" % rc)

    def set_lj(self, eps, sigma, rc):
        """Lennard-Jones between all particles, cut off (and shifted to 0) at rc (Sec. 4)."""
        r = self._lib.orc_set_lj(self._h, float(eps), float(sigma), float(rc))
        if r != ORC_OK:
            raise RuntimeError("orc_set_lj: %d" % r)

    def conservative_forces(self):
        """(forces (np, 3), energies {harmonic, fene, lj}) at the current positions."""
        n = self.n_particles
        out = np.zeros((max(n, 1), 3))
        e = np.zeros(3)
        self._lib.orc_conservative_forces(self._h, _dp(out), _dp(e))
        return out[:n], {"harmonic": float(e[0]), "fene": float(e[1]), "lj": float(e[2])}

    def md_substep(self) -> int:
        return self._lib.orc_md_substep(self._h)

    def lb_step(self) -> int:
        return self._lib.orc_lb_step(self._h)

    def cycle(self, k: int = 1):
        for _ in range(k):
            for _ in range(self.n_sub):
                rc = self.md_substep()
                assert rc == ORC_OK, rc
            rc = self.lb_step()
            assert rc == ORC_OK, rc

    # accessors -------------------------------------------------------------
    def observables(self) -> dict:
        o = np.zeros(11)
        self._lib.orc_observables(self._h, _dp(o))
        return {"mass": o[0], "p_fluid": o[1:4].copy(), "p_particles": o[4:7].copy(),
                "kT_particles": o[7], "e_kin": o[8], "lb_step": int(o[9]), "md_step": int(o[10])}

    def populations(self) -> np.ndarray:
        out = np.zeros(19 * self.n_nodes)
        self._lib.orc_get_populations(self._h, _dp(out))
        return out.reshape(19, self.n_nodes)

    def set_populations(self, f):
        f = _f64(f).reshape(-1)
        assert f.size == 19 * self.n_nodes
        self._lib.orc_set_populations(self._h, _dp(f))

    def jacc(self) -> np.ndarray:
        out = np.zeros(3 * self.n_nodes)
        self._lib.orc_get_jacc(self._h, _dp(out))
        return out.reshape(self.n_nodes, 3)

    def set_jacc(self, j):
        j = _f64(j).reshape(-1)
        assert j.size == 3 * self.n_nodes
        self._lib.orc_set_jacc(self._h, _dp(j))

    def node_field(self) -> np.ndarray:
        out = np.zeros(4 * self.n_nodes)
        self._lib.orc_get_node_field(self._h, _dp(out))
        return out.reshape(self.n_nodes, 4)

    @property
    def n_particles(self) -> int:
        return int(self._lib.orc_num_particles(self._h))

    def particles(self):
        n = self.n_particles
        pos = np.zeros(3 * max(n, 1))
        vel = np.zeros(3 * max(n, 1))
        self._lib.orc_get_particles(self._h, _dp(pos), _dp(vel))
        return pos[:3 * n].reshape(n, 3), vel[:3 * n].reshape(n, 3)

    def set_particles(self, pos=None, vel=None):
        n = self.n_particles
        p = None if pos is None else _f64(pos).reshape(n, 3)
        v = None if vel is None else _f64(vel).reshape(n, 3)
        self._lib.orc_set_particles(self._h, None if p is None else _dp(p), None if v is None else _dp(v))

    def coupling_forces(self) -> np.ndarray:
        n = self.n_particles
        out = np.zeros(3 * max(n, 1))
        self._lib.orc_get_coupling_forces(self._h, _dp(out))
        return out[:3 * n].reshape(n, 3)

    def counters(self):
        o = (ct.c_int64 * 3)()
        self._lib.orc_counters(self._h, o)
        return int(o[0]), int(o[1]), int(o[2])

    def set_counters(self, lb_step, md_step):
        self._lib.orc_set_counters(self._h, int(lb_step), int(md_step))

    # building blocks ---------------------------------------------------------
    def collide_node(self, f, F, node=0, lb_step=0) -> np.ndarray:
        f = _f64(f).reshape(19)
        F = _f64(F).reshape(3)
        out = np.zeros(19)
        self._lib.orc_collide_node(self._h, _dp(f), _dp(F), int(node), int(lb_step), _dp(out))
        return out

    def trilinear(self, R):
        R = _f64(R).reshape(3)
        corner = np.zeros(8, dtype=np.int64)
        delta = np.zeros(8)
        self._lib.orc_trilinear(self._h, _dp(R), corner.ctypes.data_as(ct.POINTER(ct.c_int64)), _dp(delta))
        return corner, delta


class Tangent:
    """Forward-mode derivative of the oracle's step (``lbmd_tangent.c``):
    the same state as ``Oracle`` carried as (value, derivative along one
    direction of zeta and the initial positions).  Ideal particles, mass 1.
    ``drag()`` returns (S, dS) with S the sum of the coupling force F_x over
    the MD steps done and the particles."""

    def __init__(self, nx, ny, nz, *, n_sub=1, variant=1, rho0=1.0, nu=1.0 / 6.0, nu_bulk=-1.0,
                 gamma_ghost=0.0, kT=0.0, zeta=1.0, body_force=(0.0, 0.0, 0.0), seed=1):
        p = OrcParams()
        p.nx, p.ny, p.nz, p.n_sub, p.variant = nx, ny, nz, n_sub, variant
        p.rho0, p.nu, p.nu_bulk, p.gamma_ghost, p.kT, p.zeta = rho0, nu, nu_bulk, gamma_ghost, kT, zeta
        for a in range(3):
            p.body_force[a] = body_force[a]
        p.seed = seed
        self.n_sub = n_sub
        self.n_nodes = nx * ny * nz
        self.np = 0
        self._h = lib().tan_create(ct.byref(p))
        if not self._h:
            raise ValueError("bad tangent parameters")

    def close(self):
        if getattr(self, "_h", None):
            lib().tan_destroy(self._h)
            self._h = None

    def __del__(self):
        self.close()

    def set_particles(self, pos, vel, dpos=None, dzeta=0.0):
        pos = _f64(pos).reshape(-1)
        vel = _f64(vel).reshape(-1)
        self.np = pos.size // 3
        d = None if dpos is None else _f64(dpos).reshape(-1)
        lib().tan_set_particles(self._h, self.np, _dp(pos), _dp(vel), None if d is None else _dp(d), float(dzeta))

    def md_substep(self):
        lib().tan_md_substep(self._h)

    def lb_step(self):
        lib().tan_lb_step(self._h)

    def cycle(self, k: int = 1):
        for _ in range(int(k)):
            for _ in range(self.n_sub):
                self.md_substep()
            self.lb_step()

    def drag(self):
        out = np.zeros(2)
        lib().tan_drag(self._h, _dp(out))
        return float(out[0]), float(out[1])

    def populations(self):
        v = np.empty(19 * self.n_nodes)
        d = np.empty(19 * self.n_nodes)
        lib().tan_get_populations(self._h, _dp(v), _dp(d))
        return v.reshape(19, -1), d.reshape(19, -1)

    def particles(self):
        n = max(self.np, 1)
        a, b, c, e = (np.empty(3 * n) for _ in range(4))
        lib().tan_get_particles(self._h, _dp(a), _dp(b), _dp(c), _dp(e))
        k = 3 * self.np
        return a[:k].reshape(-1, 3), b[:k].reshape(-1, 3), c[:k].reshape(-1, 3), e[:k].reshape(-1, 3)
