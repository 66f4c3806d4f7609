"""Seeded synthetic inputs shared by the tests, the benchmark and the oracle.

This module draws initial conditions only; it holds none of the method's
arithmetic (no lattice weights, no equilibria, no coupling).  Both the GPU
library and the CPU oracle receive the arrays it returns as plain inputs, so
initial-condition generation is input data, not shared compute.

The workloads follow the paper's set-up (Sec. 3): ideal or bead-spring point
particles at uniform-random positions in a periodic box, Maxwellian velocities
at temperature kT, the fluid initially at rest.  Every generator takes an
explicit integer seed and uses numpy's Philox bit generator, so the same seed
gives the same arrays on every machine.
"""
from __future__ import annotations

import numpy as np


def _rng(seed: int, stream: int) -> np.random.Generator:
    return np.random.Generator(np.random.Philox(key=int(seed) & (2**64 - 1), counter=[0, 0, 0, int(stream)]))


def uniform_positions(n: int, shape, seed: int) -> np.ndarray:
    """n positions uniform in [0, nx) x [0, ny) x [0, nz), float64 (n, 3)."""
    g = _rng(seed, 1)
    L = np.asarray(shape, dtype=np.float64)
    pos = g.random((int(n), 3)) * L
    # random() is in [0, 1); the product can still round up to L.
    return np.where(pos >= L, 0.0, pos)


def maxwell_velocities(n: int, kT: float, seed: int, mass=1.0) -> np.ndarray:
    """Gaussian velocities with variance kT / m per component, float64 (n, 3)."""
    g = _rng(seed, 2)
    m = np.broadcast_to(np.asarray(mass, dtype=np.float64), (int(n),))
    return g.standard_normal((int(n), 3)) * np.sqrt(float(kT) / m)[:, None]


def bead_spring_chains(n_chains: int, n_beads: int, shape, seed: int, step: float = 1.0):
    """Random-walk chains: the first bead uniform in the box, each next bead at
    distance ``step`` in a uniformly random direction (positions wrapped into
    the box).  Returns (pos (n_chains*n_beads, 3), bonds (n_chains*(n_beads-1), 2))."""
    g = _rng(seed, 3)
    L = np.asarray(shape, dtype=np.float64)
    pos = np.zeros((n_chains, n_beads, 3))
    pos[:, 0, :] = g.random((n_chains, 3)) * L
    d = g.standard_normal((n_chains, max(n_beads - 1, 0), 3))
    d /= np.linalg.norm(d, axis=2, keepdims=True)
    if n_beads > 1:
        pos[:, 1:, :] = pos[:, :1, :] + np.cumsum(step * d, axis=1)
    pos = np.mod(pos, L)
    pos = np.where(pos >= L, 0.0, pos).reshape(-1, 3)
    first = (np.arange(n_chains)[:, None] * n_beads + np.arange(n_beads - 1)[None, :]).reshape(-1)
    bonds = np.stack([first, first + 1], axis=1).astype(np.int64)
    return pos, bonds


def self_avoiding_chains(n_chains: int, n_beads: int, shape, seed: int, bond: float = 0.97, d_min: float = 0.9,
                         tries: int = 64):
    """Bead-spring chains with no two beads closer than ``d_min`` (minimum
    image): each chain starts at a uniform point, each next bead at distance
    ``bond`` from the previous one in a uniformly random direction, a trial
    that comes closer than ``d_min`` to any placed bead is redrawn (a chain
    that gets stuck is started again).  A stand-in for a relaxed
    Kremer-Grest melt: no overlaps, so Lennard-Jones forces start finite.
    Returns (pos (n_chains*n_beads, 3), bonds (n_chains*(n_beads-1), 2))."""
    g = _rng(seed, 6)
    L = np.asarray(shape, dtype=np.float64)
    nc = np.maximum((L // d_min).astype(int), 1)  # hash cells of edge >= d_min
    csz = L / nc
    grid = {}

    def key(x):
        return tuple(int(v) % int(c) for v, c in zip(np.floor(x / csz), nc))

    def free(x):
        k = key(x)
        for dx in (-1, 0, 1):
            for dy in (-1, 0, 1):
                for dz in (-1, 0, 1):
                    for y in grid.get(((k[0] + dx) % nc[0], (k[1] + dy) % nc[1], (k[2] + dz) % nc[2]), ()):
                        d = y - x
                        d -= L * np.round(d / L)
                        if float(d @ d) < d_min * d_min:
                            return False
        return True

    out = np.zeros((n_chains, n_beads, 3))
    for c in range(n_chains):
        for _attempt in range(1000):
            placed = []
            x = g.random(3) * L
            ok = free(x)
            while ok and len(placed) < n_beads:
                placed.append(x)
                grid.setdefault(key(x), []).append(x)
                if len(placed) == n_beads:
                    break
                ok = False
                for _ in range(tries):
                    d = g.standard_normal(3)
                    y = np.mod(placed[-1] + bond * d / np.linalg.norm(d), L)
                    y = np.where(y >= L, 0.0, y)
                    if free(y):
                        x, ok = y, True
                        break
            if len(placed) == n_beads:
                out[c] = np.asarray(placed)
                break
            for x in placed:  # stuck: take the chain out and start again
                lst = grid[key(x)]
                for i, y in enumerate(lst):
                    if y is x:
                        del lst[i]
                        break
        else:
            raise RuntimeError("self_avoiding_chains: could not place chain %d" % c)
    first = (np.arange(n_chains)[:, None] * n_beads + np.arange(n_beads - 1)[None, :]).reshape(-1)
    bonds = np.stack([first, first + 1], axis=1).astype(np.int64)
    return out.reshape(-1, 3), bonds


def perturbed(base: np.ndarray, amplitude: float, seed: int) -> np.ndarray:
    """base * (1 + amplitude * U(-1, 1)), elementwise: a random state near a
    caller-given reference state (e.g. populations of a fluid at rest)."""
    g = _rng(seed, 4)
    base = np.asarray(base, dtype=np.float64)
    return base * (1.0 + float(amplitude) * (2.0 * g.random(base.shape) - 1.0))


def uniform(shape, lo: float, hi: float, seed: int, stream: int = 5) -> np.ndarray:
    """Plain uniform numbers in [lo, hi) (e.g. small momentum transfers)."""
    g = _rng(seed, stream)
    return lo + (hi - lo) * g.random(shape)


def replica_configs(n_replicas: int, seed: int, edges=(12, 16, 24, 32), max_particles: int = 400,
                    zeta_range=(0.5, 5.0), n_subs=(1, 5, 10)):
    """Parameters of a batch of independent replica boxes: cubic edge drawn
    uniformly from ``edges``, particle count uniform in [1, max_particles],
    friction uniform in ``zeta_range``, MD steps per LB step drawn from
    ``n_subs``; variants alternate A, B.  Returns a dict of per-replica arrays."""
    g = _rng(seed, 11)
    edge = np.asarray(edges)[g.integers(0, len(edges), n_replicas)]
    return {
        "dims": np.stack([edge, edge, edge], axis=1).astype(np.int32),
        "n_particles": g.integers(1, max_particles + 1, n_replicas).astype(np.int32),
        "zeta": g.uniform(zeta_range[0], zeta_range[1], n_replicas),
        "n_sub": np.asarray(n_subs)[g.integers(0, len(n_subs), n_replicas)].astype(np.int32),
        "variant": ["A" if r % 2 == 0 else "B" for r in range(n_replicas)],
    }
