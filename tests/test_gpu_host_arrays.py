"""Particle upload and download through page-locked host arrays (pinned torch
tensors: asynchronous copies) give bit for bit what pageable numpy arrays
give, including into caller-owned output arrays."""
import numpy as np
import pytest

from paper_1610_02733_gb300 import inputs, lbmd

pytestmark = pytest.mark.gpu

SHAPE = (16, 12, 10)


@pytest.mark.parametrize("precision", ["fp32", "fp64"])
def test_pinned_and_pageable_host_arrays_agree(precision):
    torch = pytest.importorskip("torch")
    n = 200
    pos, vel = inputs.uniform_positions(n, SHAPE, 61), inputs.maxwell_velocities(n, 1e-4, 61)
    sims = [lbmd.LBMD(*SHAPE, variant="B", precision=precision, n_sub=5, kT=1e-4, zeta=1.0, seed=61, max_particles=n)
            for _ in range(2)]
    for s in sims:
        s.add_particles(pos, vel)
        s.cycle(1)
    new_pos = np.ascontiguousarray(inputs.uniform_positions(n, SHAPE, 62).reshape(-1))
    new_vel = np.ascontiguousarray(inputs.maxwell_velocities(n, 1e-4, 62).reshape(-1))
    sims[0].set_particles(new_pos, new_vel)
    sims[1].set_particles(torch.from_numpy(new_pos.copy()).pin_memory(), torch.from_numpy(new_vel.copy()).pin_memory())
    for s in sims:
        s.cycle(1)
    p0, v0 = sims[0].particles()
    out = (torch.empty(3 * n, dtype=torch.float64).pin_memory(), torch.empty(3 * n, dtype=torch.float64).pin_memory())
    sims[1].particles(out=out)
    assert np.array_equal(out[0].numpy().reshape(n, 3), p0)
    assert np.array_equal(out[1].numpy().reshape(n, 3), v0)
    # the same context read both ways
    sims[0].particles(out=out)
    assert np.array_equal(out[0].numpy().reshape(n, 3), p0)
    assert np.array_equal(out[1].numpy().reshape(n, 3), v0)
