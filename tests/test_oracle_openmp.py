"""The oracle's OpenMP timing build (used only for the all-cores CPU baseline)
gives bit for bit the results of the plain single-thread build that checks
the GPU path: its threads only split the LB node loops, where every node is
collided, streamed and summed on its own."""
import numpy as np
import pytest

from paper_1610_02733_gb300 import inputs


def test_openmp_build_equals_the_plain_oracle(orc):
    try:
        orc.build_openmp()
    except Exception as exc:  # pragma: no cover - hosts without an OpenMP runtime
        pytest.skip("no OpenMP build: %s" % exc)
    shape, n = (12, 10, 8), 40
    pos, vel = inputs.uniform_positions(n, shape, 3), inputs.maxwell_velocities(n, 1e-3, 3)
    runs = []
    for openmp in (False, True):
        o = orc.Oracle(*shape, n_sub=3, variant=1, kT=1e-3, zeta=1.5, seed=4, openmp=openmp)
        o.add_particles(pos, vel)
        o.cycle(3)
        runs.append((o.populations(), *o.particles(), o.node_field()))
        o.close()
    for a, b in zip(*runs):
        np.testing.assert_array_equal(a, b)
