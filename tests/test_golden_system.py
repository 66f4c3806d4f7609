"""The Kremer-Grest system the library sets up (LJ-unit conversion, the
temperature sweep's defaults) against the values the paper prints for its
test system (Sec. 4), kept as a text fixture in tests/golden/."""
import inspect
import os
from fractions import Fraction

import numpy as np

from paper_1610_02733_gb300 import lj_units, sweep

GOLDEN = os.path.join(os.path.dirname(__file__), "golden", "kremer_grest_system.txt")


def _fixture():
    out = {}
    with open(GOLDEN) as fh:
        for line in fh:
            line = line.split("#", 1)[0].strip()
            if line:
                key, value = (s.strip() for s in line.split("=", 1))
                out[key] = [s.strip() for s in value.split(",")]
    return out


def test_fixture_is_self_consistent():
    g = _fixture()
    beads = int(g["n_chains"][0]) * int(g["beads_per_chain"][0])
    assert beads == int(g["processors"][0]) * int(g["particles_per_processor"][0])  # 2560 = 8 x 320


def test_lj_cutoff_and_units_follow_the_paper():
    g = _fixture()
    assert lj_units.R_CUT_KG == 2.0 ** float(Fraction(g["lj_cutoff_log2_sigma"][0]))
    defaults = inspect.signature(lj_units.lattice_params).parameters
    assert defaults["kT"].default == float(g["kT_epsilon"][0])
    assert defaults["eta"].default == float(g["shear_viscosity"][0])
    assert defaults["rho"].default == float(g["fluid_density"][0])
    # a = sigma and tau_LB = m dt tau: the kinematic viscosity eta / rho in
    # lattice units is (eta / rho) m dt, the temperature kT (m dt)^2
    for dt in (float(x) for x in g["md_time_steps_tau"]):
        p = lj_units.lattice_params(10, dt, 5.0)
        t = 10 * dt
        assert np.isclose(p["nu"], float(g["shear_viscosity"][0]) / float(g["fluid_density"][0]) * t, rtol=1e-15)
        assert np.isclose(p["kT"], float(g["kT_epsilon"][0]) * t * t, rtol=1e-15)
        assert p["rho0"] == float(g["fluid_density"][0])
        assert p["lj_sigma"] == float(g["lattice_spacing_sigma"][0])


def test_sweep_builds_the_papers_system():
    g = _fixture()
    params = inspect.signature(sweep.build_system).parameters
    assert params["n_chains"].default == int(g["n_chains"][0])
    assert params["n_beads"].default == int(g["beads_per_chain"][0])
    assert params["box"].default == int(g["box_sigma"][0])
    assert tuple(sweep.PAPER_DTS) == tuple(float(x) for x in g["md_time_steps_tau"])
    assert tuple(sweep.PAPER_MS) == tuple(int(x) for x in g["time_scale_contrasts_m"])
    pos, bonds = sweep._chains(int(g["n_chains"][0]), int(g["beads_per_chain"][0]), int(g["box_sigma"][0]), 1)
    assert pos.shape == (2560, 3) and bonds.shape == (10 * 255, 2)
    assert float(pos.min()) >= 0.0 and float(pos.max()) < float(g["box_sigma"][0])
