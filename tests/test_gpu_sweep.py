"""The paper's temperature findings (Sec. 3, Sec. 4) on the Kremer-Grest
system at its own size (10 chains x 256 beads in (20 sigma)^3, k_B T = epsilon,
eta = 3 epsilon tau / sigma^3), with the HALF_STEP integrator, in short runs
(10 tau of equilibration, 30 tau of measurement; block standard errors about
0.3 %):

* variant A heats up at large friction and time-scale contrast (m = 10,
  dt = 0.01 tau, zeta = 20 mu/tau);
* variant B stays within 2 % there;
* A heats up alike at the same LB time step (m = 5, dt = 0.010 tau versus
  m = 10, dt = 0.005 tau);
* variant C is indistinguishable from B."""
import pytest

from paper_1610_02733_gb300 import sweep

pytestmark = pytest.mark.gpu

KW = dict(equil_tau=10.0, measure_tau=30.0, integrator="half_step")


def test_a_heats_up_b_does_not():
    a = sweep.measure_temperature("A", 10, 0.01, 20.0, **KW)
    b = sweep.measure_temperature("B", 10, 0.01, 20.0, **KW)
    assert a["T"] - 1.0 > 0.12, a
    assert abs(b["T"] - 1.0) < 0.02, b


def test_a_heat_up_depends_on_the_lb_time_step():
    a1 = sweep.measure_temperature("A", 5, 0.010, 20.0, **KW)
    a2 = sweep.measure_temperature("A", 10, 0.005, 20.0, **KW)
    assert a1["T"] - 1.0 > 0.08 and a2["T"] - 1.0 > 0.08
    assert abs(a1["T"] - a2["T"]) < 0.015, (a1, a2)


def test_c_matches_b():
    b = sweep.measure_temperature("B", 10, 0.005, 20.0, **KW)
    c = sweep.measure_temperature("C", 10, 0.005, 20.0, **KW)
    assert abs(c["T"] - b["T"]) < 0.01, (b, c)
