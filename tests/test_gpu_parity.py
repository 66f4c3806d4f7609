"""GPU parity: the CUDA path through the C ABI against the FP64 oracle, on
the same seeded inputs, element by element.

Tolerances: populations 1e-5 in FP32 and 1e-12 in FP64 after
one LB step, relative to each population's scale w_i rho0; particle and node vectors 1e-5 / 1e-12
relative to their largest magnitude.  Integer-valued results (A and B at
m = 1, repeated runs, graph replay) must match bit for bit.
"""
import numpy as np
import pytest

from gpu_common import TOL, W, assert_pops_close, assert_pops_close_per_value, assert_vec_close, pair, random_state
from paper_1610_02733_gb300 import inputs, lbmd

pytestmark = pytest.mark.gpu

# lattice shapes: tiny, ragged (not a multiple of the 256-thread block, odd
# sides), and one that spans many blocks
SHAPES = [(4, 4, 4), (10, 6, 14), (9, 7, 5), (32, 32, 32)]


def _periodic_diff(a, b, shape):
    d = a - b
    L = np.array(shape, dtype=float)
    return d - L * np.round(d / L)


@pytest.mark.parametrize("precision", ["fp32", "fp64"])
@pytest.mark.parametrize("shape", SHAPES)
@pytest.mark.parametrize("kT", [0.0, 1e-4, 1e-3])
def test_one_lb_step(precision, shape, kT):
    kw = dict(precision=precision, kT=kT, nu=0.11, nu_bulk=0.3, gamma_ghost=0.2, body_force=(1e-5, -2e-5, 3e-5),
              seed=1234)
    o, g = pair(shape, **kw)
    f0 = random_state(o, 7)
    o.set_populations(f0)
    g.set_populations(f0)
    for obj in (o, g):
        obj.md_substep()
        obj.lb_step()
    fg, fo = g.populations(), o.populations()
    assert_pops_close(fg, fo, precision)
    if kT <= 1e-4:  # no population near zero: the per-value check as stated
        assert_pops_close_per_value(fg, fo, precision)
    nf_g, nf_o = g.node_field(), o.node_field()
    assert_vec_close(nf_g[:, 0], nf_o[:, 0], precision, "rho")
    assert_vec_close(nf_g[:, 1:], nf_o[:, 1:], precision, "j")


@pytest.mark.parametrize("precision", ["fp32", "fp64"])
@pytest.mark.parametrize("variant", ["A", "B", "C"])
@pytest.mark.parametrize("shape", [(8, 8, 8), (10, 6, 14)])
def test_md_substeps_then_lb_step(precision, variant, shape):
    n_sub, n = 4, 40
    o, g = pair(shape, precision=precision, variant=variant, n_sub=n_sub, kT=1e-3, zeta=1.5, seed=77,
                max_particles=n)
    f0 = random_state(o, 3, amplitude=0.02)
    o.set_populations(f0)
    g.set_populations(f0)
    pos = inputs.uniform_positions(n, shape, 5)
    # edge cases: exactly on a node, on the upper box face, just below it,
    # negative (wrapped), far outside (wrapped)
    pos[0] = [2.0, 3.0, 1.0]
    pos[1] = [shape[0] - 1e-9, 0.5, shape[2] - 1e-12]
    pos[2] = [0.0, 0.0, 0.0]
    pos[3] = [-0.25, -3.5, 1.5]
    pos[4] = [3 * shape[0] + 0.5, 0.25, -2 * shape[2] + 0.75]
    vel = inputs.maxwell_velocities(n, 1e-3, 5)
    mass = 1.0 + inputs.uniform(n, 0.0, 2.0, 5)
    o.add_particles(pos, vel, mass)
    g.add_particles(pos, vel, mass)
    for s in range(n_sub):
        o.md_substep()
        g.md_substep()
        po, vo = o.particles()
        pg, vg = g.particles()
        assert_vec_close(vg, vo, precision, "velocity after MD step %d" % s)
        d = _periodic_diff(pg, po, shape)
        assert np.abs(d).max() <= {"fp32": 2e-5, "fp64": 1e-12}[precision], np.abs(d).max()
        assert_vec_close(g.node_field()[:, 1:], o.node_field()[:, 1:], precision, "node j after MD step %d" % s)
        assert_vec_close(g.transfer(), o.jacc(), precision, "transfer after MD step %d" % s)
    o.lb_step()
    g.lb_step()
    assert_pops_close(g.populations(), o.populations(), precision)
    ob_o, ob_g = o.observables(), g.observables()
    assert abs(ob_g["mass"] / ob_o["mass"] - 1) < {"fp32": 1e-6, "fp64": 1e-13}[precision]
    assert_vec_close(ob_g["p_particles"], ob_o["p_particles"], precision, "particle momentum")
    assert abs(ob_g["kT_particles"] / ob_o["kT_particles"] - 1) < {"fp32": 1e-5, "fp64": 1e-12}[precision]
    assert ob_g["lb_step"] == 1 and ob_g["md_step"] == n_sub


@pytest.mark.parametrize("precision", ["fp32", "fp64"])
def test_bonded_chains_several_cycles(precision):
    shape = (16, 16, 16)
    pos, bonds = inputs.bead_spring_chains(4, 16, shape, 11)
    n = pos.shape[0]
    o, g = pair(shape, precision=precision, variant="B", n_sub=10, kT=1e-4, zeta=2.0, seed=3, max_particles=n,
                max_bonds=bonds.shape[0])
    vel = inputs.maxwell_velocities(n, 1e-4, 11)
    for obj in (o, g):
        obj.add_particles(pos, vel)
        obj.add_bonds(bonds, 30.0, 1.0)
    for c in range(3):
        o.cycle(1)
        g.cycle(1)
    po, vo = o.particles()
    pg, vg = g.particles()
    # three cycles of a chaotic system: FP32 rounding has grown, still far
    # below the motion of the beads
    tol = {"fp32": 1e-3, "fp64": 1e-9}[precision]
    assert np.abs(_periodic_diff(pg, po, shape)).max() < tol
    assert np.abs(vg - vo).max() < tol * np.abs(vo).max()
    from gpu_common import W
    err = np.abs(g.populations() - o.populations()) / W[:, None]
    assert err.max() < {"fp32": 1e-5, "fp64": 1e-11}[precision]


@pytest.mark.parametrize("precision", ["fp32", "fp64"])
def test_variants_a_and_b_coincide_bitwise_at_m_equal_one(precision):
    # variant A both with the node field and with the frozen copy of the
    # compact records as the source of its frozen node velocities
    shape, n = (12, 10, 8), 50
    runs = {}
    for variant, copy in (("A", False), ("A", True), ("B", False)):
        o, g = pair(shape, precision=precision, variant=variant, n_sub=1, kT=1e-3, zeta=1.5, seed=9,
                    max_particles=n)
        g.set_frozen_copy(copy)
        g.add_particles(inputs.uniform_positions(n, shape, 2), inputs.maxwell_velocities(n, 1e-3, 2))
        g.cycle(5)
        runs[variant, copy] = (g.populations(), *g.particles())
    for key in (("A", False), ("A", True)):
        for a, b in zip(runs[key], runs["B", False]):
            np.testing.assert_array_equal(a, b)


def test_repeat_runs_and_graph_replay_are_bitwise_identical():
    shape, n = (16, 12, 10), 100
    out = []
    for mode in ("eager", "eager", "graph"):
        o, g = pair(shape, precision="fp32", variant="B", n_sub=5, kT=1e-3, zeta=1.0, seed=21, max_particles=n)
        g.add_particles(inputs.uniform_positions(n, shape, 4), inputs.maxwell_velocities(n, 1e-3, 4))
        if mode == "eager":
            g.cycle(7)
        else:
            g.run_cycles(3)
            g.run_cycles(4)
        out.append((g.populations(), *g.particles(), g.node_field()))
        assert g.counts()["lb_step"] == 7 and g.counts()["md_step"] == 35
    for a, b in zip(out[0], out[1]):
        np.testing.assert_array_equal(a, b)
    for a, b in zip(out[0], out[2]):
        np.testing.assert_array_equal(a, b)


@pytest.mark.parametrize("variant", ["A", "B", "C"])
def test_momentum_conservation_every_md_step_fp64(variant):
    shape, n = (8, 8, 8), 30
    o, g = pair(shape, precision="fp64", variant=variant, n_sub=5, kT=1e-3, zeta=2.0, seed=5, max_particles=n)
    g.add_particles(inputs.uniform_positions(n, shape, 6), inputs.maxwell_velocities(n, 1e-3, 6))
    ob0 = g.observables()
    p0 = ob0["p_fluid"] + ob0["p_particles"]
    for c in range(3):
        for s in range(5):
            g.md_substep()
            ob = g.observables()
            np.testing.assert_allclose(ob["p_fluid"] + ob["p_particles"], p0, rtol=0, atol=1e-13)
            assert abs(ob["mass"] / ob0["mass"] - 1) < 1e-14
        g.lb_step()


def test_no_particles_and_sequence_errors():
    from paper_1610_02733_gb300 import lbmd
    o, g = pair((6, 6, 6), precision="fp32", n_sub=2)
    with pytest.raises(lbmd.LbmdError) as ei:
        g.lb_step()
    assert ei.value.status == lbmd.LBMD_ERR_SEQUENCE
    g.md_substep()
    g.md_substep()
    with pytest.raises(lbmd.LbmdError):
        g.md_substep()
    g.lb_step()
    ob = g.observables()
    assert ob["kT_particles"] == 0.0 and ob["lb_step"] == 1
    with pytest.raises(lbmd.LbmdError) as ei:
        g.add_particles(np.zeros((1, 3)), np.zeros((1, 3)))
    assert ei.value.status == lbmd.LBMD_ERR_CAPACITY


def test_invalid_parameters_are_rejected():
    from paper_1610_02733_gb300 import lbmd
    for bad in (dict(n_sub=0), dict(nu=-1.0), dict(kT=-1.0), dict(gamma_ghost=1.5)):
        with pytest.raises(lbmd.LbmdError) as ei:
            lbmd.LBMD(8, 8, 8, **bad)
        assert ei.value.status == lbmd.LBMD_ERR_ARG
    with pytest.raises(lbmd.LbmdError):
        lbmd.LBMD(1, 8, 8)


def test_temperature_statistics_match_oracle():
    # FP32 GPU vs FP64 oracle on the same Philox streams over a long run:
    # the mean particle temperature agrees within 0.5 %.
    shape, n, kT = (8, 8, 8), 60, 1e-3
    o, g = pair(shape, precision="fp32", variant="B", n_sub=5, kT=kT, zeta=0.5, seed=4, max_particles=n)
    pos, vel = inputs.uniform_positions(n, shape, 4), inputs.maxwell_velocities(n, kT, 4)
    o.add_particles(pos, vel)
    g.add_particles(pos, vel)
    To, Tg = [], []
    for c in range(1500):
        o.cycle(1)
        g.run_cycles(1)
        if c >= 100:
            To.append(o.observables()["kT_particles"])
            Tg.append(g.observables()["kT_particles"])
    assert abs(np.mean(Tg) / np.mean(To) - 1.0) < 0.005


@pytest.mark.parametrize("precision", ["fp32", "fp16dev"])
def test_variant_c_several_cycles(precision):
    # variant C over several cycles, with thermal noise, in the plain and a
    # reduced-precision storage form (populations updated after every MD step)
    shape, n_sub, n = (12, 10, 8), 5, 30
    o, g = pair(shape, precision=precision, variant="C", n_sub=n_sub, kT=1e-4, zeta=1.0, seed=21, max_particles=n)
    pos, vel = inputs.uniform_positions(n, shape, 8), inputs.maxwell_velocities(n, 1e-4, 8)
    o.add_particles(pos, vel)
    g.add_particles(pos, vel)
    o.cycle(3)
    g.run_cycles(3)
    err = np.abs(g.populations() - o.populations()) / W[:, None]
    assert float(err.max()) <= {"fp32": 1e-5, "fp16dev": 2e-4}[precision]
    if precision == "fp32":
        _, vg = g.particles()
        _, vo = o.particles()
        assert_vec_close(vg, vo, "fp32", "velocities")


@pytest.mark.parametrize("integrator", ["start", "half_step"])
@pytest.mark.parametrize("precision", ["fp32", "fp64"])
@pytest.mark.parametrize("variant", ["A", "B"])
def test_variant_b_spread_paths_agree_bitwise(precision, integrator, variant):
    # the row gather (+ migrant atomics) and the all-atomic path hand over the
    # same fixed-point transfers into the compact records: bitwise equal, and
    # equal to the oracle; variant A also with its frozen node velocities
    # from a copy of the records instead of the node field (switched at a
    # cycle boundary in the middle of the run, both ways)
    shape, n = (24, 20, 18), 3000
    runs = {}
    modes = [("rows", None), ("atomic", None)]
    if variant == "A":
        modes += [("rows", (True, False)), ("atomic", (False, True))]
    for spread, copies in modes:
        o, g = pair(shape, precision=precision, variant=variant, n_sub=5, kT=1e-4, zeta=1.5, seed=41, max_particles=n,
                    integrator=integrator, spread=spread)
        pos, vel = inputs.uniform_positions(n, shape, 41), inputs.maxwell_velocities(n, 1e-4, 41)
        g.add_particles(pos, vel)
        for c in range(2):
            if copies is not None:
                g.set_frozen_copy(copies[c])
            g.cycle(1)
        runs[spread, copies] = (g.populations(), *g.particles())
    for key in runs:
        for a, b in zip(runs[key], runs["rows", None]):
            np.testing.assert_array_equal(a, b)
    o.add_particles(pos, vel)
    o.cycle(2)
    assert_pops_close(runs["rows", None][0], o.populations(), precision)
    po, vo = o.particles()
    assert np.abs(_periodic_diff(runs["rows", None][1], po, shape)).max() <= TOL[precision] * max(shape)
    assert_vec_close(runs["rows", None][2], vo, precision, "velocities")


def test_unstable_friction_step_rejected():
    # zeta dt / m = 2.5 (zeta = 5, m = 2 MD steps per LB step, unit mass)
    g = lbmd.LBMD(8, 8, 8, n_sub=2, zeta=5.0, max_particles=4)
    with pytest.raises(lbmd.LbmdError) as ei:
        g.add_particles(np.ones((1, 3)), np.zeros((1, 3)))
    assert ei.value.status == lbmd.LBMD_ERR_ARG
    g.add_particles(np.ones((1, 3)), np.zeros((1, 3)), np.array([3.0]))  # heavier: 5 / 2 / 3 < 2


@pytest.mark.parametrize("precision,nx", [("fp32", 4096), ("fp64", 2048)])
def test_longest_rows(precision, nx):
    # the longest node rows the row gather accepts (its shared memory per
    # warp grows with nx; fewer warps per block then), ragged ny, nz
    shape, n = (nx, 3, 4), 3000
    o, g = pair(shape, precision=precision, variant="B", n_sub=3, kT=1e-4, zeta=1.5, seed=61, max_particles=n,
                spread="rows")
    pos, vel = inputs.uniform_positions(n, shape, 61), inputs.maxwell_velocities(n, 1e-4, 61)
    for obj in (o, g):
        obj.add_particles(pos, vel)
        obj.cycle(2)
    assert_pops_close(g.populations(), o.populations(), precision)
    po, vo = o.particles()
    pg, vg = g.particles()
    assert np.abs(_periodic_diff(pg, po, shape)).max() <= TOL[precision] * nx
    assert_vec_close(vg, vo, precision, "velocities")
    with pytest.raises(lbmd.LbmdError):
        lbmd.LBMD(nx + 1 if precision == "fp32" else nx * 2 + 1, 2, 2, precision=precision)



def test_frozen_copy_arguments():
    g = lbmd.LBMD(8, 8, 8, variant="A", n_sub=2, max_particles=4)
    with pytest.raises(lbmd.LbmdError) as e:
        lbmd._check(g._h, lbmd.load().lbmd_set_frozen_copy(g._h, 2), "lbmd_set_frozen_copy")
    assert e.value.status == lbmd.LBMD_ERR_ARG
    g.add_particles(np.ones((1, 3)), np.zeros((1, 3)))
    g.md_substep()
    with pytest.raises(lbmd.LbmdError) as e:
        g.set_frozen_copy(True)
    assert e.value.status == lbmd.LBMD_ERR_SEQUENCE
    g.md_substep()
    g.lb_step()
    g.set_frozen_copy(True)
    g.set_frozen_copy(False)
    g.close()


@pytest.mark.parametrize("variant", ["A", "B"])
def test_calls_between_the_last_md_step_and_the_lb_step(variant):
    # reading the state between the last MD step of a cycle and the LB step
    # changes nothing; replacing the particles there gives the same bits as
    # replacing them at the cycle boundary (the LB step then re-orders the
    # new particles, instead of the next cycle treating them as having left
    # their rows): the active set only decides where the fixed-point
    # transfers are summed
    shape, n, n_sub = (24, 20, 18), 3000, 3
    pos, vel = inputs.uniform_positions(n, shape, 5), inputs.maxwell_velocities(n, 1e-4, 5)
    pos2, vel2 = inputs.uniform_positions(n, shape, 6), inputs.maxwell_velocities(n, 1e-4, 6)
    runs = {}
    for mode in ("plain", "read", "set_before", "set_after"):
        g = lbmd.LBMD(*shape, variant=variant, n_sub=n_sub, kT=1e-4, zeta=1.5, seed=17, max_particles=n)
        g.add_particles(pos, vel)
        g.cycle(1)
        for _ in range(n_sub):
            g.md_substep()
        if mode == "read":
            g.particles()
            g.observables()
        if mode == "set_before":
            g.set_particles(pos2, vel2)
        g.lb_step()
        if mode == "set_after":
            g.set_particles(pos2, vel2)
        g.run_cycles(2)
        runs[mode] = (g.populations(), *g.particles())
        g.close()
    for a, b in zip(runs["read"], runs["plain"]):
        np.testing.assert_array_equal(a, b)
    for a, b in zip(runs["set_before"], runs["set_after"]):
        np.testing.assert_array_equal(a, b)
