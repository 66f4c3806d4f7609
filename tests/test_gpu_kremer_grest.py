"""Kremer-Grest chains (Sec. 4) on the GPU against the FP64 oracle:
Lennard-Jones between all beads (cut at 2^(7/6) sigma), FENE springs, the
paper's parameters converted from LJ units, all three coupling variants.

The forces after one MD step are compared tightly (the tolerances of the
other parity tests); after several cycles the chaotic bead motion has
amplified rounding, so positions and velocities get the looser bounds of the
harmonic-chain test while the populations keep theirs.  The paper's own
system size (10 chains of 256 beads in (20 sigma)^3) is checked at its
hardest grid point (m = 10, dt = 0.01 tau, zeta = 20 mu/tau)."""
import numpy as np
import pytest

from gpu_common import TOL, W, assert_vec_close, pair
from paper_1610_02733_gb300 import inputs, lbmd, lj_units

pytestmark = pytest.mark.gpu


def _periodic_diff(a, b, shape):
    d = a - b
    L = np.asarray(shape, dtype=float)
    return d - L * np.round(d / L)


def _kg_pair(shape, n_chains, n_beads, m, dt, zeta, *, precision, variant, seed, harmonic=0):
    lp = lj_units.lattice_params(m, dt, zeta)
    pos, bonds = inputs.self_avoiding_chains(n_chains, n_beads, shape, seed)
    n = pos.shape[0]
    o, g = pair(shape, precision=precision, variant=variant, n_sub=m, kT=lp["kT"], zeta=lp["zeta"], nu=lp["nu"],
                seed=seed, max_particles=n, max_bonds=bonds.shape[0] + harmonic)
    vel = inputs.maxwell_velocities(n, lp["kT"], seed)
    for obj in (o, g):
        obj.add_particles(pos, vel)
        obj.set_lj(lp["lj_eps"], lp["lj_sigma"], lp["lj_rc"])
        obj.add_fene_bonds(bonds, lp["fene_k"], lp["fene_R0"])
        if harmonic:
            obj.add_bonds(bonds[:harmonic], 0.5 * lp["fene_k"], 0.97)
    return o, g, lp


@pytest.mark.parametrize("precision", ["fp32", "fp64"])
@pytest.mark.parametrize("variant", ["A", "B", "C"])
def test_one_md_step_with_lj_and_fene(precision, variant):
    # dense enough for many LJ pairs, ragged box, a few harmonic bonds too
    shape = (11, 9, 8)
    o, g, _ = _kg_pair(shape, 6, 24, 5, 0.005, 5.0, precision=precision, variant=variant, seed=21, harmonic=4)
    o.md_substep()
    g.md_substep()
    po, vo = o.particles()
    pg, vg = g.particles()
    assert_vec_close(vg, vo, precision, "velocities")
    assert np.abs(_periodic_diff(pg, po, shape)).max() <= {"fp32": 1e-5, "fp64": 1e-12}[precision] * max(shape)


@pytest.mark.parametrize("precision", ["fp32", "fp64"])
def test_lj_unordered_particles(precision):
    # LJ between particles in no spatial order by id (every chunk of 32 ids
    # spans the box), more than one tile of ids: the pair kernel cannot skip
    # chunks and runs over several tiles
    shape, n = (14, 12, 11), 1400
    lp = lj_units.lattice_params(5, 0.005, 5.0)
    o, g = pair(shape, precision=precision, variant="B", n_sub=5, kT=lp["kT"], zeta=lp["zeta"], nu=lp["nu"],
                seed=25, max_particles=n)
    # well separated start (> 1.07 apart, across the periodic faces too): a
    # jittered lattice whose spacing divides the box, shuffled ids
    axes = [np.arange(L // 1.05) * (L / (L // 1.05)) for L in shape]
    grid = np.stack(np.meshgrid(*axes, indexing="ij"), -1).reshape(-1, 3)
    rng = np.random.default_rng(25)
    pos = grid[rng.permutation(grid.shape[0])[:n]] + 0.02 * rng.random((n, 3))
    vel = inputs.maxwell_velocities(n, lp["kT"], 25)
    for obj in (o, g):
        obj.add_particles(pos, vel)
        obj.set_lj(lp["lj_eps"], lp["lj_sigma"], lp["lj_rc"])
    for _ in range(2):
        o.md_substep()
        g.md_substep()
    po, vo = o.particles()
    pg, vg = g.particles()
    assert_vec_close(vg, vo, precision, "velocities")
    assert np.abs(_periodic_diff(pg, po, shape)).max() <= {"fp32": 1e-5, "fp64": 1e-12}[precision] * max(shape)


@pytest.mark.parametrize("precision", ["fp32", "fp64"])
@pytest.mark.parametrize("variant", ["A", "B", "C"])
def test_chains_several_cycles(precision, variant):
    shape = (16, 12, 10)
    o, g, _ = _kg_pair(shape, 4, 32, 5, 0.005, 5.0, precision=precision, variant=variant, seed=22)
    for _ in range(3):
        o.cycle(1)
        g.cycle(1)
    po, vo = o.particles()
    pg, vg = g.particles()
    tol = {"fp32": 1e-3, "fp64": 1e-9}[precision]
    assert np.abs(_periodic_diff(pg, po, shape)).max() < tol
    assert np.abs(vg - vo).max() < tol * np.abs(vo).max()
    err = np.abs(g.populations() - o.populations()) / W[:, None]
    assert float(err.max()) <= TOL[precision]
    ob = g.observables()
    oo = o.observables()
    # total momentum of fluid + particles: the pair forces cancel up to rounding
    assert np.allclose(ob["p_fluid"] + ob["p_particles"], oo["p_fluid"] + oo["p_particles"],
                       rtol=0, atol={"fp32": 1e-5, "fp64": 1e-12}[precision] * np.abs(vo).max() * vo.shape[0])


@pytest.mark.parametrize("precision", ["fp32", "fp64"])
def test_paper_system_size(precision):
    # 10 chains x 256 beads in (20 sigma)^3, m = 10, dt = 0.01 tau,
    # zeta = 20 mu/tau, variant B; three LB cycles
    shape = (20, 20, 20)
    o, g, _ = _kg_pair(shape, 10, 256, 10, 0.01, 20.0, precision=precision, variant="B", seed=23)
    g.run_cycles(3)
    o.cycle(3)
    po, vo = o.particles()
    pg, vg = g.particles()
    tol = {"fp32": 1e-3, "fp64": 1e-9}[precision]
    assert np.abs(_periodic_diff(pg, po, shape)).max() < tol
    assert np.abs(vg - vo).max() < tol * np.abs(vo).max()
    err = np.abs(g.populations() - o.populations()) / W[:, None]
    assert float(err.max()) <= TOL[precision]


def test_bitwise_reproducible_despite_slot_order():
    # the re-ordering's slot order inside a row depends on atomics; the LJ
    # sums run over particle ids, so repeated runs agree bit for bit
    shape = (16, 12, 10)
    runs = []
    for _ in range(2):
        _, g, _ = _kg_pair(shape, 4, 32, 5, 0.005, 5.0, precision="fp32", variant="B", seed=24)
        g.run_cycles(4)
        runs.append((g.populations(), *g.particles()))
    for a, b in zip(*runs):
        np.testing.assert_array_equal(a, b)


def test_lj_argument_checks():
    g = lbmd.LBMD(8, 8, 8, max_particles=10)
    with pytest.raises(lbmd.LbmdError) as ei:
        g.set_lj(1.0, 1.0, 3.5)  # 2 r_cut + 2 = 9 > 8
    assert ei.value.status == lbmd.LBMD_ERR_ARG
    with pytest.raises(lbmd.LbmdError):
        g.set_lj(-1.0, 1.0, 1.0)
    g.set_lj(1.0, 1.0, 2.0 ** (7.0 / 6.0))
    big = lbmd.LBMD(8, 8, 8, max_particles=200000)
    with pytest.raises(lbmd.LbmdError) as ei:
        big.set_lj(1.0, 1.0, 1.0)
    assert ei.value.status == lbmd.LBMD_ERR_CAPACITY
    g.add_particles(np.array([[1.0, 1, 1], [2.0, 1, 1]]), np.zeros((2, 3)))
    with pytest.raises(lbmd.LbmdError):
        g.add_fene_bonds(np.array([[0, 1]]), 30.0, 0.0)


@pytest.mark.parametrize("integrator", ["start", "half_step"])
def test_variant_b_spread_paths_agree_bitwise(integrator):
    # variant B with conservative forces: the row gather, and the transfers
    # handed over inside the LJ / bond kernel, give the same fixed-point sums
    shape, m = (16, 12, 10), 5
    lp = lj_units.lattice_params(m, 0.005, 5.0)
    pos, bonds = inputs.self_avoiding_chains(4, 32, shape, 26)
    n = pos.shape[0]
    vel = inputs.maxwell_velocities(n, lp["kT"], 26)
    runs = {}
    for lj in (True, False):
        for spread in ("rows", "atomic"):
            g = lbmd.LBMD(*shape, variant="B", precision="fp32", n_sub=m, kT=lp["kT"], zeta=lp["zeta"], nu=lp["nu"],
                          seed=26, max_particles=n, max_bonds=bonds.shape[0], integrator=integrator, spread=spread)
            g.add_particles(pos, vel)
            if lj:
                g.set_lj(lp["lj_eps"], lp["lj_sigma"], lp["lj_rc"])
            g.add_fene_bonds(bonds, lp["fene_k"], lp["fene_R0"])
            g.run_cycles(3)
            runs[(lj, spread)] = (g.populations(), *g.particles())
        for a, b in zip(runs[(lj, "rows")], runs[(lj, "atomic")]):
            np.testing.assert_array_equal(a, b)


@pytest.mark.parametrize("precision", ["fp32", "fp64"])
def test_verlet_lists_give_the_all_pairs_bits(precision):
    # the LJ forces from the Verlet lists (built at every re-ordering) equal
    # the all-pairs loop bit for bit: the same run with the lists voided every
    # cycle (re-setting the same LJ parameters voids them until the next
    # re-ordering) must not differ
    shape, m = (20, 20, 20), 10
    lp = lj_units.lattice_params(m, 0.01, 20.0)
    pos, bonds = inputs.self_avoiding_chains(10, 256, shape, 27)
    n = pos.shape[0]
    runs = []
    for void in (False, True):
        g = lbmd.LBMD(*shape, variant="B", precision=precision, n_sub=m, kT=lp["kT"], zeta=lp["zeta"], nu=lp["nu"],
                      seed=27, max_particles=n, max_bonds=bonds.shape[0], integrator="half_step")
        g.add_particles(pos, inputs.maxwell_velocities(n, lp["kT"], 27))
        g.set_lj(lp["lj_eps"], lp["lj_sigma"], lp["lj_rc"])
        g.add_fene_bonds(bonds, lp["fene_k"], lp["fene_R0"])
        for _ in range(6):
            if void:
                g.set_lj(lp["lj_eps"], lp["lj_sigma"], lp["lj_rc"])
            g.cycle(1)
        runs.append((g.populations(), *g.particles()))
    for a, b in zip(*runs):
        np.testing.assert_array_equal(a, b)

