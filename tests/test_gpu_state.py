"""Checkpoint / resume (lbmd_save_state, lbmd_load_state): a run of 2k cycles
equals a run of k cycles, saved, restored into a fresh context and continued
for k cycles -- bit for bit (populations, positions, velocities, counters),
for the three variants, both integrators, FP32, FP64 and FP16 storage, ideal
particles with several masses and Kremer-Grest chains (LJ + FENE)."""
import numpy as np
import pytest

from paper_1610_02733_gb300 import inputs, lbmd, lj_units

pytestmark = pytest.mark.gpu

SHAPE = (16, 12, 10)


def _make(variant, precision, integrator, kg, n_sub=5):
    if kg:
        lp = lj_units.lattice_params(n_sub, 0.005, 5.0)
        pos, bonds = inputs.self_avoiding_chains(3, 24, SHAPE, 51)
        kw = dict(kT=lp["kT"], zeta=lp["zeta"], nu=lp["nu"], max_bonds=bonds.shape[0])
    else:
        lp, bonds = None, None
        pos = inputs.uniform_positions(150, SHAPE, 51)
        kw = dict(kT=1e-4, zeta=1.5)
    n = pos.shape[0]
    g = lbmd.LBMD(*SHAPE, variant=variant, precision=precision, n_sub=n_sub, seed=51, max_particles=n,
                  integrator=integrator, **kw)

    def populate(ctx):
        mass = None if kg else 1.0 + (np.arange(n) % 3)
        ctx.add_particles(pos, inputs.maxwell_velocities(n, kw["kT"], 51, 1.0 if mass is None else mass), mass)
        if kg:
            ctx.set_lj(lp["lj_eps"], lp["lj_sigma"], lp["lj_rc"])
            ctx.add_fene_bonds(bonds, lp["fene_k"], lp["fene_R0"])

    def fresh():
        return lbmd.LBMD(*SHAPE, variant=variant, precision=precision, n_sub=n_sub, seed=51, max_particles=n,
                         integrator=integrator, **kw)
    populate(g)
    return g, populate, fresh


def _state(g):
    return (g.populations(), *g.particles())


@pytest.mark.parametrize("variant", ["A", "B", "C"])
@pytest.mark.parametrize("integrator", ["start", "half_step"])
@pytest.mark.parametrize("kg", [False, True])
def test_resume_is_bitwise(variant, integrator, kg):
    k = 3
    ref, populate, fresh = _make(variant, "fp32", integrator, kg)
    ref.run_cycles(2 * k)
    want = _state(ref)
    first, _, _ = _make(variant, "fp32", integrator, kg)
    first.run_cycles(k)
    blob = first.save_state()
    second = fresh()
    second.load_state(blob)
    c = second.counts()
    assert c["lb_step"] == k and c["md_step"] == k * second.n_sub
    second.run_cycles(k)
    for a, b in zip(_state(second), want):
        np.testing.assert_array_equal(a, b)


@pytest.mark.parametrize("precision", ["fp64", "fp16dev"])
def test_resume_other_storage(precision):
    k = 2
    ref, _, fresh = _make("B", precision, "half_step", True)
    ref.run_cycles(2 * k)
    first, _, _ = _make("B", precision, "half_step", True)
    first.run_cycles(k)
    second = fresh()
    second.load_state(first.save_state())
    for _ in range(k):
        second.cycle(1)  # eager calls after the restore
    for a, b in zip(_state(second), _state(ref)):
        np.testing.assert_array_equal(a, b)


def test_state_errors():
    g, _, fresh = _make("B", "fp32", "start", False)
    g.md_substep()
    with pytest.raises(lbmd.LbmdError) as ei:
        g.save_state()
    assert ei.value.status == lbmd.LBMD_ERR_SEQUENCE
    for _ in range(g.n_sub - 1):
        g.md_substep()
    g.lb_step()
    blob = g.save_state()
    other = lbmd.LBMD(*SHAPE, variant="B", precision="fp32", n_sub=5, seed=52, max_particles=200)
    with pytest.raises(lbmd.LbmdError) as ei:
        other.load_state(blob)  # another seed
    assert ei.value.status == lbmd.LBMD_ERR_ARG
    small = lbmd.LBMD(*SHAPE, variant="B", precision="fp32", n_sub=5, seed=51, kT=1e-4, zeta=1.5, max_particles=10)
    with pytest.raises(lbmd.LbmdError) as ei:
        small.load_state(blob)
    assert ei.value.status == lbmd.LBMD_ERR_CAPACITY
    with pytest.raises(lbmd.LbmdError) as ei:
        fresh().load_state(blob[:100])
    assert ei.value.status == lbmd.LBMD_ERR_ARG
