"""Batched replicas (lbmd_batch_*) against the FP64 oracle.

Every replica of a batch must evolve as a single box with its own lattice,
particles, friction, MD steps per LB step, variant and Philox key: each is
compared, element by element, with an oracle run of that box alone.  The
batch mixes shapes (including ragged, non-cubic ones), m in {1, 2, 5, 10}
(period lcm = 10), both variants, a replica without particles and a
perturbed initial fluid state, and runs two periods (graph-replayed) plus a
few eager ticks."""
import numpy as np
import pytest

from gpu_common import TOL, W, assert_vec_close
from oracle import oracle as orc
from paper_1610_02733_gb300 import inputs, lbmd

pytestmark = pytest.mark.gpu

REPLICAS = [
    # dims, m, variant, zeta, seed, particles
    ((12, 12, 12), 1, "B", 1.0, 11, 6),
    ((10, 8, 6), 5, "A", 0.5, 12, 9),
    ((16, 12, 8), 10, "B", 2.0, 13, 40),
    ((6, 6, 6), 2, "A", 1.5, 14, 0),
    ((8, 14, 10), 5, "B", 3.0, 15, 1),
]
KT = 1e-4


def _build(precision, md_steps_eager=0):
    b = lbmd.Batch([r[0] for r in REPLICAS], n_sub=[r[1] for r in REPLICAS], variant=[r[2] for r in REPLICAS],
                   zeta=[r[3] for r in REPLICAS], seed=[r[4] for r in REPLICAS],
                   max_particles=[max(r[5], 1) for r in REPLICAS], precision=precision, kT=KT)
    oracles = []
    for i, (dims, m, var, zeta, seed, n) in enumerate(REPLICAS):
        o = orc.Oracle(*dims, n_sub=m, variant={"A": 0, "B": 1}[var], kT=KT, zeta=zeta, seed=seed)
        if n:
            pos, vel = inputs.uniform_positions(n, dims, seed), inputs.maxwell_velocities(n, 1e-3, seed)
            o.add_particles(pos, vel)
            b.add_particles(i, pos, vel)
        oracles.append(o)
    # a non-trivial flow in replica 0 (both sides start from the same state)
    f0 = inputs.perturbed(oracles[0].populations(), 0.03, 99)
    oracles[0].set_populations(f0)
    b.set_populations(0, f0)
    return b, oracles


def _oracle_steps(o, m, first, steps):
    for s in range(first, first + steps):
        o.md_substep()
        if (s + 1) % m == 0:
            o.lb_step()


@pytest.mark.parametrize("precision", ["fp64", "fp32"])
def test_replicas_match_single_box_oracle(precision):
    b, oracles = _build(precision)
    steps = 23  # two graph-replayed periods of 10 ticks and 3 eager ticks
    b.run(steps)
    assert not b.unstable().any()
    for i, (dims, m, var, zeta, seed, n) in enumerate(REPLICAS):
        _oracle_steps(oracles[i], m, 0, steps)
        c = b.counts(i)
        assert c["lb_step"] == steps // m and c["md_step"] == steps
        err = np.abs(b.populations(i) - oracles[i].populations()) / W[:, None]
        assert float(err.max()) <= TOL[precision], (i, float(err.max()))
        if n:
            pg, vg = b.particles(i)
            po, vo = oracles[i].particles()
            assert_vec_close(pg, po, precision, "replica %d positions" % i)
            assert_vec_close(vg, vo, precision, "replica %d velocities" % i)


def test_graph_replay_equals_eager_ticks():
    b1, _ = _build("fp32")
    b2, _ = _build("fp32")
    b1.run(20)
    for _ in range(20):
        b2.run(1)
    for i in range(len(REPLICAS)):
        assert np.array_equal(b1.populations(i), b2.populations(i))
        p1, v1 = b1.particles(i)
        p2, v2 = b2.particles(i)
        assert np.array_equal(p1, p2) and np.array_equal(v1, v2)


def test_kinetic_sums():
    b, _ = _build("fp64")
    b.run(10)
    k = b.kinetic()
    for i, r in enumerate(REPLICAS):
        _, v = b.particles(i)
        assert k[i, 4] == r[5]
        assert abs(k[i, 0] - float((v ** 2).sum())) <= 1e-12 * max(1e-30, float((v ** 2).sum()))
        assert np.allclose(k[i, 1:4], v.sum(axis=0), rtol=1e-12, atol=1e-300)


def test_unstable_replica_is_flagged_and_others_unaffected():
    # zeta dt / m = 5 at m = 1: the explicit friction map overshoots (|1 - 5| > 1)
    dims = [(8, 8, 8), (8, 8, 8)]
    b = lbmd.Batch(dims, n_sub=[1, 1], variant=["B", "B"], zeta=[5.0, 0.5], seed=[3, 4], max_particles=[4, 4],
                   precision="fp64", kT=KT)
    o = orc.Oracle(8, 8, 8, n_sub=1, variant=1, kT=KT, zeta=0.5, seed=4)
    for i in range(2):
        pos, vel = inputs.uniform_positions(4, dims[i], 20 + i), inputs.maxwell_velocities(4, 1e-3, 20 + i)
        b.add_particles(i, pos, vel)
        if i == 1:
            o.add_particles(pos, vel)
    b.run(60)
    assert list(b.unstable()) == [1, 0]
    _oracle_steps(o, 1, 0, 60)
    err = np.abs(b.populations(1) - o.populations()) / W[:, None]
    assert float(err.max()) <= TOL["fp64"]
    pg, vg = b.particles(1)
    po, vo = o.particles()
    assert_vec_close(vg, vo, "fp64", "stable replica velocities")


def test_tuning_choice():
    b, _ = _build("fp32")
    b.run(10)
    t = b.tuning()
    assert t["nodes_per_block"] in (64, 128, 256) and t["particle_block"] in (64, 128, 256)
    assert all(x > 0 for x in t["lb_ms"]) and all(x > 0 for x in t["particle_ms"])


@pytest.mark.parametrize("precision,cap", [("fp32", 1), ("fp32", 3), ("fp64", 2)])
def test_persistent_grid_cap_is_bitwise_neutral(precision, cap):
    # one to three blocks work through every LB item of a tick (many items
    # per block: several windows of work entries, the header ring and the
    # staging buffers rotate) and give bit for bit what the full grid gives
    b_full, _ = _build(precision)
    b_cap, _ = _build(precision)
    b_cap.set_lb_grid(cap)
    b_full.run(23)
    b_cap.run(23)
    for i in range(len(REPLICAS)):
        assert b_cap.counts(i) == b_full.counts(i)
        assert np.array_equal(b_cap.populations(i), b_full.populations(i))
        p1, v1 = b_cap.particles(i)
        p2, v2 = b_full.particles(i)
        assert np.array_equal(p1, p2) and np.array_equal(v1, v2)


def test_frozen_replica_items_are_skipped_by_a_capped_grid():
    # a large replica that turns unstable ahead of a small stable one in the
    # work table: one block skips the frozen replica's items window by window
    # and the stable replica still follows its oracle
    dims = [(24, 24, 24), (8, 6, 10)]
    b = lbmd.Batch(dims, n_sub=[1, 1], variant=["B", "A"], zeta=[5.0, 0.5], seed=[5, 6], max_particles=[4, 4],
                   precision="fp64", kT=KT)
    b.set_lb_grid(1)
    o = orc.Oracle(8, 6, 10, n_sub=1, variant=0, kT=KT, zeta=0.5, seed=6)
    for i in range(2):
        pos, vel = inputs.uniform_positions(4, dims[i], 30 + i), inputs.maxwell_velocities(4, 1e-3, 30 + i)
        b.add_particles(i, pos, vel)
        if i == 1:
            o.add_particles(pos, vel)
    b.run(40)
    assert list(b.unstable()) == [1, 0]
    _oracle_steps(o, 1, 0, 40)
    err = np.abs(b.populations(1) - o.populations()) / W[:, None]
    assert float(err.max()) <= TOL["fp64"]
    pg, vg = b.particles(1)
    po, vo = o.particles()
    assert_vec_close(pg, po, "fp64", "stable replica positions")
    assert_vec_close(vg, vo, "fp64", "stable replica velocities")


def test_negative_grid_cap_is_rejected():
    b, _ = _build("fp32")
    with pytest.raises(lbmd.LbmdError):
        b.set_lb_grid(-1)


def test_kinetic_sums_fp32():
    # FP32 velocities are summed as FP32 pairs (~44 bits): against exact sums
    # of the stored values
    import math
    b, _ = _build("fp32")
    b.run(10)
    k = b.kinetic()
    for i, r in enumerate(REPLICAS):
        _, v = b.particles(i)
        assert k[i, 4] == r[5]
        e2 = math.fsum((v ** 2).ravel())
        assert abs(k[i, 0] - e2) <= 1e-12 * max(1e-30, e2)
        for d in range(3):
            assert abs(k[i, 1 + d] - math.fsum(v[:, d])) <= 1e-12 * max(1e-30, math.fsum(np.abs(v[:, d])))


@pytest.mark.parametrize("precision,schedule", [("fp32", "period_graph"), ("fp32", "persistent"),
                                                ("fp64", "period_graph")])
def test_full_batched_configuration_sampled(precision, schedule):
    # the benchmark's batch itself (512 replicas, cubic edges {12, 16, 24, 32},
    # 1-400 particles, zeta in [0.5, 5], m in {1, 5, 10}, variants A / B
    # alternating, kT = 1e-4; FP32 as benchmarked, and FP64), 12 MD steps; a stable replica of every
    # edge and every m is checked element by element against an oracle run
    # of its own box
    R, seed0 = 512, 1
    cfg = inputs.replica_configs(R, seed0)
    seeds = np.arange(R, dtype=np.uint64) + np.uint64(seed0 * 1000)
    b = lbmd.Batch(cfg["dims"], n_sub=cfg["n_sub"], variant=cfg["variant"], zeta=cfg["zeta"], seed=seeds,
                   max_particles=cfg["n_particles"], precision=precision, kT=KT)
    for r in range(R):
        n = int(cfg["n_particles"][r])
        b.add_particles(r, inputs.uniform_positions(n, cfg["dims"][r], seed0 + r),
                        inputs.maxwell_velocities(n, KT, seed0 + r))
    b.set_schedule(schedule)
    steps = 12
    b.run(steps)
    unstable = b.unstable()
    picked = {}
    for r in range(R):
        key = (int(cfg["dims"][r][0]), int(cfg["n_sub"][r]))
        # inside the stable range of the explicit friction (zeta dt / m < 1)
        if key not in picked and not unstable[r] and cfg["zeta"][r] / cfg["n_sub"][r] < 1.0:
            picked[key] = r
    assert len(picked) == 12, sorted(picked)  # 4 edges x 3 values of m
    for (edge, m), r in sorted(picked.items()):
        dims = tuple(int(d) for d in cfg["dims"][r])
        n = int(cfg["n_particles"][r])
        o = orc.Oracle(*dims, n_sub=m, variant={"A": 0, "B": 1}[cfg["variant"][r]], kT=KT,
                       zeta=float(cfg["zeta"][r]), seed=int(seeds[r]))
        o.add_particles(inputs.uniform_positions(n, dims, seed0 + r), inputs.maxwell_velocities(n, KT, seed0 + r))
        _oracle_steps(o, m, 0, steps)
        assert b.counts(r)["lb_step"] == steps // m
        err = np.abs(b.populations(r) - o.populations()) / W[:, None]
        assert float(err.max()) <= TOL[precision], (r, edge, m, float(err.max()))
        pg, vg = b.particles(r)
        po, vo = o.particles()
        assert_vec_close(pg, po, precision, "replica %d positions" % r)
        assert_vec_close(vg, vo, precision, "replica %d velocities" % r)
        o.close()
    b.close()
