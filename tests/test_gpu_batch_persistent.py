"""Batched replicas with the persistent schedule (lbmd_batch_set_schedule,
LBMD_BATCH_PERSISTENT): one launch per run call, each thread-block cluster
running whole replicas.

Every replica is compared with an oracle run of its own box (the same
ragged batch as tests/test_gpu_batch.py: m in {1, 2, 5, 10}, both variants,
a replica without particles, a perturbed fluid), and with the per-tick
schedule bit for bit: same states after runs split into calls that do not
align with the period, for every cluster size, and across schedule
switches in the middle of a run."""
import numpy as np
import pytest

from gpu_common import TOL, W, assert_vec_close
from oracle import oracle as orc
from paper_1610_02733_gb300 import inputs, lbmd
from test_gpu_batch import KT, REPLICAS, _build, _oracle_steps

pytestmark = pytest.mark.gpu


def _assert_same(b1, b2, n_rep):
    for i in range(n_rep):
        assert b1.counts(i) == b2.counts(i), i
        assert np.array_equal(b1.populations(i), b2.populations(i)), i
        p1, v1 = b1.particles(i)
        p2, v2 = b2.particles(i)
        assert np.array_equal(p1, p2) and np.array_equal(v1, v2), i


@pytest.mark.parametrize("precision", ["fp64", "fp32"])
def test_persistent_replicas_match_single_box_oracle(precision):
    b, oracles = _build(precision)
    b.set_schedule("persistent")
    steps = 23
    for k in (7, 1, 15):  # calls that start in the middle of replicas' LB cycles
        b.run(k)
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


@pytest.mark.parametrize("precision", ["fp32", "fp64"])
@pytest.mark.parametrize("cluster", [0, 1, 2, 4, 8, 16])
def test_persistent_equals_period_graph_bitwise(precision, cluster):
    b_ref, _ = _build(precision)
    b_ref.run(23)
    b, _ = _build(precision)
    b.set_schedule("persistent", cluster)
    b.run(10)
    b.run(13)
    _assert_same(b, b_ref, len(REPLICAS))


def test_schedule_switches_mid_run():
    b_ref, _ = _build("fp32")
    b_ref.run(27)
    b, _ = _build("fp32")
    b.run(4)  # per-tick schedule, ends inside a period
    b.set_schedule("persistent", 2)
    b.run(9)
    b.set_schedule("period_graph")
    b.run(8)
    b.set_schedule("persistent")
    b.run(6)
    _assert_same(b, b_ref, len(REPLICAS))


def test_many_particles_per_thread():
    # 1100 particles on a one-block cluster (256 threads): each thread keeps
    # its particles (i, i + 256, ...) over the whole launch
    dims = [(10, 12, 8), (6, 6, 6)]
    n = [1100, 3]

    def make():
        b = lbmd.Batch(dims, n_sub=[5, 1], variant=["B", "A"], zeta=[0.8, 1.2], seed=[41, 42], max_particles=n,
                       precision="fp64", kT=KT)
        for i in range(2):
            b.add_particles(i, inputs.uniform_positions(n[i], dims[i], 50 + i),
                            inputs.maxwell_velocities(n[i], 1e-3, 50 + i))
        return b

    b_ref = make()
    b_ref.run(12)
    b = make()
    b.set_schedule("persistent", 1)
    b.run(12)
    _assert_same(b, b_ref, 2)
    o = orc.Oracle(*dims[0], n_sub=5, variant=1, kT=KT, zeta=0.8, seed=41)
    o.add_particles(inputs.uniform_positions(n[0], dims[0], 50), inputs.maxwell_velocities(n[0], 1e-3, 50))
    _oracle_steps(o, 5, 0, 12)
    err = np.abs(b.populations(0) - o.populations()) / W[:, None]
    assert float(err.max()) <= TOL["fp64"]
    pg, vg = b.particles(0)
    po, vo = o.particles()
    assert_vec_close(vg, vo, "fp64", "velocities")


def test_persistent_unstable_replica_is_flagged_and_others_unaffected():
    dims = [(8, 8, 8), (8, 8, 8), (6, 10, 8)]
    b = lbmd.Batch(dims, n_sub=[1, 1, 2], variant=["B", "B", "A"], zeta=[5.0, 0.5, 4.5], seed=[3, 4, 5],
                   max_particles=[4, 4, 4], precision="fp64", kT=KT)
    b.set_schedule("persistent")
    o = orc.Oracle(8, 8, 8, n_sub=1, variant=1, kT=KT, zeta=0.5, seed=4)
    for i in range(3):
        pos, vel = inputs.uniform_positions(4, dims[i], 20 + i), inputs.maxwell_velocities(4, 1e-3, 20 + i)
        b.add_particles(i, pos, vel)
        if i == 1:
            o.add_particles(pos, vel)
    b.run(25)
    b.run(35)
    # zeta dt / m = 5 (B, m = 1) and 4.5 / 2 = 2.25 (A, m = 2): both diverge
    assert list(b.unstable()) == [1, 0, 1]
    _oracle_steps(o, 1, 0, 60)
    err = np.abs(b.populations(1) - o.populations()) / W[:, None]
    assert float(err.max()) <= TOL["fp64"]
    pg, vg = b.particles(1)
    po, vo = o.particles()
    assert_vec_close(pg, po, "fp64", "stable replica positions")
    assert_vec_close(vg, vo, "fp64", "stable replica velocities")


def test_persistent_tuning_and_arguments():
    b, _ = _build("fp32")
    t = b.persistent_tuning()
    assert t["cluster_blocks"] in (1, 2, 4, 8, 16)
    ms = dict(zip(t["candidates"], t["period_ms"]))
    assert ms[t["cluster_blocks"]] > 0 and all(x >= 0 for x in t["period_ms"])
    assert ms[t["cluster_blocks"]] == min(x for x in t["period_ms"] if x > 0)
    with pytest.raises(lbmd.LbmdError):
        b.set_schedule("persistent", 3)
    with pytest.raises(lbmd.LbmdError):
        lbmd._bcheck(b._h, lbmd.load().lbmd_batch_set_schedule(b._h, 2, 0), "lbmd_batch_set_schedule")


@pytest.mark.parametrize("schedule_first", ["persistent", "period_graph"])
def test_particles_added_and_populations_replaced_between_runs(schedule_first):
    # particles added after a run re-order the replicas (heaviest first) under
    # the same captured launch; populations replaced at a replica's cycle
    # boundary; both schedules give the same bits
    def run(schedule):
        b, _ = _build("fp32")
        b.set_schedule(schedule)
        b.run(10)
        dims = REPLICAS[3][0]  # the replica that had no particles
        b_pos = inputs.uniform_positions(1, dims, 77)
        b.add_particles(3, b_pos, inputs.maxwell_velocities(1, 1e-3, 77))
        b.run(10)
        f = inputs.perturbed(b.populations(2), 0.02, 78)  # replica 2: m = 10, at its cycle boundary
        b.set_populations(2, f)
        b.run(5)
        return b

    b1 = run(schedule_first)
    b2 = run("period_graph" if schedule_first == "persistent" else "persistent")
    _assert_same(b1, b2, len(REPLICAS))
