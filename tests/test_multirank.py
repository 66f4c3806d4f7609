"""Host logic of the multi-GPU benchmark path on CPU: two gloo ranks, each an
independent replica, the job time is the slowest rank's, the rate counts the
units of every rank (replicas only: the workload does not shard, so there is
no data-path collective)."""
import os
import socket

import pytest


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank_main(rank, world, port, out):
    import sys
    sys.path.insert(0, os.path.dirname(os.path.dirname(os.path.abspath(__file__))))
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank), WORLD_SIZE=str(world))
    import torch.distributed as dist
    import bench
    dist.init_process_group("gloo", rank=rank, world_size=world)
    ms = 10.0 * (rank + 1)  # rank 1 is the slow one
    slowest = bench.max_over_ranks(ms, world)
    rate = bench.whole_job_rate(1000.0, world, slowest * 1e-3)
    out.put((rank, slowest, rate))
    dist.barrier()
    dist.destroy_process_group()


def test_two_gloo_ranks_max_time_and_whole_job_rate():
    torch = pytest.importorskip("torch")
    import torch.multiprocessing as mp
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_rank_main, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    res = sorted(q.get(timeout=120) for _ in procs)
    for p in procs:
        p.join(timeout=120)
        assert p.exitcode == 0
    for rank, slowest, rate in res:
        assert slowest == 20.0
        assert abs(rate - 2 * 1000.0 / 0.02) < 1e-6


def test_single_rank_is_identity():
    import bench
    assert bench.max_over_ranks(3.5, 1) == 3.5
    assert bench.whole_job_rate(10.0, 1, 2.0) == 5.0


def _replica_rank_main(rank, world, port, out):
    # one replica per rank, as the benchmark runs them (seed = base + rank),
    # computed here by the oracle in place of the GPU library; the only
    # collective is the timing reduction (and, for this test, a fingerprint
    # exchange)
    import sys
    import time
    sys.path.insert(0, os.path.dirname(os.path.dirname(os.path.abspath(__file__))))
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank), WORLD_SIZE=str(world))
    import numpy as np
    import torch
    import torch.distributed as dist
    import bench
    from oracle import oracle as orc
    from paper_1610_02733_gb300 import inputs
    dist.init_process_group("gloo", rank=rank, world_size=world)
    seed = bench.SEED + rank
    shape, n, cycles = (12, 10, 8), 40, 2
    o = orc.Oracle(*shape, n_sub=bench.N_SUB, variant=1, kT=bench.KT, zeta=bench.ZETA, seed=seed)
    o.add_particles(inputs.uniform_positions(n, shape, seed), inputs.maxwell_velocities(n, bench.KT, seed))
    t0 = time.perf_counter()
    o.cycle(cycles)
    ms = (time.perf_counter() - t0) * 1e3
    slowest = bench.max_over_ranks(ms, world)
    rate = bench.whole_job_rate(float(np.prod(shape) * cycles), world, slowest * 1e-3)
    fp = torch.tensor([o.populations().sum(), float(np.abs(o.particles()[1]).sum())], dtype=torch.float64)
    allfp = [torch.zeros(2, dtype=torch.float64) for _ in range(world)]
    dist.all_gather(allfp, fp)
    all_ms = [torch.zeros(1, dtype=torch.float64) for _ in range(world)]
    dist.all_gather(all_ms, torch.tensor([ms], dtype=torch.float64))
    out.put((rank, slowest, rate, [x.tolist() for x in allfp], [float(x) for x in all_ms]))
    o.close()
    dist.barrier()
    dist.destroy_process_group()


def test_two_gloo_ranks_run_independent_replicas():
    pytest.importorskip("torch")
    import torch.multiprocessing as mp
    from oracle import oracle as orc
    orc.build()
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_replica_rank_main, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    res = sorted(q.get(timeout=300) for _ in procs)
    for p in procs:
        p.join(timeout=300)
        assert p.exitcode == 0
    (_, s0, r0, fp, ms), (_, s1, r1, _, _) = res
    # every rank reports the slowest rank's time and the units of both
    assert s0 == s1 == max(ms)
    assert abs(r0 - 2 * 12 * 10 * 8 * 2 / (max(ms) * 1e-3)) < 1e-6 * r0 and r0 == r1
    # independent replicas: the same mass, different particle states
    assert abs(fp[0][0] - fp[1][0]) < 1e-9 * fp[0][0]
    assert fp[0][1] != fp[1][1]


def test_reference_arm_under_torchrun():
    # the launch the driver uses for N > 1, on the CPU: rank 0 alone runs the
    # oracle and prints one JSON line, the other rank exits 0 without work
    import json
    import subprocess
    import sys
    pytest.importorskip("torch")
    root = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
    cmd = [sys.executable, "-m", "torch.distributed.run", "--nnodes=1", "--nproc-per-node", "2", "--master-addr",
           "127.0.0.1", "--master-port", str(_free_port()), "bench.py", "--impl", "reference", "--gpus", "2",
           "--steps", "1", "--warmup", "0"]
    r = subprocess.run(cmd, cwd=root, capture_output=True, text=True, timeout=600)
    assert r.returncode == 0, r.stderr[-2000:]
    lines = [ln for ln in r.stdout.splitlines() if ln.startswith("{")]
    assert len(lines) == 1, r.stdout
    d = json.loads(lines[0])
    assert d["impl"] == "reference" and d["value"] > 0 and d["cpu_baseline"]["kind"] == "oracle"
    assert d["e2e"]["h2d_bytes_per_step"] == 0
