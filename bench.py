"""Benchmark of the coupled LB/MD hot path on GB300.

One step = one full LB cycle of the paper's scheme (Sec. 3): m = 10 MD steps
(interpolation, friction + noise, velocity Verlet, momentum spreading) and one
LB step (MRT collision with noise and forcing, streaming, node field), variant
B, FP32 storage and arithmetic, on the workload

    256^3 periodic D3Q19, rho = 1, nu = 1/6, kT = 1e-4,
    10^6 ideal particles (mass 1, zeta = 1) at uniform-random positions with
    Maxwellian velocities, dt_MD = tau_LB / 10.

Reported: MLUPS (lattice node updates per second) as ``value`` and
particle-substeps/s beside it, the roofline of the LB step against the
measured HBM bandwidth, an end-to-end figure through the C ABI with host
buffers, and the FP64 CPU oracle timed on a bounded sample of the same
workload.  Inputs (2.5 GB of populations) are far larger than L2, so no L2
flush is needed between steps.

Usage: python bench.py [--gpus N] [--steps K] [--warmup W] [--impl reference]
Under torchrun (N > 1) every rank runs an independent replica (the workload
does not shard); rank 0 prints the aggregate.
"""
from __future__ import annotations

import argparse
import json
import os
import statistics
import subprocess
import sys
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

METRIC = "MLUPS + particle-substeps/s (variant B, n=10) and % of HBM roofline vs plain FP32"
SHAPE = (256, 256, 256)
N_PARTICLES = 1_000_000
N_SUB = 10
KT = 1e-4
ZETA = 1.0
SEED = 1
LB_BYTES_PER_NODE = 2 * 19 * 4  # algorithmic: read and write 19 FP32 populations
PARTICLE_BYTES = 48              # algorithmic per particle and MD step: R, v read and written (FP32)
NODE_TOUCH_BYTES = 32            # ... per distinct touched node: node velocity read, transfer written
# kernels per cycle (variant B, no bonds): per MD step couple + row gather +
# migrant spread; per LB step the re-ordering (count, chunk scan, finalize,
# scatter), the next active nodes (rows, chunk scan, finalize), the collide
# with fused moments and the remaining moments
LAUNCHES_PER_CYCLE = 3 * N_SUB + 4 + 3 + 2
WORKLOAD = "256^3 D3Q19 + 1e6 ideal particles, variant B, n=10, FP32"
PRECISION = "fp32"


def _peaks():
    path = os.path.join(ROOT, "MEASURED_PEAKS.json")
    try:
        with open(path) as fh:
            d = json.load(fh)
        return float(d["hbm_gbs"]), "measured"
    except Exception:
        return 6800.0, "fallback"


class ClockSampler:
    """nvidia-smi clock/throttle sampling during the timed region."""

    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, device_index: int):
        self.dev = device_index
        self.proc = None
        self.path = os.path.join("/tmp", "lbmd_clocks_%d_%d.csv" % (os.getpid(), device_index))

    def start(self):
        try:
            self.fh = open(self.path, "w")
            self.proc = subprocess.Popen(["nvidia-smi", "-i", str(self.dev), "--query-gpu=" + self.FIELDS,
                                          "--format=csv,noheader,nounits", "-lms", "100"],
                                         stdout=self.fh, stderr=subprocess.DEVNULL)
        except Exception:
            self.proc = None

    def stop(self):
        if self.proc is None:
            return None
        time.sleep(0.25)
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except Exception:
            self.proc.kill()
        self.fh.close()
        sm, smax, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for line in open(self.path):
            parts = [p.strip() for p in line.split(",")]
            if len(parts) < 9:
                continue
            try:
                sm.append(float(parts[1]))
                smax.append(float(parts[2]))
            except ValueError:
                continue
            for name, flag in zip(names, parts[5:9]):
                if flag.lower() == "active":
                    reasons.add(name)
        os.remove(self.path)
        if not sm:
            return None
        return {"sm_mhz": statistics.median(sm), "sm_max_mhz": max(smax), "reasons": sorted(reasons),
                "samples": len(sm)}


def max_over_ranks(value: float, world: int, device="cpu") -> float:
    """The slowest rank's value (every rank runs an independent replica; the
    job's time is the longest one)."""
    if world <= 1:
        return float(value)
    import torch
    import torch.distributed as dist
    t = torch.tensor([float(value)], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def whole_job_rate(units_per_rank: float, world: int, seconds: float) -> float:
    """Units processed by all ranks per second of the slowest rank."""
    return world * units_per_rank / seconds


def _setup_gpu(torch, lbmd, inputs, seed_offset=0):
    stream = torch.cuda.Stream()
    torch.cuda.set_stream(stream)
    sim = lbmd.LBMD(*SHAPE, variant="B", precision=PRECISION, n_sub=N_SUB, kT=KT, zeta=ZETA, seed=SEED + seed_offset,
                    max_particles=N_PARTICLES, stream=stream.cuda_stream)
    pos = inputs.uniform_positions(N_PARTICLES, SHAPE, SEED + seed_offset)
    vel = inputs.maxwell_velocities(N_PARTICLES, KT, SEED + seed_offset)
    sim.add_particles(pos, vel)
    return sim, stream, pos, vel


def _plain_lb_form(torch, lbmd, stream, peak, steps=50):
    """The LB step alone: 256^3 D3Q19, no particles, kT = 1e-4, FP32 -- the
    LB kernel's roofline without the coupling (152 B/node)."""
    sim = lbmd.LBMD(*SHAPE, variant="B", precision="fp32", n_sub=1, kT=KT, seed=SEED, stream=stream.cuda_stream)
    sim.run_cycles(5)
    a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    torch.cuda.synchronize()
    a.record(stream)
    sim.run_cycles(steps)
    b.record(stream)
    torch.cuda.synchronize()
    sim.close()
    ms = a.elapsed_time(b) / steps
    n_nodes = SHAPE[0] * SHAPE[1] * SHAPE[2]
    return {"workload": "256^3 D3Q19, no particles, kT=1e-4, FP32 (an empty MD step and one LB step per cycle)",
            "value": round(n_nodes / (ms * 1e-3) / 1e6, 1), "unit": "MLUPS", "ms_per_step": round(ms, 4),
            "roofline_frac": round(LB_BYTES_PER_NODE * n_nodes / (ms * 1e-3) / 1e9 / peak, 4)}


def _time_form(torch, lbmd, inputs, stream, precision, steps, pos, vel):
    """Cycle time of the same workload with another population storage form."""
    sim = lbmd.LBMD(*SHAPE, variant="B", precision=precision, n_sub=N_SUB, kT=KT, zeta=ZETA, seed=SEED,
                    max_particles=N_PARTICLES, stream=stream.cuda_stream)
    sim.add_particles(pos, vel)
    sim.run_cycles(3)
    a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    torch.cuda.synchronize()
    a.record(stream)
    sim.run_cycles(steps)
    b.record(stream)
    torch.cuda.synchronize()
    ms = a.elapsed_time(b) / steps
    ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(5)]
    for e0, e1 in ev:
        for _ in range(N_SUB):
            sim.md_substep()
        e0.record(stream)
        sim.lb_step()
        e1.record(stream)
    torch.cuda.synchronize()
    lb_ms = sum(e0.elapsed_time(e1) for e0, e1 in ev) / len(ev)
    sim.close()
    return ms, lb_ms


ACCURACY_CYCLES = 100  # 1000 MD steps at m = 10
ACCURACY_FORMS = ("fp32", "fp16dev", "fp16dev_sr", "bf16dev", "bf16dev_sr")


def _precision_accuracy(lbmd, inputs, stream, pos, vel):
    """Per-observable errors of the storage forms on the benchmark workload
    over 1000 MD steps, each from the same initial state and Philox streams:
    the mass against N rho0, the total (fluid + particle) momentum against
    that of the initial particles (both conserved exactly in exact
    arithmetic), in units of the particles' thermal momentum sqrt(N_p m kT),
    and the particle temperature against the FP32 run."""
    import numpy as np

    n_nodes = SHAPE[0] * SHAPE[1] * SHAPE[2]
    p0 = np.asarray(vel).sum(axis=0)
    p_scale = float(np.sqrt(N_PARTICLES * KT))
    out = {"workload": WORKLOAD.replace(", FP32", "") + ", %d MD steps" % (ACCURACY_CYCLES * N_SUB)}
    for prec in ACCURACY_FORMS:
        sim = lbmd.LBMD(*SHAPE, variant="B", precision=prec, n_sub=N_SUB, kT=KT, zeta=ZETA, seed=SEED,
                        max_particles=N_PARTICLES, stream=stream.cuda_stream)
        sim.add_particles(pos, vel)
        sim.run_cycles(ACCURACY_CYCLES)
        ob = sim.observables()
        sim.close()
        row = {"mass_rel": float("%.3g" % abs(ob["mass"] / (n_nodes * 1.0) - 1.0)),
               "momentum_rel": float("%.3g" % (np.linalg.norm(ob["p_fluid"] + ob["p_particles"] - p0) / p_scale)),
               "kT_particles": float("%.6g" % ob["kT_particles"])}
        if prec != "fp32":
            row["kT_rel_vs_fp32"] = float("%.3g" % abs(ob["kT_particles"] / out["fp32"]["kT_particles"] - 1.0))
        out[prec] = row
    return out


BATCH_REPLICAS, BATCH_MD_STEPS, BATCH_SAMPLE = 512, 2000, 10


def _batched_replicas(torch, lbmd, inputs, stream, peak, schedule="period_graph", edges=(12, 16, 24, 32)):
    """The batched form: 512 independent replica boxes (cubic edges from
    {12, 16, 24, 32}, 1-400 ideal particles, zeta in [0.5, 5], m in {1, 5,
    10}, variants alternating A and B, kT = 1e-4, FP32), 2000 MD steps
    replayed from the captured period graph, with every replica's particle
    kinetic energy recorded on the device every 10 MD steps.  Reports the
    throughput and the per-replica temperature drift (stable replicas), and
    the replicas flagged unstable (explicit friction, zeta dt / m >~ 2)."""
    import numpy as np

    cfg = inputs.replica_configs(BATCH_REPLICAS, SEED, edges=edges)
    R = BATCH_REPLICAS
    b = lbmd.Batch(cfg["dims"], n_sub=cfg["n_sub"], variant=cfg["variant"], zeta=cfg["zeta"],
                   seed=np.arange(R, dtype=np.uint64) + np.uint64(SEED * 1000), max_particles=cfg["n_particles"],
                   precision="fp32", kT=KT, stream=stream.cuda_stream)
    for r in range(R):
        n = int(cfg["n_particles"][r])
        b.add_particles(r, inputs.uniform_positions(n, cfg["dims"][r], SEED + r),
                        inputs.maxwell_velocities(n, KT, SEED + r))
    b.set_schedule(schedule)
    b.run(10)  # tunes the particle kernels and captures the graph
    n_samples = BATCH_MD_STEPS // BATCH_SAMPLE + 1
    kin = torch.empty((n_samples, R, 5), dtype=torch.float64, device="cuda")
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    torch.cuda.synchronize()
    e0.record(stream)
    b.kinetic_device(kin[0].data_ptr())
    for s in range(1, n_samples):
        b.run(BATCH_SAMPLE)
        b.kinetic_device(kin[s].data_ptr())
    e1.record(stream)
    torch.cuda.synchronize()
    ms = e0.elapsed_time(e1)
    unstable = b.unstable().astype(bool)
    k = kin.cpu().numpy()
    stable = ~unstable
    nodes = cfg["dims"].prod(axis=1).astype(np.float64)
    node_updates = float((nodes * (BATCH_MD_STEPS // cfg["n_sub"]))[stable].sum())
    psteps = float(cfg["n_particles"][stable].sum()) * BATCH_MD_STEPS
    alg_bytes = LB_BYTES_PER_NODE * node_updates + PARTICLE_BYTES * psteps
    # per-replica temperature T / kT over the run; excess = mean over the
    # second half - 1, drift = least-squares slope over the second half per
    # 1000 MD steps
    T = k[:, :, 0] / (3.0 * np.maximum(k[:, :, 4], 1.0) * KT)
    half = n_samples // 2
    t = np.arange(n_samples)[half:] * BATCH_SAMPLE / 1000.0
    excess = T[half:].mean(axis=0) - 1.0
    slope = np.zeros(R)
    if stable.any():
        slope[stable] = np.polyfit(t, T[half:][:, stable], 1)[0]
    zdt = cfg["zeta"] / cfg["n_sub"]
    var = np.array(cfg["variant"])
    bins = [(0.0, 0.25), (0.25, 0.5), (0.5, 1.0), (1.0, 2.0), (2.0, 10.0)]
    temp = {}
    for v in ("A", "B"):
        sel = stable & (var == v)
        w = cfg["n_particles"].astype(np.float64)
        byb = {}
        for lo, hi in bins:
            m = sel & (zdt >= lo) & (zdt < hi)
            if m.any():
                byb["%g-%g" % (lo, hi)] = {"replicas": int(m.sum()),
                                           "excess_T": round(float((excess[m] * w[m]).sum() / w[m].sum()), 4)}
        temp[v] = {"replicas": int(sel.sum()),
                   "excess_T_weighted": round(float((excess[sel] * w[sel]).sum() / w[sel].sum()), 4),
                   "median_drift_per_1000_steps": round(float(np.median(slope[sel])), 4),
                   "by_zeta_dt": byb}
    tune = b.tuning()
    tune["persistent"] = b.persistent_tuning()
    b.close()
    return {
        "schedule": schedule,
        "workload": "512 replica boxes, edges {%s}, 1-400 ideal particles, zeta in [0.5, 5], "
                    "m in {1,5,10}, variants A/B alternating, kT=1e-4, FP32, 2000 MD steps"
                    % ",".join(str(e) for e in edges),
        "value": round(node_updates / (ms * 1e-3) / 1e6, 1), "unit": "MLUPS",
        "particle_substeps_per_s": float("%.4g" % (psteps / (ms * 1e-3))),
        "ms_total": round(ms, 2), "lb_node_updates": node_updates,
        "roofline_frac": round(alg_bytes / (ms * 1e-3) / 1e9 / peak, 4),
        "graph_launches": BATCH_MD_STEPS // 10, "tuning": tune,
        "unstable": {"count": int(unstable.sum()), "min_zeta_dt_unstable":
                     round(float(zdt[unstable].min()), 3) if unstable.any() else None,
                     "max_zeta_dt_stable": round(float(zdt[stable].max()), 3)},
        "temperature": temp,
    }


def _variant_costs(torch, lbmd, inputs, stream, pos, vel, steps, ms_b):
    """Cycle time of variants A and C on the same workload against B (the
    paper's comparison of the extra effort of B and C over A, Sec. 4)."""
    out = {}
    for v in ("A", "C"):
        sim = lbmd.LBMD(*SHAPE, variant=v, precision="fp32", n_sub=N_SUB, kT=KT, zeta=ZETA, seed=SEED,
                        max_particles=N_PARTICLES, stream=stream.cuda_stream)
        sim.add_particles(pos, vel)
        sim.run_cycles(3)
        a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        torch.cuda.synchronize()
        a.record(stream)
        sim.run_cycles(steps)
        b.record(stream)
        torch.cuda.synchronize()
        ms = a.elapsed_time(b) / steps
        out[v] = {"ms_per_cycle": round(ms, 4),
                  "value": round(SHAPE[0] * SHAPE[1] * SHAPE[2] / (ms * 1e-3) / 1e6, 1), "unit": "MLUPS"}
        sim.close()
    out["B"] = {"ms_per_cycle": round(ms_b, 4)}
    ma = out["A"]["ms_per_cycle"]
    out["extra_vs_A"] = {"B": round(ms_b / ma - 1.0, 4), "C": round(out["C"]["ms_per_cycle"] / ma - 1.0, 4)}
    return out


def _bead_spring_64_form(torch, lbmd, inputs, stream):
    """The configuration of the A-versus-B cost comparison: 64^3, 64 random-walk
    chains of 64 beads (harmonic bonds k = 30, r0 = 1, mass 1, zeta = 2),
    kT = 1e-4, n = 10, FP32, 10^4 MD steps (1000 cycles replayed from the
    captured cycle graph) for variants A and B; GPU time per cycle by CUDA
    events and the extra cost of B over A (Sec. 3: 'a few percent')."""
    shape, cycles = (64, 64, 64), 1000
    pos, bonds = inputs.bead_spring_chains(64, 64, shape, 2)
    vel = inputs.maxwell_velocities(pos.shape[0], KT, 2)
    out = {"workload": "64^3 D3Q19, 64 chains x 64 beads (harmonic k=30, r0=1), zeta=2, kT=1e-4, n=10, FP32, "
                       "10^4 MD steps"}
    ms = {}
    for v in ("A", "B"):
        sim = lbmd.LBMD(*shape, variant=v, precision="fp32", n_sub=10, kT=KT, zeta=2.0, seed=SEED,
                        max_particles=pos.shape[0], max_bonds=bonds.shape[0], stream=stream.cuda_stream)
        sim.add_particles(pos, vel)
        sim.add_bonds(bonds, 30.0, 1.0)
        sim.run_cycles(20)
        a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        torch.cuda.synchronize()
        a.record(stream)
        sim.run_cycles(cycles)
        b.record(stream)
        torch.cuda.synchronize()
        ms[v] = a.elapsed_time(b) / cycles
        sim.close()
    n_nodes = shape[0] * shape[1] * shape[2]
    for v in ("A", "B"):
        out[v] = {"ms_per_cycle": round(ms[v], 5), "value": round(n_nodes / (ms[v] * 1e-3) / 1e6, 1),
                  "unit": "MLUPS", "particle_substeps_per_s": float("%.4g" % (pos.shape[0] * 10 / (ms[v] * 1e-3)))}
    out["extra_vs_A"] = {"B": round(ms["B"] / ms["A"] - 1.0, 4)}
    return out


def _kremer_grest_form(torch, stream):
    """The paper's test system (Sec. 4): 10 Kremer-Grest chains of 256 beads in
    (20 sigma)^3, LJ units converted to lattice units, HALF_STEP integrator.
    GPU time per MD step (graph-replayed cycles, CUDA events) of variants A,
    B and C at m = 10, dt = 0.005 tau, zeta = 20 mu/tau (the paper's cost
    comparison), and the share of the all-pairs Lennard-Jones forces (B with
    the LJ forces switched off, FENE springs kept)."""
    from paper_1610_02733_gb300 import sweep

    def per_md_step(variant, lj=True, cycles=300):
        sim, lp = sweep.build_system(variant, 10, 0.005, 20.0, integrator="half_step", stream=stream.cuda_stream)
        if not lj:
            sim.set_lj(0.0, 1.0, 0.0)
        sim.run_cycles(20)
        a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        torch.cuda.synchronize()
        a.record(stream)
        sim.run_cycles(cycles)
        b.record(stream)
        torch.cuda.synchronize()
        ms = a.elapsed_time(b) / (cycles * 10)
        sim.close()
        return ms

    ms = {v: per_md_step(v) for v in ("A", "B", "C")}
    no_lj = per_md_step("B", lj=False)
    n = 2560
    return {"workload": "10 x 256-bead Kremer-Grest chains in (20 sigma)^3 (2560 beads, 20^3 lattice), m=10, "
                        "dt=0.005 tau, zeta=20 mu/tau, kT=epsilon, HALF_STEP integrator, FP32",
            "ms_per_md_step": {v: round(x, 5) for v, x in ms.items()},
            "particle_substeps_per_s": {v: float("%.4g" % (n / (x * 1e-3))) for v, x in ms.items()},
            "extra_vs_A": {v: round(ms[v] / ms["A"] - 1.0, 4) for v in ("B", "C")},
            "lj_ms_per_md_step": round(ms["B"] - no_lj, 5),
            "lj": "Verlet lists (r_cut + 0.5, rebuilt every LB step), exactly the all-pairs forces"}


def _adjoint_form(torch, lbmd, inputs):
    """The adjoint form: L = mean particle drag along x over 200 MD steps
    (32^3, 64 ideal particles, zeta = 1.5, m = 10, body force 1e-5 along x,
    kT = 1e-4 with fixed Philox counters), forward pass with a checkpoint per
    LB step and the hand-written backward pass, FP32, with the FP64 gradients
    as the accuracy reference."""
    import numpy as np

    shape, n, cycles, zeta = (32, 32, 32), 64, 20, 1.5
    pos = inputs.uniform_positions(n, shape, SEED + 7)
    vel = inputs.maxwell_velocities(n, KT, SEED + 7)
    out = {"workload": "32^3 D3Q19, 64 ideal particles, zeta=1.5, m=10, 200 MD steps, body force 1e-5, kT=1e-4, "
                       "variant B; L = mean particle drag along x; gradients w.r.t. zeta and initial positions"}
    grads = {}
    for prec in ("fp64", "fp32"):
        ad = lbmd.Adjoint(*shape, n_particles=n, n_cycles=cycles, n_sub=10, precision=prec, kT=KT,
                          body_force=(1e-5, 0.0, 0.0), seed=SEED)
        ad.forward(zeta, pos, vel)  # warm-up
        ad.backward()
        t0 = time.perf_counter()
        L = ad.forward(zeta, pos, vel)
        t1 = time.perf_counter()
        dz, dpos = ad.backward()
        t2 = time.perf_counter()
        grads[prec] = (L, dz, dpos)
        out[prec] = {"forward_ms": round((t1 - t0) * 1e3, 3), "backward_ms": round((t2 - t1) * 1e3, 3),
                     "loss": L, "dL_dzeta": dz, "dL_dR0_norm": float(np.linalg.norm(dpos))}
        ad.close()
    L64, z64, p64 = grads["fp64"]
    L32, z32, p32 = grads["fp32"]
    out["fp32_vs_fp64"] = {"loss_rel": float(abs(L32 - L64) / abs(L64)),
                           "dL_dzeta_rel": float(abs(z32 - z64) / abs(z64)),
                           "dL_dR0_rel": float(np.linalg.norm(p32 - p64) / np.linalg.norm(p64))}
    out["accuracy"] = "FP64 gradients match the oracle tangent to 1e-9 and FP64 finite differences (tests)"
    return out


def _touched_nodes(pos):
    """Distinct nodes at the corners of the particles' cells (exact)."""
    import numpy as np
    base = np.floor(pos).astype(np.int64)
    L = np.array(SHAPE)
    ids = []
    for k in range(8):
        o = np.array([k & 1, (k >> 1) & 1, (k >> 2) & 1])
        c = (base + o) % L
        ids.append(c[:, 0] + L[0] * (c[:, 1] + L[1] * c[:, 2]))
    return int(np.unique(np.concatenate(ids)).size)


def run_gpu(args):
    import numpy as np
    import torch
    import torch.distributed as dist

    from paper_1610_02733_gb300 import inputs, lbmd

    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    if world > 1:
        dist.init_process_group("nccl")
    torch.cuda.set_device(local)
    dev = torch.cuda.current_device()

    sim, stream, pos0, vel0 = _setup_gpu(torch, lbmd, inputs, seed_offset=rank)
    n_nodes = SHAPE[0] * SHAPE[1] * SHAPE[2]

    # warm-up through the product's cycle replay (captures the CUDA graphs of
    # both buffer parities on first use)
    sim.run_cycles(max(args.warmup, 2))
    stream.synchronize()

    # timed region: K full cycles replayed from the captured CUDA graphs,
    # device-resident inputs
    start, stop = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    fallback0 = sim.moments_fallback_rows()
    clocks = ClockSampler(dev)
    clocks.start()
    if world > 1:
        dist.barrier()
    torch.cuda.synchronize()
    start.record(stream)
    sim.run_cycles(args.steps)
    stop.record(stream)
    torch.cuda.synchronize()
    if world > 1:
        dist.barrier()
    clk = clocks.stop()
    # collide rows whose fused post-stream moments timed out in the timed
    # cycles (computed by the follow-up kernel instead; same results)
    fallback_rows = sim.moments_fallback_rows() - fallback0
    total_ms = max_over_ranks(start.elapsed_time(stop), world, "cuda")
    ms_per_step = total_ms / args.steps
    mlups = whole_job_rate(n_nodes * args.steps, world, total_ms * 1e-3) / 1e6
    psubsteps = whole_job_rate(N_PARTICLES * N_SUB * args.steps, world, total_ms * 1e-3)

    # breakdown: the same cycles issued call by call, with events around every
    # LB step (its kernels' per-launch duration) on the launching stream
    nb = max(5, min(args.steps, 20))
    ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(nb)]
    b0, b1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    torch.cuda.synchronize()
    b0.record(stream)
    for k in range(nb):
        for _ in range(N_SUB):
            sim.md_substep()
        ev[k][0].record(stream)
        sim.lb_step()
        ev[k][1].record(stream)
    b1.record(stream)
    torch.cuda.synchronize()
    eager_ms = b0.elapsed_time(b1) / nb
    lb_avg_ms = float(np.mean([a.elapsed_time(b) for a, b in ev]))
    md_ms = eager_ms - lb_avg_ms

    # end to end through the C ABI with host buffers: every step uploads the
    # particle state from pinned host memory, runs the cycle, and reads the
    # particles and the observables back.  Two forms: the synchronising
    # accessors, and the asynchronous ones, whose copies overlap the cycles
    # (the upload of step k + 1 and the downloads of step k run beside the
    # cycle of step k + 1), synchronised once at the end
    h_pos = torch.from_numpy(np.ascontiguousarray(pos0, dtype=np.float64).reshape(-1)).pin_memory()
    h_vel = torch.from_numpy(np.ascontiguousarray(vel0, dtype=np.float64).reshape(-1)).pin_memory()
    o_pos = [torch.empty(3 * N_PARTICLES, dtype=torch.float64).pin_memory() for _ in range(2)]
    o_vel = [torch.empty(3 * N_PARTICLES, dtype=torch.float64).pin_memory() for _ in range(2)]
    e_steps = max(1, min(args.steps, 50))

    def e2e_sync():
        for k in range(e_steps):
            sim.set_particles(h_pos, h_vel)
            sim.run_cycles(1)
            sim.particles(out=(o_pos[0], o_vel[0]))
            sim.observables()

    def e2e_async():
        sim.set_particles_async(h_pos, h_vel)
        for k in range(e_steps):
            sim.run_cycles(1)
            sim.observables_async()
            sim.particles_async(o_pos[k % 2], o_vel[k % 2])
            if k + 1 < e_steps:
                sim.set_particles_async(h_pos, h_vel)
        sim.synchronize()

    e2e_rates = {}
    for name, fn in (("synchronous", e2e_sync), ("asynchronous", e2e_async)):
        if world > 1:
            dist.barrier()
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        fn()
        torch.cuda.synchronize()
        e2e_s = max_over_ranks(time.perf_counter() - t0, world, "cuda")
        e2e_rates[name] = whole_job_rate(n_nodes * e_steps, world, e2e_s) / 1e6
    if world > 1:
        dist.barrier()
    e2e_mlups = e2e_rates["asynchronous"]

    peak, peak_kind = _peaks()
    touched = _touched_nodes(pos0)
    cycle_alg_bytes = LB_BYTES_PER_NODE * n_nodes + N_SUB * (N_PARTICLES * 48 + touched * 32)
    # rooflines of the two phases of a cycle; the one that takes longer is
    # reported as the dominant unit
    md_alg = N_PARTICLES * PARTICLE_BYTES + touched * NODE_TOUCH_BYTES
    md_step_ms = md_ms / N_SUB
    lb_roof = {"bound": "hbm", "achieved": round(LB_BYTES_PER_NODE * n_nodes / (lb_avg_ms * 1e-3) / 1e9, 1),
               "peak": peak, "unit": "GB/s", "traffic": _profiled_traffic("lb_step"),
               "kernel": "LB step: re-ordering + active nodes + lb_collide_push (fused moments) + moments_rest_kernel",
               "algorithmic_bytes": LB_BYTES_PER_NODE * n_nodes, "ms": round(lb_avg_ms, 4), "peak_source": peak_kind}
    md_roof = {"bound": "hbm", "achieved": round(md_alg / (md_step_ms * 1e-3) / 1e9, 1), "peak": peak,
               "unit": "GB/s", "traffic": _profiled_traffic("md_substep"),
               "kernel": "MD step: couple_kernel + spread_rows_kernel + migrant_spread_kernel",
               "algorithmic_bytes": md_alg, "ms": round(md_step_ms, 4), "peak_source": peak_kind}
    for r in (lb_roof, md_roof):
        r["frac"] = round(r["achieved"] / peak, 4)
        if r["traffic"]:
            # the ncu DRAM bytes over the same time, and their ratio to the
            # algorithmic bytes (the implementation's overhead)
            r["dram_frac"] = round(r["traffic"] / (r["ms"] * 1e-3) / 1e9 / peak, 4)
            r["overhead"] = round(r["traffic"] / r["algorithmic_bytes"], 3)
    dominant = md_roof if md_ms > lb_avg_ms else lb_roof
    line = {
        "metric": METRIC,
        "value": round(mlups, 1),
        "unit": "MLUPS",
        "particle_substeps_per_s": float("%.4g" % psubsteps),
        "n_gpus": world,
        "steps": args.steps,
        "warmup": args.warmup,
        "ms_per_step": round(ms_per_step, 4),
        "higher_is_better": True,
        "scaling": "weak",
        "vs_baseline": None,
        "dtype": "f32",
        "data": "synthetic (seeded uniform positions, Maxwellian velocities, fluid at rest)",
        "config": {"workload": WORKLOAD, "lattice": list(SHAPE), "particles": N_PARTICLES, "n_sub": N_SUB,
                   "kT": KT, "zeta": ZETA, "variant": "B", "l2": "inputs larger than L2 (2.5 GB populations)",
                   "parallelism": "replicas" if world > 1 else "single GPU"},
        "breakdown_ms": {"lb_step": round(lb_avg_ms, 4), "md_substeps": round(md_ms, 4),
                         "eager_cycle": round(eager_ms, 4), "graph_cycle": round(ms_per_step, 4)},
        "roofline": dominant,
        "roofline_phases": {"lb_step": lb_roof, "md_substep": md_roof},
        "cycle_roofline": {"algorithmic_bytes": cycle_alg_bytes, "touched_nodes": touched,
                           "frac": round(cycle_alg_bytes / (ms_per_step * 1e-3) / 1e9 / peak, 4)},
        "e2e": {"value": round(e2e_mlups, 1), "unit": "MLUPS", "h2d_bytes_per_step": 2 * 3 * 8 * N_PARTICLES,
                "d2h_bytes_per_step": 2 * 3 * 8 * N_PARTICLES + 80, "steps": e_steps,
                "accessors": "asynchronous (lbmd_*_async, one lbmd_synchronize at the end)",
                "synchronous_accessors_value": round(e2e_rates["synchronous"], 1)},
        "gpu_launches": args.steps * LAUNCHES_PER_CYCLE,
        "moments_fallback_rows": fallback_rows,
        "clocks": clk,
    }
    sim.close()
    if not args.no_forms:
        # the reduced-precision storage forms on the same workload, against
        # this plain FP32 path (algorithmic LB bytes 2 x 19 x 2 B per node)
        forms = {}
        for prec in ("fp16dev", "bf16dev", "fp16dev_sr", "bf16dev_sr"):
            ms, lb_ms = _time_form(torch, lbmd, inputs, stream, prec, min(args.steps, 50), pos0, vel0)
            lb_bytes = 2 * 19 * 2 * n_nodes
            forms[prec] = {"value": round(whole_job_rate(n_nodes, world, ms * 1e-3) / 1e6, 1), "unit": "MLUPS",
                           "ms_per_step": round(ms, 4), "lb_step_ms": round(lb_ms, 4),
                           "speedup_vs_fp32": round(ms_per_step / ms, 3),
                           "lb_step_speedup_vs_fp32": round(lb_avg_ms / lb_ms, 3),
                           "lb_roofline_frac": round(lb_bytes / (lb_ms * 1e-3) / 1e9 / peak, 4)}
        # the FP64 storage form (the verification precision): its cost on
        # this GPU, whose FP64 pipes issue 2 FMA per SM per clock
        ms, lb_ms = _time_form(torch, lbmd, inputs, stream, "fp64", 3, pos0, vel0)
        forms["fp64"] = {"value": round(whole_job_rate(n_nodes, world, ms * 1e-3) / 1e6, 1), "unit": "MLUPS",
                         "ms_per_step": round(ms, 3), "lb_step_ms": round(lb_ms, 3),
                         "slowdown_vs_fp32": round(ms / ms_per_step, 2),
                         "lb_roofline_frac": round(2 * 19 * 8 * n_nodes / (lb_ms * 1e-3) / 1e9 / peak, 4)}
        line["precision_forms"] = forms
        line["precision_accuracy"] = _precision_accuracy(lbmd, inputs, stream, pos0, vel0)
        line["variants"] = _variant_costs(torch, lbmd, inputs, stream, pos0, vel0, min(args.steps, 30), ms_per_step)
        line["batched_replicas"] = _batched_replicas(torch, lbmd, inputs, stream, peak)
        pers = _batched_replicas(torch, lbmd, inputs, stream, peak, "persistent")
        line["batched_replicas"]["persistent"] = {k: pers[k] for k in ("ms_total", "value", "unit", "roofline_frac")}
        line["batched_replicas"]["persistent"]["cluster_blocks"] = pers["tuning"]["persistent"]["cluster_blocks"]
        line["adjoint"] = _adjoint_form(torch, lbmd, inputs)
        line["kremer_grest"] = _kremer_grest_form(torch, stream)
        line["bead_spring_64"] = _bead_spring_64_form(torch, lbmd, inputs, stream)
        line["plain_lb"] = _plain_lb_form(torch, lbmd, stream, peak)
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        line["cpu_baseline"] = cpu_baseline()
    if rank == 0:
        print(json.dumps(line))
    if world > 1:
        dist.destroy_process_group()


def _source_hash(files):
    import hashlib
    h = hashlib.sha256()
    for f in files:
        with open(os.path.join(ROOT, "paper_1610_02733_gb300", "csrc", f), "rb") as fh:
            h.update(fh.read())
    return h.hexdigest()[:16]


def _profiled_traffic(unit):
    """DRAM bytes (read + write) per launch of `unit` from the ncu summary in
    profiles/traffic.json; None unless the kernel sources still hash to the
    value recorded with the capture, and for any workload but the benchmark's
    (the figures are for 256^3 / 10^6 particles, FP32, kT = 1e-4)."""
    if (SHAPE, N_PARTICLES, KT, PRECISION) != ((256, 256, 256), 1_000_000, 1e-4, "fp32"):
        return None
    try:
        with open(os.path.join(ROOT, "profiles", "traffic.json")) as fh:
            d = json.load(fh)[unit]
        if _source_hash(d["sources"]) != d["source_hash"]:
            return None
        return d["dram_bytes"]
    except Exception:
        return None


def _oracle_sample(edge: int, cycles: int):
    """Time the FP64 oracle on a sample of the workload: an edge^3 box at the
    same particle density (10^6 / 256^3), `cycles` full cycles."""
    from oracle import oracle as orc
    from paper_1610_02733_gb300 import inputs
    shape = (edge, edge, edge)
    n = max(1, int(round(N_PARTICLES * edge ** 3 / (SHAPE[0] * SHAPE[1] * SHAPE[2]))))
    o = orc.Oracle(*shape, n_sub=N_SUB, variant=1, kT=KT, zeta=ZETA, seed=SEED)
    o.add_particles(inputs.uniform_positions(n, shape, SEED), inputs.maxwell_velocities(n, KT, SEED))
    t0 = time.perf_counter()
    o.cycle(cycles)
    dt = time.perf_counter() - t0
    o.close()
    return dt, edge ** 3, n


def _cpu_model():
    """The host CPU's model name (lscpu), else what platform reports."""
    try:
        out = subprocess.run(["lscpu"], capture_output=True, text=True, timeout=10).stdout
        for line in out.splitlines():
            if line.lower().startswith("model name"):
                return line.split(":", 1)[1].strip()
    except Exception:
        pass
    import platform
    return platform.processor() or platform.machine()


def _oracle_full_cycles(cycles: int):
    """The oracle's OpenMP timing build (LB node loops over all host cores,
    particle loop serial) on the full workload: 256^3, 10^6 particles,
    `cycles` cycles of 10 MD steps + 1 LB step."""
    from oracle import oracle as orc
    from paper_1610_02733_gb300 import inputs
    o = orc.Oracle(*SHAPE, n_sub=N_SUB, variant=1, kT=KT, zeta=ZETA, seed=SEED, openmp=True)
    o.add_particles(inputs.uniform_positions(N_PARTICLES, SHAPE, SEED), inputs.maxwell_velocities(N_PARTICLES, KT, SEED))
    t0 = time.perf_counter()
    o.cycle(cycles)
    dt = time.perf_counter() - t0
    o.close()
    return dt


def _oracle_small_configs():
    """The oracle (OpenMP timing build, all host cores on the LB node loops)
    on BASELINE's first configuration in full -- 8^3, 10 particles, FP64,
    m = 5, 1000 MD steps, variants A and B -- and on 10 cycles (100 MD steps)
    of its second, 64^3 with 64 chains of 64 beads (harmonic k = 30, r0 = 1,
    zeta = 2, m = 10, variants A and B)."""
    from oracle import oracle as orc
    from paper_1610_02733_gb300 import inputs
    out = {}
    for v, name in ((0, "A"), (1, "B")):
        o = orc.Oracle(8, 8, 8, n_sub=5, variant=v, kT=1e-4, zeta=1.0, seed=1, openmp=True)
        o.add_particles(inputs.uniform_positions(10, (8, 8, 8), 1), inputs.maxwell_velocities(10, 1e-4, 1))
        t0 = time.perf_counter()
        o.cycle(200)
        dt = time.perf_counter() - t0
        o.close()
        out["c1_" + name] = {"value": round(512 * 200 / dt / 1e6, 4), "unit": "MLUPS", "s": round(dt, 3),
                             "sample": "8^3, 10 particles, m=5, 1000 MD steps, FP64 (the whole configuration)"}
    shape = (64, 64, 64)
    pos, bonds = inputs.bead_spring_chains(64, 64, shape, 2)
    vel = inputs.maxwell_velocities(pos.shape[0], KT, 2)
    for v, name in ((0, "A"), (1, "B")):
        o = orc.Oracle(*shape, n_sub=10, variant=v, kT=KT, zeta=2.0, seed=2, openmp=True)
        o.add_particles(pos, vel)
        o.add_bonds(bonds, 30.0, 1.0)
        t0 = time.perf_counter()
        o.cycle(10)
        dt = time.perf_counter() - t0
        o.close()
        out["c2_" + name] = {"value": round(64 ** 3 * 10 / dt / 1e6, 4), "unit": "MLUPS",
                             "particle_substeps_per_s": float("%.4g" % (pos.shape[0] * 100 / dt)), "s": round(dt, 3),
                             "sample": "10 cycles (100 MD steps) of 64^3 with 64 chains x 64 beads, m=10, FP64"}
    return out


def cpu_baseline():
    """The FP64 oracle on the host cores: 3 full cycles of the benchmark
    workload with its OpenMP timing build (all cores on the LB node loops,
    particle loop serial), and a bounded single-thread sample of the plain
    build (8 cycles of a 128^3 box at the same particle density)."""
    edge, cycles = 128, 8
    dt, nodes, n = _oracle_sample(edge, cycles)
    single = {"value": round(nodes * cycles / dt / 1e6, 4), "unit": "MLUPS", "cores": 1,
              "particle_substeps_per_s": float("%.4g" % (n * N_SUB * cycles / dt)),
              "sample": "%d cycles of a %d^3 box with %d particles (same density, n=10, variant B), FP64, "
                        "single thread, %.1f s" % (cycles, edge, n, dt)}
    cores = os.cpu_count() or 1
    out = {"kind": "oracle", "cpu_model": _cpu_model(), "nproc": cores, "single_thread": single}
    full_cycles = 3
    try:
        dt_full = _oracle_full_cycles(full_cycles)
        nodes_full = SHAPE[0] * SHAPE[1] * SHAPE[2]
        out.update({"value": round(nodes_full * full_cycles / dt_full / 1e6, 4), "unit": "MLUPS", "cores": cores,
                    "particle_substeps_per_s": float("%.4g" % (N_PARTICLES * N_SUB * full_cycles / dt_full)),
                    "sample": "%d full cycles of the workload (%dx%dx%d, %d particles, n=10, variant B), FP64, "
                              "OpenMP over %d cores on the LB node loops, particle loop serial, %.1f s" % (
                                  full_cycles, SHAPE[0], SHAPE[1], SHAPE[2], N_PARTICLES, cores, dt_full)})
    except Exception as exc:  # no OpenMP runtime on this host
        out.update({"value": single["value"], "unit": "MLUPS", "cores": 1, "sample": single["sample"],
                    "all_cores": "unavailable: %s" % exc})
    try:
        out["other_configs"] = _oracle_small_configs()
    except Exception as exc:
        out["other_configs"] = "unavailable: %s" % exc
    return out


def run_reference(args):
    """The oracle as the reference arm, on the host cores; each step is one
    cycle of a 64^3 sample of the workload at the same particle density."""
    rank = int(os.environ.get("RANK", "0"))
    if rank != 0:
        return
    edge = 64
    for _ in range(args.warmup):
        _oracle_sample(edge, 1)
    tot, nodes, n = 0.0, 0, 0
    for _ in range(args.steps):
        dt, nodes, n = _oracle_sample(edge, 1)
        tot += dt
    mlups = nodes * args.steps / tot / 1e6
    sample = "1 cycle of a %d^3 box with %d particles per step (same density, n=10, variant B), FP64" % (edge, n)
    print(json.dumps({
        "impl": "reference", "metric": METRIC, "value": round(mlups, 4), "unit": "MLUPS",
        "particle_substeps_per_s": float("%.4g" % (n * N_SUB * args.steps / tot)), "n_gpus": 0,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": round(1e3 * tot / args.steps, 3),
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
        "config": {"workload": WORKLOAD, "sample": sample},
        "cpu_baseline": {"value": round(mlups, 4), "unit": "MLUPS", "cores": 1, "kind": "oracle", "sample": sample},
        "e2e": {"value": round(mlups, 4), "unit": "MLUPS", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }))


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=100)
    ap.add_argument("--warmup", type=int, default=5)
    ap.add_argument("--impl", default="gb300", choices=["gb300", "reference"])
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-forms", action="store_true",
                    help="skip the reduced-precision, variant A/C, batched, adjoint and Kremer-Grest forms")
    ap.add_argument("--edge", type=int, default=256, help="lattice edge (profiling of smaller cases)")
    ap.add_argument("--lattice", type=int, nargs=3, metavar=("NX", "NY", "NZ"), default=None,
                    help="non-cubic lattice (profiling of smaller cases with 256-node rows)")
    ap.add_argument("--particles", type=int, default=1_000_000)
    ap.add_argument("--kT", type=float, default=1e-4, help="temperature (profiling: 0 switches the noise off)")
    ap.add_argument("--precision", default="fp32", choices=["fp32", "fp16dev", "bf16dev", "fp16dev_sr", "bf16dev_sr"],
                    help="population storage of the timed workload (profiling)")
    ap.add_argument("--only-form", default=None, choices=["batched_replicas"],
                    help="run only this form and print its JSON object (profiling)")
    ap.add_argument("--schedule", default="period_graph", choices=["period_graph", "persistent"],
                    help="schedule of the batched form with --only-form")
    ap.add_argument("--edges", type=int, nargs="+", default=[12, 16, 24, 32],
                    help="replica box edges of the batched form with --only-form")
    args = ap.parse_args()
    args.warmup = max(args.warmup, 3)
    global SHAPE, N_PARTICLES, WORKLOAD, KT, PRECISION
    KT = args.kT
    PRECISION = args.precision
    shape = tuple(args.lattice) if args.lattice else (args.edge, args.edge, args.edge)
    if shape != (256, 256, 256) or args.particles != 1_000_000 or KT != 1e-4 or PRECISION != "fp32":
        SHAPE = shape
        N_PARTICLES = args.particles
        WORKLOAD = "%dx%dx%d D3Q19 + %d ideal particles, variant B, n=10, %s storage, kT=%g" % (
            shape + (args.particles, PRECISION, KT))
    if args.impl == "reference":
        run_reference(args)
        return
    import __graft_entry__
    __graft_entry__.build()
    if args.only_form == "batched_replicas":
        import torch
        from paper_1610_02733_gb300 import inputs, lbmd
        out = _batched_replicas(torch, lbmd, inputs, torch.cuda.Stream(), _peaks()[0], args.schedule,
                                tuple(args.edges))
        print(json.dumps(out))
        return
    run_gpu(args)


if __name__ == "__main__":
    main()
