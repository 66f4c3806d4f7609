"""Temperature of a Kremer-Grest polymer system against the friction
coefficient, for the coupling variants A, B and C (Sec. 4): the paper's test
of the coupling, restated on synthetic chains.

The paper runs ten chains of 256 beads in a (20 sigma)^3 box (LJ cut at
2^(7/6) sigma, FENE springs, a = sigma, rho = 1 mu/sigma^3, k_B T = 1 epsilon,
eta = 3 epsilon tau/sigma^3), for m = 1, 5, 10 MD steps per LB step and MD
time steps dt = 0.001, 0.005, 0.010 tau, and reports the measured particle
temperature (mean kinetic energy) as a function of zeta.  It starts from a
pre-relaxed melt that is not available; here the chains are grown
self-avoiding (inputs.self_avoiding_chains) and equilibrated in the run
before the measurement window.

    python -m paper_1610_02733_gb300.sweep --out sweep.json [--quick]

Each grid point reports T / epsilon with a block-average standard error and
the GPU time per MD step; ``variant_costs`` times the three variants on the
same system (the paper's comparison of the coupling's extra effort)."""
import argparse
import functools
import json
import time

import numpy as np

from . import inputs, lbmd, lj_units

PAPER_MS = (1, 5, 10)
PAPER_DTS = (0.001, 0.005, 0.010)
ZETAS = (1.0, 2.5, 5.0, 10.0, 20.0)


@functools.lru_cache(maxsize=4)
def _chains(n_chains, n_beads, box, seed):
    return inputs.self_avoiding_chains(n_chains, n_beads, (box, box, box), seed)


def build_system(variant: str, m: int, dt: float, zeta: float, *, n_chains=10, n_beads=256, box=20, seed=1,
                 precision="fp32", integrator="start", stream=None):
    """One context holding the Kremer-Grest system at one grid point."""
    lp = lj_units.lattice_params(m, dt, zeta)
    pos, bonds = _chains(n_chains, n_beads, box, seed)
    n = pos.shape[0]
    sim = lbmd.LBMD(box, box, box, variant=variant, precision=precision, n_sub=m, kT=lp["kT"], zeta=lp["zeta"],
                    nu=lp["nu"], rho0=lp["rho0"], seed=seed, max_particles=n, max_bonds=bonds.shape[0],
                    integrator=integrator, stream=stream)
    sim.add_particles(pos, inputs.maxwell_velocities(n, lp["kT"], seed))
    sim.set_lj(lp["lj_eps"], lp["lj_sigma"], lp["lj_rc"])
    sim.add_fene_bonds(bonds, lp["fene_k"], lp["fene_R0"])
    return sim, lp


def measure_temperature(variant: str, m: int, dt: float, zeta: float, *, equil_tau=20.0, measure_tau=100.0,
                        sample_tau=0.05, n_blocks=10, **kw) -> dict:
    """Mean particle temperature T / epsilon over ``measure_tau`` after
    ``equil_tau`` (both in tau), sampled every ``sample_tau``."""
    sim, lp = build_system(variant, m, dt, zeta, **kw)
    tau_lb = lp["tau_lb"]
    every = max(1, int(round(sample_tau / tau_lb)))  # LB cycles between samples
    sim.run_cycles(max(1, int(round(equil_tau / tau_lb))))
    sim.observables()
    n_samples = max(n_blocks, int(round(measure_tau / (every * tau_lb))))
    n_samples -= n_samples % n_blocks
    temps = np.empty(n_samples)
    t0 = time.perf_counter()
    for s in range(n_samples):
        sim.run_cycles(every)
        temps[s] = lj_units.temperature_in_lj(sim.observables()["kT_particles"], lp)
    wall = time.perf_counter() - t0
    sim.close()
    blocks = temps.reshape(n_blocks, -1).mean(axis=1)
    return {"variant": variant, "m": m, "dt": dt, "zeta": zeta, "integrator": kw.get("integrator", "start"),
            "T": float(temps.mean()),
            "stderr": float(blocks.std(ddof=1) / np.sqrt(n_blocks)), "samples": int(n_samples),
            "measure_tau": n_samples * every * tau_lb,
            "ms_per_md_step": 1e3 * wall / (n_samples * every * m)}


def variant_costs(m: int, dt: float = 0.005, zeta: float = 20.0, cycles: int = 200, **kw) -> dict:
    """Wall time per MD step of variants A, B and C on the same system (graph-
    replayed cycles, synchronised at both ends), and the extra effort of B and
    C over A."""
    out = {}
    for v in ("A", "B", "C"):
        sim, _ = build_system(v, m, dt, zeta, **kw)
        sim.run_cycles(10)
        sim.observables()
        t0 = time.perf_counter()
        sim.run_cycles(cycles)
        sim.observables()
        out[v] = 1e3 * (time.perf_counter() - t0) / (cycles * m)
        sim.close()
    return {"m": m, "dt": dt, "zeta": zeta, "ms_per_md_step": out,
            "extra_vs_A": {v: out[v] / out["A"] - 1.0 for v in ("B", "C")}}


def main(argv=None):
    ap = argparse.ArgumentParser(description=__doc__.split("\n\n")[0])
    ap.add_argument("--out", default=None)
    ap.add_argument("--variants", default="A,B,C")
    ap.add_argument("--quick", action="store_true", help="shorter windows (equilibrate 10 tau, measure 30 tau)")
    ap.add_argument("--precision", default="fp32")
    ap.add_argument("--integrator", default="start", choices=["start", "half_step"],
                    help="where velocity Verlet evaluates the coupling force (lbmd_params.integrator)")
    ap.add_argument("--no-costs", action="store_true")
    ap.add_argument("--point", nargs=4, metavar=("VARIANT", "M", "DT", "ZETA"), default=None,
                    help="only run one grid point for --cycles LB cycles (e.g. under a profiler)")
    ap.add_argument("--cycles", type=int, default=100)
    args = ap.parse_args(argv)
    if args.point:
        v, m, dt, z = args.point[0], int(args.point[1]), float(args.point[2]), float(args.point[3])
        sim, lp = build_system(v, m, dt, z, precision=args.precision, integrator=args.integrator)
        sim.run_cycles(3)
        sim.observables()
        t0 = time.perf_counter()
        sim.run_cycles(args.cycles)
        ob = sim.observables()
        wall = time.perf_counter() - t0
        print(json.dumps({"variant": v, "m": m, "dt": dt, "zeta": z, "cycles": args.cycles,
                          "ms_per_md_step": 1e3 * wall / (args.cycles * m),
                          "T": lj_units.temperature_in_lj(ob["kT_particles"], lp)}))
        sim.close()
        return
    eq, ms = (10.0, 30.0) if args.quick else (20.0, 100.0)
    rows = []
    for v in args.variants.split(","):
        dts = PAPER_DTS if v != "C" else (0.005,)  # the paper compares B and C at dt = 0.005 tau
        for m in PAPER_MS:
            for dt in dts:
                for z in ZETAS:
                    r = measure_temperature(v, m, dt, z, equil_tau=eq, measure_tau=ms, precision=args.precision,
                                            integrator=args.integrator)
                    rows.append(r)
                    print(json.dumps(r), flush=True)
    costs = [] if args.no_costs else [variant_costs(m, integrator=args.integrator) for m in PAPER_MS]
    for c in costs:
        print(json.dumps(c), flush=True)
    if args.out:
        with open(args.out, "w") as fh:
            json.dump({"temperature": rows, "costs": costs}, fh, indent=1)


if __name__ == "__main__":
    main()
