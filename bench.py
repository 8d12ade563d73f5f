"""CTR-IBIM benchmark: pair-interactions/s of the full solve path on one GB300.

One step = the whole hot path for one synthetic molecule-sized problem:
setup (tube, geometry, correction weights, right-hand side), the
FP32-pair GMRES with FP64 refinement, and the polarization energy.
Default workload: ellipsoid (4, 3, 2) A with three seeded charges, h = 0.05,
tube 2h (about 178k tube nodes, 356k unknowns).

value = sum over systems of M^2 x (operator applications in the step) / time,
the pair count of every dense sum counted in full (including excluded pairs).

Usage: python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]
Under torchrun each rank runs an independent replica (no collective on the
data path); rank 0 prints one JSON line.
"""
from __future__ import annotations

import argparse
import ctypes
import json
import os
import statistics
import subprocess
import sys
import threading
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

# Algorithmic work per pair interaction (one target, one source, one orientation): the minimal FP32 form of
# the four kernels of Eq. (1.4) with their weights, an FMA counted as one FP32-pipe lane operation -- 3 sub,
# 3 for r^2, 1 for r, 1 kappa r, 9 for the three dot products, 2 inverse powers, 3 for the Yukawa factor,
# 4 for K11/K22, 1 for K12, about 11 for K21, 4 accumulations -- plus 2 SFU operations (rsqrt, ex2).  A
# launch's algorithmic work is this times M^2 interactions; the same count serves every arithmetic
# (float-float spends about ten FP32 operations per counted one, which its fraction shows).
ALG_OPS = 43
# The timed solve: GMRES restart length, FP32 inner tolerance and the solve tolerance
RESTART, INNER_TOL, SOLVE_TOL = 64, 1e-5, 1e-10
# FP32-pipe lane operations per pair evaluation as the kernels execute them, counted from the kernel source:
# one-sided evaluations (one orientation) and symmetric ones (both orientations, with the share of the
# in-warp transposed sums), for the packed FP32 and the float-float pair arithmetics (a packed f32x2
# instruction counts as two lane operations, the FMA pipe's throughput being the same either way).
# SFU work (rsqrt, ex2) and shared-memory loads are not counted.
OPS_FP32 = {"one": 41, "sym": 49}
OPS_DF64 = {"one": 423, "sym": 501}
# FP64 pipe lane operations per pair evaluation of the FP64 schedule (CUDA's exp and rsqrt included): the
# ncu count sm__inst_executed_pipe_fp64 x 32 / evaluations over one launch at h = 0.1 (69); its peak is the
# measured DFMA probe rate, there being no FP64 unit count to go by.
OPS_FP64 = {"one": 69, "sym": 69}
# DRAM bytes (read + write) per launch of the schedule kernels at the default workload (h = 0.05) from one
# ncu capture, valid only while the kernel sources hash to `sources` (otherwise reported as null); the
# profile records every re-keying after a change that leaves the kernels and the captured items unchanged.
TRAFFIC = {"profile": "profiles/dram_traffic_sched_kernels_ellipsoid_h0.05.txt", "h": 0.05,
           "sources": "2f15c2965403e8ce", "fp32": 2.659e7, "df64": 3.306e7, "fp64": None}
KERNEL_SOURCES = ("paper_2210_03699_gb300/csrc/pairkern.cuh", "paper_2210_03699_gb300/csrc/schedule.cu",
                  "paper_2210_03699_gb300/csrc/common.cuh")
# Treecode far field of the FP32 operator (FP32 charges): FMA-pipe lane operations per proxy evaluation
# counted from the kernel source (tree.cuh, k_tree_far2: 1 sub, 6 fma, 7 mul; an f32x2 instruction does
# two), plus 2 SFU operations (rsqrt, ex2).  The float-float operator's far field (k_tree_far_ff): 171
# FP32 add/sub/mul/fma instructions per evaluation (difference 11, r^2 12, d.n 18, rsqrt by one Newton
# step 16, kappa r 8, the table exponential 29, the two charge combinations and accumulations 27 and 31,
# 1 + kappa r times E 11, r^-3 8; table indexing and loads not counted), 1 SFU operation.
OPS_FAR = 14
OPS_FAR_DF = 171
SFU_FAR = 2


def kernel_sources_hash():
    import hashlib
    h = hashlib.sha256()
    for rel in KERNEL_SOURCES:
        with open(os.path.join(ROOT, rel), "rb") as f:
            h.update(f.read())
    return h.hexdigest()[:16]


def traffic_for(key, h):
    """Measured DRAM bytes per launch of kernel `key`, when the record matches this workload and source."""
    if abs(h - TRAFFIC["h"]) > 1e-12 or TRAFFIC.get(key) is None:
        return None, None
    if TRAFFIC["sources"] != kernel_sources_hash():
        return None, f"{TRAFFIC['profile']} (stale: kernel sources changed since the capture)"
    return TRAFFIC[key], TRAFFIC["profile"]


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=3)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--h", type=float, default=0.05, help="grid spacing of the ellipsoid workload")
    ap.add_argument("--precision", default="fp32_refine", choices=["fp32_refine", "fp64"])
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--cpu-seconds", type=float, default=15.0, help="target CPU time of the baseline sample")
    ap.add_argument("--skip-e2e", action="store_true")
    ap.add_argument("--skip-fp64-check", action="store_true",
                    help="do not solve the workload in plain FP64 for the error_vs_fp64 object")
    ap.add_argument("--skip-serve", action="store_true", help="do not run the bounded serving object")
    ap.add_argument("--mode", default="solve", choices=["solve", "batch", "serve", "kernels", "tree", "map"],
                    help="solve: the default single-system line; batch: many molecules in one engine; "
                         "serve: continuous-batching server under Poisson arrivals; kernels: two FP32, two "
                         "float-float and two FP64 operator applications of the ellipsoid at --h (the profiling "
                         "case); tree: the solve step with the far-field treecode on the ellipsoid at --tree-h; "
                         "map: potential maps (psi_rxn at --map-points points) of the solved ellipsoid at --h")
    ap.add_argument("--map-points", type=int, default=200000, help="map mode: points of the potential map")
    ap.add_argument("--tree-h", type=float, default=0.025, help="tree mode: grid spacing (0.025: ~714k nodes)")
    ap.add_argument("--tree-tol", type=float, default=1e-10, help="tree mode: solve tolerance")
    ap.add_argument("--tree-direct", action="store_true",
                    help="tree mode: also time the direct-sum applications at the same size")
    ap.add_argument("--oracle-solves", action="store_true",
                    help="with --impl reference: time whole oracle solves (sphere h=0.25, ellipsoid h=0.2) and one "
                         "full oracle matvec of the 500-atom molecule on the host cores, one JSON line")
    ap.add_argument("--molecules", type=int, default=64, help="batch mode: molecules in the batch")
    ap.add_argument("--max-atoms", type=int, default=2000, help="batch/serve: largest molecule")
    ap.add_argument("--requests", type=int, default=1000, help="serve mode: requests per load level")
    ap.add_argument("--capacity-requests", type=int, default=200,
                    help="serve mode: requests of the saturated run that measures capacity")
    ap.add_argument("--loads", default="0.8", help="serve mode: offered load / measured capacity (comma list)")
    ap.add_argument("--pool", type=int, default=12, help="serve mode: distinct problems requests draw from")
    ap.add_argument("--slots", type=int, default=16, help="serve mode: server slots")
    ap.add_argument("--rate", type=float, default=None,
                    help="serve mode: one run at this arrival rate (requests/s) instead of the capacity run and loads")
    ap.add_argument("--step-quantum-ms", type=float, default=20.0,
                    help="serve: pair work of one system per engine step (longer applications run in parts; 0: whole)")
    ap.add_argument("--serve-requests", type=int, default=48, help="requests per run of the default line's serve object")
    ap.add_argument("--fp64-pool-only", action="store_true",
                    help="serve mode: only time the plain FP64 one-at-a-time path on every pool problem")
    ap.add_argument("--fp64-max-M", type=int, default=120000,
                    help="serve mode: pool problems up to this size are also solved in plain FP64 one at a time")
    return ap.parse_args()


def dist_init():
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl" if _cuda() else "gloo")
    return world, rank, local


def _cuda():
    import torch
    return torch.cuda.is_available()


def barrier(world):
    if world > 1:
        import torch.distributed as dist
        dist.barrier()


def max_over_ranks(v, world):
    if world <= 1:
        return v
    import torch
    import torch.distributed as dist
    t = torch.tensor([v], dtype=torch.float64, device="cuda" if _cuda() else "cpu")
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def sum_over_ranks(v, world):
    if world <= 1:
        return v
    import torch
    import torch.distributed as dist
    t = torch.tensor([v], dtype=torch.float64, device="cuda" if _cuda() else "cpu")
    dist.all_reduce(t, op=dist.ReduceOp.SUM)
    return float(t.item())


class ClockSampler:
    """nvidia-smi clocks and throttle reasons sampled every 200 ms during the timed region."""

    FIELDS = ("clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.hw_slowdown,"
              "clocks_event_reasons.hw_thermal_slowdown,clocks_event_reasons.sw_thermal_slowdown,"
              "clocks_event_reasons.sw_power_cap")

    def __init__(self, index: int):
        self.index = index
        self.samples = []
        self._stop = threading.Event()
        self._t = None

    def _run(self):
        while not self._stop.is_set():
            try:
                out = subprocess.run(["nvidia-smi", f"--id={self.index}", f"--query-gpu={self.FIELDS}",
                                      "--format=csv,noheader,nounits"], capture_output=True, text=True, timeout=5)
                if out.returncode == 0 and out.stdout.strip():
                    self.samples.append([v.strip() for v in out.stdout.strip().split(",")])
            except Exception:  # noqa: BLE001 - sampling is best effort
                pass
            self._stop.wait(0.2)

    def __enter__(self):
        self._t = threading.Thread(target=self._run, daemon=True)
        self._t.start()
        return self

    def __exit__(self, *a):
        self._stop.set()
        if self._t:
            self._t.join(timeout=10)

    def summary(self):
        if not self.samples:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["unsampled"]}
        sm = [float(s[0]) for s in self.samples if s[0].replace(".", "").isdigit()]
        mx = [float(s[1]) for s in self.samples if s[1].replace(".", "").isdigit()]
        reasons = set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for s in self.samples:
            for nm, v in zip(names, s[3:7]):
                if v.strip().lower() == "active":
                    reasons.add(nm)
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": max(mx) if mx else None,
                "reasons": sorted(reasons), "samples": len(self.samples),
                "power_w_max": max((float(s[2]) for s in self.samples if s[2].replace(".", "").isdigit()),
                                   default=None)}


def workload(h):
    import synthetic as syn
    prob = syn.ellipsoid_problem(h=h)
    return prob, {"workload": f"ellipsoid 4x3x2 A, 3 seeded charges, h={h:g} A, tube 2h, eps_in=1, eps_out=80, "
                              f"kappa=0.1257", "grid": list(prob.grid.n), "solver": None}


class OracleSample:
    """The oracle's FP64 punctured dense sum (Eqs. 2.14-2.15) on sampled target rows, host cores."""

    def __init__(self, prob, seconds, threads=None):
        from oracle import geometry, native
        import synthetic as syn
        if threads:
            native.set_threads(threads)
        self.cores = native.max_threads()
        self.prob = prob
        geo = geometry.tube_geometry(prob.grid.n, prob.grid.origin, prob.grid.h, prob.sdist, prob.tube)
        self.M = geo.M
        self.rng = np.random.Generator(np.random.PCG64(1))
        self.p = syn.random_density(self.M, seed=2)
        # calibrate the row count to about `seconds` of CPU time
        rows = np.sort(self.rng.choice(self.M, size=min(self.M, 32 * self.cores), replace=False))
        S = self._system(rows)
        t0 = time.perf_counter()
        S.punctured_sum(self.p, rows)
        rate = rows.size * self.M / max(time.perf_counter() - t0, 1e-6)
        n_rows = int(min(self.M, max(self.cores, rate * seconds / self.M)))
        self.rows = np.sort(self.rng.choice(self.M, size=n_rows, replace=False))
        self.S = self._system(self.rows)

    def _system(self, rows):
        from oracle.system import OracleSystem
        return OracleSystem.from_problem(self.prob, rows=rows,
                                         table_cache=os.path.join(ROOT, "oracle", "_build", "cache"))

    def run(self):
        t0 = time.perf_counter()
        self.S.punctured_sum(self.p, self.rows)
        dt = time.perf_counter() - t0
        pairs = self.rows.size * self.M
        return {"value": pairs / dt, "unit": "pair-interactions/s", "cores": self.cores, "kind": "oracle",
                "sample": f"FP64 punctured dense sum of {self.rows.size} sampled target rows x {self.M} sources "
                          f"({pairs:.3g} pairs, {dt:.1f} s) of the same workload"}


def cpu_baseline(prob, seconds, threads=None):
    return OracleSample(prob, seconds, threads).run()


def run_oracle_solves():
    """Whole FP64 oracle solves (setup, GMRES to 1e-10, energy) and one full oracle matvec, host cores."""
    import synthetic as syn
    from oracle import energy, native
    from oracle.system import OracleSystem
    cache = os.path.join(ROOT, "oracle", "_build", "cache")
    out = []
    for name, prob in (("sphere R=2, h=0.25", syn.sphere_problem(h=0.25)),
                       ("ellipsoid 4x3x2, h=0.2", syn.ellipsoid_problem(h=0.2))):
        t0 = time.perf_counter()
        S = OracleSystem.from_problem(prob, table_cache=cache)
        t1 = time.perf_counter()
        psi, dpsi, info = S.solve(tol=1e-10)
        G, _ = energy.polarization_energy(S, psi, dpsi)
        t2 = time.perf_counter()
        out.append({"workload": name, "M": S.M, "setup_s": t1 - t0, "solve_s": t2 - t1, "G_pol": G,
                    "iterations": int(info.get("iterations", -1)) if isinstance(info, dict) else None})
    prob = syn.molecule_problem(n_atoms=500, seed=0, h=0.5)
    S = OracleSystem.from_problem(prob, table_cache=cache)
    p = syn.random_density(S.M, seed=2)
    t0 = time.perf_counter()
    S.punctured_sum(p)
    dt = time.perf_counter() - t0
    out.append({"workload": "molecule 500 atoms, h=0.5: one full punctured sum", "M": S.M, "matvec_s": dt,
                "pairs_per_s": S.M * S.M / dt})
    print(json.dumps({"impl": "reference", "mode": "oracle_solves", "cores": native.max_threads(), "results": out}),
          flush=True)


def run_reference(args, world, rank):
    """The oracle as it stands, timed on the host cores, as the reference arm."""
    if rank != 0:
        return
    if args.oracle_solves:
        run_oracle_solves()
        return
    prob, cfg = workload(args.h)
    cfg = dict(cfg, **solver_config(args, world))
    sample = OracleSample(prob, seconds=max(2.0, min(args.cpu_seconds, 20.0)))
    steps = []
    res = None
    for it in range(args.warmup + args.steps):
        res = sample.run()
        if it >= args.warmup:
            steps.append(res["value"])
    value = statistics.median(steps)
    line = {"impl": "reference", "metric": "CTR-IBIM matvec pair-interactions/s", "value": value,
            "unit": "pair-interactions/s", "n_gpus": args.gpus, "steps": args.steps, "warmup": args.warmup,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
            "data": "synthetic", "config": cfg,
            "cpu_baseline": {"value": value, "unit": "pair-interactions/s", "cores": res["cores"], "kind": "oracle",
                             "sample": res["sample"]},
            "e2e": {"value": value, "unit": "pair-interactions/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


def run_batch(args, ctr):
    """Batched workload: molecules with log-uniform atom counts, h in {0.5, 0.35}, one engine."""
    import torch
    import synthetic as syn
    t0 = time.perf_counter()
    specs = syn.batch_specs(args.molecules, seed=0, max_atoms=args.max_atoms)
    probs = syn.molecules_parallel(specs)
    t_gen = time.perf_counter() - t0
    opts = [ctr.Options(tube_halfwidth=p.tube, precision=ctr.FP32_REFINE, tol=1e-10) for p in probs]

    def make():
        return [ctr.CtrIbim.from_problem(p, options=o) for p, o in zip(probs, opts)]

    systems = make()
    Ms = np.array([g.M for g in systems], dtype=np.float64)
    ctr.batch_solve(systems)                        # warm-up (and autotuning)
    torch.cuda.synchronize()
    launches0 = ctr.kernel_launches()
    t0 = time.perf_counter()
    out = ctr.batch_solve(systems)
    torch.cuda.synchronize()
    t_batch = time.perf_counter() - t0
    launches = ctr.kernel_launches() - launches0
    pairs = float(np.sum(Ms ** 2 * np.array([i.matvecs_fp32 + i.matvecs_fp64 for _, _, i in out])))
    # the same systems one after another (engine of one slot each)
    t0 = time.perf_counter()
    for g in systems:
        g.solve(device=True)
    torch.cuda.synchronize()
    t_seq = time.perf_counter() - t0
    shapes = {}
    for g in systems:
        t = g.pair_tuning(ctr.FP32_REFINE)
        key = f"block {t['block_targets']}, tile {t['tile']}, chunk {t['chunk']}, unroll {t['unroll']}"
        shapes[key] = shapes.get(key, 0) + 1
    line = {"metric": "CTR-IBIM batched pair-interactions/s", "value": pairs / t_batch, "unit": "pair-interactions/s",
            "n_gpus": 1, "steps": 1, "higher_is_better": True, "dtype": "f32 pairs + f64", "data": "synthetic",
            "config": {"workload": f"{len(probs)} random-walk SES molecules, atoms log-uniform in 20-{args.max_atoms}, "
                                   f"h in {{0.5, 0.35}}, tube 2h, FP32 pairs + float-float refinement, tol 1e-10",
                       "M_min": int(Ms.min()), "M_median": int(np.median(Ms)), "M_max": int(Ms.max()),
                       "sum_M2": float(np.sum(Ms ** 2)), "generation_s": t_gen},
            "batch_s": t_batch, "solves_per_s": len(probs) / t_batch, "sequential_s": t_seq,
            "speedup_vs_sequential": t_seq / t_batch, "all_converged": all(i.converged for _, _, i in out),
            "max_iterations": int(max(i.iterations for _, _, i in out)),
            "fp32_variants": shapes, "gpu_launches": int(launches)}
    for g in systems:
        g.close()
    print(json.dumps(line), flush=True)


def fp64_pool_times(ctr, pool, max_M):
    """The plain FP64 one-at-a-time GPU path on every pool problem of at most max_M nodes: energy and
    seconds per problem (None where skipped) and each problem's node count."""
    import torch
    Ms, G64, t = [], {}, {}
    for k, p in enumerate(pool):
        with ctr.CtrIbim.from_problem(p) as G:
            Ms.append(G.M)
        if G.M > max_M:
            continue
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        with ctr.CtrIbim.from_problem(p, options=ctr.Options(tube_halfwidth=p.tube, precision=ctr.FP64,
                                                             tol=SOLVE_TOL)) as G:
            psi, dpsi, _ = G.solve(device=True)
            G64[k] = G.energy(psi, dpsi)[0]
        torch.cuda.synchronize()
        t[k] = time.perf_counter() - t0
    return Ms, G64, t


def serve_experiment(ctr, pool, n_requests, loads, slots, fp64_max_M, seed=11, cap_requests=None, quantum_ms=20.0,
                     rate=None):
    """Continuous-batching server over a pool of problems: capacity with every request submitted at once,
    then Poisson arrivals at each fraction of it; per load solves/s and p50/p99 latency (submission to
    result).  Served energies are compared with the plain FP64 one-at-a-time GPU path on every pool problem
    of at most fp64_max_M nodes (the fixed sample); requests pick pool problems uniformly, so with every
    problem in the sample 1 / (mean FP64 solve time) is that path's rate on the same mix."""
    import threading as th
    import torch

    def run_load(rate, n, sd):
        arrivals = None
        if rate is not None:
            gaps = np.random.Generator(np.random.PCG64(sd)).exponential(1.0 / rate, size=n)
            arrivals = np.cumsum(gaps) - gaps[0]
        picks = np.random.Generator(np.random.PCG64(sd + 1)).integers(0, len(pool), size=n)
        with ctr.Server(max_slots=slots, step_quantum_ms=quantum_ms) as sv:
            tickets = [None] * n
            t0 = time.perf_counter()

            def submitter():
                for i in range(n):
                    if arrivals is not None:
                        dt = arrivals[i] - (time.perf_counter() - t0)
                        if dt > 0:
                            time.sleep(dt)
                    p = pool[picks[i]]
                    tickets[i] = sv.submit_problem(p, ctr.Options(tube_halfwidth=p.tube, precision=ctr.FP32_REFINE,
                                                                  tol=SOLVE_TOL))

            thr = th.Thread(target=submitter)
            thr.start()
            thr.join()
            res = [sv.wait(t, timeout=3600) for t in tickets]
            st = sv.stats()
        lat = np.array([r.latency for r in res])
        t_first = min(r.t_submit for r in res)
        t_last = max(r.t_done for r in res)
        statuses = {}
        for r in res:
            statuses[str(r.status)] = statuses.get(str(r.status), 0) + 1
        failed = [{"pick": int(picks[i]), "status": res[i].status, "M": res[i].M,
                   "iterations": res[i].info.iterations} for i in range(n) if res[i].status != 0][:8]
        return {"requests": n, "solves_per_s": n / (t_last - t_first), "p50_s": float(np.percentile(lat, 50)),
                "p99_s": float(np.percentile(lat, 99)), "mean_s": float(lat.mean()),
                "all_ok": all(r.status == 0 for r in res), "statuses": statuses, "failed": failed,
                "peak_slots": st["peak_slots"],
                "peak_used_GB": st["peak_used_bytes"] / 1e9, "steps": st["steps"],
                "energies": [(int(picks[i]), res[i].G_pol) for i in range(n)]}

    run_load(None, min(len(pool), 4), 7)              # warm-up (autotuning, first touch)
    if rate is not None:   # one run at a fixed arrival rate (policies compared on the same arrivals)
        cap, capacity = None, None
        levels = {f"rate {rate:g}/s": run_load(rate, n_requests, seed + 2)}
    else:
        cap = run_load(None, cap_requests or n_requests, seed)   # saturated: everything submitted at once
        capacity = cap["solves_per_s"]
        levels = {f"{f:g}": run_load(f * capacity, n_requests, seed + 2) for f in loads}
    # the plain FP64 one-at-a-time GPU path on the sample
    Ms, G64, t64 = fp64_pool_times(ctr, pool, fp64_max_M)
    runs = list(levels.values()) + ([cap] if cap else [])
    errs = [abs(e / G64[k] - 1) for lv in runs for k, e in lv["energies"] if k in G64]
    for lv in runs:
        lv.pop("energies")
    n64 = len(t64)
    return {"capacity_solves_per_s": capacity, "saturated": cap, "levels": levels,
            "M_min": int(min(Ms)), "M_max": int(max(Ms)), "pool": len(pool), "slots": slots,
            "step_quantum_ms": quantum_ms,
            "fp64_solves_per_s": n64 / sum(t64.values()) if n64 else None,
            "fp64_same_mix": n64 == len(pool),
            "fp64_sample": f"{n64} of the {len(pool)} pool problems (those with M <= {fp64_max_M}), one at a time",
            "fp64_s_per_problem": {int(Ms[k]): round(v, 3) for k, v in t64.items()},
            "max_energy_err": float(max(errs)) if errs else None, "checked_requests": len(errs)}


def c5_pool(n_mol, n_sph, n_ell, max_atoms, seed=0):
    """Problems of the serving workload: SES molecules of the batched distribution (atoms log-uniform,
    h in {0.5, 0.35}), spheres of 5k-400k nodes with +-1 charges, ellipsoids at h 0.2 ... 0.035."""
    import synthetic as syn
    rng = np.random.Generator(np.random.PCG64(seed))
    pool = list(syn.molecules_parallel(syn.batch_specs(n_mol, seed=100 + seed, max_atoms=max_atoms))) if n_mol else []
    for _ in range(n_sph):
        pool.append(syn.sphere_with_nodes(int(np.exp(rng.uniform(np.log(5e3), np.log(4e5)))),
                                          q=float(rng.choice([-1.0, 1.0]))))
    for k, hh in enumerate([0.2, 0.1, 0.05, 0.035][:n_ell]):
        pool.append(syn.ellipsoid_problem(h=hh, seed=k))
    return pool


def run_serve_bounded(ctr, args):
    """The serving object of the default line: a pool of six problems of up to ~45k nodes (two molecules,
    two spheres, two ellipsoids), 48 requests at 0.8 of the measured capacity."""
    import synthetic as syn
    rng = np.random.Generator(np.random.PCG64(5))
    pool = list(syn.molecules_parallel([(60, 201, 0.5), (150, 202, 0.35)]))
    for M in (6000, 30000):
        pool.append(syn.sphere_with_nodes(M, q=float(rng.choice([-1.0, 1.0]))))
    pool += [syn.ellipsoid_problem(h=0.2, seed=1), syn.ellipsoid_problem(h=0.1, seed=2)]
    out = serve_experiment(ctr, pool, n_requests=args.serve_requests, loads=[0.8], slots=args.slots,
                           fp64_max_M=10 ** 9, quantum_ms=args.step_quantum_ms)
    out["workload"] = (f"{args.serve_requests} requests per run drawn from a pool of {len(pool)} problems (SES "
                       f"molecules of 60 and 150 atoms at h 0.5 / 0.35, spheres of 6k and 30k nodes, ellipsoids at "
                       f"h 0.2 / 0.1), FP32 pairs + float-float refinement to {SOLVE_TOL:g}; capacity with all "
                       f"requests submitted at once, then Poisson arrivals at 0.8 of it")
    return out


def run_serve(args, ctr):
    """Serving workload (C5): Poisson arrivals at fractions of the measured capacity; latency and throughput."""
    pool = c5_pool(max(1, args.pool // 3), max(1, args.pool // 3), max(1, args.pool - 2 * (args.pool // 3)),
                   args.max_atoms)
    if args.fp64_pool_only:   # only the plain FP64 one-at-a-time path on the whole pool (the same-mix rate)
        Ms, G64, t64 = fp64_pool_times(ctr, pool, 10 ** 12)
        print(json.dumps({"mode": "serve_fp64_pool", "pool": len(pool), "fp64_s_per_problem":
                          {int(Ms[k]): round(v, 3) for k, v in t64.items()},
                          "fp64_solves_per_s_same_mix": len(t64) / sum(t64.values()),
                          "G_pol": {int(Ms[k]): v for k, v in G64.items()}}), flush=True)
        return
    out = serve_experiment(ctr, pool, n_requests=args.requests, loads=[float(v) for v in args.loads.split(",") if v],
                           slots=args.slots, fp64_max_M=args.fp64_max_M, cap_requests=args.capacity_requests,
                           quantum_ms=args.step_quantum_ms, rate=args.rate)
    top = list(out["levels"])[-1] if args.rate is not None else max(out["levels"], key=float)   # highest load
    line = {"metric": "CTR-IBIM served solves/s", "value": out["levels"][top]["solves_per_s"],
            "unit": "solves/s", "n_gpus": 1, "higher_is_better": True, "dtype": "f32 pairs + f64",
            "data": "synthetic",
            "config": {"workload": f"{args.requests} requests per load level, Poisson arrivals, drawn from a pool of "
                                   f"{len(pool)} problems (SES molecules, spheres, ellipsoids), FP32 pairs + "
                                   f"float-float refinement to {SOLVE_TOL:g}", "M_min": out["M_min"],
                       "M_max": out["M_max"], "slots": args.slots, "step_quantum_ms": args.step_quantum_ms}}
    line.update(out)
    print(json.dumps(line), flush=True)


def run_kernels(args, ctr):
    """Two FP32, two float-float and two FP64 operator applications (the first of each warms up), timed."""
    import torch
    prob, cfg = workload(args.h)
    stream = torch.cuda.current_stream()
    out = {"mode": "kernels", "config": cfg}
    with ctr.CtrIbim.from_problem(prob) as G:
        x = torch.tensor(np.random.default_rng(0).uniform(-1, 1, 2 * G.M), device="cuda")
        y = torch.empty_like(x)
        out["M"] = G.M
        for pr, name in ((ctr.FP32_REFINE, "fp32"), (ctr.DF64, "df64"), (ctr.FP64, "fp64")):
            G.matvec(x, pr, out=y)
            e0 = torch.cuda.Event(enable_timing=True)
            e1 = torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            G.matvec(x, pr, out=y)
            e1.record(stream)
            torch.cuda.synchronize()
            out[name] = dict(G.pair_schedule(pr), t_matvec_ms=e0.elapsed_time(e1))
    print(json.dumps(out), flush=True)


# Potential map (Eq. 2.31 at arbitrary points): FMA-pipe lane operations per (point, node) pair of the FP32
# kernel counted from its source (potential.cu, MapFp32x2: 3 sub, 3 for r^2, 1 r, 2 for E's argument and
# E1, 3 for d.n, 2 for 1/r^3, 1 for the ratio term, 3 for the first accumulation, 2 for the second; an
# f32x2 instruction does two), plus 2 SFU operations (rsqrt, ex2).
OPS_MAP = 22


def run_map(args, ctr):
    """psi_rxn of the solved default workload on a cloud of points inside and outside the ellipsoid, in the
    three arithmetics: pair evaluations/s and the fraction of the FMA-pipe peak (FP32)."""
    import torch
    prob, cfg = workload(args.h)
    rng = np.random.Generator(np.random.PCG64(17))
    g = prob.grid
    lo = np.asarray(g.origin)
    hi = lo + g.h * (np.asarray(g.n) - 1)
    pts = rng.uniform(lo, hi, size=(args.map_points, 3))
    stream = torch.cuda.current_stream()
    out = {"mode": "map", "config": dict(cfg, points=args.map_points,
                                         points_recipe="uniform in the grid box (seed 17), both sides of the surface")}
    with ctr.CtrIbim.from_problem(prob, options=ctr.Options(tube_halfwidth=prob.tube, precision=ctr.FP32_REFINE)) as G:
        psi, dpsi, _ = G.solve(device=True)
        z = torch.tensor(pts, device="cuda")
        M = G.M
        sms = torch.cuda.get_device_properties(torch.cuda.current_device()).multi_processor_count
        peak = sms * 128 * 2070e6
        res = {}
        for prec, name, reps in ((ctr.FP32_REFINE, "fp32", 5), (ctr.DF64, "df64", 2), (ctr.FP64, "fp64", 1)):
            G.potential_map(psi, dpsi, z, prec)
            e0 = torch.cuda.Event(enable_timing=True)
            e1 = torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            for _ in range(reps):
                G.potential_map(psi, dpsi, z, prec)
            e1.record(stream)
            torch.cuda.synchronize()
            t = e0.elapsed_time(e1) * 1e-3 / reps
            res[name] = {"t_ms": t * 1e3, "pairs_per_s": args.map_points * M / t}
        res["fp32"].update({"achieved": OPS_MAP * args.map_points * M / res["fp32"]["t_ms"] * 1e3, "peak": peak,
                            "unit": "FP32-pipe lane ops/s", "frac": OPS_MAP * args.map_points * M /
                            res["fp32"]["t_ms"] * 1e3 / peak,
                            "basis": f"{OPS_MAP} FMA-pipe lane ops per (point, node) pair x {args.map_points} x {M}; "
                                     f"peak {sms} SMs x 128 lanes x 2070 MHz"})
        out.update(M=M, maps=res)
    print(json.dumps(out), flush=True)


def run_tree(args, ctr, world):
    """The solve step (setup, FP32-refined GMRES, energy) with the treecode far field, timed like the default
    line; value counts M^2 per operator application, as the direct sum would evaluate."""
    import torch
    local = torch.cuda.current_device()
    prob, cfg = workload(args.tree_h)
    opts = ctr.Options(tube_halfwidth=prob.tube, precision=ctr.FP32_REFINE, tol=args.tree_tol,
                       farfield=ctr.FARFIELD_TREECODE)
    cfg["solver"] = f"fp32_refine, GMRES restart {opts.restart}, tol {opts.tol:g}"
    cfg["farfield"] = (f"treecode degree {opts.tree_degree}, theta {opts.tree_theta}, leaf {opts.tree_leaf}; "
                       f"value counts M^2 per operator application (the direct sum's pairs)")
    cfg["l2"] = "256 MiB buffer written between timed steps (L2 flush, outside the step events)"
    cfg["parallelism"] = f"replicas x{world}"
    stream = torch.cuda.current_stream()
    sd_dev = torch.tensor(prob.sdist, dtype=torch.float64, device="cuda")
    flush = torch.empty(256 * 2 ** 20 // 4, dtype=torch.float32, device="cuda")

    def step():
        with ctr.CtrIbim.from_problem(prob, options=opts, sdist=sd_dev) as G:
            psi, dpsi, info = G.solve(device=True)
            Gp, _ = G.energy(psi, dpsi)
            return G.M, info, Gp

    for _ in range(args.warmup):
        M, info, Gp = step()
    torch.cuda.synchronize()
    ev, infos, pairs = [], [], 0.0
    launches0 = ctr.kernel_launches()
    with ClockSampler(local) as clk:
        for _ in range(args.steps):
            flush.fill_(1.0)
            e0 = torch.cuda.Event(enable_timing=True)
            e1 = torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            M, info, Gp = step()
            e1.record(stream)
            ev.append((e0, e1))
            infos.append(info)
            pairs += float(M) ** 2 * (info.matvecs_fp32 + info.matvecs_fp64)
        torch.cuda.synchronize()
    launches = ctr.kernel_launches() - launches0
    t_dev = sum(a.elapsed_time(b) for a, b in ev) * 1e-3
    value = pairs / t_dev
    # phases of one application per arithmetic, the treecode's work counts, unit-count peaks
    with ctr.CtrIbim.from_problem(prob, options=opts, sdist=sd_dev) as G:
        ph = {pr: G.time_operator(pr, reps=3) for pr in (ctr.FP32_REFINE, ctr.DF64)}
        ff = {pr: G.farfield_info(pr) for pr in (ctr.FP32_REFINE, ctr.DF64)}
        Mk = G.M
    direct = None
    if args.tree_direct:
        with ctr.CtrIbim.from_problem(prob, options=ctr.Options(tube_halfwidth=prob.tube), sdist=sd_dev) as D:
            direct = {"fp32_ms": D.time_operator(ctr.FP32_REFINE, reps=1)["pairs_ms"],
                      "df64_ms": D.time_operator(ctr.DF64, reps=1)["pairs_ms"]}
    probes = Probes()
    rate_ffma = probes.rate(0)
    rate_ex2 = probes.rate(2)
    rate_rsq = probes.rate(3)
    sms = torch.cuda.get_device_properties(local).multi_processor_count
    f_max = (clk.summary().get("sm_max_mhz") or 2070.0) * 1e6
    rate_units = sms * 128 * f_max
    sfu_evals = 1.0 / (1.0 / rate_ex2 + 1.0 / rate_rsq) if rate_ex2 and rate_rsq else None
    far_peak = min(rate_units / OPS_FAR, sfu_evals) if sfu_evals else rate_units / OPS_FAR
    i_last = infos[-1]
    n_app = {ctr.FP32_REFINE: i_last.matvecs_fp32, ctr.DF64: i_last.matvecs_fp64}
    step_s = t_dev / args.steps
    kern = []
    for pr, tag, ops in ((ctr.FP32_REFINE, "fp32", OPS_FP32["one"]), (ctr.DF64, "df64", OPS_DF64["one"])):
        near, far = ff[pr]["near_pairs"], ff[pr]["far_evaluations"]
        t_near, t_far = ph[pr]["pairs_ms"] * 1e-3, ph[pr]["far_ms"] * 1e-3
        kern.append({"bound": "alu", "kernel": f"sched_kernel<{'Fp32x2' if tag == 'fp32' else 'Df64'}Policy> "
                                               f"(treecode direct part, {tag})",
                     "achieved": near / t_near, "peak": rate_units / ops, "unit": "pair-interactions/s",
                     "frac": near / t_near / (rate_units / ops), "traffic": None,
                     "peak_basis": f"{sms} SMs x 128 FP32 lanes x {f_max / 1e6:.0f} MHz / {ops} lane ops per "
                                   f"one-sided pair; measured FFMA probe {rate_ffma:.4g}/s",
                     "t_ms": t_near * 1e3, "pairs": near, "step_share": n_app[pr] * t_near / step_s})
        if tag == "fp32":
            fname, fpeak = "k_tree_mom + k_tree_momred + k_tree_far2<2, 256> (treecode far field, FP32 charges)", far_peak
            fbasis = (f"min({sms} SMs x 128 FP32 lanes x {f_max / 1e6:.0f} MHz / {OPS_FAR} lane ops, SFU: "
                      f"1/(1/ex2 + 1/rsqrt) with the measured probes {rate_ex2:.4g}/s, {rate_rsq:.4g}/s) per proxy "
                      f"evaluation")
        else:
            fname = "k_tree_mom<double> + k_tree_momred<double> + k_tree_far_ff<2, 128> (treecode far field, float-float)"
            fpeak = rate_units / OPS_FAR_DF
            fbasis = (f"{sms} SMs x 128 FP32 lanes x {f_max / 1e6:.0f} MHz / {OPS_FAR_DF} FP32-pipe ops per "
                      f"float-float proxy evaluation")
        kern.append({"bound": "alu", "kernel": fname,
                     "achieved": far / t_far if t_far > 0 else None, "peak": fpeak,
                     "unit": "proxy evaluations/s",
                     "frac": far / t_far / fpeak if t_far > 0 else None, "traffic": None, "peak_basis": fbasis,
                     "t_ms": t_far * 1e3, "evaluations": far, "step_share": n_app[pr] * t_far / step_s})
    kern.sort(key=lambda k: -k["step_share"])
    e2e = None
    if not args.skip_e2e:
        h2d = prob.sdist.nbytes + prob.charge_xyz.nbytes + prob.charge_q.nbytes
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        with ctr.CtrIbim.from_problem(prob, options=opts) as G:
            psi, dpsi, info_e = G.solve(device=False)
            G.energy(psi, dpsi)
            e2e_pairs = float(G.M) ** 2 * (info_e.matvecs_fp32 + info_e.matvecs_fp64)
            d2h = psi.nbytes + dpsi.nbytes + 8
        torch.cuda.synchronize()
        e2e = {"value": e2e_pairs / (time.perf_counter() - t0), "unit": "pair-interactions/s",
               "h2d_bytes_per_step": int(h2d), "d2h_bytes_per_step": int(d2h)}
    cpu = None if args.no_cpu_baseline else cpu_baseline(prob, args.cpu_seconds)
    line = {
        "mode": "tree", "metric": "CTR-IBIM matvec pair-interactions/s", "value": value,
        "unit": "pair-interactions/s", "n_gpus": world, "steps": args.steps, "warmup": args.warmup,
        "ms_per_step": step_s * 1e3, "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
        "dtype": "f32 pairs + f64", "data": "synthetic",
        "config": dict(cfg, M=int(Mk), iterations=int(i_last.iterations), refinements=int(i_last.refinements),
                       matvecs_fp32=int(i_last.matvecs_fp32), matvecs_fp64=int(i_last.matvecs_fp64),
                       residual=i_last.residual, G_pol=Gp),
        "phases_ms": {"fp32": ph[ctr.FP32_REFINE], "df64": ph[ctr.DF64]},
        "farfield": {"fp32": {k: v for k, v in ff[ctr.FP32_REFINE].items() if k != "perm"},
                     "df64": {k: v for k, v in ff[ctr.DF64].items() if k != "perm"}},
        "direct_ms": direct,
        "roofline": kern[0], "roofline_second": kern[1], "kernels": kern,
        "probes": {"ffma": rate_ffma, "ex2": rate_ex2, "rsqrt": rate_rsq},
        "clocks": clk.summary(), "e2e": e2e, "gpu_launches": int(launches), "cpu_baseline": cpu,
    }
    print(json.dumps(line), flush=True)


def main():
    args = parse()
    world, rank, local = dist_init()
    if args.impl == "reference":
        run_reference(args, world, rank)
        return
    if args.mode in ("batch", "serve", "kernels", "tree", "map"):
        import torch
        torch.cuda.set_device(local)
        import paper_2210_03699_gb300 as ctr
        if rank == 0:
            if args.mode == "tree":
                run_tree(args, ctr, 1)
            else:
                {"batch": run_batch, "serve": run_serve, "kernels": run_kernels, "map": run_map}[args.mode](args, ctr)
        return
    import torch
    torch.cuda.set_device(local)
    import paper_2210_03699_gb300 as ctr

    prob, cfg = workload(args.h)
    prec = ctr.FP32_REFINE if args.precision == "fp32_refine" else ctr.FP64
    opts = ctr.Options(tube_halfwidth=prob.tube, precision=prec, tol=SOLVE_TOL, restart=RESTART,
                       inner_tol=INNER_TOL)
    cfg = dict(cfg, **solver_config(args, world))
    stream = torch.cuda.current_stream()
    sd_dev = torch.tensor(prob.sdist, dtype=torch.float64, device="cuda")
    flush = torch.empty(256 * 2 ** 20 // 4, dtype=torch.float32, device="cuda")

    def step():
        with ctr.CtrIbim.from_problem(prob, options=opts, sdist=sd_dev) as G:
            psi, dpsi, info = G.solve(device=True)
            Gp, _ = G.energy(psi, dpsi)
            return G.M, info, Gp, psi, dpsi

    for _ in range(args.warmup):
        M, info, Gp, _, _ = step()
    torch.cuda.synchronize()
    barrier(world)
    ev = []
    pairs = 0.0
    infos = []
    launches0 = ctr.kernel_launches()
    with ClockSampler(local) as clk:
        t_wall0 = time.perf_counter()
        for _ in range(args.steps):
            flush.fill_(1.0)
            e0 = torch.cuda.Event(enable_timing=True)
            e1 = torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            M, info, Gp, psi, dpsi = step()
            e1.record(stream)
            ev.append((e0, e1))
            infos.append(info)
            pairs += float(M) ** 2 * (info.matvecs_fp32 + info.matvecs_fp64)
        torch.cuda.synchronize()
        t_wall = time.perf_counter() - t_wall0
    launches = ctr.kernel_launches() - launches0
    barrier(world)
    t_dev = sum(a.elapsed_time(b) for a, b in ev) * 1e-3
    t_max = max_over_ranks(t_dev, world)
    pairs_all = sum_over_ranks(pairs, world)
    value = pairs_all / t_max
    steps_all = sum_over_ranks(float(args.steps), world)

    # kernel-level rooflines: one operator application per arithmetic, timed on the stream
    t_mv, sched = {}, {}
    with ctr.CtrIbim.from_problem(prob, options=opts, sdist=sd_dev) as G:
        x = torch.tensor(np.random.default_rng(0).uniform(-1, 1, 2 * G.M), device="cuda")
        y = torch.empty_like(x)
        timed = ((ctr.FP32_REFINE, 5), (ctr.DF64, 2)) if prec == ctr.FP32_REFINE else ((ctr.FP64, 1),)
        for pr, reps in timed:
            G.matvec(x, pr, out=y)
            e0 = torch.cuda.Event(enable_timing=True)
            e1 = torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            for _ in range(reps):
                G.matvec(x, pr, out=y)
            e1.record(stream)
            torch.cuda.synchronize()
            t_mv[pr] = e0.elapsed_time(e1) * 1e-3 / reps
            sched[pr] = G.pair_schedule(pr)
            sched[pr]["shape"] = G.pair_tuning(pr)
        Mk = G.M
        # accuracy of the timed step's result: the residual recomputed with the float-float operator
        g = torch.empty(2 * Mk, dtype=torch.float64, device="cuda")
        ctr.lib.ctr_ibim_rhs(G._h, ctypes.c_void_p(g.data_ptr()), 1)
        xs = torch.cat([psi, dpsi])
        r_true = float(torch.linalg.vector_norm(g - G.matvec(xs, ctr.DF64)) / torch.linalg.vector_norm(g))
    probes = Probes()
    rate_ffma = probes.rate(0)
    rate_ex2 = probes.rate(2)
    rate_dfma = probes.rate(4)
    # FMA-pipe lane operations per second from unit counts and clocks: SMs x 128 FP32 lanes x the SM clock
    # ceiling (sampled by nvidia-smi; 2070 MHz when unavailable).  The FFMA probe's measured rate is reported
    # beside it.
    sms = torch.cuda.get_device_properties(local).multi_processor_count
    f_max = (clk.summary().get("sm_max_mhz") or 2070.0) * 1e6
    rate_units = sms * 128 * f_max
    i_last = infos[-1]
    step_s = t_max / args.steps

    def roof(pr, ops, name, key, n_app, rate=None, what="FP32"):
        sc = sched[pr]
        peak = rate or rate_units
        alg = ALG_OPS * Mk * Mk / t_mv[pr]
        n_exec = ops["one"] * sc["one_sided_pairs"] + ops["sym"] * sc["symmetric_pairs"]
        traffic, tsrc = traffic_for(key, args.h)
        return {"bound": "alu", "kernel": name, "achieved": alg, "peak": peak,
                "unit": f"{what}-pipe lane ops/s", "frac": alg / peak, "traffic": traffic,
                "traffic_source": tsrc,
                "achieved_basis": f"algorithmic: {ALG_OPS} {what}-pipe lane ops per pair interaction x M^2 = "
                                  f"{Mk}^2 interactions per launch / the launch's CUDA-event time",
                "peak_basis": (f"{sms} SMs x 128 FP32 lanes x {f_max / 1e6:.0f} MHz = {rate_units:.4g} lane ops/s "
                               f"(unit counts and clocks); measured FFMA probe {rate_ffma:.4g}/s") if rate is None
                else f"measured DFMA probe {rate:.4g}/s",
                "pairs_per_s": Mk * Mk / t_mv[pr],
                "frac_executed": n_exec / t_mv[pr] / peak,
                "executed_basis": f"lane ops the schedule executes: {ops['one']} per one-sided and {ops['sym']} "
                                  f"per symmetric pair evaluation (both orientations)",
                "t_matvec_ms": t_mv[pr] * 1e3, "one_sided_pairs": sc["one_sided_pairs"],
                "symmetric_pairs": sc["symmetric_pairs"], "items": sc["items"],
                "partial_bytes": sc["partial_bytes"], "kernel_shape": sc["shape"], "applications_per_step": n_app,
                "step_share": n_app * t_mv[pr] / step_s}

    if prec == ctr.FP32_REFINE:
        r32 = roof(ctr.FP32_REFINE, OPS_FP32, "sched_kernel<Fp32x2Policy> (packed FP32 pair sum: inner GMRES and "
                   "residual updates)", "fp32", i_last.matvecs_fp32)
        rdf = roof(ctr.DF64, OPS_DF64, "sched_kernel<Df64Policy> (float-float pair sum, refinement residual)",
                   "df64", i_last.matvecs_fp64)
        dominant, other = (rdf, r32) if rdf["step_share"] >= r32["step_share"] else (r32, rdf)
        dominant = dict(dominant, ex2_rate=rate_ex2, dfma_rate=rate_dfma)
    else:   # plain FP64 solves: every application is the FP64 schedule, bound by the DFMA pipe
        dominant = roof(ctr.FP64, OPS_FP64, "sched_kernel<Fp64Policy> (FP64 pair sum)", "fp64",
                        i_last.matvecs_fp64, rate=rate_dfma, what="FP64")
        other = None

    # the same workload through the public API with host buffers
    e2e = None
    if not args.skip_e2e:
        h2d = prob.sdist.nbytes + prob.charge_xyz.nbytes + prob.charge_q.nbytes
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        e2e_pairs = 0.0
        for _ in range(max(1, args.steps)):
            with ctr.CtrIbim.from_problem(prob, options=opts) as G:
                psi_h, dpsi_h, info_h = G.solve(device=False)
                Gh, _ = G.energy(psi_h, dpsi_h)
                e2e_pairs += float(G.M) ** 2 * (info_h.matvecs_fp32 + info_h.matvecs_fp64)
                d2h = psi_h.nbytes + dpsi_h.nbytes + 8
        torch.cuda.synchronize()
        t_e2e = max_over_ranks(time.perf_counter() - t0, world)
        e2e = {"value": sum_over_ranks(e2e_pairs, world) / t_e2e, "unit": "pair-interactions/s",
               "h2d_bytes_per_step": int(h2d), "d2h_bytes_per_step": int(d2h),
               "solves_per_s": sum_over_ranks(float(max(1, args.steps)), world) / t_e2e}

    # the error of the timed result against the plain FP64 GPU solve of the same system (once, untimed)
    accuracy = None
    if rank == 0 and prec == ctr.FP32_REFINE and not args.skip_fp64_check:
        accuracy = fp64_check(ctr, prob, sd_dev, psi, dpsi, Gp, opts)

    serve = None
    if rank == 0 and world == 1 and not args.skip_serve:
        serve = run_serve_bounded(ctr, args)

    cpu = None
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        cpu = cpu_baseline(prob, args.cpu_seconds)

    if rank == 0:
        i0 = infos[-1]
        line = {
            "metric": "CTR-IBIM matvec pair-interactions/s", "value": value, "unit": "pair-interactions/s",
            "n_gpus": world, "steps": args.steps, "warmup": args.warmup, "ms_per_step": t_max / args.steps * 1e3,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
            "dtype": "f32 pairs + f64" if prec == ctr.FP32_REFINE else "f64", "data": "synthetic",
            "config": cfg,
            "solves_per_s": steps_all / t_max,
            "solve": {"M": int(M), "unknowns": int(2 * M), "iterations": int(i0.iterations),
                      "refinements": int(i0.refinements), "matvecs_fp32": int(i0.matvecs_fp32),
                      "matvecs_fp64": int(i0.matvecs_fp64), "residual": i0.residual,
                      "residual_recomputed_df64": r_true, "G_pol": Gp},
            "error_vs_fp64": accuracy,
            "roofline": dominant,
            "roofline_second": other,
            "clocks": clk.summary(),
            "e2e": e2e,
            "gpu_launches": int(launches),
            "wall_s": t_wall,
            "cpu_baseline": cpu,
            "serve": serve,
        }
        print(json.dumps(line), flush=True)
    if world > 1:
        import torch.distributed as dist
        dist.destroy_process_group()


def solver_config(args, world):
    """The static description of the timed solve (the same keys in both arms of the benchmark)."""
    if args.precision == "fp32_refine":
        solver = (f"fp32_refine: FP32 pairs in GMRES(restart {RESTART}, inner tol {INNER_TOL:g}), "
                  f"refinement to tol {SOLVE_TOL:g}; residual arithmetic float-float, first residual g - A x, "
                  f"later ones updated r - A d with the FP32 operator")
        residual = "float-float"
        mode = "update"
    else:
        solver = f"fp64, GMRES restart {RESTART}, tol {SOLVE_TOL:g}"
        residual = "fp64"
        mode = "full"
    return {"solver": solver, "residual": residual, "residual_mode": mode,
            "l2": "256 MiB buffer written between timed steps (L2 flush, outside the step events)",
            "parallelism": f"replicas x{world}"}


def fp64_check(ctr, prob, sd_dev, psi, dpsi, Gp, opts):
    """Plain FP64 GPU solve of the same system to the same tolerance; relative errors of the timed result."""
    import torch
    t0 = time.perf_counter()
    with ctr.CtrIbim.from_problem(prob, options=ctr.Options(tube_halfwidth=prob.tube, precision=ctr.FP64,
                                                            tol=opts.tol), sdist=sd_dev) as G:
        p64, d64, info = G.solve(device=True)
        G64, _ = G.energy(p64, d64)
    torch.cuda.synchronize()
    t = time.perf_counter() - t0

    def rel(a, b):
        return float(torch.max(torch.abs(a - b)) / torch.max(torch.abs(b)))

    return {"reference": f"plain FP64 GPU solve of the same system (CTR_FP64 pairs, GMRES to {opts.tol:g}), once",
            "G_pol_rel": abs(Gp / G64 - 1), "psi_rel_max": rel(psi, p64), "dpsi_rel_max": rel(dpsi, d64),
            "G_pol_fp64": G64, "fp64_iterations": int(info.iterations), "fp64_solve_s": t,
            "fp64_solves_per_s": 1.0 / t}


class Probes:
    """The arithmetic-throughput probes (libctr_probe.so, built beside the solver library): rates of
    dependent FFMA, f32x2 FMA, ex2, rsqrt and DFMA chains on every SM."""

    def __init__(self):
        from paper_2210_03699_gb300 import build
        self.lib = ctypes.CDLL(build.PROBE_LIB)
        self.lib.ctr_probe_rate.restype = ctypes.c_int
        self.lib.ctr_probe_rate.argtypes = [ctypes.c_int, ctypes.c_int64, ctypes.POINTER(ctypes.c_double),
                                            ctypes.POINTER(ctypes.c_double)]

    def rate(self, kind, iters=20000):
        r = ctypes.c_double()
        t = ctypes.c_double()
        st = self.lib.ctr_probe_rate(kind, iters, ctypes.byref(r), ctypes.byref(t))
        return float(r.value) if st == 0 else None


if __name__ == "__main__":
    main()
