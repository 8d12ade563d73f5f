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

# FP32-pipe lane operations per pair evaluation, counted from the kernel source (see the design notes):
# one-sided evaluations (one orientation) and symmetric ones (both orientations, with the share of the
# in-warp transposed sums), for the packed FP32 and the float-float pair arithmetics (a packed f32x2
# instruction counts as two lane operations, the FMA pipe's throughput being the same either way).
# SFU work (rsqrt, ex2) and shared-memory loads are not counted.
OPS_FP32 = {"one": 41, "sym": 50}
OPS_DF64 = {"one": 507, "sym": 501}
# FP64 pipe lane operations per pair evaluation of the FP64 schedule (CUDA's exp and rsqrt included): the
# ncu count sm__inst_executed_pipe_fp64 x 32 / evaluations over one launch at h = 0.1 (69); its peak is the
# measured DFMA probe rate, there being no FP64 unit count to go by.
OPS_FP64 = {"one": 69, "sym": 69}
# DRAM bytes (read + write) per launch of the schedule kernels at the default workload (h = 0.05), from one
# ncu capture (profiles/dram_traffic_sched_kernels_ellipsoid_h0.05.txt); None at any other size, or once
# the kernels change.
TRAFFIC_H005 = {"fp32": 2.286e8, "df64": 1.0483e9, "fp64": None}
# Treecode far field (FP32 charges): FMA-pipe lane operations per proxy evaluation counted from the kernel
# source (tree.cuh, k_tree_far2: 1 sub, 6 fma, 7 mul; an f32x2 instruction does two), plus 2 SFU operations
# (rsqrt, ex2).
OPS_FAR = 14
SFU_FAR = 2


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
    ap.add_argument("--mode", default="solve", choices=["solve", "batch", "serve", "kernels", "tree"],
                    help="solve: the default single-system line; batch: many molecules in one engine; "
                         "serve: continuous-batching server under Poisson arrivals; kernels: two FP32, two "
                         "float-float and two FP64 operator applications of the ellipsoid at --h (the profiling "
                         "case); tree: the solve step with the far-field treecode on the ellipsoid at --tree-h")
    ap.add_argument("--tree-h", type=float, default=0.025, help="tree mode: grid spacing (0.025: ~714k nodes)")
    ap.add_argument("--tree-tol", type=float, default=1e-6,
                    help="tree mode: solve tolerance (the FP32 far field sets a floor near 2e-7)")
    ap.add_argument("--tree-direct", action="store_true",
                    help="tree mode: also time the direct-sum applications at the same size")
    ap.add_argument("--oracle-solves", action="store_true",
                    help="with --impl reference: time whole oracle solves (sphere h=0.25, ellipsoid h=0.2) and one "
                         "full oracle matvec of the 500-atom molecule on the host cores, one JSON line")
    ap.add_argument("--molecules", type=int, default=64, help="batch mode: molecules in the batch")
    ap.add_argument("--max-atoms", type=int, default=2000, help="batch/serve: largest molecule")
    ap.add_argument("--requests", type=int, default=48, help="serve mode: requests per load level")
    ap.add_argument("--loads", default="0.5,0.8,0.95", help="serve mode: offered load / measured capacity")
    ap.add_argument("--pool", type=int, default=12, help="serve mode: distinct problems requests draw from")
    ap.add_argument("--slots", type=int, default=16, help="serve mode: server slots")
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
    R, V, U = ctr.tuning_info()
    line = {"metric": "CTR-IBIM batched pair-interactions/s", "value": pairs / t_batch, "unit": "pair-interactions/s",
            "n_gpus": 1, "steps": 1, "higher_is_better": True, "dtype": "f32 pairs + f64", "data": "synthetic",
            "config": {"workload": f"{len(probs)} random-walk SES molecules, atoms log-uniform in 20-{args.max_atoms}, "
                                   f"h in {{0.5, 0.35}}, tube 2h, FP32 pairs + float-float refinement, tol 1e-10",
                       "M_min": int(Ms.min()), "M_median": int(np.median(Ms)), "M_max": int(Ms.max()),
                       "sum_M2": float(np.sum(Ms ** 2)), "generation_s": t_gen},
            "batch_s": t_batch, "solves_per_s": len(probs) / t_batch, "sequential_s": t_seq,
            "speedup_vs_sequential": t_seq / t_batch, "all_converged": all(i.converged for _, _, i in out),
            "max_iterations": int(max(i.iterations for _, _, i in out)),
            "autotuned_fp32_variant": {"targets_per_thread": R, "chunk": V, "unroll": U}, "gpu_launches": int(launches)}
    for g in systems:
        g.close()
    print(json.dumps(line), flush=True)


def run_serve(args, ctr):
    """Serving: Poisson arrivals at fractions of the measured capacity; latency and throughput."""
    import threading as th
    import torch
    import synthetic as syn
    rng = np.random.Generator(np.random.PCG64(0))
    n_mol = max(1, args.pool // 3)
    mol_specs = syn.batch_specs(n_mol, seed=100, max_atoms=min(args.max_atoms, 600))
    pool = list(syn.molecules_parallel(mol_specs))
    for k in range(max(1, args.pool // 3)):
        pool.append(syn.sphere_with_nodes(int(np.exp(rng.uniform(np.log(5e3), np.log(4e5)))),
                                          q=float(rng.choice([-1.0, 1.0]))))
    for k, hh in enumerate([0.2, 0.1, 0.05][:max(1, args.pool - len(pool))]):
        pool.append(syn.ellipsoid_problem(h=hh, seed=k))
    opts = ctr.Options(precision=ctr.FP32_REFINE, tol=1e-10)

    def run_load(rate, n, seed):
        arrivals = None
        if rate is not None:
            gaps = np.random.Generator(np.random.PCG64(seed)).exponential(1.0 / rate, size=n)
            arrivals = np.cumsum(gaps) - gaps[0]
        picks = np.random.Generator(np.random.PCG64(seed + 1)).integers(0, len(pool), size=n)
        with ctr.Server(max_slots=args.slots) as sv:
            tickets = [None] * n
            t0 = time.perf_counter()

            def submitter():
                for i in range(n):
                    if arrivals is not None:
                        dt = arrivals[i] - (time.perf_counter() - t0)
                        if dt > 0:
                            time.sleep(dt)
                    p = pool[picks[i]]
                    tickets[i] = sv.submit_problem(p, ctr.Options(tube_halfwidth=p.tube, precision=opts.precision,
                                                                  tol=opts.tol))

            thr = th.Thread(target=submitter)
            thr.start()
            thr.join()
            res = [sv.wait(t, timeout=3600) for t in tickets]
            st = sv.stats()
        lat = np.array([r.latency for r in res])
        t_first = min(r.t_submit for r in res)
        t_last = max(r.t_done for r in res)
        ok = all(r.status == 0 for r in res)
        return {"solves_per_s": n / (t_last - t_first), "p50_latency_s": float(np.percentile(lat, 50)),
                "p99_latency_s": float(np.percentile(lat, 99)), "mean_latency_s": float(lat.mean()),
                "all_ok": ok, "peak_slots": st["peak_slots"], "peak_used_GB": st["peak_used_bytes"] / 1e9,
                "steps": st["steps"], "G": {int(picks[i]): res[i].G_pol for i in range(n)}}

    warm = run_load(None, min(len(pool), 4), 7)      # warm-up (autotuning, first-touch)
    cap = run_load(None, args.requests, 11)          # saturated: everything submitted at once
    capacity = cap["solves_per_s"]
    levels = {}
    for f in [float(v) for v in args.loads.split(",") if v]:
        levels[str(f)] = run_load(f * capacity, args.requests, 13)
    # the plain FP64 one-at-a-time GPU path on the same pool (energies for the error check)
    t0 = time.perf_counter()
    G64 = {}
    for k, p in enumerate(pool):
        with ctr.CtrIbim.from_problem(p, options=ctr.Options(tube_halfwidth=p.tube, precision=ctr.FP64,
                                                               tol=1e-10)) as G:
            psi, dpsi, _ = G.solve(device=True)
            G64[k] = G.energy(psi, dpsi)[0]
    torch.cuda.synchronize()
    t64 = time.perf_counter() - t0
    errs = [abs(levels[str(f)]["G"][k] / G64[k] - 1) for f in levels for k in levels[str(f)]["G"]]
    Ms = []
    for p in pool:
        with ctr.CtrIbim.from_problem(p) as G:
            Ms.append(G.M)
    for lv in list(levels.values()) + [cap]:
        lv.pop("G", None)
    line = {"metric": "CTR-IBIM served solves/s", "value": levels[max(levels, key=float)]["solves_per_s"],
            "unit": "solves/s", "n_gpus": 1, "higher_is_better": True, "dtype": "f32 pairs + f64",
            "data": "synthetic",
            "config": {"workload": f"{args.requests} requests per load level, Poisson arrivals, drawn from a pool of "
                                   f"{len(pool)} problems (SES molecules, spheres, ellipsoids), FP32 pairs + "
                                   f"float-float refinement to 1e-10", "M_min": int(min(Ms)), "M_max": int(max(Ms)),
                       "slots": args.slots},
            "capacity_solves_per_s": capacity, "saturated": cap, "levels": levels,
            "fp64_one_at_a_time_solves_per_s": len(pool) / t64,
            "max_rel_energy_error_vs_fp64_path": float(max(errs)) if errs else None}
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
    rate_ffma = ctypes_probe(ctr, 0)
    rate_ex2 = ctypes_probe(ctr, 2)
    rate_rsq = ctypes_probe(ctr, 3)
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
        kern.append({"bound": "alu", "kernel": f"k_tree_mom + k_tree_momred + k_tree_far2<"
                                               f"{'2, 256' if tag == 'fp32' else '1, 128'}> (treecode far field, "
                                               f"{tag} blocks)",
                     "achieved": far / t_far if t_far > 0 else None, "peak": far_peak,
                     "unit": "proxy evaluations/s",
                     "frac": far / t_far / far_peak if t_far > 0 else None, "traffic": None,
                     "peak_basis": f"min({sms} SMs x 128 FP32 lanes x {f_max / 1e6:.0f} MHz / {OPS_FAR} lane ops, "
                                   f"SFU: 1/(1/ex2 + 1/rsqrt) with the measured probes {rate_ex2:.4g}/s, "
                                   f"{rate_rsq:.4g}/s) per proxy evaluation",
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
    if args.mode in ("batch", "serve", "kernels", "tree"):
        import torch
        torch.cuda.set_device(local)
        import paper_2210_03699_gb300 as ctr
        if rank == 0:
            if args.mode == "tree":
                run_tree(args, ctr, 1)
            else:
                {"batch": run_batch, "serve": run_serve, "kernels": run_kernels}[args.mode](args, ctr)
        return
    import torch
    torch.cuda.set_device(local)
    import paper_2210_03699_gb300 as ctr

    prob, cfg = workload(args.h)
    prec = ctr.FP32_REFINE if args.precision == "fp32_refine" else ctr.FP64
    opts = ctr.Options(tube_halfwidth=prob.tube, precision=prec, tol=1e-10)
    cfg["solver"] = f"{args.precision}, GMRES restart {opts.restart}, tol {opts.tol:g}"
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
            M, info, Gp = step()
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

    # kernel-level rooflines: FP32 and float-float operator applications, timed on the stream
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
        Mk = G.M
    rate_ffma = ctypes_probe(ctr, 0)
    rate_ex2 = ctypes_probe(ctr, 2)
    rate_dfma = ctypes_probe(ctr, 4)
    # FMA-pipe lane operations per second from unit counts and clocks: SMs x 128 FP32 lanes x the SM clock
    # ceiling (sampled by nvidia-smi; 2070 MHz when unavailable).  The FFMA probe's measured rate is reported
    # beside it.
    sms = torch.cuda.get_device_properties(local).multi_processor_count
    f_max = (clk.summary().get("sm_max_mhz") or 2070.0) * 1e6
    rate_units = sms * 128 * f_max

    def roof(pr, ops, name, key, rate=None):
        sc = sched[pr]
        n_ops = ops["one"] * sc["one_sided_pairs"] + ops["sym"] * sc["symmetric_pairs"]
        peak = (rate or rate_units) * Mk * Mk / n_ops
        ach = Mk * Mk / t_mv[pr]
        return {"bound": "alu", "kernel": name, "achieved": ach, "peak": peak, "unit": "pair-interactions/s",
                "frac": ach / peak, "traffic": TRAFFIC_H005[key] if abs(args.h - 0.05) < 1e-12 else None,
                "peak_basis": f"{sms} SMs x 128 FP32 lanes x {f_max / 1e6:.0f} MHz = {rate_units:.4g} lane ops/s "
                              f"x M^2 / FMA-pipe lane ops of the schedule ({ops['one']} per one-sided and "
                              f"{ops['sym']} per symmetric pair evaluation); measured FFMA probe {rate_ffma:.4g}/s",
                "t_matvec_ms": t_mv[pr] * 1e3, "one_sided_pairs": sc["one_sided_pairs"],
                "symmetric_pairs": sc["symmetric_pairs"], "items": sc["items"]}

    i_last = infos[-1]
    if prec == ctr.FP32_REFINE:
        r32 = roof(ctr.FP32_REFINE, OPS_FP32, "sched_kernel<Fp32x2Policy> (packed FP32 pair sum, inner GMRES)",
                   "fp32")
        rdf = roof(ctr.DF64, OPS_DF64, "sched_kernel<Df64Policy> (float-float pair sum, refinement residual)",
                   "df64")
        share32 = i_last.matvecs_fp32 * t_mv[ctr.FP32_REFINE]
        sharedf = i_last.matvecs_fp64 * t_mv[ctr.DF64]
        dominant, other = (rdf, r32) if sharedf >= share32 else (r32, rdf)
        dominant = dict(dominant, ex2_rate=rate_ex2, dfma_rate=rate_dfma,
                        step_share=max(share32, sharedf) / (t_max / args.steps))
        other = dict(other, step_share=min(share32, sharedf) / (t_max / args.steps))
    else:   # plain FP64 solves: every application is the FP64 schedule, bound by the DFMA pipe
        dominant = roof(ctr.FP64, OPS_FP64, "sched_kernel<Fp64Policy> (FP64 pair sum)", "fp64", rate=rate_dfma)
        dominant["bound"] = "alu"
        dominant["peak_basis"] = (f"measured DFMA probe {rate_dfma:.4g}/s x M^2 / FP64-pipe lane ops of the "
                                  f"schedule ({OPS_FP64['one']} per pair evaluation, ncu count)")
        dominant = dict(dominant, step_share=i_last.matvecs_fp64 * t_mv[ctr.FP64] / (t_max / args.steps))
        other = None

    # e2e through the public API with host buffers
    e2e = None
    if not args.skip_e2e:
        h2d = prob.sdist.nbytes + prob.charge_xyz.nbytes + prob.charge_q.nbytes
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        e2e_pairs = 0.0
        for _ in range(max(1, args.steps)):
            with ctr.CtrIbim.from_problem(prob, options=opts) as G:
                psi, dpsi, info = G.solve(device=False)
                Gp, _ = G.energy(psi, dpsi)
                e2e_pairs += float(G.M) ** 2 * (info.matvecs_fp32 + info.matvecs_fp64)
                d2h = psi.nbytes + dpsi.nbytes + 8
        torch.cuda.synchronize()
        t_e2e = max_over_ranks(time.perf_counter() - t0, world)
        e2e = {"value": sum_over_ranks(e2e_pairs, world) / t_e2e, "unit": "pair-interactions/s",
               "h2d_bytes_per_step": int(h2d), "d2h_bytes_per_step": int(d2h)}

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
            "config": dict(cfg, M=int(M), unknowns=int(2 * M), iterations=int(i0.iterations),
                           refinements=int(i0.refinements), matvecs_fp32=int(i0.matvecs_fp32),
                           matvecs_fp64=int(i0.matvecs_fp64), residual=i0.residual, G_pol=Gp),
            "roofline": dominant,
            "roofline_second": other,
            "clocks": clk.summary(),
            "e2e": e2e,
            "gpu_launches": int(launches),
            "wall_s": t_wall,
            "cpu_baseline": cpu,
        }
        print(json.dumps(line), flush=True)
    if world > 1:
        import torch.distributed as dist
        dist.destroy_process_group()


def ctypes_probe(ctr, kind, iters=20000):
    import ctypes
    L = ctr.lib
    L.ctr_probe_rate.restype = ctypes.c_int
    L.ctr_probe_rate.argtypes = [ctypes.c_int, ctypes.c_int64, ctypes.POINTER(ctypes.c_double),
                                 ctypes.POINTER(ctypes.c_double)]
    r = ctypes.c_double()
    s = ctypes.c_double()
    st = L.ctr_probe_rate(kind, iters, ctypes.byref(r), ctypes.byref(s))
    return float(r.value) if st == 0 else None


if __name__ == "__main__":
    main()
