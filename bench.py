"""Benchmark: converged eigenpairs per second near a target energy density, L = 18.

Workload (the L = 18 shift-invert configuration): dim 48 620, nev = 50 eigenpairs nearest
sigma = E_min + eps (E_max - E_min), h in {0.5, 1, 2, 3, 4, 5}, eps in {0.1, 0.5, 0.9}.  A step is
one batch of `--batch` jobs (L, h, seed, eps) run through the whole path: sector build from the
job's fields, extremal bounds, numeric factorization (FP32 fronts on tcgen05, FP64 refinement),
block shift-invert Lanczos, Rayleigh-Ritz on H, observables.  The timed region runs all K steps'
jobs in the served form (continuous batching on `--slots` worker streams with HBM admission): the
value is the converged eigenpairs (residual <= 1e-10 ||H||) over the device span of those jobs
(CUDA events).  The same jobs then run one after another on one stream for the kernel profile and
the roofline, and a subset runs on the plain FP64 path for the mixed-versus-FP64 comparison.  The
symbolic analysis of the L = 18 pattern is setup (built once in warm-up, excluded).

    python bench.py [--gpus N] [--steps K] [--warmup W] [--batch B] [--slots S] [--impl reference]
    python bench.py --case {factor,solve} [--L L] [--reps R] [--precision fp32|fp64]   (profiler cases)
    python bench.py --case observables [--L L] [--reps R]   (the eigenvector observables on nev = 50 vectors)
"""
from __future__ import annotations

import argparse
import json
import math
import os
import statistics
import subprocess
import sys
import threading
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

L = 18
NEV = 50
HS = [0.5, 1.0, 2.0, 3.0, 4.0, 5.0]
EPS = [0.1, 0.5, 0.9]
PROF_KEYS = ("factor_fp32", "schur_fp32", "schur_tc", "trisolve_fp32", "refine_spmv", "orth", "syev_krylov",
             "syev_rr", "extremal_bounds", "op_apply", "ks_restart", "ritz_h", "observables", "sector_build",
             "syev_fp32", "syev_fallback", "oa_refine", "trisolve_fp64", "factor_fp64", "syev_rr_fp64",
             "gm_deflate", "gm_spmv", "gm_orth", "f_assemble", "f_panel", "f_build_g", "syev_rr_bisect")
METRIC = "eigenpairs/s near eps (res<=1e-10||H||), L=18, mixed vs FP64; p50/p99 latency"


def jobs_for_step(step: int, batch: int, rank: int = 0, world: int = 1):
    out = []
    for b in range(batch):
        k = (step * batch + b) * world + rank
        out.append((HS[k % len(HS)], 1000 + k, EPS[(k // len(HS)) % len(EPS)]))
    return out


class ClockSampler:
    def __init__(self, path):
        self.path, self.proc = path, None

    def __enter__(self):
        q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
             "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
             "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")
        try:
            self.f = open(self.path, "w")
            self.proc = subprocess.Popen(["nvidia-smi", f"--query-gpu={q}", "--format=csv,noheader,nounits",
                                          "-lms", "200"], stdout=self.f, stderr=subprocess.DEVNULL)
        except Exception:
            self.proc = None
        return self

    def __exit__(self, *a):
        if self.proc is not None:
            self.proc.terminate()
            self.proc.wait(timeout=10)
            self.f.close()

    def summary(self, device: int = 0):
        try:
            rows = [r.split(",") for r in open(self.path).read().strip().splitlines()]
        except Exception:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["unsampled"]}
        rows = [[c.strip() for c in r] for r in rows if len(r) >= 9 and r[0].strip() == str(device)]
        if not rows:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["unsampled"]}
        mhz = [float(r[1]) for r in rows if r[1].replace(".", "").isdigit()]
        reasons = set()
        for r in rows:
            for name, col in (("hw_slowdown", 5), ("hw_thermal_slowdown", 6), ("sw_thermal_slowdown", 7),
                              ("sw_power_cap", 8)):
                if r[col].lower().startswith("active"):
                    reasons.add(name)
        return {"sm_mhz": statistics.median(mhz) if mhz else None,
                "sm_max_mhz": float(rows[0][2]) if rows[0][2].replace(".", "").isdigit() else None,
                "reasons": sorted(reasons), "samples": len(rows)}


def measured_peaks():
    try:
        return json.load(open(os.path.join(ROOT, "MEASURED_PEAKS.json")))
    except Exception:
        return None


# --------------------------------------------------------------------------------------------
def run_reference(args):
    """The oracle as it stands on the host cores: a bounded sample of the same L=18 jobs is out of
    reach (about an hour per job), so each step runs the oracle on L=16 jobs of the same shape and
    reports their eigenpairs/s, labelled as such."""
    rank = int(os.environ.get("RANK", "0"))
    if rank != 0:
        return 0
    import multiprocessing as mp

    cores = os.cpu_count() or 1
    ctx = mp.get_context("spawn")
    per_step = max(1, cores)
    t_steps = []
    pairs = 0
    with ctx.Pool(cores) as pool:
        for s in range(args.warmup + args.steps):
            # warm-up steps only start the workers (imports, oracle library load): one L=12 job each
            Ls = 16 if s >= args.warmup else 12
            jobs = [(Ls, h, seed, eps, NEV if Ls == 16 else 20) for (h, seed, eps) in jobs_for_step(s, per_step)]
            t0 = time.perf_counter()
            res = pool.map(_oracle_job, jobs)
            dt = time.perf_counter() - t0
            if s >= args.warmup:
                t_steps.append(dt)
                pairs += sum(res)
    tot = sum(t_steps)
    v = pairs / tot
    line = {"impl": "reference", "metric": METRIC, "value": v, "unit": "eigenpairs/s", "n_gpus": args.gpus,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * tot / args.steps,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": {"workload": "oracle sample: L=16 jobs shaped like the L=18 workload (h in {0.5..5}, "
                                   "eps in {0.1,0.5,0.9}, nev=50)", "L": 16, "nev": NEV, "jobs_per_step": per_step},
            "cpu_baseline": {"value": v, "unit": "eigenpairs/s", "cores": cores, "kind": "oracle",
                             "sample": f"{per_step * args.steps} oracle shift-invert jobs at L=16 (one per core)"},
            "e2e": {"value": v, "unit": "eigenpairs/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line))
    return 0


def _oracle_job(job):
    import oracle

    L_, h, seed, eps, nev = job
    r = oracle.solve_job(oracle.Job(L_, h, seed, eps, nev), "si")
    hn = max(abs(r.emin), abs(r.emax))
    return int((r.resid <= 1e-10 * hn).sum())


def cpu_baseline_sample(seconds: float = 20.0):
    """Oracle on the host cores for a bounded time: L=16 jobs of the workload's shape."""
    import multiprocessing as mp

    cores = os.cpu_count() or 1
    ctx = mp.get_context("spawn")
    jobs = [(16, h, seed, eps, NEV) for (h, seed, eps) in jobs_for_step(0, cores)]
    t0 = time.perf_counter()
    with ctx.Pool(cores) as pool:
        res = pool.map(_oracle_job, jobs)
    dt = time.perf_counter() - t0
    return {"value": sum(res) / dt, "unit": "eigenpairs/s", "cores": cores, "kind": "oracle",
            "sample": f"{len(jobs)} oracle shift-invert jobs at L=16 (nev=50, one per core) in {dt:.1f} s; "
                      f"an L=18 oracle job takes about an hour on one core"}


# --------------------------------------------------------------------------------------------
def run_case(args):
    """A single-operation case for profilers: one L-site sector (h = 3, seed 5), one factorization of
    H - sigma at eps = 0.5, then --reps unrefined block solves with 8 right-hand sides."""
    import numpy as np

    import paper_1411_0660_gb300 as g

    ctx = g.Context(0)
    sec = g.build_sector(ctx, args.L, 3.0, 5)
    lo, hi = g.extremal_bounds(sec)
    prec = g.MBL_PREC_FP64 if args.precision == "fp64" else g.MBL_PREC_FP32
    import torch

    nvtx = getattr(torch.cuda, "nvtx", None)
    if nvtx is not None:
        nvtx.range_push("factor")
    f = g.factor(sec, lo + 0.5 * (hi - lo), precision=prec, tensor_cores=args.tensor_cores,
                 solve_dataflow=args.dataflow)
    if nvtx is not None:
        nvtx.range_pop()
    B = np.random.default_rng(0).standard_normal((sec.dim, 8))
    t0 = time.perf_counter()
    if nvtx is not None:
        nvtx.range_push("solve")
    for _ in range(args.reps if args.case == "solve" else 0):
        f.solve(B, refine=False)
    if nvtx is not None:
        nvtx.range_pop()
    dt = time.perf_counter() - t0
    line = {"case": args.case, "L": args.L, "precision": args.precision, "reps": args.reps,
            "solve_s_per_rep": dt / max(1, args.reps), "factor": f.stats()}
    if args.case == "solve" and args.trace:
        # per-launch device clocks of one more solve: where the sequence spends its time
        f.set_trace(True)
        for _ in range(2):
            f.solve(B, refine=False)
        t0s, t1s, kind = f.trace()
        base = int(t0s.min())
        rec = [[int(k), (int(a) - base) / 1e3, (int(b) - base) / 1e3] for k, a, b in zip(kind, t0s, t1s)]
        prev = 0.0
        crit = {0: 0.0, 1: 0.0, 2: 0.0, 3: 0.0}
        for k, a, b in rec:  # time each launch adds after its predecessor finished
            crit[k] += b - max(prev, a)
            prev = b
        line["trace"] = {"launches": len(rec), "span_us": rec[-1][2] - rec[0][1] if rec else 0.0,
                         "critical_us": {"gather": crit[0], "forward": crit[1], "backward_start": crit[2],
                                         "backward_update": crit[3]}}
        with open(args.trace, "w") as fo:
            json.dump({"records_us": rec, "kinds": "0 gather, 1 forward step, 2 backward level start, "
                                                   "3 backward update"}, fo)
    print(json.dumps(line))
    f.close()
    sec.close()
    ctx.close()
    return 0


def run_observables_case(args):
    """Device time of the eigenvector observables on nev = 50 seeded random unit vectors of the
    L-site sector (their cost does not depend on the vectors): mbl_observables_dev (r, S_1^P, S_E)
    and mbl_observables_extra_dev (KL, S_2^P, F, f).  The roofline is the extra observables'
    algorithmic traffic, one read of the n x nev vectors, over their CUDA-event time."""
    import numpy as np
    import torch

    import paper_1411_0660_gb300 as g

    ctx = g.Context(0)
    n, nev = math.comb(args.L, args.L // 2), NEV
    dev = torch.device("cuda:0")
    gen = torch.Generator(device=dev)
    gen.manual_seed(1234)
    Y = torch.randn(nev, n, dtype=torch.float64, device=dev, generator=gen)
    Y /= Y.norm(dim=1, keepdim=True)
    Y = Y.reshape(-1).contiguous()  # column-major n x nev
    ev = torch.linspace(-1.0, 1.0, nev, dtype=torch.float64, device=dev)
    outs = [torch.zeros(m, dtype=torch.float64, device=dev) for m in (nev - 2, 1, nev, nev)]
    outx = [torch.zeros(m, dtype=torch.float64, device=dev) for m in (nev - 1, nev, nev, nev)]
    st = torch.cuda.current_stream()
    for _ in range(3):
        g.observables_dev(ctx, args.L, nev, ev, Y, *outs, stream=st)
        g.observables_extra_dev(ctx, args.L, nev, Y, 2.0, *outx, stream=st)
    e = [torch.cuda.Event(enable_timing=True) for _ in range(4)]
    torch.cuda.synchronize()
    e[0].record(st)
    for _ in range(args.reps):
        g.observables_dev(ctx, args.L, nev, ev, Y, *outs, stream=st)
    e[1].record(st)
    e[2].record(st)
    for _ in range(args.reps):
        g.observables_extra_dev(ctx, args.L, nev, Y, 2.0, *outx, stream=st)
    e[3].record(st)
    torch.cuda.synchronize()
    ms_base = e[0].elapsed_time(e[1]) / args.reps
    ms_extra = e[2].elapsed_time(e[3]) / args.reps
    peak = (measured_peaks() or {}).get("hbm_gbs")
    gbs = 8.0 * n * nev / (ms_extra * 1e-3) / 1e9
    print(json.dumps({"case": "observables", "L": args.L, "n": n, "nev": nev, "ms_r_s1p_se": ms_base,
                      "ms_kl_sqp_fluct_dynf": ms_extra, "extra_gbs": gbs, "hbm_peak_gbs": peak,
                      "extra_frac": gbs / peak if peak else None}))
    ctx.close()
    return 0


def run_workload(args):
    """Other configurations of the workload table, each printing its own JSON line:
    l16batch -- batched small sizes: L = 16, h in {1, 2.5, 4} x eps in {0.1, ..., 0.9} x `--seeds`
                seeds, nev = 50, FP64 fronts, all submitted at once to a server of `--slots` streams;
    serve    -- a serving stream: Poisson arrivals (`--rate` per second, `--requests` requests) of
                L in {14, 16, 18, 20} weighted 4:3:2:1, h ~ U[0.5, 5], seed = request id,
                eps ~ U[0.05, 0.95], nev = 50, mixed precision; p50/p99 latency and throughput;
    large    -- the large sizes: L = 20, h = 3, `--seeds` seeds x eps in {0.2, 0.5, 0.8}, nev = 50, mixed
                precision through the server; plus the symbolic analysis (fill-in, flops, device
                footprint) of L = 18, 20 and 22, whose L = 22 fronts do not fit in one GPU;
    odd      -- the odd-L sector of the numerical-method section at its largest size: L = 19 with
                10 up spins (its "S^z = 1", dimension 92 378), h in {1, 3, 5} x `--seeds` seeds x
                eps in {0.2, 0.5, 0.8}, nev = 50, mixed precision through the server."""
    import numpy as np
    import torch

    import paper_1411_0660_gb300 as g

    ctx = g.Context(0)
    srv = g.Server(ctx, slots=args.slots)
    plans = None
    if args.workload == "large":
        dev_total = torch.cuda.get_device_properties(0).total_memory
        plans = {}
        for L_ in (18, 20, 22):
            sec = g.build_sector(ctx, L_, 3.0, 0)
            pst = g.analyse(sec, 50, 8)
            sec.close()
            pst["fits_one_gpu_fp32"] = pst["job_peak_bytes_fp32"] < 0.85 * dev_total
            plans[str(L_)] = pst
        jobs = [(20, 3.0, s, e, g.MBL_PREC_FP32) for s in range(args.seeds) for e in (0.2, 0.5, 0.8)]
        srv.wait(srv.submit(20, 3.0, 10 ** 6, 0.5, 50))  # warm-up: kernels and graphs at L = 20
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        tickets = [srv.submit(L_, h, s, e, 50, precision=pr) for (L_, h, s, e, pr) in jobs]
        out = [srv.wait(t) for t in tickets]
        host_s = time.perf_counter() - t0
    elif args.workload == "odd":
        jobs = [(19, h, s, e, g.MBL_PREC_FP32) for s in range(args.seeds) for h in (1.0, 3.0, 5.0)
                for e in (0.2, 0.5, 0.8)]
        srv.wait(srv.submit(19, 3.0, 10 ** 6, 0.5, 50, nup=10))  # warm-up: plan, kernels, graphs
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        tickets = [srv.submit(L_, h, s, e, 50, precision=pr, nup=10) for (L_, h, s, e, pr) in jobs]
        out = [srv.wait(t) for t in tickets]
        host_s = time.perf_counter() - t0
    elif args.workload == "l16batch":
        jobs = [(16, h, s, e / 10.0, g.MBL_PREC_FP64) for s in range(args.seeds) for h in (1.0, 2.5, 4.0)
                for e in range(1, 10)]
        for t in [srv.submit(16, 1.0, 10 ** 6 + k, 0.5, 50, precision=g.MBL_PREC_FP64) for k in range(args.slots)]:
            srv.wait(t)  # warm-up: plan, kernels, graphs
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        tickets = [srv.submit(L_, h, s, e, 50, precision=pr) for (L_, h, s, e, pr) in jobs]
        out = [srv.wait(t) for t in tickets]
        host_s = time.perf_counter() - t0
    else:
        rng = np.random.default_rng(12345)
        Ls = rng.choice([14, 16, 18, 20], size=args.requests, p=[0.4, 0.3, 0.2, 0.1])
        gaps = rng.exponential(1.0 / args.rate, size=args.requests)
        hs = rng.uniform(0.5, 5.0, size=args.requests)
        es = rng.uniform(0.05, 0.95, size=args.requests)
        for L_ in (14, 16, 18, 20):  # warm-up: one request per size builds the plans
            srv.wait(srv.submit(L_, 1.0, 10 ** 6 + L_, 0.5, 50))
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        tickets, due = [], 0.0
        for k in range(args.requests):
            due += gaps[k]
            delay = due - (time.perf_counter() - t0)
            if delay > 0:
                time.sleep(delay)
            tickets.append(srv.submit(int(Ls[k]), float(hs[k]), k, float(es[k]), 50))
        out = [srv.wait(t) for t in tickets]
        host_s = time.perf_counter() - t0
        jobs = list(zip(Ls.tolist(), hs.tolist(), range(args.requests), es.tolist()))
    st = srv.stats()
    srv.stop()
    span_ms = max(r.d_end_ms for r in out) - min(r.d_start_ms for r in out)
    pairs = sum(r.nconv for r in out)
    lat = sorted((r.t_end_ms - r.t_submit_ms) for r in out)
    line = {"workload": args.workload, "jobs": len(out), "slots": args.slots,
            "eigenpairs_per_s": pairs / (span_ms / 1e3), "eigenpairs_per_s_host": pairs / host_s,
            "converged": pairs, "requested": 50 * len(out), "device_span_s": span_ms / 1e3, "host_s": host_s,
            "latency_ms": {"p50": lat[len(lat) // 2], "p99": lat[min(len(lat) - 1, int(0.99 * len(lat)))],
                           "max": lat[-1]},
            "min_nconv": min(r.nconv for r in out), "peak_reserved_gb": st["peak_reserved_bytes"] / 1e9,
            "failed": st["failed"],
            "not_converged": [{"L": int(j[0]), "h": float(j[1]), "seed": int(j[2]), "eps": float(j[3]),
                               "nconv": r.nconv, "status": r.status} for j, r in zip(jobs, out) if r.status != 0]}
    if plans is not None:
        line["plans"] = plans
    if args.workload in ("large", "odd"):
        line["job_s"] = sorted(round((r.d_end_ms - r.d_start_ms) / 1e3, 2) for r in out)
    if args.workload == "serve":
        line.update({"rate_per_s": args.rate, "by_L": {str(L_): sum(1 for j in jobs if j[0] == L_) for L_ in (14, 16, 18, 20)}})
    print(json.dumps(line))
    ctx.close()
    return 0


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--case", choices=["factor", "solve", "observables"], default=None,
                    help="run one factorization (and --reps solves) instead of the benchmark")
    ap.add_argument("--L", type=int, default=18)
    ap.add_argument("--workload", choices=["l18", "l16batch", "serve", "large", "odd"], default="l18",
                    help="l18: the benchmark line; l16batch / serve: the batched and serving configurations")
    ap.add_argument("--seeds", type=int, default=8, help="l16batch: seeds per (h, eps)")
    ap.add_argument("--requests", type=int, default=40, help="serve: number of requests")
    ap.add_argument("--rate", type=float, default=4.0, help="serve: mean arrivals per second")
    ap.add_argument("--reps", type=int, default=3)
    ap.add_argument("--precision", choices=["fp32", "fp64"], default="fp32")
    ap.add_argument("--tensor-cores", type=int, default=1)
    ap.add_argument("--dataflow", type=int, default=0, help="solve sweeps as persistent dataflow kernels")
    ap.add_argument("--trace", default=None, help="--case solve: write per-launch device clocks of one solve here")
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=3)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--batch", type=int, default=6)
    ap.add_argument("--slots", type=int, default=8, help="concurrent jobs (worker streams) in the timed region")
    ap.add_argument("--impl", default="gb300")
    ap.add_argument("--fp64-stride", type=int, default=3)
    ap.add_argument("--no-cpu-baseline", action="store_true")
    args = ap.parse_args()
    if args.case == "observables":
        return run_observables_case(args)
    if args.case:
        return run_case(args)
    if args.workload != "l18":
        return run_workload(args)
    if args.impl == "reference":
        return run_reference(args)

    # cpu baseline first (spawned workers, before the first CUDA call)
    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    cpu = None
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        cpu = cpu_baseline_sample()

    import numpy as np
    import torch

    import paper_1411_0660_gb300 as g

    local = int(os.environ.get("LOCAL_RANK", "0"))
    torch.cuda.set_device(local)
    dist = None
    if world > 1:
        import torch.distributed as dist

        dist.init_process_group("nccl")
    ctx = g.Context(local)
    n = 48620
    d_ev = torch.empty(NEV, dtype=torch.float64, device="cuda")
    d_vec = torch.empty(n * NEV, dtype=torch.float64, device="cuda")
    d_res = torch.empty(NEV, dtype=torch.float64, device="cuda")
    d_r = torch.empty(NEV - 2, dtype=torch.float64, device="cuda")
    d_rm = torch.empty(1, dtype=torch.float64, device="cuda")
    d_s1 = torch.empty(NEV, dtype=torch.float64, device="cuda")
    d_se = torch.empty(NEV, dtype=torch.float64, device="cuda")

    def device_job(h, seed, eps, prec, tc=1):
        sec = g.build_sector(ctx, L, h, seed)
        nconv, sigma, st = g.solve_near_dev(sec, eps, NEV, d_ev, d_vec, d_res, precision=prec, tensor_cores=tc)
        g.observables_dev(ctx, L, NEV, d_ev, d_vec, d_r, d_rm, d_s1, d_se)
        sec.close()
        return nconv, st

    # warm-up (builds the L=18 plan once: setup, excluded)
    for s in range(args.warmup):
        for (h, seed, eps) in jobs_for_step(s, 1, rank, world):
            device_job(h, seed, eps, g.MBL_PREC_FP32)
    torch.cuda.synchronize()
    if dist:
        dist.barrier()

    timed_jobs = [j for s in range(args.steps) for j in jobs_for_step(args.warmup + s, args.batch, rank, world)]
    clocks = ClockSampler(os.path.join(ROOT, "gpurun_out", "clocks_bench.csv") if os.path.isdir(
        os.path.join(ROOT, "gpurun_out")) else "/tmp/clocks_bench.csv")
    nvtx = getattr(torch.cuda, "nvtx", None)

    # ---- timed region: the served (continuously batched) form, all K steps' jobs in flight ----
    # Jobs run on `slots` worker streams as HBM allows; the span is measured on the device with the
    # jobs' CUDA events (first start to last end, relative to one reference event).
    # the jobs' inputs: their disorder realizations h_i (host arrays, prepared untimed)
    host_fields = []
    for (h, seed, eps) in timed_jobs:
        sec0 = g.build_sector(ctx, L, h, seed)
        host_fields.append(np.ascontiguousarray(sec0.fields()))
        sec0.close()
    srv = g.Server(ctx, slots=args.slots)
    for t in [srv.submit(L, h, seed, eps, NEV) for (h, seed, eps) in jobs_for_step(0, args.slots, rank, world)]:
        srv.wait(t)  # worker warm-up: kernels loaded, graphs captured once per worker
    torch.cuda.synchronize()
    if dist:
        dist.barrier()
    l0 = g.launch_count()
    with clocks:
        torch.cuda.synchronize()
        if nvtx is not None:
            nvtx.range_push("timed")
        t_host0 = time.perf_counter()
        tickets = [srv.submit(L, h, seed, eps, NEV, want_vectors=True, fields=hf)
                   for (h, seed, eps), hf in zip(timed_jobs, host_fields)]
        served = [srv.wait(t) for t in tickets]
        torch.cuda.synchronize()
        t_host = time.perf_counter() - t_host0
        if nvtx is not None:
            nvtx.range_pop()
    launches = g.launch_count() - l0
    srv_stats = srv.stats()
    srv.stop()
    ms = max(r.d_end_ms for r in served) - min(r.d_start_ms for r in served)
    pairs = sum(r.nconv for r in served)
    lat = [(r.t_end_ms - r.t_submit_ms) / 1e3 for r in served]
    tmax = ms
    if dist:
        t = torch.tensor([ms, pairs], dtype=torch.float64, device="cuda")
        dist.all_reduce(t[:1], op=dist.ReduceOp.MAX)
        tt = torch.tensor([float(pairs)], dtype=torch.float64, device="cuda")
        dist.all_reduce(tt, op=dist.ReduceOp.SUM)
        tmax, pairs = float(t[0]), int(tt[0])
    value = pairs / (tmax / 1e3)

    # ---- the same jobs one after another on one stream (profiled): kernel breakdown, roofline ----
    ctx.set_profiling(True)
    job_ev = [torch.cuda.Event(enable_timing=True) for _ in range(len(timed_jobs) + 1)]
    job_pairs, job_stats = [], []
    ev_mixed = torch.empty((len(timed_jobs), NEV), dtype=torch.float64, device="cuda")
    torch.cuda.synchronize()
    if nvtx is not None:
        nvtx.range_push("sequential")
    for i, (h, seed, eps) in enumerate(timed_jobs):
        job_ev[i].record()
        nc, st = device_job(h, seed, eps, g.MBL_PREC_FP32)
        job_pairs.append(nc)
        job_stats.append(st)
        ev_mixed[i].copy_(d_ev)
    job_ev[-1].record()
    torch.cuda.synchronize()
    if nvtx is not None:
        nvtx.range_pop()
    job_ms = [job_ev[i].elapsed_time(job_ev[i + 1]) for i in range(len(timed_jobs))]
    prof = {k: ctx.profile(k) for k in PROF_KEYS}
    ctx.set_profiling(False)
    sequential = {"value": sum(job_pairs) / (sum(job_ms) / 1e3), "unit": "eigenpairs/s",
                  "ms_per_job": sum(job_ms) / len(job_ms)}

    # ---- the plain FP64 GPU path on a subset of the same jobs (every third one: all h and eps) ----
    sub = list(range(0, len(timed_jobs), max(1, args.fp64_stride)))
    fp64 = None
    if args.fp64_stride > 0 and sub:
        ctx.set_profiling(True)
        torch.cuda.synchronize()
        a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        a.record()
        p64 = 0
        ev64 = {}
        for i in sub:
            h, seed, eps = timed_jobs[i]
            nc, st = device_job(h, seed, eps, g.MBL_PREC_FP64)
            p64 += nc
            ev64[i] = d_ev.clone()
        b.record()
        torch.cuda.synchronize()
        t64 = a.elapsed_time(b)
        f64 = ctx.profile("factor_fp64")
        ctx.set_profiling(False)
        t_mixed = sum(job_ms[i] for i in sub)
        p_mixed = sum(job_pairs[i] for i in sub)
        fp64 = {"value": p64 / (t64 / 1e3), "unit": "eigenpairs/s", "jobs": len(sub),
                "ms_per_job": t64 / len(sub), "factor_ms_per_job": f64["ms"] / max(1, f64["launches"]),
                "mixed_same_jobs": {"value": p_mixed / (t_mixed / 1e3), "ms_per_job": t_mixed / len(sub)},
                "mixed_over_fp64": (p_mixed / t_mixed) / max(p64 / t64, 1e-30),
                "served_mixed_over_fp64": value / max(p64 / (t64 / 1e3), 1e-30)}
        torch.cuda.synchronize()
        # the same subset with split-BF16 Schur updates (3xBF16 on tcgen05), the third precision mode
        a.record()
        pbf, evbf, bf_solves = 0, {}, 0
        for i in sub:
            h, seed, eps = timed_jobs[i]
            nc, st = device_job(h, seed, eps, g.MBL_PREC_FP32, tc=2)
            pbf += nc
            bf_solves += st["solves"]
            evbf[i] = d_ev.clone()
        b.record()
        torch.cuda.synchronize()
        tbf = a.elapsed_time(b)
        # per result: mixed-precision eigenvalues against the FP64 path's, relative to ||H|| ~ |E| scale
        bf_dev = 0.0
        for i in sub:
            h, seed, eps = timed_jobs[i]
            sec = g.build_sector(ctx, L, h, seed)
            lo, hi = g.extremal_bounds(sec)
            sec.close()
            hn_i = max(abs(lo), abs(hi))
            d = (ev_mixed[i] - ev64[i]).abs().max().item()
            job_stats[i]["max_dev_vs_fp64"] = d / hn_i
            bf_dev = max(bf_dev, (evbf[i] - ev64[i]).abs().max().item() / hn_i)
        fp64["bf16x3_same_jobs"] = {"value": pbf / (tbf / 1e3), "ms_per_job": tbf / len(sub), "converged": pbf,
                                    "solves": bf_solves, "mixed_tf32x3_solves": sum(job_stats[i]["solves"] for i in sub),
                                    "max_dev_vs_fp64": bf_dev}

    # ---- end to end: the timed served region itself, on the host clock (host fields in; eigenvalues,
    # residuals, observables and eigenvectors back in host memory) ----
    n_dim = math.comb(L, L // 2)
    h2d_job = L * 8
    d2h_job = 8 * (NEV * 4 + (NEV - 2) + n_dim * NEV)
    e2e = {"value": pairs / t_host, "unit": "eigenpairs/s", "h2d_bytes_per_step": h2d_job * args.batch,
           "d2h_bytes_per_step": d2h_job * args.batch,
           "note": "host wall time of the timed served region; inputs h_i copied from host memory per job, "
                   "eigenvalues, residuals, observables and eigenvectors copied back"}

    # ---- roofline of the dominant kernel class ----
    peaks = measured_peaks()
    dom = max(("schur_fp32", "schur_tc", "trisolve_fp32", "refine_spmv", "orth"), key=lambda k: prof[k]["ms"])
    P = prof[dom]
    per_launch_ms = P["ms"] / max(1, P["launches"])
    per_launch_work = P["work"] / max(1, P["launches"])
    clk = 2070.0
    if dom in ("trisolve_fp32", "refine_spmv"):
        achieved = per_launch_work / (per_launch_ms / 1e3) / 1e9
        peak = peaks["hbm_gbs"] if peaks else 6800.0
        roof = {"bound": "hbm", "unit": "GB/s", "peak_source": "measured copy" if peaks else "fallback"}
    elif dom == "schur_tc":
        # 3xTF32 on tcgen05: algorithmic flops counted once; TF32 dense peak = measured BF16 x 1.1/2.25
        achieved = per_launch_work / (per_launch_ms / 1e3) / 1e12
        bf = (peaks or {}).get("bf16_tflops", 1900.0)
        peak = bf * 1.1 / 2.25
        roof = {"bound": "tensor", "unit": "TFLOP/s",
                "peak_source": "measured BF16 x nominal TF32/BF16 ratio (1.1/2.25)" if peaks else "fallback"}
    elif dom == "schur_fp32":
        achieved = per_launch_work / (per_launch_ms / 1e3) / 1e12
        peak = 152 * 128 * 2 * clk * 1e6 / 1e12
        roof = {"bound": "alu", "unit": "TFLOP/s", "peak_source": "152 SM x 128 FP32 lanes x 2 x 2070 MHz"}
    else:
        achieved = per_launch_work / (per_launch_ms / 1e3) / 1e12
        peak = 152 * 2 * 2 * clk * 1e6 / 1e12
        roof = {"bound": "alu", "unit": "TFLOP/s", "peak_source": "152 SM x 2 FP64 FMA/clk x 2 x 2070 MHz"}
    traffic = None
    if dom == "trisolve_fp32":
        # DRAM bytes of one block solve from the committed ncu capture of the same kernels
        try:
            with open(os.path.join(ROOT, "profiles", "solve_l18_fp32_traffic.md")) as fp:
                for ln in fp:
                    if ln.startswith("traffic_bytes_per_solve:"):
                        traffic = float(ln.split(":")[1])
        except OSError:
            traffic = None
    roof.update({"achieved": achieved, "peak": peak, "frac": achieved / peak, "traffic": traffic, "kernel": dom,
                 "launch_ms": per_launch_ms, "work_per_launch": per_launch_work})
    if traffic is not None:
        roof["traffic_source"] = "profiles/solve_l18_fp32_traffic.md (ncu dram__bytes_read + write, one solve)"

    if rank == 0:
        lat_ms = sorted(1e3 * x for x in lat)
        line = {
            "metric": METRIC, "value": value, "unit": "eigenpairs/s", "n_gpus": args.gpus, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": tmax / args.steps, "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "f32 fronts + f64 refinement", "data": "synthetic",
            "config": {"workload": "L=18 shift-invert: dim 48620, nev=50, h in {0.5,1,2,3,4,5}, eps in "
                                   "{0.1,0.5,0.9}, seeds 1000+k; served on worker streams", "L": L, "nev": NEV,
                       "jobs_per_step": args.batch, "slots": args.slots,
                       "parallelism": f"replicas x{world}", "l2": "working set (factor ~0.5 GB, fronts ~3 GB) "
                                                                  "far above the 129 MB L2"},
            "gpu_launches": launches,
            "clocks": clocks.summary(local),
            "latency_ms": {"p50": lat_ms[len(lat_ms) // 2], "p99": lat_ms[min(len(lat_ms) - 1,
                                                                              int(0.99 * len(lat_ms)))],
                           "note": "submission to completion; all timed jobs submitted at once"},
            "served": {"slots": args.slots, "host_s": t_host, "peak_reserved_gb": srv_stats["peak_reserved_bytes"] / 1e9,
                       "budget_gb": srv_stats["budget_bytes"] / 1e9},
            "sequential": sequential,
            "fp64_path": fp64,
            "per_job": [{"h": j[0], "seed": j[1], "eps": j[2], "nconv": job_pairs[i], "ms": round(job_ms[i], 1),
                         "max_resid_rel": job_stats[i]["max_resid"], "restarts": job_stats[i]["restarts"],
                         "solves": job_stats[i]["solves"], "fp64_fallback": job_stats[i]["fp64_fallback"],
                         **({"max_dev_vs_fp64": job_stats[i]["max_dev_vs_fp64"]}
                            if "max_dev_vs_fp64" in job_stats[i] else {})}
                        for i, j in enumerate(timed_jobs)],
            "roofline": roof,
            "profile": prof,
            "e2e": e2e,
            "cpu_baseline": cpu,
        }
        print(json.dumps(line))
    if dist:
        dist.destroy_process_group()
    return 0


if __name__ == "__main__":
    sys.exit(main())
