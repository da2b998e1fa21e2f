"""Benchmark: converged eigenpairs per second near a target energy density, L = 18.

Workload (the L = 18 shift-invert configuration): dim 48 620, nev = 50 eigenpairs nearest
sigma = E_min + eps (E_max - E_min), h in {0.5, 1, 2, 3, 4, 5}, eps in {0.1, 0.5, 0.9}.  A step is
one batch of `--batch` jobs (L, h, seed, eps) run through the whole path: sector build from the
job's fields, extremal bounds, numeric factorization (FP32 fronts on tcgen05, FP64 refinement),
block shift-invert Lanczos, Rayleigh-Ritz on H, observables.  The timed region runs all K steps'
jobs in the served form (continuous batching on `--slots` worker streams with HBM admission): the
value is the converged eigenpairs (residual <= 1e-10 ||H||) over the device span of those jobs
(CUDA events).  After it, on the first `--compare-jobs` jobs and the same server: `--repeats`
served mixed runs (the spread of the value) and one served FP64 run (mixed versus FP64 in the same
form); then the same jobs one after another on one stream for the kernel profile and the roofline,
and every `--fp64-stride`-th of them on the FP64 and split-BF16 paths one after another.  The
symbolic analysis of the L = 18 pattern is setup (built once in warm-up, excluded).  One compact
JSON line goes to stdout; the per-job records and the full profile go to `--detail`.

    python bench.py [--gpus N] [--steps K] [--warmup W] [--batch B] [--slots S] [--impl reference]
    python bench.py --case {factor,solve} [--L L] [--reps R] [--precision fp32|fp64]   (profiler cases)
    python bench.py --case observables [--L L] [--reps R]   (the eigenvector observables on nev = 50 vectors)
    python bench.py --workload {l16batch,serve,large,odd,l22,campaign}   (the other configurations)
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
WORKLOAD = ("L=18 shift-invert, dim 48620, nev=50, h in {0.5,1,2,3,4,5}, eps in {0.1,0.5,0.9}, "
            "seeds 1000+k")
# job-time classes of the compact line (device ms per job of the sequential profiled pass)
BREAKDOWN = ("factor_fp32", "schur_tc", "f_panel", "f_build_g", "trisolve_fp32", "gm_deflate", "gm_orth",
             "gm_spmv", "orth", "syev_krylov", "syev_rr", "ritz_h", "extremal_bounds", "observables")


def reduce_over_ranks(ms: float, pairs: int, dist, device: str = "cuda"):
    """Whole-job figures of a multi-rank run: the slowest rank's span (MAX) and the converged pairs of
    all ranks (SUM), through torch.distributed collectives on `device`."""
    import torch

    t = torch.tensor([float(ms)], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    tt = torch.tensor([float(pairs)], dtype=torch.float64, device=device)
    dist.all_reduce(tt, op=dist.ReduceOp.SUM)
    return float(t[0]), int(tt[0])


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


_ORDERING = {"band": 0, "cover": 1, "modes": 2, "auto": 3, "hybrid": 4}
_ordering = 3


def _context(device):
    """A library context whose symbolic analyses use the ordering chosen on the command line."""
    ctx = g.Context(device)
    ctx.set_ordering(_ordering)
    return ctx


def profiled_traffic(name, algorithmic_bytes):
    """DRAM bytes per solve from a committed ncu summary under profiles/, or None when that capture
    was taken on a different factorization (its algorithmic bytes per solve are not this run's within
    1%: another ordering or sector), or when the summary is missing."""
    traffic = alg = None
    try:
        with open(os.path.join(ROOT, "profiles", name)) as fp:
            for ln in fp:
                if ln.startswith("traffic_bytes_per_solve:"):
                    traffic = float(ln.split(":")[1])
                elif ln.startswith("algorithmic_bytes_per_solve:"):
                    alg = float(ln.split(":")[1])
    except OSError:
        return None
    if traffic is None or alg is None or abs(alg - algorithmic_bytes) > 0.01 * algorithmic_bytes:
        return None
    return traffic


def measured_peaks():
    try:
        return json.load(open(os.path.join(ROOT, "MEASURED_PEAKS.json")))
    except Exception:
        return None


# --------------------------------------------------------------------------------------------
def oracle_l18_scale(Ls: int = 16):
    """Ratio (mean oracle seconds per L = Ls job) / (mean per L = 18 job) of the stored oracle runs in
    tests/golden (same oracle, one core each, jobs of the L = 18 workload's shape): an L = 18 oracle job
    takes about half an hour, so the L = 18 rate is the timed L = Ls rate times this ratio."""
    t = {}
    for L_ in (Ls, 18):
        with open(os.path.join(ROOT, "tests", "golden", f"oracle_L{L_}.json")) as f:
            js = json.load(f)["jobs"]
        t[L_] = sum(j["oracle_seconds"] for j in js) / len(js)
    return t[Ls] / t[18], t[Ls], t[18]


def _oracle_pool_rate(pool, jobs):
    t0 = time.perf_counter()
    res = pool.map(_oracle_job, jobs)
    return sum(res), time.perf_counter() - t0


def run_reference(args):
    """The oracle as it stands on the host cores.  Each timed step runs one job of the L = 18 workload's
    shape per core at a smaller size (a bounded sample: an L = 18 oracle job takes about half an hour):
    L = 16 (about 30 s a step) for up to 5 steps, L = 14 (about 1.5 s) for more, so that the whole run
    ends within a few minutes.  The reported value is that rate carried to L = 18 by the stored oracle
    timings of the same shapes (oracle_l18_scale), labelled as extrapolated, with the measured rate
    beside it."""
    rank = int(os.environ.get("RANK", "0"))
    if rank != 0:
        return 0
    import multiprocessing as mp

    cores = os.cpu_count() or 1
    ctx = mp.get_context("spawn")
    per_step = max(1, cores)
    t_steps = []
    pairs = 0
    Lsample = 16 if args.steps <= 5 else 14
    with ctx.Pool(cores) as pool:
        for s in range(args.warmup + args.steps):
            # warm-up steps only start the workers (imports, oracle library load): one L=12 job each
            Ls = Lsample if s >= args.warmup else 12
            jobs = [(Ls, h, seed, eps, NEV if Ls == Lsample else 20) for (h, seed, eps) in jobs_for_step(s, per_step)]
            p, dt = _oracle_pool_rate(pool, jobs)
            if s >= args.warmup:
                t_steps.append(dt)
                pairs += p
    tot = sum(t_steps)
    v16 = pairs / tot
    scale, t16, t18 = oracle_l18_scale(Lsample)
    v = v16 * scale
    cpu = {"value": v, "unit": "eigenpairs/s", "cores": cores, "kind": "oracle",
           "sample": f"{per_step * args.steps} oracle shift-invert jobs at L={Lsample} (one per core, nev=50) "
                     f"timed: {v16:.3f} eigenpairs/s; carried to L=18 by the stored oracle seconds per job "
                     f"(L={Lsample} {t16:.1f} s, L=18 {t18:.0f} s, ratio {scale:.5f}): extrapolated",
           f"value_l{Lsample}_measured": v16, "extrapolated": True}
    line = {"impl": "reference", "metric": METRIC, "value": v, "unit": "eigenpairs/s", "n_gpus": args.gpus,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * tot / args.steps,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": {"workload": WORKLOAD, "L": L, "nev": NEV, "jobs_per_step": per_step,
                       "sample_L": Lsample, "extrapolated_to_L": 18},
            "cpu_baseline": cpu,
            "e2e": {"value": v, "unit": "eigenpairs/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line))
    return 0


def _oracle_job(job):
    import oracle

    L_, h, seed, eps, nev = job
    r = oracle.solve_job(oracle.Job(L_, h, seed, eps, nev), "si")
    hn = max(abs(r.emin), abs(r.emax))
    return int((r.resid <= 1e-10 * hn).sum())


def _round_floats(x, sig: int = 6):
    """The line's floats to `sig` significant digits (the line stays under about 3 KB; the detail file
    keeps full precision)."""
    if isinstance(x, float):
        return float(f"{x:.{sig}g}") if math.isfinite(x) else x
    if isinstance(x, dict):
        return {k: _round_floats(v, sig) for k, v in x.items()}
    if isinstance(x, list):
        return [_round_floats(v, sig) for v in x]
    return x


def cpu_baseline_sample():
    """Oracle on the host cores: one L = 16 job of the workload's shape per core (about 20-35 s),
    carried to L = 18 by the stored oracle timings and labelled as extrapolated."""
    import multiprocessing as mp

    cores = os.cpu_count() or 1
    ctx = mp.get_context("spawn")
    jobs = [(16, h, seed, eps, NEV) for (h, seed, eps) in jobs_for_step(0, cores)]
    with ctx.Pool(cores) as pool:
        p, dt = _oracle_pool_rate(pool, jobs)
    v16 = p / dt
    scale, t16, t18 = oracle_l18_scale()
    return {"value": v16 * scale, "unit": "eigenpairs/s", "cores": cores, "kind": "oracle",
            "sample": f"{len(jobs)} oracle shift-invert jobs at L=16 (nev=50, one per core) in {dt:.1f} s = "
                      f"{v16:.3f} eigenpairs/s; carried to L=18 by the stored oracle seconds per job "
                      f"(L=16 {t16:.1f} s, L=18 {t18:.0f} s): extrapolated",
            "value_l16_measured": v16, "extrapolated": True}


# --------------------------------------------------------------------------------------------
def run_batch_case(args):
    """Profiler case of the batched solve: --batch factorizations of L-site sectors (h = 3, seeds 5, 6,
    ..., eps = 0.5), then --reps unrefined block solves of all of them in shared launches (8
    right-hand sides each), inside an NVTX range "solve".  Prints the CUDA-event time per batched
    solve and the achieved algorithmic bandwidth."""
    import numpy as np
    import torch

    import paper_1411_0660_gb300 as g

    ctx = _context(0)
    K = args.batch
    secs, facts = [], []
    for k in range(K):
        sec = g.build_sector(ctx, args.L, 3.0, 5 + k)
        lo, hi = g.extremal_bounds(sec)
        secs.append(sec)
        facts.append(g.factor(sec, lo + 0.5 * (hi - lo), precision=g.MBL_PREC_FP32))
    n, p = secs[0].dim, 8
    gen = torch.Generator(device="cuda")
    gen.manual_seed(7)
    d_b = [torch.randn(n * p, dtype=torch.float64, device="cuda", generator=gen) for _ in range(K)]
    d_x = [torch.zeros_like(b) for b in d_b]
    for _ in range(2):
        g.factor_solve_batch_dev(facts, d_b, d_x, p)
    st = facts[0].stats()
    nvtx = getattr(torch.cuda, "nvtx", None)
    torch.cuda.synchronize()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    if nvtx is not None:
        nvtx.range_push("solve")
    e0.record()
    for _ in range(args.reps):
        g.factor_solve_batch_dev(facts, d_b, d_x, p)
    e1.record()
    torch.cuda.synchronize()
    if nvtx is not None:
        nvtx.range_pop()
    ms = e0.elapsed_time(e1) / args.reps
    algo = K * (2.0 * (st["nnz_l"] + n) * 4 + 16.0 * n * p)
    peak = (measured_peaks() or {}).get("hbm_gbs")
    gbs = algo / (ms * 1e-3) / 1e9
    print(json.dumps({"case": "solve_batch", "L": args.L, "jobs": K, "reps": args.reps, "ms_per_batched_solve": ms,
                      "ms_per_solve": ms / K, "algorithmic_bytes": algo, "achieved_gbs": gbs,
                      "frac_of_measured_hbm": gbs / peak if peak else None}))
    for f in facts:
        f.close()
    for s_ in secs:
        s_.close()
    ctx.close()
    return 0


def run_case(args):
    """A single-operation case for profilers: one L-site sector (h = 3, seed 5), one factorization of
    H - sigma at eps = 0.5, then --reps unrefined block solves with 8 right-hand sides (with
    --batch K > 1: the batched solve of K factorizations, run_batch_case)."""
    import numpy as np

    import paper_1411_0660_gb300 as g

    if args.case == "solve" and args.batch > 1 and args.batch_case:
        return run_batch_case(args)
    ctx = _context(0)
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

    ctx = _context(0)
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


def run_l22(args):
    """The largest sector of the paper's campaign: L = 22 (dimension 705 432), h = 3, seed `--seeds`
    jobs from 0, eps = 0.5, nev = 50, FP32 fronts in the memory-lean arena with FP64 refinement, one
    job after another on the direct path.  Prints the analysis (fill-in, flops, whole and lean arena,
    job peak), and per job the wall time, factorization time, solves and convergence."""
    import torch

    import paper_1411_0660_gb300 as g

    ctx = _context(0)
    out = {"workload": "l22", "L": 22, "n": math.comb(22, 11), "jobs": []}
    for seed in range(args.seeds):
        sec = g.build_sector(ctx, 22, 3.0, seed)
        if seed == 0:
            t0 = time.perf_counter()
            a = g.analyse(sec, NEV, 8)
            a["host_s"] = time.perf_counter() - t0
            out["plan"] = {k: a[k] for k in ("nnz_l", "flops", "max_front", "tree_levels", "front_bytes_fp32",
                                             "front_peak_bytes_fp32", "solve_factor_bytes_fp32",
                                             "job_peak_bytes_fp32", "ms_analyse", "host_s")}
        torch.cuda.synchronize()
        free0 = torch.cuda.mem_get_info()[0]
        t0 = time.perf_counter()
        try:
            res = g.solve_near(sec, 0.5, NEV, allow_partial=True)
        except g.MblError as e:
            out["jobs"].append({"seed": seed, "error": str(e), "s": time.perf_counter() - t0})
            sec.close()
            continue
        dt = time.perf_counter() - t0
        lo, hi = g.extremal_bounds(sec)
        hn = max(abs(lo), abs(hi))
        sec.close()
        out["jobs"].append({"seed": seed, "s": dt, "nconv": res.nconv, "max_resid_over_H": float(res.resid.max() / hn),
                            "sigma": res.sigma, "stats": res.stats, "free_gb_before": free0 / 1e9})
    out["eigenpairs_per_s"] = sum(j.get("nconv", 0) for j in out["jobs"]) / sum(j["s"] for j in out["jobs"])
    print(json.dumps(out))
    ctx.close()
    return 0


def run_campaign_workload(args):
    """Disorder-averaging campaign: L in {12, 14, 16}, h in {1, 2, 2.5, 3, 3.5, 4, 4.5, 5, 6}, `--seeds`
    realizations each, eps = 0.5, nev = 20, through the server; the gap ratio binned per realization,
    mean and standard error per (L, h), the collapse g[(h - h_c) L^(1/nu)] (cubic, w = 0.8) and a
    bootstrap of it, and the weak / strong disorder means against the GOE / Poisson values."""
    import paper_1411_0660_gb300 as g
    from paper_1411_0660_gb300 import campaign as cp

    ctx = _context(0)
    Ls, hs = [12, 14, 16], [1.0, 2.0, 2.5, 3.0, 3.5, 4.0, 4.5, 5.0, 6.0]
    data = cp.run_campaign(ctx, Ls, hs, range(args.seeds), eps=0.5, nev=20, observable="r", slots=args.slots)
    L, h, Q, dQ = cp.points(data)
    table = {f"L{int(a)}_h{b}": [round(q, 4), round(e, 4)] for a, b, q, e in zip(L, h, Q, dQ)}
    fit = cp.collapse_fit(L, h, Q, dQ, w=0.8, L_min=12, hc_range=(2.0, 5.5), nu_range=(0.3, 2.5))
    boot = cp.bootstrap_fit(data, samples=40, seed=1, w=0.8, L_min=12, hc_range=(2.0, 5.5), nu_range=(0.3, 2.5))
    out = {"workload": "campaign", "observable": "r", "eps": 0.5, "nev": 20, "seeds": args.seeds,
           "jobs": data["jobs"], "converged": data["converged"], "requested": data["requested"],
           "seconds": data["seconds"], "eigenpairs_per_s": data["converged"] / data["seconds"],
           "r_mean_stderr": table, "collapse": {"hc": fit["hc"], "nu": fit["nu"], "chi2_per_dof": fit["chi2_per_dof"],
                                                "points": fit["points"], "hc_std": boot["hc_std"],
                                                "nu_std": boot["nu_std"], "bootstrap_fits": boot["fits"]},
           "paper": {"r_goe": 0.5307, "r_poisson": 2 * math.log(2) - 1, "hc_eps05": 3.72, "nu_eps05": 0.91}}
    print(json.dumps(out))
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
                footprint) of L = 18, 20 and 22 (at L = 22 only the memory-lean fronts arena fits);
    odd      -- the odd-L sector of the numerical-method section at its largest size: L = 19 with
                10 up spins (its "S^z = 1", dimension 92 378), h in {1, 3, 5} x `--seeds` seeds x
                eps in {0.2, 0.5, 0.8}, nev = 50, mixed precision through the server."""
    import numpy as np
    import torch

    import paper_1411_0660_gb300 as g

    ctx = _context(0)
    srv = g.Server(ctx, slots=args.slots)
    plans = None
    if args.workload == "large":
        dev_total = torch.cuda.get_device_properties(0).total_memory
        plans = {}
        for L_ in (18, 20, 22):
            sec = g.build_sector(ctx, L_, 3.0, 0)
            pst = g.analyse(sec, 50, 8)
            sec.close()
            pst["fits_one_gpu_fp32"] = pst["job_peak_bytes_fp32"] < dev_total - 4e9
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


def served_run(srv, jobs, fields, precision=None, want_vectors=False):
    """Submit every job at once to the server and wait for all: converged pairs, the device span
    (first job start to last job end, CUDA events), the host wall time and per-job latencies."""
    import paper_1411_0660_gb300 as g

    prec = g.MBL_PREC_FP32 if precision is None else precision
    t0 = time.perf_counter()
    tickets = [srv.submit(L, h, seed, eps, NEV, precision=prec, want_vectors=want_vectors, fields=hf)
               for (h, seed, eps), hf in zip(jobs, fields)]
    out = [srv.wait(t) for t in tickets]
    host_s = time.perf_counter() - t0
    span_ms = max(r.d_end_ms for r in out) - min(r.d_start_ms for r in out)
    pairs = sum(r.nconv for r in out)
    return {"pairs": pairs, "span_ms": span_ms, "host_s": host_s, "value": pairs / (span_ms / 1e3),
            "lat_ms": sorted(r.t_end_ms - r.t_submit_ms for r in out), "results": out}


def _pct(xs, q):
    xs = sorted(xs)
    return xs[min(len(xs) - 1, int(q * len(xs)))]


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--case", choices=["factor", "solve", "observables"], default=None,
                    help="run one factorization (and --reps solves) instead of the benchmark")
    ap.add_argument("--L", type=int, default=18)
    ap.add_argument("--workload", choices=["l18", "l16batch", "serve", "large", "odd", "l22", "campaign"],
                    default="l18",
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
    ap.add_argument("--compare-jobs", type=int, default=18,
                    help="jobs of the comparison arms (served FP64 vs served mixed, repeats, profiled pass)")
    ap.add_argument("--repeats", type=int, default=3, help="served mixed runs of the comparison jobs (spread)")
    ap.add_argument("--fp64-stride", type=int, default=3,
                    help="sequential FP64 and split-BF16 passes on every stride-th comparison job (0: skip)")
    ap.add_argument("--detail", default="/tmp/bench_detail.json",
                    help="file for the per-job records and the full kernel-class profile")
    ap.add_argument("--clocks-csv", default="/tmp/clocks_bench.csv",
                    help="nvidia-smi samples taken during the timed region")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--batch-jobs", type=int, default=16, help="served form: jobs per batched solve launch (1: off)")
    ap.add_argument("--batch-window-us", type=float, default=300.0, help="served form: batcher collection window")
    ap.add_argument("--batch-lanes", type=int, default=2, help="served form: streams of batched solves")
    ap.add_argument("--ordering", choices=sorted(_ORDERING), default="auto",
                    help="fill-reducing ordering of the symbolic analysis")
    ap.add_argument("--cache-fraction", type=float, default=0.0,
                    help="served form: share of HBM keeping finished jobs' factorizations (0: off; the "
                         "workload's realizations are all distinct, and the comparison arms rerun the "
                         "same jobs, which a cache would answer from stored factorizations)")
    args = ap.parse_args()
    global _ordering
    _ordering = _ORDERING[args.ordering]
    args.batch_case = args.case == "solve" and "--batch" in sys.argv
    if args.case == "observables":
        return run_observables_case(args)
    if args.case:
        return run_case(args)
    if args.workload == "l22":
        return run_l22(args)
    if args.workload == "campaign":
        return run_campaign_workload(args)
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
    ctx = _context(local)
    n = math.comb(L, L // 2)
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
    clocks = ClockSampler(args.clocks_csv)
    nvtx = getattr(torch.cuda, "nvtx", None)

    # the jobs' inputs: their disorder realizations h_i (host arrays, prepared untimed)
    host_fields = []
    plan = None
    for (h, seed, eps) in timed_jobs:
        sec0 = g.build_sector(ctx, L, h, seed)
        host_fields.append(np.ascontiguousarray(sec0.fields()))
        if plan is None:  # the plan the served jobs use (built by the warm-up already)
            plan = g.analyse(sec0, NEV, 8)
        sec0.close()
    ordering_used = {v: k for k, v in _ORDERING.items()}[int(plan["ordering"])]
    srv = g.Server(ctx, slots=args.slots, batch_jobs=args.batch_jobs, batch_window_us=args.batch_window_us,
                   batch_lanes=args.batch_lanes, cache_fraction=args.cache_fraction)
    for t in [srv.submit(L, h, seed, eps, NEV) for (h, seed, eps) in jobs_for_step(0, args.slots, rank, world)]:
        srv.wait(t)  # worker warm-up: kernels loaded, graphs captured once per worker
    for t in [srv.submit(L, h, seed, eps, NEV, precision=g.MBL_PREC_FP64)
              for (h, seed, eps) in jobs_for_step(1, 2, rank, world)]:
        srv.wait(t)  # FP64 kernels and graphs too (used by the comparison arm after the timed region)
    torch.cuda.synchronize()
    if dist:
        dist.barrier()

    # ---- timed region: the served (continuously batched) form, all K steps' jobs in flight ----
    # Jobs run on `slots` worker streams as HBM allows; the span is measured on the device with the
    # jobs' CUDA events (first start to last end).  The host wall time of the same region, with the
    # fields copied in and eigenpairs, vectors and observables copied back per job, is the e2e number.
    l0 = g.launch_count()
    b0 = srv.stats()
    with clocks:
        torch.cuda.synchronize()
        if nvtx is not None:
            nvtx.range_push("timed")
        main_run = served_run(srv, timed_jobs, host_fields, want_vectors=True)
        torch.cuda.synchronize()
        if nvtx is not None:
            nvtx.range_pop()
    launches = g.launch_count() - l0
    srv_stats = srv.stats()
    # the batched solves of the timed region (CUDA events around each batch on the batcher's stream)
    served_solve = {k: srv_stats[k] - b0[k]
                    for k in ("solve_batches", "batched_solves", "batch_ms", "batch_bytes", "batch_busy_ms")}
    ms = main_run["span_ms"]
    pairs = main_run["pairs"]
    t_host = main_run["host_s"]
    tmax = ms
    if dist:
        tmax, pairs = reduce_over_ranks(ms, pairs, dist, "cuda")
    value = pairs / (tmax / 1e3)
    served_res = main_run.pop("results")

    # ---- comparison arms on the first `compare_jobs` jobs, same server (same slots) ----
    cmp_idx = list(range(min(args.compare_jobs, len(timed_jobs))))
    cmp_jobs = [timed_jobs[i] for i in cmp_idx]
    cmp_fields = [host_fields[i] for i in cmp_idx]
    reps = []
    for _ in range(max(1, args.repeats)):
        r = served_run(srv, cmp_jobs, cmp_fields)
        r.pop("results")
        reps.append(r)
    s64 = served_run(srv, cmp_jobs, cmp_fields, precision=g.MBL_PREC_FP64)
    s64_res = s64.pop("results")
    srv.stop()
    rep_vals = [r["value"] for r in reps]
    served_mixed_cmp = statistics.median(rep_vals)

    # ---- the comparison jobs one after another on one stream (profiled): kernel breakdown, roofline ----
    ctx.set_profiling(True)
    job_ev = [torch.cuda.Event(enable_timing=True) for _ in range(len(cmp_jobs) + 1)]
    job_pairs, job_stats = [], []
    ev_mixed = torch.empty((len(cmp_jobs), NEV), dtype=torch.float64, device="cuda")
    torch.cuda.synchronize()
    if nvtx is not None:
        nvtx.range_push("sequential")
    for i, (h, seed, eps) in enumerate(cmp_jobs):
        job_ev[i].record()
        nc, st = device_job(h, seed, eps, g.MBL_PREC_FP32)
        job_pairs.append(nc)
        job_stats.append(st)
        ev_mixed[i].copy_(d_ev)
    job_ev[-1].record()
    torch.cuda.synchronize()
    if nvtx is not None:
        nvtx.range_pop()
    job_ms = [job_ev[i].elapsed_time(job_ev[i + 1]) for i in range(len(cmp_jobs))]
    prof = {k: ctx.profile(k) for k in PROF_KEYS}
    ctx.set_profiling(False)
    seq_mixed = sum(job_pairs) / (sum(job_ms) / 1e3)

    # mixed against FP64 eigenvalues, per job (served FP64 results), relative to ||H||
    dev_vs_fp64 = []
    for i, (h, seed, eps) in enumerate(cmp_jobs):
        sec = g.build_sector(ctx, L, h, seed)
        lo, hi = g.extremal_bounds(sec)
        sec.close()
        hn_i = max(abs(lo), abs(hi))
        d = float(np.abs(ev_mixed[i].cpu().numpy() - s64_res[i].evals).max()) / hn_i
        job_stats[i]["max_dev_vs_fp64"] = d
        dev_vs_fp64.append(d)

    # ---- sequential FP64 and split-BF16 on every stride-th comparison job ----
    seq = None
    sub = list(range(0, len(cmp_jobs), args.fp64_stride)) if args.fp64_stride > 0 else []
    if sub:
        a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        torch.cuda.synchronize()
        a.record()
        p64 = 0
        for i in sub:
            nc, st = device_job(*cmp_jobs[i], g.MBL_PREC_FP64)
            p64 += nc
        b.record()
        torch.cuda.synchronize()
        t64 = a.elapsed_time(b)
        a.record()
        pbf, bf_solves, bf_dev = 0, 0, 0.0
        for i in sub:
            nc, st = device_job(*cmp_jobs[i], g.MBL_PREC_FP32, tc=2)
            pbf += nc
            bf_solves += st["solves"]
            bf_dev = max(bf_dev, float(np.abs(d_ev.cpu().numpy() - s64_res[i].evals).max()))
        b.record()
        torch.cuda.synchronize()
        tbf = a.elapsed_time(b)
        t_mixed = sum(job_ms[i] for i in sub)
        p_mixed = sum(job_pairs[i] for i in sub)
        seq = {"jobs": len(sub), "mixed": p_mixed / (t_mixed / 1e3), "fp64": p64 / (t64 / 1e3),
               "bf16x3": pbf / (tbf / 1e3), "mixed_over_fp64": (p_mixed / t_mixed) / max(p64 / t64, 1e-30),
               "ms_per_job": {"mixed": t_mixed / len(sub), "fp64": t64 / len(sub), "bf16x3": tbf / len(sub)},
               "solves": {"tf32x3": sum(job_stats[i]["solves"] for i in sub), "bf16x3": bf_solves}}

    # ---- end to end: the timed served region itself, on the host clock ----
    h2d_job = L * 8
    d2h_job = 8 * (NEV * 4 + (NEV - 2) + n * NEV)
    # host wall of the timed served region: fields h_i in per job; eigenvalues, residuals,
    # observables and eigenvectors back to host memory
    e2e = {"value": pairs / t_host, "unit": "eigenpairs/s", "h2d_bytes_per_step": h2d_job * args.batch,
           "d2h_bytes_per_step": d2h_job * args.batch}

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
        roof = {"bound": "hbm", "unit": "GB/s", "peak_source": "of measured copy" if peaks else "of fallback"}
    elif dom == "schur_tc":
        achieved = per_launch_work / (per_launch_ms / 1e3) / 1e12
        bf = (peaks or {}).get("bf16_tflops", 1900.0)
        peak = bf * 1.1 / 2.25
        roof = {"bound": "tensor", "unit": "TFLOP/s",
                "peak_source": "of measured BF16 x nominal TF32/BF16 (1.1/2.25)" if peaks else "of fallback"}
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
        traffic = profiled_traffic("solve_l18_fp32_traffic.md", per_launch_work)
    roof.update({"achieved": achieved, "peak": peak, "frac": achieved / peak, "traffic": traffic, "kernel": dom,
                 "launch_ms": per_launch_ms, "work_per_launch": per_launch_work})
    roof_seq = {"kernel": dom, "achieved": achieved, "frac": achieved / peak, "launch_ms": per_launch_ms}
    if served_solve["solve_batches"] > 0 and dom == "trisolve_fp32":
        # the served form's solves: one launch of the batched sequence per batch of jobs, timed with
        # CUDA events on the batcher's stream inside the timed region
        nb = served_solve["solve_batches"]
        kmean = served_solve["batched_solves"] / nb
        per_launch_ms = served_solve["batch_ms"] / nb
        per_launch_work = served_solve["batch_bytes"] / nb
        achieved = per_launch_work / (per_launch_ms / 1e3) / 1e9
        traffic = profiled_traffic("solve_l18_fp32_batch_traffic.md", per_launch_work / kmean)
        traffic = traffic * kmean if traffic is not None else None
        roof = {"bound": "hbm", "unit": "GB/s", "peak_source": roof["peak_source"], "achieved": achieved,
                "peak": peak, "frac": achieved / peak, "traffic": traffic,
                "kernel": "trisolve_fp32 batched (served, timed region)", "launch_ms": per_launch_ms,
                "work_per_launch": per_launch_work, "jobs_per_launch": kmean, "launches": nb,
                "sequential": roof_seq}
        if served_solve["batch_busy_ms"] > 0:
            # all batches' bytes over the time during which at least one was executing: the lanes'
            # batches overlap, so this is the class's aggregate rate, where `achieved` is per launch
            agg = served_solve["batch_bytes"] / (served_solve["batch_busy_ms"] / 1e3) / 1e9
            roof["aggregate"] = {"achieved": agg, "frac": agg / peak, "busy_ms": served_solve["batch_busy_ms"]}

    if rank == 0:
        nj = len(cmp_jobs)
        line = {
            "metric": METRIC, "value": value, "unit": "eigenpairs/s", "n_gpus": args.gpus, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": tmax / args.steps, "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "f32 fronts + f64 refinement", "data": "synthetic",
            "config": {"workload": WORKLOAD + f"; served on {args.slots} worker streams", "L": L, "nev": NEV,
                       "jobs_per_step": args.batch, "slots": args.slots, "parallelism": f"replicas x{world}",
                       "l2": "inputs > L2 (factor > 0.3 GB/job)", "ordering": f"{args.ordering} ({ordering_used}, nnz(L) = {int(plan['nnz_l'])})"},
            "gpu_launches": launches,
            "clocks": clocks.summary(local),
            "latency_ms": {"p50": _pct(main_run["lat_ms"], 0.5), "p99": _pct(main_run["lat_ms"], 0.99)},
            "jobs": {"n": len(served_res), "converged": sum(r.nconv for r in served_res),
                     "requested": NEV * len(served_res), "min_nconv": min(r.nconv for r in served_res),
                     "max_resid_over_H": max(float(s["max_resid"]) for s in job_stats),
                     "fp64_fallbacks": sum(int(s["fp64_fallback"]) for s in job_stats)},
            "repeats": {"n": len(rep_vals), "jobs": nj, "values": [round(v, 2) for v in rep_vals],
                        "spread": (max(rep_vals) - min(rep_vals)) / statistics.median(rep_vals)},
            "mixed_vs_fp64": {"jobs": nj, "served_mixed": served_mixed_cmp, "served_fp64": s64["value"],
                              "served_ratio": served_mixed_cmp / max(s64["value"], 1e-30),
                              "fp64_converged": s64["pairs"], "max_eval_dev_over_H": max(dev_vs_fp64),
                              "sequential": seq},
            "ms_per_job": {k: round(prof[k]["ms"] / nj, 2) for k in BREAKDOWN},
            "sequential_mixed": {"value": seq_mixed, "ms_per_job": sum(job_ms) / nj,
                                 "solves_per_job": sum(s["solves"] for s in job_stats) / nj},
            "served": {"host_s": t_host, "peak_reserved_gb": srv_stats["peak_reserved_bytes"] / 1e9},
            "roofline": roof,
            "e2e": e2e,
            "cpu_baseline": cpu,
            "detail": args.detail,
        }
        detail = {"per_job": [{"h": j[0], "seed": j[1], "eps": j[2], "nconv": job_pairs[i], "ms": job_ms[i],
                               **{k: v for k, v in job_stats[i].items()}} for i, j in enumerate(cmp_jobs)],
                  "served_latency_ms": main_run["lat_ms"], "profile": prof, "line": line}
        try:
            with open(args.detail, "w") as fo:
                json.dump(detail, fo)
        except OSError:
            line["detail"] = None
        sys.stdout.flush()
        print(json.dumps(_round_floats(line)), flush=True)
    if dist:
        dist.destroy_process_group()
    return 0


if __name__ == "__main__":
    sys.exit(main())
