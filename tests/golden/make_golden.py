"""Write oracle results for sizes the oracle cannot redo inside a test (L = 14, 16, 18).

Calls only the CPU oracle (oracle/); nothing here comes from the GPU path.  Each job is
(L, h, seed, eps, nev); the file keeps E_min, E_max, sigma, the nev eigenvalues nearest sigma,
their residuals, the gap ratios and S_1^P / S^E of each eigenvector.  Run:

    python tests/golden/make_golden.py L14        # 9 jobs, seconds
    python tests/golden/make_golden.py L16        # 9 jobs, minutes
    python tests/golden/make_golden.py L18        # 3 jobs, about an hour each on one core
"""
import json
import multiprocessing as mp
import os
import sys
import time

HERE = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, os.path.dirname(os.path.dirname(HERE)))

SETS = {
    # the same shape at L=14 (the reference arm's per-step sample when many steps are asked for)
    "L14": [(14, h, 0, eps, 50) for h in (1.0, 2.5, 4.0) for eps in (0.1, 0.5, 0.9)],
    # the batched L=16 workload shape: h in {1, 2.5, 4}, eps in {0.1, 0.5, 0.9}, nev = 50
    "L16": [(16, h, 0, eps, 50) for h in (1.0, 2.5, 4.0) for eps in (0.1, 0.5, 0.9)],
    # the L=18 workload shape: h in {0.5, 3, 5}, eps in {0.1, 0.5, 0.9}, nev = 50
    "L18": [(18, 0.5, 0, 0.1, 50), (18, 3.0, 0, 0.5, 50), (18, 5.0, 1, 0.9, 50)],
}


def run(job):
    import oracle

    L, h, seed, eps, nev = job
    t = time.time()
    r = oracle.solve_job(oracle.Job(L, h, seed, eps, nev), "si")
    return {
        "L": L, "h": h, "seed": seed, "eps": eps, "nev": nev,
        "emin": r.emin, "emax": r.emax, "sigma": r.sigma,
        "evals": [float(x) for x in r.evals], "resid": [float(x) for x in r.resid],
        "r": [None if x != x else float(x) for x in r.r], "r_mean": r.r_mean,
        "s1p": [float(x) for x in r.s1p], "se": [float(x) for x in r.se],
        "oracle_seconds": time.time() - t,
    }


def main():
    name = sys.argv[1]
    jobs = SETS[name]
    ctx = mp.get_context("spawn")
    with ctx.Pool(min(len(jobs), os.cpu_count() or 1)) as pool:
        out = pool.map(run, jobs)
    doc = {"_source": "oracle/ (plain CPU FP64 shift-invert: minimum-degree LDL^T, Lanczos with full "
                      "reorthogonalization, Rayleigh-Ritz on H), written by tests/golden/make_golden.py",
           "jobs": out}
    with open(os.path.join(HERE, f"oracle_{name}.json"), "w") as f:
        json.dump(doc, f, indent=1)


if __name__ == "__main__":
    main()
