"""Disorder averaging and finite-size-scaling collapse of the eigenpair observables.

The numerical-method section of arXiv:1411.0660 averages each observable over the eigenstates of a
target packet and over disorder realizations; since eigenstates of one realization are correlated,
the values are first averaged per realization (one bin each) and the error bar is the standard error
over these bins.  Its supplement extracts h_c and nu from the scaling ansatz Q = g[(h - h_c) L^(1/nu)]
with g a polynomial of degree three, fitted in a window of half-width w (0.8) in h around h_c and for
L >= L_min, and estimates the statistical error of (h_c, nu) by a bootstrap over realizations.

This module runs such a campaign through the library's server (every eigenpair and observable comes
from the GPU path) and does the statistics on the host with numpy:

    ctx = Context(0)
    data = run_campaign(ctx, Ls=[12, 14, 16], hs=[2, 2.5, 3, 3.5, 4, 4.5, 5], seeds=range(40),
                        eps=0.5, nev=20, observable="r")
    fit = collapse_fit(*points(data), w=0.8, L_min=12)
"""
from __future__ import annotations

import math

import numpy as np


# ---------------------------------------------------------------------------------------------
# binning over realizations
# ---------------------------------------------------------------------------------------------
def realization_mean(values) -> float:
    """The bin of one realization: the mean of an observable over its eigenstates (NaN entries, e.g.
    gap ratios of exactly degenerate levels, are left out)."""
    v = np.asarray(values, dtype=np.float64)
    v = v[~np.isnan(v)]
    return float(v.mean()) if len(v) else math.nan


def mean_stderr(bins):
    """Mean and standard error (sample standard deviation / sqrt(count)) of per-realization bins."""
    b = np.asarray(bins, dtype=np.float64)
    b = b[~np.isnan(b)]
    if len(b) == 0:
        return math.nan, math.nan
    if len(b) == 1:
        return float(b[0]), math.nan
    return float(b.mean()), float(b.std(ddof=1) / math.sqrt(len(b)))


def points(data, observable: str | None = None):
    """Arrays (L, h, Q, dQ) of the campaign's (L, h) means and standard errors."""
    keys = sorted(data["bins"])
    L = np.array([k[0] for k in keys], dtype=np.float64)
    h = np.array([k[1] for k in keys], dtype=np.float64)
    ms = [mean_stderr(data["bins"][k]) for k in keys]
    return L, h, np.array([m for m, _ in ms]), np.array([s for _, s in ms])


# ---------------------------------------------------------------------------------------------
# scaling collapse
# ---------------------------------------------------------------------------------------------
def _chi2(hc, nu, L, h, Q, dQ, w, deg=3):
    """Weighted least-squares misfit of the points with |h - h_c| <= w to a polynomial of degree `deg`
    in x = (h - h_c) L^(1/nu); returns (chi2, points used, coefficients)."""
    m = np.abs(h - hc) <= w
    if m.sum() <= deg + 1:
        return math.inf, int(m.sum()), None
    x = (h[m] - hc) * L[m] ** (1.0 / nu)
    wt = 1.0 / dQ[m]
    A = np.vander(x, deg + 1, increasing=True) * wt[:, None]
    b = Q[m] * wt
    coef, *_ = np.linalg.lstsq(A, b, rcond=None)
    r = A @ coef - b
    return float(r @ r), int(m.sum()), coef


def collapse_fit(L, h, Q, dQ, w: float = 0.8, L_min: float = 0, hc_range=(1.0, 6.0), nu_range=(0.3, 3.0),
                 deg: int = 3):
    """Best (h_c, nu) of the ansatz Q = g[(h - h_c) L^(1/nu)], g a polynomial of degree `deg` fitted in
    the window |h - h_c| <= w over the sizes L >= L_min, by minimizing the weighted misfit per degree
    of freedom: a grid over (h_c, nu) in the given ranges, then two finer grids around the best point
    (within the ranges; a best point on a range's edge means the data do not fix that parameter)."""
    L, h, Q, dQ = (np.asarray(a, dtype=np.float64) for a in (L, h, Q, dQ))
    keep = (L >= L_min) & np.isfinite(Q) & np.isfinite(dQ) & (dQ > 0)
    L, h, Q, dQ = L[keep], h[keep], Q[keep], dQ[keep]

    def score(hc, nu):
        c2, npts, _ = _chi2(hc, nu, L, h, Q, dQ, w, deg)
        dof = npts - (deg + 1) - 2
        return c2 / dof if dof > 0 else math.inf

    best = (math.inf, None, None)
    hc_lo, hc_hi = hc_range
    nu_lo, nu_hi = nu_range
    for hstep, nstep in ((0.05, 0.05), (0.01, 0.01), (0.002, 0.002)):
        for hc in np.arange(hc_lo, hc_hi + 1e-12, hstep):
            for nu in np.arange(nu_lo, nu_hi + 1e-12, nstep):
                s = score(hc, nu)
                if s < best[0]:
                    best = (s, float(hc), float(nu))
        if best[1] is None:
            break
        # finer grids around the best point, within the given ranges
        hc_lo, hc_hi = max(hc_range[0], best[1] - 5 * hstep), min(hc_range[1], best[1] + 5 * hstep)
        nu_lo, nu_hi = max(nu_range[0], best[2] - 5 * nstep), min(nu_range[1], best[2] + 5 * nstep)
    if best[1] is None:
        raise ValueError("collapse_fit: too few points in the window")
    c2, npts, coef = _chi2(best[1], best[2], L, h, Q, dQ, w, deg)
    return {"hc": best[1], "nu": best[2], "chi2_per_dof": best[0], "points": npts, "coef": coef.tolist()}


def bootstrap_fit(data, samples: int = 100, seed: int = 0, **fit_kw):
    """Statistical error of (h_c, nu): the collapse refitted on `samples` resamplings of the
    realizations of every (L, h) (drawn with replacement), standard deviations of the fits."""
    rng = np.random.default_rng(seed)
    hcs, nus = [], []
    keys = sorted(data["bins"])
    for _ in range(samples):
        L, h, Q, dQ = [], [], [], []
        for k in keys:
            b = np.asarray(data["bins"][k], dtype=np.float64)
            b = b[~np.isnan(b)]
            if len(b) < 2:
                continue
            m, s = mean_stderr(b[rng.integers(0, len(b), len(b))])
            if not (s > 0):
                continue
            L.append(k[0])
            h.append(k[1])
            Q.append(m)
            dQ.append(s)
        try:
            f = collapse_fit(L, h, Q, dQ, **fit_kw)
        except ValueError:
            continue
        hcs.append(f["hc"])
        nus.append(f["nu"])
    return {"hc_std": float(np.std(hcs, ddof=1)) if len(hcs) > 1 else math.nan,
            "nu_std": float(np.std(nus, ddof=1)) if len(nus) > 1 else math.nan, "fits": len(hcs)}


# ---------------------------------------------------------------------------------------------
# the campaign on the GPU
# ---------------------------------------------------------------------------------------------
OBSERVABLES = ("r", "s1p", "se_per_site")


def run_campaign(ctx, Ls, hs, seeds, eps: float = 0.5, nev: int = 20, observable: str = "r", slots: int = 8,
                 precision: int | None = None):
    """Every (L, h, seed) job through the server (continuous batching over `slots` workers); per job
    the bin of `observable` over its nev eigenstates (gap ratio r, participation entropy S_1^P, or
    entanglement entropy per site S_E / L).  Returns {"bins": {(L, h): [bin per realization]},
    "jobs", "converged", "seconds"}."""
    import time

    from . import MBL_PREC_FP32, Server

    if observable not in OBSERVABLES:
        raise ValueError(f"observable must be one of {OBSERVABLES}")
    srv = Server(ctx, slots=slots)
    jobs = [(L, float(h), int(s)) for L in Ls for h in hs for s in seeds]
    t0 = time.perf_counter()
    tickets = [srv.submit(L, h, s, eps, nev, precision=MBL_PREC_FP32 if precision is None else precision)
               for (L, h, s) in jobs]
    bins: dict = {}
    conv = 0
    for (L, h, s), t in zip(jobs, tickets):
        res = srv.wait(t)
        conv += res.nconv
        if observable == "r":
            v = res.r
        elif observable == "s1p":
            v = res.s1p
        else:
            v = res.se / L
        bins.setdefault((L, h), []).append(realization_mean(v))
    dt = time.perf_counter() - t0
    srv.stop()
    return {"bins": bins, "jobs": len(jobs), "converged": conv, "requested": nev * len(jobs), "seconds": dt,
            "eps": eps, "nev": nev, "observable": observable}
