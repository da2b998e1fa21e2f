"""Disorder averaging and scaling collapse (host statistics, no GPU): per-realization bins and their
standard error against numpy's definitions; the collapse fit recovers (h_c, nu) from data made with a
known scaling function; the bootstrap gives a spread of the order of the noise.  The numerical-method
section (binning per realization, standard error over bins) and its supplement (cubic polynomial in a
window of half-width w around h_c, bootstrap) define the procedure."""
import math

import numpy as np
import pytest

from paper_1411_0660_gb300 import campaign as cp


def test_bins_and_standard_error():
    rng = np.random.default_rng(0)
    per_state = [rng.normal(0.5, 0.1, 20) for _ in range(30)]
    per_state[3][5] = np.nan  # a gap ratio of two exactly degenerate levels
    bins = [cp.realization_mean(v) for v in per_state]
    assert abs(bins[3] - np.nanmean(per_state[3])) < 1e-15
    m, s = cp.mean_stderr(bins)
    assert abs(m - np.mean(bins)) < 1e-15
    assert abs(s - np.std(bins, ddof=1) / math.sqrt(len(bins))) < 1e-15
    assert math.isnan(cp.mean_stderr([0.3])[1])


def _synthetic(hc, nu, Ls, hs, noise, seed, reals=40):
    """Realization bins of Q = g[(h - hc) L^(1/nu)] + noise, g(x) = 0.45 - 0.04 x + 0.002 x^3."""
    rng = np.random.default_rng(seed)
    g = lambda x: 0.45 - 0.04 * x + 0.002 * x ** 3
    bins = {}
    for L in Ls:
        for h in hs:
            q = g((h - hc) * L ** (1.0 / nu))
            bins[(L, h)] = list(q + rng.normal(0.0, noise, reals))
    return {"bins": bins}


def test_collapse_recovers_known_exponents():
    data = _synthetic(3.7, 0.9, [12, 14, 16, 18], np.arange(2.6, 4.81, 0.2), 0.004, 1)
    fit = cp.collapse_fit(*cp.points(data), w=0.8, L_min=12, hc_range=(2.5, 5.0), nu_range=(0.4, 2.0))
    assert abs(fit["hc"] - 3.7) < 0.08 and abs(fit["nu"] - 0.9) < 0.15
    assert fit["chi2_per_dof"] < 3.0
    # the same data with a wrong nu collapse worse
    L, h, Q, dQ = cp.points(data)
    c_true = cp._chi2(3.7, 0.9, L, h, Q, dQ, 0.8)[0]
    c_bad = cp._chi2(3.7, 2.0, L, h, Q, dQ, 0.8)[0]
    assert c_bad > 3 * c_true


def test_bootstrap_spread_is_finite_and_small():
    data = _synthetic(3.2, 0.8, [12, 14, 16], np.arange(2.2, 4.21, 0.25), 0.004, 2, reals=30)
    b = cp.bootstrap_fit(data, samples=20, seed=3, w=0.8, L_min=12, hc_range=(2.2, 4.5), nu_range=(0.4, 2.0))
    assert b["fits"] >= 15
    assert 0.0 < b["hc_std"] < 0.3 and 0.0 < b["nu_std"] < 0.6


def test_fit_rejects_too_few_points():
    with pytest.raises(ValueError):
        cp.collapse_fit([12, 14], [3.0, 3.0], [0.4, 0.5], [0.01, 0.01], w=0.8)
