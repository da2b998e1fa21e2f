"""GPU path versus stored oracle results at the workload sizes (needs a GB300).

tests/golden/oracle_L16.json and oracle_L18.json were written by tests/golden/make_golden.py from
the CPU oracle alone (minimum-degree LDL^T shift-invert Lanczos, Rayleigh-Ritz on H).  The GPU
runs the same jobs in the configuration the benchmark times (FP32 fronts with FP64 refinement,
block 8) and, at L=18, also with FP64 fronts.  Tolerances as in parity.py: sigma and eigenvalues
within 1e-10 ||H||, the same window (edge ties accepted), residuals <= 1e-10 ||H||, gap ratios
within 1e-8 and entropies within 1e-8 for well-conditioned eigenvectors.
"""
import json
import os

import numpy as np
import pytest

from parity import EIG_TOL, OBS_TOL, well_conditioned

pytestmark = pytest.mark.gpu

GOLD = os.path.join(os.path.dirname(__file__), "golden")


def _jobs(name):
    with open(os.path.join(GOLD, f"oracle_{name}.json")) as f:
        return json.load(f)["jobs"]


CASES = [(j, 1) for j in _jobs("L16")] + [(j, p) for j in _jobs("L18") for p in (1, 0)]


@pytest.fixture(scope="module")
def g():
    import paper_1411_0660_gb300 as g

    return g


@pytest.fixture(scope="module")
def ctx(g):
    c = g.Context(0)
    yield c
    c.close()


@pytest.mark.parametrize("job,prec", CASES,
                         ids=[f"L{j['L']}-h{j['h']}-s{j['seed']}-e{j['eps']}-{'fp32' if p else 'fp64'}"
                              for j, p in CASES])
def test_matches_stored_oracle(g, ctx, job, prec):
    L, h, seed, eps, nev = job["L"], job["h"], job["seed"], job["eps"], job["nev"]
    hn = max(abs(job["emin"]), abs(job["emax"]))
    sec = g.build_sector(ctx, L, h, seed)
    lo, hi = g.extremal_bounds(sec)
    assert abs(lo - job["emin"]) <= EIG_TOL * hn and abs(hi - job["emax"]) <= EIG_TOL * hn
    res = g.solve_near(sec, eps, nev, precision=prec)
    r, rm, s1, se = g.observables(ctx, L, res.evals, res.evecs)
    sec.close()
    assert res.nconv == nev
    assert abs(res.sigma - job["sigma"]) <= EIG_TOL * hn
    ev_o = np.asarray(job["evals"])
    # both are the nev nearest eigenvalues: pair them in ascending order unless the window edge
    # has a tie (then every GPU value must sit on an oracle value)
    d = np.abs(np.sort(res.evals) - np.sort(ev_o))
    if d.max() > EIG_TOL * hn:
        near = np.array([np.min(np.abs(ev_o - x)) for x in res.evals])
        assert near.max() <= EIG_TOL * hn
        pytest.skip("window edge tie: eigenvalues matched individually, observables not paired")
    assert np.max(res.resid) <= EIG_TOL * hn
    r_o = np.array([np.nan if x is None else x for x in job["r"]])
    both = ~np.isnan(r_o) & ~np.isnan(r)
    assert np.max(np.abs(r[both] - r_o[both]), initial=0.0) <= OBS_TOL
    ok = well_conditioned(ev_o, res.evals, res.resid) & well_conditioned(ev_o, ev_o, np.asarray(job["resid"]))
    assert np.max(np.abs(s1 - np.asarray(job["s1p"]))[ok], initial=0.0) <= OBS_TOL
    assert np.max(np.abs(se - np.asarray(job["se"]))[ok], initial=0.0) <= OBS_TOL
