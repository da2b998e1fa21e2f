"""Serving through the C ABI (needs a GB300): requests of mixed L, precision and eps run side by
side on worker streams; each result must equal the single-call result (build_sector + solve_near
+ observables) within the parity tolerances, and the dense oracle at L=12.  HBM admission: a budget
that fits one job at a time serializes the jobs; an oversized request fails with MBL_ERR_OOM.
"""
import numpy as np
import pytest

from parity import EIG_TOL, OBS_TOL, well_conditioned

pytestmark = pytest.mark.gpu

MIX = [  # (L, h, seed, eps, nev, precision)
    (12, 2.0, 0, 0.5, 20, 1),
    (14, 3.0, 1, 0.3, 20, 1),
    (12, 1.0, 2, 0.8, 10, 0),
    (14, 0.5, 3, 0.5, 16, 0),
    (10, 4.0, 4, 0.1, 12, 1),
    (14, 5.0, 5, 0.9, 20, 1),
]


@pytest.fixture(scope="module")
def g():
    import paper_1411_0660_gb300 as g

    return g


@pytest.fixture(scope="module")
def ctx(g):
    c = g.Context(0)
    yield c
    c.close()


def _alone(g, ctx, L, h, seed, eps, nev, prec):
    sec = g.build_sector(ctx, L, h, seed)
    res = g.solve_near(sec, eps, nev, precision=prec)
    r, rm, s1, se = g.observables(ctx, L, res.evals, res.evecs)
    lo, hi = g.extremal_bounds(sec)
    sec.close()
    return res, (r, rm, s1, se), max(abs(lo), abs(hi))


def test_mix_equals_alone(g, ctx, orc):
    srv = g.Server(ctx, slots=3)
    tickets = [srv.submit(L, h, s, e, nev, precision=p, want_vectors=True) for (L, h, s, e, nev, p) in MIX]
    served = [srv.wait(t, 300.0) for t in tickets]
    st = srv.stats()
    srv.stop()
    assert st["completed"] == len(MIX) and st["failed"] == 0
    for job, out in zip(MIX, served):
        L, h, seed, eps, nev, prec = job
        assert out is not None and out.status == 0 and out.nconv == nev
        res, (r, rm, s1, se), hn = _alone(g, ctx, *job)
        assert abs(out.sigma - res.sigma) <= EIG_TOL * hn
        assert np.max(np.abs(out.evals - res.evals)) <= EIG_TOL * hn
        assert np.max(out.resid) <= EIG_TOL * hn
        assert np.max(np.abs(out.r - r)) <= OBS_TOL
        ok = well_conditioned(out.evals, out.evals, out.resid)
        assert np.max(np.abs(out.s1p - s1)[ok], initial=0.0) <= OBS_TOL
        assert np.max(np.abs(out.se - se)[ok], initial=0.0) <= OBS_TOL
        # the served eigenvectors themselves satisfy H y = lambda y
        sec = g.build_sector(ctx, L, h, seed)
        HY = sec.spmv(out.evecs)
        sec.close()
        assert np.max(np.linalg.norm(HY - out.evecs * out.evals, axis=0)) <= EIG_TOL * hn
        if L == 12:
            w = orc.syev(orc.csr(L, orc.fields(L, h, seed)).dense(), vectors=False)
            near = np.sort(w[np.argsort(np.abs(w - out.sigma), kind="stable")[:nev]])
            assert np.max(np.abs(near - out.evals)) <= EIG_TOL * hn


def test_admission_serializes_when_one_job_fits(g, ctx):
    probe = g.Server(ctx, slots=1)
    t = probe.submit(14, 3.0, 7, 0.5, 20)
    one = probe.wait(t, 300.0)
    probe.stop()
    srv = g.Server(ctx, slots=3, hbm_budget_bytes=int(1.5 * one.reserved_bytes))
    ts = [srv.submit(14, 3.0, 7 + k, 0.5, 20) for k in range(3)]
    outs = sorted((srv.wait(t, 300.0) for t in ts), key=lambda o: o.t_admit_ms)
    st = srv.stats()
    srv.stop()
    assert all(o.status == 0 for o in outs)
    assert st["peak_reserved_bytes"] <= int(1.5 * one.reserved_bytes)
    for a, b in zip(outs, outs[1:]):
        assert b.t_admit_ms >= a.t_end_ms - 1e-3  # at most one job holds HBM at a time


def test_jobs_overlap_when_memory_allows(g, ctx):
    srv = g.Server(ctx, slots=3)
    ts = [srv.submit(14, 2.0, 20 + k, 0.5, 20) for k in range(3)]
    outs = [srv.wait(t, 300.0) for t in ts]
    srv.stop()
    assert all(o.status == 0 for o in outs)
    spans = sorted((o.t_admit_ms, o.t_end_ms) for o in outs)
    assert any(spans[i + 1][0] < spans[i][1] for i in range(len(spans) - 1))


def test_oversized_request_and_bad_arguments(g, ctx):
    srv = g.Server(ctx, slots=1, hbm_budget_bytes=1 << 20)
    t = srv.submit(12, 1.0, 0, 0.5, 10)
    with pytest.raises(g.MblError) as e:
        srv.wait(t, 300.0)
    assert e.value.code == 2
    with pytest.raises(g.MblError) as e:
        srv.submit(13, 1.0, 0, 0.5, 10)
    assert e.value.code == 1
    with pytest.raises(g.MblError) as e:
        srv.submit(12, 1.0, 0, 1.5, 10)
    assert e.value.code == 1
    srv.stop()


def test_repeated_request_reuses_the_live_factor(g, ctx, orc):
    """Serving residency: a request identical to a finished one takes its sector and factorization
    from the cache (no new factorization) and returns the same eigenpairs; a cache of size zero never
    reuses; the oracle confirms the reused result."""
    L, h, seed, eps, nev = 14, 2.0, 80, 0.4, 20
    srv = g.Server(ctx, slots=2, cache_fraction=0.25)
    a = srv.wait(srv.submit(L, h, seed, eps, nev, want_vectors=True), 300.0)
    b = srv.wait(srv.submit(L, h, seed, eps, nev, want_vectors=True), 300.0)
    c = srv.wait(srv.submit(L, h, seed + 1, eps, nev), 300.0)  # another realization: no reuse
    st = srv.stats()
    srv.stop()
    assert a.status == 0 and b.status == 0 and c.status == 0
    assert a.factor_reused == 0 and b.factor_reused == 1 and c.factor_reused == 0
    assert st["cache_hits"] == 1
    H = orc.csr(L, orc.fields(L, h, seed))
    emin, emax = orc.extremal_bounds(H)
    hn = max(abs(emin), abs(emax))
    assert np.max(np.abs(a.evals - b.evals)) <= EIG_TOL * hn
    for j in range(nev):
        y = b.evecs[:, j]
        assert np.linalg.norm(H.matvec(y) - b.evals[j] * y) <= EIG_TOL * hn
    srv0 = g.Server(ctx, slots=1, cache_fraction=0.0)
    x = srv0.wait(srv0.submit(L, h, seed, eps, nev), 300.0)
    y = srv0.wait(srv0.submit(L, h, seed, eps, nev), 300.0)
    st0 = srv0.stats()
    srv0.stop()
    assert x.factor_reused == 0 and y.factor_reused == 0 and st0["cache_hits"] == 0
