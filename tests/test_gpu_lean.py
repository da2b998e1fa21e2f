"""Memory-lean fronts arena (needs a GB300).

The lean arena backs each region of fronts with device memory only from its level's assembly to
its parents' assembly, and releases a front's factor columns once they are copied to the solve
factor.  The arithmetic is the same as with the whole arena, so the factorizations must give
bit-identical solves, and a shift-invert job in lean mode must match the oracle.  The analysis must
report a lean peak below the whole arena (the figure that makes the largest sector fit one GPU).
"""
import numpy as np
import pytest

from parity import EIG_TOL, window_equivalent

pytestmark = pytest.mark.gpu

ARENA_LEAN, ARENA_FULL = 1, 2


@pytest.fixture(scope="module")
def g():
    import paper_1411_0660_gb300 as g

    return g


@pytest.fixture(scope="module")
def ctx(g):
    c = g.Context(0)
    yield c
    c.close()


@pytest.mark.parametrize("L,prec,tc", [(14, 1, 1), (14, 0, 1), (16, 1, 1), (16, 1, 2), (13, 1, 1)])
def test_lean_arena_factor_bit_identical(g, ctx, L, prec, tc):
    nup = None if L % 2 == 0 else (L + 1) // 2
    sec = g.build_sector(ctx, L, 2.5, 70, nup=nup)
    lo, hi = g.extremal_bounds(sec)
    sigma = lo + 0.45 * (hi - lo)
    B = np.random.default_rng(11).standard_normal((sec.dim, 8))
    fs = [g.factor(sec, sigma, precision=prec, tensor_cores=tc, arena_mode=m) for m in (ARENA_FULL, ARENA_LEAN)]
    st = [f.stats() for f in fs]
    assert st[0]["perturbed"] == st[1]["perturbed"] and st[0]["negative"] == st[1]["negative"]
    assert st[1]["front_bytes"] < st[0]["front_bytes"]
    X = [f.solve(B, refine=False) for f in fs]
    assert np.array_equal(X[0].view(np.uint64), X[1].view(np.uint64))
    for f in fs:
        f.close()
    sec.close()


def test_lean_arena_solve_near_matches_oracle(g, ctx, orc):
    L, h, seed, eps, nev = 14, 3.0, 71, 0.5, 30
    sec = g.build_sector(ctx, L, h, seed)
    res = g.solve_near(sec, eps, nev, arena_mode=ARENA_LEAN)
    sec.close()
    assert res.nconv == nev
    H = orc.csr(L, orc.fields(L, h, seed))
    emin, emax = orc.extremal_bounds(H)
    hn = max(abs(emin), abs(emax))
    sigma = emin + eps * (emax - emin)
    spectrum = orc.nearest_shift_invert(H, sigma, nev + 12, hn).evals
    assert window_equivalent(res.evals, spectrum, sigma, nev, hn)
    for j in range(nev):
        y = res.evecs[:, j]
        assert np.linalg.norm(H.matvec(y) - res.evals[j] * y) <= EIG_TOL * hn


def test_analysis_reports_lean_peak(g, ctx):
    sec = g.build_sector(ctx, 20, 3.0, 0)
    a = g.analyse(sec, 50, 8)
    sec.close()
    # the whole arena would exceed 8 GiB at L = 20, so the automatic mode is lean
    assert a["front_peak_bytes_fp32"] < 0.5 * a["front_bytes_fp32"]
    assert a["job_peak_bytes_fp32"] < a["front_bytes_fp32"]
    with pytest.raises(g.MblError):
        sec2 = g.build_sector(ctx, 12, 1.0, 0)
        try:
            g.factor(sec2, 0.0, arena_mode=3)
        finally:
            sec2.close()
