"""General magnetization sectors on the GPU versus the oracle (needs a GB300): the odd-L sectors of
the numerical-method section (its "S^z = 1", read as n_up = (L + 1)/2) and sectors away from half
filling.  Same bars as the S^z = 0 parity tests: bit-exact basis, ranks and CSR; eigenvalues within
1e-10 ||H|| and the same window; residuals <= 1e-10 ||H||; observables within 1e-8 for
well-conditioned eigenvectors.
"""
import math

import numpy as np
import pytest

from parity import EIG_TOL, OBS_TOL, well_conditioned, window_equivalent

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def g():
    import paper_1411_0660_gb300 as g

    return g


@pytest.fixture(scope="module")
def ctx(g):
    return g.Context(0)


@pytest.mark.parametrize("L,nup", [(3, 1), (3, 2), (5, 2), (7, 4), (9, 5), (12, 3), (13, 7), (14, 5), (15, 8),
                                   (17, 9), (6, 0), (6, 6)])
def test_sector_basis_rank_csr_bit_exact(g, ctx, orc, L, nup):
    h, seed = 2.5, 300 + L + nup
    sec = g.build_sector(ctx, L, h, seed, nup=nup)
    assert sec.dim == math.comb(L, nup) and sec.nup == nup and sec.L == L
    st = orc.basis(L, nup)
    assert np.array_equal(sec.basis(), st)
    assert np.array_equal(sec.rank(st), np.arange(sec.dim))
    # states of another sector, or with a bit beyond the chain, are not in this one
    bad = np.array([(1 << (nup + 1)) - 1 if nup < L else 0, 1 << L], dtype=np.uint32)
    assert np.all(sec.rank(bad) == -1)
    hi = orc.fields(L, h, seed)
    assert np.array_equal(sec.fields().view(np.uint64), hi.view(np.uint64))
    rp, col, val = sec.csr()
    H = orc.csr(L, hi, 1.0, st)
    assert np.array_equal(rp, H.rowptr) and np.array_equal(col, H.col)
    assert np.array_equal(val.view(np.uint64), H.val.view(np.uint64))
    sec.close()


def test_sector_arguments_are_validated(g, ctx):
    with pytest.raises(g.MblError):
        g.build_sector(ctx, 15, 1.0, 0)  # odd L needs a sector
    with pytest.raises(g.MblError):
        g.build_sector(ctx, 12, 1.0, 0, nup=13)
    with pytest.raises(g.MblError):
        g.build_sector(ctx, 23, 1.0, 0, nup=11)
    with pytest.raises(g.MblError):
        g.observables(ctx, 13, np.zeros(3), np.zeros((1716, 3)))  # odd L without nup


@pytest.mark.parametrize("L,nup,h,seed", [(13, 7, 2.0, 1), (15, 8, 0.5, 2), (14, 4, 3.0, 3)])
def test_sector_extremal_bounds(g, ctx, orc, L, nup, h, seed):
    sec = g.build_sector(ctx, L, h, seed, nup=nup)
    lo, hi = g.extremal_bounds(sec)
    H = orc.csr(L, orc.fields(L, h, seed), 1.0, orc.basis(L, nup))
    if H.n <= 924:
        w = orc.syev(H.dense(), vectors=False)
        wlo, whi = w[0], w[-1]
    else:
        wlo, whi = orc.extremal_bounds(H)
    hn = max(abs(wlo), abs(whi))
    assert abs(lo - wlo) <= 1e-12 * hn and abs(hi - whi) <= 1e-12 * hn


@pytest.mark.parametrize("L,nup,h,seed,eps,nev,prec", [
    (13, 7, 2.0, 11, 0.5, 20, 0),
    (13, 7, 3.0, 12, 0.2, 50, 1),
    (11, 4, 1.0, 13, 0.7, 30, 1),
    (15, 8, 3.0, 14, 0.5, 50, 1),
])
def test_sector_solve_near_and_observables(g, ctx, orc, L, nup, h, seed, eps, nev, prec):
    sec = g.build_sector(ctx, L, h, seed, nup=nup)
    res = g.solve_near(sec, eps, nev, precision=prec)
    st = orc.basis(L, nup)
    H = orc.csr(L, orc.fields(L, h, seed), 1.0, st)
    if H.n <= 3432:
        spectrum = orc.syev(H.dense(), vectors=False)
        sigma = spectrum[0] + eps * (spectrum[-1] - spectrum[0])
        hn = max(abs(spectrum[0]), abs(spectrum[-1]))
    else:
        emin, emax = orc.extremal_bounds(H)
        sigma = emin + eps * (emax - emin)
        hn = max(abs(emin), abs(emax))
        spectrum = orc.nearest_shift_invert(H, sigma, nev + 12, hn).evals
    assert abs(res.sigma - sigma) <= 1e-12 * hn
    assert res.nconv == nev
    assert window_equivalent(res.evals, spectrum, sigma, nev, hn)
    Y = res.evecs
    res_o = np.array([np.linalg.norm(H.matvec(Y[:, j]) - res.evals[j] * Y[:, j]) for j in range(nev)])
    assert np.all(res_o <= EIG_TOL * hn)
    assert np.abs(Y.T @ Y - np.eye(nev)).max() < 1e-10
    r_g, rm_g, s1_g, se_g = g.observables(ctx, L, res.evals, Y, nup=nup)
    r_o, rm_o = orc.gap_ratio(res.evals)
    assert np.allclose(r_g, r_o, atol=1e-12, equal_nan=True)
    kl_g, sq_g, fl_g, df_g = g.observables_extra(ctx, L, Y, 2.0, nup=nup)
    # the vectors compared are chosen by the oracle's residuals, not the GPU's own report
    mask = well_conditioned(spectrum, res.evals, res_o)
    for j in np.nonzero(mask)[0]:
        y = Y[:, j]
        assert abs(s1_g[j] - orc.s1p(y)) <= OBS_TOL
        assert abs(se_g[j] - orc.entanglement(L, y, st)) <= OBS_TOL
        assert abs(sq_g[j] - orc.sqp(y, 2.0)) <= OBS_TOL
        assert abs(fl_g[j] - orc.fluct(L, y, st)) <= OBS_TOL
        assert abs(df_g[j] - orc.dynf(L, y, st)) <= OBS_TOL
    for j in range(nev - 1):
        if mask[j] and mask[j + 1]:
            assert abs(kl_g[j] - orc.kl(Y[:, j], Y[:, j + 1])) <= 1e-8 * max(1.0, abs(kl_g[j]))
    sec.close()


def test_sector_jobs_through_the_server(g, ctx, orc):
    """An odd-L job and an off-half-filling job served side by side give the direct path's
    eigenvalues and observables."""
    jobs = [(13, 7, 2.0, 21, 0.5), (12, 4, 1.5, 22, 0.3)]
    srv = g.Server(ctx, slots=2)
    tickets = [srv.submit(L, h, seed, eps, 20, want_vectors=True, nup=nup) for (L, nup, h, seed, eps) in jobs]
    out = [srv.wait(t) for t in tickets]
    srv.stop()
    for (L, nup, h, seed, eps), r in zip(jobs, out):
        assert r.status == 0 and r.nconv == 20 and r.dim == math.comb(L, nup)
        sec = g.build_sector(ctx, L, h, seed, nup=nup)
        d = g.solve_near(sec, eps, 20)
        hn = max(abs(v) for v in g.extremal_bounds(sec))
        assert np.abs(np.sort(r.evals) - np.sort(d.evals)).max() <= 1e-10 * hn
        st = orc.basis(L, nup)
        H = orc.csr(L, orc.fields(L, h, seed), 1.0, st)
        for j in range(20):
            y = r.evecs[:, j]
            assert np.linalg.norm(H.matvec(y) - r.evals[j] * y) <= EIG_TOL * hn
        sec.close()
    with pytest.raises(g.MblError):
        srv2 = g.Server(ctx, slots=1)
        try:
            srv2.submit(13, 1.0, 0, 0.5, 10)  # odd L needs nup
        finally:
            srv2.stop()
