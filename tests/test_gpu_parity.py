"""GPU path versus the CPU oracle, element by element, through the C ABI (needs a GB300).

Bit-exact: fields, basis, ranks, CSR.  Floating point: eigenvalues within 1e-10 ||H||, the same
window (ties at the edge accepted), residuals <= 1e-10 ||H||, observables within 1e-8 for
well-conditioned eigenvectors (see parity.py).
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


# ---------------------------------------------------------------- bit-exact setup ----------
@pytest.mark.parametrize("L", [2, 4, 6, 10, 14, 18, 22])
def test_fields_basis_rank_bit_exact(g, ctx, orc, L):
    sec = g.build_sector(ctx, L, 2.5, 1000 + L)
    assert np.array_equal(sec.fields().view(np.uint64), orc.fields(L, 2.5, 1000 + L).view(np.uint64))
    st = sec.basis()
    assert sec.dim == math.comb(L, L // 2)
    if L <= 20:
        assert np.array_equal(st, orc.basis(L))
    r = sec.rank(st)
    assert np.array_equal(r, np.arange(sec.dim))
    # wrong popcount (0, all up, L/2 + 1 up) or a bit beyond the chain
    bad = np.array([0, (1 << L) - 1, (1 << (L // 2 + 1)) - 1, ((1 << (L // 2)) - 1) << (32 - L // 2)],
                   dtype=np.uint32)
    assert np.all(sec.rank(bad) == -1)


@pytest.mark.parametrize("L,h,seed,J", [(2, 1.0, 3, 1.0), (4, 0.0, 0, 1.0), (8, 3.0, 5, 0.7), (12, 2.0, 0, 1.0),
                                        (16, 5.0, 11, 1.0)])
def test_csr_bit_exact(g, ctx, orc, L, h, seed, J):
    hi = orc.fields(L, h, seed)
    sec = g.build_sector_fields(ctx, L, hi, J) if J != 1.0 else g.build_sector(ctx, L, h, seed)
    rp, col, val = sec.csr()
    H = orc.csr(L, hi, J)
    assert np.array_equal(rp, H.rowptr)
    assert np.array_equal(col, H.col)
    assert np.array_equal(val.view(np.uint64), H.val.view(np.uint64))


def test_spmv(g, ctx, orc):
    L = 14
    sec = g.build_sector(ctx, L, 3.0, 2)
    H = orc.csr(L, orc.fields(L, 3.0, 2))
    X = np.random.default_rng(0).standard_normal((sec.dim, 5))
    Y = sec.spmv(X, shift=0.37)
    for q in range(5):
        want = H.matvec(X[:, q], 0.37)
        assert np.abs(Y[:, q] - want).max() <= 1e-13 * np.abs(want).max()


# ---------------------------------------------------------------- extremal bounds ----------
@pytest.mark.parametrize("L,h,seed", [(4, 1.0, 0), (8, 2.0, 1), (10, 0.5, 2), (12, 3.0, 3), (14, 5.0, 4), (16, 0.5, 5)])
def test_extremal_bounds(g, ctx, orc, L, h, seed):
    sec = g.build_sector(ctx, L, h, seed)
    lo, hi = g.extremal_bounds(sec)
    H = orc.csr(L, orc.fields(L, h, seed))
    if H.n <= 924:
        w = orc.syev(H.dense(), vectors=False)
        wlo, whi = w[0], w[-1]
    else:
        wlo, whi = orc.extremal_bounds(H)
    hn = max(abs(wlo), abs(whi))
    assert abs(lo - wlo) <= 1e-12 * hn and abs(hi - whi) <= 1e-12 * hn


# ---------------------------------------------------------------- factorization -------------
@pytest.mark.parametrize("prec", [0, 1])
@pytest.mark.parametrize("L,h,seed,eps", [(12, 2.0, 0, 0.5), (14, 3.0, 1, 0.3), (16, 1.0, 2, 0.7)])
def test_factor_solve_and_inertia(g, ctx, orc, prec, L, h, seed, eps):
    sec = g.build_sector(ctx, L, h, seed)
    lo, hi = g.extremal_bounds(sec)
    sigma = lo + eps * (hi - lo)
    f = g.factor(sec, sigma, precision=prec)
    st = f.stats()
    assert st["n"] == sec.dim and st["nnz_l"] > 0 and st["max_front"] > 0
    H = orc.csr(L, orc.fields(L, h, seed))
    B = np.random.default_rng(1).standard_normal((sec.dim, 3))
    X = f.solve(B, refine=True)
    hn = max(abs(lo), abs(hi))
    for q in range(3):
        r = H.matvec(X[:, q], sigma) - B[:, q]
        assert np.linalg.norm(r) <= 1e-13 * ((hn + abs(sigma)) * np.linalg.norm(X[:, q]) + np.linalg.norm(B[:, q]))
    if prec == 0 and L <= 14 and st["perturbed"] == 0:
        w = orc.syev(H.dense(), vectors=False) if L <= 12 else None
        if w is not None:
            assert st["negative"] == int(np.sum(w < sigma))


@pytest.mark.parametrize("prec", [0, 1])
def test_factor_solve_dev_matches_host(g, ctx, orc, prec):
    """The device-array solve runs the same kernels as the host-array one: bit-identical unrefined
    blocks (40 right-hand sides: a block of 32 and a ragged block of 8), refined solves to the
    refinement tolerance."""
    import torch

    L, h, seed = 14, 2.0, 7
    sec = g.build_sector(ctx, L, h, seed)
    lo, hi = g.extremal_bounds(sec)
    sigma = lo + 0.4 * (hi - lo)
    f = g.factor(sec, sigma, precision=prec)
    B = np.random.default_rng(3).standard_normal((sec.dim, 40))
    d_b = torch.from_numpy(np.asfortranarray(B).ravel(order="F")).cuda()
    d_x = torch.zeros_like(d_b)
    f.solve_dev(d_b, d_x, 40, refine=False)
    torch.cuda.synchronize()
    X = d_x.cpu().numpy().reshape(40, sec.dim).T
    assert np.array_equal(X, f.solve(B, refine=False))
    f.solve_dev(d_b, d_x, 40, refine=True)
    torch.cuda.synchronize()
    X = d_x.cpu().numpy().reshape(40, sec.dim).T
    H = orc.csr(L, orc.fields(L, h, seed))
    hn = max(abs(lo), abs(hi))
    for q in (0, 17, 39):
        r = H.matvec(X[:, q], sigma) - B[:, q]
        assert np.linalg.norm(r) <= 1e-13 * ((hn + abs(sigma)) * np.linalg.norm(X[:, q]) + np.linalg.norm(B[:, q]))
    with pytest.raises(g.MblError):
        f.solve_dev(d_b, d_x, 0)
    f.close()
    sec.close()


def test_bounds_factor_and_solves_are_bit_reproducible(g, ctx):
    """The extremal bounds, the factorization (every Schur-update mode) and the unrefined and
    refined block solves give the same bits when repeated: none of their reductions depends on
    the order in which CTAs or warps run."""
    L, h, seed = 14, 5.0, 23
    b = []
    for _ in range(2):
        sec = g.build_sector(ctx, L, h, seed)
        b.append(g.extremal_bounds(sec))
        sec.close()
    assert b[0] == b[1]
    sec = g.build_sector(ctx, L, h, seed)
    lo, hi = b[0]
    sigma = lo + 0.1 * (hi - lo)
    B = np.random.default_rng(4).standard_normal((sec.dim, 8))
    for kw in (dict(precision=1, tensor_cores=1), dict(precision=1, tensor_cores=0), dict(precision=0)):
        xs = []
        for _ in range(2):
            f = g.factor(sec, sigma, **kw)
            xs.append(f.solve(B, refine=False))
            xs.append(f.solve(B, refine=False))
            f.close()
        for x in xs[1:]:
            assert np.array_equal(x.view(np.uint64), xs[0].view(np.uint64))
    f = g.factor(sec, sigma, precision=1)
    xr = [f.solve(B, refine=True) for _ in range(2)]
    assert np.array_equal(xr[0].view(np.uint64), xr[1].view(np.uint64))
    f.close()
    sec.close()


@pytest.mark.parametrize("L,h,seed,eps,prec", [(14, 1.0, 3, 0.5, 1), (14, 1.0, 3, 0.5, 0), (16, 5.0, 1023, 0.1, 1)])
def test_solve_near_is_bit_reproducible(g, ctx, L, h, seed, eps, prec):
    """Two whole shift-invert runs on the same sector, and a third on a freshly built copy of it,
    return the same bits: eigenvalues, eigenvectors and residuals, and the same solve count.  Every
    reduction of the Krylov layer (block Gram-Schmidt, the projected matrix, the small eigensolves,
    the refinement's norms) sums in an order that does not depend on how CTAs or warps are scheduled."""
    sec = g.build_sector(ctx, L, h, seed)
    rs = [g.solve_near(sec, eps, 30, precision=prec) for _ in range(2)]
    sec.close()
    sec = g.build_sector(ctx, L, h, seed)
    rs.append(g.solve_near(sec, eps, 30, precision=prec))
    sec.close()
    for r in rs[1:]:
        assert r.stats["solves"] == rs[0].stats["solves"]
        assert np.array_equal(r.evals.view(np.uint64), rs[0].evals.view(np.uint64))
        assert np.array_equal(r.evecs.view(np.uint64), rs[0].evecs.view(np.uint64))
        assert np.array_equal(r.resid.view(np.uint64), rs[0].resid.view(np.uint64))


# ---------------------------------------------------------------- eigenpairs + observables ---
def _reference(orc, H, L, eps, nev):
    """Oracle spectrum around sigma: the full dense spectrum up to L = 12, else the nev + 12
    eigenvalues nearest sigma from the oracle's shift-invert path (enough to test the window and the
    gaps of every wanted level)."""
    if H.n <= 924:
        w = orc.syev(H.dense(), vectors=False)
        return w, w[0] + eps * (w[-1] - w[0]), max(abs(w[0]), abs(w[-1]))
    emin, emax = orc.extremal_bounds(H)
    sigma = emin + eps * (emax - emin)
    hn = max(abs(emin), abs(emax))
    e = orc.nearest_shift_invert(H, sigma, min(H.n, nev + 12), hn)
    return e.evals, sigma, hn


def _check_job(g, ctx, orc, L, h, seed, eps, nev, prec, block=8, **kw):
    sec = g.build_sector(ctx, L, h, seed)
    res = g.solve_near(sec, eps, nev, precision=prec, block=block, **kw)
    H = orc.csr(L, orc.fields(L, h, seed))
    spectrum, sigma, hn = _reference(orc, H, L, eps, nev)
    assert abs(res.sigma - sigma) <= 1e-12 * hn
    assert res.nconv == nev
    assert window_equivalent(res.evals, spectrum, sigma, nev, hn)
    # residuals recomputed with the oracle's H
    Y = res.evecs
    res_o = np.zeros(nev)
    for j in range(nev):
        res_o[j] = np.linalg.norm(H.matvec(Y[:, j]) - res.evals[j] * Y[:, j])
        assert res_o[j] <= EIG_TOL * hn
        assert abs(np.linalg.norm(Y[:, j]) - 1) < 1e-12
    assert np.abs(Y.T @ Y - np.eye(nev)).max() < 1e-10
    # observables on the GPU versus the oracle on the same (GPU) eigenvectors' definitions; which
    # vectors are well enough conditioned to compare is decided from the oracle's residuals
    r_g, rm_g, s1_g, se_g = g.observables(ctx, L, res.evals, res.evecs)
    r_o, rm_o = orc.gap_ratio(res.evals)
    assert np.allclose(r_g, r_o, atol=1e-12, equal_nan=True)
    mask = well_conditioned(spectrum, res.evals, res_o)
    st = orc.basis(L)
    for j in np.nonzero(mask)[0]:
        assert abs(s1_g[j] - orc.s1p(Y[:, j])) <= OBS_TOL
        assert abs(se_g[j] - orc.entanglement(L, Y[:, j], st)) <= OBS_TOL
    return res, spectrum, hn


@pytest.mark.parametrize("ordering", ["BAND", "MODES", "COVER", "HYBRID"])
def test_every_ordering_matches_the_oracle(g, orc, ordering):
    """Every fill-reducing ordering factors the same matrix (in exact arithmetic a symmetric
    permutation of one LDL^T), so each must give the oracle's eigenpairs: L = 14, h = 2.5, seed 3,
    eps = 0.5, 20 pairs, FP32 fronts.  A context of its own, so the shared one keeps the default."""
    code = getattr(g, f"MBL_ORDER_{ordering}")
    c = g.Context(0)
    try:
        c.set_ordering(code)
        sec = g.build_sector(c, 14, 2.5, 3)
        assert g.analyse(sec, 20, 8)["ordering"] == code
        sec.close()
        _check_job(g, c, orc, 14, 2.5, 3, 0.5, 20, 1)
        with pytest.raises(g.MblError):
            c.set_ordering(7)
    finally:
        c.close()


@pytest.mark.parametrize("prec", [0, 1])
def test_config_L12_h2_seed0(g, ctx, orc, prec):
    """Headline small case: L=12, h=2.0, seed 0, eps=0.5, nev=20 (FP64 and FP32 fronts)."""
    res, spectrum, hn = _check_job(g, ctx, orc, 12, 2.0, 0, 0.5, 20, prec)
    # oracle eigenpairs and observables on the oracle's own eigenvectors
    job = orc.solve_job(orc.Job(12, 2.0, 0, 0.5, 20), "dense")
    assert np.abs(np.sort(res.evals) - job.evals).max() <= EIG_TOL * hn
    H = orc.csr(12, orc.fields(12, 2.0, 0))
    res_o = np.array([np.linalg.norm(H.matvec(res.evecs[:, j]) - res.evals[j] * res.evecs[:, j]) for j in range(20)])
    mask = well_conditioned(spectrum, job.evals, job.resid) & well_conditioned(spectrum, res.evals, res_o)
    _, _, s1_g, se_g = g.observables(ctx, 12, res.evals, res.evecs)
    assert np.all(np.abs(s1_g - job.s1p)[mask] <= OBS_TOL)
    assert np.all(np.abs(se_g - job.se)[mask] <= OBS_TOL)
    assert abs(np.nanmean(job.r) - np.nanmean(orc.gap_ratio(res.evals)[0])) <= 1e-8


@pytest.mark.parametrize("L,h,seed,eps,nev,prec", [(12, 0.5, 3, 0.1, 20, 1), (12, 5.0, 4, 0.9, 30, 1),
                                                   (14, 3.0, 5, 0.5, 50, 1), (14, 1.0, 6, 0.2, 50, 0),
                                                   (12, 4.0, 7, 0.0, 10, 1), (12, 4.0, 7, 1.0, 10, 1)])
def test_solve_near_matrix(g, ctx, orc, L, h, seed, eps, nev, prec):
    _check_job(g, ctx, orc, L, h, seed, eps, nev, prec)


@pytest.mark.parametrize("block", [1, 4, 16])
def test_block_sizes(g, ctx, orc, block):
    _check_job(g, ctx, orc, 12, 2.5, 8, 0.6, 16, 1, block=block)


@pytest.mark.parametrize("prec", [0, 1])
@pytest.mark.parametrize("L", [12, 16])
def test_dataflow_solve_matches_level_sequence(g, ctx, prec, L):
    """The persistent dataflow sweeps compute the same block solve as the launch sequence."""
    sec = g.build_sector(ctx, L, 2.0, 31)
    lo, hi = g.extremal_bounds(sec)
    sigma = lo + 0.45 * (hi - lo)
    B = np.random.default_rng(2).standard_normal((sec.dim, 8))
    fs = [g.factor(sec, sigma, precision=prec, solve_dataflow=df) for df in (0, 1)]
    X = [f.solve(B, refine=False) for f in fs]
    # the two schedules sum in different orders: in FP64 they agree to rounding; in FP32 each is as
    # far from the exact solve as the other (the refined FP64 solution is the yardstick)
    if prec == 0:
        assert np.max(np.abs(X[1] - X[0])) <= 1e-10 * np.max(np.abs(X[0]))
    else:
        xr = fs[0].solve(B, refine=True)
        e0, e1 = (np.max(np.abs(x - xr)) for x in X)
        scale = np.max(np.abs(xr))
        assert e0 <= 1e-2 * scale and e1 <= 1e-2 * scale
        assert np.max(np.abs(X[1] - X[0])) <= 2.0 * max(e0, e1) + 1e-6 * scale


def test_dataflow_solve_near(g, ctx, orc):
    _check_job(g, ctx, orc, 14, 3.0, 5, 0.5, 50, 1, solve_dataflow=1)


@pytest.mark.parametrize("L,h,seed,eps,prec", [(16, 1.0, 1, 0.4, 0), (16, 2.5, 1, 0.6, 0)])
def test_window_has_no_spurious_ritz_values(g, ctx, orc, L, h, seed, eps, prec):
    """Jobs where plain Rayleigh-Ritz on H kept a spurious interior Ritz value in the window: every
    returned pair must be an eigenpair (oracle residual), and the window [min, max] must hold exactly
    nev eigenvalues, counted by the oracle's LDL^T inertia (Sylvester) at both ends."""
    nev = 50
    sec = g.build_sector(ctx, L, h, seed)
    res = g.solve_near(sec, eps, nev, precision=prec)
    lo, hi = g.extremal_bounds(sec)
    sec.close()
    hn = max(abs(lo), abs(hi))
    assert res.nconv == nev
    H = orc.csr(L, orc.fields(L, h, seed))
    for j in range(nev):
        assert np.linalg.norm(H.matvec(res.evecs[:, j]) - res.evals[j] * res.evecs[:, j]) <= EIG_TOL * hn
    ev = np.sort(res.evals)
    gap_lo, gap_hi = 0.5 * (ev[1] - ev[0]), 0.5 * (ev[-1] - ev[-2])
    F = orc.LDLT(H)
    below_lo = F.factor(ev[0] - min(gap_lo, 1e-9 * hn)).negative
    below_hi = F.factor(ev[-1] + min(gap_hi, 1e-9 * hn)).negative
    assert below_hi - below_lo == nev


@pytest.mark.parametrize("L,nev", [(2, 1), (2, 2), (4, 6), (6, 5), (8, 12), (10, 40)])
def test_dense_route_small_sectors(g, ctx, orc, L, nev):
    _check_job(g, ctx, orc, L, 1.5, 9, 0.5, nev, 1)


def test_observables_on_oracle_vectors(g, ctx, orc):
    job = orc.solve_job(orc.Job(12, 3.0, 2, 0.4, 20), "dense")
    r, rm, s1, se = g.observables(ctx, 12, job.evals, job.evecs)
    assert np.allclose(r, job.r, atol=1e-13, equal_nan=True)
    assert abs(rm - job.r_mean) < 1e-13
    assert np.abs(s1 - job.s1p).max() < 1e-11
    assert np.abs(se - job.se).max() < 1e-11


def test_invalid_arguments(g, ctx):
    with pytest.raises(g.MblError) as e:
        g.build_sector(ctx, 7, 1.0, 0)
    assert e.value.code == 1
    with pytest.raises(g.MblError):
        g.build_sector(ctx, 24, 1.0, 0)
    sec = g.build_sector(ctx, 12, 1.0, 0)
    with pytest.raises(g.MblError):
        g.solve_near(sec, 1.5, 10)
    with pytest.raises(g.MblError):
        g.solve_near(sec, 0.5, 0)
    with pytest.raises(g.MblError):
        g.solve_near(sec, 0.5, sec.dim + 1)


def test_analyse_matches_factorization(g, ctx):
    """The symbolic analysis alone predicts what a factorization then reports."""
    sec = g.build_sector(ctx, 14, 2.0, 3)
    a = g.analyse(sec, 50, 8)
    f = g.factor(sec, 0.1, precision=1)
    st = f.stats()
    assert a["nnz_l"] == st["nnz_l"] and a["n"] == st["n"] and a["max_front"] == st["max_front"]
    assert a["flops"] == st["flops"] and a["tree_levels"] == st["tree_levels"]
    assert a["front_bytes_fp32"] == st["front_bytes"]
    assert a["job_peak_bytes_fp64"] > a["job_peak_bytes_fp32"] > a["front_bytes_fp32"]
    with pytest.raises(g.MblError):
        g.analyse(sec, 0, 8)
