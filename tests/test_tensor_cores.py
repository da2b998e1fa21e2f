"""tcgen05 Schur updates (3xTF32, FP32 accumulation in tensor memory) against the FP32 CUDA-core
updates on the same factorization, and the refined shift-invert results through them (GPU)."""
import numpy as np
import pytest

from parity import EIG_TOL, window_equivalent

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def g():
    import paper_1411_0660_gb300 as g

    return g


@pytest.fixture(scope="module")
def ctx(g):
    return g.Context(0)


@pytest.mark.parametrize("L", [12, 14, 16])
def test_tc_factor_matches_cuda_cores(g, ctx, orc, L):
    sec = g.build_sector(ctx, L, 3.0, 1)
    lo, hi = g.extremal_bounds(sec)
    sigma = lo + 0.45 * (hi - lo)
    f_s = g.factor(sec, sigma, precision=1, tensor_cores=0)
    f_t = g.factor(sec, sigma, precision=1, tensor_cores=1)
    B = np.random.default_rng(2).standard_normal((sec.dim, 4))
    X = f_s.solve(B, refine=True)
    Xs = f_s.solve(B, refine=False)
    Xt = f_t.solve(B, refine=False)
    es = np.linalg.norm(Xs - X) / np.linalg.norm(X)
    et = np.linalg.norm(Xt - X) / np.linalg.norm(X)
    # both unrefined solves carry FP32-level factor error; 3xTF32 must not be much worse
    assert et < max(20 * es, 1e-5)
    H = orc.csr(L, orc.fields(L, 3.0, 1))
    Xr = f_t.solve(B, refine=True)
    hn = max(abs(lo), abs(hi))
    for q in range(4):
        r = H.matvec(Xr[:, q], sigma) - B[:, q]
        assert np.linalg.norm(r) <= 1e-13 * ((hn + abs(sigma)) * np.linalg.norm(Xr[:, q]) + np.linalg.norm(B[:, q]))
    assert f_t.stats()["negative"] == f_s.stats()["negative"]


@pytest.mark.parametrize("L,h,seed,eps,nev", [(12, 2.0, 0, 0.5, 20), (14, 4.0, 3, 0.3, 40)])
def test_tc_solve_near(g, ctx, orc, L, h, seed, eps, nev):
    sec = g.build_sector(ctx, L, h, seed)
    res = g.solve_near(sec, eps, nev, precision=1, tensor_cores=1)
    H = orc.csr(L, orc.fields(L, h, seed))
    emin, emax = orc.extremal_bounds(H)
    hn = max(abs(emin), abs(emax))
    sigma = emin + eps * (emax - emin)
    e = orc.nearest_shift_invert(H, sigma, nev + 12, hn)
    assert res.nconv == nev
    assert window_equivalent(res.evals, e.evals, sigma, nev, hn)
    for j in range(nev):
        assert np.linalg.norm(H.matvec(res.evecs[:, j]) - res.evals[j] * res.evecs[:, j]) <= EIG_TOL * hn


@pytest.mark.parametrize("L", [12, 16])
def test_bf16x3_factor(g, ctx, orc, L):
    """tcgen05 with split-BF16 operands (hi*hi + hi*lo + lo*hi, FP32 accumulation): the same inertia
    as the CUDA-core factor, an unrefined solve within the expected loss of about 5 bits against
    3xTF32, and FP64 refinement through it to the FP64 backward-error target."""
    sec = g.build_sector(ctx, L, 3.0, 1)
    lo, hi = g.extremal_bounds(sec)
    sigma = lo + 0.45 * (hi - lo)
    f_s = g.factor(sec, sigma, precision=1, tensor_cores=0)
    f_b = g.factor(sec, sigma, precision=1, tensor_cores=2)
    assert f_b.stats()["negative"] == f_s.stats()["negative"]
    B = np.random.default_rng(3).standard_normal((sec.dim, 4))
    X = f_s.solve(B, refine=True)
    es = np.linalg.norm(f_s.solve(B, refine=False) - X) / np.linalg.norm(X)
    eb = np.linalg.norm(f_b.solve(B, refine=False) - X) / np.linalg.norm(X)
    assert eb < max(2000 * es, 1e-2)
    H = orc.csr(L, orc.fields(L, 3.0, 1))
    Xr = f_b.solve(B, refine=True)
    hn = max(abs(lo), abs(hi))
    for q in range(4):
        r = H.matvec(Xr[:, q], sigma) - B[:, q]
        assert np.linalg.norm(r) <= 1e-13 * ((hn + abs(sigma)) * np.linalg.norm(Xr[:, q]) + np.linalg.norm(B[:, q]))


def test_bf16x3_solve_near(g, ctx, orc):
    L, h, seed, eps, nev = 14, 2.0, 7, 0.5, 40
    sec = g.build_sector(ctx, L, h, seed)
    res = g.solve_near(sec, eps, nev, precision=1, tensor_cores=2)
    H = orc.csr(L, orc.fields(L, h, seed))
    emin, emax = orc.extremal_bounds(H)
    hn = max(abs(emin), abs(emax))
    sigma = emin + eps * (emax - emin)
    e = orc.nearest_shift_invert(H, sigma, nev + 12, hn)
    assert res.nconv == nev
    assert window_equivalent(res.evals, e.evals, sigma, nev, hn)
    for j in range(nev):
        assert np.linalg.norm(H.matvec(res.evecs[:, j]) - res.evals[j] * res.evecs[:, j]) <= EIG_TOL * hn


def test_tensor_core_mode_is_validated(g, ctx):
    sec = g.build_sector(ctx, 10, 1.0, 2)
    with pytest.raises(g.MblError):
        g.factor(sec, 0.0, precision=1, tensor_cores=3)


def test_schur_tile_autotuning_recorded(g, ctx):
    """The FP32 fronts' trailing update is autotuned per size class of trailing block (tcgen05 128 x 128
    tiles against CUDA-core 64 x 64 tiles, timed on a synthetic front of the class): every class the
    plan's panel steps have gets a choice and two timings; FP32 fronts on CUDA cores are not tuned."""
    sec = g.build_sector(ctx, 16, 2.0, 90)
    lo, hi = g.extremal_bounds(sec)
    f = g.factor(sec, lo + 0.5 * (hi - lo), precision=1, tensor_cores=1)
    st = f.stats()
    f.close()
    tuned = [c for c in range(8) if st["tune_choice"][c] >= 0]
    assert tuned == list(range(8))
    present = [c for c in range(8) if st["tune_us_tc"][c] > 0]
    assert present, st
    for c in present:
        assert st["tune_us_cc"][c] > 0 and st["tune_choice"][c] in (0, 1)
        assert st["tune_choice"][c] == (1 if st["tune_us_tc"][c] <= st["tune_us_cc"][c] else 0)
    f0 = g.factor(sec, lo + 0.5 * (hi - lo), precision=1, tensor_cores=0)
    assert all(c == -1 for c in f0.stats()["tune_choice"])
    f0.close()
    sec.close()
