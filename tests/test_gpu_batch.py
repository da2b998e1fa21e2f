"""Batched triangular solves (needs a GB300).

Jobs of one sector shape share a symbolic plan, so their block solves are one launch sequence on
different buffers.  mbl_factor_solve_batch_dev runs K factorizations' solves in shared launches:
each result must be bit-identical to the factorization's own unrefined solve.  The server batches its
workers' solves the same way: served results with batching must match the oracle's eigenpairs like
unbatched ones, and the batches must actually hold several jobs.
"""
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
    c = g.Context(0)
    yield c
    c.close()


def _dev(B):
    import torch

    return torch.from_numpy(np.asfortranarray(B).ravel(order="F")).cuda()


@pytest.mark.parametrize("prec,nrhs", [(1, 8), (0, 8), (1, 37)])
def test_batch_solve_bit_identical_to_single_solves(g, ctx, prec, nrhs):
    import torch

    L = 14
    jobs = [(1.0, 50, 0.3), (3.0, 51, 0.5), (5.0, 52, 0.8)]
    secs, facts = [], []
    for h, seed, eps in jobs:
        sec = g.build_sector(ctx, L, h, seed)
        lo, hi = g.extremal_bounds(sec)
        secs.append(sec)
        facts.append(g.factor(sec, lo + eps * (hi - lo), precision=prec))
    n = secs[0].dim
    rng = np.random.default_rng(9)
    d_b = [_dev(rng.standard_normal((n, nrhs))) for _ in jobs]
    single = []
    for f, b in zip(facts, d_b):
        x = torch.zeros_like(b)
        f.solve_dev(b, x, nrhs, refine=False)
        torch.cuda.synchronize()
        single.append(x.cpu().numpy())
    d_x = [torch.full_like(b, np.nan) for b in d_b]
    g.factor_solve_batch_dev(facts, d_b, d_x, nrhs)
    torch.cuda.synchronize()
    for x1, x in zip(single, d_x):
        assert np.array_equal(x.cpu().numpy().view(np.uint64), x1.view(np.uint64))
    # a sub-batch in another order gives the same bits too
    d_x2 = [torch.zeros_like(b) for b in d_b[:2]]
    g.factor_solve_batch_dev([facts[1], facts[0]], [d_b[1], d_b[0]], d_x2, nrhs)
    torch.cuda.synchronize()
    assert np.array_equal(d_x2[0].cpu().numpy(), single[1]) and np.array_equal(d_x2[1].cpu().numpy(), single[0])
    for f in facts:
        f.close()
    for s in secs:
        s.close()


def test_batch_solve_rejects_mixed_plans_and_duplicates(g, ctx):
    import torch

    s12 = g.build_sector(ctx, 12, 2.0, 1)
    s14 = g.build_sector(ctx, 14, 2.0, 1)
    f12 = g.factor(s12, 0.1)
    f14 = g.factor(s14, 0.1)
    f14d = g.factor(s14, 0.2, precision=0)
    b12 = torch.zeros(s12.dim * 2, dtype=torch.float64, device="cuda")
    b14 = torch.zeros(s14.dim * 2, dtype=torch.float64, device="cuda")
    with pytest.raises(g.MblError):
        g.factor_solve_batch_dev([f12, f14], [b12, b14], [b12.clone(), b14.clone()], 2)
    with pytest.raises(g.MblError):
        g.factor_solve_batch_dev([f14, f14d], [b14, b14], [b14.clone(), b14.clone()], 2)
    with pytest.raises(g.MblError):
        g.factor_solve_batch_dev([f14, f14], [b14, b14], [b14.clone(), b14.clone()], 2)
    for f in (f12, f14, f14d):
        f.close()
    s12.close()
    s14.close()


def test_served_solves_are_batched_and_correct(g, ctx, orc):
    jobs = [(14, 0.5 + k, 60 + k, 0.2 + 0.12 * k, 20, 1 if k < 4 else 0) for k in range(6)]
    srv = g.Server(ctx, slots=6, batch_jobs=16, batch_window_us=300.0)
    tickets = [srv.submit(L, h, s, e, nev, precision=p, want_vectors=True) for (L, h, s, e, nev, p) in jobs]
    out = [srv.wait(t, 600.0) for t in tickets]
    st = srv.stats()
    srv.stop()
    assert st["failed"] == 0
    assert st["solve_batches"] > 0 and st["batched_solves"] > st["solve_batches"]  # more than one job per launch
    assert st["batch_ms"] > 0 and st["batch_bytes"] > 0
    for (L, h, seed, eps, nev, prec), r in zip(jobs, out):
        assert r.status == 0 and r.nconv == nev
        H = orc.csr(L, orc.fields(L, h, seed))
        emin, emax = orc.extremal_bounds(H)
        hn = max(abs(emin), abs(emax))
        sigma = emin + eps * (emax - emin)
        assert abs(r.sigma - sigma) <= 1e-12 * hn
        spectrum = orc.nearest_shift_invert(H, sigma, nev + 12, hn).evals
        assert window_equivalent(r.evals, spectrum, sigma, nev, hn)
        for j in range(nev):
            y = r.evecs[:, j]
            assert np.linalg.norm(H.matvec(y) - r.evals[j] * y) <= EIG_TOL * hn
    # the same jobs without batching give the same eigenvalues
    srv1 = g.Server(ctx, slots=6, batch_jobs=1)
    out1 = [srv1.wait(t, 600.0) for t in [srv1.submit(L, h, s, e, nev, precision=p) for (L, h, s, e, nev, p) in jobs]]
    st1 = srv1.stats()
    srv1.stop()
    assert st1["solve_batches"] == 0
    for (L, h, seed, eps, nev, prec), a, b in zip(jobs, out, out1):
        sec = g.build_sector(ctx, L, h, seed)
        hn = max(abs(v) for v in g.extremal_bounds(sec))
        sec.close()
        assert np.max(np.abs(a.evals - b.evals)) <= EIG_TOL * hn
