"""GPU observables of the characterization section and its supplement versus the CPU oracle,
element by element through the C ABI (needs a GB300): KL divergence of adjacent eigenvectors,
S_q^P, bipartite fluctuation F and dynamic spin fraction f.

The kernels reduce the same weights p_i = y_i^2 / |y|^2 in another order than the oracle, so the
tolerance is 1e-8 (the observables tolerance), far above the rounding differences (~1e-13).
"""
import math

import numpy as np
import pytest

from parity import OBS_TOL

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def g():
    import paper_1411_0660_gb300 as g

    return g


@pytest.fixture(scope="module")
def ctx(g):
    return g.Context(0)


def _oracle_extra(orc, L, Y, q, st):
    nev = Y.shape[1]
    kl = np.array([orc.kl(Y[:, k], Y[:, k + 1]) for k in range(nev - 1)])
    sqp = np.array([orc.sqp(Y[:, j], q) for j in range(nev)])
    fl = np.array([orc.fluct(L, Y[:, j], st) for j in range(nev)])
    dy = np.array([orc.dynf(L, Y[:, j], st) for j in range(nev)])
    return kl, sqp, fl, dy


def _close(a, b, tol=OBS_TOL):
    a, b = np.asarray(a), np.asarray(b)
    same_inf = np.isinf(a) & np.isinf(b) & (np.sign(a) == np.sign(b))
    same_nan = np.isnan(a) & np.isnan(b)
    fin = ~(same_inf | same_nan)
    return bool(np.all(np.abs(a[fin] - b[fin]) <= tol * np.maximum(1.0, np.abs(b[fin]))))


@pytest.mark.parametrize("L,q", [(6, 0.5), (8, 2.0), (12, 3.0), (14, 2.0), (16, 2.0)])
def test_extra_observables_random_and_special_vectors(g, ctx, orc, L, q):
    st = orc.basis(L)
    n = len(st)
    rng = np.random.default_rng(100 + L)
    cols = [rng.standard_normal(n) * np.exp(-rng.uniform(0, 6, n)) for _ in range(5)]
    e = np.zeros(n)
    e[n // 2] = 1.0
    cols += [e, np.ones(n), rng.standard_normal(n)]  # a basis state (KL to it and from it infinite)
    Y = np.column_stack(cols)
    kl, sqp, fl, dy = g.observables_extra(ctx, L, Y, q)
    okl, osq, ofl, ody = _oracle_extra(orc, L, Y, q, st)
    assert _close(kl, okl) and _close(sqp, osq) and _close(fl, ofl) and _close(dy, ody)
    assert math.isinf(kl[4]) and np.isfinite(kl[5])  # q_i = 0 < p_i from column 4 to the basis state


@pytest.mark.parametrize("L", [2, 4])
def test_extra_observables_smallest_sectors(g, ctx, orc, L):
    st = orc.basis(L)
    n = len(st)
    Y = np.random.default_rng(L).standard_normal((n, n))
    Y[:, 0] = 0.0
    Y[0, 0] = 1.0  # a basis state
    for q in (0.5, 2.0):
        kl, sqp, fl, dy = g.observables_extra(ctx, L, Y, q)
        assert all(_close(a, b) for a, b in zip((kl, sqp, fl, dy), _oracle_extra(orc, L, Y, q, st)))
        assert abs(dy[0]) < 1e-14 and abs(fl[0]) < 1e-14 and abs(sqp[0]) < 1e-14


def test_extra_observables_on_solved_eigenvectors(g, ctx, orc):
    L, nev = 14, 40
    sec = g.build_sector(ctx, L, 3.0, 4)
    res = g.solve_near(sec, 0.5, nev)
    sec.close()
    order = np.argsort(res.evals)
    Y = res.evecs[:, order]
    st = orc.basis(L)
    kl, sqp, fl, dy = g.observables_extra(ctx, L, Y, 2.0)
    okl, osq, ofl, ody = _oracle_extra(orc, L, Y, 2.0, st)
    assert _close(kl, okl) and _close(sqp, osq) and _close(fl, ofl) and _close(dy, ody)
    assert np.all(kl > 0) and np.all((dy >= -1e-14) & (dy <= 1 + 1e-14))
    assert np.all(sqp <= math.log(math.comb(L, L // 2)) + 1e-12)


def test_extra_observables_device_entry_and_errors(g, ctx, orc):
    torch = pytest.importorskip("torch")
    L, nev = 10, 6
    st = orc.basis(L)
    n = len(st)
    Y = np.random.default_rng(9).standard_normal((n, nev))
    dev = torch.device("cuda:0")
    dY = torch.tensor(Y.T.copy(), dtype=torch.float64, device=dev).reshape(-1)  # column-major
    outs = [torch.zeros(m, dtype=torch.float64, device=dev) for m in (nev - 1, nev, nev, nev)]
    g.observables_extra_dev(ctx, L, nev, dY, 2.0, *outs)
    torch.cuda.synchronize()
    ref = _oracle_extra(orc, L, Y, 2.0, st)
    for o, r in zip(outs, ref):
        assert _close(o.cpu().numpy(), r)
    for bad_q in (1.0, 0.0, -2.0):
        with pytest.raises(g.MblError):
            g.observables_extra(ctx, L, Y, bad_q)
    with pytest.raises(g.MblError):
        g.observables_extra(ctx, 11, Y, 2.0)
