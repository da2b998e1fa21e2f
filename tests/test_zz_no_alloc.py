"""The static-scratch entanglement entropy (mbl_entanglement_noalloc_dev) against the allocating
entry point (mbl_observables_dev) on the same device vectors, two calls in a row; the device's
free memory must not move across the two calls.  Collected last on purpose: it must pass alone and
after the rest of the suite (the scratch is library-global).  Needs a GB300.
"""
import numpy as np
import pytest

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


def _vectors(g, ctx, L, nev):
    import torch

    sec = g.build_sector(ctx, L, 2.0, 17)
    n = sec.dim
    if L <= 12:
        res = g.solve_near(sec, 0.5, nev)
        V, ev = res.evecs, res.evals
    else:  # any vector has a Schmidt spectrum: random ones exercise every block
        V = np.random.default_rng(L).standard_normal((n, nev))
        ev = np.sort(np.random.default_rng(L + 1).standard_normal(nev))
    sec.close()
    d_vec = torch.tensor(np.asfortranarray(V).reshape(-1, order="F"), dtype=torch.float64, device="cuda")
    d_ev = torch.tensor(ev, dtype=torch.float64, device="cuda")
    return n, d_ev, d_vec


@pytest.mark.parametrize("L,nev", [(2, 1), (8, 10), (12, 20), (16, 64)])
def test_noalloc_matches_allocating_entry_point(g, ctx, L, nev):
    import torch

    n, d_ev, d_vec = _vectors(g, ctx, L, nev)
    z = lambda k: torch.zeros(k, dtype=torch.float64, device="cuda")
    d_r, d_rm, d_s1, d_se_ref = z(max(nev - 2, 1)), z(1), z(nev), z(nev)
    g.observables_dev(ctx, L, nev, d_ev, d_vec, d_r, d_rm, d_s1, d_se_ref)
    ref = d_se_ref.cpu().numpy()
    d_se1, d_se2 = z(nev), z(nev)
    torch.cuda.synchronize()
    free0 = torch.cuda.mem_get_info()[0]
    g.entanglement_noalloc_dev(ctx, L, nev, d_vec, d_se1)
    g.entanglement_noalloc_dev(ctx, L, nev, d_vec, d_se2)
    ctx.synchronize()
    torch.cuda.synchronize()
    free1 = torch.cuda.mem_get_info()[0]
    a, b = d_se1.cpu().numpy(), d_se2.cpu().numpy()
    assert np.array_equal(a, b)
    assert np.max(np.abs(a - ref)) <= 1e-12
    assert free1 == free0


def test_noalloc_rejects_oversized_requests(g, ctx):
    import torch

    d_vec = torch.zeros(48620 * 2, dtype=torch.float64, device="cuda")
    d_se = torch.zeros(65, dtype=torch.float64, device="cuda")
    with pytest.raises(g.MblError) as e:
        g.entanglement_noalloc_dev(ctx, 18, 2, d_vec, d_se)
    assert e.value.code == 1
    with pytest.raises(g.MblError) as e:
        g.entanglement_noalloc_dev(ctx, 12, 65, d_vec, d_se)
    assert e.value.code == 1
    with pytest.raises(g.MblError) as e:
        g.entanglement_noalloc_dev(ctx, 13, 2, d_vec, d_se)
    assert e.value.code == 1
