"""The static-scratch entanglement entropy (mbl_entanglement_noalloc_dev) against the allocating
entry point (mbl_observables_dev) on the same device vectors, two calls in a row; the device's
free memory must not move across the two calls.  Collected last on purpose: it must pass alone and
after the rest of the suite (the scratch is library-global).  Needs a GB300.
"""
import json
import os
import subprocess
import sys

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


_FRESH = r"""
import json, sys
import numpy as np
import torch
sys.path.insert(0, sys.argv[1])
import paper_1411_0660_gb300 as g
ctx = g.Context(0)
L, nev = 12, 16
n = 924
V = np.random.default_rng(5).standard_normal((n, nev))
d_vec = torch.tensor(V.T.copy().reshape(-1), dtype=torch.float64, device="cuda")
d_se = torch.zeros(nev, dtype=torch.float64, device="cuda")
d_ev = torch.tensor(np.linspace(-1.0, 1.0, nev), dtype=torch.float64, device="cuda")
z = lambda k: torch.zeros(k, dtype=torch.float64, device="cuda")
d_r, d_rm, d_s1, d_ref = z(nev - 2), z(1), z(nev), z(nev)
torch.cuda.synchronize()
free0 = torch.cuda.mem_get_info()[0]
g.entanglement_noalloc_dev(ctx, L, nev, d_vec, d_se)  # the process's first eigensolver call
ctx.synchronize()
torch.cuda.synchronize()
free1 = torch.cuda.mem_get_info()[0]
g.observables_dev(ctx, L, nev, d_ev, d_vec, d_r, d_rm, d_s1, d_ref)
torch.cuda.synchronize()
print(json.dumps({"free0": free0, "free1": free1, "se": d_se.cpu().tolist(), "ref": d_ref.cpu().tolist()}))
"""


def test_noalloc_first_call_in_a_fresh_process_does_not_allocate():
    """A caller that cannot allocate may make this its first eigensolver call of the process: the
    kernels it launches were loaded when the context was created, so free device memory is unchanged
    across the call; the result equals the allocating entry point's."""
    root = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
    out = subprocess.run([sys.executable, "-c", _FRESH, root], capture_output=True, text=True, timeout=600)
    assert out.returncode == 0, out.stderr[-2000:]
    r = json.loads(out.stdout.strip().splitlines()[-1])
    assert r["free1"] == r["free0"]
    assert np.max(np.abs(np.array(r["se"]) - np.array(r["ref"]))) <= 1e-12


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
