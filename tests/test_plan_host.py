"""Host-only checks of the symbolic analysis (no GPU): the library's plan builder is compiled
with a small checker (tests/plan_check.cpp) and run on the patterns of several sectors, including
odd L and sectors away from half filling.  The checker verifies the invariants the numeric
factorization and the solves rely on: a permutation ordering; supernodes that partition the
columns; front row lists whose contribution rows belong to ancestors and nest into the parent's
rows; an L structure that holds the pattern of P A P^T; nnz(L); solve panels that tile every
front's fully summed block with consistent offsets into the packed solve factor; solve steps that
cover every panel once; a forward gather that writes every front row once; and dataflow item
lists whose dependencies are met in list order.  All three fill-reducing orderings are checked, and
the two optional ones (band or cover-refined separators over all modes) are checked to need less
fill and fewer flops than the default band separators of a fixed mode sequence."""
import os
import subprocess

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
CSRC = os.path.join(ROOT, "paper_1411_0660_gb300", "csrc")


@pytest.fixture(scope="module")
def checker(tmp_path_factory):
    from paper_1411_0660_gb300 import build

    inc = build._cuda_include()
    libdir = os.path.join(os.path.dirname(inc), "lib64")
    if not os.path.isdir(libdir):
        libdir = os.path.join(os.path.dirname(inc), "lib")
    exe = str(tmp_path_factory.mktemp("plan") / "plan_check")
    cmd = ["g++", "-O2", "-std=c++17", "-pthread", "-I" + inc, "-I" + os.path.join(ROOT, "include"), "-I" + CSRC,
           os.path.join(ROOT, "tests", "plan_check.cpp"), os.path.join(CSRC, "symbolic.cpp"), "-o", exe,
           "-L" + libdir, "-lcudart", "-Wl,-rpath," + libdir]
    subprocess.run(cmd, check=True, capture_output=True)
    return exe


@pytest.mark.parametrize("L,nup", [(2, 1), (8, 4), (10, 5), (11, 5), (12, 3), (13, 7), (14, 7), (15, 8), (16, 8), (17, 9), (18, 9),
                                   (12, 1), (9, 0)])
@pytest.mark.parametrize("ordering", [0, 1, 2, 4])
def test_plan_invariants(checker, L, nup, ordering):
    r = subprocess.run([checker, str(L), str(nup), str(ordering)], capture_output=True, text=True, timeout=120)
    assert r.returncode == 0 and r.stdout.startswith("ok"), r.stdout + r.stderr


def _stats(checker, L, nup, ordering):
    r = subprocess.run([checker, str(L), str(nup), str(ordering)], capture_output=True, text=True, timeout=120)
    assert r.returncode == 0 and r.stdout.startswith("ok"), r.stdout + r.stderr
    return {k: float(v) for k, v in (t.split("=") for t in r.stdout.split()[1:])}


@pytest.mark.parametrize("L,nup", [(14, 7), (16, 8), (18, 9), (17, 9)])
def test_cover_ordering_reduces_fill(checker, L, nup):
    """A minimum cover of the edges crossing a threshold inside a band is never larger than the band,
    and the cover ordering also searches every mode: fill-in and flops shrink, the largest front
    does not grow by more than a few percent."""
    band, cover, modes, hybrid = (_stats(checker, L, nup, o) for o in (0, 1, 2, 4))
    assert cover["nnz_l"] < 0.9 * band["nnz_l"], (cover, band)
    assert cover["flops"] < 0.85 * band["flops"], (cover, band)
    assert cover["max_front"] <= 1.05 * band["max_front"], (cover, band)
    # the cover refines the best band among the same modes: never more fill than that band alone
    assert cover["nnz_l"] <= modes["nnz_l"] <= band["nnz_l"], (cover, modes, band)
    # the hybrid takes covers only where subgraphs are large: between the two, and fewer supernodes
    assert cover["nnz_l"] <= hybrid["nnz_l"] <= modes["nnz_l"], (cover, hybrid, modes)
    assert hybrid["supernodes"] <= cover["supernodes"], (hybrid, cover)


@pytest.mark.parametrize("L,nup,resolved", [(16, 8, 0), (17, 9, 0), (18, 9, 2), (18, 4, 0)])
def test_auto_ordering_by_sector_dimension(checker, L, nup, resolved):
    """The default picks the modes ordering for sectors of dimension >= 40000 and the band ordering
    below, and builds exactly the plan that ordering builds."""
    auto, explicit = _stats(checker, L, nup, 3), _stats(checker, L, nup, resolved)
    assert auto["ordering"] == resolved
    assert auto == explicit


def test_unknown_ordering_is_rejected(checker):
    r = subprocess.run([checker, "8", "4", "7"], capture_output=True, text=True, timeout=60)
    assert r.returncode != 0
