"""Host-side logic of the benchmark (no GPU): the DRAM traffic it copies into its roofline from a
committed ncu summary is used only for the factorization that summary was captured on."""
import pytest

pytest.importorskip("torch")
import bench  # noqa: E402


def _alg_bytes(name):
    import os

    with open(os.path.join(bench.ROOT, "profiles", name)) as fp:
        for ln in fp:
            if ln.startswith("algorithmic_bytes_per_solve:"):
                return float(ln.split(":")[1])
    raise AssertionError(f"{name} states no algorithmic bytes")


@pytest.mark.parametrize("name", ["solve_l18_fp32_traffic.md", "solve_l18_fp32_batch_traffic.md"])
def test_traffic_only_for_the_captured_factor(name):
    alg = _alg_bytes(name)
    t = bench.profiled_traffic(name, alg)
    assert t is not None and t > alg  # DRAM bytes of the capture, above the algorithmic bytes
    assert bench.profiled_traffic(name, alg * 1.005) == t  # within 1%: the same factor
    # a smaller factor (another ordering) or another sector: no stale figure
    assert bench.profiled_traffic(name, alg * 0.73) is None
    assert bench.profiled_traffic(name, alg * 1.5) is None
    assert bench.profiled_traffic("no_such_summary.md", alg) is None


def test_orderings_named_like_the_library():
    from paper_1411_0660_gb300 import _capi

    assert bench._ORDERING == {"band": _capi.MBL_ORDER_BAND, "cover": _capi.MBL_ORDER_COVER,
                               "modes": _capi.MBL_ORDER_MODES, "auto": _capi.MBL_ORDER_AUTO,
                               "hybrid": _capi.MBL_ORDER_HYBRID}
