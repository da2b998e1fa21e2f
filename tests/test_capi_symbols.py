"""Host-side checks of the C-ABI library (no GPU): it builds for sm_103a, loads, and exports
every entry point that include/mblsi.h declares; the Python binding declares each one."""
import ctypes
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _declared():
    txt = open(os.path.join(ROOT, "include", "mblsi.h")).read()
    txt = re.sub(r"/\*.*?\*/", "", txt, flags=re.S)
    return sorted(set(re.findall(r"\b(mbl_[a-z0-9_]+)\s*\(", txt)))


@pytest.fixture(scope="module")
def libpath():
    from paper_1411_0660_gb300 import build

    return build.build()


def test_library_exports_every_declared_symbol(libpath):
    lib = ctypes.CDLL(libpath)
    names = _declared()
    assert len(names) >= 20
    missing = [n for n in names if not hasattr(lib, n)]
    assert not missing, missing


def test_binding_covers_every_declared_symbol():
    from paper_1411_0660_gb300 import _capi

    bound = {n for n, _, _ in _capi.SIGNATURES}
    assert set(_declared()) == bound


def test_missing_library_fails_loudly(tmp_path, monkeypatch):
    from paper_1411_0660_gb300 import _capi

    monkeypatch.setattr(_capi, "_lib", None)
    monkeypatch.setattr(_capi, "lib_path", lambda: str(tmp_path / "absent.so"))
    with pytest.raises(ImportError):
        _capi.load(build_if_missing=False)


def test_no_gpu_calls_needed_to_load(libpath):
    # loading and querying static strings touches no device
    from paper_1411_0660_gb300 import _capi

    lib = _capi.load()
    assert b"sm_103a" in lib.mbl_version()
    assert lib.mbl_status_string(4) == b"not converged"


def _prototypes():
    """name -> number of parameters of every function prototype in include/mblsi.h."""
    txt = open(os.path.join(ROOT, "include", "mblsi.h")).read()
    txt = re.sub(r"/\*.*?\*/", "", txt, flags=re.S)
    out = {}
    for m in re.finditer(r"\b(mbl_[a-z0-9_]+)\s*\(([^;{]*?)\)\s*;", txt):
        params = m.group(2).strip()
        out[m.group(1)] = 0 if params in ("", "void") else params.count(",") + 1
    return out


def test_binding_parameter_counts_match_the_header():
    """Each ctypes signature has as many parameters as its C prototype (a missing or extra
    argument would otherwise only surface as a wrong value on the GPU)."""
    from paper_1411_0660_gb300 import _capi

    proto = _prototypes()
    bad = [(n, len(args), proto[n]) for n, _, args in _capi.SIGNATURES if n in proto and len(args) != proto[n]]
    assert not bad, bad
    assert len(proto) >= 20
