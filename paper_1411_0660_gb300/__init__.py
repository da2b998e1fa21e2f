"""GB300 (sm_103a) shift-invert exact diagonalization of the random-field Heisenberg chain.

Python face of libmblsi (include/mblsi.h): every step runs in the library's CUDA kernels; this
module only marshals arguments.  Method: Luitz, Laflorencie, Alet, arXiv:1411.0660 (Eq. 1, the
numerical-method section, and the observables of the characterization section).

    ctx = Context(0)
    sec = build_sector(ctx, L=16, h=3.0, seed=7)
    emin, emax = extremal_bounds(sec)
    res = solve_near(sec, eps=0.5, nev=50)
    r, r_mean, s1p, se = observables(ctx, 16, res.evals, res.evecs)
"""
from __future__ import annotations

import ctypes
import math
import sys
from dataclasses import dataclass

import numpy as np

from . import _capi
from ._capi import (MBL_ORDER_AUTO, MBL_ORDER_BAND, MBL_ORDER_COVER, MBL_ORDER_HYBRID, MBL_ORDER_MODES,
                    MBL_PREC_FP32, MBL_PREC_FP64, FactorStats, Opts, PlanStats, SolveStats)

__all__ = ["Context", "Sector", "Factorization", "MblError", "build_sector", "build_sector_fields",
           "extremal_bounds", "factor", "solve_near", "solve_near_dev", "observables", "observables_dev",
           "default_opts", "launch_count", "factor_solve_batch_dev", "entanglement_noalloc_dev", "Server", "ServedResult", "MBL_PREC_FP32", "MBL_PREC_FP64",
           "MBL_ORDER_AUTO", "MBL_ORDER_BAND", "MBL_ORDER_COVER", "MBL_ORDER_MODES", "MBL_ORDER_HYBRID"]


class MblError(RuntimeError):
    def __init__(self, code: int, msg: str):
        super().__init__(f"[{code}] {msg}")
        self.code = code


def _lib():
    return _capi.load()


def _check(rc: int, ctx_handle=None):
    if rc != _capi.MBL_OK:
        msg = _lib().mbl_last_error(ctx_handle)
        raise MblError(rc, msg.decode() if msg else "")


def _ptr(a: np.ndarray):
    return a.ctypes.data_as(ctypes.c_void_p)


def default_opts(**kw) -> Opts:
    o = Opts()
    _lib().mbl_opts_default(ctypes.byref(o))
    for k, v in kw.items():
        setattr(o, k, v)
    return o


class Context:
    def __init__(self, device: int = 0, hbm_budget_bytes: int = 0):
        h = ctypes.c_void_p()
        _check(_lib().mbl_ctx_create(device, hbm_budget_bytes, ctypes.byref(h)))
        self.handle = h

    def set_profiling(self, on: bool = True):
        _check(_lib().mbl_ctx_set_profiling(self.handle, 1 if on else 0), self.handle)

    def set_ordering(self, ordering: int):
        """Ordering of the symbolic analyses built from now on: MBL_ORDER_AUTO (the default),
        MBL_ORDER_BAND, MBL_ORDER_MODES, MBL_ORDER_COVER or MBL_ORDER_HYBRID."""
        _check(_lib().mbl_ctx_set_ordering(self.handle, int(ordering)), self.handle)

    def profile(self, name: str) -> dict:
        n, ms, w = ctypes.c_int64(), ctypes.c_double(), ctypes.c_double()
        _check(_lib().mbl_ctx_profile_get(self.handle, name.encode(), ctypes.byref(n), ctypes.byref(ms),
                                          ctypes.byref(w)), self.handle)
        return {"launches": n.value, "ms": ms.value, "work": w.value}

    def synchronize(self):
        _check(_lib().mbl_ctx_synchronize(self.handle), self.handle)

    def close(self):
        if getattr(self, "handle", None):
            _lib().mbl_ctx_destroy(self.handle)
            self.handle = None

    def __del__(self):
        # at interpreter shutdown the release order is arbitrary and the CUDA runtime may be going
        # away: leave the memory to process exit instead of calling into the library
        if sys.is_finalizing():
            return
        try:
            self.close()
        except Exception:
            pass


class Sector:
    def __init__(self, ctx: Context, handle, L: int):
        self.ctx, self.handle, self.L = ctx, handle, L
        n, nnz = ctypes.c_int64(), ctypes.c_int64()
        _check(_lib().mbl_sector_info(handle, ctypes.byref(n), ctypes.byref(nnz)), ctx.handle)
        self.dim, self.nnz = n.value, nnz.value
        ln, nu = ctypes.c_int(), ctypes.c_int()
        _check(_lib().mbl_sector_shape(handle, ctypes.byref(ln), ctypes.byref(nu)), ctx.handle)
        self.nup = nu.value  # up spins of every basis state

    def basis(self) -> np.ndarray:
        out = np.zeros(self.dim, dtype=np.uint32)
        _check(_lib().mbl_sector_copy_basis(self.handle, _ptr(out)), self.ctx.handle)
        return out

    def csr(self):
        rp = np.zeros(self.dim + 1, dtype=np.int64)
        col = np.zeros(self.nnz, dtype=np.int32)
        val = np.zeros(self.nnz, dtype=np.float64)
        _check(_lib().mbl_sector_copy_csr(self.handle, _ptr(rp), _ptr(col), _ptr(val)), self.ctx.handle)
        return rp, col, val

    def fields(self) -> np.ndarray:
        out = np.zeros(self.L, dtype=np.float64)
        _check(_lib().mbl_sector_copy_fields(self.handle, _ptr(out)), self.ctx.handle)
        return out

    def rank(self, states) -> np.ndarray:
        st = np.ascontiguousarray(states, dtype=np.uint32)
        out = np.zeros(len(st), dtype=np.int64)
        _check(_lib().mbl_sector_rank(self.handle, _ptr(st), len(st), _ptr(out)), self.ctx.handle)
        return out

    def spmv(self, x: np.ndarray, shift: float = 0.0) -> np.ndarray:
        X = np.asfortranarray(x, dtype=np.float64)
        if X.ndim == 1:
            X = X[:, None]
        Y = np.zeros_like(X, order="F")
        _check(_lib().mbl_spmv(self.handle, float(shift), _ptr(X), _ptr(Y), X.shape[1]), self.ctx.handle)
        return Y[:, 0] if np.ndim(x) == 1 else Y

    def close(self):
        if getattr(self, "handle", None):
            _lib().mbl_sector_destroy(self.handle)
            self.handle = None

    def __del__(self):
        # at interpreter shutdown the release order is arbitrary and the CUDA runtime may be going
        # away: leave the memory to process exit instead of calling into the library
        if sys.is_finalizing():
            return
        try:
            self.close()
        except Exception:
            pass


def launch_count() -> int:
    """Kernels launched by the library so far (all contexts)."""
    return int(_lib().mbl_launch_count())


def build_sector(ctx: Context, L: int, h: float, seed: int, nup: int | None = None) -> Sector:
    """Sector with nup up spins (None: the S^z_tot = 0 sector of even L)."""
    h_ = ctypes.c_void_p()
    sd = ctypes.c_uint64(seed & (2**64 - 1))
    if nup is None:
        rc = _lib().mbl_build_sector(ctx.handle, L, float(h), sd, ctypes.byref(h_))
    else:
        rc = _lib().mbl_build_sector_nup(ctx.handle, L, nup, float(h), sd, ctypes.byref(h_))
    _check(rc, ctx.handle)
    return Sector(ctx, h_, L)


def build_sector_fields(ctx: Context, L: int, h_i, J: float = 1.0, nup: int | None = None) -> Sector:
    hi = np.ascontiguousarray(h_i, dtype=np.float64)
    h_ = ctypes.c_void_p()
    if nup is None:
        rc = _lib().mbl_build_sector_fields(ctx.handle, L, _ptr(hi), float(J), ctypes.byref(h_))
    else:
        rc = _lib().mbl_build_sector_fields_nup(ctx.handle, L, nup, _ptr(hi), float(J), ctypes.byref(h_))
    _check(rc, ctx.handle)
    return Sector(ctx, h_, L)


def extremal_bounds(sec: Sector):
    lo, hi = ctypes.c_double(), ctypes.c_double()
    _check(_lib().mbl_extremal_bounds(sec.handle, ctypes.byref(lo), ctypes.byref(hi)), sec.ctx.handle)
    return lo.value, hi.value


def analyse(sec: Sector, nev: int = 50, block: int = 8) -> dict:
    """Symbolic analysis of the sector's L (cached): predicted fill-in, flops and device footprint."""
    s = PlanStats()
    _check(_lib().mbl_analyse(sec.handle, nev, block, ctypes.byref(s)), sec.ctx.handle)
    return {f: getattr(s, f) for f, _ in PlanStats._fields_}


class Factorization:
    def __init__(self, sec: Sector, handle):
        self.sec, self.handle = sec, handle

    def stats(self) -> dict:
        s = FactorStats()
        _check(_lib().mbl_factor_stats_get(self.handle, ctypes.byref(s)), self.sec.ctx.handle)
        out = {}
        for f, _ in FactorStats._fields_:
            v = getattr(s, f)
            out[f] = list(v) if isinstance(v, ctypes.Array) else v
        return out

    def set_trace(self, on: bool = True):
        """Record per-launch start/end device clocks of later solves (diagnostic)."""
        _check(_lib().mbl_factor_trace(self.handle, 1 if on else 0), self.sec.ctx.handle)

    def trace(self):
        """(t0_ns, t1_ns, kind) arrays of the latest traced solve; kind 0 gather, 1 forward step,
        2 backward level start, 3 backward update."""
        cnt = ctypes.c_int()
        _check(_lib().mbl_factor_trace_get(self.handle, None, None, None, 0, ctypes.byref(cnt)), self.sec.ctx.handle)
        n = cnt.value
        t0 = np.zeros(max(n, 1), dtype=np.uint64)
        t1 = np.zeros(max(n, 1), dtype=np.uint64)
        kind = np.zeros(max(n, 1), dtype=np.int32)
        _check(_lib().mbl_factor_trace_get(self.handle, t0.ctypes.data, t1.ctypes.data, kind.ctypes.data, n,
                                           ctypes.byref(cnt)), self.sec.ctx.handle)
        return t0[:n], t1[:n], kind[:n]

    def solve(self, b: np.ndarray, refine: bool = True) -> np.ndarray:
        B = np.asfortranarray(b, dtype=np.float64)
        if B.ndim == 1:
            B = B[:, None]
        X = np.zeros_like(B, order="F")
        _check(_lib().mbl_factor_solve(self.handle, _ptr(B), _ptr(X), B.shape[1], 1 if refine else 0),
               self.sec.ctx.handle)
        return X[:, 0] if np.ndim(b) == 1 else X

    def solve_dev(self, d_b, d_x, nrhs: int, refine: bool = False, stream=None):
        """Device variant of solve: d_b, d_x are float64 CUDA tensors holding n x nrhs column-major
        blocks (nrhs contiguous vectors of length n)."""
        s = ctypes.c_void_p(stream.cuda_stream) if stream is not None else None
        _check(_lib().mbl_factor_solve_dev(self.handle, ctypes.c_void_p(d_b.data_ptr()), ctypes.c_void_p(d_x.data_ptr()),
                                           nrhs, 1 if refine else 0, s), self.sec.ctx.handle)

    def close(self):
        if getattr(self, "handle", None):
            _lib().mbl_factor_destroy(self.handle)
            self.handle = None

    def __del__(self):
        # at interpreter shutdown the release order is arbitrary and the CUDA runtime may be going
        # away: leave the memory to process exit instead of calling into the library
        if sys.is_finalizing():
            return
        try:
            self.close()
        except Exception:
            pass


def factor_solve_batch_dev(facts, d_bs, d_xs, nrhs: int, stream=None):
    """Unrefined solves of several factorizations of one sector shape in shared launches:
    d_xs[k] = (L D L^T)_k^-1 d_bs[k] (torch float64 CUDA tensors, n x nrhs column-major)."""
    K = len(facts)
    fa = (ctypes.c_void_p * K)(*[f.handle.value for f in facts])
    ba = (ctypes.c_void_p * K)(*[t.data_ptr() for t in d_bs])
    xa = (ctypes.c_void_p * K)(*[t.data_ptr() for t in d_xs])
    s = ctypes.c_void_p(stream.cuda_stream) if stream is not None else None
    _check(_lib().mbl_factor_solve_batch_dev(fa, K, ba, xa, nrhs, s), facts[0].sec.ctx.handle)


def factor(sec: Sector, sigma: float, opts: Opts | None = None, **kw) -> Factorization:
    o = opts if opts is not None else default_opts(**kw)
    h = ctypes.c_void_p()
    _check(_lib().mbl_factor(sec.handle, float(sigma), ctypes.byref(o), ctypes.byref(h)), sec.ctx.handle)
    return Factorization(sec, h)


@dataclass
class NearResult:
    evals: np.ndarray
    evecs: np.ndarray  # dim x nev (column j = eigenvector j)
    resid: np.ndarray
    nconv: int
    sigma: float
    stats: dict


def solve_near(sec: Sector, eps: float, nev: int, opts: Opts | None = None, allow_partial: bool = False,
               **kw) -> NearResult:
    o = opts if opts is not None else default_opts(**kw)
    ev = np.zeros(nev)
    vec = np.zeros((sec.dim, nev), order="F")
    res = np.zeros(nev)
    nc, sg, st = ctypes.c_int(), ctypes.c_double(), SolveStats()
    rc = _lib().mbl_solve_near(sec.handle, float(eps), nev, ctypes.byref(o), _ptr(ev), _ptr(vec), _ptr(res),
                               ctypes.byref(nc), ctypes.byref(sg), ctypes.byref(st))
    if not (allow_partial and rc == _capi.MBL_ERR_NOT_CONVERGED):
        _check(rc, sec.ctx.handle)
    return NearResult(ev, vec, res, nc.value, sg.value, {f: getattr(st, f) for f, _ in SolveStats._fields_})


def solve_near_dev(sec: Sector, eps: float, nev: int, d_evals, d_evecs, d_resid, stream=None,
                   opts: Opts | None = None, **kw):
    """Device variant: d_* are torch CUDA tensors (float64) of sizes nev, dim*nev, nev."""
    o = opts if opts is not None else default_opts(**kw)
    nc, sg, st = ctypes.c_int(), ctypes.c_double(), SolveStats()
    s = ctypes.c_void_p(stream.cuda_stream) if stream is not None else None
    _check(_lib().mbl_solve_near_dev(sec.handle, float(eps), nev, ctypes.byref(o), ctypes.c_void_p(d_evals.data_ptr()),
                                     ctypes.c_void_p(d_evecs.data_ptr()), ctypes.c_void_p(d_resid.data_ptr()),
                                     ctypes.byref(nc), ctypes.byref(sg), ctypes.byref(st), s), sec.ctx.handle)
    return nc.value, sg.value, {f: getattr(st, f) for f, _ in SolveStats._fields_}


def observables(ctx: Context, L: int, evals: np.ndarray, evecs: np.ndarray, nup: int | None = None):
    """r, r_mean, S_1^P, S^E of eigenpairs of the sector (L, nup) (None: S^z_tot = 0, even L)."""
    ev = np.ascontiguousarray(evals, dtype=np.float64)
    V = np.asfortranarray(evecs, dtype=np.float64)
    nev = len(ev)
    r = np.zeros(max(nev - 2, 1))
    rm = np.zeros(1)
    s1p = np.zeros(nev)
    se = np.zeros(nev)
    tail = (_ptr(ev), _ptr(V), _ptr(r), _ptr(rm), _ptr(s1p), _ptr(se))
    if nup is None:
        rc = _lib().mbl_observables(ctx.handle, L, nev, *tail)
    else:
        rc = _lib().mbl_observables_nup(ctx.handle, L, nup, nev, *tail)
    _check(rc, ctx.handle)
    return r[: max(nev - 2, 0)], float(rm[0]), s1p, se


def observables_dev(ctx: Context, L: int, nev: int, d_evals, d_evecs, d_r, d_rmean, d_s1p, d_se, stream=None,
                    nup: int | None = None):
    s = ctypes.c_void_p(stream.cuda_stream) if stream is not None else None
    tail = tuple(ctypes.c_void_p(t.data_ptr()) for t in (d_evals, d_evecs, d_r, d_rmean, d_s1p, d_se)) + (s,)
    if nup is None:
        rc = _lib().mbl_observables_dev(ctx.handle, L, nev, *tail)
    else:
        rc = _lib().mbl_observables_nup_dev(ctx.handle, L, nup, nev, *tail)
    _check(rc, ctx.handle)


def observables_extra(ctx: Context, L: int, evecs: np.ndarray, q: float = 2.0, nup: int | None = None):
    """KL of adjacent columns (nev - 1), S_q^P, bipartite fluctuation F and dynamic fraction f of
    the columns of evecs (dim x nev, ascending eigenvalues) of the sector (L, nup)."""
    V = np.asfortranarray(evecs, dtype=np.float64)
    nev = V.shape[1]
    kl = np.zeros(max(nev - 1, 1))
    sqp, fl, dyn = np.zeros(nev), np.zeros(nev), np.zeros(nev)
    tail = (_ptr(V), float(q), _ptr(kl), _ptr(sqp), _ptr(fl), _ptr(dyn))
    if nup is None:
        rc = _lib().mbl_observables_extra(ctx.handle, L, nev, *tail)
    else:
        rc = _lib().mbl_observables_extra_nup(ctx.handle, L, nup, nev, *tail)
    _check(rc, ctx.handle)
    return kl[: max(nev - 1, 0)], sqp, fl, dyn


def observables_extra_dev(ctx: Context, L: int, nev: int, d_evecs, q, d_kl, d_sqp, d_fluct, d_dynf, stream=None,
                          nup: int | None = None):
    s = ctypes.c_void_p(stream.cuda_stream) if stream is not None else None
    tail = (ctypes.c_void_p(d_evecs.data_ptr()), float(q)) + tuple(
        ctypes.c_void_p(t.data_ptr()) for t in (d_kl, d_sqp, d_fluct, d_dynf)) + (s,)
    if nup is None:
        rc = _lib().mbl_observables_extra_dev(ctx.handle, L, nev, *tail)
    else:
        rc = _lib().mbl_observables_extra_nup_dev(ctx.handle, L, nup, nev, *tail)
    _check(rc, ctx.handle)


def entanglement_noalloc_dev(ctx: Context, L: int, nev: int, d_evecs, d_se, stream=None):
    """S^E of nev device vectors with no device allocation (static library scratch; L <= 16,
    nev <= 64).  d_evecs: torch float64 CUDA tensor of dim*nev (column-major), d_se: nev.
    Calls on one device must not overlap."""
    s = ctypes.c_void_p(stream.cuda_stream) if stream is not None else None
    _check(_lib().mbl_entanglement_noalloc_dev(ctx.handle, L, nev, ctypes.c_void_p(d_evecs.data_ptr()),
                                               ctypes.c_void_p(d_se.data_ptr()), s), ctx.handle)


# ------------------------------------------------------------------------------------------
# Serving (continuous batching with HBM admission): a thin face of mbl_server_* / mbl_submit /
# mbl_poll / mbl_wait.
# ------------------------------------------------------------------------------------------
@dataclass
class ServedResult:
    status: int
    nconv: int
    L: int
    dim: int
    sigma: float
    evals: np.ndarray
    resid: np.ndarray
    r: np.ndarray
    r_mean: float
    s1p: np.ndarray
    se: np.ndarray
    evecs: np.ndarray | None
    t_submit_ms: float
    t_admit_ms: float
    t_end_ms: float
    d_start_ms: float
    d_end_ms: float
    reserved_bytes: int
    factor_reused: int = 0


def _dim_of(L: int, nup: int = 0) -> int:
    """Dimension C(L, nup) of a sector (nup = 0: the S^z_tot = 0 sector, L/2 up spins)."""
    return math.comb(L, nup if nup > 0 else L // 2)


class Server:
    """Worker threads of a context serving (L, h, seed, eps, nev) requests as memory allows."""

    def __init__(self, ctx: Context, slots: int = 4, hbm_budget_bytes: int = 0, batch_jobs: int = 16,
                 batch_window_us: float = 300.0, cache_fraction: float = 0.25, batch_lanes: int = 2):
        """`batch_jobs` > 1 batches the workers' triangular solves of one sector size into shared
        launches (at most that many jobs per launch, waiting up to `batch_window_us` while one of the
        `batch_lanes` streams is idle); 1 turns it off.  `cache_fraction` of the budget keeps finished
        jobs' live factorizations for repeated requests."""
        self.ctx = ctx
        self._req = {}
        _check(_lib().mbl_server_batching(ctx.handle, batch_jobs, float(batch_window_us), int(batch_lanes)),
               ctx.handle)
        _check(_lib().mbl_server_cache(ctx.handle, float(cache_fraction)), ctx.handle)
        _check(_lib().mbl_server_start(ctx.handle, slots, hbm_budget_bytes), ctx.handle)

    def submit(self, L: int, h: float, seed: int, eps: float, nev: int, precision: int = MBL_PREC_FP32,
               want_vectors: bool = False, fields: np.ndarray | None = None, nup: int = 0) -> int:
        """Queue a job; `fields` (h_i, length L) replaces the seeded disorder of (h, seed); `nup`
        selects the sector (0: S^z_tot = 0 of even L)."""
        fp = None
        if fields is not None:
            fields = np.ascontiguousarray(fields, dtype=np.float64)
            if fields.shape != (L,):
                raise ValueError("fields must have length L")
            fp = _ptr(fields)
        q = _capi.Request(L, float(h), seed, fp, float(eps), nev, precision, 1 if want_vectors else 0, nup)
        t = ctypes.c_uint64()
        _check(_lib().mbl_submit(self.ctx.handle, ctypes.byref(q), ctypes.byref(t)), self.ctx.handle)
        self._req[t.value] = (L, nup, nev, want_vectors)
        return t.value

    def _collect(self, ticket: int, timeout_s: float | None):
        L, nup, nev, vec = self._req[ticket]
        n = _dim_of(L, nup)
        ev, rs, r, s1, se = (np.zeros(nev), np.zeros(nev), np.zeros(max(nev - 2, 1)), np.zeros(nev),
                             np.zeros(nev))
        V = np.zeros((n, nev), order="F") if vec else None
        out = _capi.Result()
        out.evals, out.resid, out.r, out.s1p, out.se = (_ptr(ev), _ptr(rs), _ptr(r), _ptr(s1), _ptr(se))
        out.evecs = _ptr(V) if vec else None
        if timeout_s is None:
            rc = _lib().mbl_poll(self.ctx.handle, ticket, ctypes.byref(out))
        else:
            rc = _lib().mbl_wait(self.ctx.handle, ticket, float(timeout_s), ctypes.byref(out))
        if rc == _capi.MBL_PENDING:
            return None
        del self._req[ticket]
        if rc not in (_capi.MBL_OK, _capi.MBL_ERR_NOT_CONVERGED):
            _check(rc, self.ctx.handle)
        return ServedResult(rc, out.nconv, out.L, out.dim, out.sigma, ev, rs, r[: max(nev - 2, 0)], out.r_mean, s1,
                            se, V, out.t_submit_ms, out.t_admit_ms, out.t_end_ms, out.d_start_ms, out.d_end_ms,
                            out.reserved_bytes, out.factor_reused)

    def poll(self, ticket: int):
        """The result if finished, else None (non-blocking)."""
        return self._collect(ticket, None)

    def wait(self, ticket: int, timeout_s: float = 0.0):
        """Block until finished (timeout_s <= 0: no limit); None if the timeout expired."""
        return self._collect(ticket, timeout_s)

    def stats(self) -> dict:
        st = _capi.ServerStats()
        _check(_lib().mbl_server_stats_get(self.ctx.handle, ctypes.byref(st)), self.ctx.handle)
        return {f: getattr(st, f) for f, _ in _capi.ServerStats._fields_}

    def stop(self):
        if self.ctx.handle:
            _lib().mbl_server_stop(self.ctx.handle)

