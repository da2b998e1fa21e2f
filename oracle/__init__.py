"""Plain CPU FP64 oracle for the shift-invert exact diagonalization of the random-field
Heisenberg chain (Luitz, Laflorencie, Alet, arXiv:1411.0660).

TEST INFRASTRUCTURE ONLY.  Only ``tests/``, ``__graft_entry__.smoke()`` and the CPU-baseline
leg of ``bench.py`` may import this package.  It shares no code with the GPU library: the C
source next to this file is compiled on its own with gcc and loaded through ctypes.

What each function computes and the passage it follows:

* ``fields``            Eq. 1, h_i uniform on [-h, h] (SplitMix64 stream, a stated reading)
* ``basis``             magnetization sectors of the numerical-method section (S^z = 0 of even
                        L; for odd L its "S^z = 1", read as n_up = (L + 1) / 2) or any n_up;
                        brute force
* ``csr``               Eq. 1 restricted to the sector, binary search of flipped states
* ``syev``              dense Householder + implicit QL
* ``extremal_bounds``   E_0, E_max of the numerical-method section
* ``nearest``           eigenpairs closest to the target, numerical-method section
* ``gap_ratio``         r^(n), "level statistics" paragraph
* ``s1p``               S_1^P, "Hilbert space localization" paragraph
* ``entanglement``      S^E = -Tr rho_A ln rho_A, A = sites 0 .. floor(L/2) - 1, "entanglement
                        entropy" paragraph
* ``kl``                KL divergence of nearby eigenstates, "level statistics and eigenvectors
                        similarity" paragraph
* ``sqp``               S_q^P, q != 1, "Hilbert space localization" paragraph
* ``fluct``             bipartite fluctuation F of S^z_A, "entanglement entropy" paragraph
* ``dynf``              dynamic spin fraction f, supplementary section on the dynamical spin fraction
"""
from __future__ import annotations

import ctypes
import os
import platform
import subprocess
from dataclasses import dataclass

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "mbl_oracle.c")
_LIB = os.path.join(_HERE, "_build", "liborc.so")

_f64p = np.ctypeslib.ndpointer(dtype=np.float64, flags="C_CONTIGUOUS")
_i64p = np.ctypeslib.ndpointer(dtype=np.int64, flags="C_CONTIGUOUS")
_i32p = np.ctypeslib.ndpointer(dtype=np.int32, flags="C_CONTIGUOUS")
_u32p = np.ctypeslib.ndpointer(dtype=np.uint32, flags="C_CONTIGUOUS")


def build(force: bool = False) -> str:
    """Compile the oracle with gcc (no FMA contraction; portable flags only)."""
    os.makedirs(os.path.dirname(_LIB), exist_ok=True)
    stamp = os.path.join(os.path.dirname(_LIB), "ARCH")
    if not (os.path.exists(stamp) and open(stamp).read().strip() == platform.machine()):
        force = True
    if force or not os.path.exists(_LIB) or os.path.getmtime(_LIB) < max(
        os.path.getmtime(_SRC), os.path.getmtime(os.path.join(_HERE, "mbl_oracle.h"))
    ):
        tmp = _LIB + f".{os.getpid()}.tmp"
        subprocess.check_call(
            ["gcc", "-O2", "-std=c11", "-fPIC", "-shared", "-ffp-contract=off", "-o", tmp, _SRC, "-lm"]
        )
        os.replace(tmp, _LIB)
        with open(stamp, "w") as f:
            f.write(platform.machine())
    return _LIB


_lib = None


def lib():
    global _lib
    if _lib is None:
        build()
        L = ctypes.CDLL(_LIB)
        L.orc_fields.argtypes = [ctypes.c_int, ctypes.c_double, ctypes.c_uint64, _f64p]
        L.orc_binom.argtypes = [ctypes.c_int, ctypes.c_int]
        L.orc_binom.restype = ctypes.c_int64
        L.orc_basis.argtypes = [ctypes.c_int, ctypes.c_void_p]
        L.orc_basis.restype = ctypes.c_int64
        L.orc_basis_sector.argtypes = [ctypes.c_int, ctypes.c_int, ctypes.c_void_p]
        L.orc_basis_sector.restype = ctypes.c_int64
        L.orc_nnz.argtypes = [ctypes.c_int, _u32p, ctypes.c_int64]
        L.orc_nnz.restype = ctypes.c_int64
        L.orc_csr.argtypes = [ctypes.c_int, _f64p, ctypes.c_double, _u32p, ctypes.c_int64, _i64p, _i32p, _f64p]
        L.orc_spmv.argtypes = [ctypes.c_int64, _i64p, _i32p, _f64p, ctypes.c_double, _f64p, _f64p]
        L.orc_syev.argtypes = [ctypes.c_int, _f64p, _f64p, ctypes.c_int]
        L.orc_stev.argtypes = [ctypes.c_int, _f64p, _f64p, _f64p, ctypes.c_void_p]
        L.orc_extremal_lanczos.argtypes = [ctypes.c_int64, _i64p, _i32p, _f64p, ctypes.c_double,
                                           ctypes.c_uint64, ctypes.POINTER(ctypes.c_double),
                                           ctypes.POINTER(ctypes.c_double)]
        L.orc_nearest_dense.argtypes = [ctypes.c_int64, _i64p, _i32p, _f64p, ctypes.c_double, ctypes.c_int,
                                        ctypes.POINTER(ctypes.c_double), ctypes.POINTER(ctypes.c_double),
                                        ctypes.POINTER(ctypes.c_double), _f64p, ctypes.c_void_p]
        L.orc_ldlt_analyse.argtypes = [ctypes.c_int64, _i64p, _i32p]
        L.orc_ldlt_analyse.restype = ctypes.c_void_p
        L.orc_ldlt_factor.argtypes = [ctypes.c_void_p, _i64p, _i32p, _f64p, ctypes.c_double, ctypes.c_double]
        L.orc_ldlt_solve.argtypes = [ctypes.c_void_p, _f64p, _f64p]
        for nm in ("orc_ldlt_nnz", "orc_ldlt_negative", "orc_ldlt_perturbed"):
            getattr(L, nm).argtypes = [ctypes.c_void_p]
            getattr(L, nm).restype = ctypes.c_int64
        L.orc_ldlt_free.argtypes = [ctypes.c_void_p]
        L.orc_kl.argtypes = [ctypes.c_int64, _f64p, _f64p]
        L.orc_kl.restype = ctypes.c_double
        L.orc_sqp.argtypes = [ctypes.c_int64, _f64p, ctypes.c_double]
        L.orc_sqp.restype = ctypes.c_double
        L.orc_fluct.argtypes = [ctypes.c_int, _u32p, ctypes.c_int64, _f64p]
        L.orc_fluct.restype = ctypes.c_double
        L.orc_dynf.argtypes = [ctypes.c_int, _u32p, ctypes.c_int64, _f64p]
        L.orc_dynf.restype = ctypes.c_double
        L.orc_nearest_shift_invert.argtypes = [ctypes.c_int64, _i64p, _i32p, _f64p, ctypes.c_double, ctypes.c_int,
                                               ctypes.c_double, _f64p, _f64p, _f64p]
        L.orc_gap_ratio.argtypes = [ctypes.c_int, _f64p, _f64p, ctypes.POINTER(ctypes.c_double)]
        L.orc_s1p.argtypes = [ctypes.c_int64, _f64p]
        L.orc_s1p.restype = ctypes.c_double
        L.orc_entanglement.argtypes = [ctypes.c_int, _u32p, ctypes.c_int64, _f64p]
        L.orc_entanglement.restype = ctypes.c_double
        _lib = L
    return _lib


# ---------------------------------------------------------------------------------------------
def fields(L: int, h: float, seed: int) -> np.ndarray:
    out = np.zeros(L, dtype=np.float64)
    lib().orc_fields(L, float(h), ctypes.c_uint64(seed & (2**64 - 1)), out)
    return out


def binom(n: int, k: int) -> int:
    return int(lib().orc_binom(n, k))


def default_nup(L: int) -> int:
    """Up spins of the sector the numerical-method section uses at chain length L: S^z = 0
    (L/2) for even L; for odd L its "S^z = 1" read as sum_i sigma^z_i = n_up - n_down = 1."""
    return L // 2 if L % 2 == 0 else (L + 1) // 2


def basis(L: int, nup: int | None = None) -> np.ndarray:
    k = default_nup(L) if nup is None else nup
    n = lib().orc_basis_sector(L, k, None)
    if n < 0:
        raise ValueError(f"invalid sector L={L}, nup={k}")
    st = np.zeros(n, dtype=np.uint32)
    lib().orc_basis_sector(L, k, st.ctypes.data)
    return st


@dataclass
class CSR:
    n: int
    rowptr: np.ndarray
    col: np.ndarray
    val: np.ndarray

    def matvec(self, x: np.ndarray, shift: float = 0.0) -> np.ndarray:
        x = np.ascontiguousarray(x, dtype=np.float64)
        y = np.zeros(self.n, dtype=np.float64)
        lib().orc_spmv(self.n, self.rowptr, self.col, self.val, float(shift), x, y)
        return y

    def dense(self) -> np.ndarray:
        A = np.zeros((self.n, self.n))
        for i in range(self.n):
            for p in range(self.rowptr[i], self.rowptr[i + 1]):
                A[i, self.col[p]] = self.val[p]
        return A


def csr(L: int, hi: np.ndarray, J: float = 1.0, states: np.ndarray | None = None) -> CSR:
    st = basis(L) if states is None else states
    n = len(st)
    hi = np.ascontiguousarray(hi, dtype=np.float64)
    nnz = lib().orc_nnz(L, st, n)
    rowptr = np.zeros(n + 1, dtype=np.int64)
    col = np.zeros(nnz, dtype=np.int32)
    val = np.zeros(nnz, dtype=np.float64)
    lib().orc_csr(L, hi, float(J), st, n, rowptr, col, val)
    return CSR(n, rowptr, col, val)


def syev(A: np.ndarray, vectors: bool = True):
    n = A.shape[0]
    M = np.asfortranarray(A, dtype=np.float64).copy(order="F")
    flat = M.reshape(-1, order="F").copy()
    w = np.zeros(n)
    rc = lib().orc_syev(n, flat, w, 1 if vectors else 0)
    if rc != 0:
        raise RuntimeError("QL iteration did not converge")
    if vectors:
        return w, flat.reshape((n, n), order="F")
    return w


def stev(d: np.ndarray, e: np.ndarray):
    n = len(d)
    w = np.zeros(n)
    zl = np.zeros(n)
    ee = np.zeros(max(n, 1))
    ee[: n - 1] = e
    lib().orc_stev(n, np.ascontiguousarray(d, dtype=np.float64), ee, w, zl.ctypes.data)
    return w, zl


def extremal_bounds(H: CSR, tol: float = 1e-13, seed: int = 0xB0B) -> tuple[float, float]:
    emin, emax = ctypes.c_double(), ctypes.c_double()
    steps = lib().orc_extremal_lanczos(H.n, H.rowptr, H.col, H.val, tol, seed, ctypes.byref(emin), ctypes.byref(emax))
    if steps < 0:
        raise RuntimeError(f"extremal Lanczos did not converge in {-steps} steps")
    return emin.value, emax.value


@dataclass
class Eigs:
    evals: np.ndarray
    evecs: np.ndarray  # n x nev
    resid: np.ndarray
    emin: float
    emax: float
    sigma: float


def nearest_dense(H: CSR, eps: float, nev: int) -> Eigs:
    ev = np.zeros(nev)
    vec = np.zeros(H.n * nev)
    emin, emax, sig = ctypes.c_double(), ctypes.c_double(), ctypes.c_double()
    rc = lib().orc_nearest_dense(H.n, H.rowptr, H.col, H.val, float(eps), nev, ctypes.byref(emin),
                                 ctypes.byref(emax), ctypes.byref(sig), ev, vec.ctypes.data)
    if rc != 0:
        raise RuntimeError(f"dense eigensolver failed ({rc})")
    V = vec.reshape((nev, H.n)).T.copy()
    res = np.array([np.linalg.norm(H.matvec(V[:, j]) - ev[j] * V[:, j]) for j in range(nev)])
    return Eigs(ev, V, res, emin.value, emax.value, sig.value)


def nearest_shift_invert(H: CSR, sigma: float, nev: int, hnorm: float, emin=np.nan, emax=np.nan) -> Eigs:
    ev = np.zeros(nev)
    vec = np.zeros(H.n * nev)
    res = np.zeros(nev)
    rc = lib().orc_nearest_shift_invert(H.n, H.rowptr, H.col, H.val, float(sigma), nev, float(hnorm), ev, vec, res)
    if rc < 0:
        raise RuntimeError(f"shift-invert Lanczos did not converge ({rc})")
    return Eigs(ev, vec.reshape((nev, H.n)).T.copy(), res, emin, emax, sigma)


class LDLT:
    """Sparse LDL^T of H - sigma I (minimum-degree order, no pivoting, static perturbation)."""

    def __init__(self, H: CSR):
        self.H = H
        self._h = lib().orc_ldlt_analyse(H.n, H.rowptr, H.col)
        if not self._h:
            raise MemoryError("ordering failed")

    def factor(self, sigma: float, tiny: float = 0.0):
        lib().orc_ldlt_factor(self._h, self.H.rowptr, self.H.col, self.H.val, float(sigma), float(tiny))
        return self

    def solve(self, b: np.ndarray) -> np.ndarray:
        x = np.zeros(self.H.n)
        lib().orc_ldlt_solve(self._h, np.ascontiguousarray(b, dtype=np.float64), x)
        return x

    @property
    def nnz(self) -> int:
        return int(lib().orc_ldlt_nnz(self._h))

    @property
    def negative(self) -> int:
        return int(lib().orc_ldlt_negative(self._h))

    @property
    def perturbed(self) -> int:
        return int(lib().orc_ldlt_perturbed(self._h))

    def __del__(self):
        if getattr(self, "_h", None):
            lib().orc_ldlt_free(self._h)
            self._h = None


def gap_ratio(evals: np.ndarray):
    nev = len(evals)
    r = np.zeros(max(nev - 2, 0))
    rm = ctypes.c_double()
    lib().orc_gap_ratio(nev, np.ascontiguousarray(evals, dtype=np.float64), r if nev > 2 else np.zeros(1),
                        ctypes.byref(rm))
    return r, rm.value


def s1p(y: np.ndarray) -> float:
    y = np.ascontiguousarray(y, dtype=np.float64)
    return float(lib().orc_s1p(len(y), y))


def entanglement(L: int, y: np.ndarray, states: np.ndarray | None = None) -> float:
    st = basis(L) if states is None else states
    y = np.ascontiguousarray(y, dtype=np.float64)
    return float(lib().orc_entanglement(L, st, len(st), y))


def kl(y: np.ndarray, z: np.ndarray) -> float:
    y = np.ascontiguousarray(y, dtype=np.float64)
    z = np.ascontiguousarray(z, dtype=np.float64)
    return float(lib().orc_kl(len(y), y, z))


def sqp(y: np.ndarray, q: float) -> float:
    y = np.ascontiguousarray(y, dtype=np.float64)
    return float(lib().orc_sqp(len(y), y, float(q)))


def fluct(L: int, y: np.ndarray, states: np.ndarray | None = None) -> float:
    st = basis(L) if states is None else states
    y = np.ascontiguousarray(y, dtype=np.float64)
    return float(lib().orc_fluct(L, st, len(st), y))


def dynf(L: int, y: np.ndarray, states: np.ndarray | None = None) -> float:
    st = basis(L) if states is None else states
    y = np.ascontiguousarray(y, dtype=np.float64)
    return float(lib().orc_dynf(L, st, len(st), y))


# ---------------------------------------------------------------------------------------------
DENSE_MAX_N = 3432  # L <= 14: full dense diagonalization; larger sectors use shift-invert


@dataclass
class Job:
    L: int
    h: float
    seed: int
    eps: float
    nev: int
    J: float = 1.0
    nup: int | None = None  # up spins of the sector (None: default_nup(L))


@dataclass
class JobResult:
    emin: float
    emax: float
    sigma: float
    evals: np.ndarray
    evecs: np.ndarray
    resid: np.ndarray
    r: np.ndarray
    r_mean: float
    s1p: np.ndarray
    se: np.ndarray


def solve_job(job: Job, method: str = "auto", hi: np.ndarray | None = None) -> JobResult:
    """The whole path for one (L, h, seed, eps, nev): fields, sector, H, E_min/E_max,
    sigma = E_min + eps (E_max - E_min), the nev eigenpairs nearest sigma, observables."""
    st = basis(job.L, job.nup)
    if hi is None:
        hi = fields(job.L, job.h, job.seed)
    H = csr(job.L, hi, job.J, st)
    if method == "auto":
        method = "dense" if H.n <= DENSE_MAX_N else "si"
    if method == "dense":
        e = nearest_dense(H, job.eps, job.nev)
    else:
        emin, emax = extremal_bounds(H)
        sigma = emin + job.eps * (emax - emin)
        hn = max(abs(emin), abs(emax))
        e = nearest_shift_invert(H, sigma, job.nev, hn, emin, emax)
    r, rm = gap_ratio(e.evals)
    s1 = np.array([s1p(e.evecs[:, j]) for j in range(job.nev)])
    se = np.array([entanglement(job.L, e.evecs[:, j], st) for j in range(job.nev)])
    return JobResult(e.emin, e.emax, e.sigma, e.evals, e.evecs, e.resid, r, rm, s1, se)
