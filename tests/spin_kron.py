"""Independent full-Hilbert-space construction of the chain by Kronecker products (test helper).

Used only to pin the oracle: it builds Eq. 1 in the 2^L-dimensional space from 2x2 spin
matrices with numpy, a route that shares nothing with the oracle's bit-manipulation CSR.
Site i is the i-th least significant tensor factor; local state 1 is spin up.
"""
import numpy as np

SZ = np.array([[-0.5, 0.0], [0.0, 0.5]])
SP = np.array([[0.0, 0.0], [1.0, 0.0]])  # |up><down|
SM = SP.T
I2 = np.eye(2)


def site_op(op, i, L):
    """op acting on site i (bit i) of an L-site chain."""
    out = np.array([[1.0]])
    for s in range(L - 1, -1, -1):  # most significant factor first
        out = np.kron(out, op if s == i else I2)
    return out


def hamiltonian_full(L, hi, J=1.0):
    dim = 2**L
    H = np.zeros((dim, dim))
    for i in range(L):
        j = (i + 1) % L
        H += J * (site_op(SZ, i, L) @ site_op(SZ, j, L))
        H += 0.5 * J * (site_op(SP, i, L) @ site_op(SM, j, L) + site_op(SM, i, L) @ site_op(SP, j, L))
        H += hi[i] * site_op(SZ, i, L)
    return H


def total_spin_sq(L):
    Sx = sum(0.5 * (site_op(SP, i, L) + site_op(SM, i, L)) for i in range(L))
    Sy_sq = -0.25 * sum((site_op(SP, i, L) - site_op(SM, i, L)) for i in range(L)) @ sum(
        (site_op(SP, i, L) - site_op(SM, i, L)) for i in range(L)
    )
    Sz = sum(site_op(SZ, i, L) for i in range(L))
    return Sx @ Sx + Sy_sq + Sz @ Sz


def sector_indices(L, m_up):
    return np.array([s for s in range(2**L) if bin(s).count("1") == m_up], dtype=np.int64)


def schmidt_entropy(L, y_full):
    """S^E of a full-space vector for A = low L/2 bits, via numpy SVD of the reshaped vector."""
    LA = L // 2
    M = y_full.reshape(2 ** (L - LA), 2**LA)  # row index = high bits (B), column = low bits (A)
    s = np.linalg.svd(M, compute_uv=False)
    p = s**2 / np.sum(s**2)
    p = p[p > 1e-15]
    return float(-np.sum(p * np.log(p)))
