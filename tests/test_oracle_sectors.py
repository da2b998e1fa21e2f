"""Pins of the oracle's general magnetization sectors (odd L, n_up != L/2) against constructions
that share nothing with it: the full 2^L Hamiltonian from Kronecker products, closed forms of the
one-magnon band, the spin-flip symmetry between sectors, and hand-computed Schmidt spectra.

The numerical-method section uses the S^z = 0 sector of even L and the "S^z = 1" sector of odd L
(L = 15, 17, 19), read here as n_up - n_down = 1.
"""
import math

import numpy as np
import pytest

from spin_kron import hamiltonian_full, schmidt_entropy, sector_indices


@pytest.mark.parametrize("L", [2, 3, 4, 5, 7, 9, 12])
def test_sector_basis_dimension_order_popcount(orc, L):
    for nup in range(L + 1):
        st = orc.basis(L, nup)
        assert len(st) == math.comb(L, nup)
        assert np.all(np.diff(st.astype(np.int64)) > 0)
        assert all(bin(int(s)).count("1") == nup for s in st)
        assert np.all(st < (1 << L))
    with pytest.raises(ValueError):
        orc.basis(L, L + 1)


def test_default_sector_of_the_paper(orc):
    assert [orc.default_nup(L) for L in (12, 14, 15, 17, 19, 22)] == [6, 7, 8, 9, 10, 11]
    assert np.array_equal(orc.basis(16), orc.basis(16, 8))


@pytest.mark.parametrize("L,nup,J", [(3, 1, 1.0), (3, 2, 1.0), (5, 2, 0.8), (5, 3, 1.0), (6, 2, 1.0),
                                     (7, 4, 1.2), (8, 3, 1.0), (9, 5, 1.0)])
def test_sector_csr_matches_kronecker_construction(orc, L, nup, J):
    rng = np.random.default_rng(100 * L + nup)
    hi = rng.uniform(-2, 2, L)
    idx = sector_indices(L, nup)
    want = hamiltonian_full(L, hi, J)[np.ix_(idx, idx)]
    got = orc.csr(L, hi, J, orc.basis(L, nup)).dense()
    assert np.abs(got - want).max() < 1e-13


@pytest.mark.parametrize("L", [5, 6, 7])
def test_sectors_assemble_the_full_spectrum(orc, L):
    """H conserves S^z_tot, so the sectors' spectra together are the spectrum of H on all 2^L
    states (a plausible slip in one sector's basis or CSR changes the union)."""
    hi = np.random.default_rng(L).uniform(-1.5, 1.5, L)
    parts = []
    for nup in range(L + 1):
        H = orc.csr(L, hi, 1.0, orc.basis(L, nup))
        parts.append(orc.syev(H.dense(), vectors=False))
    got = np.sort(np.concatenate(parts))
    want = np.linalg.eigvalsh(hamiltonian_full(L, hi, 1.0))
    assert np.abs(got - want).max() < 1e-12


@pytest.mark.parametrize("L", [3, 4, 5, 8, 9, 11])
def test_one_magnon_band_closed_form(orc, L):
    """One up spin in a zero field on a ring: the two bonds at the flipped site turn from +J/4 to
    -J/4 and the spin hops with amplitude J/2, so E(q) = J (L/4 - 1) + J cos q, q = 2 pi m / L."""
    J = 0.9
    H = orc.csr(L, np.zeros(L), J, orc.basis(L, 1))
    got = np.sort(orc.syev(H.dense(), vectors=False))
    want = np.sort([J * (L / 4 - 1) + J * math.cos(2 * math.pi * m / L) for m in range(L)])
    assert np.abs(got - want).max() < 1e-13


@pytest.mark.parametrize("L,nup", [(7, 3), (9, 4), (8, 3)])
def test_spin_flip_maps_sector_to_mirror_sector(orc, L, nup):
    """Flipping every spin maps the sector n_up with fields h_i to n_up' = L - n_up with -h_i."""
    hi = np.random.default_rng(L + nup).uniform(-2, 2, L)
    a = orc.syev(orc.csr(L, hi, 1.0, orc.basis(L, nup)).dense(), vectors=False)
    b = orc.syev(orc.csr(L, -hi, 1.0, orc.basis(L, L - nup)).dense(), vectors=False)
    assert np.abs(np.sort(a) - np.sort(b)).max() < 1e-12


def test_entanglement_odd_chain_hand_value(orc):
    """L = 3, one up spin, A = site 0, B = sites 1 and 2: (|up down down> + |down up down>)/sqrt2
    has two equal Schmidt weights, S^E = ln 2; a basis state has S^E = 0."""
    st = orc.basis(3, 1)  # [0b001, 0b010, 0b100]
    y = np.array([1.0, 1.0, 0.0]) / math.sqrt(2)
    assert abs(orc.entanglement(3, y, st) - math.log(2)) < 1e-14
    assert abs(orc.entanglement(3, np.array([0.0, 0.0, 1.0]), st)) < 1e-14
    # W state over all three sites: the cut leaves weights 1/3 (A up) and 2/3 (A down)
    w = np.ones(3) / math.sqrt(3)
    want = -(1 / 3) * math.log(1 / 3) - (2 / 3) * math.log(2 / 3)
    assert abs(orc.entanglement(3, w, st) - want) < 1e-14


@pytest.mark.parametrize("L,nup", [(5, 2), (5, 3), (7, 4), (7, 3), (6, 2), (9, 5)])
def test_entanglement_general_sector_vs_library_svd(orc, L, nup):
    idx = sector_indices(L, nup)
    st = orc.basis(L, nup)
    rng = np.random.default_rng(L * 10 + nup)
    for _ in range(3):
        y = rng.standard_normal(len(idx))
        full = np.zeros(2**L)
        full[idx] = y
        assert abs(orc.entanglement(L, y, st) - schmidt_entropy(L, full)) < 1e-12


@pytest.mark.parametrize("L,nup", [(5, 3), (7, 4)])
def test_fluct_odd_chain_closed_forms(orc, L, nup):
    """A basis state has a definite S^z_A (F = 0); the equal superposition of two states whose
    S^z_A differ by 1 has F = 1/4."""
    st = orc.basis(L, nup)
    e0 = np.zeros(len(st))
    e0[0] = 1.0
    assert abs(orc.fluct(L, e0, st)) < 1e-15
    LA = L // 2

    def mA(s):
        return bin(int(s) & ((1 << LA) - 1)).count("1") - LA / 2

    j = next(k for k in range(len(st)) if abs(mA(st[k]) - mA(st[0])) == 1)
    y = np.zeros(len(st))
    y[0] = y[j] = 1 / math.sqrt(2)
    assert abs(orc.fluct(L, y, st) - 0.25) < 1e-15


@pytest.mark.parametrize("L,nup", [(7, 4), (9, 5), (8, 3)])
def test_dynf_general_sector_limits(orc, L, nup):
    """f = 1 - |<M>|^2 / <M^+ M>, M = sum_j S^z_j e^{2 pi i j / L}: a basis state has a definite M
    (f = 0); the uniform vector of the sector is translation invariant, so <M> = 0 (f = 1)."""
    st = orc.basis(L, nup)
    for k in (0, len(st) // 2, len(st) - 1):
        e = np.zeros(len(st))
        e[k] = 1.0
        s = int(st[k])
        M = sum((0.5 if (s >> j) & 1 else -0.5) * np.exp(2j * math.pi * j / L) for j in range(L))
        if abs(M) > 1e-12:
            assert abs(orc.dynf(L, e, st)) < 1e-14
    u = np.ones(len(st)) / math.sqrt(len(st))
    assert abs(orc.dynf(L, u, st) - 1.0) < 1e-14
