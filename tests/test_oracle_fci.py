"""Pins of the determinant-space oracle (direct CI) against the Fock-space oracle."""
import numpy as np
import pytest

from oracle import fock, fci
from paper_1605_02611_gb300 import synth


@pytest.mark.parametrize("K", [2, 3])
def test_fci_equals_fock_all_sectors(K):
    h, eri = synth.integrals(K, 100 + K)
    H = fock.hamiltonian(h, eri)
    for Na in range(K + 1):
        for Nb in range(K + 1):
            idx, sgn = fci.jw_map(K, Na, Nb)
            Hs = H[idx][:, idx].toarray() * np.outer(sgn, sgn)
            Hf = fci.hamiltonian(h, eri, Na, Nb).toarray()
            assert np.abs(Hs - Hf).max() < 1e-12


def test_fci_equals_fock_k4_half_filling():
    K = 4
    h, eri = synth.integrals(K, 44)
    H = fock.hamiltonian(h, eri)
    idx, sgn = fci.jw_map(K, 2, 2)
    Hs = H[idx][:, idx].toarray() * np.outer(sgn, sgn)
    Hf = fci.hamiltonian(h, eri, 2, 2).toarray()
    assert np.abs(Hs - Hf).max() < 1e-12


def test_direct_ci_sigma_matches_matrix():
    K, Na, Nb = 5, 3, 2
    h, eri = synth.integrals(K, 9)
    Hf = fci.hamiltonian(h, eri, Na, Nb)
    c = np.random.default_rng(0).normal(size=(Hf.shape[0], 3))
    assert np.abs(fci.sigma(h, eri, Na, Nb, c) - Hf @ c).max() < 1e-12


def test_slater_condon_diagonal():
    K, Na, Nb = 5, 2, 3
    h, eri = synth.integrals(K, 12)
    Hf = fci.hamiltonian(h, eri, Na, Nb).toarray()
    sa, sb = fci.strings(K, Na), fci.strings(K, Nb)
    for ia in range(0, len(sa), 3):
        for ib in range(0, len(sb), 4):
            oa = [p for p in range(K) if (sa[ia] >> p) & 1]
            ob = [p for p in range(K) if (sb[ib] >> p) & 1]
            d = fci.slater_condon_diag(h, eri, oa, ob)
            assert abs(Hf[ia * len(sb) + ib, ia * len(sb) + ib] - d) < 1e-12


def test_integral_symmetries():
    """Synthetic (pq|rs) is 8-fold symmetric, so v_pqrs = <pq|sr> = v_qpsr (Eq. longrangeh)."""
    K = 4
    h, eri = synth.integrals(K, 1)
    assert np.allclose(h, h.T)
    assert np.allclose(eri, eri.transpose(1, 0, 2, 3))
    assert np.allclose(eri, eri.transpose(2, 3, 0, 1))
    assert np.allclose(eri, eri.transpose(0, 1, 3, 2))
    v = eri.transpose(0, 2, 3, 1)  # v_pqrs = (ps|qr)
    assert np.allclose(v, v.transpose(1, 0, 3, 2))
