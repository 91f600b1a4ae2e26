"""Pins of the brute-force Fock-space oracle against closed forms (Eq. longrangeh)."""
import numpy as np
import pytest

from oracle import fock, fci
from paper_1605_02611_gb300 import synth


def test_anticommutation():
    K = 2
    cd, c = fock.operators(K)
    eye = np.eye(4 ** K)
    for x in range(2 * K):
        for y in range(2 * K):
            ac = (c[x] @ cd[y] + cd[y] @ c[x]).toarray()
            assert np.allclose(ac, eye * (x == y))
            cc = (cd[x] @ cd[y] + cd[y] @ cd[x]).toarray()
            assert np.allclose(cc, 0.0)


def test_noninteracting_spectrum():
    """eri = 0: the ground state fills the lowest orbitals of h in each spin."""
    K = 3
    h, _ = synth.integrals(K, 11)
    eri = np.zeros((K,) * 4)
    H = fock.hamiltonian(h, eri)
    eps = np.linalg.eigvalsh(h)
    for Na in range(K + 1):
        for Nb in range(K + 1):
            idx = fock.sector_indices(K, Na, Nb)
            w = np.linalg.eigvalsh(H[idx][:, idx].toarray())
            assert abs(w[0] - (eps[:Na].sum() + eps[:Nb].sum())) < 1e-12


def test_hubbard_atom():
    """One orbital: energies 0, e, e, 2e + U."""
    h = np.array([[-0.7]])
    eri = np.array([[[[1.3]]]])
    H = fock.hamiltonian(h, eri).toarray()
    assert np.allclose(np.sort(np.diag(H)), np.sort([0.0, -0.7, -0.7, -1.4 + 1.3]))
    assert np.allclose(H, np.diag(np.diag(H)))


@pytest.mark.parametrize("t,U", [(1.0, 4.0), (0.3, 1.7), (1.0, 0.0)])
def test_hubbard_dimer(t, U):
    """Two sites, two electrons, S_z = 0: E0 = (U - sqrt(U^2 + 16 t^2)) / 2."""
    h, eri = synth.hubbard_integrals(2, t, U)
    H = fock.hamiltonian(h, eri)
    idx = fock.sector_indices(2, 1, 1)
    w = np.linalg.eigvalsh(H[idx][:, idx].toarray())
    assert abs(w[0] - 0.5 * (U - np.sqrt(U * U + 16 * t * t))) < 1e-12
    Hc = fci.hamiltonian(h, eri, 1, 1).toarray()
    assert abs(np.linalg.eigvalsh(Hc)[0] - w[0]) < 1e-12


def test_closed_shell_determinant_energy():
    """<D|H|D> for doubly occupied orbitals 0..n-1: 2 sum h_ii + sum_ij [2(ii|jj) - (ij|ji)]."""
    K, n = 3, 2
    h, eri = synth.integrals(K, 5)
    H = fock.hamiltonian(h, eri)
    occ = [1] * (2 * n) + [0] * (2 * (K - n))
    j = fock.index_of(occ, K)
    ref = 2 * sum(h[i, i] for i in range(n))
    ref += sum(2 * eri[i, i, k, k] - eri[i, k, k, i] for i in range(n) for k in range(n))
    assert abs(H[j, j] - ref) < 1e-12


def test_conservation_and_hermiticity():
    K = 3
    h, eri = synth.integrals(K, 3)
    H = fock.hamiltonian(h, eri)
    na, nb = fock.number_ops(K)
    assert abs(H - H.T).max() < 1e-13
    assert abs(H @ na - na @ H).max() < 1e-12
    assert abs(H @ nb - nb @ H).max() < 1e-12
