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


def _slater_condon(h, eri, d1, d2):
    """<d2|H|d1> by the Slater-Condon rules (Szabo & Ostlund, Tables 2.3-2.4),
    for determinants given as ascending lists of spin-orbital keys s*K + p
    (alpha block first, the creation order of the determinant basis)."""
    K = h.shape[0]

    def one(x, y):
        return h[x % K, y % K] if x // K == y // K else 0.0

    def anti(x, y, z, w):  # <xy||zw>, <xy|zw> = (x z|y w) with matching spins
        g = eri[x % K, z % K, y % K, w % K] if (x // K == z // K and y // K == w // K) else 0.0
        if x // K == w // K and y // K == z // K:
            g -= eri[x % K, w % K, y % K, z % K]
        return g

    gone = [x for x in d1 if x not in d2]   # occupied in d1 only
    new = [x for x in d2 if x not in d1]    # occupied in d2 only
    if len(gone) > 2:
        return 0.0
    if not gone:
        return (sum(one(i, i) for i in d1)
                + 0.5 * sum(anti(i, j, i, j) for i in d1 for j in d1))
    # d1 with the removed orbitals replaced in place by the added ones, then the
    # parity of the sort that brings it to d2's ascending order
    lst = list(d1)
    for m, p in zip(gone, new):
        lst[lst.index(m)] = p
    inv = sum(1 for a in range(len(lst)) for b in range(a + 1, len(lst)) if lst[a] > lst[b])
    sign = -1.0 if inv % 2 else 1.0
    if len(gone) == 1:
        (m,), (p,) = gone, new
        return sign * (one(p, m) + sum(anti(p, n, m, n) for n in d1))
    (m, n), (p, q) = gone, new
    return sign * anti(p, q, m, n)


def test_slater_condon_off_diagonal_k8():
    """Every element of sampled columns of the K=8, N=8 direct-CI Hamiltonian
    (4900 determinants) equals the Slater-Condon value: diagonal, single and
    double excitations with their phases, and zero beyond doubles."""
    K, Na, Nb = 8, 4, 4
    h, eri = synth.integrals(K, 1605)
    sa, sb = fci.strings(K, Na), fci.strings(K, Nb)
    n = len(sa) * len(sb)

    def det(i):
        ia, ib = divmod(i, len(sb))
        return ([p for p in range(K) if (sa[ia] >> p) & 1]
                + [K + p for p in range(K) if (sb[ib] >> p) & 1])

    cols = np.random.default_rng(8).choice(n, size=6, replace=False)
    c = np.zeros((n, len(cols)))
    c[cols, np.arange(len(cols))] = 1.0
    Hc = fci.sigma(h, eri, Na, Nb, c)
    dets = [det(i) for i in range(n)]
    counts = [0, 0, 0]
    for j, col in enumerate(cols):
        d1 = dets[col]
        for i in range(n):
            ref = _slater_condon(h, eri, d1, dets[i])
            assert abs(Hc[i, j] - ref) < 1e-12, (col, i, Hc[i, j], ref)
            nexc = len(set(dets[i]) - set(d1))
            if 0 < nexc <= 2 and ref != 0.0:
                counts[nexc] += 1
    assert counts[1] > 0 and counts[2] > 0   # both rules were exercised
