"""The seeded input generators shared by the oracle, the library tests and the bench
(host logic, CPU): integrals, bond sectors and random MPS / two-site tensors."""
import math

import numpy as np
import pytest

from paper_1605_02611_gb300 import synth


@pytest.mark.parametrize("K,std", [(6, 0.1), (10, 0.05)])
def test_integrals_recipe(K, std):
    h, eri = synth.integrals(K, 1605, offdiag_std=std)
    assert np.array_equal(h, h.T)
    assert np.array_equal(np.diag(h), -2.0 + 0.5 * np.arange(K))
    off = h[np.triu_indices(K, 1)]
    assert abs(off.std() - std) < 0.5 * std          # loose: a few dozen draws
    for perm in [(1, 0, 2, 3), (0, 1, 3, 2), (2, 3, 0, 1)]:
        assert np.allclose(eri, eri.transpose(perm), atol=1e-15)
    G = eri.reshape(K * K, K * K)
    w = np.linalg.eigvalsh(G)
    assert w.min() > -1e-12                         # sum of B (x) B: positive semidefinite
    assert int((w > 1e-10 * w.max()).sum()) <= 2 * K  # rank <= number of B^L
    h2, eri2 = synth.integrals(K, 1605, offdiag_std=std)
    assert np.array_equal(h, h2) and np.array_equal(eri, eri2)
    h3, _ = synth.integrals(K, 1606, offdiag_std=std)
    assert not np.array_equal(h, h3)


@pytest.mark.parametrize("K,Na,Nb,M", [(6, 3, 3, 10**6), (8, 4, 3, 10**6), (12, 6, 6, 64), (16, 8, 8, 200)])
def test_bond_sectors(K, Na, Nb, M):
    bonds = synth.bond_sectors(K, Na, Nb, M)
    assert len(bonds) == K + 1
    assert bonds[0].qn == [(0, 0)] and bonds[0].dim == [1]
    assert bonds[K].qn == [(Na, Nb)] and bonds[K].dim == [1]
    for b, bs in enumerate(bonds):
        assert bs.total <= M
        assert bs.qn == sorted(bs.qn) and all(d > 0 for d in bs.dim)
        d = dict(zip(bs.qn, bs.dim))
        for (na, nb), dim in d.items():
            # never more than the Fock space on either side can hold
            fl = math.comb(b, na) * math.comb(b, nb)
            fr = math.comb(K - b, Na - na) * math.comb(K - b, Nb - nb)
            assert dim <= min(fl, fr)
            if b > 0:   # reachable from the previous bond through one site
                prev = dict(zip(bonds[b - 1].qn, bonds[b - 1].dim))
                assert dim <= sum(prev.get((na - a, nb - c), 0) for a, c in synth.LOCAL_QN)
        lab = bs.labels()
        assert lab.shape == (bs.total, 2)
    if M >= 10**6:  # no truncation: the exact Schmidt ranks min(left, right Fock dim)
        for b, bs in enumerate(bonds):
            for (na, nb), dim in zip(bs.qn, bs.dim):
                fl = math.comb(b, na) * math.comb(b, nb)
                fr = math.comb(K - b, Na - na) * math.comb(K - b, Nb - nb)
                assert dim == min(fl, fr)


def test_largest_remainder_respects_caps_and_total():
    w = np.array([5.0, 1.0, 1.0, 0.5])
    dims = synth._largest_remainder(w, [3, 10, 10, 10], 12)
    assert sum(dims) == 12 and dims[0] == 3
    assert synth._largest_remainder(w, [1, 1, 1, 1], 12) == [1, 1, 1, 1]


def _block_mask(ll, rl):
    m = np.zeros((len(ll), 4, len(rl)), dtype=bool)
    for n, (a, c) in enumerate(synth.LOCAL_QN):
        m[:, n, :] = (ll[:, None, 0] + a == rl[None, :, 0]) & (ll[:, None, 1] + c == rl[None, :, 1])
    return m


def test_random_mps_block_structure():
    K, N = 6, 6
    bonds, T = synth.random_mps(K, N, 0, 16, 3)
    for k, A in enumerate(T):
        assert A.shape == (bonds[k].total, 4, bonds[k + 1].total)
        m = _block_mask(bonds[k].labels(), bonds[k + 1].labels())
        assert np.all(A[~m] == 0.0) and np.any(A[m] != 0.0)


def test_random_isometric_mps_gauge():
    K, N, M, c = 8, 8, 24, 3
    bonds, T = synth.random_isometric_mps(K, N, 0, M, 11, c)
    for k, A in enumerate(T):
        m = _block_mask(bonds[k].labels(), bonds[k + 1].labels())
        assert np.all(A[~m] == 0.0)
        Dl, _, Dr = A.shape
        if k < c:      # left isometry: sum_{l,n} A[l,n,r] A[l,n,r'] = delta
            X = A.reshape(Dl * 4, Dr)
            assert np.allclose(X.T @ X, np.eye(Dr), atol=1e-12)
        elif k > c + 1:  # right isometry: sum_{n,r} A[l,n,r] A[l',n,r] = delta
            X = A.reshape(Dl, 4 * Dr)
            assert np.allclose(X @ X.T, np.eye(Dl), atol=1e-12)
        else:
            assert abs(np.linalg.norm(A) - 1.0) < 1e-12


def test_random_psi_structure_and_norm():
    bonds = synth.bond_sectors(8, 4, 4, 20)
    psi = synth.random_psi(bonds[3], bonds[5], 2)
    ll, rl = bonds[3].labels(), bonds[5].labels()
    for n1, (a1, c1) in enumerate(synth.LOCAL_QN):
        for n2, (a2, c2) in enumerate(synth.LOCAL_QN):
            ok = (ll[:, None, 0] + a1 + a2 == rl[None, :, 0]) & (ll[:, None, 1] + c1 + c2 == rl[None, :, 1])
            assert np.all(psi[:, n1, n2, :][~ok] == 0.0)
    assert abs(np.linalg.norm(psi) - 1.0) < 1e-12
