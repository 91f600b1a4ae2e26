"""Pins of the projected-H_eff two-site DMRG oracle."""
import numpy as np
import pytest

from oracle import dmrg, fci, mps
from paper_1605_02611_gb300 import synth


def _fci_e0(h, eri, Na, Nb):
    import scipy.sparse.linalg as spla
    H = fci.hamiltonian(h, eri, Na, Nb)
    if H.shape[0] < 300:
        return np.linalg.eigvalsh(H.toarray())[0]
    return spla.eigsh(H, k=1, which="SA", tol=1e-14)[0][0]


@pytest.mark.parametrize("K,N,two_sz", [(4, 4, 0), (5, 4, 2), (6, 6, 0)])
def test_full_m_equals_fci(K, N, two_sz):
    """M >= 4^(K/2): the MPS is exact (Schmidt form), so DMRG = FCI."""
    h, eri = synth.integrals(K, 20 + K)
    bonds, T = synth.random_mps(K, N, two_sz, 4 ** (K // 2), 3)
    E, D, T2, lab = dmrg.dmrg(h, eri, N, two_sz, T, [b.labels() for b in bonds], [4 ** (K // 2)] * 2)
    e0 = _fci_e0(h, eri, (N + two_sz) // 2, (N - two_sz) // 2)
    assert abs(E[-1] - e0) < 1e-10


@pytest.mark.slow
def test_k8_m256_equals_fci():
    cfg = synth.WORKLOADS["k8_m256_fp64"]
    h, eri = synth.integrals(8, cfg["seed"], cfg["offdiag_std"])
    bonds, T = synth.random_mps(8, 8, 0, 256, cfg["seed"])
    E, D, _, _ = dmrg.dmrg(h, eri, 8, 0, T, [b.labels() for b in bonds], [256, 256])
    assert abs(E[-1] - _fci_e0(h, eri, 4, 4)) < 1e-10


def test_truncated_is_variational_and_gauge():
    K, N = 6, 6
    h, eri = synth.integrals(K, 77)
    bonds, T = synth.random_mps(K, N, 0, 12, 5)
    E, D, T2, lab = dmrg.dmrg(h, eri, N, 0, T, [b.labels() for b in bonds], [12, 12, 12])
    e0 = _fci_e0(h, eri, 3, 3)
    for e in E:
        assert e >= e0 - 1e-10
    assert E[2] <= E[0] + 1e-9
    assert max(len(x) for x in lab) <= 12
    # after the final right-to-left pass, sites 2..K-1 are right-orthonormal
    for k in range(2, K):
        A = T2[k].reshape(T2[k].shape[0], -1)
        assert np.allclose(A @ A.T, np.eye(A.shape[0]), atol=1e-12)


def test_projected_heff_hermitian_and_conserving():
    K, N = 5, 5
    h, eri = synth.integrals(K, 4)
    bonds, T = synth.random_mps(K, N, 1, 9, 8)
    Na, Nb = 3, 2
    k = 1
    lab = [b.labels() for b in bonds]
    mask = mps.allowed_mask(lab[k], lab[k + 2])
    rng = np.random.default_rng(1)
    x = rng.normal(size=mask.shape) * mask
    y = rng.normal(size=mask.shape) * mask
    sx = mps.sigma(T, k, x, h, eri, Na, Nb)
    sy = mps.sigma(T, k, y, h, eri, Na, Nb)
    assert abs(np.vdot(x, sy) - np.vdot(sx, y)) < 1e-12 * (1 + abs(np.vdot(x, sy)))
    assert np.abs(sx[~mask]).max() < 1e-14


def test_truncation_rule_keeps_multiplets():
    lams = [(0.5, 0, 0), (0.2, 1, 0), (0.2, 2, 0), (0.1, 0, 1), (1e-20, 1, 1)]
    assert [x[:2] for x in dmrg.truncation_select(lams, 2)] == [(0.5, 0)]
    assert len(dmrg.truncation_select(lams, 3)) == 3
    assert len(dmrg.truncation_select(lams, 10)) == 4


@pytest.mark.parametrize("K,N,two_sz,M", [(5, 5, 1, 9), (6, 6, 0, 12), (6, 4, 2, 7)])
def test_right_canonicalize_keeps_state_and_gauge(K, N, two_sz, M):
    """Bringing the start MPS to right-canonical form is a change of gauge only:
    the contracted state is unchanged, every site k >= 2 becomes
    right-orthonormal (sum over n, r of A^n[l, r] A^n[l', r] = delta_ll'), and
    the quantum-number block structure of every tensor survives."""
    bonds, T = synth.random_mps(K, N, two_sz, M, 40 + K)
    lab = [b.labels() for b in bonds]
    T2 = dmrg.right_canonicalize(T, lab)
    before, after = mps.full_state(T), mps.full_state(T2)
    assert np.abs(after - before).max() < 1e-12 * np.abs(before).max()
    for k in range(2, K):
        A = T2[k].reshape(T2[k].shape[0], -1)
        assert np.allclose(A @ A.T, np.eye(A.shape[0]), atol=1e-12)
    for k in range(K):
        # entries outside the allowed (q_l + q(n) = q_r) pattern stay exactly zero
        q = lab[k][:, None, None, :] + mps.LOCAL_QN[None, :, None, :]
        allowed = np.all(q == lab[k + 1][None, None, :, :], axis=-1)
        assert np.all(T2[k][~allowed] == 0.0)
