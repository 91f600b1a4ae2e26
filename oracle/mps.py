"""Renormalised bases and the projected two-site effective Hamiltonian (oracle).

Test infrastructure only.  An MPS is a list of dense tensors A[k] of shape
[D_k, 4, D_{k+1}] (Eq. FSMPS, one spatial orbital per site, local index
n = n_alpha + 2 n_beta) together with per-bond sector labels (n_alpha, n_beta)
of the block left of the bond.  Nothing here assumes canonical form.

* left_basis(k):  columns are |l_alpha> of Eq. (lbasis) for the block of
  sites 0..k-1, as vectors of the Jordan-Wigner Fock basis of ``oracle.fock``;
* right_basis(k): rows are |r_alpha> of Eq. (rbasis) for sites k..K-1;
* the two-site product basis |l n_k n_k+1 r> (Eq. MPSCform with two explicit
  sites) maps a wavefunction psi[l, n1, n2, r] to the Fock vector P psi, and
  the effective Hamiltonian is H_eff = P^T H P.  ``sigma`` returns P^T H P psi
  with H applied in the determinant space by ``oracle.fci.sigma``.
"""
from __future__ import annotations

import numpy as np

from . import fci

LOCAL_QN = np.array([(0, 0), (1, 0), (0, 1), (1, 1)], dtype=np.int64)


def left_basis(tensors, k: int) -> np.ndarray:
    """U[(n_0..n_{k-1}), alpha] for bond k (k sites on the left)."""
    U = np.ones((1, 1))
    for j in range(k):
        A = tensors[j]
        U = np.einsum("al,lnr->anr", U, A).reshape(-1, A.shape[2])
    return U


def right_basis(tensors, k: int) -> np.ndarray:
    """V[alpha, (n_k..n_{K-1})] for bond k (sites k..K-1 on the right)."""
    V = np.ones((1, 1))
    for j in range(len(tensors) - 1, k - 1, -1):
        A = tensors[j]
        V = np.einsum("lnr,rb->lnb", A, V).reshape(A.shape[0], -1)
    return V


def full_state(tensors) -> np.ndarray:
    """Psi^{n_1..n_K} as a flat Fock vector."""
    return left_basis(tensors, len(tensors)).reshape(-1)


class TwoSiteProjector:
    """The map psi[l,n1,n2,r] -> Fock vector for the sites (k, k+1)."""

    def __init__(self, tensors, k: int, Na: int, Nb: int):
        K = len(tensors)
        self.K, self.k, self.Na, self.Nb = K, k, Na, Nb
        self.U = left_basis(tensors, k)
        self.V = right_basis(tensors, k + 2)
        self.jw_idx, self.jw_sgn = fci.jw_map(K, Na, Nb)

    @property
    def shape(self):
        return (self.U.shape[1], 4, 4, self.V.shape[0])

    def project(self, psi: np.ndarray) -> np.ndarray:
        """Fock vector -> determinant vector (sector restriction with JW signs)."""
        v = np.einsum("al,lijr,rb->aijb", self.U, psi, self.V, optimize=True).reshape(-1)
        return v[self.jw_idx] * self.jw_sgn

    def unproject(self, c: np.ndarray) -> np.ndarray:
        v = np.zeros(4 ** self.K)
        v[self.jw_idx] = c * self.jw_sgn
        v = v.reshape(self.U.shape[0], 4, 4, self.V.shape[1])
        return np.einsum("al,aijb,rb->lijr", self.U, v, self.V, optimize=True)


def sigma(tensors, k: int, psi: np.ndarray, h, eri, Na: int, Nb: int,
          proj: TwoSiteProjector | None = None) -> np.ndarray:
    """sigma = P^T H P psi for the two-site product basis at sites (k, k+1)."""
    P = proj if proj is not None else TwoSiteProjector(tensors, k, Na, Nb)
    c = P.project(psi)
    return P.unproject(fci.sigma(h, eri, Na, Nb, c))


def allowed_mask(lab_l: np.ndarray, lab_r: np.ndarray) -> np.ndarray:
    """Boolean [D_l,4,4,D_r]: q_l + q(n1) + q(n2) == q_r (both components)."""
    q = (lab_l[:, None, None, None, :] + LOCAL_QN[None, :, None, None, :]
         + LOCAL_QN[None, None, :, None, :])
    return np.all(q == lab_r[None, None, None, :, :], axis=-1)


def heff_dense(tensors, k: int, h, eri, Na: int, Nb: int, mask: np.ndarray) -> np.ndarray:
    """Explicit H_eff restricted to the allowed entries (columns in mask order)."""
    P = TwoSiteProjector(tensors, k, Na, Nb)
    idx = np.flatnonzero(mask.reshape(-1))
    n = len(idx)
    cols = []
    for j in range(n):
        e = np.zeros(mask.size)
        e[idx[j]] = 1.0
        cols.append(P.project(e.reshape(mask.shape)))
    Pm = np.stack(cols, axis=1)  # [ndet, n]
    HP = fci.sigma(h, eri, Na, Nb, Pm)
    return Pm.T @ HP
