"""Two-site DMRG sweep over the projected effective Hamiltonian (oracle).

Test infrastructure only.  Follows the three steps of a sweep step in Sec.
"The DMRG in renormalization group language": blocking (the two-site product
basis |l n_k n_k+1 r>), solving (lowest eigenpair of H_eff = P^T H P, see
``oracle.mps``), decimation (SVD of psi reshaped to (l n_k) x (n_k+1 r), keep
at most M singular vectors: the Schmidt form of Sec. "Matrix product states").

Readings where the paper is silent (shared, by statement only, with the
library):
* sweep schedule: one sweep = left-to-right over pairs (k, k+1), k = 0..K-3,
  each followed by a left-move truncation, then right-to-left over
  k = K-2..1, each followed by a right-move truncation; the sweep energy is
  the eigenvalue of its last step;
* truncation: singular values are grouped by the quantum number of the cut;
  weights lambda = s^2 below 1e-14 are dropped; the rest are sorted by
  (-lambda, sector order, index); if more than M remain, keep the first M
  except those within relative 1e-8 of the first dropped value (a
  degenerate multiplet is never split);
* the initial MPS (random, from the seeded generator) is first brought to
  right-canonical form by QR, from site K-1 down to site 2.
"""
from __future__ import annotations

import numpy as np
import scipy.sparse.linalg as spla

from . import mps as omps

TRUNC_WMIN = 1e-14
TRUNC_TIE = 1e-8


def _labels_from(dims_by_q):
    lab = []
    for q, d in dims_by_q:
        lab += [q] * d
    return np.array(lab, dtype=np.int64).reshape(-1, 2)


def right_canonicalize(tensors, labels):
    """QR from the right, per left sector; returns new tensors (labels unchanged)."""
    T = [t.copy() for t in tensors]
    K = len(T)
    for k in range(K - 1, 1, -1):
        A = T[k]
        Dl = A.shape[0]
        mat = A.reshape(Dl, -1)
        newA = np.zeros_like(mat)
        Rfull = np.zeros((Dl, Dl))
        lab = labels[k]
        for q in np.unique(lab, axis=0):
            rows = np.flatnonzero(np.all(lab == q, axis=1))
            sub = mat[rows]
            cols = np.flatnonzero(np.any(sub != 0, axis=0))
            # rows of sub must be orthonormalised: sub = R Q  (LQ via QR of transpose)
            Q, R = np.linalg.qr(sub[:, cols].T)
            newA[np.ix_(rows, cols)] = Q.T
            Rfull[np.ix_(rows, rows)] = R.T
        T[k] = newA.reshape(A.shape)
        T[k - 1] = np.einsum("lnr,rs->lns", T[k - 1], Rfull)
    return T


def truncation_select(lams, M):
    """lams: list of (lambda, group, index).  Returns the kept list (same order rule)."""
    cand = sorted([x for x in lams if x[0] >= TRUNC_WMIN], key=lambda x: (-x[0], x[1], x[2]))
    if len(cand) <= M:
        return cand
    t = cand[M][0]
    return [x for x in cand[:M] if x[0] > t * (1.0 + TRUNC_TIE)]


def decimate(psi, lab_l, lab_r, M, direction):
    """Split psi[l,n1,n2,r] into (left tensor, right tensor, new labels, discarded weight).

    direction 'left' (sweep moving right): left tensor is left-orthonormal U,
    right tensor is S V^T.  'right': left tensor is U S, right tensor is V^T.
    """
    Dl, _, _, Dr = psi.shape
    rows_q = (lab_l[:, None, :] + omps.LOCAL_QN[None, :, :]).reshape(-1, 2)   # (l,n1)
    cols_q = (lab_r[None, :, :] - omps.LOCAL_QN[:, None, :]).reshape(-1, 2)   # (n2,r)
    mat = psi.reshape(Dl * 4, 4 * Dr)
    groups = sorted({tuple(q) for q in rows_q} & {tuple(q) for q in cols_q})
    svd = {}
    lams = []
    for g, q in enumerate(groups):
        r = np.flatnonzero(np.all(rows_q == q, axis=1))
        c = np.flatnonzero(np.all(cols_q == q, axis=1))
        U, s, Vt = np.linalg.svd(mat[np.ix_(r, c)], full_matrices=False)
        svd[g] = (r, c, U, s, Vt)
        lams += [(s[i] ** 2, g, i) for i in range(len(s))]
    total = sum(x[0] for x in lams)
    kept = truncation_select(lams, M)
    kept_w = sum(x[0] for x in kept)
    by_g = {}
    for lam, g, i in kept:
        by_g.setdefault(g, []).append(i)
    new_dims = [(groups[g], len(sorted(by_g[g]))) for g in sorted(by_g)]
    Dn = sum(d for _, d in new_dims)
    left = np.zeros((Dl * 4, Dn))
    right = np.zeros((Dn, 4 * Dr))
    off = 0
    for g in sorted(by_g):
        idx = sorted(by_g[g])
        r, c, U, s, Vt = svd[g]
        n = len(idx)
        if direction == "left":
            left[r, off:off + n] = U[:, idx]
            right[off:off + n][:, c] = s[idx, None] * Vt[idx]
        else:
            left[r, off:off + n] = U[:, idx] * s[None, idx]
            right[off:off + n][:, c] = Vt[idx]
        off += n
    return (left.reshape(Dl, 4, Dn), right.reshape(Dn, 4, Dr), _labels_from(new_dims),
            float(total - kept_w))


def solve(tensors, k, psi0, mask, h, eri, Na, Nb, tol=1e-12):
    """Lowest eigenpair of H_eff on the allowed subspace (Lanczos, or dense if small)."""
    P = omps.TwoSiteProjector(tensors, k, Na, Nb)
    idx = np.flatnonzero(mask.reshape(-1))
    n = len(idx)
    shape = mask.shape

    def mv(x):
        full = np.zeros(mask.size)
        full[idx] = np.asarray(x).reshape(-1)
        return omps.sigma(tensors, k, full.reshape(shape), h, eri, Na, Nb, P).reshape(-1)[idx]

    if n <= 200:
        Hm = np.stack([mv(np.eye(n)[j]) for j in range(n)], axis=1)
        w, v = np.linalg.eigh(0.5 * (Hm + Hm.T))
        e, x = w[0], v[:, 0]
    else:
        op = spla.LinearOperator((n, n), matvec=mv, dtype=float)
        v0 = psi0.reshape(-1)[idx]
        if not np.any(v0):
            v0 = None
        w, v = spla.eigsh(op, k=1, which="SA", tol=tol, v0=v0, ncv=min(n, 40))
        e, x = w[0], v[:, 0]
    out = np.zeros(mask.size)
    out[idx] = x
    return float(e), out.reshape(shape)


def dmrg(h, eri, N, two_sz, tensors, labels, Ms, tol=1e-12):
    """Two-site DMRG.  labels[b] = per-index (na, nb) of bond b.  Returns
    (energies per sweep, max discarded weight per sweep, tensors, labels)."""
    Na, Nb = (N + two_sz) // 2, (N - two_sz) // 2
    K = len(tensors)
    T = right_canonicalize(tensors, labels)
    lab = [np.asarray(x, dtype=np.int64).reshape(-1, 2) for x in labels]
    energies, discarded = [], []
    for M in Ms:
        dmax = 0.0
        e = None
        # left to right
        for k in range(0, K - 2):
            psi = np.einsum("lnm,mor->lnor", T[k], T[k + 1])
            mask = omps.allowed_mask(lab[k], lab[k + 2])
            e, x = solve(T, k, psi, mask, h, eri, Na, Nb, tol)
            A, B, newlab, dw = decimate(x, lab[k], lab[k + 2], M, "left")
            T[k], lab[k + 1] = A, newlab
            T[k + 1] = B
            dmax = max(dmax, dw)
        # right to left
        for k in range(K - 2, 0, -1):
            psi = np.einsum("lnm,mor->lnor", T[k], T[k + 1])
            mask = omps.allowed_mask(lab[k], lab[k + 2])
            e, x = solve(T, k, psi, mask, h, eri, Na, Nb, tol)
            A, B, newlab, dw = decimate(x, lab[k], lab[k + 2], M, "right")
            T[k], T[k + 1], lab[k + 1] = A, B, newlab
            dmax = max(dmax, dw)
        energies.append(e)
        discarded.append(dmax)
    return energies, discarded, T, lab
