"""Brute-force Fock-space Hamiltonian from Jordan-Wigner matrices (oracle).

Test infrastructure only.  Eq. (longrangeh) with spin made explicit: spatial
orbitals p = 0..K-1, spin-orbital x = 2p + s (s = 0 alpha, 1 beta), ordering
0a, 0b, 1a, 1b, ...  A basis state is the occupation pattern of all 2K
spin-orbitals; its index is sum_k n_k 4^(K-1-k) with n_k = n_ka + 2 n_kb, which
is the row-major order of an MPS amplitude Psi^{n_1 ... n_K} (Eq. FSMPS).  The
state with pattern n is prod_{x ascending} (a_x^dag)^{n_x} |vac>.

    H = sum_{pq,s} h_pq a+_{ps} a_{qs}
      + 1/2 sum_{pqrs,s,t} (pq|rs) a+_{ps} a+_{rt} a_{st} a_{qs}

which is Eq. (longrangeh) with v_{pqrs} = <pq|sr> = (ps|qr) for spin-orbitals.
"""
from __future__ import annotations

import numpy as np
import scipy.sparse as sp


def occupation(index: int, K: int) -> list:
    """Occupation bits of spin-orbitals 0..2K-1 for a basis index."""
    occ = []
    for k in range(K):
        n = (index >> (2 * (K - 1 - k))) & 3
        occ += [n & 1, (n >> 1) & 1]
    return occ


def index_of(occ, K: int) -> int:
    idx = 0
    for k in range(K):
        n = occ[2 * k] + 2 * occ[2 * k + 1]
        idx = idx * 4 + n
    return idx


def creation(K: int, x: int) -> sp.csr_matrix:
    """a_x^dagger as a sparse 4^K x 4^K matrix (Jordan-Wigner sign over y < x)."""
    dim = 4 ** K
    rows, cols, vals = [], [], []
    for j in range(dim):
        occ = occupation(j, K)
        if occ[x]:
            continue
        sign = -1.0 if sum(occ[:x]) % 2 else 1.0
        occ2 = list(occ)
        occ2[x] = 1
        rows.append(index_of(occ2, K))
        cols.append(j)
        vals.append(sign)
    return sp.csr_matrix((vals, (rows, cols)), shape=(dim, dim))


def operators(K: int):
    """Lists (cdag[x], c[x]) for all 2K spin-orbitals."""
    cd = [creation(K, x) for x in range(2 * K)]
    return cd, [m.T.tocsr() for m in cd]


def hamiltonian(h: np.ndarray, eri: np.ndarray, ops=None) -> sp.csr_matrix:
    """Full Fock-space H (sparse), written term by term from Eq. (longrangeh)."""
    K = h.shape[0]
    cd, c = ops if ops is not None else operators(K)
    dim = 4 ** K
    H = sp.csr_matrix((dim, dim))
    for p in range(K):
        for q in range(K):
            if h[p, q] == 0.0:
                continue
            for s in range(2):
                H = H + h[p, q] * (cd[2 * p + s] @ c[2 * q + s])
    for p in range(K):
        for q in range(K):
            for r in range(K):
                for s_ in range(K):
                    g = eri[p, q, r, s_]
                    if g == 0.0:
                        continue
                    for s in range(2):
                        for t in range(2):
                            term = (cd[2 * p + s] @ cd[2 * r + t]) @ (c[2 * s_ + t] @ c[2 * q + s])
                            H = H + 0.5 * g * term
    return H.tocsr()


def number_ops(K: int, ops=None):
    """(N_alpha, N_beta) operators as sparse matrices."""
    cd, c = ops if ops is not None else operators(K)
    na = sum(cd[2 * p] @ c[2 * p] for p in range(K))
    nb = sum(cd[2 * p + 1] @ c[2 * p + 1] for p in range(K))
    return na.tocsr(), nb.tocsr()


def sector_indices(K: int, Na: int, Nb: int) -> np.ndarray:
    """Basis indices of the (N_alpha, N_beta) sector, ascending."""
    out = []
    for j in range(4 ** K):
        occ = occupation(j, K)
        if sum(occ[0::2]) == Na and sum(occ[1::2]) == Nb:
            out.append(j)
    return np.array(out, dtype=np.int64)
