"""Determinant-space (full CI) Hamiltonian of Eq. (longrangeh) (oracle).

Test infrastructure only.  Determinants of fixed (N_alpha, N_beta) are pairs of
occupation strings (bit masks over the K spatial orbitals, ascending integer
order); the determinant (I_a, I_b) is

    prod_{p in I_a, ascending} a+_{p alpha}  prod_{p in I_b, ascending} a+_{p beta} |vac>

and the CI vector is c[I_a, I_b].  H is written with the spin-summed
excitation operators E_pq = sum_s a+_{ps} a_{qs}:

    H = sum_pq k_pq E_pq + 1/2 sum_pqrs (pq|rs) E_pq E_rs,
    k_pq = h_pq - 1/2 sum_r (pr|rq),

which follows from Eq. (longrangeh) by one anticommutation
(E_pq E_rs = delta_qr E_ps + sum a+_{ps} a+_{rt} a_{st} a_{qs}).  Its action on
a vector is the string-driven direct-CI algorithm of Knowles & Handy
(Chem. Phys. Lett. 111, 315 (1984)): D_rs = E_rs c, G_pq = sum_rs (pq|rs) D_rs,
sigma = sum_pq k_pq D_pq + 1/2 sum_pq E_pq G_pq.
"""
from __future__ import annotations

import itertools
from functools import lru_cache

import numpy as np
import scipy.sparse as sp


@lru_cache(maxsize=None)
def strings(K: int, n: int) -> tuple:
    """All bit strings of K orbitals with n electrons, ascending."""
    out = []
    for occ in itertools.combinations(range(K), n):
        out.append(sum(1 << p for p in occ))
    return tuple(sorted(out))


def _popcount_below(mask: int, p: int) -> int:
    return bin(mask & ((1 << p) - 1)).count("1")


@lru_cache(maxsize=None)
def excitation_table(K: int, n: int) -> dict:
    """(p, q) -> (src, dst, sign): <dst| a+_p a_q |src> = sign for one spin."""
    strs = strings(K, n)
    pos = {s: i for i, s in enumerate(strs)}
    table = {}
    for p in range(K):
        for q in range(K):
            src, dst, sgn = [], [], []
            for i, s in enumerate(strs):
                if not (s >> q) & 1:
                    continue
                s1 = s & ~(1 << q)
                sign = -1 if _popcount_below(s, q) % 2 else 1
                if (s1 >> p) & 1:
                    continue
                sign *= -1 if _popcount_below(s1, p) % 2 else 1
                t = s1 | (1 << p)
                src.append(i)
                dst.append(pos[t])
                sgn.append(sign)
            table[(p, q)] = (np.array(src, dtype=np.int64), np.array(dst, dtype=np.int64),
                             np.array(sgn, dtype=float))
    return table


def _apply_E(c: np.ndarray, ta, tb, p: int, q: int) -> np.ndarray:
    """E_pq c for c of shape [n_a, n_b, ...]."""
    out = np.zeros_like(c)
    src, dst, sgn = ta[(p, q)]
    if len(src):
        out[dst] += sgn.reshape((-1,) + (1,) * (c.ndim - 1)) * c[src]
    src, dst, sgn = tb[(p, q)]
    if len(src):
        shape = (1, -1) + (1,) * (c.ndim - 2)
        out[:, dst] += sgn.reshape(shape) * c[:, src]
    return out


def sigma(h: np.ndarray, eri: np.ndarray, Na: int, Nb: int, c: np.ndarray) -> np.ndarray:
    """H c for a CI vector c (flat [n_a*n_b] or [n_a*n_b, nvec])."""
    K = h.shape[0]
    ta, tb = excitation_table(K, Na), excitation_table(K, Nb)
    na, nb = len(strings(K, Na)), len(strings(K, Nb))
    extra = c.shape[1:] if c.ndim > 1 else ()
    cc = c.reshape((na, nb) + extra)
    kk = h - 0.5 * np.einsum("prrq->pq", eri)
    D = np.stack([_apply_E(cc, ta, tb, r, s) for r in range(K) for s in range(K)])
    G = np.tensordot(eri.reshape(K * K, K * K), D, axes=(1, 0))
    out = np.tensordot(kk.reshape(-1), D, axes=(0, 0))
    for pq in range(K * K):
        p, q = divmod(pq, K)
        out += 0.5 * _apply_E(G[pq], ta, tb, p, q)
    return out.reshape(c.shape)


def E_matrix(K: int, Na: int, Nb: int, p: int, q: int) -> sp.csr_matrix:
    """E_pq as a sparse matrix on the determinant space."""
    ta, tb = excitation_table(K, Na), excitation_table(K, Nb)
    na, nb = len(strings(K, Na)), len(strings(K, Nb))
    rows, cols, vals = [], [], []
    src, dst, sgn = ta[(p, q)]
    for i, j, v in zip(src, dst, sgn):
        rows.append(j * nb + np.arange(nb))
        cols.append(i * nb + np.arange(nb))
        vals.append(np.full(nb, v))
    src, dst, sgn = tb[(p, q)]
    for i, j, v in zip(src, dst, sgn):
        rows.append(np.arange(na) * nb + j)
        cols.append(np.arange(na) * nb + i)
        vals.append(np.full(na, v))
    n = na * nb
    if not rows:
        return sp.csr_matrix((n, n))
    return sp.csr_matrix((np.concatenate(vals), (np.concatenate(rows), np.concatenate(cols))),
                         shape=(n, n))


def hamiltonian(h: np.ndarray, eri: np.ndarray, Na: int, Nb: int) -> sp.csr_matrix:
    """Explicit sparse H on the determinant space (same formula as ``sigma``)."""
    K = h.shape[0]
    kk = h - 0.5 * np.einsum("prrq->pq", eri)
    E = [[E_matrix(K, Na, Nb, p, q) for q in range(K)] for p in range(K)]
    n = E[0][0].shape[0]
    H = sp.csr_matrix((n, n))
    for p in range(K):
        for q in range(K):
            if kk[p, q] != 0.0:
                H = H + kk[p, q] * E[p][q]
            G = sp.csr_matrix((n, n))
            for r in range(K):
                for s in range(K):
                    if eri[p, q, r, s] != 0.0:
                        G = G + eri[p, q, r, s] * E[r][s]
            H = H + 0.5 * (E[p][q] @ G)
    return H.tocsr()


def slater_condon_diag(h: np.ndarray, eri: np.ndarray, occ_a, occ_b) -> float:
    """<D|H|D> = sum_i h_ii + 1/2 sum_ij [(ii|jj) - delta_{s_i s_j} (ij|ji)] (spin-orbitals)."""
    so = [(p, 0) for p in occ_a] + [(p, 1) for p in occ_b]
    e = sum(h[p, p] for p, _ in so)
    for (p, s) in so:
        for (q, t) in so:
            e += 0.5 * eri[p, p, q, q]
            if s == t:
                e -= 0.5 * eri[p, q, q, p]
    return float(e)


def jw_map(K: int, Na: int, Nb: int):
    """Determinant -> (Fock-space index, sign) for the Jordan-Wigner basis of
    ``oracle.fock`` (interleaved order 0a,0b,1a,1b,...).  The interleaved product
    equals sign times the alpha-first product, sign = (-1)^{#(i beta, j alpha), i<j}.
    """
    sa, sb = strings(K, Na), strings(K, Nb)
    idx = np.zeros(len(sa) * len(sb), dtype=np.int64)
    sgn = np.zeros(len(sa) * len(sb))
    for ia, a in enumerate(sa):
        for ib, b in enumerate(sb):
            j = 0
            swaps = 0
            for k in range(K):
                na_, nb_ = (a >> k) & 1, (b >> k) & 1
                j = j * 4 + na_ + 2 * nb_
                if na_:
                    swaps += _popcount_below(b, k)
            idx[ia * len(sb) + ib] = j
            sgn[ia * len(sb) + ib] = -1.0 if swaps % 2 else 1.0
    return idx, sgn


def ground_state(h: np.ndarray, eri: np.ndarray, Na: int, Nb: int, nroots: int = 1):
    """Lowest eigenvalues of the explicit determinant-space H (dense eigh)."""
    H = hamiltonian(h, eri, Na, Nb).toarray()
    w, v = np.linalg.eigh(H)
    return w[:nroots], v[:, :nroots]
