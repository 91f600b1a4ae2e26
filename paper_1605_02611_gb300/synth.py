"""Seeded synthetic inputs shared by the CUDA path, the CPU oracle and the bench.

This module draws random numbers and lays out structure only; it holds none of
the DMRG arithmetic (no operator algebra, no contractions of the method).  The
one matrix factorisation here is the QR of Gaussian matrices used to draw
random isometries (random orthonormal bases), a standard way to sample them.

Workload recipe (the paper's own test system, H20/STO-3G, Sec. "Hamiltonian
compression", is not available here, so these stand in for it):

* one-electron integrals h_pq: symmetric, diagonal -2 + 0.5 p (p = 0..K-1),
  off-diagonal N(0, std^2) drawn on the upper triangle and mirrored;
* two-electron integrals in chemists' order (pq|rs) = sum_{L<2K} B^L_pq B^L_rs
  with every B^L symmetric, entries N(0, b_std^2) (upper triangle incl. the
  diagonal, mirrored), which makes (pq|rs) 8-fold symmetric and positive
  semidefinite as a (pq),(rs) matrix, like a real Coulomb kernel;
* random MPS tensors with U(1)xU(1) block structure.  Bond sectors are labelled
  by the particle counts (n_alpha, n_beta) of the block left of the bond; the
  local basis of a spatial-orbital site is n = n_alpha + 2 n_beta, i.e.
  |0>, |up>, |dn>, |up dn>.
"""
from __future__ import annotations

import math
from dataclasses import dataclass

import numpy as np


def _sym_normal(rng: np.random.Generator, K: int, std: float) -> np.ndarray:
    a = rng.normal(0.0, std, size=(K, K))
    u = np.triu(a)
    return u + np.triu(u, 1).T


def integrals(K: int, seed: int, offdiag_std: float = 0.1, b_std: float = 0.1):
    """Return (h, eri): h[K,K] and eri[K,K,K,K] = (pq|rs), float64, C order."""
    rng = np.random.default_rng(seed)
    h = _sym_normal(rng, K, offdiag_std)
    h[np.arange(K), np.arange(K)] = -2.0 + 0.5 * np.arange(K)
    B = np.stack([_sym_normal(rng, K, b_std) for _ in range(2 * K)])
    eri = np.einsum("lpq,lrs->pqrs", B, B, optimize=True)
    return np.ascontiguousarray(h), np.ascontiguousarray(eri)


# --- bond sectors -----------------------------------------------------------

LOCAL_QN = [(0, 0), (1, 0), (0, 1), (1, 1)]  # n = n_alpha + 2 n_beta


@dataclass
class BondSectors:
    """Sorted list of sectors (na, nb) with their dimensions."""
    qn: list          # list[(na, nb)]
    dim: list         # list[int]

    @property
    def total(self) -> int:
        return int(sum(self.dim))

    def labels(self) -> np.ndarray:
        """Per-index (na, nb) labels, shape [total, 2], int32."""
        out = np.zeros((self.total, 2), dtype=np.int32)
        i = 0
        for (na, nb), d in zip(self.qn, self.dim):
            out[i:i + d] = (na, nb)
            i += d
        return out


def _reachable(b: int, K: int, Na: int, Nb: int):
    out = []
    for na in range(0, min(b, Na) + 1):
        if Na - na > K - b:
            continue
        for nb in range(0, min(b, Nb) + 1):
            if Nb - nb > K - b:
                continue
            out.append((na, nb))
    return out


def bond_sectors(K: int, Na: int, Nb: int, M: int, spread: float = 0.5):
    """Sector dimensions for every bond 0..K of an MPS with bond dimension <= M.

    Target weight of a sector is (left Fock dim * right Fock dim)^spread; M is
    shared out by largest remainder, then every dimension is capped so that it
    never exceeds what the neighbouring bond and one site can supply (so the
    tensors can be full rank).
    """
    bonds = []
    for b in range(K + 1):
        secs = _reachable(b, K, Na, Nb)
        fl = [math.comb(b, na) * math.comb(b, nb) for na, nb in secs]
        fr = [math.comb(K - b, Na - na) * math.comb(K - b, Nb - nb) for na, nb in secs]
        cap = [min(x, y) for x, y in zip(fl, fr)]
        w = np.array([(x * y) ** spread for x, y in zip(fl, fr)], dtype=float)
        if sum(cap) <= M:
            dims = list(cap)
        else:
            dims = _largest_remainder(w, cap, M)
        bonds.append(dict(zip(secs, dims)))
    # enforce neighbour consistency both ways until stable
    for _ in range(4 * K + 4):
        changed = False
        for b in range(K):
            for q, d in list(bonds[b + 1].items()):
                inc = sum(bonds[b].get((q[0] - a, q[1] - c), 0) for a, c in LOCAL_QN)
                if d > inc:
                    bonds[b + 1][q] = inc
                    changed = True
        for b in range(K, 0, -1):
            for q, d in list(bonds[b - 1].items()):
                out = sum(bonds[b].get((q[0] + a, q[1] + c), 0) for a, c in LOCAL_QN)
                if d > out:
                    bonds[b - 1][q] = out
                    changed = True
        if not changed:
            break
    res = []
    for b in range(K + 1):
        items = sorted((q, d) for q, d in bonds[b].items() if d > 0)
        res.append(BondSectors([q for q, _ in items], [d for _, d in items]))
    return res


def _largest_remainder(w: np.ndarray, cap, M: int):
    cap = np.array(cap, dtype=np.int64)
    dims = np.zeros_like(cap)
    free = np.ones(len(cap), dtype=bool)
    left = M
    # water-filling with caps
    while left > 0 and free.any():
        share = w * free
        if share.sum() <= 0:
            break
        ideal = left * share / share.sum()
        add = np.minimum(np.floor(ideal).astype(np.int64), cap - dims)
        if add.sum() == 0:
            order = np.argsort(-(ideal - np.floor(ideal)) - 1e-9 * np.arange(len(w)))
            for i in order:
                if left == 0:
                    break
                if free[i] and dims[i] < cap[i]:
                    dims[i] += 1
                    left -= 1
            break
        dims += add
        left -= int(add.sum())
        free = dims < cap
    return [int(x) for x in dims]


def random_mps(K: int, N: int, two_sz: int, M: int, seed: int, spread: float = 0.5):
    """Random QN-block MPS: returns (bonds, tensors).

    tensors[k] is a dense float64 array [D_k, 4, D_{k+1}] that is zero outside
    the allowed blocks (right label = left label + local label).  Entries are
    N(0, 1/(4 D_k)) so that norms stay O(1) along the chain.  The tensors are
    NOT canonical.
    """
    Na, Nb = (N + two_sz) // 2, (N - two_sz) // 2
    bonds = bond_sectors(K, Na, Nb, M, spread)
    rng = np.random.default_rng(seed)
    tensors = []
    for k in range(K):
        L, R = bonds[k], bonds[k + 1]
        ll, rl = L.labels(), R.labels()
        A = rng.normal(0.0, 1.0 / math.sqrt(4 * L.total), size=(L.total, 4, R.total))
        for n, (a, c) in enumerate(LOCAL_QN):
            mask = (ll[:, None, 0] + a == rl[None, :, 0]) & (ll[:, None, 1] + c == rl[None, :, 1])
            A[:, n, :] *= mask
        tensors.append(np.ascontiguousarray(A))
    return bonds, tensors


def random_isometric_mps(K: int, N: int, two_sz: int, M: int, seed: int, center: int, spread: float = 0.5):
    """Random QN-block MPS in mixed-canonical form around sites (center, center+1).

    Sites left of `center` are random left isometries (for every right sector
    the stacked (l, n) x r block has orthonormal columns), sites right of
    center+1 random right isometries (orthonormal rows per left sector): the
    Q factors of Gaussian random matrices.  The two centre tensors are
    Gaussian.  Returns (bonds, tensors) like random_mps.
    """
    Na, Nb = (N + two_sz) // 2, (N - two_sz) // 2
    bonds = bond_sectors(K, Na, Nb, M, spread)
    rng = np.random.default_rng(seed)
    tensors = []
    for k in range(K):
        L, R = bonds[k], bonds[k + 1]
        ll, rl = L.labels(), R.labels()
        A = np.zeros((L.total, 4, R.total))
        if k < center:
            # rows (l, n) grouped by right sector
            for (qa, qb), d, off in zip(R.qn, R.dim, np.cumsum([0] + R.dim[:-1])):
                rows = [(l, n) for n, (a, c) in enumerate(LOCAL_QN)
                        for l in range(L.total) if ll[l, 0] + a == qa and ll[l, 1] + c == qb]
                Q, _ = np.linalg.qr(rng.normal(size=(len(rows), d)))
                for i, (l, n) in enumerate(rows):
                    A[l, n, off:off + d] = Q[i]
        elif k > center + 1:
            for (qa, qb), d, off in zip(L.qn, L.dim, np.cumsum([0] + L.dim[:-1])):
                cols = [(n, r) for n, (a, c) in enumerate(LOCAL_QN)
                        for r in range(R.total) if qa + a == rl[r, 0] and qb + c == rl[r, 1]]
                Q, _ = np.linalg.qr(rng.normal(size=(len(cols), d)))
                for i, (n, r) in enumerate(cols):
                    A[off:off + d, n, r] = Q[i]
        else:
            A = rng.normal(size=(L.total, 4, R.total))
            for n, (a, c) in enumerate(LOCAL_QN):
                mask = (ll[:, None, 0] + a == rl[None, :, 0]) & (ll[:, None, 1] + c == rl[None, :, 1])
                A[:, n, :] *= mask
            A /= np.linalg.norm(A)
        tensors.append(np.ascontiguousarray(A))
    return bonds, tensors


def random_psi(bl: BondSectors, br: BondSectors, seed: int) -> np.ndarray:
    """Random two-site wavefunction [D_l, 4, 4, D_r] with the block structure of the
    total quantum number fixed by the bond labels (ql + q(n1) + q(n2) = qr)."""
    rng = np.random.default_rng(seed)
    ll, rl = bl.labels(), br.labels()
    psi = rng.normal(0.0, 1.0, size=(bl.total, 4, 4, br.total))
    for n1, (a1, c1) in enumerate(LOCAL_QN):
        for n2, (a2, c2) in enumerate(LOCAL_QN):
            mask = ((ll[:, None, 0] + a1 + a2 == rl[None, :, 0])
                    & (ll[:, None, 1] + c1 + c2 == rl[None, :, 1]))
            psi[:, n1, n2, :] *= mask
    nrm = np.linalg.norm(psi)
    return psi / nrm if nrm > 0 else psi


def hubbard_integrals(K: int, t: float, U: float):
    """Open-chain Hubbard model as integrals: h = -t on neighbours, (pp|pp) = U."""
    h = np.zeros((K, K))
    for p in range(K - 1):
        h[p, p + 1] = h[p + 1, p] = -t
    eri = np.zeros((K, K, K, K))
    for p in range(K):
        eri[p, p, p, p] = U
    return h, eri


# configurations of the workloads (sizes, seeds), named by what they are
BASE_SEED = 1605

WORKLOADS = {
    "k8_m256_fp64": dict(K=8, N=8, two_sz=0, M=[256] * 8, seed=BASE_SEED, offdiag_std=0.1),
    "k24_m512_ramp": dict(K=24, N=24, two_sz=0, M=[128, 256] + [512] * 8, seed=BASE_SEED + 1,
                          offdiag_std=0.1),
    "k40_m2000_ramp": dict(K=40, N=40, two_sz=0, M=[250, 500, 1000, 2000, 2000, 2000],
                           seed=BASE_SEED + 2, offdiag_std=0.05),
}
