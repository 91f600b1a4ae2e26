"""Tensor-core H_eff.psi and diagonal against the oracle, element by element, on
the operand path the K=40 bench runs: the W-contracted (blocking) sums formed
on the tensor cores (three BF16 slices, FP32 accumulation).  By default that
path is taken only by sums of at least 1e5 terms (the switch site K/2 of large
problems); here the threshold is lowered to one term so that every blocking
sum of both sides of a small problem takes it.  The two-site positions are
the central ones, whose right site is the MPO's switch site.

Tolerance: three BF16 slices carry the operands to ~2^-24, and the FP32
accumulation in the tensor cores leaves ~1e-5 relative (rounding toward
zero); 2e-4 of the largest element bounds both with margin.
"""
import numpy as np
import pytest

from oracle import fci
from oracle import mps as omps
from paper_1605_02611_gb300 import synth

from gpu_util import context_with_mps, rel_err, require_gpu

pytestmark = pytest.mark.gpu

TOL_X3 = 2e-4


def _oracle_diag_sample(T, k, h, eri, Na, Nb, mask, idx):
    """Diagonal elements e_i . H_eff e_i of the oracle's P^T H P at flat indices idx
    (indices into the allowed entries in mask order)."""
    P = omps.TwoSiteProjector(T, k, Na, Nb)
    flat = np.flatnonzero(mask.reshape(-1))
    cols = []
    for i in idx:
        e = np.zeros(mask.size)
        e[flat[i]] = 1.0
        cols.append(P.project(e.reshape(mask.shape)))
    Pm = np.stack(cols, axis=1)
    HP = fci.sigma(h, eri, Na, Nb, Pm)
    return np.einsum("di,di->i", Pm, HP)


@pytest.mark.parametrize("K,N,two_sz,M,k", [
    (8, 8, 0, 60, 3),     # right site 4 = K/2 (switch site)
    (10, 10, 0, 200, 4),  # right site 5 = K/2, bonds of 200
    (9, 9, 1, 60, 3),     # odd K, S_z = 1/2: operator classes without elements at some bonds
])
def test_tc_w_sums_sigma_and_diag_vs_oracle(K, N, two_sz, M, k):
    require_gpu()
    seed = 500 + 10 * K + two_sz
    Na, Nb = (N + two_sz) // 2, (N - two_sz) // 2
    h, eri = synth.integrals(K, seed)
    bonds, T = synth.random_isometric_mps(K, N, two_sz, M, seed + 1, k, 0.5)
    psi = synth.random_psi(bonds[k], bonds[k + 2], seed + 2)
    ref = omps.sigma(T, k, psi, h, eri, Na, Nb)
    ctx = context_with_mps(h, eri, N, two_sz, bonds, T)
    ctx.set_precision(2)
    ctx.set_tc_combos(True, 1)
    ctx.prepare(k)
    y, _ = ctx.sigma(ctx.pack(psi))
    r = ctx.pack(ref)
    err = rel_err(y, r)
    print(f"K={K} 2Sz={two_sz}: tensor-core sums + sigma max-element error {err:.2e}")
    assert err < TOL_X3
    # diagonal of H_eff from the tensor-core sums: a sample of elements (every block
    # contributes) against the oracle's explicit e_i . P^T H P e_i
    d = ctx.diag()
    lab = [b.labels() for b in bonds]
    mask = omps.allowed_mask(lab[k], lab[k + 2])
    rng = np.random.default_rng(seed)
    n = int(mask.sum())
    idx = np.unique(np.concatenate([rng.choice(n, size=min(n, 160), replace=False), [0, n - 1]]))
    dref = _oracle_diag_sample(T, k, h, eri, Na, Nb, mask, idx)
    # the library's packed order differs from the mask order: map through the layout
    ordered = np.zeros(mask.shape)
    ordered[mask] = np.arange(n)
    pos = ctx.pack(ordered).astype(np.int64)      # packed slot -> mask-order index
    inv = np.empty(n, dtype=np.int64)
    inv[pos] = np.arange(n)
    got = d[inv[idx]]
    derr = np.abs(got - dref).max() / np.abs(dref).max()
    print(f"K={K} 2Sz={two_sz}: diagonal max-element error {derr:.2e}")
    assert derr < TOL_X3
    ctx.close()


def test_tc_sigma_multi_tile_multi_chunk_vs_oracle():
    """Three-slice tensor-core sigma at K=10, M=1000 (sectors of ~100 rows: several
    128-row tiles per group and 64-wide K steps per term), with the operator terms
    cut into many chunks by a small intermediate budget, against the oracle."""
    require_gpu()
    K, N, M, k, seed = 10, 10, 1000, 3, 5
    h, eri = synth.integrals(K, seed)
    bonds, T = synth.random_isometric_mps(K, N, 0, M, seed + 1, k, 0.5)
    psi = synth.random_psi(bonds[k], bonds[k + 2], seed + 2)
    ref = omps.sigma(T, k, psi, h, eri, 5, 5)
    ctx = context_with_mps(h, eri, N, 0, bonds, T)
    ctx.set_precision(2)
    ctx.set_chunk_budget(4)
    ctx.prepare(k)
    assert max(ctx.layout[:, 1].max(), ctx.layout[:, 5].max()) > 64
    y, _ = ctx.sigma(ctx.pack(psi))
    err = rel_err(y, ctx.pack(ref))
    print(f"K=10 M=1000 three-slice multi-chunk sigma max-element error {err:.2e}")
    assert err < TOL_X3
    ctx.close()
