"""Tensor-core (tcgen05) mixed-precision sigma against the FP64 path and the oracle.

Accuracy cases use mixed-canonical (isometric) MPS, the regime of a DMRG
sweep, where the renormalised operators have norms of the order of |H|.
"""
import numpy as np
import pytest

from oracle import fci, mps as omps
from paper_1605_02611_gb300 import synth

from gpu_util import context_with_mps, rel_err, require_gpu

pytestmark = pytest.mark.gpu


def _pair(K, N, M, k, seed, spread=0.5):
    require_gpu()
    h, eri = synth.integrals(K, seed)
    bonds, T = synth.random_isometric_mps(K, N, 0, M, seed + 1, k, spread)
    ctx = context_with_mps(h, eri, N, 0, bonds, T)
    ctx.prepare(k)
    x = ctx.pack(synth.random_psi(bonds[k], bonds[k + 2], seed + 2))
    ref, fl64 = ctx.sigma(x)
    return ctx, x, ref, fl64


CASES = [(6, 20, 2), (10, 1000, 3), (12, 300, 5)]


@pytest.mark.parametrize("K,M,k", CASES)
def test_bf16_single_pass_close_to_fp64(K, M, k):
    ctx, x, ref, fl64 = _pair(K, K, M, k, 100 + K)
    ctx.set_precision(1)
    ctx.prepare(k)
    y, fl = ctx.sigma(x)
    assert fl == fl64                     # same algorithmic flop count
    assert np.linalg.norm(y - ref) / np.linalg.norm(ref) < 1e-2


@pytest.mark.parametrize("K,M,k", CASES)
def test_bf16_two_slices_close_to_fp64(K, M, k):
    """Two BF16 slices carry the operands to ~2^-16; three products."""
    ctx, x, ref, _ = _pair(K, K, M, k, 250 + K)
    ctx.set_precision(3)
    ctx.prepare(k)
    y, _ = ctx.sigma(x)
    err = np.linalg.norm(y - ref) / np.linalg.norm(ref)
    print(f"two-slice sigma relative error K={K} M={M}: {err:.2e}")
    assert err < 1e-4


@pytest.mark.parametrize("K,M,k", CASES)
def test_bf16_three_slices_close_to_fp64(K, M, k):
    """Three BF16 slices carry the operands to ~2^-24; what remains is the
    tensor-core FP32 accumulation, which rounds toward zero (a small systematic
    shrink of |sigma|, measured ~1e-5 to 3e-5 relative here)."""
    ctx, x, ref, _ = _pair(K, K, M, k, 200 + K)
    ctx.set_precision(2)
    ctx.prepare(k)
    y, _ = ctx.sigma(x)
    assert np.linalg.norm(y - ref) / np.linalg.norm(ref) < 1e-4
    # the error is mostly a uniform shrink: after removing the best scale it is smaller
    a = (y @ ref) / (ref @ ref)
    assert np.linalg.norm(y - a * ref) <= np.linalg.norm(y - ref)


def test_three_slices_against_oracle():
    require_gpu()
    K, N, M, k = 6, 6, 20, 2
    h, eri = synth.integrals(K, 5)
    bonds, T = synth.random_isometric_mps(K, N, 0, M, 6, k)
    psi = synth.random_psi(bonds[k], bonds[k + 2], 7)
    ref = omps.sigma(T, k, psi, h, eri, 3, 3)
    ctx = context_with_mps(h, eri, N, 0, bonds, T)
    ctx.set_precision(2)
    ctx.prepare(k)
    y, _ = ctx.sigma(ctx.pack(psi))
    r = ctx.pack(ref)
    assert np.linalg.norm(y - r) / np.linalg.norm(r) < 1e-5


def test_mixed_dmrg_k8_energy_equals_fci():
    """Tensor-core sweep (three BF16 slices) with the FP64 refinement step: K=8, M=256 vs FCI."""
    require_gpu()
    import scipy.sparse.linalg as spla
    cfg = synth.WORKLOADS["k8_m256_fp64"]
    h, eri = synth.integrals(8, cfg["seed"], cfg["offdiag_std"])
    bonds, T = synth.random_mps(8, 8, 0, 256, cfg["seed"])
    ctx = context_with_mps(h, eri, 8, 0, bonds, T)
    out = ctx.run([256] * 3, [1e-6, 1e-6, 1e-9], precision=2)
    e0 = spla.eigsh(fci.hamiltonian(h, eri, 4, 4), k=1, which="SA", tol=1e-14)[0][0]
    assert abs(out["energy"][-1] - e0) < 1e-9


def test_mixed_vs_fp64_truncated_sweeps():
    """K=12, M=64, six sweeps from the same start: tensor-core sweeps (FP64 last step)
    reach the FP64 sweep energy within 1e-6 Eh."""
    require_gpu()
    K, N, M = 12, 12, 64
    h, eri = synth.integrals(K, 1606)
    bonds, T = synth.random_mps(K, N, 0, M, 1607)
    e = {}
    for prec in (0, 2, 3):
        ctx = context_with_mps(h, eri, N, 0, bonds, T)
        e[prec] = ctx.run([M] * 6, [1e-6, 1e-7, 1e-8, 1e-9, 1e-9, 1e-9], precision=prec)["energy"]
        ctx.close()
    print("three-slice - fp64 sweep energies:", e[2] - e[0])
    print("two-slice - fp64 sweep energies:", e[3] - e[0])
    assert abs(e[2][-1] - e[0][-1]) < 1e-6
    assert abs(e[3][-1] - e[0][-1]) < 1e-6


@pytest.mark.parametrize("precision", [1, 2, 3])
def test_chunked_plans_match_unchunked(precision):
    """A small intermediate budget splits the operator terms into many chunks
    (the regime of large bonds); results must not depend on the chunking and
    must stay finite (the shared intermediate buffer is reused between chunks)."""
    ctx, x, ref, _ = _pair(10, 10, 1000, 3, 400)
    ctx.set_chunk_budget(1)
    ctx.prepare(3)
    y64c, _ = ctx.sigma(x)
    assert np.linalg.norm(y64c - ref) / np.linalg.norm(ref) < 1e-12
    ctx.set_precision(precision)
    ctx.set_chunk_budget(2048)
    ctx.prepare(3)
    y1, _ = ctx.sigma(x)
    tol = 1e-2 if precision == 1 else 1e-4
    for mb in (4, 1):
        ctx.set_chunk_budget(mb)
        ctx.prepare(3)
        for _ in range(2):
            yc, _ = ctx.sigma(x)
            assert np.all(np.isfinite(yc))
            assert np.linalg.norm(yc - ref) / np.linalg.norm(ref) < tol
            # another partition of the term sums: FP32 tensor-core accumulation in another order
            assert np.linalg.norm(yc - y1) / np.linalg.norm(y1) < 1e-5
