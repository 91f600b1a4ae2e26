"""Tensor-core H_eff.psi on the TMA-staged work lists (precisions 4, 5, 6: one
BF16 pass, three and two BF16 slices per operand) against the oracle and the
FP64 path, element by element; and the Davidson refinement of a step.

One BF16 pass rounds psi, both W-contracted operators and the intermediate X
to 8 significant bits (2^-9 relative each) and accumulates in FP32; with the
cancellations between terms of H_eff the result carries a few 1e-3 relative
error at these sizes: bars 1e-2 in norm and 2e-2 of the largest element.
Three (two) slices carry the operands to ~2^-24 (~2^-16); what remains is the
FP32 accumulation in the tensor cores (~1e-5): bars 1e-4 and 2e-4.
"""
import numpy as np
import pytest

from oracle import mps as omps
from paper_1605_02611_gb300 import synth

from gpu_util import context_with_mps, rel_err, require_gpu

pytestmark = pytest.mark.gpu

CASES = [
    (6, 6, 0, 20, 2),       # small blocks, one tile per group
    (9, 9, 1, 60, 3),       # odd K, S_z = 1/2, switch site on the right
    (10, 10, 0, 1000, 3),   # sectors of ~100: K blocks over two 64-wide steps, several row tiles
    (12, 12, 0, 300, 5),    # more bond states
]
TOL = {4: (1e-2, 2e-2), 5: (1e-4, 2e-4), 6: (1e-4, 2e-4)}


def _case(K, N, two_sz, M, k, seed):
    require_gpu()
    Na, Nb = (N + two_sz) // 2, (N - two_sz) // 2
    h, eri = synth.integrals(K, seed)
    bonds, T = synth.random_isometric_mps(K, N, two_sz, M, seed + 1, k, 0.5)
    psi = synth.random_psi(bonds[k], bonds[k + 2], seed + 2)
    return h, eri, bonds, T, psi, Na, Nb


@pytest.mark.parametrize("precision", [4, 5, 6])
@pytest.mark.parametrize("K,N,two_sz,M,k", CASES)
def test_tma_sigma_vs_oracle_and_fp64(K, N, two_sz, M, k, precision):
    h, eri, bonds, T, psi, Na, Nb = _case(K, N, two_sz, M, k, 700 + K)
    ctx = context_with_mps(h, eri, N, two_sz, bonds, T)
    ctx.prepare(k)
    x = ctx.pack(psi)
    y64, fl64 = ctx.sigma(x)
    ctx.set_precision(precision)
    ctx.prepare(k)
    y, fl = ctx.sigma(x)
    assert fl == fl64                       # same algorithmic flop count
    st = ctx.plan_stats()
    assert st["stage1_tiles"] > 0 and st["stage2_tiles"] > 0 and st["chunks"] == 1
    e_norm = np.linalg.norm(y - y64) / np.linalg.norm(y64)
    e_max = rel_err(y, y64)
    print(f"K={K} M={M} precision {precision}: TMA sigma vs FP64: {e_norm:.2e} (norm), {e_max:.2e} (max element)")
    tn, tm = TOL[precision]
    assert e_norm < tn and e_max < tm
    if K <= 10:
        ref = ctx.pack(omps.sigma(T, k, psi, h, eri, Na, Nb))
        assert rel_err(y64, ref) < 1e-11    # the FP64 path is the oracle's H_eff.psi
        assert rel_err(y, ref) < tm
    # a second call on the same work lists gives the same vector up to the order of
    # the FP32 reductions of split stage-2 tiles
    y2, _ = ctx.sigma(x)
    assert np.linalg.norm(y2 - y) <= 1e-5 * np.linalg.norm(y)
    ctx.close()


@pytest.mark.parametrize("precision", [4, 5])
def test_tma_chunks_match_one_chunk(precision):
    """A small budget for the X intermediates cuts the bond states into chunks that
    share one buffer (rows a chunk does not write are cleared first): same sigma."""
    h, eri, bonds, T, psi, Na, Nb = _case(10, 10, 0, 1000, 3, 777)
    ctx = context_with_mps(h, eri, 10, 0, bonds, T)
    ctx.set_precision(precision)
    ctx.prepare(3)
    x = ctx.pack(psi)
    y1, _ = ctx.sigma(x)
    ctx.set_tma_budget(2)
    ctx.prepare(3)
    assert ctx.plan_stats()["chunks"] > 1
    for _ in range(2):
        yc, _ = ctx.sigma(x)
        assert np.all(np.isfinite(yc))
        assert np.linalg.norm(yc - y1) <= 1e-5 * np.linalg.norm(y1)
    ctx.close()


def test_refined_step_matches_fp64_step():
    """One two-site step at K=10, M=200 from a random isometric MPS (about 130 FP64
    Davidson iterations): the single-pass solve alone ends ~1e-3 relative off (its
    operator rounds to 8 bits); refined with the three-slice operator the step's
    eigenvalue is the FP64 step's within 1e-6 relative."""
    h, eri, bonds, T, psi, Na, Nb = _case(10, 10, 0, 200, 4, 790)
    e = {}
    for label, prec, ref in (("fp64", 0, -1), ("one pass", 4, -1), ("refined", 4, 5)):
        ctx = context_with_mps(h, eri, 10, 0, bonds, T)
        ctx.set_precision(prec)
        ctx.set_refinement(ref, 60)
        ctx.prepare(4)
        e[label], _, it, _ = ctx.step(4, 0, 200, 1e-8, 260)
        print(f"{label}: E {e[label]:.10f}, {it} iterations")
        ctx.close()
    assert abs(e["one pass"] - e["fp64"]) < 1e-2 * abs(e["fp64"])
    assert abs(e["refined"] - e["fp64"]) < 1e-6 * abs(e["fp64"])
