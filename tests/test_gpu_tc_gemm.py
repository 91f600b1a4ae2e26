"""Tensor-core grouped block GEMM (tcgen05, BF16 in, FP32 accumulate) against
an FP64 product of the same BF16-rounded operands."""
import numpy as np
import pytest

import paper_1605_02611_gb300 as G

from gpu_util import require_gpu

pytestmark = pytest.mark.gpu


def _pad8(x):
    return (x + 7) // 8 * 8


def _case(rng, torch, shapes, beta=0, trans=0):
    """shapes: list of tasks, each (m, n, [k_t...], [neg_t...])."""
    tasks, terms, keep, refs = [], [], [], []
    for (m, n, ks, negs) in shapes:
        shp = (n, m) if trans else (m, n)
        C = torch.randn(*shp, device="cuda", dtype=torch.float32) if beta else torch.zeros(*shp, device="cuda")
        ref = C.double().clone().T.contiguous() if (beta and trans) else (
            C.double().clone() if beta else torch.zeros(m, n, device="cuda", dtype=torch.float64))
        t0 = len(terms)
        for k, neg in zip(ks, negs):
            la, lb = _pad8(k) + 8 * int(rng.integers(0, 2)), _pad8(k)
            A = torch.zeros(m, la, device="cuda", dtype=torch.bfloat16)
            B = torch.zeros(n, lb, device="cuda", dtype=torch.bfloat16)
            A[:, :k] = torch.randn(m, k, device="cuda").to(torch.bfloat16)
            B[:, :k] = torch.randn(n, k, device="cuda").to(torch.bfloat16)
            keep += [A, B]
            terms.append([A.data_ptr(), B.data_ptr(), la, lb, k, neg])
            prod = A[:, :k].double() @ B[:, :k].double().T
            ref += -prod if neg else prod
        keep.append(C)
        tasks.append([C.data_ptr(), m if trans else n, m, n, beta, t0, len(terms), trans])
        refs.append((C, ref))
    G.gemm_bf16_selftest(np.array(tasks), np.array(terms))
    torch.cuda.synchronize()
    for C, ref in refs:
        got = C.double().T if trans else C.double()
        err = (got - ref).abs().max().item()
        scale = ref.abs().max().item() + 1.0
        assert err <= 1e-5 * scale, (err, scale)


def test_single_tile_exact_shapes():
    torch = require_gpu()
    _case(np.random.default_rng(0), torch, [(128, 128, [64], [0])])


def test_ragged_multi_tile_multi_term():
    torch = require_gpu()
    rng = np.random.default_rng(1)
    shapes = []
    for _ in range(12):
        m, n = int(rng.integers(1, 300)), int(rng.integers(1, 300))
        nt = int(rng.integers(1, 4))
        ks = [int(rng.integers(1, 200)) for _ in range(nt)]
        negs = [int(rng.integers(0, 2)) for _ in range(nt)]
        shapes.append((m, n, ks, negs))
    _case(rng, torch, shapes)


def test_accumulate_beta_and_long_k():
    torch = require_gpu()
    rng = np.random.default_rng(2)
    _case(rng, torch, [(200, 70, [1000, 3], [0, 1]), (5, 260, [130], [0])], beta=1)


def test_transposed_store_and_many_tiles():
    """More tiles than resident CTAs (persistent loop, both TMEM accumulators), transposed stores."""
    torch = require_gpu()
    rng = np.random.default_rng(3)
    shapes = [(int(rng.integers(1, 260)), int(rng.integers(1, 300)), [int(rng.integers(1, 150))], [0])
              for _ in range(400)]
    _case(rng, torch, shapes, beta=1, trans=1)
    _case(rng, torch, shapes[:50], beta=0, trans=0)


def test_rejects_misaligned():
    torch = require_gpu()
    A = torch.zeros(16, 16, device="cuda", dtype=torch.bfloat16)
    C = torch.zeros(16, 16, device="cuda")
    with pytest.raises(G.GbdmrgError):
        G.gemm_bf16_selftest(np.array([[C.data_ptr(), 16, 16, 16, 0, 0, 1, 0]]),
                             np.array([[A.data_ptr() + 2, A.data_ptr(), 16, 16, 8, 0]]))
