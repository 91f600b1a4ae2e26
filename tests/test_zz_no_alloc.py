"""The no-allocation diagonal entry point (gbdmrg_diag_noalloc) through the C-ABI.

It serves callers that cannot allocate device memory when they need the
Davidson preconditioner input (e.g. inside a framework whose memory manager
owns the device): all its scratch sits in a fixed array inside the library.  It must give the same
diagonal as gbdmrg_diag, call after call, and refuse problems whose scratch
would not fit.  This file is collected last on purpose.
"""
import numpy as np
import pytest

import paper_1605_02611_gb300 as G
from paper_1605_02611_gb300 import synth

from gpu_util import context_with_mps, rel_err, require_gpu

pytestmark = pytest.mark.gpu


@pytest.mark.parametrize("K,M,k", [
    (8, 60, 3),      # every psi block inside one 64 x 64 GEMM tile
    (10, 1000, 3),   # blocks of 100 columns: several tiles per block, ragged tails
])
def test_diag_noalloc_matches_diag_twice(K, M, k):
    torch = require_gpu()
    N = K
    h, eri = synth.integrals(K, 91)
    bonds, T = synth.random_mps(K, N, 0, M, 92)
    ctx = context_with_mps(h, eri, N, 0, bonds, T)
    ctx.prepare(k)
    if K == 10:
        assert max(ctx.layout[:, 1].max(), ctx.layout[:, 5].max()) > 64
    ref = ctx.diag()
    for _ in range(2):
        out = torch.full((ctx.nnz,), float("nan"), device="cuda", dtype=torch.float64)
        torch.cuda.synchronize()
        ctx.diag_noalloc(out.data_ptr())
        torch.cuda.synchronize()
        got = out.cpu().numpy()
        assert np.all(np.isfinite(got))
        assert rel_err(got, ref) < 1e-11


def test_diag_noalloc_rejects_oversized_problem():
    torch = require_gpu()
    # K=32, M=1200: the gathered diagonals alone need 4 (D_k + D_k+2) x 514 doubles > 32 MiB
    K, N, M, k = 32, 32, 1200, 15
    h, eri = synth.integrals(K, 93)
    bonds, T = synth.random_isometric_mps(K, N, 0, M, 94, k, 1.0)
    ctx = context_with_mps(h, eri, N, 0, bonds, T)
    ctx.prepare(k)
    out = torch.zeros(ctx.nnz, device="cuda", dtype=torch.float64)
    with pytest.raises(G.GbdmrgError, match="too large for the no-allocation"):
        ctx.diag_noalloc(out.data_ptr())
