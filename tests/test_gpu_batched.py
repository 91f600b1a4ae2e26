"""Batched tensor-core sigma: several independent two-site problems fused into
one launch per stage (and replayed as a CUDA graph) against the same problems
run one by one, and against the FP64 path."""
import numpy as np
import pytest

import paper_1605_02611_gb300 as G
from paper_1605_02611_gb300 import synth

from gpu_util import context_with_mps, require_gpu

pytestmark = pytest.mark.gpu

# (K, M, k): different orbital counts, bond dimensions and sweep positions, so
# the concatenated work lists differ in shape and number of chunks
PROBLEMS = [(6, 20, 2), (10, 1000, 3), (12, 300, 5)]


def _problems(torch, precision=2, chunk_mb=None):
    out = []
    for i, (K, M, k) in enumerate(PROBLEMS):
        h, eri = synth.integrals(K, 300 + i)
        bonds, T = synth.random_isometric_mps(K, K, 0, M, 310 + i, k, 0.5)
        ctx = context_with_mps(h, eri, K, 0, bonds, T)
        ctx.prepare(k)
        x = ctx.pack(synth.random_psi(bonds[k], bonds[k + 2], 320 + i))
        y64, _ = ctx.sigma(x)
        ctx.set_precision(precision)
        if chunk_mb:
            ctx.set_chunk_budget(chunk_mb)
        ctx.keep_host_plans(True)
        ctx.prepare(k)
        y, _ = ctx.sigma(x)
        xd = torch.tensor(x, device="cuda")
        yd = torch.zeros_like(xd)
        out.append(dict(ctx=ctx, x=x, y64=y64, y=y, xd=xd, yd=yd))
    torch.cuda.synchronize()
    return out


@pytest.mark.parametrize("use_graph,precision,chunk_mb", [(False, 2, None), (True, 2, None), (True, 3, 1)])
def test_batched_matches_individual(use_graph, precision, chunk_mb):
    torch = require_gpu()
    ps = _problems(torch, precision, chunk_mb)
    b = G.Batch([p["ctx"] for p in ps])
    for rep in range(3):  # with a graph: eager + capture, then two replays
        for p in ps:
            p["yd"].zero_()
        torch.cuda.synchronize()
        ms, fl = b.sigma([p["xd"].data_ptr() for p in ps], [p["yd"].data_ptr() for p in ps], use_graph)
        assert ms > 0 and fl > 0
        for p in ps:
            yb = p["yd"].cpu().numpy()
            ref = p["y"]
            assert np.all(np.isfinite(yb))
            # same products and slices; only the order of the FP32 split-K atomics differs
            assert np.linalg.norm(yb - ref) / np.linalg.norm(ref) < 1e-6
            assert np.linalg.norm(yb - p["y64"]) / np.linalg.norm(p["y64"]) < 1e-4
    b.close()


def test_batched_flops_are_the_sum():
    torch = require_gpu()
    ps = _problems(torch)
    b = G.Batch([p["ctx"] for p in ps])
    _, fl = b.sigma([p["xd"].data_ptr() for p in ps], [p["yd"].data_ptr() for p in ps], False)
    each = [p["ctx"].sigma(p["x"])[1] for p in ps]
    assert fl == pytest.approx(sum(each), rel=1e-12)
    b.close()


def test_batched_rejects_unsuitable_contexts():
    torch = require_gpu()
    K, M, k = 6, 20, 2
    h, eri = synth.integrals(K, 7)
    bonds, T = synth.random_isometric_mps(K, K, 0, M, 8, k)
    ctx = context_with_mps(h, eri, K, 0, bonds, T)
    with pytest.raises(G.GbdmrgError):      # not prepared
        G.Batch([ctx])
    ctx.prepare(k)
    with pytest.raises(G.GbdmrgError):      # FP64 plan: no tensor-core work lists
        G.Batch([ctx])
    ctx.set_precision(2)
    ctx.prepare(k)
    with pytest.raises(G.GbdmrgError):      # host copies of the work lists not kept
        G.Batch([ctx])
    ctx.keep_host_plans(True)
    ctx.prepare(k)
    G.Batch([ctx]).close()
    del torch
