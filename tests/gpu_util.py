"""Helpers for the GPU tests: build/load the library, open contexts."""
import numpy as np
import pytest

import paper_1605_02611_gb300 as G


def require_gpu():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    G.load()  # raises (does not skip) when the extension is missing on a GPU machine
    return torch


def context_with_mps(h, eri, N, two_sz, bonds, tensors):
    ctx = G.Context(h, eri, N, two_sz)
    ctx.set_mps(tensors, [b.labels() for b in bonds])
    return ctx


def rel_err(a, b):
    return float(np.abs(a - b).max() / max(np.abs(b).max(), 1e-300))
