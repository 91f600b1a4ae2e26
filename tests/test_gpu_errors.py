"""Error behaviour of the C-ABI on a GPU: every failure is a status code, never a crash."""
import numpy as np
import pytest

import paper_1605_02611_gb300 as G
from paper_1605_02611_gb300 import synth

from gpu_util import require_gpu

pytestmark = pytest.mark.gpu


def test_state_errors():
    require_gpu()
    h, eri = synth.integrals(4, 1)
    ctx = G.Context(h, eri, 4, 0)
    with pytest.raises(G.GbdmrgError, match="ESTATE"):
        ctx.prepare(1)                      # MPS not set
    bonds, T = synth.random_mps(4, 4, 0, 8, 1)
    lab = [b.labels() for b in bonds]
    with pytest.raises(G.GbdmrgError, match="EINVAL"):
        ctx.set_mps([T[0]], [np.array([[1, 0]]), lab[1]])   # left boundary must be (0, 0)
    ctx.set_mps(T, lab)
    with pytest.raises(G.GbdmrgError, match="EINVAL"):
        ctx.prepare(3)                      # k + 1 == K
    with pytest.raises(G.GbdmrgError, match="EINVAL"):
        ctx.run([0], 1e-8)                  # non-positive M


def test_invalid_problem():
    require_gpu()
    h, eri = synth.integrals(3, 1)
    with pytest.raises(G.GbdmrgError):
        G.Context(h, eri, 7, 1)             # N > 2K
    with pytest.raises(G.GbdmrgError):
        G.Context(h + np.triu(np.ones_like(h), 1), eri, 2, 0)
