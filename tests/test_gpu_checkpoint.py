"""Checkpoint / resume of the MPS: a saved and reloaded state continues the
sweep exactly as the original one, and bad files are rejected."""
import os

import numpy as np
import pytest

import paper_1605_02611_gb300 as G
from paper_1605_02611_gb300 import synth

from gpu_util import context_with_mps, require_gpu

pytestmark = pytest.mark.gpu


def _run(tmp_path):
    K, M = 8, 64
    h, eri = synth.integrals(K, 77)
    bonds, T = synth.random_mps(K, K, 0, M, 78)
    a = context_with_mps(h, eri, K, 0, bonds, T)
    a.run([M] * 2, 1e-8)
    path = os.path.join(str(tmp_path), "mps.ckpt")
    a.save(path)
    return h, eri, K, M, a, path


def test_resume_continues_identically(tmp_path):
    require_gpu()
    h, eri, K, M, a, path = _run(tmp_path)
    b = G.Context(h, eri, K, 0)
    b.load(path)
    for k in range(K):
        assert np.array_equal(a.get_mps(k), b.get_mps(k))
    for bd in range(K + 1):
        assert np.array_equal(a.get_bond(bd), b.get_bond(bd))
    ea = a.run([M], 1e-9)["energy"]
    eb = b.run([M], 1e-9)["energy"]
    assert ea[0] == eb[0]          # FP64 path: the same deterministic sweep
    a.close()
    b.close()


def test_bad_checkpoints_are_rejected(tmp_path):
    require_gpu()
    h, eri, K, M, a, path = _run(tmp_path)
    raw = open(path, "rb").read()
    # truncated file
    bad = os.path.join(str(tmp_path), "short.ckpt")
    open(bad, "wb").write(raw[: len(raw) // 2])
    b = G.Context(h, eri, K, 0)
    with pytest.raises(G.GbdmrgError, match="EIO"):
        b.load(bad)
    # not a checkpoint
    junk = os.path.join(str(tmp_path), "junk.ckpt")
    open(junk, "wb").write(b"x" * 64)
    with pytest.raises(G.GbdmrgError, match="EIO"):
        b.load(junk)
    with pytest.raises(G.GbdmrgError, match="EIO"):
        b.load(os.path.join(str(tmp_path), "missing.ckpt"))
    # another problem size
    h6, eri6 = synth.integrals(6, 1)
    c = G.Context(h6, eri6, 6, 0)
    with pytest.raises(G.GbdmrgError, match="EINVAL"):
        c.load(path)
    # a context without an MPS cannot be saved
    with pytest.raises(G.GbdmrgError, match="ESTATE"):
        c.save(os.path.join(str(tmp_path), "empty.ckpt"))
    # the failed loads left b without an MPS; a good file still loads
    b.load(path)
    assert np.array_equal(a.get_mps(3), b.get_mps(3))
    for x in (a, b, c):
        x.close()
