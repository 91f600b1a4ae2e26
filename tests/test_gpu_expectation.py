"""Expectation values from the environments of a converged MPS, against the
sweep energy and against an FCI-vector expectation computed by the oracle."""
import os

import numpy as np
import pytest

import paper_1605_02611_gb300 as G
from oracle import fci
from paper_1605_02611_gb300 import synth

from gpu_util import context_with_mps, require_gpu

pytestmark = pytest.mark.gpu


def test_energy_and_one_body_expectation(tmp_path):
    require_gpu()
    K, N, M = 6, 6, 64          # M = 4^3: the MPS is exact
    h, eri = synth.integrals(K, 91)
    bonds, T = synth.random_mps(K, N, 0, M, 92)
    ctx = context_with_mps(h, eri, N, 0, bonds, T)
    e = ctx.run([M] * 4, 1e-10)["energy"][-1]
    for k in (0, 1):
        ctx.prepare(k)
        assert abs(ctx.expectation() - e) < 1e-9
    # a one-body operator t (eri = 0) in the same state, against <c|T|c> of the FCI vector
    rng = np.random.default_rng(93)
    t = rng.normal(size=(K, K))
    t = 0.5 * (t + t.T)
    path = os.path.join(str(tmp_path), "gs.ckpt")
    ctx.save(path)
    ot = G.Context(t, np.zeros((K, K, K, K)), N, 0)
    ot.load(path)
    ot.prepare(1)
    val = ot.expectation()
    w, c = fci.ground_state(h, eri, N // 2, N // 2)
    c = c[:, 0]
    Tm = fci.hamiltonian(t, np.zeros((K, K, K, K)), N // 2, N // 2)
    ref = float(c @ (Tm @ c))
    assert abs(val - ref) < 1e-7
    assert abs(e - w[0]) < 1e-9
    with pytest.raises(G.GbdmrgError):
        G.Context(t, np.zeros((K, K, K, K)), N, 0).expectation()   # not prepared
    ctx.close()
    ot.close()
