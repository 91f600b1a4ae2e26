"""Learned Davidson preconditioner on the GPU against the FP64 NumPy reference
(oracle/mlp.py): forward passes, loss gradients, features and training pairs,
the preconditioner itself, and DMRG energies with the network in the loop."""
import numpy as np
import pytest

import paper_1605_02611_gb300 as G
from oracle import fci
from oracle import mlp as omlp
from paper_1605_02611_gb300 import synth

from gpu_util import context_with_mps, require_gpu

pytestmark = pytest.mark.gpu


def _bf16(a):
    """Round to the nearest BF16 (ties to even), returned as float64."""
    a = np.asarray(a, dtype=np.float32)
    u = a.view(np.uint32).astype(np.uint64)
    u = (u + 0x7FFF + ((u >> 16) & 1)) & 0xFFFF0000
    return u.astype(np.uint32).view(np.float32).astype(np.float64)


def _params(seed, w3=0.2):
    rng = np.random.default_rng(seed)
    p = {"W1": rng.normal(0, 1 / np.sqrt(5), (256, 5)), "b1": rng.normal(0, 0.1, 256),
         "W2": rng.normal(0, 1 / 16, (256, 256)), "b2": rng.normal(0, 0.1, 256),
         "W3": rng.normal(0, w3, 256), "b3": np.array([0.05])}
    for k in ("W1", "W2", "W3"):
        p[k] = _bf16(p[k])          # the network rounds its weights to BF16: use representable values
    for k in ("b1", "b2", "b3"):
        p[k] = np.asarray(p[k], dtype=np.float32).astype(np.float64)
    return omlp.flatten(p)


def _features(seed, n):
    return np.random.default_rng(seed).normal(size=(n, 5)).astype(np.float32)


def test_forward_matches_oracle():
    require_gpu()
    net = G.Mlp(seed=1)
    th = _params(2)
    net.set_params(th)
    assert np.array_equal(net.get_params(), th.astype(np.float32))
    F = _features(3, 1000)
    ref, _ = omlp.forward(th, F.astype(np.float64))
    g = net.forward(F, inference=False)
    assert np.max(np.abs(g - ref)) / np.max(np.abs(ref)) < 1e-5
    # inference numerics: h1 rounded to BF16 before the tensor-core layer
    gi = net.forward(F, inference=True)
    assert np.max(np.abs(gi - ref)) / np.max(np.abs(ref)) < 2e-2
    net.close()


@pytest.mark.parametrize("n", [1, 37, 512, 3000])
def test_loss_gradient_matches_oracle(n):
    require_gpu()
    net = G.Mlp(seed=4)
    th = _params(5)
    net.set_params(th)
    F = _features(6, n)
    rng = np.random.default_rng(7)
    P = rng.normal(size=n).astype(np.float32)
    T = rng.normal(size=n).astype(np.float32)
    Lr, gr = omlp.loss_grad(th, F.astype(np.float64), P.astype(np.float64), T.astype(np.float64))
    L, g = net.loss_grad(F, P, T)
    assert L == pytest.approx(Lr, rel=1e-5)
    gp, rp = omlp.unflatten(g.astype(np.float64)), omlp.unflatten(gr)
    for name in ("W1", "b1", "W2", "b2", "W3", "b3"):
        err = np.max(np.abs(gp[name] - rp[name])) / max(np.max(np.abs(rp[name])), 1e-30)
        assert err < 1e-3, name
    net.close()


def test_untrained_network_is_the_diagonal_preconditioner():
    require_gpu()
    net = G.Mlp(seed=8)
    p = omlp.unflatten(net.get_params().astype(np.float64))
    assert np.all(p["W3"] == 0) and p["b3"][0] == 0
    F = _features(9, 100)
    assert np.all(net.forward(F) == 0) and np.all(net.forward(F, inference=True) == 0)
    net.close()


def _prepared(K, M, k, seed):
    h, eri = synth.integrals(K, seed)
    bonds, T = synth.random_isometric_mps(K, K, 0, M, seed + 1, k)
    ctx = context_with_mps(h, eri, K, 0, bonds, T)
    blk = ctx.prepare(k)
    blocks = [(int(b[6]), int(b[1] * b[5])) for b in blk]
    return ctx, blocks


def test_precondition_matches_oracle():
    require_gpu()
    ctx, blocks = _prepared(8, 60, 3, 11)
    d = ctx.diag()
    rng = np.random.default_rng(12)
    r = rng.normal(size=ctx.nnz)
    theta = float(np.min(d)) - 0.3
    t0 = ctx.precondition(r, theta)          # diagonal preconditioner (no network)
    assert np.allclose(t0, omlp.diag_correction(r, d, theta), rtol=1e-14, atol=0)
    net = G.Mlp(seed=13)
    th = _params(14, w3=0.05)
    net.set_params(th)
    ctx.set_preconditioner(net)
    t = ctx.precondition(r, theta)
    ref = omlp.precondition(th, r, d, theta, blocks)
    assert np.linalg.norm(t - ref) / np.linalg.norm(ref) < 1e-2
    ctx.close()
    net.close()


def test_pairs_match_oracle():
    require_gpu()
    ctx, blocks = _prepared(8, 60, 3, 21)
    d = ctx.diag()
    rng = np.random.default_rng(22)
    n = ctx.nnz
    psi = rng.normal(size=n)
    psi /= np.linalg.norm(psi)
    x = psi + 0.2 * rng.normal(size=n)
    x /= np.linalg.norm(x)
    r = rng.normal(size=n) * 0.1
    theta = float(np.min(d)) - 0.1
    F, P, T, idx = ctx.make_pairs(x, r, theta, psi, 500, 23)
    assert len(idx) == 500 and idx.min() >= 0 and idx.max() < n
    Fr = omlp.features(r, d, theta, blocks)[idx]
    Pr, Tr = omlp.pair_values(x, r, d, theta, psi)
    assert np.allclose(F, Fr, rtol=1e-6, atol=1e-6)
    assert np.allclose(P, Pr[idx], rtol=1e-6, atol=1e-6)
    assert np.allclose(T, Tr[idx], rtol=1e-6, atol=1e-6)
    _, _, _, idx2 = ctx.make_pairs(x, r, theta, psi, 500, 23)   # deterministic in the seed
    assert np.array_equal(idx, idx2)
    ctx.close()


def _harvest_and_train(K, M, sweeps, seed, cap=20000, per=200, epochs=30):
    h, eri = synth.integrals(K, seed)
    bonds, T = synth.random_mps(K, K, 0, M, seed + 1)
    ctx = context_with_mps(h, eri, K, 0, bonds, T)
    ctx.set_harvest(cap, per, seed)
    out = ctx.run([M] * sweeps, 1e-8)
    F, P, Tt = ctx.get_harvest()
    net = G.Mlp(seed=seed)
    l0, l1 = net.train(F, P, Tt, epochs=epochs, batch=1024, lr=1e-3, seed=seed)
    return h, eri, ctx, net, out, (F, P, Tt), (l0, l1)


def test_harvest_and_training_lower_the_loss():
    require_gpu()
    _, _, ctx, net, out, (F, P, T), (l0, l1) = _harvest_and_train(8, 64, 2, 31)
    assert len(P) > 1000
    assert np.all(np.isfinite(F)) and np.all(np.abs(P) <= 100) and np.all(np.abs(T) <= 100)
    L_diag = float(np.mean((P.astype(np.float64) - T) ** 2))   # network output 0
    L_net, _ = net.loss_grad(F, P, T)
    assert l1 < l0
    assert L_net < L_diag
    ctx.close()
    net.close()


def test_dmrg_with_learned_preconditioner_reaches_fci():
    """K=8, N=8, M=256 (exact): whichever preconditioner, the energy is the FCI one."""
    require_gpu()
    import scipy.sparse.linalg as spla
    h, eri, ctx, net, _, _, _ = _harvest_and_train(8, 256, 2, 41)
    e_fci = spla.eigsh(fci.hamiltonian(h, eri, 4, 4), k=1, which="SA", tol=1e-14)[0][0]
    bonds, T = synth.random_mps(8, 8, 0, 256, 43)
    c2 = context_with_mps(h, eri, 8, 0, bonds, T)
    c2.set_preconditioner(net)
    out = c2.run([256] * 4, 1e-9)
    assert abs(out["energy"][-1] - e_fci) < 1e-9
    assert c2.precond_counters()["learned"] > 0
    ctx.close()
    c2.close()
    net.close()


def test_learned_preconditioner_iterations():
    """Sweeps from the same state with the diagonal and with the trained network:
    same energies; the Davidson iteration counts are what the network gains (or
    loses) against the diagonal preconditioner."""
    require_gpu()
    K, M = 12, 128
    h, eri, ctx, net, out, _, _ = _harvest_and_train(K, M, 3, 51, cap=60000, per=300)
    tensors = [ctx.get_mps(k) for k in range(K)]
    labels = [ctx.get_bond(b) for b in range(K + 1)]
    res = {}
    for name, pre in (("diag", None), ("mlp", net)):
        c = G.Context(h, eri, K, 0)
        c.set_mps(tensors, labels)
        c.set_preconditioner(pre)
        o = c.run([M] * 2, 1e-8)
        res[name] = (o["energy"], int(np.sum(o["davidson_iters"])), c.precond_counters())
        c.close()
    (e_d, it_d, _), (e_m, it_m, cnt) = res["diag"], res["mlp"]
    print(f"Davidson iterations over 2 sweeps: diagonal {it_d}, learned {it_m} "
          f"(learned applications {cnt['learned']}, fallbacks {cnt['fallbacks']})")
    assert np.allclose(e_d, e_m, atol=1e-8)
    assert cnt["learned"] > 0
    ctx.close()
    net.close()
