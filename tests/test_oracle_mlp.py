"""Pins of the learned-preconditioner reference (oracle/mlp.py) against things
fixed independently of its code: finite differences, closed-form values,
special cases and hand-computed features."""
import math

import numpy as np
import pytest

from oracle import mlp


def _params(seed, scale=0.3):
    rng = np.random.default_rng(seed)
    th = rng.normal(0.0, scale, mlp.NPARAMS)
    return th


def _batch(seed, B=7):
    rng = np.random.default_rng(seed)
    return rng.normal(size=(B, mlp.NFEAT)), rng.normal(size=B), rng.normal(size=B)


def test_layout_size():
    assert mlp.NPARAMS == 256 * 5 + 256 + 256 * 256 + 256 + 256 + 1
    th = _params(0)
    assert np.array_equal(mlp.flatten(mlp.unflatten(th)), th)


def test_gelu_closed_forms():
    # x Phi(x): Phi(1) = 0.8413447460685429, Phi(-1) = 1 - Phi(1), Phi(0) = 1/2
    assert mlp.gelu(np.array([1.0]))[0] == pytest.approx(0.8413447460685429, abs=1e-15)
    assert mlp.gelu(np.array([-1.0]))[0] == pytest.approx(-(1 - 0.8413447460685429), abs=1e-15)
    assert mlp.gelu(np.array([0.0]))[0] == 0.0
    x = np.linspace(-4, 4, 17)
    assert np.allclose(mlp.gelu(x) - mlp.gelu(-x), x, atol=1e-15)   # Phi(x) + Phi(-x) = 1
    assert mlp.gelu(np.array([40.0]))[0] == 40.0
    # derivative: phi(0) term vanishes at 0, so gelu'(0) = 1/2
    assert mlp.gelu_grad(np.array([0.0]))[0] == pytest.approx(0.5, abs=1e-15)
    h = 1e-6
    fd = (mlp.gelu(x + h) - mlp.gelu(x - h)) / (2 * h)
    assert np.allclose(mlp.gelu_grad(x), fd, atol=1e-8)


def test_gradient_matches_finite_differences():
    th = _params(1)
    F, P, T = _batch(2)
    L, g = mlp.loss_grad(th, F, P, T)
    assert L == pytest.approx(mlp.loss(th, F, P, T), rel=1e-14)
    rng = np.random.default_rng(3)
    # a few entries of every parameter group
    idx, o = [], 0
    for _, shp in mlp.SHAPES:
        sz = int(np.prod(shp))
        idx += list(o + rng.choice(sz, size=min(sz, 6), replace=False))
        o += sz
    h = 1e-5
    for i in idx:
        tp, tm = th.copy(), th.copy()
        tp[i] += h
        tm[i] -= h
        fd = (mlp.loss(tp, F, P, T) - mlp.loss(tm, F, P, T)) / (2 * h)
        assert g[i] == pytest.approx(fd, rel=1e-6, abs=1e-9), i


def test_zero_output_layer():
    """W3 = 0: g = b3 for every input, and no gradient reaches the hidden layers."""
    th = _params(4)
    p = mlp.unflatten(th)
    p["W3"][:] = 0.0
    p["b3"][:] = 0.25
    th = mlp.flatten(p)
    F, P, T = _batch(5, B=11)
    g, _ = mlp.forward(th, F)
    assert np.all(g == 0.25)
    L, grad = mlp.loss_grad(th, F, P, T)
    gp = mlp.unflatten(grad)
    for name in ("W1", "b1", "W2", "b2"):
        assert np.all(gp[name] == 0.0)
    e = 1.25 * P - T
    assert gp["b3"][0] == pytest.approx(np.mean(2 * e * P), rel=1e-14)
    assert L == pytest.approx(np.mean(e * e), rel=1e-14)


def test_features_by_hand():
    r = np.array([3.0, 4.0, 0.0, 0.0])
    d = np.array([1.0, 2.0, 3.0, 5.0])
    F = mlp.features(r, d, 1.0, [(0, 2), (2, 2)])
    # |r| = 5, sqrt(n) = 2
    assert np.allclose(F[:, 0], [1.2, 1.6, 0.0, 0.0], atol=1e-15)
    assert np.allclose(F[:, 1], np.arcsinh([0.0, 1.0, 2.0, 4.0]), atol=1e-15)
    assert np.allclose(F[:, 2], [0.0, 1 / 1.01, 2 / 4.01, 4 / 16.01], atol=1e-15)
    # block 0: rms = sqrt(12.5), times 2/5 = sqrt(2); block 1: rms 0
    assert np.allclose(F[:, 3], [math.asinh(math.sqrt(2))] * 2 + [0.0] * 2, atol=1e-15)
    assert np.allclose(F[:, 4], [math.asinh(0.5)] * 2 + [math.asinh(3.0)] * 2, atol=1e-15)


def test_pair_target_is_the_exact_correction():
    rng = np.random.default_rng(6)
    n = 50
    x = rng.normal(size=n)
    x /= np.linalg.norm(x)
    tau0 = rng.normal(size=n) * 0.1
    tau0 -= (tau0 @ x) * x                      # orthogonal to x
    psi = (x + tau0) / np.linalg.norm(x + tau0)
    r = rng.normal(size=n)
    d = rng.normal(size=n) + 3.0
    P, T = mlp.pair_values(x, r, d, -1.0, psi)
    s = math.sqrt(n) / np.linalg.norm(tau0)
    assert np.allclose(T, np.clip(tau0 * s, -100, 100), atol=1e-12)
    assert np.allclose(P, np.clip(r / (-1.0 - d) * s, -100, 100), atol=1e-12)


def test_precondition_reduces_to_diagonal():
    th = _params(7)
    p = mlp.unflatten(th)
    p["W3"][:] = 0.0
    p["b3"][:] = 0.0
    rng = np.random.default_rng(8)
    r = rng.normal(size=12)
    d = rng.normal(size=12)
    d[3] = -0.5 + 1e-12                        # near-zero denominator: clamped
    t = mlp.precondition(mlp.flatten(p), r, d, -0.5, [(0, 5), (5, 7)])
    assert np.array_equal(t, r / np.where(np.abs(-0.5 - d) < 1e-8, np.sign(-0.5 - d) * 1e-8, -0.5 - d))
    p["b3"][:] = 1.0
    t2 = mlp.precondition(mlp.flatten(p), r, d, -0.5, [(0, 5), (5, 7)])
    assert np.allclose(t2, 2 * t, rtol=1e-15)
