"""Learned Davidson preconditioner: plain FP64 NumPy reference.  TEST INFRASTRUCTURE ONLY.

The paper solves each two-site problem for its lowest eigenpair (Sec. "The
DMRG in renormalization group language", the solving step) without naming the
eigensolver.  The library uses Davidson's method, whose usual preconditioner
turns the residual r = H_eff x - theta x into the correction t_i = r_i /
(theta - d_i), d = diag(H_eff).  The learned preconditioner keeps that form
and multiplies each element by (1 + g(f_i)), g a small network of per-element
features with quantum-number-block context:

    delta_i = d_i - theta
    f_0 = r_i sqrt(n) / |r|                       (residual, unit RMS)
    f_1 = asinh(delta_i)                          (diagonal shift, log scale)
    f_2 = delta_i / (delta_i^2 + 0.01)            (smoothly clamped 1/delta)
    f_3 = asinh(rms_b(r) sqrt(n) / |r|)           (block residual RMS, relative)
    f_4 = asinh(mean_b(d) - theta)                (block mean of the diagonal)

where b is the QN block holding element i and n the number of elements.

Network (3 layers, GELU, hidden width 256):
    a1 = W1 f + b1, h1 = gelu(a1); a2 = W2 h1 + b2, h2 = gelu(a2); g = W3 . h2 + b3
with gelu(x) = x Phi(x) (Phi the standard normal CDF, written with erf).

Training pairs come from the method itself: for a Ritz vector x_j of Davidson
iteration j and the converged vector psi, the exact correction with unit
weight on x_j is tau = psi / (x_j . psi) - x_j.  A pair stores the features,
P = p_i s and T = tau_i s with p_i = r_i / (theta - d_i) (denominator clamped to
|.| >= 1e-8) and s = sqrt(n) / |tau|; both are clipped to [-100, 100].  The
loss is the mean of ((1 + g) P - T)^2.

Pinned in tests/test_oracle_mlp.py: central finite differences of the loss
against the analytic gradient, the W3 = 0 special case (g = b3 exactly, zero
gradient for the hidden layers), gelu against its closed form values and
derivative, features against values written out by hand, and the target
against a vector constructed to have a known correction.
"""
from __future__ import annotations

import math

import numpy as np

HIDDEN = 256
NFEAT = 5
CLIP = 100.0
DEN_EPS = 1e-8

# flat parameter layout, shared by the library's C-ABI (order and shapes)
SHAPES = [("W1", (HIDDEN, NFEAT)), ("b1", (HIDDEN,)), ("W2", (HIDDEN, HIDDEN)), ("b2", (HIDDEN,)),
          ("W3", (HIDDEN,)), ("b3", (1,))]
NPARAMS = sum(int(np.prod(s)) for _, s in SHAPES)


def unflatten(theta):
    out, o = {}, 0
    for name, shp in SHAPES:
        sz = int(np.prod(shp))
        out[name] = np.asarray(theta[o:o + sz], dtype=np.float64).reshape(shp)
        o += sz
    return out


def flatten(p):
    return np.concatenate([np.asarray(p[name], dtype=np.float64).ravel() for name, _ in SHAPES])


_erf = np.vectorize(math.erf, otypes=[np.float64])


def gelu(x):
    return 0.5 * x * (1.0 + _erf(x / math.sqrt(2.0)))


def gelu_grad(x):
    # d/dx [x Phi(x)] = Phi(x) + x phi(x)
    return 0.5 * (1.0 + _erf(x / math.sqrt(2.0))) + x * np.exp(-0.5 * x * x) / math.sqrt(2.0 * math.pi)


def forward(theta, F):
    """g for every row of F (n x 5); also returns the intermediates."""
    p = unflatten(theta)
    a1 = F @ p["W1"].T + p["b1"]
    h1 = gelu(a1)
    a2 = h1 @ p["W2"].T + p["b2"]
    h2 = gelu(a2)
    g = h2 @ p["W3"] + p["b3"][0]
    return g, (a1, h1, a2, h2)


def loss(theta, F, P, T):
    g, _ = forward(theta, F)
    return float(np.mean(((1.0 + g) * P - T) ** 2))


def loss_grad(theta, F, P, T):
    """Loss and its gradient with respect to the flat parameters (backpropagation)."""
    p = unflatten(theta)
    g, (a1, h1, a2, h2) = forward(theta, F)
    B = F.shape[0]
    e = (1.0 + g) * P - T
    L = float(np.mean(e * e))
    dg = 2.0 * e * P / B
    grads = {"W3": h2.T @ dg, "b3": np.array([dg.sum()])}
    da2 = np.outer(dg, p["W3"]) * gelu_grad(a2)
    grads["W2"] = da2.T @ h1
    grads["b2"] = da2.sum(axis=0)
    da1 = (da2 @ p["W2"]) * gelu_grad(a1)
    grads["W1"] = da1.T @ F
    grads["b1"] = da1.sum(axis=0)
    return L, flatten(grads)


def features(r, d, theta, blocks):
    """Per-element features; blocks = list of (offset, size) covering 0..n-1."""
    r = np.asarray(r, dtype=np.float64)
    d = np.asarray(d, dtype=np.float64)
    n = r.size
    rn = float(np.linalg.norm(r))
    F = np.zeros((n, NFEAT))
    delta = d - theta
    F[:, 0] = r * math.sqrt(n) / rn
    F[:, 1] = np.arcsinh(delta)
    F[:, 2] = delta / (delta * delta + 0.01)
    for off, sz in blocks:
        sl = slice(off, off + sz)
        rms = math.sqrt(float(np.sum(r[sl] ** 2)) / sz)
        F[sl, 3] = math.asinh(rms * math.sqrt(n) / rn)
        F[sl, 4] = math.asinh(float(np.mean(d[sl])) - theta)
    return F


def diag_correction(r, d, theta):
    """The diagonal (Davidson) correction p_i = r_i / (theta - d_i), |denominator| >= 1e-8."""
    den = theta - np.asarray(d, dtype=np.float64)
    den = np.where(np.abs(den) < DEN_EPS, np.where(den < 0, -DEN_EPS, DEN_EPS), den)
    return np.asarray(r, dtype=np.float64) / den


def pair_values(x, r, d, theta, psi):
    """(P, T) for every element: diagonal correction and exact correction, both
    scaled by sqrt(n)/|tau| and clipped."""
    x = np.asarray(x, dtype=np.float64)
    psi = np.asarray(psi, dtype=np.float64)
    c = float(x @ psi)
    tau = psi / c - x
    s = math.sqrt(x.size) / float(np.linalg.norm(tau))
    P = np.clip(diag_correction(r, d, theta) * s, -CLIP, CLIP)
    T = np.clip(tau * s, -CLIP, CLIP)
    return P, T


def precondition(theta_params, r, d, theta, blocks):
    """The learned correction t = (1 + g(f)) p."""
    F = features(r, d, theta, blocks)
    g, _ = forward(theta_params, F)
    return (1.0 + g) * diag_correction(r, d, theta)
