"""CUDA path (through the C-ABI) against the CPU oracle, element by element.

Tolerances: FP64 sigma vectors to relative 1e-11 and energies to 1e-9 Eh.
"""
import numpy as np
import pytest

from oracle import dmrg as odmrg
from oracle import fci, mps as omps
from paper_1605_02611_gb300 import synth

from gpu_util import context_with_mps, rel_err, require_gpu

pytestmark = pytest.mark.gpu


def _sigma_case(K, N, two_sz, M, k, seed):
    require_gpu()
    h, eri = synth.integrals(K, seed)
    bonds, T = synth.random_mps(K, N, two_sz, M, seed + 1)
    Na, Nb = (N + two_sz) // 2, (N - two_sz) // 2
    psi = synth.random_psi(bonds[k], bonds[k + 2], seed + 2)
    ref = omps.sigma(T, k, psi, h, eri, Na, Nb)
    ctx = context_with_mps(h, eri, N, two_sz, bonds, T)
    ctx.prepare(k)
    sig, flops = ctx.sigma(ctx.pack(psi))
    return ctx, psi, ref, sig, flops


@pytest.mark.parametrize("K,N,two_sz,M,k", [
    (4, 4, 0, 16, 1),      # full space, middle
    (5, 5, 1, 12, 0),      # left edge, odd N, S_z = 1/2
    (5, 5, 1, 12, 3),      # right edge
    (6, 6, 0, 20, 2),      # truncated, centre
    (6, 4, 2, 9, 1),       # S_z = 1, ragged small sectors
])
def test_sigma_matches_oracle_small(K, N, two_sz, M, k):
    ctx, psi, ref, sig, flops = _sigma_case(K, N, two_sz, M, k, 10 * K + k)
    assert rel_err(sig, ctx.pack(ref)) < 1e-11
    assert flops > 0


def test_sigma_matches_oracle_multi_tile():
    """Sector dimensions above the 64 x 64 tile with ragged tails (K=10, M=1000, bond 5 sectors of 100)."""
    ctx, psi, ref, sig, flops = _sigma_case(10, 10, 0, 1000, 3, 5)
    assert max(ctx.layout[:, 1].max(), ctx.layout[:, 5].max()) > 64
    assert rel_err(sig, ctx.pack(ref)) < 1e-11


def test_diag_matches_oracle():
    require_gpu()
    K, N, M, k = 5, 5, 10, 1
    h, eri = synth.integrals(K, 8)
    bonds, T = synth.random_mps(K, N, 1, M, 9)
    lab = [b.labels() for b in bonds]
    mask = omps.allowed_mask(lab[k], lab[k + 2])
    Heff = omps.heff_dense(T, k, h, eri, 3, 2, mask)
    ref = np.zeros(mask.shape)
    ref[mask] = np.diag(Heff)
    ctx = context_with_mps(h, eri, N, 1, bonds, T)
    ctx.prepare(k)
    d = ctx.diag()
    assert rel_err(d, ctx.pack(ref)) < 1e-11


def test_heff_hermitian_k12():
    """<x|H y> = <H x|y> (the paper's Hermitian-conjugate symmetry) at K=12, M=160."""
    require_gpu()
    K, N = 12, 12
    h, eri = synth.integrals(K, 12)
    bonds, T = synth.random_mps(K, N, 0, 160, 13)
    ctx = context_with_mps(h, eri, N, 0, bonds, T)
    ctx.prepare(5)
    rng = np.random.default_rng(0)
    x = rng.normal(size=ctx.nnz)
    y = rng.normal(size=ctx.nnz)
    hx, _ = ctx.sigma(x)
    hy, _ = ctx.sigma(y)
    a, b = x @ hy, hx @ y
    assert abs(a - b) < 1e-12 * (abs(a) + np.linalg.norm(hx) * np.linalg.norm(y))


def _fci_e0(h, eri, Na, Nb):
    import scipy.sparse.linalg as spla
    H = fci.hamiltonian(h, eri, Na, Nb)
    return spla.eigsh(H, k=1, which="SA", tol=1e-14)[0][0]


def test_dmrg_k8_m256_equals_fci():
    """K=8, N=8, M=256: exact MPS, so the sweep energy equals FCI (4900 determinants)."""
    require_gpu()
    cfg = synth.WORKLOADS["k8_m256_fp64"]
    h, eri = synth.integrals(8, cfg["seed"], cfg["offdiag_std"])
    bonds, T = synth.random_mps(8, 8, 0, 256, cfg["seed"])
    ctx = context_with_mps(h, eri, 8, 0, bonds, T)
    out = ctx.run([256] * 4, 1e-9)
    e0 = _fci_e0(h, eri, 4, 4)
    assert abs(out["energy"][-1] - e0) < 1e-9
    assert np.all(out["energy"] >= e0 - 1e-9)


@pytest.mark.parametrize("K,N,two_sz,M", [(6, 6, 0, 12), (7, 6, 2, 10)])
def test_dmrg_truncated_matches_oracle(K, N, two_sz, M):
    """Same start MPS and schedule: per-sweep energies of the GPU sweep and the oracle sweep."""
    require_gpu()
    h, eri = synth.integrals(K, 40 + K)
    bonds, T = synth.random_mps(K, N, two_sz, M, 41 + K)
    ref, _, _, _ = odmrg.dmrg(h, eri, N, two_sz, T, [b.labels() for b in bonds], [M] * 3)
    ctx = context_with_mps(h, eri, N, two_sz, bonds, T)
    out = ctx.run([M] * 3, 1e-10)
    assert np.abs(out["energy"] - np.array(ref)).max() < 1e-9
    for b in range(K + 1):
        assert len(ctx.get_bond(b)) <= M


def test_canonical_form_after_run():
    """After the right-to-left half sweep, sites 2..K-1 are right-orthonormal (sum_n A A^T = 1)."""
    require_gpu()
    K, N, M = 6, 6, 12
    h, eri = synth.integrals(K, 3)
    bonds, T = synth.random_mps(K, N, 0, M, 4)
    ctx = context_with_mps(h, eri, N, 0, bonds, T)
    ctx.run([M], 1e-9)
    for k in range(2, K):
        A = ctx.get_mps(k)
        A = A.reshape(A.shape[0], -1)
        assert np.allclose(A @ A.T, np.eye(A.shape[0]), atol=1e-12)


@pytest.mark.parametrize("direction", [0, 1])
def test_step_energy_matches_oracle_solve(direction):
    """gbdmrg_step on a mixed-canonical MPS: the Davidson eigenvalue equals the
    lowest eigenvalue of the projected H_eff (oracle), and the returned psi is
    its eigenvector (up to sign)."""
    require_gpu()
    K, N, M, k = 6, 6, 16, 2
    h, eri = synth.integrals(K, 61)
    bonds, T = synth.random_isometric_mps(K, N, 0, M, 62, k)
    lab = [b.labels() for b in bonds]
    mask = omps.allowed_mask(lab[k], lab[k + 2])
    psi0 = np.einsum("lnm,mor->lnor", T[k], T[k + 1])
    e_ref, x_ref = odmrg.solve(T, k, psi0, mask, h, eri, 3, 3, tol=1e-13)
    ctx = context_with_mps(h, eri, N, 0, bonds, T)
    ctx.prepare(k)
    e, dw, it, psi = ctx.step(k, direction, M, 1e-10, 300, want_psi=True)
    assert abs(e - e_ref) < 1e-9
    ref = ctx.pack(x_ref)
    assert min(np.abs(psi - ref).max(), np.abs(psi + ref).max()) < 1e-7
    assert 0 <= dw < 1e-2


def test_sigma_flops_host_matches_plan():
    require_gpu()
    import paper_1605_02611_gb300 as G
    K, N, M, k = 8, 8, 40, 3
    h, eri = synth.integrals(K, 71)
    bonds, T = synth.random_mps(K, N, 0, M, 72)
    ctx = context_with_mps(h, eri, N, 0, bonds, T)
    ctx.prepare(k)
    _, fl = ctx.sigma(np.ones(ctx.nnz))
    assert fl == G.sigma_flops_host(h, eri, N, 0, k, bonds[k].labels(), bonds[k + 2].labels())
