"""Environment (renormalised-operator) updates on the tensor cores against the FP64
updates: three BF16 slices (gbdmrg_set_env_precision(ctx, 2), FP32-level) and the
exact splitting (precision 3: every block scaled by a power of two and split into
six 7-bit integer slices, exact products and sums in the FP32 accumulators, the
levels added in two-float registers and stored in FP64).

The updates of Eqs. leftrenorm/rightrenorm (blocking, then decimation with the
new site tensor, Eq. prenormdec) build every environment up to the two-site
position in gbdmrg_prepare; H_eff.psi and <psi|H|psi> at that position then
test the environments element by element through their only use.
"""
import numpy as np
import pytest

from oracle import mps as omps
from paper_1605_02611_gb300 import synth

from gpu_util import context_with_mps, rel_err, require_gpu

pytestmark = pytest.mark.gpu


@pytest.mark.parametrize("K,N,two_sz,M,k", [
    (8, 8, 0, 60, 3),      # left environments up to bond 3, right ones down to bond 5
    (9, 9, 1, 60, 4),      # odd K, S_z = 1/2
    (10, 10, 0, 1000, 4),  # sectors of ~100 (several K steps per block)
])
def test_tc_environments_give_the_fp64_sigma(K, N, two_sz, M, k):
    require_gpu()
    seed = 900 + K
    Na, Nb = (N + two_sz) // 2, (N - two_sz) // 2
    h, eri = synth.integrals(K, seed)
    bonds, T = synth.random_isometric_mps(K, N, two_sz, M, seed + 1, k, 0.5)
    psi = synth.random_psi(bonds[k], bonds[k + 2], seed + 2)
    out = {}
    for envp in (0, 2):
        ctx = context_with_mps(h, eri, N, two_sz, bonds, T)
        ctx.set_env_precision(envp)
        ctx.prepare(k)
        out[envp] = (ctx.sigma(ctx.pack(psi))[0], ctx.expectation())
        ctx.close()
    err = rel_err(out[2][0], out[0][0])
    de = abs(out[2][1] - out[0][1])
    print(f"K={K} M={M}: sigma with tensor-core environments vs FP64 environments {err:.2e}; "
          f"<H> difference {de:.2e} Eh")
    # three BF16 slices and FP32 accumulation: FP32-level agreement, not FP64
    assert err < 1e-5
    assert de < 1e-5 * max(1.0, abs(out[0][1]))
    if K <= 9:
        ref = omps.sigma(T, k, psi, h, eri, Na, Nb)
        ctx = context_with_mps(h, eri, N, two_sz, bonds, T)
        ctx.prepare(k)
        assert rel_err(out[2][0], ctx.pack(ref)) < 1e-5
        ctx.close()


def test_tc_environment_sweeps_match_fp64():
    """K=12, M=64, six sweeps from the same start: tensor-core sigma (three slices on the
    TMA-staged work lists) and tensor-core environment updates, with the FP64 last
    step of each sweep, end within 5e-5 Eh of the FP64 sweep energy (measured 2.2e-5:
    the environments carry FP32-level errors into that last step, which is why the
    FP64 update stays the default)."""
    require_gpu()
    K, N, M = 12, 12, 64
    h, eri = synth.integrals(K, 1606)
    bonds, T = synth.random_mps(K, N, 0, M, 1607)
    e = {}
    for label, prec, envp in (("fp64", 0, 0), ("tc", 5, 2)):
        ctx = context_with_mps(h, eri, N, 0, bonds, T)
        ctx.set_env_precision(envp)
        e[label] = ctx.run([M] * 6, [1e-6, 1e-7, 1e-8, 1e-9, 1e-9, 1e-9], precision=prec)["energy"]
        ctx.close()
    print("tensor-core - fp64 sweep energies:", e["tc"] - e["fp64"])
    assert abs(e["tc"][-1] - e["fp64"][-1]) < 5e-5


@pytest.mark.parametrize("K,N,two_sz,M,k,spread", [
    (8, 8, 0, 60, 3, 0.5),
    (9, 9, 1, 60, 4, 0.5),
    (10, 10, 0, 1000, 4, 0.5),
    (12, 12, 0, 1000, 3, 4.0),   # a sector of 400 states at bond 6: contractions cut into 128-column sums
])
def test_exact_tc_environments_give_the_fp64_sigma(K, N, two_sz, M, k, spread):
    """Six 7-bit slices carry every block to ~2^-42 of its largest element: the
    environments agree with the FP64 ones to ~1e-10, far below the tensor-core sigma's
    own error and the 1e-6 Eh energy target."""
    require_gpu()
    seed = 900 + K
    h, eri = synth.integrals(K, seed)
    bonds, T = synth.random_isometric_mps(K, N, two_sz, M, seed + 1, k, spread)
    if spread > 1:
        assert max(bonds[6].dim) > 128
    psi = synth.random_psi(bonds[k], bonds[k + 2], seed + 2)
    out = {}
    for envp in (0, 3):
        ctx = context_with_mps(h, eri, N, two_sz, bonds, T)
        ctx.set_env_precision(envp)
        ctx.prepare(k)
        out[envp] = (ctx.sigma(ctx.pack(psi))[0], ctx.expectation())
        ctx.close()
    err = rel_err(out[3][0], out[0][0])
    de = abs(out[3][1] - out[0][1])
    print(f"K={K} M={M}: sigma with exact tensor-core environments vs FP64 environments {err:.2e}; "
          f"<H> difference {de:.2e} Eh")
    assert err < 1e-9
    assert de < 1e-9 * max(1.0, abs(out[0][1]))


def test_exact_tc_environment_sweeps_match_fp64():
    """K=12, M=64, six sweeps: exact tensor-core environment updates with the FP64 sigma
    reach the FP64 sweep energies within 1e-9 Eh, and with the three-slice tensor-core
    sigma within 1e-6 Eh."""
    require_gpu()
    K, N, M = 12, 12, 64
    h, eri = synth.integrals(K, 1606)
    bonds, T = synth.random_mps(K, N, 0, M, 1607)
    e = {}
    for label, prec, envp in (("fp64", 0, 0), ("fp64 exact env", 0, 3), ("tc exact env", 5, 3)):
        ctx = context_with_mps(h, eri, N, 0, bonds, T)
        ctx.set_env_precision(envp)
        e[label] = ctx.run([M] * 6, [1e-6, 1e-7, 1e-8, 1e-9, 1e-9, 1e-9], precision=prec)["energy"]
        ctx.close()
    print("exact env (fp64 sigma) - fp64:", e["fp64 exact env"] - e["fp64"])
    print("exact env (tc sigma) - fp64:", e["tc exact env"] - e["fp64"])
    assert abs(e["fp64 exact env"][-1] - e["fp64"][-1]) < 1e-9
    assert abs(e["tc exact env"][-1] - e["fp64"][-1]) < 1e-6
