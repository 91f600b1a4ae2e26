"""Library MPO builder (host code, no GPU) against the brute-force Fock-space oracle."""
import os
import subprocess
import sys

import numpy as np
import pytest

import paper_1605_02611_gb300 as G
from oracle import fock
from paper_1605_02611_gb300 import synth


@pytest.fixture(scope="module")
def lib():
    try:
        return G.load()
    except RuntimeError as e:
        pytest.skip(str(e))


@pytest.mark.parametrize("K", [1, 2, 3, 4])
def test_mpo_equals_fock_hamiltonian(lib, K):
    """W[1]...W[K] (Eq. wproduct) reproduces H of Eq. (longrangeh) exactly."""
    h, eri = synth.integrals(K, 300 + K)
    dims, D = G.mpo_build_host(h, eri, K, K % 2, dense=True)
    H = fock.hamiltonian(h, eri).toarray()
    assert np.abs(D - H).max() < 1e-12 * max(1.0, np.abs(H).max())


def test_mpo_hubbard_sparse_integrals(lib):
    h, eri = synth.hubbard_integrals(4, 1.0, 3.0)
    dims, D = G.mpo_build_host(h, eri, 4, 0, dense=True)
    H = fock.hamiltonian(h, eri).toarray()
    assert np.abs(D - H).max() < 1e-12
    # nearest-neighbour hopping + on-site U: bond dimension stays O(1)
    assert dims.max() <= 6


@pytest.mark.parametrize("K", [5, 8, 13])
def test_bond_dimension_profile(lib, K):
    """Dense integrals: D(b) = 2 + 4K + 2n^2 - n with n = 2 min(b, K-b) spin-orbitals
    on the shorter side (normal/complementary split with the switch at K/2)."""
    h, eri = synth.integrals(K, 2)
    dims, _ = G.mpo_build_host(h, eri, K, K % 2)
    assert dims[0] == 1 and dims[K] == 1
    for b in range(1, K):
        n = 2 * min(b, K - b) if b <= K // 2 else 2 * (K - b)
        assert dims[b] == 2 + 4 * K + 2 * n * n - n, (b, dims[b])


def test_invalid_problems_rejected(lib):
    h, eri = synth.integrals(3, 1)
    with pytest.raises(G.GbdmrgError):
        G.mpo_build_host(h, eri, 3, 0)          # parity of N and 2Sz differ
    bad = h.copy()
    bad[0, 1] += 1e-3
    with pytest.raises(G.GbdmrgError):
        G.mpo_build_host(bad, eri, 2, 0)        # h1 not symmetric
    e2 = eri.copy()
    e2[0, 1, 2, 2] += 1e-3
    with pytest.raises(G.GbdmrgError):
        G.mpo_build_host(h, e2, 2, 0)           # eri not 8-fold symmetric
    nan = h.copy()
    nan[1, 1] = np.nan
    with pytest.raises(G.GbdmrgError):
        G.mpo_build_host(nan, eri, 2, 0)


def test_header_symbols_exported(lib):
    """Every function declared in include/gbdmrg.h is exported by the library."""
    import re
    hdr = open(os.path.join(os.path.dirname(__file__), "..", "include", "gbdmrg.h")).read()
    names = set(re.findall(r"\b(gbdmrg_[a-z_]+)\s*\(", hdr))
    assert names, "no declarations found"
    for n in names:
        assert hasattr(lib, n), n
    assert names <= set(G.SIGNATURES), names - set(G.SIGNATURES)


def test_plan_knobs_reject_bad_arguments(lib):
    """The plan knobs and the autotuner reject null contexts and empty lists on the
    host, before any device work."""
    import ctypes as C
    EINVAL = 1
    assert lib.gbdmrg_set_split(None, 4.0) == EINVAL
    assert lib.gbdmrg_get_plan_params(None, None, None) == EINVAL
    none = (C.c_void_p * 1)(None)
    assert lib.gbdmrg_autotune(0, none, 3, None, 0, None, 0, None, None, None) == EINVAL
    assert lib.gbdmrg_autotune(1, none, 3, None, 0, None, 0, None, None, None) == EINVAL
    assert lib.gbdmrg_autotune(1, None, 3, None, 0, None, 0, None, None, None) == EINVAL
    assert lib.gbdmrg_set_stage1_stacked(None, 1) == EINVAL
    assert lib.gbdmrg_set_tc_combos(None, 1, 0) == EINVAL


def test_context_without_gpu_fails_loudly(lib):
    """No CPU fallback: without a CUDA device creating a context is an error."""
    torch = pytest.importorskip("torch")
    if torch.cuda.is_available():
        pytest.skip("a GPU is present")
    h, eri = synth.integrals(4, 1)
    with pytest.raises(G.GbdmrgError):
        G.Context(h, eri, 4, 0)


def test_missing_library_is_an_error(tmp_path):
    root = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
    code = ("import paper_1605_02611_gb300 as G\n"
            f"G.load({str(tmp_path / 'libgbdmrg.so')!r})\n")
    p = subprocess.run([sys.executable, "-c", code], cwd=root, capture_output=True, text=True, timeout=120)
    assert p.returncode != 0 and "missing" in p.stderr
