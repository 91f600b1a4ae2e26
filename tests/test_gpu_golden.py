"""Full-M DMRG on the GPU (FP64 path and three-slice tensor-core path with the
FP64 refinement step) against the stored exact energies of tests/golden/."""
import numpy as np
import pytest

from paper_1605_02611_gb300 import synth

from gpu_util import context_with_mps, require_gpu
from test_golden import golden

pytestmark = pytest.mark.gpu

FULL_M = {4: 16, 5: 16, 6: 64, 8: 256}


@pytest.mark.parametrize("precision", [0, 2])
@pytest.mark.parametrize("row", golden(), ids=lambda r: f"K{r[0]}")
def test_full_m_dmrg_reaches_golden_energy(row, precision):
    require_gpu()
    K, N, tsz, seed, std, e = row
    M = FULL_M[K]
    h, eri = synth.integrals(K, seed, std)
    bonds, T = synth.random_mps(K, N, tsz, M, seed + 5)
    ctx = context_with_mps(h, eri, N, tsz, bonds, T)
    out = ctx.run([M] * 4, [1e-6, 1e-8, 1e-9, 1e-9], precision=precision)
    assert abs(out["energy"][-1] - e) < 1e-9
    assert np.all(out["energy"] >= e - 1e-9)      # variational
    ctx.close()
