"""Stored exact energies (tests/golden/fci_energies.txt, written by
tests/golden/make_golden.py from the oracle's full CI) against independent
routes: the Fock-space Hamiltonian for K <= 5 and a sparse Lanczos solve."""
import os

import numpy as np
import pytest
import scipy.sparse.linalg as spla

from oracle import fci, fock
from paper_1605_02611_gb300 import synth

HERE = os.path.dirname(os.path.abspath(__file__))


def golden():
    rows = []
    with open(os.path.join(HERE, "golden", "fci_energies.txt")) as f:
        for line in f:
            if line.startswith("#") or not line.strip():
                continue
            K, N, tsz, seed, std, e = line.split()
            rows.append((int(K), int(N), int(tsz), int(seed), float(std), float(e)))
    return rows


@pytest.mark.parametrize("row", golden(), ids=lambda r: f"K{r[0]}")
def test_golden_energy(row):
    K, N, tsz, seed, std, e = row
    h, eri = synth.integrals(K, seed, std)
    na, nb = (N + tsz) // 2, (N - tsz) // 2
    if K <= 5:
        # second quantisation written out on the whole Fock space, restricted to the sector
        H = fock.hamiltonian(h, eri)
        sel = fock.sector_indices(K, na, nb)
        w = np.linalg.eigvalsh(H[sel][:, sel].toarray())[0]
    else:
        w = spla.eigsh(fci.hamiltonian(h, eri, na, nb), k=1, which="SA", tol=1e-14)[0][0]
    assert abs(w - e) < 1e-10
