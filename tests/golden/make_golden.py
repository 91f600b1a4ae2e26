"""Write the stored reference values of tests/golden/ (calls only the oracle).

    python tests/golden/make_golden.py

fci_energies.txt: the exact ground-state energy (full CI in the determinant
space of fixed N_alpha, N_beta; the oracle's Slater-Condon / direct-CI
Hamiltonian, diagonalised densely) of the seeded synthetic Hamiltonians used by
the tests and the K=8 workload.  Columns: K N two_sz seed offdiag_std E0.
"""
import os
import sys

HERE = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, os.path.dirname(os.path.dirname(HERE)))

import numpy as np  # noqa: E402

from oracle import fci  # noqa: E402
from paper_1605_02611_gb300 import synth  # noqa: E402

CASES = [(4, 4, 0, 11, 0.1), (5, 5, 1, 7, 0.1), (6, 6, 0, 91, 0.1), (8, 8, 0, synth.BASE_SEED, 0.1)]


def main():
    lines = ["# K N two_sz seed offdiag_std E0 (exact, oracle full CI)"]
    for K, N, tsz, seed, std in CASES:
        h, eri = synth.integrals(K, seed, std)
        na, nb = (N + tsz) // 2, (N - tsz) // 2
        w, _ = fci.ground_state(h, eri, na, nb)
        lines.append(f"{K} {N} {tsz} {seed} {std} {w[0]:.15f}")
    with open(os.path.join(HERE, "fci_energies.txt"), "w") as f:
        f.write("\n".join(lines) + "\n")


if __name__ == "__main__":
    main()
