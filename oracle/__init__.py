"""CPU oracle for the two-site DMRG hot path.  TEST INFRASTRUCTURE ONLY.

Only ``tests/``, ``__graft_entry__.smoke()`` and ``bench.py`` (its CPU-baseline
leg and ``--impl reference``) may import or run anything in this package.  The
CUDA library never calls into it and shares no code with it.

What it computes, and from which definition:

* ``fock``  -- the Hamiltonian of Eq. (longrangeh) as an explicit matrix on the
  whole Fock space, built from Jordan-Wigner creation/annihilation matrices
  (second quantisation written out; K <= 5 spatial orbitals).
* ``fci``   -- the same Hamiltonian on the determinant space of fixed
  (N_alpha, N_beta), applied by the string-driven direct-CI algorithm
  (Knowles & Handy, Chem. Phys. Lett. 111, 315 (1984)) and, for small cases,
  as an explicit matrix from the Slater-Condon rules.
* ``mps``   -- the renormalised left/right bases of Eqs. (lbasis)/(rbasis) as
  explicit vectors, and the two-site effective Hamiltonian as the projection
  of H onto the product basis |l n_k n_k+1 r> (Eq. MPSCform, two-site form):
  sigma = P^T H P psi.  This is the plain definition of H_eff.psi, independent
  of any MPO.
* ``dmrg``  -- the two-site sweep of Sec. "The DMRG in renormalization group
  language": blocking, solving (lowest eigenpair of the projected H_eff),
  decimation (SVD truncation to M states).

Parity pins live in ``tests/test_oracle_*.py``: closed forms (Hubbard dimer,
non-interacting spectra, closed-shell determinant energy), brute force on the
Fock space, Hermiticity, conservation laws, and DMRG = FCI at full M.
"""
