// Quantum-chemistry MPO with normal and complementary operators.
//
// The MPO W[k] of Eq. (wproduct) is built from the left-right decomposition of
// Eq. (Hdecomp): at every bond each Hamiltonian term is represented by one
// bond operator ("state"), chosen as in the paper's normal/complementary
// scheme:
//   * nothing emitted yet           -> I      (left op = 1, right op carries the term)
//   * everything emitted            -> H      (left op = H^L part, right op = 1)
//   * one operator emitted          -> normal  a+_x / a_x           (right side complementary, S-type)
//   * three operators emitted       -> compl   indexed by the pending a_x / a+_x (left S-type)
//   * two emitted, two pending      -> normal pair (A = a+a+, B = a+a, aa) while the
//                                      left block has <= floor(K/2) sites, otherwise
//                                      compl pair (P, Q type on the left): the switch
//                                      of Sec. "MPO representation of quantum chemistry
//                                      Hamiltonians" (complementary side moves at K/2).
// Integral coefficients are applied at the site where a term leaves a normal
// (or I) state and enters a complementary (or H) state; every other transition
// is structural.  This is the element-wise blocking with non-zero metadata of
// Sec. "Efficient implementation of expectation values": W is stored as a list
// of non-zero (row, col, 4x4 site operator) entries.
//
// Fermion signs: Jordan-Wigner with spin-orbital order 0a,0b,1a,1b,...; local
// site basis n = n_alpha + 2 n_beta.  A term is first stably sorted by
// spin-orbital (sign of the permutation), and on each spin-orbital y the local
// factor is (product of its sigma+/-) * Z^(number of term operators on later
// spin-orbitals) -- so the MPO is a plain (bosonic) tensor product and the
// renormalised operators need no extra signs.
#pragma once
#include <array>
#include <cstdint>
#include <string>
#include <unordered_map>
#include <vector>

namespace gbdmrg {

struct FOp {            // one fermion operator on spin-orbital x
  int8_t cre;           // 1 = a+, 0 = a
  int16_t x;            // 2*site + spin
};

// Bond operator identity.  kind: 0 = I, 1 = H, 2 = normal(ops), 3 = compl(ops)
struct StateKey {
  int8_t kind = 0;
  int8_t n = 0;
  FOp ops[2] = {{0, 0}, {0, 0}};
  uint64_t pack() const;
};

struct BondState {
  StateKey key;
  int dna = 0, dnb = 0;   // quantum-number change of the LEFT operator
  int parity = 0;         // fermion parity of the left operator
};

struct WEntry {
  int row, col;           // state indices at bond k and bond k+1
  double m[16];           // 4x4 site operator, m[n*4 + n'] = <n| w |n'>
};

struct MPO {
  int K = 0;
  std::vector<std::vector<BondState>> bonds;  // K+1 bonds
  std::vector<std::vector<WEntry>> W;         // K sites
  int state_I(int b) const;                   // index of I at bond b (-1 if absent)
  int state_H(int b) const;
};

// Build from h[K*K] (symmetric) and eri[K^4] = (pq|rs) (chemists' order).
// Coefficients with |c| <= drop_tol are skipped.
MPO build_mpo(int K, const double* h, const double* eri, double drop_tol = 1e-14);

// Contract the MPO to a dense 4^K x 4^K matrix (row-major), K <= 6.  Debug/tests.
void mpo_to_dense(const MPO& mpo, std::vector<double>& out);

}  // namespace gbdmrg
