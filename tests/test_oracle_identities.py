"""The paper's operator identities checked on the Fock space (CPU).

Spin-orbital form with spin suppressed, as in Eq. (longrangeh): t_pq and
v_pqrs = <pq|sr> over the 2K spin-orbitals of ``oracle.fock`` (order 0a, 0b,
1a, ...), with v_pqrs = (ps|qr) when the spins of p, s and of q, r agree.
These pin the Hamiltonian convention of the oracle to the decomposition the
MPO is built from (Eq. Hdecomp and the blocking rule Eq. prenormrule).
"""
import itertools

import numpy as np
import pytest

from oracle import fock
from paper_1605_02611_gb300 import synth

K = 3
N_SO = 2 * K


@pytest.fixture(scope="module")
def system():
    h, eri = synth.integrals(K, 5)
    t = np.zeros((N_SO, N_SO))
    v = np.zeros((N_SO,) * 4)
    for x, y in itertools.product(range(N_SO), repeat=2):
        if x % 2 == y % 2:
            t[x, y] = h[x // 2, y // 2]
    for p, q, r, s in itertools.product(range(N_SO), repeat=4):
        if p % 2 == s % 2 and q % 2 == r % 2:
            v[p, q, r, s] = eri[p // 2, s // 2, q // 2, r // 2]
    cd, c = fock.operators(K)
    cd = [m.toarray() for m in cd]
    c = [m.toarray() for m in c]
    H = fock.hamiltonian(h, eri).toarray()
    w = v - v.transpose(1, 0, 2, 3)   # w_pqrs = v_pqrs - v_qprs
    return dict(t=t, v=v, w=w, cd=cd, c=c, H=H)


def _block_h(s, B):
    """H restricted to the spin-orbitals B (Eqs. lefth / righth)."""
    t, v, cd, c = s["t"], s["v"], s["cd"], s["c"]
    m = np.zeros_like(s["H"])
    for p, q in itertools.product(B, repeat=2):
        m += t[p, q] * (cd[p] @ c[q])
    for p, q, r, u in itertools.product(B, repeat=4):
        if v[p, q, r, u]:
            m += 0.5 * v[p, q, r, u] * (cd[p] @ cd[q] @ c[r] @ c[u])
    return m


def test_longrangeh_in_spin_orbitals_is_the_oracle_h(system):
    """Eq. (longrangeh) written over spin-orbitals with v_pqrs = <pq|sr> is the oracle's H."""
    assert np.abs(_block_h(system, range(N_SO)) - system["H"]).max() < 1e-12


def test_integral_identities(system):
    """v_pqrs = v_qpsr (Eq. longrangeh); w_pqrs = v_pqrs - v_qprs = v_pqrs - v_pqsr and
    x_pqrs = v_pqrs - v_qprs - v_pqsr + v_qpsr = 2 w_pqrs (Eq. norm_complementary)."""
    v, w = system["v"], system["w"]
    assert np.abs(v - v.transpose(1, 0, 3, 2)).max() < 1e-15
    assert np.abs(w - (v - v.transpose(0, 1, 3, 2))).max() < 1e-15
    x = v - v.transpose(1, 0, 2, 3) - v.transpose(0, 1, 3, 2) + v.transpose(1, 0, 3, 2)
    assert np.abs(x - 2 * w).max() < 1e-15
    assert np.abs(w).max() > 1e-3   # not vacuous


@pytest.mark.parametrize("k", range(1, N_SO))
def test_hdecomp_as_printed_is_exact(system, k):
    """Eq. Hdecomp with its printed prefactors (1/2 on the S, A-P and B-Q sums, P built
    from v, Q from w, S from t and w) equals H at every cut of the spin-orbital chain."""
    s = system
    t, v, w, cd, c = s["t"], s["v"], s["w"], s["cd"], s["c"]
    L, R = range(k), range(k, N_SO)

    def S(p, B):
        m = sum(t[p, q] * c[q] for q in B)
        for q, r, u in itertools.product(B, repeat=3):
            if w[p, q, r, u]:
                m = m + w[p, q, r, u] * (cd[q] @ c[r] @ c[u])
        return m

    def P(p, q):
        return sum(v[p, q, r, u] * (c[r] @ c[u]) for r, u in itertools.product(R, repeat=2))

    def Q(p, q):
        return sum(w[p, r, q, u] * (cd[r] @ c[u]) for r, u in itertools.product(R, repeat=2))

    def hc(m):
        return m + m.T

    Hd = _block_h(s, L) + _block_h(s, R)
    Hd = Hd + 0.5 * (hc(sum(cd[p] @ S(p, R) for p in L)) + hc(sum(cd[p] @ S(p, L) for p in R)))
    Hd = Hd + 0.5 * hc(sum((cd[p] @ cd[q]) @ P(p, q) for p in L for q in L))
    Hd = Hd - 0.5 * hc(sum((cd[p] @ c[q]) @ Q(p, q) for p in L for q in L))
    assert np.abs(Hd - s["H"]).max() < 1e-12


def test_prenormrule_cross_term_uses_w(system):
    """Eq. prenormrule: P^{R_k}_pq = P^{R_k+1}_pq + P^k_pq + sum_{s in R_k+1} w_pqks a_k a_s
    (P^k_pq = 0 for a single spin-orbital) at every cut; the same rule with v_pqks in the
    cross term, as the text beside Eq. pwform writes [A_0], does not hold."""
    s = system
    v, w, c = s["v"], s["w"], s["c"]
    bad = 0.0
    for k in range(1, N_SO - 1):
        Rk, Rk1 = range(k, N_SO), range(k + 1, N_SO)
        for p, q in itertools.product(range(k), repeat=2):
            full = sum(v[p, q, r, u] * (c[r] @ c[u]) for r, u in itertools.product(Rk, repeat=2))
            inner = sum(v[p, q, r, u] * (c[r] @ c[u]) for r, u in itertools.product(Rk1, repeat=2))
            with_w = inner + sum(w[p, q, k, u] * (c[k] @ c[u]) for u in Rk1)
            with_v = inner + sum(v[p, q, k, u] * (c[k] @ c[u]) for u in Rk1)
            assert np.abs(with_w - full).max() < 1e-13, (k, p, q)
            bad = max(bad, np.abs(with_v - full).max())
    assert bad > 1e-3


def test_unique_two_electron_integrals(system):
    """Appendix form of the two-body part: (1/2) sum v_pqrs a+_p a+_q a_r a_s equals
    sum g_pqrs a+_p a+_q a_r a_s with g_pqrs = w_pqrs for p < q, r < s and 0 otherwise."""
    s = system
    v, w, cd, c = s["v"], s["w"], s["cd"], s["c"]
    h2 = np.zeros_like(s["H"])
    g2 = np.zeros_like(s["H"])
    for p, q, r, u in itertools.product(range(N_SO), repeat=4):
        op = None
        if v[p, q, r, u]:
            op = cd[p] @ cd[q] @ c[r] @ c[u]
            h2 += 0.5 * v[p, q, r, u] * op
        if p < q and r < u and w[p, q, r, u]:
            g2 += w[p, q, r, u] * (op if op is not None else cd[p] @ cd[q] @ c[r] @ c[u])
    assert np.abs(h2).max() > 1e-3
    assert np.abs(h2 - g2).max() < 1e-12
