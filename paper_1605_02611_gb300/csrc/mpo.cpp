// MPO builder: see mpo.hpp for the construction and its correspondence to
// Eqs. (Hdecomp), (renormrule), (prenormrule) of the paper.
#include "mpo.hpp"

#include <algorithm>
#include <thread>
#include <mutex>
#include <exception>
#include <atomic>
#include <cmath>
#include <map>
#include <stdexcept>
#include <unordered_map>
#include <utility>
#include <vector>

namespace gbdmrg {

uint64_t StateKey::pack() const {
  uint64_t v = (uint64_t)kind | ((uint64_t)n << 2);
  for (int i = 0; i < n; ++i)
    v |= (uint64_t)((uint64_t)ops[i].cre | ((uint64_t)ops[i].x << 1)) << (4 + 13 * i);
  return v;
}

static StateKey unpack_key(uint64_t v) {
  StateKey k;
  k.kind = v & 3;
  k.n = (v >> 2) & 3;
  for (int i = 0; i < k.n; ++i) {
    uint64_t o = (v >> (4 + 13 * i)) & 0x1fff;
    k.ops[i].cre = o & 1;
    k.ops[i].x = (int16_t)(o >> 1);
  }
  return k;
}

int MPO::state_I(int b) const {
  for (size_t i = 0; i < bonds[b].size(); ++i)
    if (bonds[b][i].key.kind == 0) return (int)i;
  return -1;
}
int MPO::state_H(int b) const {
  for (size_t i = 0; i < bonds[b].size(); ++i)
    if (bonds[b][i].key.kind == 1) return (int)i;
  return -1;
}

namespace {

struct Term {
  int n;
  FOp o[4];
};

inline uint64_t term_pack(const FOp* o, int n) {
  uint64_t v = (uint64_t)n;
  for (int i = 0; i < n; ++i)
    v |= (uint64_t)((uint64_t)o[i].cre | ((uint64_t)o[i].x << 1)) << (3 + 13 * i);
  return v;
}

inline void term_unpack(uint64_t v, Term& t) {
  t.n = v & 7;
  for (int i = 0; i < t.n; ++i) {
    uint64_t o = (v >> (3 + 13 * i)) & 0x1fff;
    t.o[i].cre = o & 1;
    t.o[i].x = (int16_t)(o >> 1);
  }
}

// stable sort by spin-orbital, returns permutation sign (swaps of distinct x only)
inline int stable_sort_sign(FOp* o, int n) {
  int sign = 1;
  for (int i = 1; i < n; ++i) {
    FOp cur = o[i];
    int j = i - 1;
    while (j >= 0 && o[j].x > cur.x) {
      o[j + 1] = o[j];
      sign = -sign;
      --j;
    }
    o[j + 1] = cur;
  }
  return sign;
}

// 2x2 single spin-orbital matrices, index [n][n']
struct M2 {
  double a[2][2];
};
inline M2 m2_id() { return {{{1, 0}, {0, 1}}}; }
inline M2 m2_mul(const M2& x, const M2& y) {
  M2 r{};
  for (int i = 0; i < 2; ++i)
    for (int j = 0; j < 2; ++j) r.a[i][j] = x.a[i][0] * y.a[0][j] + x.a[i][1] * y.a[1][j];
  return r;
}
inline M2 m2_sigma(int cre) {
  M2 r{};
  if (cre) r.a[1][0] = 1.0; else r.a[0][1] = 1.0;
  return r;
}
inline M2 m2_z() { return {{{1, 0}, {0, -1}}}; }

// Local 4x4 operator on site s for the term operators located there (sorted,
// given in order) with 'pend' operators of the term on later sites.
void local_op(const FOp* ops, int nops, int site, int pend, double* m) {
  M2 la = m2_id(), lb = m2_id();
  int nb_ops = 0;
  for (int i = 0; i < nops; ++i)
    if (ops[i].x == 2 * site + 1) ++nb_ops;
  for (int i = 0; i < nops; ++i) {
    if (ops[i].x == 2 * site) la = m2_mul(la, m2_sigma(ops[i].cre));
    else lb = m2_mul(lb, m2_sigma(ops[i].cre));
  }
  if ((nb_ops + pend) & 1) la = m2_mul(la, m2_z());
  if (pend & 1) lb = m2_mul(lb, m2_z());
  for (int n = 0; n < 4; ++n)
    for (int np = 0; np < 4; ++np)
      m[n * 4 + np] = la.a[n & 1][np & 1] * lb.a[n >> 1][np >> 1];
}

struct EntryAcc {
  double m[16];
  bool structural;
};

// Open-addressing hash table with 64-bit keys (stored as key + 1, 0 = empty),
// linear probing, values in a dense vector in insertion order.  Much lighter
// than node-based maps for the tens of millions of insertions of a K=40 build.
template <class V>
class FlatMap {
 public:
  explicit FlatMap(size_t expect = 16) { rehash(capacity_for(expect)); }
  // value of key k, default-constructed on first use
  V& operator[](uint64_t k) {
    if (2 * (vals_.size() + 1) > slots_.size()) rehash(2 * slots_.size());
    size_t i = mix(k) & mask_;
    for (;;) {
      const uint64_t s = keys_[i];
      if (s == 0) {
        keys_[i] = k + 1;
        slots_[i] = (uint32_t)vals_.size();
        vals_.emplace_back();
        order_.push_back(k);
        return vals_.back();
      }
      if (s == k + 1) return vals_[slots_[i]];
      i = (i + 1) & mask_;
    }
  }
  const V* find(uint64_t k) const {
    size_t i = mix(k) & mask_;
    for (;;) {
      const uint64_t s = keys_[i];
      if (s == 0) return nullptr;
      if (s == k + 1) return &vals_[slots_[i]];
      i = (i + 1) & mask_;
    }
  }
  size_t size() const { return vals_.size(); }
  uint64_t key(size_t j) const { return order_[j]; }
  const V& value(size_t j) const { return vals_[j]; }
  V& value(size_t j) { return vals_[j]; }

 private:
  // finaliser of MurmurHash3 (Appleby): spreads the bits of packed keys
  static uint64_t mix(uint64_t x) {
    x ^= x >> 33;
    x *= 0xff51afd7ed558ccdULL;
    x ^= x >> 33;
    x *= 0xc4ceb9fe1a85ec53ULL;
    x ^= x >> 33;
    return x;
  }
  static size_t capacity_for(size_t n) {
    size_t c = 16;
    while (c < 2 * n) c <<= 1;
    return c;
  }
  void rehash(size_t cap) {
    keys_.assign(cap, 0);
    slots_.assign(cap, 0);
    mask_ = cap - 1;
    for (size_t j = 0; j < order_.size(); ++j) {
      size_t i = mix(order_[j]) & mask_;
      while (keys_[i] != 0) i = (i + 1) & mask_;
      keys_[i] = order_[j] + 1;
      slots_[i] = (uint32_t)j;
    }
  }
  std::vector<uint64_t> keys_;
  std::vector<uint32_t> slots_;
  std::vector<V> vals_;
  std::vector<uint64_t> order_;
  size_t mask_ = 0;
};

// run f(0..n-1) on n host threads (the calling thread takes 0); the first
// exception thrown by any of them is rethrown
template <class F>
void run_parallel(int n, F&& f) {
  std::exception_ptr fail;
  std::mutex mu;
  auto body = [&](int w) {
    try {
      f(w);
    } catch (...) {
      std::lock_guard<std::mutex> lk(mu);
      if (!fail) fail = std::current_exception();
    }
  };
  std::vector<std::thread> pool;
  for (int w = 1; w < n; ++w) pool.emplace_back(body, w);
  body(0);
  for (auto& th : pool) th.join();
  if (fail) std::rethrow_exception(fail);
}

}  // namespace

MPO build_mpo(int K, const double* h, const double* eri, double drop_tol) {
  if (K < 1 || K > 200) throw std::runtime_error("K out of range");
  // 1) unique sorted terms with accumulated coefficients
  FlatMap<double> terms((size_t)K * K * K * K);
  auto add = [&](FOp* o, int n, double c) {
    // zero operator: repeated creator or annihilator on the same spin-orbital
    for (int i = 0; i < n; ++i)
      for (int j = i + 1; j < n; ++j)
        if (o[i].cre == o[j].cre && o[i].x == o[j].x) return;
    int sg = stable_sort_sign(o, n);
    terms[term_pack(o, n)] += sg * c;
  };
  for (int p = 0; p < K; ++p)
    for (int q = 0; q < K; ++q) {
      double c = h[p * K + q];
      if (std::fabs(c) <= drop_tol) continue;
      for (int s = 0; s < 2; ++s) {
        FOp o[2] = {{1, (int16_t)(2 * p + s)}, {0, (int16_t)(2 * q + s)}};
        add(o, 2, c);
      }
    }
  for (int p = 0; p < K; ++p)
    for (int q = 0; q < K; ++q)
      for (int r = 0; r < K; ++r)
        for (int s_ = 0; s_ < K; ++s_) {
          double g = eri[((size_t)(p * K + q) * K + r) * K + s_];
          if (std::fabs(g) <= drop_tol) continue;
          for (int s = 0; s < 2; ++s)
            for (int t = 0; t < 2; ++t) {
              // 1/2 (pq|rs) a+_{ps} a+_{rt} a_{st} a_{qs}
              FOp o[4] = {{1, (int16_t)(2 * p + s)}, {1, (int16_t)(2 * r + t)},
                          {0, (int16_t)(2 * s_ + t)}, {0, (int16_t)(2 * q + s)}};
              add(o, 4, 0.5 * g);
            }
        }

  const int half = K / 2;
  // 2) route every term.  Sites are divided among host threads; every thread
  // scans all terms and records the transitions at its own sites, so each site's
  // entries accumulate in the same (term) order whatever the number of threads.
  std::vector<FlatMap<EntryAcc>> acc(K);  // per site: (from state, to state) -> W entry
  auto state_at = [&](const Term& t, int b) -> StateKey {
    int e = 0;
    for (int i = 0; i < t.n; ++i)
      if (t.o[i].x / 2 < b) ++e;
    StateKey k;
    if (e == 0) { k.kind = 0; return k; }
    if (e == t.n) { k.kind = 1; return k; }
    if (t.n == 2 || e == 1) {
      k.kind = 2; k.n = 1; k.ops[0] = t.o[0];
      if (t.n == 2 && e != 1) throw std::logic_error("bad state");
      return k;
    }
    if (e == 3) { k.kind = 3; k.n = 1; k.ops[0] = t.o[3]; return k; }
    // e == 2 of 4
    if (b <= half) { k.kind = 2; k.n = 2; k.ops[0] = t.o[0]; k.ops[1] = t.o[1]; }
    else { k.kind = 3; k.n = 2; k.ops[0] = t.o[2]; k.ops[1] = t.o[3]; }
    return k;
  };
  const unsigned hw = std::max(1u, std::thread::hardware_concurrency());
  const int nw = (int)std::min<unsigned>(std::min(hw, 16u), (unsigned)K);
  // owner of each site: the switch site K/2 sees a transition of most terms, so it
  // gets a worker of its own; the others are dealt out round-robin
  std::vector<int> owner(K);
  {
    int w = nw > 1 ? 1 : 0;
    for (int s = 0; s < K; ++s) {
      if (s == half && nw > 1) { owner[s] = 0; continue; }
      owner[s] = w;
      w = nw > 1 ? 1 + (w % (nw - 1)) : 0;
    }
  }
  std::vector<FlatMap<std::pair<int, int>>> alive_w(nw);  // key -> [first bond, last bond]
  auto route = [&](int w) {
    FlatMap<std::pair<int, int>>& alive = alive_w[w];
    auto note_alive = [&](uint64_t key, int b) {
      const size_t before = alive.size();
      std::pair<int, int>& r = alive[key];
      if (alive.size() != before) r = std::make_pair(b, b);
      else { r.first = std::min(r.first, b); r.second = std::max(r.second, b); }
    };
    Term t;
    for (size_t ti = 0; ti < terms.size(); ++ti) {
      double c = terms.value(ti);
      if (std::fabs(c) <= drop_tol) continue;
      term_unpack(terms.key(ti), t);
      // the state only changes at sites carrying operators of the term and at the
      // switch site K/2, so only those sites are visited
      int ev[5], nev = 0;
      for (int i = 0; i < t.n; ++i) ev[nev++] = t.o[i].x / 2;
      if (half < K) ev[nev++] = half;
      std::sort(ev, ev + nev);
      nev = (int)(std::unique(ev, ev + nev) - ev);
      if (w == 0) {
        note_alive(state_at(t, 0).pack(), 0);
        note_alive(state_at(t, K).pack(), K);
      }
      for (int e = 0; e < nev; ++e) {
        const int s = ev[e];
        if (owner[s] != w) continue;
        StateKey prev = state_at(t, s), nxt = state_at(t, s + 1);
        uint64_t pk = prev.pack(), nk = nxt.pack();
        FOp site_ops[4];
        int ns = 0, later = 0;
        for (int i = 0; i < t.n; ++i) {
          int si = t.o[i].x / 2;
          if (si == s) site_ops[ns++] = t.o[i];
          else if (si > s) ++later;
        }
        if (nk == pk && ns == 0) continue;
        note_alive(pk, s);
        note_alive(nk, s + 1);
        bool coef = (prev.kind == 0 || prev.kind == 2) && (nxt.kind == 1 || nxt.kind == 3);
        double m[16];
        local_op(site_ops, ns, s, later, m);
        // state keys use 30 bits: the pair packs into one 64-bit key
        const size_t before = acc[s].size();
        EntryAcc& slot = acc[s][(pk << 30) | nk];
        if (acc[s].size() != before) {
          for (int i = 0; i < 16; ++i) slot.m[i] = 0.0;
          slot.structural = false;
        }
        if (coef) {
          for (int i = 0; i < 16; ++i) slot.m[i] += c * m[i];
          slot.structural = false;
        } else if (!slot.structural) {
          for (int i = 0; i < 16; ++i) slot.m[i] = m[i];
          slot.structural = true;
        }
      }
    }
  };
  run_parallel(nw, route);
  FlatMap<std::pair<int, int>> alive;
  for (int w = 0; w < nw; ++w)
    for (size_t j = 0; j < alive_w[w].size(); ++j) {
      const std::pair<int, int>& v = alive_w[w].value(j);
      const size_t before = alive.size();
      std::pair<int, int>& r = alive[alive_w[w].key(j)];
      if (alive.size() != before) r = v;
      else { r.first = std::min(r.first, v.first); r.second = std::max(r.second, v.second); }
    }
  // 3) bond state lists (deterministic order)
  MPO mpo;
  mpo.K = K;
  mpo.bonds.resize(K + 1);
  std::vector<std::unordered_map<uint64_t, int>> index(K + 1);
  {
    std::vector<std::vector<uint64_t>> keys(K + 1);
    for (size_t j = 0; j < alive.size(); ++j)
      for (int b = alive.value(j).first; b <= alive.value(j).second; ++b) keys[b].push_back(alive.key(j));
    for (int b = 0; b <= K; ++b) {
      auto& v = keys[b];
      std::vector<BondState> st;
      for (uint64_t kk : v) {
        BondState bs;
        bs.key = unpack_key(kk);
        int da = 0, db = 0;
        for (int i = 0; i < bs.key.n; ++i) {
          int d = bs.key.ops[i].cre ? 1 : -1;
          if (bs.key.ops[i].x & 1) db += d; else da += d;
        }
        if (bs.key.kind == 3) { da = -da; db = -db; }
        bs.dna = da; bs.dnb = db;
        bs.parity = bs.key.n & 1;
        st.push_back(bs);
      }
      std::sort(st.begin(), st.end(), [](const BondState& a, const BondState& b2) {
        if (a.dna != b2.dna) return a.dna < b2.dna;
        if (a.dnb != b2.dnb) return a.dnb < b2.dnb;
        return a.key.pack() < b2.key.pack();
      });
      for (size_t i = 0; i < st.size(); ++i) index[b][st[i].key.pack()] = (int)i;
      mpo.bonds[b] = std::move(st);
    }
  }
  // 4) entries: routed transitions + pass-throughs
  mpo.W.resize(K);
  std::atomic<int> next_site{0};
  run_parallel(nw, [&](int) {
    for (int s; (s = next_site.fetch_add(1)) < K;) {
    auto& out = mpo.W[s];
    for (size_t j = 0; j < acc[s].size(); ++j) {
      const uint64_t kk = acc[s].key(j);
      const EntryAcc& a = acc[s].value(j);
      WEntry e;
      e.row = index[s].at(kk >> 30);
      e.col = index[s + 1].at(kk & ((1ULL << 30) - 1));
      bool nz = false;
      for (int i = 0; i < 16; ++i) { e.m[i] = a.m[i]; if (std::fabs(e.m[i]) > 0) nz = true; }
      if (nz) out.push_back(e);
    }
    for (const auto& kv : index[s]) {
      auto it = index[s + 1].find(kv.first);
      if (it == index[s + 1].end()) continue;
      WEntry e;
      e.row = kv.second;
      e.col = it->second;
      int par = mpo.bonds[s][kv.second].parity;
      for (int i = 0; i < 16; ++i) e.m[i] = 0;
      const double pz[4] = {1, -1, -1, 1};
      for (int n = 0; n < 4; ++n) e.m[n * 5] = par ? pz[n] : 1.0;
      out.push_back(e);
    }
    std::sort(out.begin(), out.end(), [](const WEntry& a, const WEntry& b) {
      return a.col != b.col ? a.col < b.col : a.row < b.row;
    });
    }
  });
  return mpo;
}

void mpo_to_dense(const MPO& mpo, std::vector<double>& out) {
  const int K = mpo.K;
  if (K > 6) throw std::runtime_error("mpo_to_dense: K too large");
  // T[state] is a (4^b x 4^b) matrix
  std::vector<std::vector<double>> T(mpo.bonds[0].size());
  int I0 = mpo.state_I(0);
  T[I0] = {1.0};
  size_t dim = 1;
  for (int s = 0; s < K; ++s) {
    size_t nd = dim * 4;
    std::vector<std::vector<double>> Tn(mpo.bonds[s + 1].size());
    for (const auto& e : mpo.W[s]) {
      const auto& src = T[e.row];
      if (src.empty()) continue;
      auto& dst = Tn[e.col];
      if (dst.empty()) dst.assign(nd * nd, 0.0);
      for (size_t i = 0; i < dim; ++i)
        for (size_t j = 0; j < dim; ++j) {
          double v = src[i * dim + j];
          if (v == 0) continue;
          for (int n = 0; n < 4; ++n)
            for (int np = 0; np < 4; ++np) {
              double w = e.m[n * 4 + np];
              if (w != 0) dst[(i * 4 + n) * nd + (j * 4 + np)] += v * w;
            }
        }
    }
    T.swap(Tn);
    dim = nd;
  }
  int H = mpo.state_H(K);
  out = T[H];
}

}  // namespace gbdmrg
