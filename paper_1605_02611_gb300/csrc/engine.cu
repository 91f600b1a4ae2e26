// Two-site DMRG engine (see engine.hpp).  Host code here only plans work
// lists; every arithmetic step on the MPS, environments and wavefunctions runs
// in the kernels of kernels.cu (cuSOLVER syevd serves the dense symmetric
// eigenproblems of the decimation step).
#include <algorithm>
#include <cstdint>
#include <cstdio>
#include <chrono>
#include <cmath>
#include <cstring>
#include <exception>
#include <map>
#include <mutex>
#include <numeric>
#include <thread>
#include <tuple>

#include "engine.hpp"
#include "mlp.hpp"

namespace gbdmrg {

void cuda_check(cudaError_t e, const char* what) {
  if (e == cudaSuccess) return;
  if (e == cudaErrorMemoryAllocation)
    throw Error(ST_ENOMEM, std::string(what) + ": " + cudaGetErrorString(e));
  throw Error(ST_ECUDA, std::string(what) + ": " + cudaGetErrorString(e));
}

static void solver_check(cusolverStatus_t s, const char* what) {
  if (s != CUSOLVER_STATUS_SUCCESS) throw Error(ST_ECUDA, std::string(what) + ": cusolver status " + std::to_string((int)s));
}

void* dev_alloc(size_t bytes, cudaStream_t s) {
  void* p = nullptr;
  if (bytes == 0) return nullptr;
  cuda_check(cudaMallocAsync(&p, bytes, s), "cudaMallocAsync");
  return p;
}
void dev_free(void* p, cudaStream_t s) {
  if (p) cudaFreeAsync(p, s);
}

int Bond::find(int a, int b) const {
  int lo = 0, hi = nsec() - 1;
  while (lo <= hi) {
    int mid = (lo + hi) >> 1;
    if (qa[mid] == a && qb[mid] == b) return mid;
    if (qa[mid] < a || (qa[mid] == a && qb[mid] < b)) lo = mid + 1;
    else hi = mid - 1;
  }
  return -1;
}

void Bond::add(int a, int b, int d) {
  qa.push_back(a);
  qb.push_back(b);
  dim.push_back(d);
  off.push_back(total);
  total += d;
}

OpLayout make_op_layout(const Bond& b, int da, int db) {
  OpLayout L;
  L.da = da;
  L.db = db;
  L.blk_of_col.assign(b.nsec(), -1);
  long off = 0;
  for (int j = 0; j < b.nsec(); ++j) {
    int i = b.find(b.qa[j] + da, b.qb[j] + db);
    if (i < 0) continue;
    L.blk_of_col[j] = (int)L.blocks.size();
    L.blocks.push_back({i, j, b.dim[i], b.dim[j], off});
    off += (long)b.dim[i] * b.dim[j];
  }
  L.nnz = off;
  return L;
}

size_t Env::bytes() const {
  size_t s = 0;
  for (size_t i = 0; i < cls.size(); ++i) s += (size_t)nslot[i] * cls[i].nnz * sizeof(double);
  return s;
}

void SiteT::layout(const Bond& l, const Bond& r) {
  L = l;
  R = r;
  blocks.clear();
  bn.clear();
  lookup.assign((size_t)l.nsec() * 4, -1);
  long off = 0;
  for (int ql = 0; ql < l.nsec(); ++ql)
    for (int n = 0; n < 4; ++n) {
      int qr = r.find(l.qa[ql] + LQA[n], l.qb[ql] + LQB[n]);
      if (qr < 0) continue;
      lookup[ql * 4 + n] = (int)blocks.size();
      blocks.push_back({ql, qr, l.dim[ql], r.dim[qr], off});
      bn.push_back(n);
      off += (long)l.dim[ql] * r.dim[qr];
    }
  nnz = off;
}

void PsiLayout::build(const Bond& l, const Bond& r, int sa, int sb) {
  L = l;
  R = r;
  da = sa;
  db = sb;
  blocks.clear();
  b1.clear();
  b2.clear();
  lookup.assign((size_t)l.nsec() * 16, -1);
  long off = 0;
  for (int ql = 0; ql < l.nsec(); ++ql)
    for (int n1 = 0; n1 < 4; ++n1)
      for (int n2 = 0; n2 < 4; ++n2) {
        int qr = r.find(l.qa[ql] + LQA[n1] + LQA[n2] + sa, l.qb[ql] + LQB[n1] + LQB[n2] + sb);
        if (qr < 0) continue;
        lookup[(ql * 4 + n1) * 4 + n2] = (int)blocks.size();
        blocks.push_back({ql, qr, l.dim[ql], r.dim[qr], off});
        b1.push_back(n1);
        b2.push_back(n2);
        off += (long)l.dim[ql] * r.dim[qr];
      }
  nnz = off;
}

// ---------------------------------------------------------------- GEMM plans

int GemmBuilder::begin(double* C, int ldc, int m, int n, int beta) {
  tasks.push_back({C, ldc, m, n, beta, (int)terms.size(), (int)terms.size()});
  return (int)tasks.size() - 1;
}

void GemmBuilder::term(const double* A, int lda, const double* B, int ldb, int k, int flags, double alpha,
                       int m, int n) {
  if (k <= 0 || m <= 0 || n <= 0) return;
  terms.push_back({A, B, lda, ldb, k, flags, alpha});
  tasks.back().t1 = (int)terms.size();
  flops += 2.0 * m * n * k;
}

void GemmBuilder::end() {
  GemmTask& t = tasks.back();
  if (t.t1 == t.t0) {
    tasks.pop_back();
    return;
  }
  int idx = (int)tasks.size() - 1;
  for (int r0 = 0; r0 < t.m; r0 += GEMM_TM)
    for (int c0 = 0; c0 < t.n; c0 += GEMM_TN) tiles.push_back({idx, r0, c0});
}

void GemmPlan::upload(const std::vector<GemmTile>& ti, const std::vector<GemmTask>& ta,
                      const std::vector<GemmTerm>& te, cudaStream_t s) {
  tiles.upload(ti, s);
  tasks.upload(ta, s);
  terms.upload(te, s);
  ntiles = (int)ti.size();
}

void GemmPlan::run(cudaStream_t s) const {
  if (ntiles == 0) return;
  launch_gemm(tiles.p, ntiles, tasks.p, terms.p, s);
  cuda_check(cudaGetLastError(), "gemm launch");
}

static void run_builder(Context& c, GemmBuilder& g) {
  if (g.tasks.empty()) return;
  c.other_flops_total += g.flops;
  GemmPlan p;
  p.upload(g.tiles, g.tasks, g.terms, c.stream);
  p.run(c.stream);
  // host vectors must outlive the async upload: synchronise before they go
  cuda_check(cudaStreamSynchronize(c.stream), "sync");
}

static void run_copies(Context& c, const std::vector<CopyJob>& jobs) {
  if (jobs.empty()) return;
  int mx = 0;
  for (auto& j : jobs) mx = std::max(mx, j.rows * j.cols);
  DArr<CopyJob> d;
  d.upload(jobs, c.stream);
  launch_copy(d.p, (int)jobs.size(), mx, c.stream);
  cuda_check(cudaGetLastError(), "copy launch");
  cuda_check(cudaStreamSynchronize(c.stream), "sync");
}

// ---------------------------------------------------------------- context

Context::~Context() {
  left.clear();
  right.clear();
  sites.clear();
  lt.combo.release();
  rt.combo.release();
  plan = SigmaPlan();
  // device arrays are freed on the context stream: release them before it goes
  mlp_s.reset();
  harvest.F.release();
  harvest.P.release();
  harvest.T.release();
  if (stream) cudaStreamSynchronize(stream);
  if (solver) cusolverDnDestroy(solver);
  if (ev0) cudaEventDestroy(ev0);
  if (ev1) cudaEventDestroy(ev1);
  for (int i = 0; i < kAux; ++i) {
    if (aux_solver[i]) cusolverDnDestroy(aux_solver[i]);
    if (aux[i]) cudaStreamDestroy(aux[i]);
  }
  for (int i = 0; i <= kAux; ++i)
    if (aux_ev[i]) cudaEventDestroy(aux_ev[i]);
  if (own_stream && stream) cudaStreamDestroy(stream);
}

void ctx_init(Context& c) {
  if (!c.stream) {
    cuda_check(cudaStreamCreateWithFlags(&c.stream, cudaStreamNonBlocking), "stream create");
    c.own_stream = true;
  }
  int dev = 0;
  cuda_check(cudaGetDevice(&dev), "get device");
  cudaMemPool_t pool;
  cuda_check(cudaDeviceGetDefaultMemPool(&pool, dev), "mem pool");
  uint64_t thr = UINT64_MAX;
  cudaMemPoolSetAttribute(pool, cudaMemPoolAttrReleaseThreshold, &thr);
  cuda_check(cudaEventCreate(&c.ev0), "event");
  cuda_check(cudaEventCreate(&c.ev1), "event");
  for (int i = 0; i < Context::kAux; ++i) {
    cuda_check(cudaStreamCreateWithFlags(&c.aux[i], cudaStreamNonBlocking), "aux stream");
    solver_check(cusolverDnCreate(&c.aux_solver[i]), "cusolverDnCreate");
    solver_check(cusolverDnSetStream(c.aux_solver[i], c.aux[i]), "cusolverDnSetStream");
  }
  for (int i = 0; i <= Context::kAux; ++i)
    cuda_check(cudaEventCreateWithFlags(&c.aux_ev[i], cudaEventDisableTiming), "aux event");
  solver_check(cusolverDnCreate(&c.solver), "cusolverDnCreate");
  solver_check(cusolverDnSetStream(c.solver, c.stream), "cusolverDnSetStream");
  c.mpo = build_mpo(c.K, c.h1.data(), c.eri.data());
  c.sites.resize(c.K);
  c.site_set.assign(c.K, false);
  c.left.resize(c.K + 1);
  c.right.resize(c.K + 1);
}

static Bond bond_from_labels(int D, const int* qn) {
  Bond b;
  int i = 0;
  while (i < D) {
    int a = qn[2 * i], bb = qn[2 * i + 1];
    int j = i;
    while (j < D && qn[2 * j] == a && qn[2 * j + 1] == bb) ++j;
    if (b.nsec() && (a < b.qa.back() || (a == b.qa.back() && bb <= b.qb.back())))
      throw Error(ST_EINVAL, "bond labels must be grouped and sorted by (n_alpha, n_beta)");
    b.add(a, bb, j - i);
    i = j;
  }
  return b;
}

static bool same_bond(const Bond& x, const Bond& y) {
  return x.qa == y.qa && x.qb == y.qb && x.dim == y.dim;
}

void set_site_dense(Context& c, int k, int Dl, int Dr, const int* qn_l, const int* qn_r, const double* A) {
  if (k < 0 || k >= c.K) throw Error(ST_EINVAL, "site out of range");
  Bond l = bond_from_labels(Dl, qn_l), r = bond_from_labels(Dr, qn_r);
  if (k == 0 && !(l.nsec() == 1 && l.qa[0] == 0 && l.qb[0] == 0 && l.dim[0] == 1))
    throw Error(ST_EINVAL, "left boundary bond must be one state with (0,0)");
  if (k == c.K - 1 && !(r.nsec() == 1 && r.qa[0] == c.Na && r.qb[0] == c.Nb && r.dim[0] == 1))
    throw Error(ST_EINVAL, "right boundary bond must be one state with (N_alpha, N_beta)");
  if (k > 0 && c.site_set[k - 1] && !same_bond(c.sites[k - 1].R, l))
    throw Error(ST_EINVAL, "left bond does not match the right bond of the previous site");
  if (k + 1 < c.K && c.site_set[k + 1] && !same_bond(c.sites[k + 1].L, r))
    throw Error(ST_EINVAL, "right bond does not match the left bond of the next site");
  SiteT& s = c.sites[k];
  s.layout(l, r);
  std::vector<double> h(s.nnz, 0.0);
  for (size_t b = 0; b < s.blocks.size(); ++b) {
    const Block& B = s.blocks[b];
    int n = s.bn[b];
    for (int i = 0; i < B.rows; ++i)
      for (int j = 0; j < B.cols; ++j) {
        double v = A[((size_t)(l.off[B.rs] + i) * 4 + n) * Dr + r.off[B.cs] + j];
        if (!std::isfinite(v)) throw Error(ST_EINVAL, "non-finite MPS entry");
        h[B.off + (long)i * B.cols + j] = v;
      }
  }
  s.d.upload(h, c.stream);
  cuda_check(cudaStreamSynchronize(c.stream), "sync");
  c.site_set[k] = true;
  c.prepared = -1;
}

// ---------------------------------------------------------------- checkpoint

namespace {
const char kMagic[8] = {'G', 'B', 'D', 'M', 'R', 'G', 'v', '1'};

struct FileCloser {
  void operator()(FILE* f) const {
    if (f) std::fclose(f);
  }
};

void put(FILE* f, const void* p, size_t n) {
  if (n && std::fwrite(p, 1, n, f) != n) throw Error(ST_EIO, "checkpoint: write failed");
}
void get(FILE* f, void* p, size_t n) {
  if (n && std::fread(p, 1, n, f) != n) throw Error(ST_EIO, "checkpoint: file truncated or unreadable");
}
void put_bond(FILE* f, const Bond& b) {
  const int32_t ns = b.nsec();
  put(f, &ns, 4);
  for (int i = 0; i < ns; ++i) {
    const int32_t v[3] = {b.qa[i], b.qb[i], b.dim[i]};
    put(f, v, 12);
  }
}
Bond get_bond(FILE* f) {
  int32_t ns = 0;
  get(f, &ns, 4);
  if (ns < 0 || ns > (1 << 20)) throw Error(ST_EIO, "checkpoint: corrupt bond");
  Bond b;
  for (int i = 0; i < ns; ++i) {
    int32_t v[3];
    get(f, v, 12);
    if (v[2] <= 0) throw Error(ST_EIO, "checkpoint: corrupt bond");
    if (i > 0 && !(v[0] > b.qa.back() || (v[0] == b.qa.back() && v[1] > b.qb.back())))
      throw Error(ST_EIO, "checkpoint: bond sectors out of order");
    b.add(v[0], v[1], v[2]);
  }
  return b;
}
}  // namespace

void save_mps(Context& c, const char* path) {
  for (int j = 0; j < c.K; ++j)
    if (!c.site_set[j]) throw Error(ST_ESTATE, "MPS tensor of site " + std::to_string(j) + " not set");
  std::unique_ptr<FILE, FileCloser> f(std::fopen(path, "wb"));
  if (!f) throw Error(ST_EIO, std::string("checkpoint: cannot open ") + path + " for writing");
  put(f.get(), kMagic, 8);
  const int32_t hdr[4] = {c.K, c.N, c.two_sz, 0};
  put(f.get(), hdr, 16);
  std::vector<double> h;
  for (int k = 0; k < c.K; ++k) {
    const SiteT& st = c.sites[k];
    put_bond(f.get(), st.L);
    put_bond(f.get(), st.R);
    const int64_t nnz = st.nnz;
    put(f.get(), &nnz, 8);
    h.resize(st.nnz);
    if (st.nnz) cuda_check(cudaMemcpy(h.data(), st.d.p, st.nnz * sizeof(double), cudaMemcpyDeviceToHost), "d2h");
    put(f.get(), h.data(), st.nnz * sizeof(double));
  }
  if (std::fflush(f.get()) != 0) throw Error(ST_EIO, "checkpoint: write failed");
}

void load_mps(Context& c, const char* path) {
  std::unique_ptr<FILE, FileCloser> f(std::fopen(path, "rb"));
  if (!f) throw Error(ST_EIO, std::string("checkpoint: cannot open ") + path);
  char magic[8];
  get(f.get(), magic, 8);
  if (std::memcmp(magic, kMagic, 8) != 0) throw Error(ST_EIO, "checkpoint: not an MPS checkpoint of this library");
  int32_t hdr[4];
  get(f.get(), hdr, 16);
  if (hdr[0] != c.K || hdr[1] != c.N || hdr[2] != c.two_sz)
    throw Error(ST_EINVAL, "checkpoint: K, N or 2S_z differ from this problem");
  // read everything first: the context's MPS changes only if the whole file is valid
  std::vector<SiteT> sites(c.K);
  std::vector<std::vector<double>> data(c.K);
  for (int k = 0; k < c.K; ++k) {
    Bond l = get_bond(f.get()), r = get_bond(f.get());
    if (k > 0 && !same_bond(sites[k - 1].R, l)) throw Error(ST_EIO, "checkpoint: bonds of neighbouring sites differ");
    sites[k].layout(l, r);
    int64_t nnz = 0;
    get(f.get(), &nnz, 8);
    if (nnz != sites[k].nnz) throw Error(ST_EIO, "checkpoint: block sizes do not match the bond sectors");
    data[k].resize(nnz);
    get(f.get(), data[k].data(), nnz * sizeof(double));
    for (double v : data[k])
      if (!std::isfinite(v)) throw Error(ST_EIO, "checkpoint: non-finite MPS entry");
  }
  const Bond& l0 = sites[0].L;
  const Bond& rK = sites[c.K - 1].R;
  if (!(l0.nsec() == 1 && l0.qa[0] == 0 && l0.qb[0] == 0 && l0.dim[0] == 1) ||
      !(rK.nsec() == 1 && rK.qa[0] == c.Na && rK.qb[0] == c.Nb && rK.dim[0] == 1))
    throw Error(ST_EIO, "checkpoint: boundary bonds do not fit this problem");
  for (int k = 0; k < c.K; ++k) {
    c.sites[k] = std::move(sites[k]);
    c.sites[k].d.upload(data[k], c.stream);
    cuda_check(cudaStreamSynchronize(c.stream), "sync");
    c.site_set[k] = true;
  }
  for (auto& e : c.left) e.valid = false;   // environments of the previous MPS
  for (auto& e : c.right) e.valid = false;
  c.prepared = -1;
}

void get_site_dense(Context& c, int k, std::vector<double>& A) {
  SiteT& s = c.sites[k];
  std::vector<double> h(s.nnz);
  if (s.nnz) cuda_check(cudaMemcpy(h.data(), s.d.p, s.nnz * sizeof(double), cudaMemcpyDeviceToHost), "d2h");
  int Dl = s.L.total, Dr = s.R.total;
  A.assign((size_t)Dl * 4 * Dr, 0.0);
  for (size_t b = 0; b < s.blocks.size(); ++b) {
    const Block& B = s.blocks[b];
    int n = s.bn[b];
    for (int i = 0; i < B.rows; ++i)
      for (int j = 0; j < B.cols; ++j)
        A[((size_t)(s.L.off[B.rs] + i) * 4 + n) * Dr + s.R.off[B.cs] + j] = h[B.off + (long)i * B.cols + j];
  }
}

// ---------------------------------------------------------------- environments

void env_alloc(Context& c, Env& e, const Bond& b, const std::vector<BondState>& st) {
  e = Env();
  e.bond = b;
  std::map<std::pair<int, int>, int> cmap;
  e.st_cls.assign(st.size(), -1);
  e.st_slot.assign(st.size(), -1);
  for (size_t i = 0; i < st.size(); ++i) {
    auto key = std::make_pair(st[i].dna, st[i].dnb);
    auto it = cmap.find(key);
    int ci;
    if (it == cmap.end()) {
      ci = (int)e.cls.size();
      cmap[key] = ci;
      e.cls.push_back(make_op_layout(b, key.first, key.second));
      e.nslot.push_back(0);
    } else ci = it->second;
    e.st_cls[i] = ci;
    e.st_slot[i] = e.nslot[ci]++;
  }
  e.data.resize(e.cls.size());
  for (size_t ci = 0; ci < e.cls.size(); ++ci) {
    size_t n = (size_t)e.nslot[ci] * e.cls[ci].nnz;
    e.data[ci].alloc(n, c.stream);
    if (n) cuda_check(cudaMemsetAsync(e.data[ci].p, 0, n * sizeof(double), c.stream), "memset");
  }
  e.valid = true;
}

void env_boundary_left(Context& c, Env& e) {
  Bond b;
  b.add(0, 0, 1);
  env_alloc(c, e, b, c.mpo.bonds[0]);
  int I = c.mpo.state_I(0);
  double one = 1.0;
  cuda_check(cudaMemcpyAsync(e.op(I), &one, sizeof(double), cudaMemcpyHostToDevice, c.stream), "h2d");
  cuda_check(cudaStreamSynchronize(c.stream), "sync");
}

void env_boundary_right(Context& c, Env& e) {
  Bond b;
  b.add(c.Na, c.Nb, 1);
  env_alloc(c, e, b, c.mpo.bonds[c.K]);
  int H = c.mpo.state_H(c.K);
  double one = 1.0;
  cuda_check(cudaMemcpyAsync(e.op(H), &one, sizeof(double), cudaMemcpyHostToDevice, c.stream), "h2d");
  cuda_check(cudaStreamSynchronize(c.stream), "sync");
}

// f(lo, hi) over contiguous parts of [0, n) on up to 16 host threads (the calling
// thread takes the first part); the first exception of any part is rethrown
template <class F>
static void parallel_ranges(size_t n, F&& f) {
  const size_t hw = std::max(1u, std::thread::hardware_concurrency());
  const size_t nt = std::max<size_t>(1, std::min<size_t>({hw, 16, n / 1024 + 1}));
  std::exception_ptr fail;
  std::mutex mu;
  auto part = [&](size_t t) {
    try {
      f(n * t / nt, n * (t + 1) / nt);
    } catch (...) {
      std::lock_guard<std::mutex> lk(mu);
      if (!fail) fail = std::current_exception();
    }
  };
  std::vector<std::thread> pool;
  for (size_t t = 1; t < nt; ++t) pool.emplace_back(part, t);
  part(0);
  for (auto& th : pool) th.join();
  if (fail) std::rethrow_exception(fail);
}

// The blocking sums of one side: for every (bond state beta, site slot nn) the list
// of (environment state, W coefficient) terms, in the order of the W entries, stored
// as one array with offsets (slot i = beta * 16 + nn owns [start[i], start[i + 1])).
struct TildeLists {
  std::vector<long> start;
  std::vector<std::pair<int, double>> items;
  size_t size() const { return start.size() - 1; }
  size_t len(size_t i) const { return (size_t)(start[i + 1] - start[i]); }
  const std::pair<int, double>* at(size_t i) const { return items.data() + start[i]; }
};

// lists of W[site]: by_col = the blocking sums over rows (left side) or over columns.
// Each thread owns a range of bond states and scans all entries for them.
static TildeLists tilde_lists(const MPO& mpo, int site, int nmid, bool by_col) {
  TildeLists tl;
  const size_t n = (size_t)nmid * 16;
  const auto& W = mpo.W[site];
  tl.start.assign(n + 1, 0);
  parallel_ranges((size_t)nmid, [&](size_t lo, size_t hi) {
    for (const auto& e : W) {
      const size_t b = (size_t)(by_col ? e.col : e.row);
      if (b < lo || b >= hi) continue;
      for (int nn = 0; nn < 16; ++nn)
        if (e.m[nn] != 0.0) tl.start[b * 16 + nn + 1]++;
    }
  });
  for (size_t i = 0; i < n; ++i) tl.start[i + 1] += tl.start[i];
  tl.items.resize((size_t)tl.start[n]);
  parallel_ranges((size_t)nmid, [&](size_t lo, size_t hi) {
    std::vector<long> fill(tl.start.begin() + lo * 16, tl.start.begin() + hi * 16);
    for (const auto& e : W) {
      const size_t b = (size_t)(by_col ? e.col : e.row);
      if (b < lo || b >= hi) continue;
      for (int nn = 0; nn < 16; ++nn)
        if (e.m[nn] != 0.0) tl.items[(size_t)fill[(b - lo) * 16 + nn]++] = {by_col ? e.row : e.col, e.m[nn]};
    }
  });
  return tl;
}

static void finish_tilde(Context& c, Env& env, const TildeLists& lists, Tilde& t, bool approx) {
  t.env = &env;
  t.ref.assign(t.nmid, {});
  const size_t n = lists.size();
  // operator class of every slot (-1: empty), checked to be the same for all terms
  std::vector<int> cls_of(n, -1);
  parallel_ranges(n, [&](size_t lo, size_t hi) {
    for (size_t i = lo; i < hi; ++i) {
      const size_t len = lists.len(i);
      if (!len) continue;
      const auto* L = lists.at(i);
      const int cls = env.st_cls[L[0].first];
      for (size_t j = 0; j < len; ++j)
        if (env.st_cls[L[j].first] != cls) throw Error(ST_ECUDA, "internal: mixed operator classes in a blocking sum");
      // a class without elements (no sector pair at this bond) contributes nothing: the
      // slot stays empty, so that no zero-size sum shares an address with another one
      if (env.cls[cls].nnz > 0) cls_of[i] = cls;
    }
  });
  // slots with several terms become materialised sums: their output offsets, output
  // index and term range, in slot order
  std::vector<long> off(n, -1), tstart(n, 0);
  std::vector<int> oidx(n, -1);
  size_t total = 0, nterms = 0;
  int nouts = 0;
  for (size_t i = 0; i < n; ++i) {
    const size_t len = lists.len(i);
    if (len > 1 && cls_of[i] >= 0) {
      off[i] = (long)total;
      total += env.cls[cls_of[i]].nnz;
      tstart[i] = (long)nterms;
      nterms += len;
      oidx[i] = nouts++;
    }
  }
  t.combo.alloc(total, c.stream);
  std::vector<ComboOut> outs((size_t)nouts);
  std::vector<ComboTerm> terms(nterms);
  std::mutex mu;
  long mx = 0, flops = 0;
  parallel_ranges(n, [&](size_t lo, size_t hi) {
    long my_mx = 0, my_flops = 0;
    for (size_t i = lo; i < hi; ++i) {
      const size_t len = lists.len(i);
      if (!len || cls_of[i] < 0) continue;
      const auto* L = lists.at(i);
      const int cls = cls_of[i];
      TRef& r = t.ref[i / 16][i % 16];
      r.cls = cls;
      if (len == 1) {
        r.p = env.op(L[0].first);
        r.coef = L[0].second;
      } else {
        r.p = t.combo.p + off[i];
        r.coef = 1.0;
        const long nnz = env.cls[cls].nnz;
        for (size_t j = 0; j < len; ++j) terms[(size_t)tstart[i] + j] = {env.op(L[j].first), L[j].second};
        outs[(size_t)oidx[i]] = ComboOut{t.combo.p + off[i], nnz, (int)tstart[i], (int)(tstart[i] + (long)len)};
        my_mx = std::max(my_mx, nnz);
        my_flops += 2L * (long)len * nnz;
      }
    }
    std::lock_guard<std::mutex> lk(mu);
    mx = std::max(mx, my_mx);
    flops += my_flops;
  });
  t.combo_flops = flops;
  c.other_flops_total += (double)t.combo_flops;
  if (!outs.empty() && approx && c.tc_combos && c.precision > 0 && (long)terms.size() >= c.tc_combo_min_terms) {
    std::vector<int> out_cls(outs.size());
    for (size_t i = 0; i < n; ++i)
      if (oidx[i] >= 0) out_cls[(size_t)oidx[i]] = cls_of[i];
    combos_tc(c, env, outs, terms, out_cls);
  } else if (!outs.empty()) {
    DArr<ComboOut> d_o;
    DArr<ComboTerm> d_t;
    d_o.upload(outs, c.stream);
    d_t.upload(terms, c.stream);
    launch_combo(d_o.p, (int)outs.size(), mx, d_t.p, c.stream);
    cuda_check(cudaGetLastError(), "combo launch");
    cuda_check(cudaStreamSynchronize(c.stream), "sync");
  }
}

void build_tilde_left(Context& c, Env& L, int site, Tilde& t, bool approx) {
  t.nmid = (int)c.mpo.bonds[site + 1].size();
  finish_tilde(c, L, tilde_lists(c.mpo, site, t.nmid, true), t, approx);
}

void build_tilde_right(Context& c, Env& R, int site, Tilde& t, bool approx) {
  t.nmid = (int)c.mpo.bonds[site].size();
  finish_tilde(c, R, tilde_lists(c.mpo, site, t.nmid, false), t, approx);
}

// column sector of a W-contracted operator block whose row sector is `row`
static inline int tilde_col(const Bond& b, const OpLayout& L, int row) {
  return b.find(b.qa[row] - L.da, b.qb[row] - L.db);
}

static size_t budget_elems(Context& c) { return (size_t)c.chunk_budget_mb * (1u << 20) / sizeof(double); }

void env_update_left(Context& c, Tilde& lt, const SiteT& A, int site, Env& out) {
  if (c.env_precision == 3) {
    env_update_exact(c, lt, A, site, out, true);
    return;
  }
  if (c.env_precision == 2) {
    env_update_tc(c, lt, A, site, out, true);
    return;
  }
  const auto& st = c.mpo.bonds[site + 1];
  const Bond& Lb = A.L;
  const Bond& Rb = A.R;
  Env& Lenv = *lt.env;
  env_alloc(c, out, Rb, st);
  const int nR = Rb.nsec();
  // intermediate sizes per state
  std::vector<size_t> tsz(st.size(), 0);
  for (size_t beta = 0; beta < st.size(); ++beta)
    for (int n1 = 0; n1 < 4; ++n1)
      for (int j = 0; j < nR; ++j) {
        int ql = Lb.find(Rb.qa[j] + st[beta].dna - LQA[n1], Rb.qb[j] + st[beta].dnb - LQB[n1]);
        if (ql >= 0) tsz[beta] += (size_t)Lb.dim[ql] * Rb.dim[j];
      }
  size_t budget = budget_elems(c);
  size_t b0 = 0;
  while (b0 < st.size()) {
    size_t b1 = b0, tot = 0;
    while (b1 < st.size() && (b1 == b0 || tot + tsz[b1] <= budget)) tot += tsz[b1++];
    DArr<double> T;
    T.alloc(tot, c.stream);
    GemmBuilder g1, g2;
    size_t toff = 0;
    for (size_t beta = b0; beta < b1; ++beta) {
      std::vector<long> tpos((size_t)4 * nR, -1);
      for (int n1 = 0; n1 < 4; ++n1)
        for (int j = 0; j < nR; ++j) {
          int ql = Lb.find(Rb.qa[j] + st[beta].dna - LQA[n1], Rb.qb[j] + st[beta].dnb - LQB[n1]);
          if (ql < 0) continue;
          int m = Lb.dim[ql], n = Rb.dim[j];
          g1.begin(T.p + toff, n, m, n, 0);
          for (int n1p = 0; n1p < 4; ++n1p) {
            const TRef& r = lt.ref[beta][n1 * 4 + n1p];
            if (!r.p) continue;
            const OpLayout& Lay = Lenv.cls[r.cls];
            int qlp = tilde_col(Lb, Lay, ql);
            if (qlp < 0) continue;
            int bl = Lay.blk_of_col[qlp];
            if (bl < 0 || Lay.blocks[bl].rs != ql) continue;
            int ab = A.blk(qlp, n1p);
            if (ab < 0 || A.blocks[ab].cs != j) continue;
            g1.term(r.p + Lay.blocks[bl].off, Lb.dim[qlp], A.d.p + A.blocks[ab].off, n, Lb.dim[qlp], GT_BN,
                    r.coef, m, n);
          }
          size_t before = g1.tasks.size();
          g1.end();
          if (g1.tasks.size() == before) {
            tpos[n1 * nR + j] = (long)toff;
            toff += (size_t)m * n;
          }
        }
      const OpLayout& Lo = out.lay((int)beta);
      double* obase = out.op((int)beta);
      for (const Block& ob : Lo.blocks) {
        int qa = ob.rs, qap = ob.cs;
        g2.begin(obase + ob.off, ob.cols, ob.rows, ob.cols, 0);
        for (int n1 = 0; n1 < 4; ++n1) {
          int ql = Lb.find(Rb.qa[qa] - LQA[n1], Rb.qb[qa] - LQB[n1]);
          if (ql < 0) continue;
          int ab = A.blk(ql, n1);
          if (ab < 0 || A.blocks[ab].cs != qa) continue;
          long tp = tpos[n1 * nR + qap];
          if (tp < 0) continue;
          g2.term(A.d.p + A.blocks[ab].off, Rb.dim[qa], T.p + tp, Rb.dim[qap], Lb.dim[ql], GT_TA | GT_BN, 1.0,
                  ob.rows, ob.cols);
        }
        g2.end();
      }
    }
    run_builder(c, g1);
    run_builder(c, g2);
    b0 = b1;
  }
}

void env_update_right(Context& c, Tilde& rt, const SiteT& B, int site, Env& out) {
  if (c.env_precision == 3) {
    env_update_exact(c, rt, B, site, out, false);
    return;
  }
  if (c.env_precision == 2) {
    env_update_tc(c, rt, B, site, out, false);
    return;
  }
  const auto& st = c.mpo.bonds[site];
  const Bond& Lb = B.L;
  const Bond& Rb = B.R;
  Env& Renv = *rt.env;
  env_alloc(c, out, Lb, st);
  const int nL = Lb.nsec();
  std::vector<size_t> tsz(st.size(), 0);
  for (size_t beta = 0; beta < st.size(); ++beta)
    for (int n2 = 0; n2 < 4; ++n2)
      for (int j = 0; j < nL; ++j) {
        int qr = Rb.find(Lb.qa[j] + st[beta].dna + LQA[n2], Lb.qb[j] + st[beta].dnb + LQB[n2]);
        if (qr >= 0) tsz[beta] += (size_t)Lb.dim[j] * Rb.dim[qr];
      }
  size_t budget = budget_elems(c);
  size_t b0 = 0;
  while (b0 < st.size()) {
    size_t b1 = b0, tot = 0;
    while (b1 < st.size() && (b1 == b0 || tot + tsz[b1] <= budget)) tot += tsz[b1++];
    DArr<double> T;
    T.alloc(tot, c.stream);
    GemmBuilder g1, g2;
    size_t toff = 0;
    for (size_t beta = b0; beta < b1; ++beta) {
      std::vector<long> tpos((size_t)4 * nL, -1);
      for (int n2 = 0; n2 < 4; ++n2)
        for (int j = 0; j < nL; ++j) {
          int qr = Rb.find(Lb.qa[j] + st[beta].dna + LQA[n2], Lb.qb[j] + st[beta].dnb + LQB[n2]);
          if (qr < 0) continue;
          int m = Lb.dim[j], n = Rb.dim[qr];
          g1.begin(T.p + toff, n, m, n, 0);
          for (int n2p = 0; n2p < 4; ++n2p) {
            const TRef& r = rt.ref[beta][n2 * 4 + n2p];
            if (!r.p) continue;
            const OpLayout& Lay = Renv.cls[r.cls];
            int qrp = Rb.find(Lb.qa[j] + LQA[n2p], Lb.qb[j] + LQB[n2p]);
            if (qrp < 0) continue;
            int bl = Lay.blk_of_col[qrp];
            if (bl < 0 || Lay.blocks[bl].rs != qr) continue;
            int bb = B.blk(j, n2p);
            if (bb < 0 || B.blocks[bb].cs != qrp) continue;
            g1.term(B.d.p + B.blocks[bb].off, Rb.dim[qrp], r.p + Lay.blocks[bl].off, Rb.dim[qrp], Rb.dim[qrp], 0,
                    r.coef, m, n);
          }
          size_t before = g1.tasks.size();
          g1.end();
          if (g1.tasks.size() == before) {
            tpos[n2 * nL + j] = (long)toff;
            toff += (size_t)m * n;
          }
        }
      const OpLayout& Lo = out.lay((int)beta);
      double* obase = out.op((int)beta);
      for (const Block& ob : Lo.blocks) {
        int qb = ob.rs, qbp = ob.cs;
        g2.begin(obase + ob.off, ob.cols, ob.rows, ob.cols, 0);
        for (int n2 = 0; n2 < 4; ++n2) {
          int qr = Rb.find(Lb.qa[qb] + LQA[n2], Lb.qb[qb] + LQB[n2]);
          if (qr < 0) continue;
          int bb = B.blk(qb, n2);
          if (bb < 0 || B.blocks[bb].cs != qr) continue;
          long tp = tpos[n2 * nL + qbp];
          if (tp < 0) continue;
          g2.term(B.d.p + B.blocks[bb].off, Rb.dim[qr], T.p + tp, Rb.dim[qr], Rb.dim[qr], 0, 1.0, ob.rows,
                  ob.cols);
        }
        g2.end();
      }
    }
    run_builder(c, g1);
    run_builder(c, g2);
    b0 = b1;
  }
}

// ---------------------------------------------------------------- sigma

void build_sigma_plan(Context& c, Tilde& lt, Tilde& rt, int k, SigmaPlan& plan) {
  const auto& mid = c.mpo.bonds[k + 1];
  Env& Lenv = *lt.env;
  Env& Renv = *rt.env;
  const Bond& Lb = Lenv.bond;
  const Bond& Rb = Renv.bond;
  plan = SigmaPlan();
  PsiLayout& P = plan.psi;
  P.build(Lb, Rb);
  plan.in.alloc(P.nnz, c.stream);
  plan.out.alloc(P.nnz, c.stream);
  if (c.precision >= 4) {
    build_tma_plan(c, lt, rt, k, plan, c.precision == 4 ? 1 : c.precision == 5 ? 3 : 2);
    return;
  }
  if (c.precision > 0) {
    build_mixed_plan(c, lt, rt, k, plan, c.precision == 1 ? 1 : c.precision == 2 ? 3 : 2);
    return;
  }
  const int nL = Lb.nsec();
  // X_beta layout = psi layout shifted by dQ_beta; X stored transposed per block
  std::vector<size_t> xsz(mid.size(), 0);
  for (size_t beta = 0; beta < mid.size(); ++beta)
    for (int ql = 0; ql < nL; ++ql)
      for (int n1 = 0; n1 < 4; ++n1)
        for (int n2 = 0; n2 < 4; ++n2) {
          int qr = Rb.find(Lb.qa[ql] + LQA[n1] + LQA[n2] + mid[beta].dna,
                           Lb.qb[ql] + LQB[n1] + LQB[n2] + mid[beta].dnb);
          if (qr >= 0) xsz[beta] += (size_t)Lb.dim[ql] * Rb.dim[qr];
        }
  size_t budget = budget_elems(c);
  size_t maxchunk = 0;
  std::vector<std::pair<size_t, size_t>> chunks;
  {
    size_t b0 = 0;
    while (b0 < mid.size()) {
      size_t b1 = b0, tot = 0;
      while (b1 < mid.size() && (b1 == b0 || tot + xsz[b1] <= budget)) tot += xsz[b1++];
      chunks.push_back({b0, b1});
      maxchunk = std::max(maxchunk, tot);
      b0 = b1;
    }
  }
  plan.X.alloc(maxchunk, c.stream);
  for (auto ch : chunks) {
    GemmBuilder g1, g2;
    size_t xoff = 0;
    std::vector<std::vector<long>> xpos(ch.second - ch.first);
    for (size_t beta = ch.first; beta < ch.second; ++beta) {
      auto& xp = xpos[beta - ch.first];
      xp.assign((size_t)nL * 16, -1);
      for (int qlp = 0; qlp < nL; ++qlp)
        for (int n1p = 0; n1p < 4; ++n1p)
          for (int n2 = 0; n2 < 4; ++n2) {
            int qr = Rb.find(Lb.qa[qlp] + LQA[n1p] + LQA[n2] + mid[beta].dna,
                             Lb.qb[qlp] + LQB[n1p] + LQB[n2] + mid[beta].dnb);
            if (qr < 0) continue;
            int m = Rb.dim[qr], n = Lb.dim[qlp];  // X^T block: qr rows, ql' cols
            g1.begin(plan.X.p + xoff, n, m, n, 0);
            for (int n2p = 0; n2p < 4; ++n2p) {
              const TRef& r = rt.ref[beta][n2 * 4 + n2p];
              if (!r.p) continue;
              int pb = P.blk(qlp, n1p, n2p);
              if (pb < 0) continue;
              int qrp = P.blocks[pb].cs;
              const OpLayout& Lay = Renv.cls[r.cls];
              int bl = Lay.blk_of_col[qrp];
              if (bl < 0 || Lay.blocks[bl].rs != qr) continue;
              g1.term(r.p + Lay.blocks[bl].off, Rb.dim[qrp], plan.in.p + P.blocks[pb].off, Rb.dim[qrp],
                      Rb.dim[qrp], 0, r.coef, m, n);
            }
            size_t before = g1.tasks.size();
            g1.end();
            if (g1.tasks.size() == before) {
              xp[(qlp * 4 + n1p) * 4 + n2] = (long)xoff;
              xoff += (size_t)m * n;
            }
          }
    }
    for (size_t pb = 0; pb < P.blocks.size(); ++pb) {
      const Block& ob = P.blocks[pb];
      int ql = ob.rs, n1 = P.b1[pb], n2 = P.b2[pb];
      g2.begin(plan.out.p + ob.off, ob.cols, ob.rows, ob.cols, 1);
      for (size_t beta = ch.first; beta < ch.second; ++beta) {
        const auto& xp = xpos[beta - ch.first];
        for (int n1p = 0; n1p < 4; ++n1p) {
          const TRef& r = lt.ref[beta][n1 * 4 + n1p];
          if (!r.p) continue;
          const OpLayout& Lay = Lenv.cls[r.cls];
          int qlp = tilde_col(Lb, Lay, ql);
          if (qlp < 0) continue;
          int bl = Lay.blk_of_col[qlp];
          if (bl < 0 || Lay.blocks[bl].rs != ql) continue;
          long xo = xp[(qlp * 4 + n1p) * 4 + n2];
          if (xo < 0) continue;
          g2.term(r.p + Lay.blocks[bl].off, Lb.dim[qlp], plan.X.p + xo, Lb.dim[qlp], Lb.dim[qlp], 0, r.coef,
                  ob.rows, ob.cols);
        }
      }
      g2.end();
    }
    plan.stage1.emplace_back();
    plan.stage1.back().upload(g1.tiles, g1.tasks, g1.terms, c.stream);
    plan.stage2.emplace_back();
    plan.stage2.back().upload(g2.tiles, g2.tasks, g2.terms, c.stream);
    plan.flops += g1.flops + g2.flops;
    cuda_check(cudaStreamSynchronize(c.stream), "sync");
  }
}

void run_sigma(Context& c, SigmaPlan& plan, const double* x, double* y) {
  if (plan.tm) {
    run_tma_sigma(c, plan, x, y);
    return;
  }
  if (plan.mx) {
    run_mixed_sigma(c, plan, x, y);
    return;
  }
  const size_t bytes = plan.psi.nnz * sizeof(double);
  if (x != plan.in.p) cuda_check(cudaMemcpyAsync(plan.in.p, x, bytes, cudaMemcpyDeviceToDevice, c.stream), "d2d");
  cuda_check(cudaMemsetAsync(plan.out.p, 0, bytes, c.stream), "memset");
  for (size_t i = 0; i < plan.stage1.size(); ++i) {
    plan.stage1[i].run(c.stream);
    plan.stage2[i].run(c.stream);
  }
  if (y != plan.out.p) cuda_check(cudaMemcpyAsync(y, plan.out.p, bytes, cudaMemcpyDeviceToDevice, c.stream), "d2d");
}

void compute_diag(Context& c, Tilde& lt, Tilde& rt, int k, const PsiLayout& P, double* diag) {
  const auto& mid = c.mpo.bonds[k + 1];
  Env& Lenv = *lt.env;
  Env& Renv = *rt.env;
  const Bond& Lb = Lenv.bond;
  const Bond& Rb = Renv.bond;
  std::vector<int> zb;
  for (size_t beta = 0; beta < mid.size(); ++beta)
    if (mid[beta].dna == 0 && mid[beta].dnb == 0) zb.push_back((int)beta);
  const int nz = (int)zb.size();
  cuda_check(cudaMemsetAsync(diag, 0, P.nnz * sizeof(double), c.stream), "memset");
  if (nz == 0) return;
  DArr<double> DL, DR;
  DL.alloc((size_t)4 * Lb.total * nz, c.stream);
  DR.alloc((size_t)4 * Rb.total * nz, c.stream);
  cuda_check(cudaMemsetAsync(DL.p, 0, DL.n * sizeof(double), c.stream), "memset");
  cuda_check(cudaMemsetAsync(DR.p, 0, DR.n * sizeof(double), c.stream), "memset");
  std::vector<DiagJob> jobs;
  int mx = 0;
  for (int z = 0; z < nz; ++z) {
    int beta = zb[z];
    for (int n = 0; n < 4; ++n) {
      const TRef& rl = lt.ref[beta][n * 5];
      if (rl.p) {
        const OpLayout& Lay = Lenv.cls[rl.cls];
        for (const Block& b : Lay.blocks) {
          if (b.rs != b.cs) continue;
          jobs.push_back({rl.p + b.off, DL.p + ((size_t)n * Lb.total + Lb.off[b.rs]) * nz + z, b.rows, b.cols, nz,
                          rl.coef});
          mx = std::max(mx, b.rows);
        }
      }
      const TRef& rr = rt.ref[beta][n * 5];
      if (rr.p) {
        const OpLayout& Lay = Renv.cls[rr.cls];
        for (const Block& b : Lay.blocks) {
          if (b.rs != b.cs) continue;
          jobs.push_back({rr.p + b.off, DR.p + ((size_t)n * Rb.total + Rb.off[b.rs]) * nz + z, b.rows, b.cols, nz,
                          rr.coef});
          mx = std::max(mx, b.rows);
        }
      }
    }
  }
  if (!jobs.empty()) {
    DArr<DiagJob> dj;
    dj.upload(jobs, c.stream);
    launch_diag_extract(dj.p, (int)jobs.size(), mx, c.stream);
    cuda_check(cudaGetLastError(), "diag extract");
    cuda_check(cudaStreamSynchronize(c.stream), "sync");
  }
  GemmBuilder g;
  for (size_t pb = 0; pb < P.blocks.size(); ++pb) {
    const Block& ob = P.blocks[pb];
    int n1 = P.b1[pb], n2 = P.b2[pb];
    g.begin(diag + ob.off, ob.cols, ob.rows, ob.cols, 0);
    g.term(DL.p + ((size_t)n1 * Lb.total + Lb.off[ob.rs]) * nz, nz, DR.p + ((size_t)n2 * Rb.total + Rb.off[ob.cs]) * nz,
           nz, nz, 0, 1.0, ob.rows, ob.cols);
    g.end();
  }
  run_builder(c, g);
}

void make_psi(Context& c, const SiteT& TL, const SiteT& TR, const PsiLayout& P, double* psi) {
  cuda_check(cudaMemsetAsync(psi, 0, P.nnz * sizeof(double), c.stream), "memset");
  GemmBuilder g;
  for (size_t pb = 0; pb < P.blocks.size(); ++pb) {
    const Block& ob = P.blocks[pb];
    int ql = ob.rs, n1 = P.b1[pb], n2 = P.b2[pb];
    int tl = TL.blk(ql, n1);
    if (tl < 0) continue;
    int qm = TL.blocks[tl].cs;
    int tr = TR.blk(qm, n2);
    if (tr < 0 || TR.blocks[tr].cs != ob.cs) continue;
    g.begin(psi + ob.off, ob.cols, ob.rows, ob.cols, 0);
    g.term(TL.d.p + TL.blocks[tl].off, TL.R.dim[qm], TR.d.p + TR.blocks[tr].off, ob.cols, TL.R.dim[qm], GT_BN, 1.0,
           ob.rows, ob.cols);
    g.end();
  }
  run_builder(c, g);
}

void prepare_two_site(Context& c, int k) {
  if (k < 0 || k + 1 >= c.K) throw Error(ST_EINVAL, "two-site position out of range");
  for (int j = 0; j < c.K; ++j)
    if (!c.site_set[j]) throw Error(ST_ESTATE, "MPS tensor of site " + std::to_string(j) + " not set");
  env_boundary_left(c, c.left[0]);
  for (int j = 0; j < k; ++j) {
    Tilde t;
    build_tilde_left(c, c.left[j], j, t);
    env_update_left(c, t, c.sites[j], j, c.left[j + 1]);
  }
  env_boundary_right(c, c.right[c.K]);
  for (int j = c.K - 1; j >= k + 2; --j) {
    Tilde t;
    build_tilde_right(c, c.right[j + 1], j, t);
    env_update_right(c, t, c.sites[j], j, c.right[j]);
  }
  // these sums feed only the sigma and the diagonal
  build_tilde_left(c, c.left[k], k, c.lt, true);
  build_tilde_right(c, c.right[k + 2], k + 1, c.rt, true);
  build_sigma_plan(c, c.lt, c.rt, k, c.plan);
  cuda_check(cudaStreamSynchronize(c.stream), "sync");
  c.prepared = k;
}

// ---------------------------------------------------------------- Davidson

struct DotHelper {
  DArr<double> part, out;
  int nblk = 128;
  std::vector<double> host;
  void init(int maxm, cudaStream_t s) {
    part.alloc((size_t)maxm * nblk, s);
    out.alloc(maxm, s);
    host.resize(maxm);
  }
  // dots of rows V[0..m) (stride ldv) with x, returned on host
  const std::vector<double>& dots(Context& c, const double* V, long ldv, int m, const double* x, long n) {
    launch_multidot(V, ldv, m, x, n, part.p, nblk, out.p, c.stream);
    cuda_check(cudaMemcpyAsync(host.data(), out.p, m * sizeof(double), cudaMemcpyDeviceToHost, c.stream), "d2h");
    cuda_check(cudaStreamSynchronize(c.stream), "sync");
    return host;
  }
};

// Davidson on the device: the subspace vectors, their sigma vectors, the projected
// matrix G, the Rayleigh-Ritz eigenproblem (rr_kernel, FP64 Jacobi), the Ritz
// vector, the residual, the correction and its orthogonalisation all stay in device
// memory.  The host reads three scalars per iteration (Ritz value, residual norm and
// norm of the new direction, one 24-byte copy) to decide convergence, and the sigma
// timings (CUDA events) once at the end.
double davidson(Context& c, SigmaPlan& plan, const double* diag, double* psi, const DavidsonOpts& o, int* iters) {
  const long n = plan.psi.nnz;
  const int ms = (int)std::max<long>(2, std::min<long>(std::min(o.max_sub, RR_MAX_SUB), n));
  const int nblk = 128;
  DArr<double> V, S, x, hx, r, t, coef, ocoef, G, part, scal;
  V.alloc((size_t)ms * n, c.stream);
  S.alloc((size_t)ms * n, c.stream);
  x.alloc(n, c.stream);
  hx.alloc(n, c.stream);
  r.alloc(n, c.stream);
  t.alloc(n, c.stream);
  coef.alloc(ms, c.stream);
  ocoef.alloc(ms + 1, c.stream);
  G.alloc((size_t)ms * ms, c.stream);
  part.alloc((size_t)(ms + 1) * nblk, c.stream);
  // scal: [0] Ritz value, [1] |r|^2, [2] |t|^2, [3] |psi|^2, [4] |x|^2
  scal.alloc(8, c.stream);
  cuda_check(cudaMemsetAsync(G.p, 0, G.n * sizeof(double), c.stream), "memset");
  double* th_d = scal.p;
  // sigma vectors timed with CUDA events on the context stream, read after the solve
  std::vector<std::pair<cudaEvent_t, cudaEvent_t>> evs;
  auto event = [&]() {
    cudaEvent_t e;
    cuda_check(cudaEventCreate(&e), "event");
    return e;
  };
  auto release_events = [&]() {
    for (auto& pr : evs) {
      cudaEventDestroy(pr.first);
      cudaEventDestroy(pr.second);
    }
    evs.clear();
  };
  auto sigma_of = [&](const double* in, double* out) {
    evs.push_back({event(), event()});
    cuda_check(cudaEventRecord(evs.back().first, c.stream), "record");
    run_sigma(c, plan, in, out);
    cuda_check(cudaEventRecord(evs.back().second, c.stream), "record");
    c.sigma_flops_total += plan.flops;
    c.sigma_calls++;
  };
  auto read = [&](int i0, int cnt, double* h) {
    cuda_check(cudaMemcpyAsync(h, scal.p + i0, cnt * sizeof(double), cudaMemcpyDeviceToHost, c.stream), "d2h");
    cuda_check(cudaStreamSynchronize(c.stream), "sync");
  };
  auto dots = [&](const double* Vb, long ldv, int m, const double* y, double* out) {
    launch_multidot(Vb, ldv, m, y, n, part.p, nblk, out, c.stream);
  };
  // two passes of classical Gram-Schmidt of t against V[0..m), then |t|^2
  auto orthogonalise = [&](int m) {
    for (int pass = 0; pass < 2; ++pass) {
      dots(V.p, n, m, t.p, ocoef.p);
      launch_sub_combine(V.p, n, m, ocoef.p, n, t.p, c.stream);
    }
    dots(t.p, 0, 1, t.p, scal.p + 2);
  };
  double h3[3] = {0, 0, 0};
  int it = 0;
  double theta = 0;
  const bool use_mlp = c.mlp != nullptr;
  const bool harvest = c.harvest.per_iter > 0 && c.harvest.count < c.harvest.cap;
  std::vector<DArr<double>> sv_x, sv_r;  // saved Ritz vectors / residuals
  std::vector<double> sv_theta, sv_rn;
  try {
    dots(psi, 0, 1, psi, scal.p + 3);
    read(3, 1, h3);
    if (!(h3[0] > 0) || !std::isfinite(h3[0])) throw Error(ST_EINVAL, "Davidson: zero or non-finite start vector");
    launch_scale_rsqrt(n, psi, scal.p + 3, V.p, c.stream);
    sigma_of(V.p, S.p);
    dots(V.p, 0, 1, S.p, ocoef.p);
    launch_gcol(ocoef.p, 1, G.p, ms, 0, c.stream);
    int m = 1;
    double best_rn = 1e300;
    int since_best = 0;
    // learned preconditioner and training-pair collection
    if (use_mlp || harvest) {
      c.mlp_s.reset(new MlpScratch());
      mlp_scratch_build(*c.mlp_s, use_mlp ? c.mlp : nullptr, plan.psi, c.stream);
      mlp_scratch_set_diag(*c.mlp_s, diag, c.stream);
    }
    double prev_rn = 1e300;
    for (; it < o.max_iter; ++it) {
      // Rayleigh-Ritz, Ritz vector, residual, diagonal correction
      if (!launch_rr(G.p, ms, m, coef.p, th_d, c.stream)) throw Error(ST_EINVAL, "Davidson: subspace too large");
      launch_combine_vectors(V.p, n, m, coef.p, n, x.p, c.stream);
      launch_combine_vectors(S.p, n, m, coef.p, n, hx.p, c.stream);
      launch_resid(n, hx.p, x.p, th_d, r.p, c.stream);
      dots(r.p, 0, 1, r.p, scal.p + 1);
      launch_precond_dev(n, r.p, diag, th_d, 1e-8, t.p, c.stream);
      // a full subspace restarts from the Ritz vector (harmless if this iteration
      // turns out converged: x and hx are kept)
      int mb = m;
      if (m == ms) {
        cuda_check(cudaMemcpyAsync(V.p, x.p, n * sizeof(double), cudaMemcpyDeviceToDevice, c.stream), "d2d");
        cuda_check(cudaMemcpyAsync(S.p, hx.p, n * sizeof(double), cudaMemcpyDeviceToDevice, c.stream), "d2d");
        dots(x.p, 0, 1, x.p, scal.p + 4);
        cuda_check(cudaMemsetAsync(G.p, 0, G.n * sizeof(double), c.stream), "memset");
        launch_restart_g(G.p, th_d, scal.p + 4, c.stream);  // x normalised up to rounding
        mb = 1;
      }
      orthogonalise(mb);
      read(0, 3, h3);
      theta = h3[0];
      const double rn = std::sqrt(h3[1]);
      double tn = std::sqrt(h3[2]);
      if (!std::isfinite(rn) || !std::isfinite(theta))
        throw Error(ST_ENOCONV, "Davidson: non-finite residual (iteration " + std::to_string(it) + ", subspace " +
                                    std::to_string(m) + ", theta " + std::to_string(theta) + ")");
      if (rn <= o.tol) break;
      if (harvest && sv_x.size() < 7 && (it == 0 || it == 1 || it == 2 || it == 4 || it == 7 || it == 11 || it == 16)) {
        sv_x.emplace_back();
        sv_r.emplace_back();
        sv_x.back().alloc(n, c.stream);
        sv_r.back().alloc(n, c.stream);
        cuda_check(cudaMemcpyAsync(sv_x.back().p, x.p, n * sizeof(double), cudaMemcpyDeviceToDevice, c.stream), "d2d");
        cuda_check(cudaMemcpyAsync(sv_r.back().p, r.p, n * sizeof(double), cudaMemcpyDeviceToDevice, c.stream), "d2d");
        sv_theta.push_back(theta);
        sv_rn.push_back(rn);
      }
      if (o.stagnation > 0) {
        // only near the operator's rounding floor (tensor-core sigma: ~1e-5 of |theta|)
        if (rn < 0.9 * best_rn) {
          best_rn = rn;
          since_best = 0;
        } else if (++since_best >= o.stagnation && rn < o.floor * std::fabs(theta)) {
          break;
        }
      }
      if (use_mlp) {
        bool learned = false;
        if (rn < prev_rn) learned = mlp_precondition(*c.mlp, *c.mlp_s, r.p, diag, theta, rn, t.p, c.stream);
        if (learned) {
          ++c.mlp_applied;
          orthogonalise(mb);
          read(2, 1, h3 + 2);
          tn = std::sqrt(h3[2]);
        } else {
          // the diagonal correction computed above is the fallback when the residual
          // did not decrease or the network produced a non-finite value
          ++c.mlp_fallbacks;
        }
      }
      prev_rn = rn;
      m = mb;
      if (!(tn > 1e-14)) break;  // subspace exhausted: the Ritz pair is exact in it
      launch_scale_rsqrt(n, t.p, scal.p + 2, V.p + (size_t)m * n, c.stream);
      sigma_of(V.p + (size_t)m * n, S.p + (size_t)m * n);
      dots(V.p, n, m + 1, S.p + (size_t)m * n, ocoef.p);
      launch_gcol(ocoef.p, m + 1, G.p, ms, m, c.stream);
      ++m;
    }
    dots(x.p, 0, 1, x.p, scal.p + 4);
    launch_scale_rsqrt(n, x.p, scal.p + 4, psi, c.stream);
    cuda_check(cudaStreamSynchronize(c.stream), "sync");
    for (auto& pr : evs) {
      float ems = 0;
      cuda_check(cudaEventElapsedTime(&ems, pr.first, pr.second), "elapsed");
      c.sigma_time_total += 1e-3 * ems;
    }
    release_events();
  } catch (...) {
    cudaStreamSynchronize(c.stream);
    release_events();
    throw;
  }
  if (plan.tensor() && plan_error(c, plan)) throw Error(ST_ETIMEOUT, "tensor-core GEMM: a bounded wait ran out");
  if (harvest) {
    Harvest& H = c.harvest;
    for (size_t j = 0; j < sv_x.size() && H.count < H.cap; ++j) {
      const long ns = std::min<long>(H.per_iter, H.cap - H.count);
      const uint64_t key = H.seed * 0x100000001B3ULL + (uint64_t)H.solves * 64 + j;
      // iterates with |x . psi| < 0.5 are skipped: their unit-weight correction is ill-defined
      H.count += mlp_make_pairs(*c.mlp_s, sv_x[j].p, sv_r[j].p, diag, sv_theta[j], sv_rn[j], psi, ns, key,
                                H.F.p + H.count * 5, H.P.p + H.count, H.T.p + H.count, nullptr, 0.5, c.stream);
    }
    ++H.solves;
  }
  if (iters) *iters = it;
  return theta;
}

// <psi|H|psi> / <psi|psi> for the two-site wavefunction of the current MPS at the
// prepared position (the MPS contracted with its own environments)
double expectation(Context& c) {
  if (c.prepared < 0) throw Error(ST_ESTATE, "call gbdmrg_prepare first");
  const int k = c.prepared;
  SigmaPlan& plan = c.plan;
  const long n = plan.psi.nnz;
  DArr<double> psi, sig;
  psi.alloc(n, c.stream);
  sig.alloc(n, c.stream);
  make_psi(c, c.sites[k], c.sites[k + 1], plan.psi, psi.p);
  run_sigma(c, plan, psi.p, sig.p);
  if (plan.tensor() && plan_error(c, plan)) throw Error(ST_ETIMEOUT, "tensor-core GEMM: a bounded wait ran out");
  DotHelper dh;
  dh.init(1, c.stream);
  const double num = dh.dots(c, psi.p, 0, 1, sig.p, n)[0];
  const double den = dh.dots(c, psi.p, 0, 1, psi.p, n)[0];
  if (!(den > 0)) throw Error(ST_ESTATE, "the MPS has zero norm at this position");
  return num / den + c.ecore;
}

// ---------------------------------------------------------------- decimation

double decimate(Context& c, const PsiLayout& P, const double* psi, int M, int direction, SiteT& left, SiteT& right) {
  const Bond& Lb = P.L;
  const Bond& Rb = P.R;
  struct Seg { int q, n, off; };
  std::map<std::pair<int, int>, std::pair<std::vector<Seg>, std::vector<Seg>>> gm;
  for (int ql = 0; ql < Lb.nsec(); ++ql)
    for (int n1 = 0; n1 < 4; ++n1) {
      auto key = std::make_pair(Lb.qa[ql] + LQA[n1], Lb.qb[ql] + LQB[n1]);
      gm[key].first.push_back({ql, n1, 0});
    }
  for (int qr = 0; qr < Rb.nsec(); ++qr)
    for (int n2 = 0; n2 < 4; ++n2) {
      auto key = std::make_pair(Rb.qa[qr] - LQA[n2], Rb.qb[qr] - LQB[n2]);
      gm[key].second.push_back({qr, n2, 0});
    }
  struct Group { int qa, qb, nr, nc; std::vector<Seg> rows, cols; size_t moff, goff; };
  std::vector<Group> groups;
  size_t mtot = 0, gtot = 0;
  for (auto& kv : gm) {
    if (kv.second.first.empty() || kv.second.second.empty()) continue;
    Group g;
    g.qa = kv.first.first;
    g.qb = kv.first.second;
    g.rows = kv.second.first;
    g.cols = kv.second.second;
    g.nr = g.nc = 0;
    for (auto& s : g.rows) { s.off = g.nr; g.nr += Lb.dim[s.q]; }
    for (auto& s : g.cols) { s.off = g.nc; g.nc += Rb.dim[s.q]; }
    int d = direction == 0 ? g.nr : g.nc;
    g.moff = mtot;
    g.goff = gtot;
    mtot += (size_t)g.nr * g.nc;
    gtot += (size_t)d * d;
    groups.push_back(g);
  }
  DArr<double> Mat, Gram;
  Mat.alloc(mtot, c.stream);
  Gram.alloc(gtot, c.stream);
  cuda_check(cudaMemsetAsync(Mat.p, 0, mtot * sizeof(double), c.stream), "memset");
  // gather psi blocks into the dense group matrices
  std::vector<CopyJob> jobs;
  for (auto& g : groups)
    for (auto& rs : g.rows)
      for (auto& cs : g.cols) {
        int pb = P.blk(rs.q, rs.n, cs.n);
        if (pb < 0 || P.blocks[pb].cs != cs.q) continue;
        const Block& b = P.blocks[pb];
        jobs.push_back({psi + b.off, Mat.p + g.moff + (size_t)rs.off * g.nc + cs.off, b.rows, b.cols, b.cols, g.nc, 0,
                        1.0});
      }
  run_copies(c, jobs);
  GemmBuilder gb;
  for (auto& g : groups) {
    double* Mg = Mat.p + g.moff;
    if (direction == 0) {
      gb.begin(Gram.p + g.goff, g.nr, g.nr, g.nr, 0);
      gb.term(Mg, g.nc, Mg, g.nc, g.nc, 0, 1.0, g.nr, g.nr);
    } else {
      gb.begin(Gram.p + g.goff, g.nc, g.nc, g.nc, 0);
      gb.term(Mg, g.nc, Mg, g.nc, g.nr, GT_TA | GT_BN, 1.0, g.nc, g.nc);
    }
    gb.end();
  }
  run_builder(c, gb);
  // eigen-decomposition of every group Gram matrix
  int maxd = 0;
  for (auto& g : groups) maxd = std::max(maxd, direction == 0 ? g.nr : g.nc);
  DArr<double> evals;
  size_t etot = 0;
  for (auto& g : groups) etot += direction == 0 ? g.nr : g.nc;
  evals.alloc(std::max<size_t>(etot, 1), c.stream);
  int lwork = 0;
  solver_check(cusolverDnDsyevd_bufferSize(c.solver, CUSOLVER_EIG_MODE_VECTOR, CUBLAS_FILL_MODE_UPPER, maxd, Gram.p,
                                           maxd, evals.p, &lwork),
               "syevd_bufferSize");
  // the group eigenproblems are independent: spread them over the auxiliary
  // streams (one workspace each), joined back into the context stream
  const int na = Context::kAux;
  DArr<double> work;
  work.alloc((size_t)std::max(lwork, 1) * na, c.stream);
  DArr<int> info;
  info.alloc(groups.size() + 1, c.stream);
  cuda_check(cudaEventRecord(c.aux_ev[na], c.stream), "record");
  for (int a = 0; a < na; ++a) cuda_check(cudaStreamWaitEvent(c.aux[a], c.aux_ev[na], 0), "wait");
  size_t eo = 0;
  std::vector<size_t> eoff(groups.size());
  std::vector<size_t> order(groups.size());
  std::iota(order.begin(), order.end(), 0);
  std::sort(order.begin(), order.end(), [&](size_t x, size_t y) {
    int dx = direction == 0 ? groups[x].nr : groups[x].nc, dy = direction == 0 ? groups[y].nr : groups[y].nc;
    return dx > dy;
  });
  for (size_t gi = 0; gi < groups.size(); ++gi) {
    eoff[gi] = eo;
    eo += direction == 0 ? groups[gi].nr : groups[gi].nc;
  }
  for (size_t q = 0; q < order.size(); ++q) {
    const size_t gi = order[q];
    auto& g = groups[gi];
    int d = direction == 0 ? g.nr : g.nc;
    const int a = (int)(q % na);
    solver_check(cusolverDnDsyevd(c.aux_solver[a], CUSOLVER_EIG_MODE_VECTOR, CUBLAS_FILL_MODE_UPPER, d, Gram.p + g.goff, d,
                                  evals.p + eoff[gi], work.p + (size_t)a * std::max(lwork, 1), lwork, info.p + gi),
                 "syevd");
  }
  for (int a = 0; a < na; ++a) {
    cuda_check(cudaEventRecord(c.aux_ev[a], c.aux[a]), "record");
    cuda_check(cudaStreamWaitEvent(c.stream, c.aux_ev[a], 0), "wait");
  }
  std::vector<double> ev(etot);
  std::vector<int> hinfo(groups.size());
  cuda_check(cudaMemcpyAsync(ev.data(), evals.p, etot * sizeof(double), cudaMemcpyDeviceToHost, c.stream), "d2h");
  if (!groups.empty())
    cuda_check(cudaMemcpyAsync(hinfo.data(), info.p, groups.size() * sizeof(int), cudaMemcpyDeviceToHost, c.stream),
               "d2h");
  cuda_check(cudaStreamSynchronize(c.stream), "sync");
  for (int v : hinfo)
    if (v != 0) throw Error(ST_ENOCONV, "syevd failed in decimation");
  // selection: weights >= 1e-14, sorted by (-w, group, index-from-top); keep M, never split a multiplet
  struct Cand { double w; int g, i; };
  std::vector<Cand> cand;
  double total = 0;
  for (size_t gi = 0; gi < groups.size(); ++gi) {
    int d = direction == 0 ? groups[gi].nr : groups[gi].nc;
    for (int i = 0; i < d; ++i) {
      double w = ev[eoff[gi] + d - 1 - i];
      total += std::max(w, 0.0);
      if (w >= 1e-14) cand.push_back({w, (int)gi, i});
    }
  }
  std::sort(cand.begin(), cand.end(), [](const Cand& a, const Cand& b) {
    if (a.w != b.w) return a.w > b.w;
    if (a.g != b.g) return a.g < b.g;
    return a.i < b.i;
  });
  size_t keep = cand.size();
  if ((long)cand.size() > M) {
    double t = cand[M].w;
    keep = 0;
    for (int i = 0; i < M; ++i)
      if (cand[i].w > t * (1.0 + 1e-8)) keep = i + 1;
  }
  std::vector<int> nk(groups.size(), 0);
  double kept = 0;
  for (size_t i = 0; i < keep; ++i) {
    nk[cand[i].g]++;
    kept += cand[i].w;
  }
  if (keep == 0) throw Error(ST_ENOCONV, "decimation kept no states");
  Bond nb;
  std::vector<int> gsec(groups.size(), -1);
  for (size_t gi = 0; gi < groups.size(); ++gi)
    if (nk[gi] > 0) {
      gsec[gi] = nb.nsec();
      nb.add(groups[gi].qa, groups[gi].qb, nk[gi]);
    }
  left.layout(Lb, nb);
  right.layout(nb, Rb);
  left.d.alloc(left.nnz, c.stream);
  right.d.alloc(right.nnz, c.stream);
  cuda_check(cudaMemsetAsync(left.d.p, 0, left.nnz * sizeof(double), c.stream), "memset");
  cuda_check(cudaMemsetAsync(right.d.p, 0, right.nnz * sizeof(double), c.stream), "memset");
  // product with the kept eigenvectors: kept vectors are the last nk columns of the
  // column-major eigenvector matrix, i.e. rows [d-nk, d) of its row-major view
  size_t ctot = 0;
  std::vector<size_t> coff(groups.size());
  for (size_t gi = 0; gi < groups.size(); ++gi) {
    coff[gi] = ctot;
    ctot += (size_t)nk[gi] * (direction == 0 ? groups[gi].nc : groups[gi].nr);
  }
  DArr<double> Cm;
  Cm.alloc(std::max<size_t>(ctot, 1), c.stream);
  GemmBuilder g2;
  std::vector<CopyJob> out;
  for (size_t gi = 0; gi < groups.size(); ++gi) {
    if (!nk[gi]) continue;
    auto& g = groups[gi];
    int d = direction == 0 ? g.nr : g.nc;
    const double* Uk = Gram.p + g.goff + (size_t)(d - nk[gi]) * d;  // nk x d row-major
    double* Mg = Mat.p + g.moff;
    int s = gsec[gi];
    if (direction == 0) {
      // C = Uk * Mg  (nk x nc)
      g2.begin(Cm.p + coff[gi], g.nc, nk[gi], g.nc, 0);
      g2.term(Uk, d, Mg, g.nc, g.nr, GT_BN, 1.0, nk[gi], g.nc);
      g2.end();
      for (auto& rs : g.rows) {  // A^{n1}[ql, a] = Uk[a][rowoff + i]
        int b = left.blk(rs.q, rs.n);
        out.push_back({Uk + rs.off, left.d.p + left.blocks[b].off, Lb.dim[rs.q], nk[gi], d, nk[gi], 1, 1.0});
      }
      for (auto& cs : g.cols) {  // center[a, n2, qr] = C[a][coloff + j]
        int b = right.blk(s, cs.n);
        if (b < 0 || right.blocks[b].cs != cs.q) continue;
        out.push_back({Cm.p + coff[gi] + cs.off, right.d.p + right.blocks[b].off, nk[gi], Rb.dim[cs.q], g.nc,
                       Rb.dim[cs.q], 0, 1.0});
      }
    } else {
      // C = Mg * Vk^T  (nr x nk)
      g2.begin(Cm.p + coff[gi], nk[gi], g.nr, nk[gi], 0);
      g2.term(Mg, g.nc, Uk, d, g.nc, 0, 1.0, g.nr, nk[gi]);
      g2.end();
      for (auto& cs : g.cols) {  // B^{n2}[a, qr] = Vk[a][coloff + j]
        int b = right.blk(s, cs.n);
        if (b < 0 || right.blocks[b].cs != cs.q) continue;
        out.push_back({Uk + cs.off, right.d.p + right.blocks[b].off, nk[gi], Rb.dim[cs.q], d, Rb.dim[cs.q], 0, 1.0});
      }
      for (auto& rs : g.rows) {  // center[ql, n1, a] = C[rowoff + i][a]
        int b = left.blk(rs.q, rs.n);
        out.push_back({Cm.p + coff[gi] + (size_t)rs.off * nk[gi], left.d.p + left.blocks[b].off, Lb.dim[rs.q], nk[gi],
                       nk[gi], nk[gi], 0, 1.0});
      }
    }
  }
  run_builder(c, g2);
  run_copies(c, out);
  return std::max(0.0, total - kept);
}

// ---------------------------------------------------------------- canonical form

// rows of X (r x cols, row-major) = L * Q with orthonormal rows Q (MGS, twice)
static void lq_rows(int r, int cols, std::vector<double>& X, std::vector<double>& L) {
  L.assign((size_t)r * r, 0.0);
  for (int i = 0; i < r; ++i) {
    double* xi = &X[(size_t)i * cols];
    for (int pass = 0; pass < 2; ++pass)
      for (int j = 0; j < i; ++j) {
        const double* qj = &X[(size_t)j * cols];
        double d = 0;
        for (int e = 0; e < cols; ++e) d += qj[e] * xi[e];
        for (int e = 0; e < cols; ++e) xi[e] -= d * qj[e];
        L[(size_t)i * r + j] += d;
      }
    double nr = 0;
    for (int e = 0; e < cols; ++e) nr += xi[e] * xi[e];
    nr = std::sqrt(nr);
    if (!(nr > 1e-300)) throw Error(ST_EINVAL, "initial MPS tensor is rank deficient");
    for (int e = 0; e < cols; ++e) xi[e] /= nr;
    L[(size_t)i * r + i] = nr;
  }
}

void right_canonicalize(Context& c) {
  std::vector<std::vector<double>> H(c.K);
  for (int k = 0; k < c.K; ++k) {
    H[k].resize(c.sites[k].nnz);
    if (c.sites[k].nnz)
      cuda_check(cudaMemcpy(H[k].data(), c.sites[k].d.p, c.sites[k].nnz * sizeof(double), cudaMemcpyDeviceToHost),
                 "d2h");
  }
  for (int k = c.K - 1; k >= 2; --k) {
    SiteT& A = c.sites[k];
    SiteT& P = c.sites[k - 1];
    for (int q = 0; q < A.L.nsec(); ++q) {
      int r = A.L.dim[q];
      int cols = 0;
      std::vector<int> bl;
      for (int n = 0; n < 4; ++n) {
        int b = A.blk(q, n);
        if (b >= 0) { bl.push_back(b); cols += A.blocks[b].cols; }
      }
      if (cols < r) throw Error(ST_EINVAL, "initial MPS bond larger than what the next site supplies");
      std::vector<double> X((size_t)r * cols), L;
      int co = 0;
      for (int b : bl) {
        const Block& B = A.blocks[b];
        for (int i = 0; i < r; ++i)
          for (int j = 0; j < B.cols; ++j) X[(size_t)i * cols + co + j] = H[k][B.off + (long)i * B.cols + j];
        co += B.cols;
      }
      lq_rows(r, cols, X, L);
      co = 0;
      for (int b : bl) {
        const Block& B = A.blocks[b];
        for (int i = 0; i < r; ++i)
          for (int j = 0; j < B.cols; ++j) H[k][B.off + (long)i * B.cols + j] = X[(size_t)i * cols + co + j];
        co += B.cols;
      }
      // previous site blocks (., ., q) <- block * L
      for (size_t b = 0; b < P.blocks.size(); ++b) {
        const Block& B = P.blocks[b];
        if (B.cs != q) continue;
        std::vector<double> tmp((size_t)B.rows * r, 0.0);
        for (int i = 0; i < B.rows; ++i)
          for (int j = 0; j < r; ++j) {
            double s = 0;
            for (int l = 0; l < r; ++l) s += H[k - 1][B.off + (long)i * r + l] * L[(size_t)l * r + j];
            tmp[(size_t)i * r + j] = s;
          }
        std::copy(tmp.begin(), tmp.end(), H[k - 1].begin() + B.off);
      }
    }
  }
  for (int k = 0; k < c.K; ++k)
    if (c.sites[k].nnz)
      cuda_check(cudaMemcpy(c.sites[k].d.p, H[k].data(), c.sites[k].nnz * sizeof(double), cudaMemcpyHostToDevice),
                 "h2d");
}

// ---------------------------------------------------------------- sweeps

double two_site_step(Context& c, int k, int dir, int M, const DavidsonOpts& o, bool free_used, int* iters,
                     double* discarded, const double* psi0, double* psi_out, long* nnz_out) {
  if (!c.left[k].valid || !c.right[k + 2].valid)
    throw Error(ST_ESTATE, "environments of the two-site step are not built");
  auto now = [&]() {
    cuda_check(cudaStreamSynchronize(c.stream), "sync");
    return std::chrono::steady_clock::now();
  };
  auto t0 = now();
  double f0 = c.other_flops_total + c.sigma_flops_total;
  auto lap = [&](int ph) {
    auto t1 = now();
    c.phase_s[ph] += std::chrono::duration<double>(t1 - t0).count();
    const double f1 = c.other_flops_total + c.sigma_flops_total;
    c.phase_flops[ph] += f1 - f0;
    t0 = t1;
    f0 = f1;
  };
  // the side that the environment update does not use feeds only the sigma and the diagonal
  Tilde lt, rt;
  cudaEvent_t ev0 = nullptr, ev1 = nullptr;
  cuda_check(cudaEventCreate(&ev0), "event");
  cuda_check(cudaEventCreate(&ev1), "event");
  cuda_check(cudaEventRecord(ev0, c.stream), "event");
  build_tilde_left(c, c.left[k], k, lt, dir == 1);
  build_tilde_right(c, c.right[k + 2], k + 1, rt, dir == 0);
  cuda_check(cudaEventRecord(ev1, c.stream), "event");
  const double f_tilde = c.other_flops_total + c.sigma_flops_total;
  // no synchronisation here: the host part of the sigma plan overlaps the GPU work of the
  // W-contracted sums (all device work is ordered on the context stream); the sums' phase
  // time is their event time, the plan's the rest until the plan is on the device
  SigmaPlan plan;
  build_sigma_plan(c, lt, rt, k, plan);
  {
    auto t1 = now();
    float ms = 0.f;
    cuda_check(cudaEventElapsedTime(&ms, ev0, ev1), "event time");
    cudaEventDestroy(ev0);
    cudaEventDestroy(ev1);
    const double total = std::chrono::duration<double>(t1 - t0).count(), tsum = std::min(total, 1e-3 * ms);
    const double f1 = c.other_flops_total + c.sigma_flops_total;
    c.phase_s[0] += tsum;
    c.phase_flops[0] += f_tilde - f0;
    c.phase_s[1] += total - tsum;
    c.phase_flops[1] += f1 - f_tilde;
    t0 = t1;
    f0 = f1;
  }
  DArr<double> psi, diag;
  psi.alloc(plan.psi.nnz, c.stream);
  diag.alloc(plan.psi.nnz, c.stream);
  if (psi0)
    cuda_check(cudaMemcpyAsync(psi.p, psi0, plan.psi.nnz * sizeof(double), cudaMemcpyDeviceToDevice, c.stream), "d2d");
  else
    make_psi(c, c.sites[k], c.sites[k + 1], plan.psi, psi.p);
  compute_diag(c, lt, rt, k, plan.psi, diag.p);
  lap(2);
  DavidsonOpts od = o;
  if (plan.tensor() && od.stagnation == 0) od.stagnation = 6;
  // the residual of a one-pass BF16 operator stalls near 1e-2 |theta| (operands
  // rounded to 8 bits); sliced operands near 1e-5
  const bool one_pass = c.precision == 1 || c.precision == 4;
  od.floor = one_pass ? 2e-2 : 2e-4;
  // Refinement: after the solve with the tensor-core operator, the Ritz vector
  // starts a second solve with the more accurate operator of precision
  // refine_precision (the residual and the eigenvalue of that solve are those of the
  // accurate operator); at most refine_iters iterations of the budget go to it
  const bool refine = plan.tensor() && c.refine_precision >= 0 && c.refine_precision != c.precision;
  if (refine) od.max_iter = std::max(1, o.max_iter - c.refine_iters);
  double e = davidson(c, plan, diag.p, psi.p, od, iters);
  if (refine) {
    const int keep = c.precision;
    plan = SigmaPlan();
    c.precision = c.refine_precision;
    try {
      // the sums that fed only the tensor-core sigma are formed again in FP64 for an
      // FP64 refinement
      if (c.precision == 0) {
        if (dir == 0)
          build_tilde_right(c, c.right[k + 2], k + 1, rt, true);
        else
          build_tilde_left(c, c.left[k], k, lt, true);
      }
      build_sigma_plan(c, lt, rt, k, plan);
      DavidsonOpts o2 = o;
      o2.max_iter = std::max(1, std::min(c.refine_iters, o.max_iter - (iters ? *iters : 0)));
      o2.stagnation = plan.tensor() ? 6 : 0;
      o2.floor = 2e-4;
      int it2 = 0;
      e = davidson(c, plan, diag.p, psi.p, o2, &it2);
      if (iters) *iters += it2;
    } catch (...) {
      c.precision = keep;
      throw;
    }
    c.precision = keep;
  }
  if (psi_out)
    cuda_check(cudaMemcpyAsync(psi_out, psi.p, plan.psi.nnz * sizeof(double), cudaMemcpyDeviceToDevice, c.stream),
               "d2d");
  if (nnz_out) *nnz_out = plan.psi.nnz;
  lap(3);
  SiteT A, B;
  double dw = decimate(c, plan.psi, psi.p, M, dir, A, B);
  if (discarded) *discarded = dw;
  c.sites[k] = std::move(A);
  c.sites[k + 1] = std::move(B);
  // the H_eff work lists (tens of GB for tensor-core plans of large bonds) are not needed
  // by the environment update
  plan = SigmaPlan();
  psi.release();
  diag.release();
  lap(4);
  if (dir == 0) {
    env_update_left(c, lt, c.sites[k], k, c.left[k + 1]);
    if (free_used) c.right[k + 2] = Env();
  } else {
    env_update_right(c, rt, c.sites[k + 1], k + 1, c.right[k + 1]);
    if (free_used) c.left[k + 1] = Env();
  }
  lap(5);
  c.prepared = -1;
  return e;
}

double count_sigma_flops(const MPO& mpo, int k, const Bond& Lb, const Bond& Rb) {
  const auto& mid = mpo.bonds[k + 1];
  // which (n, n') site-operator slots of the W-contracted operators are non-zero
  std::vector<uint16_t> lmask(mid.size(), 0), rmask(mid.size(), 0);
  for (const auto& e : mpo.W[k])
    for (int nn = 0; nn < 16; ++nn)
      if (e.m[nn] != 0.0) lmask[e.col] |= (uint16_t)(1u << nn);
  for (const auto& e : mpo.W[k + 1])
    for (int nn = 0; nn < 16; ++nn)
      if (e.m[nn] != 0.0) rmask[e.row] |= (uint16_t)(1u << nn);
  // The count of one bond state depends only on its quantum-number change and its two
  // slot patterns, so states are grouped by that key.  Every term is an integer and all
  // sums stay far below 2^53, so the total is exact in any order.
  std::map<std::tuple<int, int, uint16_t, uint16_t>, long> mult;
  for (size_t beta = 0; beta < mid.size(); ++beta)
    mult[std::make_tuple(mid[beta].dna, mid[beta].dnb, rmask[beta], lmask[beta])]++;
  double fl = 0;
  std::vector<char> xhas((size_t)Lb.nsec() * 16);
  for (const auto& km : mult) {
    const int da = std::get<0>(km.first), db = std::get<1>(km.first);
    const uint16_t rm = std::get<2>(km.first), lm = std::get<3>(km.first);
    double f = 0;
    std::fill(xhas.begin(), xhas.end(), 0);
    for (int qlp = 0; qlp < Lb.nsec(); ++qlp)
      for (int n1p = 0; n1p < 4; ++n1p)
        for (int n2 = 0; n2 < 4; ++n2) {
          int qr = Rb.find(Lb.qa[qlp] + LQA[n1p] + LQA[n2] + da, Lb.qb[qlp] + LQB[n1p] + LQB[n2] + db);
          if (qr < 0) continue;
          for (int n2p = 0; n2p < 4; ++n2p) {
            if (!((rm >> (n2 * 4 + n2p)) & 1)) continue;
            int qrp = Rb.find(Lb.qa[qlp] + LQA[n1p] + LQA[n2p], Lb.qb[qlp] + LQB[n1p] + LQB[n2p]);
            if (qrp < 0) continue;
            f += 2.0 * Rb.dim[qr] * Lb.dim[qlp] * Rb.dim[qrp];
            xhas[(qlp * 4 + n1p) * 4 + n2] = 1;
          }
        }
    for (int ql = 0; ql < Lb.nsec(); ++ql)
      for (int n1 = 0; n1 < 4; ++n1)
        for (int n2 = 0; n2 < 4; ++n2) {
          int qr = Rb.find(Lb.qa[ql] + LQA[n1] + LQA[n2], Lb.qb[ql] + LQB[n1] + LQB[n2]);
          if (qr < 0) continue;
          for (int n1p = 0; n1p < 4; ++n1p) {
            if (!((lm >> (n1 * 4 + n1p)) & 1)) continue;
            // the W-contracted operator changes the quantum number by dQ_beta - q(n1) + q(n1')
            int qlp = Lb.find(Lb.qa[ql] - (da - LQA[n1] + LQA[n1p]), Lb.qb[ql] - (db - LQB[n1] + LQB[n1p]));
            if (qlp < 0 || !xhas[(qlp * 4 + n1p) * 4 + n2]) continue;
            f += 2.0 * Lb.dim[ql] * Rb.dim[qr] * Lb.dim[qlp];
          }
        }
    fl += f * (double)km.second;
  }
  return fl;
}

void run_sweeps(Context& c, int nsweeps, const int* M, const double* tol, int max_iter, SweepStats& st) {
  if (c.K < 3) throw Error(ST_EINVAL, "sweeps need K >= 3");
  for (int j = 0; j < c.K; ++j)
    if (!c.site_set[j]) throw Error(ST_ESTATE, "MPS tensor of site " + std::to_string(j) + " not set");
  c.prepared = -1;
  c.have_plan = false;
  right_canonicalize(c);
  env_boundary_left(c, c.left[0]);
  env_boundary_right(c, c.right[c.K]);
  for (int j = c.K - 1; j >= 2; --j) {
    Tilde t;
    build_tilde_right(c, c.right[j + 1], j, t);
    env_update_right(c, t, c.sites[j], j, c.right[j]);
  }
  const int K = c.K;
  for (int s = 0; s < nsweeps; ++s) {
    auto t0 = std::chrono::steady_clock::now();
    double f0 = c.sigma_flops_total, s0 = c.sigma_time_total;
    double dmax = 0, e = 0;
    int iters = 0;
    DavidsonOpts o;
    o.tol = tol[s];
    o.max_iter = max_iter;
    auto step = [&](int k, int dir) {
      int it = 0;
      double dw = 0;
      try {
        e = two_site_step(c, k, dir, M[s], o, true, &it, &dw);
      } catch (const Error& err) {
        throw Error(err.code, std::string(err.what()) + " (sweep " + std::to_string(s) + ", sites " +
                                  std::to_string(k) + "," + std::to_string(k + 1) + ", direction " +
                                  std::to_string(dir) + ", M " + std::to_string(M[s]) + ", precision " +
                                  std::to_string(c.precision) + ")");
      }
      iters += it;
      dmax = std::max(dmax, dw);
    };
    for (int k = 0; k <= K - 3; ++k) step(k, 0);
    if (!c.right[K].valid) env_boundary_right(c, c.right[K]);
    for (int k = K - 2; k >= 2; --k) step(k, 1);
    {
      // Refinement of the mixed-precision sweep: the last step (sites 1, 2,
      // small bonds next to the edge) is solved with the FP64 sigma, so the
      // reported energy is an FP64-converged eigenvalue (residual checked in
      // FP64) of the basis the tensor-core sweep produced.
      const int keep = c.precision;
      c.precision = 0;
      try {
        step(1, 1);
      } catch (...) {
        c.precision = keep;
        throw;
      }
      c.precision = keep;
    }
    cuda_check(cudaStreamSynchronize(c.stream), "sync");
    auto t1 = std::chrono::steady_clock::now();
    st.energy.push_back(e + c.ecore);
    st.discarded.push_back(dmax);
    st.seconds.push_back(std::chrono::duration<double>(t1 - t0).count());
    st.sigma_flops.push_back(c.sigma_flops_total - f0);
    st.sigma_seconds.push_back(c.sigma_time_total - s0);
    st.davidson_iters.push_back(iters);
  }
}

}  // namespace gbdmrg
