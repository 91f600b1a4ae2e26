// Mixed-precision sigma vector on the tensor cores (tcgen05, BF16 operands,
// FP32 accumulation).  Same two-stage contraction as the FP64 plan:
//   stage 1: X_beta^T[qr, ql'] = sum_{n2'} Rt_beta^{n2 n2'}[qr, qr'] psi[ql', n1', n2', qr']^T
//   stage 2: sigma[ql, qr]   += sum_{beta, n1'} Lt_beta^{n1 n1'}[ql, ql'] X_beta^T[qr, ql']^T
// with every operand stored as 1 or 3 BF16 slices (x = s0 + s1 + s2, each the
// BF16 rounding of the remainder).  With 3 slices the products s_i t_j with
// i + j <= 2 are summed (6 tensor-core products), which carries the operands
// to about 2^-24 relative accuracy; with 1 slice it is a single BF16 pass.
// Coefficients +-1 of the W-contracted operators become the negate bit of the
// instruction descriptor; other coefficients are folded into a scaled copy.
#include <cuda_bf16.h>

#include <algorithm>
#include <atomic>
#include <cmath>
#include <cstdint>
#include <cstring>
#include <exception>
#include <limits>
#include <map>
#include <mutex>
#include <thread>
#include <unordered_map>
#include <unordered_set>

#include "engine.hpp"
#include "kernels_tc.hpp"
#include "kernels_tma.hpp"

namespace gbdmrg {

namespace {

inline int pad8(int x) { return (x + 7) & ~7; }

// FP64 block -> nsl BF16 slices; writes wcols columns per row (the block's columns
// and its zero padding), rows ldd elements apart in the destination
struct ConvJob {
  const double* src;
  __nv_bfloat16* dst;
  long slice_stride;
  int rows, cols, lds, ldd, nsl;
  double scale;
  int wcols;
};

// Elements of a job spread over the grid (32-bit division when the job has fewer than
// 2^31 elements, as every job of these layouts has).  The FP64 value y is split once into
// a + lo (two FP32 values, a = fl32(y), lo = fl32(y - a)), and the BF16 slices are taken
// from a by exact FP32 subtractions, lo entering the last slice: two FP64 operations per
// element instead of several per slice (the FP64 units of this GPU issue at a small
// fraction of the FP32 rate).  The slices carry y to ~2^-25 relative for three slices,
// as a direct FP64 splitting does.
__device__ __forceinline__ void conv_element(const ConvJob& jb, long i, int j) {
  const double y = j < jb.cols ? jb.scale * jb.src[i * jb.lds + j] : 0.0;
  float a = __double2float_rn(y);
  const float lo = jb.nsl > 1 ? __double2float_rn(y - (double)a) : 0.0f;
  __nv_bfloat16* d = jb.dst + i * jb.ldd + j;
  for (int sl = 0; sl < jb.nsl; ++sl) {
    const __nv_bfloat16 h = __float2bfloat16_rn(sl + 1 == jb.nsl ? a + lo : a);
    d[(long)sl * jb.slice_stride] = h;
    a -= __bfloat162float(h);
  }
}

__global__ void conv_kernel(const ConvJob* __restrict__ jobs) {
  const ConvJob jb = jobs[blockIdx.y];
  const long n = (long)jb.rows * jb.wcols;
  if (n < (1L << 31)) {
    const unsigned w = (unsigned)jb.wcols;
    for (unsigned e = blockIdx.x * blockDim.x + threadIdx.x; e < (unsigned)n; e += gridDim.x * blockDim.x) {
      const unsigned i = e / w;
      conv_element(jb, (long)i, (int)(e - i * w));
    }
  } else {
    for (long e = (long)blockIdx.x * blockDim.x + threadIdx.x; e < n; e += (long)gridDim.x * blockDim.x)
      conv_element(jb, e / jb.wcols, (int)(e % jb.wcols));
  }
}

// transposed gather FP32 -> FP64: dst[i * cols + j] = src[j * lds + i]
struct UnconvJob {
  const float* src;
  double* dst;
  int rows, cols, lds;
};

__global__ void unconv_kernel(const UnconvJob* __restrict__ jobs) {
  const UnconvJob jb = jobs[blockIdx.y];
  const long n = (long)jb.rows * jb.cols;
  for (long e = (long)blockIdx.x * blockDim.x + threadIdx.x; e < n; e += (long)gridDim.x * blockDim.x) {
    const int i = (int)(e / jb.cols), j = (int)(e % jb.cols);
    jb.dst[e] = (double)jb.src[(long)j * jb.lds + i];
  }
}

// blocks per job of the per-job copy kernels (blockIdx.y = job): with many jobs one block
// each (its threads stride over the job), so that no launch holds thousands of idle
// blocks sized for its largest job; with few jobs enough blocks for the largest
static long job_blocks(int njobs, long maxel) {
  if (njobs >= 1024) return 1;
  return std::min<long>(std::max<long>(1, (maxel + 255) / 256), 64);
}

void launch_unconv(const UnconvJob* jobs, int njobs, long maxel, cudaStream_t s) {
  for (int o0 = 0; o0 < njobs; o0 += 65535) {
    int no = std::min(65535, njobs - o0);
    const long g = job_blocks(njobs, maxel);
    unconv_kernel<<<dim3((unsigned)g, no), 256, 0, s>>>(jobs + o0);
    count_launches(1);
  }
  cuda_check(cudaGetLastError(), "unconv launch");
}

// zero n elements at p + s * stride for every slice s < nsl
struct ZeroJob {
  __nv_bfloat16* p;
  long n, stride;
  int nsl;
};

__global__ void zero_kernel(const ZeroJob* __restrict__ jobs) {
  const ZeroJob jb = jobs[blockIdx.y];
  const __nv_bfloat16 z = __float2bfloat16_rn(0.0f);
  for (int sl = 0; sl < jb.nsl; ++sl)
    for (long e = (long)blockIdx.x * blockDim.x + threadIdx.x; e < jb.n; e += (long)gridDim.x * blockDim.x)
      jb.p[sl * jb.stride + e] = z;
}

void launch_zero(const ZeroJob* jobs, int njobs, long maxel, cudaStream_t s) {
  for (int o0 = 0; o0 < njobs; o0 += 65535) {
    int no = std::min(65535, njobs - o0);
    const long g = job_blocks(njobs, maxel);
    zero_kernel<<<dim3((unsigned)g, no), 256, 0, s>>>(jobs + o0);
    count_launches(1);
  }
  cuda_check(cudaGetLastError(), "zero launch");
}

void launch_conv(const DArr<ConvJob>& jobs, int njobs, long maxel, cudaStream_t s) {
  for (int o0 = 0; o0 < njobs; o0 += 65535) {
    int no = std::min(65535, njobs - o0);
    const long g = job_blocks(njobs, maxel);
    conv_kernel<<<dim3((unsigned)g, no), 256, 0, s>>>(jobs.p + o0);
    count_launches(1);
  }
  cuda_check(cudaGetLastError(), "conv launch");
}

struct TcBuilder {
  std::vector<TcTile> tiles;
  std::vector<TcTask> tasks;
  std::vector<TcTerm> terms;
  void begin(const TcTask& t) {
    tasks.push_back(t);
    tasks.back().t0 = tasks.back().t1 = (int)terms.size();
  }
  void term(const __nv_bfloat16* A, long sA, int lda, const __nv_bfloat16* B, long sB, int ldb, int k, bool neg,
            int nsl) {
    if (k <= 0) return;
    terms.push_back({A, B, sA, sB, lda, ldb, k, neg ? 1 : 0, nsl});
    tasks.back().t1 = (int)terms.size();
  }
  bool end() {
    TcTask& t = tasks.back();
    if (t.t1 == t.t0) { tasks.pop_back(); return false; }
    const int idx = (int)tasks.size() - 1;
    for (int r0 = 0; r0 < t.m; r0 += TC_TILE_M)
      for (int c0 = 0; c0 < t.n; c0 += TC_TILE_N) tiles.push_back({idx, r0, c0});
    return true;
  }
};

}  // namespace

struct TcPlan {
  DArr<TcTile> tiles;
  DArr<TcTask> tasks;
  DArr<TcTerm> terms;
  int ntiles = 0;
  // host copies, kept when the plan may be fused into a batched launch
  std::vector<TcTile> htiles;
  std::vector<TcTask> htasks;
  std::vector<TcTerm> hterms;
  // regions of the shared X buffer to clear before this launch (stage 1 of a
  // multi-chunk plan: blocks of X that no term of this chunk writes)
  DArr<ZeroJob> zeros;
  std::vector<ZeroJob> hzeros;
  int nzeros = 0;
  long zmax = 0;
};

void run_zeros(const TcPlan& tp, cudaStream_t s) {
  if (tp.nzeros) launch_zero(tp.zeros.p, tp.nzeros, tp.zmax, s);
}

struct MixedPlan {
  int nsl = 1;
  DArr<__nv_bfloat16> psi_b, X_b, mirror;
  DArr<float> sig_f;
  DArr<ConvJob> psi_jobs;
  DArr<UnconvJob> sig_jobs;
  std::vector<ConvJob> h_psi_jobs;
  std::vector<UnconvJob> h_sig_jobs;
  int n_psi_jobs = 0, n_sig_jobs = 0;
  long psi_maxel = 0, sig_maxel = 0;
  long sig_total = 0;
  std::vector<TcPlan> stage1, stage2;
  DArr<int> err;
  // stacked right operands of stage 1 (stage1_stacked): nsl slices of rs_total elements
  DArr<__nv_bfloat16> rstack;
  long rs_total = 0;
};

void mixed_plan_free(MixedPlan* p) { delete p; }

// padded BF16 layout of one operator class: per-block offsets (elements)
static std::vector<long> padded_offsets(const OpLayout& L, long* total) {
  std::vector<long> off(L.blocks.size());
  long t = 0;
  for (size_t b = 0; b < L.blocks.size(); ++b) {
    off[b] = t;
    t += (long)L.blocks[b].rows * pad8(L.blocks[b].cols);
  }
  *total = t;
  return off;
}

namespace {

// BF16 mirror of the operators referenced by a W-contracted side
struct MirrorRef {
  long off = -1;      // element offset of slice 0 in the mirror buffer
  long stride = 0;    // slice stride
  bool neg = false;
  const std::vector<long>* boff = nullptr;  // padded block offsets of its class
};

}  // namespace

void build_mixed_plan(Context& c, Tilde& lt, Tilde& rt, int k, SigmaPlan& plan, int nsl) {
  const auto& mid = c.mpo.bonds[k + 1];
  Env& Lenv = *lt.env;
  Env& Renv = *rt.env;
  const Bond& Lb = Lenv.bond;
  const Bond& Rb = Renv.bond;
  auto* mx = new MixedPlan();
  plan.mx.reset(mx);
  mx->nsl = nsl;
  PsiLayout& P = plan.psi;
  const int nL = Lb.nsec();
  // ---- operator mirrors (one per distinct referenced operator and scale)
  std::vector<std::vector<long>> loff(Lenv.cls.size()), roff(Renv.cls.size());
  std::vector<long> lsz(Lenv.cls.size()), rsz(Renv.cls.size());
  for (size_t i = 0; i < Lenv.cls.size(); ++i) loff[i] = padded_offsets(Lenv.cls[i], &lsz[i]);
  for (size_t i = 0; i < Renv.cls.size(); ++i) roff[i] = padded_offsets(Renv.cls[i], &rsz[i]);
  struct MirrorKeyHash {
    size_t operator()(const std::pair<const double*, double>& k) const {
      uint64_t b;
      std::memcpy(&b, &k.second, sizeof b);
      return std::hash<uint64_t>()((uint64_t)(uintptr_t)k.first * 0x9e3779b97f4a7c15ULL ^ b);
    }
  };
  std::unordered_map<std::pair<const double*, double>, MirrorRef, MirrorKeyHash> mref;
  long mtot = 0;
  // mirrors in the order of their first reference: (operator, scale, class, side, offset)
  struct NewMirror {
    const double* p;
    double scale;
    int cls;
    bool left;
    long off;
  };
  std::vector<NewMirror> created;
  std::vector<std::array<MirrorRef, 16>> lm(mid.size()), rm(mid.size());
  auto mirror_of = [&](const TRef& r, bool left) -> MirrorRef {
    const double a = std::fabs(r.coef);
    const double scale = a == 1.0 ? 1.0 : r.coef;
    auto key = std::make_pair(r.p, scale);
    auto it = mref.find(key);
    MirrorRef m;
    if (it == mref.end()) {
      const long sz = left ? lsz[r.cls] : rsz[r.cls];
      m.off = mtot;
      m.stride = sz;
      m.boff = left ? &loff[r.cls] : &roff[r.cls];
      mtot += sz * nsl;
      mref.emplace(key, m);
      created.push_back({r.p, scale, r.cls, left, m.off});
    } else m = it->second;
    m.neg = (a == 1.0 && r.coef < 0);
    return m;
  };
  const bool stacked = c.stage1_stacked;
  for (size_t beta = 0; beta < mid.size(); ++beta)
    for (int nn = 0; nn < 16; ++nn) {
      if (lt.ref[beta][nn].p) lm[beta][nn] = mirror_of(lt.ref[beta][nn], true);
      if (rt.ref[beta][nn].p && !stacked) rm[beta][nn] = mirror_of(rt.ref[beta][nn], false);
    }
  // one conversion job per block of every mirror, filled on host threads (each mirror's
  // jobs are contiguous, in the order the mirrors were first referenced)
  mx->mirror.alloc(std::max<long>(mtot, 8), c.stream);
  std::vector<size_t> jstart(created.size() + 1, 0);
  for (size_t i = 0; i < created.size(); ++i)
    jstart[i + 1] = jstart[i] + (created[i].left ? Lenv.cls[created[i].cls] : Renv.cls[created[i].cls]).blocks.size();
  std::vector<ConvJob> conv(jstart.back());
  long maxel = 0;
  {
    std::mutex mu;
    auto fill = [&](size_t lo, size_t hi) {
      long mymax = 0;
      for (size_t i = lo; i < hi; ++i) {
        const NewMirror& nm = created[i];
        const OpLayout& L = nm.left ? Lenv.cls[nm.cls] : Renv.cls[nm.cls];
        const long sz = nm.left ? lsz[nm.cls] : rsz[nm.cls];
        const std::vector<long>& boff = nm.left ? loff[nm.cls] : roff[nm.cls];
        for (size_t b = 0; b < L.blocks.size(); ++b) {
          const Block& B = L.blocks[b];
          conv[jstart[i] + b] = ConvJob{nm.p + B.off, mx->mirror.p + nm.off + boff[b], sz, B.rows, B.cols, B.cols,
                                        pad8(B.cols), nsl, nm.scale, pad8(B.cols)};
          mymax = std::max<long>(mymax, (long)B.rows * pad8(B.cols));
        }
      }
      std::lock_guard<std::mutex> lk(mu);
      maxel = std::max(maxel, mymax);
    };
    const size_t nt = std::max<size_t>(1, std::min<size_t>({std::max(1u, std::thread::hardware_concurrency()), 16,
                                                             created.size() / 256 + 1}));
    std::vector<std::thread> pool;
    for (size_t t = 1; t < nt; ++t) pool.emplace_back(fill, created.size() * t / nt, created.size() * (t + 1) / nt);
    fill(0, created.size() / nt);
    for (auto& th : pool) th.join();
  }
  {
    DArr<ConvJob> dj;
    dj.upload(conv, c.stream);
    if (!conv.empty()) launch_conv(dj, (int)conv.size(), maxel, c.stream);
    cuda_check(cudaStreamSynchronize(c.stream), "sync");
  }
  // ---- group layout.  psi reshaped to (l n1) x (n2 r) is block diagonal in the
  // quantum number g of the cut; per group the row blocks (ql, n1) and column
  // blocks (n2, qr) are stacked (each padded to a multiple of 8) into one matrix
  // Psi_g (R_g x C_g).  X_beta^T and sigma^T use the same stacked blocks, so the
  // tensor-core tiles span a whole group instead of one small block.
  std::map<std::pair<int, int>, int> gidx;
  std::vector<std::pair<int, int>> gq;
  std::vector<std::vector<std::array<int, 3>>> grow, gcol;  // (ql, n1, off), (n2, qr, off)
  std::vector<int> gR, gC;
  {
    std::map<std::pair<int, int>, std::pair<std::vector<std::array<int, 3>>, std::vector<std::array<int, 3>>>> tmp;
    for (int ql = 0; ql < nL; ++ql)
      for (int n1 = 0; n1 < 4; ++n1) tmp[{Lb.qa[ql] + LQA[n1], Lb.qb[ql] + LQB[n1]}].first.push_back({ql, n1, 0});
    for (int qr = 0; qr < Rb.nsec(); ++qr)
      for (int n2 = 0; n2 < 4; ++n2) tmp[{Rb.qa[qr] - LQA[n2], Rb.qb[qr] - LQB[n2]}].second.push_back({n2, qr, 0});
    for (auto& kv : tmp) {
      if (kv.second.first.empty() || kv.second.second.empty()) continue;
      gidx[kv.first] = (int)gq.size();
      gq.push_back(kv.first);
      auto rows = kv.second.first, cols = kv.second.second;
      int R = 0, C = 0;
      for (auto& r : rows) { r[2] = R; R += pad8(Lb.dim[r[0]]); }
      for (auto& cc : cols) { cc[2] = C; C += pad8(Rb.dim[cc[1]]); }
      grow.push_back(rows);
      gcol.push_back(cols);
      gR.push_back(R);
      gC.push_back(C);
    }
  }
  const int ng = (int)gq.size();
  // (ql, n1) -> (group, row offset); (n2, qr) -> (group, col offset)
  std::vector<std::array<int, 2>> rpos((size_t)nL * 4, {-1, 0}), cpos((size_t)Rb.nsec() * 4, {-1, 0});
  for (int g = 0; g < ng; ++g) {
    for (auto& r : grow[g]) rpos[r[0] * 4 + r[1]] = {g, r[2]};
    for (auto& cc : gcol[g]) cpos[cc[1] * 4 + cc[0]] = {g, cc[2]};
  }
  auto group_of = [&](int a, int b) {
    auto it = gidx.find({a, b});
    return it == gidx.end() ? -1 : it->second;
  };
  std::vector<long> goff(ng), sgoff(ng);
  long ptot = 0, stot = 0;
  for (int g = 0; g < ng; ++g) {
    goff[g] = ptot;
    ptot += (long)gR[g] * gC[g];
    sgoff[g] = stot;
    stot += (long)gC[g] * gR[g];
  }
  mx->psi_b.alloc(std::max<long>(ptot * nsl, 8), c.stream);
  cuda_check(cudaMemsetAsync(mx->psi_b.p, 0, mx->psi_b.n * sizeof(__nv_bfloat16), c.stream), "memset");
  mx->sig_total = std::max<long>(stot, 1);
  mx->sig_f.alloc(mx->sig_total, c.stream);
  {
    std::vector<ConvJob> pj;
    std::vector<UnconvJob> sj;
    for (size_t b = 0; b < P.blocks.size(); ++b) {
      const Block& B = P.blocks[b];
      const int n1 = P.b1[b], n2 = P.b2[b];
      const auto rp = rpos[B.rs * 4 + n1];
      const auto cp = cpos[B.cs * 4 + n2];
      if (rp[0] < 0 || rp[0] != cp[0]) throw Error(ST_ECUDA, "internal: psi block outside its group");
      const int g = rp[0];
      pj.push_back({plan.in.p + B.off, mx->psi_b.p + goff[g] + (long)rp[1] * gC[g] + cp[1], ptot, B.rows, B.cols,
                    B.cols, gC[g], nsl, 1.0, pad8(B.cols)});
      mx->psi_maxel = std::max<long>(mx->psi_maxel, (long)B.rows * pad8(B.cols));
      sj.push_back({mx->sig_f.p + sgoff[g] + (long)cp[1] * gR[g] + rp[1], plan.out.p + B.off, B.rows, B.cols, gR[g]});
      mx->sig_maxel = std::max<long>(mx->sig_maxel, (long)B.rows * B.cols);
    }
    mx->psi_jobs.upload(pj, c.stream);
    mx->n_psi_jobs = (int)pj.size();
    mx->sig_jobs.upload(sj, c.stream);
    mx->n_sig_jobs = (int)sj.size();
    mx->h_psi_jobs = pj;
    mx->h_sig_jobs = sj;
  }
  mx->err.alloc(1, c.stream);
  cuda_check(cudaMemsetAsync(mx->err.p, 0, sizeof(int), c.stream), "memset");
  // ---- stacked right operands (stage1_stacked): for every (beta, g') with g = g' + dQ_beta
  // the matrix Rt_beta[(n2, qr) blocks of g, (n2', qr') blocks of g'] (C_g x C_g', the
  // column layout of Psi_g'), absent site blocks and padding zero, scaled by the W
  // coefficient of each block
  std::vector<long> soff;
  if (stacked) {
    soff.assign(mid.size() * (size_t)ng, -1);
    std::vector<ConvJob> sj;
    long stot = 0, smax = 0;
    for (size_t beta = 0; beta < mid.size(); ++beta)
      for (int gp = 0; gp < ng; ++gp) {
        const int g = group_of(gq[gp].first + mid[beta].dna, gq[gp].second + mid[beta].dnb);
        if (g < 0) continue;
        const size_t j0 = sj.size();
        for (const auto& cb : gcol[g]) {
          const int n2 = cb[0], qr = cb[1];
          for (int n2p = 0; n2p < 4; ++n2p) {
            const TRef& r = rt.ref[beta][n2 * 4 + n2p];
            if (!r.p) continue;
            const int qrp = Rb.find(gq[gp].first + LQA[n2p], gq[gp].second + LQB[n2p]);
            if (qrp < 0) continue;
            const auto cpp = cpos[qrp * 4 + n2p];
            if (cpp[0] != gp) continue;
            const OpLayout& Lay = Renv.cls[r.cls];
            const int bl = Lay.blk_of_col[qrp];
            if (bl < 0 || Lay.blocks[bl].rs != qr) continue;
            const Block& B = Lay.blocks[bl];
            // dst holds the element offset until the buffer exists
            sj.push_back({r.p + B.off, (__nv_bfloat16*)(intptr_t)(stot + (long)cb[2] * gC[gp] + cpp[1]), 0, B.rows,
                          B.cols, B.cols, gC[gp], nsl, r.coef, pad8(B.cols)});
            smax = std::max<long>(smax, (long)B.rows * pad8(B.cols));
          }
        }
        if (sj.size() > j0) {
          soff[beta * ng + gp] = stot;
          stot += (long)gC[g] * gC[gp];
        }
      }
    mx->rs_total = std::max<long>(stot, 8);
    mx->rstack.alloc((size_t)mx->rs_total * nsl, c.stream);
    cuda_check(cudaMemsetAsync(mx->rstack.p, 0, mx->rstack.n * sizeof(__nv_bfloat16), c.stream), "memset");
    for (auto& j : sj) {
      j.dst = mx->rstack.p + (intptr_t)j.dst;
      j.slice_stride = mx->rs_total;
    }
    DArr<ConvJob> dj;
    dj.upload(sj, c.stream);
    if (!sj.empty()) launch_conv(dj, (int)sj.size(), smax, c.stream);
    cuda_check(cudaStreamSynchronize(c.stream), "sync");
  }
  // ---- X_beta^T per (beta, g'): C_g x R_g' with g = g' + dQ_beta; chunking over beta
  std::vector<size_t> xsz(mid.size(), 0);
  for (size_t beta = 0; beta < mid.size(); ++beta)
    for (int gp = 0; gp < ng; ++gp) {
      int g = group_of(gq[gp].first + mid[beta].dna, gq[gp].second + mid[beta].dnb);
      if (g >= 0) xsz[beta] += (size_t)gC[g] * gR[gp];
    }
  const size_t budget = (size_t)c.chunk_budget_mb * (1u << 20) / (2 * nsl);
  std::vector<std::pair<size_t, size_t>> chunks;
  size_t maxchunk = 0;
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
  mx->X_b.alloc(std::max<size_t>(maxchunk * nsl, 8), c.stream);
  cuda_check(cudaMemsetAsync(mx->X_b.p, 0, mx->X_b.n * sizeof(__nv_bfloat16), c.stream), "memset");
  const long xstride = (long)maxchunk;
  const __nv_bfloat16* mir = mx->mirror.p;
  const bool multi = chunks.size() > 1;
  // the chunks' work lists are independent: built on host threads, uploaded in order
  struct ChunkLists {
    TcBuilder g1, g2;
    std::vector<ZeroJob> zj;
  };
  auto build_chunk = [&](std::pair<size_t, size_t> ch, ChunkLists& out) {
    TcBuilder& g1 = out.g1;
    TcBuilder& g2 = out.g2;
    std::vector<ZeroJob>& zj = out.zj;
    size_t xoff = 0;
    // X^T offsets of this chunk: [beta - b0][g'] (-1 if absent or never written)
    std::vector<std::vector<long>> xpos(ch.second - ch.first, std::vector<long>(ng, -1));
    for (size_t beta = ch.first; beta < ch.second; ++beta) {
      auto& xp = xpos[beta - ch.first];
      for (int gp = 0; gp < ng; ++gp) {
        const int g = group_of(gq[gp].first + mid[beta].dna, gq[gp].second + mid[beta].dnb);
        if (g < 0) continue;
        const long base = (long)xoff;
        if (stacked) {
          // one task: X_beta^T (C_g x R_g') = (Psi_g' Rt_beta^T)^T over the whole group
          const long so = soff[beta * ng + gp];
          if (so < 0) continue;
          TcTask t{};
          t.Cb = mx->X_b.p + base;
          t.slice_stride = xstride;
          t.ldcb = gR[gp];
          t.m = gR[gp];
          t.n = gC[g];
          t.nslices = nsl;
          t.trans = 1;
          g1.begin(t);
          g1.term(mx->psi_b.p + goff[gp], ptot, gC[gp], mx->rstack.p + so, mx->rs_total, gC[gp], gC[gp], false, nsl);
          g1.end();
          xp[gp] = base;
          xoff += (size_t)gC[g] * gR[gp];
          continue;
        }
        bool any = false;
        std::vector<ZeroJob> empty_cb;  // column blocks of X^T without a term
        // stage 1: X_beta[rows of g', (n2, qr) block of g] = sum_{n2'} Psi_g'[:, (n2', qr')] Rt^{n2 n2'}[qr, qr']^T,
        // stored transposed into X^T (rows (n2, qr) of g, columns = rows of g')
        for (const auto& cb : gcol[g]) {
          const int n2 = cb[0], qr = cb[1];
          TcTask t{};
          t.Cb = mx->X_b.p + base + (long)cb[2] * gR[gp];
          t.slice_stride = xstride;
          t.ldcb = gR[gp];
          t.m = gR[gp];
          t.n = Rb.dim[qr];
          t.nslices = nsl;
          t.trans = 1;
          g1.begin(t);
          for (int n2p = 0; n2p < 4; ++n2p) {
            const TRef& r = rt.ref[beta][n2 * 4 + n2p];
            if (!r.p) continue;
            const int qrp = Rb.find(gq[gp].first + LQA[n2p], gq[gp].second + LQB[n2p]);
            if (qrp < 0) continue;
            const auto cpp = cpos[qrp * 4 + n2p];
            if (cpp[0] != gp) continue;
            const OpLayout& Lay = Renv.cls[r.cls];
            const int bl = Lay.blk_of_col[qrp];
            if (bl < 0 || Lay.blocks[bl].rs != qr) continue;
            const MirrorRef& mr = rm[beta][n2 * 4 + n2p];
            const int kk = Rb.dim[qrp];
            g1.term(mx->psi_b.p + goff[gp] + cpp[1], ptot, gC[gp], mir + mr.off + (*mr.boff)[bl], mr.stride, pad8(kk),
                    kk, mr.neg, nsl);
          }
          if (g1.end())
            any = true;
          else
            empty_cb.push_back({mx->X_b.p + base + (long)cb[2] * gR[gp], (long)Rb.dim[qr] * gR[gp], xstride, nsl});
        }
        if (any) {
          xp[gp] = base;
          xoff += (size_t)gC[g] * gR[gp];
          // with several chunks the X buffer is shared, so rows that stay exactly zero
          // here may hold another chunk's values: clear them (one chunk: zero from the start)
          if (multi) zj.insert(zj.end(), empty_cb.begin(), empty_cb.end());
        }
      }
    }
    // stage 2: sigma^T_g[:, (ql, n1) block] += sum_{beta, n1'} X_beta^T[:, (ql', n1')] Lt^{n1 n1'}[ql, ql']^T.
    // Long term lists are split into parts that accumulate atomically (split-K), so
    // that there are enough tiles for every resident CTA.
    TcBuilder g2all;
    for (int g = 0; g < ng; ++g)
      for (const auto& rb : grow[g]) {
        const int ql = rb[0], n1 = rb[1];
        TcTask t{};
        t.C = mx->sig_f.p + sgoff[g] + rb[2];
        t.ldc = gR[g];
        t.m = gC[g];
        t.n = Lb.dim[ql];
        t.beta = 2;
        g2all.begin(t);
        for (size_t beta = ch.first; beta < ch.second; ++beta) {
          const int gp = group_of(gq[g].first - mid[beta].dna, gq[g].second - mid[beta].dnb);
          if (gp < 0) continue;
          const long xo = xpos[beta - ch.first][gp];
          if (xo < 0) continue;
          for (int n1p = 0; n1p < 4; ++n1p) {
            const TRef& r = lt.ref[beta][n1 * 4 + n1p];
            if (!r.p) continue;
            const OpLayout& Lay = Lenv.cls[r.cls];
            const int qlp = Lb.find(Lb.qa[ql] - Lay.da, Lb.qb[ql] - Lay.db);
            if (qlp < 0) continue;
            const int bl = Lay.blk_of_col[qlp];
            if (bl < 0 || Lay.blocks[bl].rs != ql) continue;
            const auto rpp = rpos[qlp * 4 + n1p];
            if (rpp[0] != gp) continue;
            const MirrorRef& mr = lm[beta][n1 * 4 + n1p];
            const int kk = Lb.dim[qlp];
            g2all.term(mx->X_b.p + xo + rpp[1], xstride, gR[gp], mir + mr.off + (*mr.boff)[bl], mr.stride, pad8(kk),
                       kk, mr.neg, nsl);
          }
        }
        g2all.end();
      }
    {
      // k-steps per task and the split that gives about split_tps tiles per SM
      long total = 0;
      std::vector<long> w(g2all.tasks.size(), 0);
      for (size_t i = 0; i < g2all.tasks.size(); ++i) {
        for (int t = g2all.tasks[i].t0; t < g2all.tasks[i].t1; ++t) w[i] += (g2all.terms[t].k + 63) / 64;
        total += w[i] * ((g2all.tasks[i].m + 127) / 128);
      }
      const long target = c.split_tps > 0
                              ? std::max<long>(1, total / std::max<long>(1, std::lround(c.split_tps * 152)))
                              : std::numeric_limits<long>::max();
      for (size_t i = 0; i < g2all.tasks.size(); ++i) {
        const TcTask& tk = g2all.tasks[i];
        long acc = 0;
        int t0 = tk.t0;
        for (int t = tk.t0; t < tk.t1; ++t) {
          acc += (g2all.terms[t].k + 63) / 64;
          if (acc >= target || t + 1 == tk.t1) {
            TcTask part = tk;
            g2.begin(part);
            for (int u = t0; u <= t; ++u) g2.terms.push_back(g2all.terms[u]);
            g2.tasks.back().t1 = (int)g2.terms.size();
            g2.end();
            t0 = t + 1;
            acc = 0;
          }
        }
      }
    }
    // longest tiles first (static round-robin over persistent CTAs)
    auto order = [&](TcBuilder& g) {
      std::vector<long> w(g.tasks.size(), 0);
      for (size_t i = 0; i < g.tasks.size(); ++i)
        for (int t = g.tasks[i].t0; t < g.tasks[i].t1; ++t) w[i] += (g.terms[t].k + 63) / 64;
      std::stable_sort(g.tiles.begin(), g.tiles.end(),
                       [&](const TcTile& a, const TcTile& b) { return w[a.task] > w[b.task]; });
    };
    order(g2);
  };
  std::vector<ChunkLists> lists(chunks.size());
  {
    const unsigned hw = std::max(1u, std::thread::hardware_concurrency());
    const size_t nth = std::min<size_t>(chunks.size(), std::min(hw, 16u));
    std::atomic<size_t> next{0};
    std::exception_ptr fail;
    std::mutex fail_mu;
    auto worker = [&] {
      for (size_t i; (i = next.fetch_add(1)) < chunks.size();) {
        try {
          build_chunk(chunks[i], lists[i]);
        } catch (...) {
          std::lock_guard<std::mutex> lk(fail_mu);
          if (!fail) fail = std::current_exception();
        }
      }
    };
    std::vector<std::thread> pool;
    for (size_t t = 1; t < nth; ++t) pool.emplace_back(worker);
    worker();
    for (auto& th : pool) th.join();
    if (fail) std::rethrow_exception(fail);
  }
  for (ChunkLists& cl : lists) {
    TcBuilder& g1 = cl.g1;
    TcBuilder& g2 = cl.g2;
    std::vector<ZeroJob>& zj = cl.zj;
    auto keep = [&](TcPlan& tp, TcBuilder& g) {
      tp.tiles.upload(g.tiles, c.stream);
      tp.tasks.upload(g.tasks, c.stream);
      tp.terms.upload(g.terms, c.stream);
      tp.ntiles = (int)g.tiles.size();
      cuda_check(cudaStreamSynchronize(c.stream), "sync");
      if (c.keep_host_plans) {
        tp.htiles.swap(g.tiles);
        tp.htasks.swap(g.tasks);
        tp.hterms.swap(g.terms);
      }
    };
    mx->stage1.emplace_back();
    keep(mx->stage1.back(), g1);
    {
      TcPlan& tp = mx->stage1.back();
      tp.nzeros = (int)zj.size();
      for (const ZeroJob& z : zj) tp.zmax = std::max(tp.zmax, z.n);
      tp.zeros.upload(zj, c.stream);
      tp.hzeros = zj;
      cuda_check(cudaStreamSynchronize(c.stream), "sync");
    }
    mx->stage2.emplace_back();
    keep(mx->stage2.back(), g2);
  }
  plan.flops = count_sigma_flops(c.mpo, k, Lb, Rb);
}

void run_mixed_sigma(Context& c, SigmaPlan& plan, const double* x, double* y) {
  MixedPlan& mx = *plan.mx;
  const size_t n = plan.psi.nnz;
  if (x != plan.in.p) cuda_check(cudaMemcpyAsync(plan.in.p, x, n * sizeof(double), cudaMemcpyDeviceToDevice, c.stream), "d2d");
  if (mx.n_psi_jobs) launch_conv(mx.psi_jobs, mx.n_psi_jobs, mx.psi_maxel, c.stream);
  cuda_check(cudaMemsetAsync(mx.sig_f.p, 0, mx.sig_total * sizeof(float), c.stream), "memset");
  for (size_t i = 0; i < mx.stage1.size(); ++i) {
    auto& s1 = mx.stage1[i];
    auto& s2 = mx.stage2[i];
    run_zeros(s1, c.stream);
    cuda_check(launch_gemm_bf16_tc(s1.tiles.p, s1.ntiles, s1.tasks.p, s1.terms.p, mx.err.p, c.stream, mx.nsl),
               "tc stage 1");
    cuda_check(launch_gemm_bf16_tc(s2.tiles.p, s2.ntiles, s2.tasks.p, s2.terms.p, mx.err.p, c.stream, mx.nsl),
               "tc stage 2");
  }
  if (mx.n_sig_jobs) launch_unconv(mx.sig_jobs.p, mx.n_sig_jobs, mx.sig_maxel, c.stream);
  if (y != plan.out.p) cuda_check(cudaMemcpyAsync(y, plan.out.p, n * sizeof(double), cudaMemcpyDeviceToDevice, c.stream), "d2d");
}

int mixed_error(Context& c, SigmaPlan& plan) {
  int h = 0;
  cuda_check(cudaMemcpyAsync(&h, plan.mx->err.p, sizeof(int), cudaMemcpyDeviceToHost, c.stream), "d2h");
  cuda_check(cudaStreamSynchronize(c.stream), "sync");
  return h;
}

// ---------------------------------------------------------------- TMA-staged single-pass plan

// H_eff.psi in one BF16 pass with both stages as TMA-staged grouped GEMMs over a few
// large matrices (one tensor map each):
//   stage 1, per input group g': X_g'^T = A1_g' Psi_g'^T, where A1_g' stacks, for every
//     bond state beta and every (n2, qr) column block of the output group g = g' + dQ_beta,
//     the row block [Rt_beta^{n2 n2'}[qr, qr'] over the column blocks (n2', qr') of g'];
//     row blocks with the same pattern of non-zero site blocks n2' are stacked together,
//     and a tile multiplies only the K blocks of its pattern (no product with an absent
//     site block).  Each output row goes through a row map to its place in X_g'^T, whose
//     rows are, per beta, the column blocks of g in the row order of sigma^T_g.
//   stage 2, per output block: sigma^T_g[rows, (ql, n1)] += sum_{beta, n1'}
//     X_g'^T[beta rows, (ql', n1')] Lt_beta^{n1 n1'}[ql, ql']^T, a long contraction over
//     the operator terms (the paper's sum over left-right terms, Eq. Hpartition), cut
//     into parts that add with FP32 vector reductions.
// Every block is padded to 16 rows and columns with zeros, so a K step of 16 never
// mixes two blocks and padding contributes exact zeros.
struct TmaPlan {
  int nsl = 1;  // BF16 slices per operand (1: one pass; 2 or 3: slice products i + j < nsl)
  DArr<__nv_bfloat16> psi_b, a1, xt, lmir;
  long x_stride = 0;  // slice stride of the X intermediates
  DArr<float> sig_t;
  long sig_total = 0;
  DArr<ConvJob> psi_jobs, a1_jobs, l_jobs;
  int n_psi_jobs = 0, n_a1_jobs = 0, n_l_jobs = 0;
  long psi_maxel = 0, a1_maxel = 0, l_maxel = 0;
  DArr<UnconvJob> sig_jobs;
  int n_sig_jobs = 0;
  long sig_maxel = 0;
  DArr<CUtensorMap> maps;
  DArr<long> rowmap;
  DArr<int2> cbtab;  // (first column, width) of the column blocks of every input group
  // device copies of a launch's copy lists
  struct Lists {
    DArr<int> cta_stage, sorder, tpiece0;
    DArr<long> sfirst;
    DArr<TmStage> stages;
    DArr<TmPiece> pieces;
    int grid = 0;
    long total = 0;
    // the stage counts on the host (reduce mode: sets the tiles' stages and segments,
    // so it comes before the tiles are uploaded); throws on a malformed term
    void plan(int mode, std::vector<TmTile>& tiles, const std::vector<TmTerm>& terms, cudaStream_t s) {
      TmListPlan lp;
      if (!tma_plan_lists(mode, tiles, terms, lp)) throw Error(ST_ECUDA, "internal: malformed TMA term list");
      grid = lp.grid;
      total = lp.total;
      cta_stage.upload(lp.cta_stage, s);
      sorder.upload(lp.sorder, s);
      sfirst.upload(lp.sfirst, s);
      tpiece0.upload(lp.tpiece0, s);
      stages.alloc((size_t)std::max<long>(lp.total, 1), s);
      pieces.alloc((size_t)std::max<long>(lp.total, 1) * tma_pieces(mode), s);
    }
    // the lists themselves, on the device, from the uploaded tiles and terms
    void fill(int mode, const TmTile* d_tiles, int ntiles, const TmTerm* d_terms, cudaStream_t s) {
      cuda_check(launch_fill_lists(mode, d_tiles, ntiles, d_terms, tpiece0.p, sorder.p, sfirst.p, total, stages.p,
                                   pieces.p, s),
                 "list fill");
    }
    TmListsDev dev() const { return {grid, cta_stage.p, stages.p, pieces.p}; }
  };
  struct Chunk {
    DArr<TmTile> t1, t2;
    DArr<TmTerm> m1, m2;
    Lists l1, l2;
    int n1 = 0, n2 = 0;
    DArr<ZeroJob> z;
    int nz = 0;
    long zmax = 0;
  };
  std::vector<Chunk> chunks;
  DArr<int> err;
  double stats[9] = {0, 0, 0, 0, 0, 0, 0, 0, 0};
};

void tma_plan_free(TmaPlan* p) { delete p; }

void tma_plan_stats(const SigmaPlan& plan, double* out) {
  for (int i = 0; i < 9; ++i) out[i] = plan.tm ? plan.tm->stats[i] : 0.0;
}

namespace {
inline int pad16(int x) { return (x + 15) & ~15; }
}  // namespace

// conversion jobs must write inside their destination buffer
static void check_conv_jobs(const std::vector<ConvJob>& jobs, const DArr<__nv_bfloat16>& buf) {
  for (const ConvJob& j : jobs)
    if (j.rows < 1 || j.wcols < j.cols || j.ldd < j.wcols || j.dst < buf.p ||
        j.dst + (long)(j.rows - 1) * j.ldd + j.wcols > buf.p + buf.n)
      throw Error(ST_ECUDA, "internal: conversion job outside its buffer");
}

namespace {
// stages of a reduce-mode tile: its pieces (ceil(k / TM_PACK_COLS) per slice pair of every
// term) packed TM_PACK_SLOTS to a stage
long packed_stages(const std::vector<TmTerm>& m, int t0, int t1) {
  long pieces = 0;
  for (int t = t0; t < t1; ++t) {
    const int nsl = std::max(1, (m[t].neg >> 4) & 15);
    pieces += (long)((m[t].k + TM_PACK_COLS - 1) / TM_PACK_COLS) * (nsl * (nsl + 1) / 2);
  }
  return (pieces + TM_PACK_SLOTS - 1) / TM_PACK_SLOTS;
}

}  // namespace

void build_tma_plan(Context& c, Tilde& lt, Tilde& rt, int k, SigmaPlan& plan, int nsl) {
  const auto& mid = c.mpo.bonds[k + 1];
  Env& Lenv = *lt.env;
  Env& Renv = *rt.env;
  const Bond& Lb = Lenv.bond;
  const Bond& Rb = Renv.bond;
  const PsiLayout& P = plan.psi;
  auto* tp = new TmaPlan();
  plan.tm.reset(tp);
  if (nsl < 1 || nsl > 3) throw Error(ST_EINVAL, "TMA plan: 1 to 3 slices");
  tp->nsl = nsl;
  const int nL = Lb.nsec(), nR = Rb.nsec();
  const int nmid = (int)mid.size();
  // slice pairs (i, j), i + j < nsl, per term (expanded by the kernel, level by level)
  const int npair = nsl == 1 ? 1 : nsl == 2 ? 3 : 6;
  // ---- groups of the cut: rows (ql, n1) and columns (n2, qr), blocks padded to 16
  std::map<std::pair<int, int>, int> gidx;
  std::vector<std::pair<int, int>> gq;
  std::vector<std::vector<std::array<int, 3>>> grow, gcol;  // (ql, n1, off), (n2, qr, off)
  std::vector<int> gR, gC;
  {
    std::map<std::pair<int, int>, std::pair<std::vector<std::array<int, 3>>, std::vector<std::array<int, 3>>>> tmp;
    for (int ql = 0; ql < nL; ++ql)
      for (int n1 = 0; n1 < 4; ++n1) tmp[{Lb.qa[ql] + LQA[n1], Lb.qb[ql] + LQB[n1]}].first.push_back({ql, n1, 0});
    for (int qr = 0; qr < nR; ++qr)
      for (int n2 = 0; n2 < 4; ++n2) tmp[{Rb.qa[qr] - LQA[n2], Rb.qb[qr] - LQB[n2]}].second.push_back({n2, qr, 0});
    for (auto& kv : tmp) {
      if (kv.second.first.empty() || kv.second.second.empty()) continue;
      gidx[kv.first] = (int)gq.size();
      gq.push_back(kv.first);
      auto rows = kv.second.first, cols = kv.second.second;
      int R = 0, C = 0;
      for (auto& r : rows) { r[2] = R; R += pad16(Lb.dim[r[0]]); }
      for (auto& cc : cols) { cc[2] = C; C += pad16(Rb.dim[cc[1]]); }
      grow.push_back(rows);
      gcol.push_back(cols);
      gR.push_back(R);
      gC.push_back(C);
    }
  }
  const int ng = (int)gq.size();
  // (group, offset, index of the block in its group) of every row block (ql, n1) and
  // column block (n2, qr)
  std::vector<std::array<int, 3>> rpos((size_t)nL * 4, {-1, 0, -1}), cpos((size_t)nR * 4, {-1, 0, -1});
  for (int g = 0; g < ng; ++g) {
    for (size_t i = 0; i < grow[g].size(); ++i) rpos[grow[g][i][0] * 4 + grow[g][i][1]] = {g, grow[g][i][2], (int)i};
    for (size_t i = 0; i < gcol[g].size(); ++i) cpos[gcol[g][i][1] * 4 + gcol[g][i][0]] = {g, gcol[g][i][2], (int)i};
  }
  auto group_of = [&](int a, int b) {
    auto it = gidx.find({a, b});
    return it == gidx.end() ? -1 : it->second;
  };
  // output group of bond state beta for input group g' (-1: none)
  std::vector<int> gout((size_t)nmid * ng, -1);
  for (int beta = 0; beta < nmid; ++beta)
    for (int gp = 0; gp < ng; ++gp)
      gout[(size_t)beta * ng + gp] = group_of(gq[gp].first + mid[beta].dna, gq[gp].second + mid[beta].dnb);
  // input group g' = g - dQ_beta of bond state beta for output group g (-1: none)
  std::vector<int> gin((size_t)nmid * ng, -1);
  for (int beta = 0; beta < nmid; ++beta)
    for (int g = 0; g < ng; ++g)
      gin[(size_t)beta * ng + g] = group_of(gq[g].first - mid[beta].dna, gq[g].second - mid[beta].dnb);
  // ---- Psi_g (BF16, R_g x C_g) and sigma^T_g (FP32, C_g x R_g)
  std::vector<long> goff(ng), sgoff(ng);
  long ptot = 0, stot = 0;
  for (int g = 0; g < ng; ++g) {
    goff[g] = ptot;
    ptot += (long)gR[g] * gC[g];
    sgoff[g] = stot;
    stot += (long)gC[g] * gR[g];
  }
  tp->psi_b.alloc(std::max<long>(ptot, 8) * nsl, c.stream);
  cuda_check(cudaMemsetAsync(tp->psi_b.p, 0, tp->psi_b.n * sizeof(__nv_bfloat16), c.stream), "memset");
  tp->sig_total = std::max<long>(stot, 4);
  tp->sig_t.alloc(tp->sig_total, c.stream);
  {
    std::vector<ConvJob> pj;
    std::vector<UnconvJob> sj;
    for (size_t b = 0; b < P.blocks.size(); ++b) {
      const Block& B = P.blocks[b];
      const auto rp = rpos[B.rs * 4 + P.b1[b]];
      const auto cp = cpos[B.cs * 4 + P.b2[b]];
      if (rp[0] < 0 || rp[0] != cp[0]) throw Error(ST_ECUDA, "internal: psi block outside its group");
      const int g = rp[0];
      pj.push_back({plan.in.p + B.off, tp->psi_b.p + goff[g] + (long)rp[1] * gC[g] + cp[1], std::max<long>(ptot, 8),
                    B.rows, B.cols, B.cols, gC[g], nsl, 1.0, pad16(B.cols)});
      tp->psi_maxel = std::max<long>(tp->psi_maxel, (long)B.rows * pad16(B.cols));
      sj.push_back({tp->sig_t.p + sgoff[g] + (long)cp[1] * gR[g] + rp[1], plan.out.p + B.off, B.rows, B.cols, gR[g]});
      tp->sig_maxel = std::max<long>(tp->sig_maxel, (long)B.rows * B.cols);
    }
    check_conv_jobs(pj, tp->psi_b);
    for (const UnconvJob& u : sj)
      if (u.src < tp->sig_t.p || u.src + (long)(u.cols - 1) * u.lds + u.rows > tp->sig_t.p + tp->sig_total)
        throw Error(ST_ECUDA, "internal: gather job outside sigma^T");
    tp->psi_jobs.upload(pj, c.stream);
    tp->n_psi_jobs = (int)pj.size();
    tp->sig_jobs.upload(sj, c.stream);
    tp->n_sig_jobs = (int)sj.size();
    cuda_check(cudaStreamSynchronize(c.stream), "sync");
  }
  // ---- stage-1 row blocks: per input group g', every (beta, n2) with at least one
  // non-zero site block n2' of Rt_beta towards the column blocks of g'
  struct RowBlk {
    int beta, n2, qr, rows, mask;
    int bl[4];  // per n2' in the mask: the operator block of Rt_beta^{n2 n2'}
  };
  std::vector<std::vector<RowBlk>> rb(ng);
  for (int gp = 0; gp < ng; ++gp)
    for (int beta = 0; beta < nmid; ++beta) {
      const int g = gout[(size_t)beta * ng + gp];
      if (g < 0) continue;
      for (const auto& cb : gcol[g]) {
        const int n2 = cb[0], qr = cb[1];
        RowBlk x{beta, n2, qr, Rb.dim[qr], 0, {-1, -1, -1, -1}};
        for (int n2p = 0; n2p < 4; ++n2p) {
          const TRef& r = rt.ref[beta][n2 * 4 + n2p];
          if (!r.p) continue;
          const int qrp = Rb.find(gq[gp].first + LQA[n2p], gq[gp].second + LQB[n2p]);
          if (qrp < 0 || cpos[qrp * 4 + n2p][0] != gp) continue;
          const OpLayout& Lay = Renv.cls[r.cls];
          const int bl = Lay.blk_of_col[qrp];
          if (bl < 0 || Lay.blocks[bl].rs != qr) continue;
          x.mask |= 1 << n2p;
          x.bl[n2p] = bl;
        }
        if (x.mask) rb[gp].push_back(x);
      }
    }
  std::vector<char> xhas((size_t)nmid * ng, 0);  // [beta][g'] has X^T rows
  for (int gp = 0; gp < ng; ++gp)
    for (const RowBlk& x : rb[gp]) xhas[(size_t)x.beta * ng + gp] = 1;
  // chunks of bond states whose X^T fit the budget (one chunk unless the budget is small)
  std::vector<size_t> xsz(nmid, 0);
  for (int beta = 0; beta < nmid; ++beta)
    for (int gp = 0; gp < ng; ++gp)
      if (xhas[(size_t)beta * ng + gp]) xsz[beta] += (size_t)gC[gout[(size_t)beta * ng + gp]] * gR[gp];
  const size_t budget = (size_t)std::max<long>(1, c.tma_budget_mb) * (1u << 20) / (sizeof(__nv_bfloat16) * nsl);
  std::vector<std::pair<int, int>> chunks;
  for (int b0 = 0; b0 < nmid;) {
    int b1 = b0;
    size_t tot = 0;
    while (b1 < nmid && (b1 == b0 || tot + xsz[b1] <= budget)) tot += xsz[b1++];
    chunks.push_back({b0, b1});
    b0 = b1;
  }
  const int nch = (int)chunks.size();
  std::vector<int> chunk_of(nmid, 0);
  for (int ci = 0; ci < nch; ++ci)
    for (int b = chunks[ci].first; b < chunks[ci].second; ++b) chunk_of[b] = ci;
  // X^T layout per chunk: regions per g' (Sum_beta C_g(beta) rows x R_g' columns);
  // xrow[beta][g'] = first row of beta's block in its region
  std::vector<std::vector<long>> xreg(nch, std::vector<long>(ng, 0)), xregrows(nch, std::vector<long>(ng, 0));
  std::vector<long> xrow((size_t)nmid * ng, -1);
  size_t maxchunk = 0;
  for (int ci = 0; ci < nch; ++ci) {
    long off = 0;
    for (int gp = 0; gp < ng; ++gp) {
      xreg[ci][gp] = off;
      long rows = 0;
      for (int beta = chunks[ci].first; beta < chunks[ci].second; ++beta)
        if (xhas[(size_t)beta * ng + gp]) {
          xrow[(size_t)beta * ng + gp] = rows;
          rows += gC[gout[(size_t)beta * ng + gp]];
        }
      xregrows[ci][gp] = rows;
      off += rows * gR[gp];
    }
    maxchunk = std::max(maxchunk, (size_t)off);
  }
  tp->x_stride = (long)std::max<size_t>(maxchunk, 8);
  tp->xt.alloc((size_t)tp->x_stride * nsl, c.stream);
  cuda_check(cudaMemsetAsync(tp->xt.p, 0, tp->xt.n * sizeof(__nv_bfloat16), c.stream), "memset");
  // ---- A1 per g': row blocks sorted by (chunk, mask), beta order kept inside a run
  for (int gp = 0; gp < ng; ++gp)
    std::stable_sort(rb[gp].begin(), rb[gp].end(), [&](const RowBlk& a, const RowBlk& b) {
      if (chunk_of[a.beta] != chunk_of[b.beta]) return chunk_of[a.beta] < chunk_of[b.beta];
      return a.mask < b.mask;
    });
  std::vector<long> a1off(ng), a1rows(ng);
  long a1tot = 0;
  for (int gp = 0; gp < ng; ++gp) {
    long rows = 0;
    for (const RowBlk& x : rb[gp]) rows += x.rows;
    a1off[gp] = a1tot;
    a1rows[gp] = rows;
    a1tot += rows * gC[gp];
  }
  const long a1s = std::max<long>(a1tot, 8);
  tp->a1.alloc(a1s * nsl, c.stream);
  cuda_check(cudaMemsetAsync(tp->a1.p, 0, tp->a1.n * sizeof(__nv_bfloat16), c.stream), "memset");
  struct Run {
    int chunk, mask;
    long r0, r1;
  };
  std::vector<std::vector<Run>> runs(ng);
  // per A1 row: its row in the X^T region of its chunk (columns: blocks of g', each its
  // own submatrix of the region)
  std::vector<std::vector<long>> rowdst(ng);
  std::vector<ConvJob> aconv;
  for (int gp = 0; gp < ng; ++gp) {
    long row = 0;
    rowdst[gp].assign((size_t)a1rows[gp], -1);
    for (const RowBlk& x : rb[gp]) {
      const int ci = chunk_of[x.beta];
      if (runs[gp].empty() || runs[gp].back().chunk != ci || runs[gp].back().mask != x.mask)
        runs[gp].push_back({ci, x.mask, row, row});
      runs[gp].back().r1 = row + x.rows;
      const long xr0 = xrow[(size_t)x.beta * ng + gp] + (long)cpos[x.qr * 4 + x.n2][1];
      for (int i = 0; i < x.rows; ++i) rowdst[gp][(size_t)(row + i)] = xr0 + i;
      for (int n2p = 0; n2p < 4; ++n2p) {
        if (!((x.mask >> n2p) & 1)) continue;
        const TRef& r = rt.ref[x.beta][x.n2 * 4 + n2p];
        const Block& B = Renv.cls[r.cls].blocks[x.bl[n2p]];
        // the K block (n2', qr') of g': submatrix of a1rows x pad16(d(qr')) at column offset coff
        const int coff = cpos[B.cs * 4 + n2p][1];
        const int w = pad16(B.cols);
        aconv.push_back({r.p + B.off, tp->a1.p + a1off[gp] + a1rows[gp] * coff + row * w, a1s, B.rows, B.cols, B.cols,
                         w, nsl, r.coef, w});
        tp->a1_maxel = std::max<long>(tp->a1_maxel, (long)B.rows * pad16(B.cols));
      }
      row += x.rows;
    }
  }
  check_conv_jobs(aconv, tp->a1);
  tp->a1_jobs.upload(aconv, c.stream);
  tp->n_a1_jobs = (int)aconv.size();
  // ---- left mirror: every distinct (operator, scale) referenced by Lt, all its blocks,
  // each padded to 16 rows and columns; blocks of one padded width w share one matrix of
  // w columns (a box past the width then reads zeros without touching memory)
  std::map<int, int> wcls;  // padded width -> class
  std::vector<int> wcls_w;
  for (const OpLayout& L : Lenv.cls)
    for (const Block& B : L.blocks)
      if (!wcls.count(pad16(B.cols))) {
        wcls[pad16(B.cols)] = (int)wcls_w.size();
        wcls_w.push_back(pad16(B.cols));
      }
  const int nwc = (int)wcls_w.size();
  std::vector<long> lrows_c(nwc, 0);
  struct MirKeyHash {
    size_t operator()(const std::pair<const double*, double>& kk) const {
      uint64_t b;
      std::memcpy(&b, &kk.second, sizeof b);
      return std::hash<uint64_t>()((uint64_t)(uintptr_t)kk.first * 0x9e3779b97f4a7c15ULL ^ b);
    }
  };
  std::unordered_map<std::pair<const double*, double>, int, MirKeyHash> lm_id;
  std::vector<std::vector<long>> mblk_row;  // per mirror, per block: row in its width class
  struct PendL {  // one block of a new mirror: source, width class, row in the class, shape
    const double* src;
    int cls;
    long crow;
    int rows, cols;
    double scale;
  };
  std::vector<PendL> lpend;
  std::vector<std::array<int, 16>> lmid((size_t)nmid);
  std::vector<std::array<char, 16>> lneg((size_t)nmid);
  for (int beta = 0; beta < nmid; ++beta)
    for (int nn = 0; nn < 16; ++nn) {
      lmid[beta][nn] = -1;
      lneg[beta][nn] = 0;
      const TRef& r = lt.ref[beta][nn];
      if (!r.p) continue;
      const double a = std::fabs(r.coef);
      const double scale = a == 1.0 ? 1.0 : r.coef;
      auto key = std::make_pair(r.p, scale);
      auto it = lm_id.find(key);
      if (it == lm_id.end()) {
        const int id = (int)mblk_row.size();
        it = lm_id.emplace(key, id).first;
        const OpLayout& L = Lenv.cls[r.cls];
        mblk_row.emplace_back(L.blocks.size());
        for (size_t b = 0; b < L.blocks.size(); ++b) {
          const Block& B = L.blocks[b];
          const int wc = wcls[pad16(B.cols)];
          mblk_row[id][b] = lrows_c[wc];
          lpend.push_back({r.p + B.off, wc, lrows_c[wc], B.rows, B.cols, scale});
          lrows_c[wc] += pad16(B.rows);
        }
      }
      lmid[beta][nn] = it->second;
      lneg[beta][nn] = (a == 1.0 && r.coef < 0) ? 1 : 0;
    }
  std::vector<long> lbase(nwc, 0);
  long ltot = 0;
  for (int wc = 0; wc < nwc; ++wc) {
    lbase[wc] = ltot;
    ltot += lrows_c[wc] * wcls_w[wc];
  }
  const long ls = std::max<long>(ltot, 8);
  tp->lmir.alloc(ls * nsl, c.stream);
  cuda_check(cudaMemsetAsync(tp->lmir.p, 0, tp->lmir.n * sizeof(__nv_bfloat16), c.stream), "memset");
  std::vector<ConvJob> lconv;
  lconv.reserve(lpend.size());
  for (const PendL& pl : lpend) {
    const int w = wcls_w[pl.cls];
    lconv.push_back({pl.src, tp->lmir.p + lbase[pl.cls] + pl.crow * w, ls, pl.rows, pl.cols, pl.cols, w, nsl, pl.scale,
                     w});
    tp->l_maxel = std::max<long>(tp->l_maxel, (long)pl.rows * w);
  }
  check_conv_jobs(lconv, tp->lmir);
  tp->l_jobs.upload(lconv, c.stream);
  tp->n_l_jobs = (int)lconv.size();
  // ---- tensor maps
  std::vector<CUtensorMap> maps;
  // every map must lie inside its buffer (a box outside the map's extent reads zeros,
  // but the extent itself is trusted by the hardware)
  struct MapInfo {
    long rows, cols;
    int box, boxc;
  };
  std::vector<MapInfo> minfo;
  // one map per slice, at consecutive indices (slice i of a map m is m + i)
  auto add_map = [&](const DArr<__nv_bfloat16>& buf, long off, long stride, long rows, long cols, long ld,
                     int box_rows, int box_cols) {
    const int first = (int)maps.size();
    for (int sl = 0; sl < nsl; ++sl) {
      const long o = off + sl * stride;
      if (o < 0 || rows < 1 || cols < 1 || ld < cols || ld % 8 != 0 || o % 8 != 0 ||
          (size_t)(o + (rows - 1) * ld + cols) > buf.n)
        throw Error(ST_ECUDA, "internal: tensor map outside its buffer");
      CUtensorMap m;
      if (!encode_bf16_map(&m, buf.p + o, (uint64_t)rows, (uint64_t)cols, (uint64_t)ld, (uint32_t)box_rows,
                           (uint32_t)box_cols))
        throw Error(ST_ECUDA, "cuTensorMapEncodeTiled failed");
      maps.push_back(m);
      minfo.push_back({rows, cols, box_rows, box_cols});
    }
    return first;
  };
  const int n1max = tma_max_n(TM_MODE_STORE_BF16), n2max = tma_max_n(TM_MODE_REDUCE_F32);
  const int bc1 = tma_box_cols(TM_MODE_STORE_BF16), bc2 = tma_box_cols(TM_MODE_REDUCE_F32);
  std::vector<std::vector<std::array<int, 3>>> nt1(ng);  // per g': (row0, width, Psi map) of the stage-1 N tiles
  // A1 of g': one map per K block (column block of g', a1rows x its padded width)
  std::vector<std::vector<int>> a1map(ng);
  for (int gp = 0; gp < ng; ++gp) {
    if (a1rows[gp] == 0) continue;
    const int parts = (gR[gp] + n1max - 1) / n1max;
    int r0 = 0;
    for (int p = 0; p < parts; ++p) {
      const int w = std::min(gR[gp] - r0, pad16((gR[gp] - r0 + (parts - p) - 1) / (parts - p)));
      nt1[gp].push_back(
          {r0, w, add_map(tp->psi_b, goff[gp], std::max<long>(ptot, 8), gR[gp], gC[gp], gC[gp], w, bc1)});
      r0 += w;
    }
    for (const auto& cc : gcol[gp]) {
      const int w = pad16(Rb.dim[cc[1]]);
      a1map[gp].push_back(add_map(tp->a1, a1off[gp] + a1rows[gp] * cc[2], a1s, a1rows[gp], w, w, 128, bc1));
    }
  }
  // X^T region of (chunk, g'): one submatrix (and map) per column block (ql', n1') of g',
  // xrows x its padded width; the table cbtab lists (first column, width) per g'
  std::vector<std::vector<std::vector<int>>> xtmap(nch, std::vector<std::vector<int>>(ng));
  std::vector<int2> cbtab;
  std::vector<int> cbt0(ng), cbt1(ng);
  for (int gp = 0; gp < ng; ++gp) {
    cbt0[gp] = (int)cbtab.size();
    for (const auto& rr : grow[gp]) cbtab.push_back(make_int2(rr[2], pad16(Lb.dim[rr[0]])));
    cbt1[gp] = (int)cbtab.size();
  }
  for (int ci = 0; ci < nch; ++ci)
    for (int gp = 0; gp < ng; ++gp)
      if (xregrows[ci][gp] > 0)
        for (const auto& rr : grow[gp]) {
          const int w = pad16(Lb.dim[rr[0]]);
          xtmap[ci][gp].push_back(add_map(tp->xt, xreg[ci][gp] + xregrows[ci][gp] * rr[2], tp->x_stride,
                                          xregrows[ci][gp], w, w, 128, bc2));
        }
  // left mirror: per width class one map per box height
  std::vector<std::vector<int>> lmap(nwc, std::vector<int>(n2max / 16 + 1, -1));
  for (int wc = 0; wc < nwc; ++wc)
    if (lrows_c[wc] > 0)
      for (int h = 16; h <= n2max; h += 16)
        lmap[wc][h / 16] = add_map(tp->lmir, lbase[wc], ls, lrows_c[wc], wcls_w[wc], wcls_w[wc], h, bc2);
  tp->cbtab.upload(cbtab, c.stream);
  tp->maps.alloc(std::max<size_t>(maps.size(), 1), c.stream);
  if (!maps.empty())
    cuda_check(cudaMemcpyAsync(tp->maps.p, maps.data(), maps.size() * sizeof(CUtensorMap), cudaMemcpyHostToDevice,
                               c.stream),
               "h2d");
  // ---- work lists per chunk
  std::vector<long> rowmap;
  double st1_tiles = 0, st1_steps = 0, st2_tiles = 0, st2_steps = 0, st1_fl = 0, st2_fl = 0;
  tp->chunks.resize(nch);
  for (int ci = 0; ci < nch; ++ci) {
    TmaPlan::Chunk& ch = tp->chunks[ci];
    std::vector<TmTile> t1, t2;
    std::vector<TmTerm> m1, m2;
    std::vector<ZeroJob> zj;
    // stage 1: per g', per (chunk, mask) run, 128-row tiles x N tiles
    for (int gp = 0; gp < ng; ++gp)
      for (const Run& run : runs[gp]) {
        if (run.chunk != ci) continue;
        for (long r0 = run.r0; r0 < run.r1; r0 += 128) {
          const long moff = (long)rowmap.size();
          for (long i = 0; i < 128; ++i)
            rowmap.push_back(r0 + i < run.r1 ? rowdst[gp][(size_t)(r0 + i)] : -1);
          for (const auto& nt : nt1[gp]) {
            TmTile tl{};
            tl.t0 = (int)m1.size();
            int ksum = 0;
            for (int n2p = 0; n2p < 4; ++n2p) {
              if (!((run.mask >> n2p) & 1)) continue;
              // the K block of n2': the column block (n2', qr') of g'
              const int qrp = Rb.find(gq[gp].first + LQA[n2p], gq[gp].second + LQB[n2p]);
              const int coff = cpos[qrp * 4 + n2p][1];
              const int cbi = cpos[qrp * 4 + n2p][2];
              const int kk = pad16(Rb.dim[qrp]);
              // one term for all slice pairs (expanded by the kernel)
              m1.push_back({a1map[gp][cbi], nt[2], 0, (int)r0, coff, nt[0], kk, nsl << 4});
              ksum += kk * npair;
              st1_steps += (kk + 63) / 64 * npair;
            }
            tl.t1 = (int)m1.size();
            tl.nseg = 1;
            tl.xbase = xreg[ci][gp];
            tl.xrows = xregrows[ci][gp];
            tl.cb0 = cbt0[gp];
            tl.cb1 = cbt1[gp];
            tl.n = nt[1];
            tl.m_valid = 128;
            tl.ldo = gR[gp];
            tl.out_off = nt[0];
            tl.rowmap_off = moff;
            t1.push_back(tl);
            st1_fl += 2.0 * 128 * nt[1] * ksum;
          }
        }
      }
    // X^T rows of this chunk that stage 1 does not write: zero them before the chunk
    // (with one chunk the buffer is zero from the start)
    if (nch > 1) {
      for (int gp = 0; gp < ng; ++gp) {
        std::unordered_set<long> written;
        for (const RowBlk& x : rb[gp])
          if (chunk_of[x.beta] == ci) written.insert(((long)x.beta * 4 + x.n2) * nR + x.qr);
        for (int beta = chunks[ci].first; beta < chunks[ci].second; ++beta) {
          if (!xhas[(size_t)beta * ng + gp]) continue;
          const int g = gout[(size_t)beta * ng + gp];
          for (const auto& cb : gcol[g]) {
            if (written.count(((long)beta * 4 + cb[0]) * nR + cb[1])) continue;
            const long r0 = xrow[(size_t)beta * ng + gp] + cb[2];
            for (const auto& rr : grow[gp]) {
              const int w = pad16(Lb.dim[rr[0]]);
              const long e0 = xreg[ci][gp] + xregrows[ci][gp] * rr[2] + r0 * w;
              zj.push_back({tp->xt.p + e0, (long)pad16(Rb.dim[cb[1]]) * w, tp->x_stride, nsl});
            }
          }
        }
      }
    }
    // stage 2: per output block (g, (ql, n1) column block, N part), 128-row tiles, terms
    // over the chunk's bond states; long term lists cut into parts (split-K)
    struct Pending {
      TmTile tl;
      std::vector<TmTerm> terms;
    };
    std::vector<Pending> pend;
    long total_steps = 0;
    for (int g = 0; g < ng; ++g)
      for (const auto& rbk : grow[g]) {
        const int ql = rbk[0], n1 = rbk[1];
        const int dql = Lb.dim[ql];
        for (int c0 = 0; c0 < pad16(dql); c0 += n2max) {
          const int nw = std::min(n2max, pad16(dql) - c0);
          // the block's terms for the first row tile; other row tiles shift the X^T row
          std::vector<TmTerm> base;
          for (int beta = chunks[ci].first; beta < chunks[ci].second; ++beta) {
            const int gp = gin[(size_t)beta * ng + g];
            if (gp < 0 || !xhas[(size_t)beta * ng + gp]) continue;
            for (int n1p = 0; n1p < 4; ++n1p) {
              const TRef& r = lt.ref[beta][n1 * 4 + n1p];
              if (!r.p) continue;
              const OpLayout& Lay = Lenv.cls[r.cls];
              const int qlp = Lb.find(Lb.qa[ql] - Lay.da, Lb.qb[ql] - Lay.db);
              if (qlp < 0) continue;
              const int bl = Lay.blk_of_col[qlp];
              if (bl < 0 || Lay.blocks[bl].rs != ql) continue;
              const auto rpp = rpos[qlp * 4 + n1p];
              if (rpp[0] != gp) continue;
              const int mid_ = lmid[beta][n1 * 4 + n1p];
              const int wc = wcls[pad16(Lb.dim[qlp])];
              base.push_back({xtmap[ci][gp][rpp[2]], lmap[wc][nw / 16], 0, (int)xrow[(size_t)beta * ng + gp], 0,
                              (int)(mblk_row[mid_][bl] + c0), pad16(Lb.dim[qlp]), (int)lneg[beta][n1 * 4 + n1p]});
            }
          }
          if (base.empty()) continue;
          for (TmTerm& t : base) t.neg |= nsl << 4;  // all slice pairs, expanded by the kernel
          long steps = 0;  // pieces (stage 2 packs TM_PACK_SLOTS per K step)
          for (const TmTerm& t : base) steps += (t.k + bc2 - 1) / bc2 * npair;
          for (int r0 = 0; r0 < gC[g]; r0 += 128) {
            Pending pd;
            pd.tl = TmTile{};
            pd.tl.n = nw;
            pd.tl.m_valid = std::min(128, gC[g] - r0);
            pd.tl.ldo = gR[g];
            pd.tl.out_off = sgoff[g] + (long)r0 * gR[g] + rbk[2] + c0;
            pd.terms = base;
            for (TmTerm& t : pd.terms) t.ay += r0;
            total_steps += steps;
            pend.push_back(std::move(pd));
          }
        }
      }
    const long target = c.split_tps > 0 ? std::max<long>(1, total_steps / std::max<long>(1, std::lround(c.split_tps * 152)))
                                        : std::numeric_limits<long>::max();
    for (Pending& pd : pend) {
      long acc = 0;
      size_t t0 = 0;
      for (size_t t = 0; t < pd.terms.size(); ++t) {
        acc += (pd.terms[t].k + bc2 - 1) / bc2 * npair;
        if (acc >= target || t + 1 == pd.terms.size()) {
          TmTile tl = pd.tl;
          tl.t0 = (int)m2.size();
          long ks = 0;
          for (size_t u = t0; u <= t; ++u) {
            m2.push_back(pd.terms[u]);
            ks += (long)pd.terms[u].k * npair;
          }
          tl.t1 = (int)m2.size();
          const long stages = packed_stages(m2, tl.t0, tl.t1);
          if (stages > (1L << 30)) throw Error(ST_ECUDA, "internal: stage-2 tile too long");
          t2.push_back(tl);
          st2_steps += stages;
          st2_fl += 2.0 * 128 * tl.n * ks;
          t0 = t + 1;
          acc = 0;
        }
      }
    }
    // longest tiles first (static round-robin over the persistent CTAs); tiles of equal
    // length keep their order, so the N tiles of one row tile stay adjacent
    auto order = [](std::vector<TmTile>& t, const std::vector<TmTerm>& m) {
      std::vector<std::pair<long, int>> key(t.size());
      for (size_t i = 0; i < t.size(); ++i) {
        long ks = 0;
        for (int j = t[i].t0; j < t[i].t1; ++j) ks += (m[j].k + 63) / 64;
        key[i] = {-ks, (int)i};
      }
      std::stable_sort(key.begin(), key.end(),
                       [](const std::pair<long, int>& a, const std::pair<long, int>& b) { return a.first < b.first; });
      std::vector<TmTile> out(t.size());
      for (size_t i = 0; i < t.size(); ++i) out[i] = t[(size_t)key[i].second];
      t.swap(out);
    };
    order(t1, m1);
    order(t2, m2);
    // the copy lists of both launches (stage 2: sets every tile's stages and segments);
    // their pieces follow from the terms checked below
    ch.l1.plan(TM_MODE_STORE_BF16, t1, m1, c.stream);
    ch.l2.plan(TM_MODE_REDUCE_F32, t2, m2, c.stream);
    st1_tiles += (double)t1.size();
    st2_tiles += (double)t2.size();
    // every access of the kernels checked against its buffer before anything runs:
    // operand boxes (their coordinates, alignment and widths), the rows stage 1 stores
    // through the row map and the blocks stage 2 reduces into
    auto check_terms = [&](const std::vector<TmTile>& tt, const std::vector<TmTerm>& mm, int nmax, int bc) {
      for (const TmTile& tl : tt) {
        if (tl.n < 16 || tl.n > nmax || tl.n % 16 || tl.t0 < 0 || tl.t1 <= tl.t0 || tl.t1 > (int)mm.size())
          throw Error(ST_ECUDA, "internal: malformed TMA tile");
        for (int t = tl.t0; t < tl.t1; ++t) {
          const TmTerm& m = mm[t];
          if (((m.neg >> 4) & 15) != nsl || m.amap < 0 || m.amap + nsl > (int)minfo.size() || m.bmap < 0 ||
              m.bmap + nsl > (int)minfo.size() ||
              minfo[m.amap].box != 128 || minfo[m.bmap].box != tl.n || minfo[m.amap].boxc != bc ||
              minfo[m.bmap].boxc != bc || m.k < 16 || m.k % 16 || m.ax % 16 || m.bx % 16 || m.ax < 0 || m.bx < 0 ||
              m.ay < 0 || m.by < 0 || m.ax + m.k > minfo[m.amap].cols + bc - 1 ||
              m.bx + m.k > minfo[m.bmap].cols + bc - 1)
            throw Error(ST_ECUDA, "internal: malformed TMA term");
        }
      }
    };
    check_terms(t1, m1, n1max, bc1);
    check_terms(t2, m2, n2max, bc2);
    {
      // the column blocks of every input group in increasing, disjoint column order, so
      // that a chunk's block is found by binary search (the kernel takes the one block
      // that holds the chunk)
      for (int gp = 0; gp < ng; ++gp)
        for (int e = cbt0[gp] + 1; e < cbt1[gp]; ++e)
          if (cbtab[(size_t)e].x < cbtab[(size_t)e - 1].x + cbtab[(size_t)e - 1].y)
            throw Error(ST_ECUDA, "internal: overlapping column blocks");
      std::atomic<int> bad{0}, next{0};
      auto check_range = [&]() {
        for (int i0 = next.fetch_add(1024); i0 < (int)t1.size() && !bad.load(); i0 = next.fetch_add(1024))
          for (int ti = i0; ti < std::min<int>((int)t1.size(), i0 + 1024); ++ti) {
            const TmTile& tl = t1[(size_t)ti];
            if (tl.rowmap_off < 0 || tl.rowmap_off + 128 > (long)rowmap.size() || tl.cb0 < 0 ||
                tl.cb1 > (int)cbtab.size() || tl.cb0 >= tl.cb1) {
              bad = 1;  // row map or column blocks out of range
              return;
            }
            long dmax = -1;
            for (int r = 0; r < 128; ++r) {
              const long d = rowmap[(size_t)(tl.rowmap_off + r)];
              if (d < -1 || d >= tl.xrows) {
                bad = 2;  // row outside its X region
                return;
              }
              dmax = std::max(dmax, d);
            }
            // every 8-column chunk of the tile lies in one column block; its highest row
            // stays inside the buffer (addresses grow with the row)
            for (int cc = 0; cc < tl.n; cc += 8) {
              const long col = tl.out_off + cc;
              int lo = tl.cb0, hi = tl.cb1 - 1;  // the last block starting at or before col
              while (lo < hi) {
                const int mid = (lo + hi + 1) / 2;
                if (cbtab[(size_t)mid].x <= col) lo = mid; else hi = mid - 1;
              }
              const int2 cb = cbtab[(size_t)lo];
              if (!(col >= cb.x && col + 8 <= cb.x + cb.y)) {
                bad = 3;  // column outside the column blocks
                return;
              }
              const long a0 = tl.xbase + tl.xrows * cb.x + (col - cb.x);
              if (a0 < 0 || a0 % 8 || cb.y % 8 || (dmax >= 0 && a0 + dmax * cb.y + 8 > tp->x_stride)) {
                bad = 4;  // store outside the X buffer
                return;
              }
            }
          }
      };
      const int nth = (int)std::max(1u, std::min(16u, std::thread::hardware_concurrency()));
      std::vector<std::thread> th;
      for (int w = 1; w < nth; ++w) th.emplace_back(check_range);
      check_range();
      for (auto& x : th) x.join();
      if (bad) throw Error(ST_ECUDA, "internal: stage-1 tile check failed (" + std::to_string(bad.load()) + ")");
    }
    for (const TmTile& tl : t2) {
      const long stages = packed_stages(m2, tl.t0, tl.t1);
      if (tl.pad != stages || stages < 1 || tl.nseg != (int)((stages + TM_SEG_KSTEPS - 1) / TM_SEG_KSTEPS))
        throw Error(ST_ECUDA, "internal: stage-2 stage or segment count");
    }

    for (const TmTile& tl : t2)
      if (tl.m_valid < 1 || tl.m_valid > 128 || tl.out_off < 0 || tl.out_off % 4 || tl.ldo % 4 ||
          tl.out_off + (long)(tl.m_valid - 1) * tl.ldo + tl.n > tp->sig_total)
        throw Error(ST_ECUDA, "internal: stage-2 reduction outside sigma^T");
    for (const ZeroJob& z : zj)
      if (z.p < tp->xt.p || z.p + (long)(z.nsl - 1) * z.stride + z.n > tp->xt.p + tp->xt.n)
        throw Error(ST_ECUDA, "internal: zero job outside X");
    ch.t1.upload(t1, c.stream);
    ch.m1.upload(m1, c.stream);
    ch.n1 = (int)t1.size();
    ch.t2.upload(t2, c.stream);
    ch.m2.upload(m2, c.stream);
    ch.n2 = (int)t2.size();
    ch.l1.fill(TM_MODE_STORE_BF16, ch.t1.p, ch.n1, ch.m1.p, c.stream);
    ch.l2.fill(TM_MODE_REDUCE_F32, ch.t2.p, ch.n2, ch.m2.p, c.stream);
    ch.nz = (int)zj.size();
    for (const ZeroJob& z : zj) ch.zmax = std::max(ch.zmax, z.n);
    ch.z.upload(zj, c.stream);
    cuda_check(cudaStreamSynchronize(c.stream), "sync");
  }
  tp->rowmap.upload(rowmap, c.stream);
  // the operator stacks depend only on the environments: filled once per plan
  if (tp->n_a1_jobs) launch_conv(tp->a1_jobs, tp->n_a1_jobs, tp->a1_maxel, c.stream);
  if (tp->n_l_jobs) launch_conv(tp->l_jobs, tp->n_l_jobs, tp->l_maxel, c.stream);
  tp->err.alloc(1, c.stream);
  cuda_check(cudaMemsetAsync(tp->err.p, 0, sizeof(int), c.stream), "memset");
  cuda_check(cudaStreamSynchronize(c.stream), "sync");
  tp->stats[0] = st1_tiles;
  tp->stats[1] = st1_steps;
  tp->stats[2] = st2_tiles;
  tp->stats[3] = st2_steps;
  tp->stats[4] = st1_fl;
  tp->stats[5] = st2_fl;
  tp->stats[6] = (double)maxchunk * 2;
  tp->stats[7] = (double)a1tot * 2;
  tp->stats[8] = nch;
  plan.flops = count_sigma_flops(c.mpo, k, Lb, Rb);
}

void run_tma_sigma(Context& c, SigmaPlan& plan, const double* x, double* y) {
  TmaPlan& tp = *plan.tm;
  const size_t n = plan.psi.nnz;
  if (x != plan.in.p) cuda_check(cudaMemcpyAsync(plan.in.p, x, n * sizeof(double), cudaMemcpyDeviceToDevice, c.stream), "d2d");
  if (tp.n_psi_jobs) launch_conv(tp.psi_jobs, tp.n_psi_jobs, tp.psi_maxel, c.stream);
  cuda_check(cudaMemsetAsync(tp.sig_t.p, 0, tp.sig_total * sizeof(float), c.stream), "memset");
  for (auto& ch : tp.chunks) {
    if (ch.nz) launch_zero(ch.z.p, ch.nz, ch.zmax, c.stream);
    cuda_check(launch_gemm_tma(TM_MODE_STORE_BF16, ch.t1.p, ch.n1, ch.m1.p, tp.maps.p, tp.rowmap.p, tp.cbtab.p,
                               tp.xt.p, tp.nsl, tp.x_stride, tp.err.p, c.stream, ch.l1.dev()),
               "tma stage 1");
    cuda_check(launch_gemm_tma(TM_MODE_REDUCE_F32, ch.t2.p, ch.n2, ch.m2.p, tp.maps.p, tp.rowmap.p, tp.cbtab.p,
                               tp.sig_t.p, 1, 0, tp.err.p, c.stream, ch.l2.dev()),
               "tma stage 2");
  }
  if (tp.n_sig_jobs) launch_unconv(tp.sig_jobs.p, tp.n_sig_jobs, tp.sig_maxel, c.stream);
  if (y != plan.out.p) cuda_check(cudaMemcpyAsync(y, plan.out.p, n * sizeof(double), cudaMemcpyDeviceToDevice, c.stream), "d2d");
}

int plan_error(Context& c, SigmaPlan& plan) {
  int h = 0;
  int* p = plan.mx ? plan.mx->err.p : plan.tm ? plan.tm->err.p : nullptr;
  if (!p) return 0;
  cuda_check(cudaMemcpyAsync(&h, p, sizeof(int), cudaMemcpyDeviceToHost, c.stream), "d2h");
  cuda_check(cudaStreamSynchronize(c.stream), "sync");
  return h;
}

// ---------------------------------------------------------------- environment update on the tensor cores

namespace {

// transposed FP64 block -> nsl BF16 slices: dst[j * ldd + i] = slices of scale * src[i * lds + j]
// for i < rows, j < cols; zeros for rows <= i < wrows (the padded contraction columns)
struct ConvTJob {
  const double* src;
  __nv_bfloat16* dst;
  long slice_stride;
  int rows, cols, lds, ldd, nsl, wrows;
  double scale;
};

__global__ void convt_kernel(const ConvTJob* __restrict__ jobs) {
  const ConvTJob jb = jobs[blockIdx.y];
  const long n = (long)jb.cols * jb.wrows;
  for (long e = (long)blockIdx.x * blockDim.x + threadIdx.x; e < n; e += (long)gridDim.x * blockDim.x) {
    const int j = (int)(e / jb.wrows), i = (int)(e % jb.wrows);
    double v = i < jb.rows ? jb.scale * jb.src[(long)i * jb.lds + j] : 0.0;
    __nv_bfloat16* d = jb.dst + (long)j * jb.ldd + i;
    for (int s = 0; s < jb.nsl; ++s) {
      const __nv_bfloat16 h = __double2bfloat16(v);
      d[s * jb.slice_stride] = h;
      v -= (double)__bfloat162float(h);
    }
  }
}

__global__ void f32_to_f64_kernel(const float* __restrict__ src, double* __restrict__ dst, long n) {
  for (long e = (long)blockIdx.x * blockDim.x + threadIdx.x; e < n; e += (long)gridDim.x * blockDim.x)
    dst[e] = (double)src[e];
}

}  // namespace

// L_{k+1}[beta] = sum (A^{n1})^T Lt_beta^{n1 n1'} A^{n1'} (left, Eqs. leftrenorm / prenormdec) or
// R_k[beta] = sum B^{n2} Rt_beta^{n2 n2'} (B^{n2'})^T (right), both stages as tensor-core
// grouped GEMMs with every operand in three BF16 slices (six products, FP32 accumulation):
//   left : stage 1 T^T_beta[n1][j, ql] = sum_{n1'} At^{n1'}[j, ql'] Lt^{n1 n1'}[ql, ql']   (At = A^T per block)
//          stage 2 L'[qa, qa']       = sum_{n1} At^{n1}[qa, ql] T^T_beta[n1][qa', ql]
//   right: stage 1 T_beta[n2][j, qr] = sum_{n2'} B^{n2'}[j, qr'] Rt^{n2 n2'}[qr, qr']
//          stage 2 R'[qb, qb']       = sum_{n2} B^{n2}[qb, qr] T_beta[n2][qb', qr]
// The intermediates are BF16 slices of the FP32 results; the new operators are
// accumulated in FP32 and stored in FP64.
void env_update_tc(Context& c, Tilde& t, const SiteT& A, int site, Env& out, bool left) {
  constexpr int NSL = 3;
  const auto& st = left ? c.mpo.bonds[site + 1] : c.mpo.bonds[site];
  const Bond& Lb = A.L;
  const Bond& Rb = A.R;
  Env& env = *t.env;
  const Bond& ob = left ? Rb : Lb;  // bond of the new operators
  env_alloc(c, out, ob, st);
  const int no = ob.nsec();
  // ---- site-tensor mirror: left: At per block [d(qr) x pad8(d(ql))]; right: [d(ql) x pad8(d(qr))]
  std::vector<long> soff(A.blocks.size());
  long stot = 0;
  for (size_t b = 0; b < A.blocks.size(); ++b) {
    const Block& B = A.blocks[b];
    soff[b] = stot;
    stot += left ? (long)B.cols * pad8(B.rows) : (long)B.rows * pad8(B.cols);
  }
  const long ss = std::max<long>(stot, 8);
  DArr<__nv_bfloat16> smir;
  smir.alloc((size_t)ss * NSL, c.stream);
  {
    if (left) {
      std::vector<ConvTJob> jobs;
      long mx = 0;
      for (size_t b = 0; b < A.blocks.size(); ++b) {
        const Block& B = A.blocks[b];
        jobs.push_back({A.d.p + B.off, smir.p + soff[b], ss, B.rows, B.cols, B.cols, pad8(B.rows), NSL, pad8(B.rows),
                        1.0});
        mx = std::max<long>(mx, (long)B.cols * pad8(B.rows));
      }
      DArr<ConvTJob> dj;
      dj.upload(jobs, c.stream);
      for (int o0 = 0; o0 < (int)jobs.size(); o0 += 65535) {
        const int nj = std::min(65535, (int)jobs.size() - o0);
        const long g = std::min<long>(std::max<long>(1, (mx + 255) / 256), 64);
        convt_kernel<<<dim3((unsigned)g, nj), 256, 0, c.stream>>>(dj.p + o0);
        count_launches(1);
      }
      cuda_check(cudaGetLastError(), "convt launch");
      cuda_check(cudaStreamSynchronize(c.stream), "sync");
    } else {
      std::vector<ConvJob> jobs;
      long mx = 0;
      for (size_t b = 0; b < A.blocks.size(); ++b) {
        const Block& B = A.blocks[b];
        jobs.push_back({A.d.p + B.off, smir.p + soff[b], ss, B.rows, B.cols, B.cols, pad8(B.cols), NSL, 1.0,
                        pad8(B.cols)});
        mx = std::max<long>(mx, (long)B.rows * pad8(B.cols));
      }
      DArr<ConvJob> dj;
      dj.upload(jobs, c.stream);
      if (!jobs.empty()) launch_conv(dj, (int)jobs.size(), mx, c.stream);
      cuda_check(cudaStreamSynchronize(c.stream), "sync");
    }
  }
  // ---- W-contracted operator mirror: every distinct (operator, scale), all blocks,
  // row-major with leading dimension pad8(cols)
  std::vector<std::vector<long>> boff(env.cls.size());
  std::vector<long> bsz(env.cls.size());
  for (size_t i = 0; i < env.cls.size(); ++i) boff[i] = padded_offsets(env.cls[i], &bsz[i]);
  struct KeyHash {
    size_t operator()(const std::pair<const double*, double>& kk) const {
      uint64_t b;
      std::memcpy(&b, &kk.second, sizeof b);
      return std::hash<uint64_t>()((uint64_t)(uintptr_t)kk.first * 0x9e3779b97f4a7c15ULL ^ b);
    }
  };
  std::unordered_map<std::pair<const double*, double>, long, KeyHash> moff;
  std::vector<std::array<long, 16>> mref(st.size());
  std::vector<std::array<char, 16>> mneg(st.size());
  long mtot = 0;
  std::vector<std::pair<const TRef*, long>> created;
  for (size_t beta = 0; beta < st.size(); ++beta)
    for (int nn = 0; nn < 16; ++nn) {
      mref[beta][nn] = -1;
      mneg[beta][nn] = 0;
      const TRef& r = t.ref[beta][nn];
      if (!r.p) continue;
      const double a = std::fabs(r.coef);
      const double scale = a == 1.0 ? 1.0 : r.coef;
      auto key = std::make_pair(r.p, scale);
      auto it = moff.find(key);
      if (it == moff.end()) {
        it = moff.emplace(key, mtot).first;
        created.push_back({&r, mtot});
        mtot += bsz[r.cls];
      }
      mref[beta][nn] = it->second;
      mneg[beta][nn] = (a == 1.0 && r.coef < 0) ? 1 : 0;
    }
  const long ms_ = std::max<long>(mtot, 8);
  DArr<__nv_bfloat16> omir;
  omir.alloc((size_t)ms_ * NSL, c.stream);
  {
    std::vector<ConvJob> jobs;
    long mx = 0;
    for (const auto& cr : created) {
      const TRef& r = *cr.first;
      const double a = std::fabs(r.coef);
      const double scale = a == 1.0 ? 1.0 : r.coef;
      const OpLayout& L = env.cls[r.cls];
      for (size_t b = 0; b < L.blocks.size(); ++b) {
        const Block& B = L.blocks[b];
        jobs.push_back({r.p + B.off, omir.p + cr.second + boff[r.cls][b], ms_, B.rows, B.cols, B.cols, pad8(B.cols),
                        NSL, scale, pad8(B.cols)});
        mx = std::max<long>(mx, (long)B.rows * pad8(B.cols));
      }
    }
    DArr<ConvJob> dj;
    dj.upload(jobs, c.stream);
    if (!jobs.empty()) launch_conv(dj, (int)jobs.size(), mx, c.stream);
    cuda_check(cudaStreamSynchronize(c.stream), "sync");
  }
  // ---- FP32 staging of the new operators (same layout as their FP64 data)
  std::vector<DArr<float>> f32(out.cls.size());
  for (size_t ci = 0; ci < out.cls.size(); ++ci) {
    f32[ci].alloc(std::max<size_t>(out.data[ci].n, 1), c.stream);
    cuda_check(cudaMemsetAsync(f32[ci].p, 0, f32[ci].n * sizeof(float), c.stream), "memset");
  }
  auto f32_op = [&](int beta) {
    return f32[out.st_cls[beta]].p + (size_t)out.st_slot[beta] * out.cls[out.st_cls[beta]].nnz;
  };
  // ---- the intermediate blocks per bond state: left (n1, j): d(j) x pad8(d(ql));
  // right (n2, j): d(j) x pad8(d(qr))
  const Bond& ib = left ? Lb : Rb;  // bond of the contracted index of stage 1
  auto inner_of = [&](int beta, int n, int j) -> int {
    // left: ql with ql + q(n1) + dQ_beta = qr_j; right: qr with qr = ql_j + dQ + q(n2)
    if (left) return Lb.find(Rb.qa[j] + st[beta].dna - LQA[n], Rb.qb[j] + st[beta].dnb - LQB[n]);
    return Rb.find(Lb.qa[j] + st[beta].dna + LQA[n], Lb.qb[j] + st[beta].dnb + LQB[n]);
  };
  std::vector<size_t> tsz(st.size(), 0);
  for (size_t beta = 0; beta < st.size(); ++beta)
    for (int n = 0; n < 4; ++n)
      for (int j = 0; j < no; ++j) {
        const int q = inner_of((int)beta, n, j);
        if (q >= 0) tsz[beta] += (size_t)ob.dim[j] * pad8(ib.dim[q]);
      }
  const size_t budget = std::max<size_t>(1, (size_t)c.chunk_budget_mb * (1u << 20) / (2 * NSL));
  for (size_t b0 = 0; b0 < st.size();) {
    size_t b1 = b0, tot = 0;
    while (b1 < st.size() && (b1 == b0 || tot + tsz[b1] <= budget)) tot += tsz[b1++];
    const long ts = std::max<long>((long)tot, 8);
    DArr<__nv_bfloat16> T;
    T.alloc((size_t)ts * NSL, c.stream);
    cuda_check(cudaMemsetAsync(T.p, 0, T.n * sizeof(__nv_bfloat16), c.stream), "memset");
    TcBuilder g1, g2;
    size_t toff = 0;
    double fl = 0;
    for (size_t beta = b0; beta < b1; ++beta) {
      std::vector<long> tpos((size_t)4 * no, -1);
      for (int n = 0; n < 4; ++n)
        for (int j = 0; j < no; ++j) {
          const int q = inner_of((int)beta, n, j);
          if (q < 0) continue;
          const int m = ob.dim[j], nn = ib.dim[q];
          TcTask tk{};
          tk.Cb = T.p + toff;
          tk.slice_stride = ts;
          tk.ldcb = pad8(nn);
          tk.m = m;
          tk.n = nn;
          tk.nslices = NSL;
          g1.begin(tk);
          for (int np = 0; np < 4; ++np) {
            const int slot = n * 4 + np;
            const TRef& r = t.ref[beta][slot];
            if (!r.p) continue;
            const OpLayout& Lay = env.cls[r.cls];
            int qp, bl, sb;
            if (left) {
              qp = Lb.find(Lb.qa[q] - Lay.da, Lb.qb[q] - Lay.db);  // ql'
              if (qp < 0) continue;
              bl = Lay.blk_of_col[qp];
              if (bl < 0 || Lay.blocks[bl].rs != q) continue;
              sb = A.blk(qp, np);
              if (sb < 0 || A.blocks[sb].cs != j) continue;
            } else {
              qp = Rb.find(Lb.qa[j] + LQA[np], Lb.qb[j] + LQB[np]);  // qr'
              if (qp < 0) continue;
              bl = Lay.blk_of_col[qp];
              if (bl < 0 || Lay.blocks[bl].rs != q) continue;
              sb = A.blk(j, np);
              if (sb < 0 || A.blocks[sb].cs != qp) continue;
            }
            const int kk = ib.dim[qp];
            g1.term(smir.p + soff[sb], ss, pad8(kk), omir.p + mref[beta][slot] + boff[r.cls][bl], ms_, pad8(kk), kk,
                    mneg[beta][slot] != 0, NSL);
            fl += 2.0 * m * nn * kk;
          }
          if (g1.end()) {
            tpos[(size_t)n * no + j] = (long)toff;
            toff += (size_t)m * pad8(nn);
          }
        }
      const OpLayout& Lo = out.lay((int)beta);
      float* obase = f32_op((int)beta);
      for (const Block& B : Lo.blocks) {
        TcTask tk{};
        tk.C = obase + B.off;
        tk.ldc = B.cols;
        tk.m = B.rows;
        tk.n = B.cols;
        g2.begin(tk);
        for (int n = 0; n < 4; ++n) {
          int q, sb;
          if (left) {
            q = Lb.find(Rb.qa[B.rs] - LQA[n], Rb.qb[B.rs] - LQB[n]);  // ql of A^{n}[ql, qa]
            if (q < 0) continue;
            sb = A.blk(q, n);
            if (sb < 0 || A.blocks[sb].cs != B.rs) continue;
          } else {
            q = Rb.find(Lb.qa[B.rs] + LQA[n], Lb.qb[B.rs] + LQB[n]);  // qr of B^{n}[qb, qr]
            if (q < 0) continue;
            sb = A.blk(B.rs, n);
            if (sb < 0 || A.blocks[sb].cs != q) continue;
          }
          const long tp = tpos[(size_t)n * no + B.cs];
          if (tp < 0) continue;
          const int kk = ib.dim[q];
          g2.term(smir.p + soff[sb], ss, pad8(kk), T.p + tp, ts, pad8(kk), kk, false, NSL);
          fl += 2.0 * B.rows * B.cols * kk;
        }
        g2.end();
      }
    }
    c.other_flops_total += fl;
    DArr<int> err;
    err.alloc(1, c.stream);
    cuda_check(cudaMemsetAsync(err.p, 0, sizeof(int), c.stream), "memset");
    DArr<TcTile> t1, t2;
    DArr<TcTask> k1, k2;
    DArr<TcTerm> m1, m2;
    t1.upload(g1.tiles, c.stream);
    k1.upload(g1.tasks, c.stream);
    m1.upload(g1.terms, c.stream);
    t2.upload(g2.tiles, c.stream);
    k2.upload(g2.tasks, c.stream);
    m2.upload(g2.terms, c.stream);
    cuda_check(launch_gemm_bf16_tc(t1.p, (int)g1.tiles.size(), k1.p, m1.p, err.p, c.stream, NSL), "tc env stage 1");
    cuda_check(launch_gemm_bf16_tc(t2.p, (int)g2.tiles.size(), k2.p, m2.p, err.p, c.stream, NSL), "tc env stage 2");
    int h = 0;
    cuda_check(cudaMemcpyAsync(&h, err.p, sizeof(int), cudaMemcpyDeviceToHost, c.stream), "d2h");
    cuda_check(cudaStreamSynchronize(c.stream), "sync");
    if (h) throw Error(ST_ETIMEOUT, "tensor-core GEMM: a bounded wait ran out");
    b0 = b1;
  }
  for (size_t ci = 0; ci < out.cls.size(); ++ci) {
    const long n = (long)out.data[ci].n;
    if (n <= 0) continue;
    f32_to_f64_kernel<<<(unsigned)std::min<long>((n + 255) / 256, 152 * 16), 256, 0, c.stream>>>(f32[ci].p,
                                                                                                  out.data[ci].p, n);
    count_launches(1);
  }
  cuda_check(cudaGetLastError(), "f32 to f64");
  cuda_check(cudaStreamSynchronize(c.stream), "sync");
}

// ---------------------------------------------------------------- exact environment update

// Environment update (Eqs. leftrenorm/rightrenorm, prenormmatrix/prenormdec) on the
// tensor cores with FP64-level results: every FP64 block is scaled by a power of two and
// split into TM_EXACT_SLICES integer slices of 7 bits, exact in BF16; the products of two
// slices summed over a block's K (<= 128 columns, products <= 2^14) are exact integers in
// the FP32 accumulators; pairs of slices of one level i + j share a weight and accumulate
// together (still exact), and the levels are added with their powers of two in two-float
// (hi + lo) registers and stored in FP64.  Dropped pairs (i + j >= slices) and the
// remainder of the splitting are below 2^-42 of each block's largest element.
//   left : E1  T^T_beta[n1][j, ql] = sum_{n1'} At^{n1'}[j, ql'] Lt^{n1 n1'}[ql, ql']
//          E2  L'[qa, qa']        = sum_{n1} At^{n1}[qa, ql] T^T_beta[n1][qa', ql]
//   right: E1  T_beta[n2][j, qr]  = sum_{n2'} B^{n2'}[j, qr'] Rt^{n2 n2'}[qr, qr']
//          E2  R'[qb, qb']        = sum_{n2} B^{n2}[qb, qr] T_beta[n2][qb', qr]
constexpr int TM_EXACT_SLICES = 6;

namespace {

// matrices of one padded width (K dimension) holding blocks stacked by rows
struct WidthClasses {
  std::map<int, int> cls;  // width -> class
  std::vector<int> w;
  std::vector<long> rows, base;
  int of(int width) {
    auto it = cls.find(width);
    if (it != cls.end()) return it->second;
    const int c = (int)w.size();
    cls[width] = c;
    w.push_back(width);
    rows.push_back(0);
    base.push_back(0);
    return c;
  }
  long place(int c, int nrows) {  // row offset of a new block of nrows rows (padded to 16)
    const long r = rows[c];
    rows[c] += pad16(nrows);
    return r;
  }
  long finish() {
    long t = 0;
    for (size_t c = 0; c < w.size(); ++c) {
      base[c] = t;
      t += rows[c] * w[c];
    }
    return std::max<long>(t, 8);
  }
};

}  // namespace

void env_update_exact(Context& c, Tilde& t, const SiteT& A, int site, Env& out, bool left) {
  constexpr int NSL = TM_EXACT_SLICES;
  const auto& st = left ? c.mpo.bonds[site + 1] : c.mpo.bonds[site];
  const Bond& Lb = A.L;
  const Bond& Rb = A.R;
  Env& env = *t.env;
  const Bond& ob = left ? Rb : Lb;  // bond of the new operators
  const Bond& ib = left ? Lb : Rb;  // bond of the contracted index
  env_alloc(c, out, ob, st);
  const int no = ob.nsec();
  const int nmax = tma_max_n(TM_MODE_EXACT_F64);
  std::vector<SplitJob> split1;  // site and operator blocks
  int nexpo = 0;
  // ---- site tensor: left At blocks [d(qr) x d(ql)], right B blocks [d(ql) x d(qr)]; K = columns
  WidthClasses sc;
  std::vector<int> s_cls(A.blocks.size()), s_exp(A.blocks.size());
  std::vector<long> s_row(A.blocks.size());
  for (size_t b = 0; b < A.blocks.size(); ++b) {
    const Block& B = A.blocks[b];
    const int rows = left ? B.cols : B.rows, kdim = left ? B.rows : B.cols;
    s_cls[b] = sc.of(pad16(kdim));
    s_row[b] = sc.place(s_cls[b], rows);
    s_exp[b] = nexpo++;
  }
  const long ss = sc.finish();
  DArr<__nv_bfloat16> smir;
  smir.alloc((size_t)ss * NSL, c.stream);
  cuda_check(cudaMemsetAsync(smir.p, 0, smir.n * sizeof(__nv_bfloat16), c.stream), "memset");
  for (size_t b = 0; b < A.blocks.size(); ++b) {
    const Block& B = A.blocks[b];
    const int w = sc.w[s_cls[b]];
    split1.push_back({A.d.p + B.off, smir.p + sc.base[s_cls[b]] + s_row[b] * w, ss, B.rows, B.cols, B.cols, w,
                      left ? B.cols : pad16(B.cols), left ? 1 : 0, s_exp[b], 1.0});
  }
  // ---- W-contracted operators: every distinct (operator, coefficient), all blocks; K = columns
  WidthClasses oc;
  struct KeyHash {
    size_t operator()(const std::pair<const double*, double>& kk) const {
      uint64_t b;
      std::memcpy(&b, &kk.second, sizeof b);
      return std::hash<uint64_t>()((uint64_t)(uintptr_t)kk.first * 0x9e3779b97f4a7c15ULL ^ b);
    }
  };
  std::unordered_map<std::pair<const double*, double>, int, KeyHash> mid_of;
  std::vector<std::vector<long>> m_row;  // per mirror, per block
  std::vector<std::vector<int>> m_exp;
  std::vector<int> m_cls_of_ref;
  struct PendO {
    const double* src;
    int cls;
    long row;
    int rows, cols, ex;
    double coef;
  };
  std::vector<PendO> opend;
  std::vector<std::array<int, 16>> mref(st.size());
  for (size_t beta = 0; beta < st.size(); ++beta)
    for (int nn = 0; nn < 16; ++nn) {
      mref[beta][nn] = -1;
      const TRef& r = t.ref[beta][nn];
      if (!r.p) continue;
      auto key = std::make_pair(r.p, r.coef);
      auto it = mid_of.find(key);
      if (it == mid_of.end()) {
        const int id = (int)m_row.size();
        it = mid_of.emplace(key, id).first;
        const OpLayout& L = env.cls[r.cls];
        m_row.emplace_back(L.blocks.size());
        m_exp.emplace_back(L.blocks.size());
        for (size_t b = 0; b < L.blocks.size(); ++b) {
          const Block& B = L.blocks[b];
          const int cl = oc.of(pad16(B.cols));
          m_row[id][b] = oc.place(cl, B.rows);
          m_exp[id][b] = nexpo++;
          opend.push_back({r.p + B.off, cl, m_row[id][b], B.rows, B.cols, m_exp[id][b], r.coef});
        }
      }
      mref[beta][nn] = it->second;
    }
  const long os = oc.finish();
  DArr<__nv_bfloat16> omir;
  omir.alloc((size_t)os * NSL, c.stream);
  cuda_check(cudaMemsetAsync(omir.p, 0, omir.n * sizeof(__nv_bfloat16), c.stream), "memset");
  for (const PendO& po : opend) {
    const int w = oc.w[po.cls];
    split1.push_back({po.src, omir.p + oc.base[po.cls] + po.row * w, os, po.rows, po.cols, po.cols, w, po.cols, 0,
                      po.ex, po.coef});
  }
  // ---- intermediate T blocks (FP64) per (beta, n, j): d(j) x d(q) with q the inner sector
  auto inner_of = [&](size_t beta, int n, int j) -> int {
    if (left) return Lb.find(Rb.qa[j] + st[beta].dna - LQA[n], Rb.qb[j] + st[beta].dnb - LQB[n]);
    return Rb.find(Lb.qa[j] + st[beta].dna + LQA[n], Lb.qb[j] + st[beta].dnb + LQB[n]);
  };
  // the source terms (site block, mirror, operator block) of the T block (beta, n, j)
  auto sources = [&](size_t beta, int n, int j, int q, std::vector<std::array<int, 3>>& src, double& fl) {
    src.clear();
    for (int np = 0; np < 4; ++np) {
      const int slot = n * 4 + np;
      const TRef& r = t.ref[beta][slot];
      if (!r.p) continue;
      const OpLayout& Lay = env.cls[r.cls];
      int qp, bl, sb;
      if (left) {
        qp = Lb.find(Lb.qa[q] - Lay.da, Lb.qb[q] - Lay.db);
        if (qp < 0) continue;
        bl = Lay.blk_of_col[qp];
        if (bl < 0 || Lay.blocks[bl].rs != q) continue;
        sb = A.blk(qp, np);
        if (sb < 0 || A.blocks[sb].cs != j) continue;
      } else {
        qp = Rb.find(Lb.qa[j] + LQA[np], Lb.qb[j] + LQB[np]);
        if (qp < 0) continue;
        bl = Lay.blk_of_col[qp];
        if (bl < 0 || Lay.blocks[bl].rs != q) continue;
        sb = A.blk(j, np);
        if (sb < 0 || A.blocks[sb].cs != qp) continue;
      }
      src.push_back({sb, mref[beta][slot], bl});
      fl += 2.0 * ob.dim[j] * ib.dim[q] * ib.dim[qp];
    }
  };
  // chunks of bond states whose T blocks (FP64 + slices, 18 bytes per element) fit the budget
  std::vector<size_t> tsz(st.size(), 0);
  for (size_t beta = 0; beta < st.size(); ++beta)
    for (int n = 0; n < 4; ++n)
      for (int j = 0; j < no; ++j) {
        const int q = inner_of(beta, n, j);
        if (q >= 0) tsz[beta] += (size_t)pad16(ob.dim[j]) * pad16(ib.dim[q]);
      }
  const size_t budget = std::max<size_t>(1, (size_t)c.chunk_budget_mb * (1u << 20) / (8 + 2 * NSL));
  // split of the site and operator blocks (shared by all chunks)
  const int nexpo_fixed = nexpo;
  int max_texp = 0;
  for (size_t b0 = 0, b1; b0 < st.size(); b0 = b1) {
    size_t tot = 0;
    for (b1 = b0; b1 < st.size() && (b1 == b0 || tot + tsz[b1] <= budget); ++b1) tot += tsz[b1];
    int cnt = 0;
    for (size_t beta = b0; beta < b1; ++beta)
      for (int n = 0; n < 4; ++n)
        for (int j = 0; j < no; ++j) cnt += inner_of(beta, n, j) >= 0;
    max_texp = std::max(max_texp, cnt);
  }
  DArr<int> expo;
  expo.alloc(std::max(nexpo_fixed + max_texp, 1), c.stream);
  DArr<int> err;
  err.alloc(1, c.stream);
  cuda_check(cudaMemsetAsync(err.p, 0, sizeof(int), c.stream), "memset");
  DArr<SplitJob> dj1;
  dj1.upload(split1, c.stream);
  for (const SplitJob& j : split1)
    if (j.rows < 1 || j.cols < 1 || j.expo < 0 || j.expo >= nexpo_fixed) throw Error(ST_ECUDA, "internal: split job");
  cuda_check(launch_split_exact(dj1.p, (int)split1.size(), NSL, expo.p, c.stream), "exact split");
  // tensor maps of the site and operator classes (per slice; operators per box height)
  std::vector<CUtensorMap> maps;
  auto add_map = [&](const DArr<__nv_bfloat16>& buf, long off, long stride, long rows, int w, int box) {
    const int first = (int)maps.size();
    for (int sl = 0; sl < NSL; ++sl) {
      const long o = off + sl * stride;
      if (rows < 1 || o < 0 || o % 8 || (size_t)(o + rows * w) > buf.n)
        throw Error(ST_ECUDA, "internal: tensor map outside its buffer");
      CUtensorMap m;
      if (!encode_bf16_map(&m, buf.p + o, (uint64_t)rows, (uint64_t)w, (uint64_t)w, (uint32_t)box))
        throw Error(ST_ECUDA, "cuTensorMapEncodeTiled failed");
      maps.push_back(m);
    }
    return first;
  };
  std::vector<int> smap(sc.w.size(), -1);
  for (size_t k = 0; k < sc.w.size(); ++k)
    if (sc.rows[k] > 0) smap[k] = add_map(smir, sc.base[k], ss, sc.rows[k], sc.w[k], 128);
  std::vector<std::vector<int>> omap(oc.w.size(), std::vector<int>(nmax / 16 + 1, -1));
  for (size_t k = 0; k < oc.w.size(); ++k)
    if (oc.rows[k] > 0)
      for (int h = 16; h <= nmax; h += 16) omap[k][h / 16] = add_map(omir, oc.base[k], os, oc.rows[k], oc.w[k], h);
  const size_t nfixed_maps = maps.size();
  double fl = 0;
  std::vector<std::array<int, 3>> src;
  for (size_t b0 = 0, b1; b0 < st.size(); b0 = b1) {
    size_t tot = 0;
    for (b1 = b0; b1 < st.size() && (b1 == b0 || tot + tsz[b1] <= budget); ++b1) tot += tsz[b1];
    maps.resize(nfixed_maps);
    // T layout of this chunk: FP64 blocks, their slices by width class, their exponents
    const size_t nb = b1 - b0;
    std::vector<long> tpos(nb * 4 * no, -1), t_row(nb * 4 * no, -1);
    std::vector<int> t_cls(nb * 4 * no, -1), t_exp(nb * 4 * no, -1);
    WidthClasses tcw;
    long ttot = 0;
    int nte = nexpo_fixed;
    struct E1 {
      size_t tix;
      int r0, c0, m_valid, nvalid, cols;
      size_t s0, s1;  // range in srcs
    };
    std::vector<E1> e1x;
    std::vector<std::array<int, 3>> srcs;
    for (size_t beta = b0; beta < b1; ++beta)
      for (int n = 0; n < 4; ++n)
        for (int j = 0; j < no; ++j) {
          const int q = inner_of(beta, n, j);
          if (q < 0) continue;
          sources(beta, n, j, q, src, fl);
          if (src.empty()) continue;
          const size_t tix = ((beta - b0) * 4 + n) * no + j;
          const int rows = ob.dim[j], cols = ib.dim[q];
          tpos[tix] = ttot;
          ttot += (long)rows * cols;
          t_cls[tix] = tcw.of(pad16(cols));
          t_row[tix] = tcw.place(t_cls[tix], rows);
          t_exp[tix] = nte++;
          const size_t s0 = srcs.size();
          srcs.insert(srcs.end(), src.begin(), src.end());
          for (int r0 = 0; r0 < rows; r0 += 128)
            for (int c0 = 0; c0 < cols; c0 += nmax)
              e1x.push_back({tix, r0, c0, std::min(128, rows - r0), std::min(nmax, cols - c0), cols, s0, srcs.size()});
        }
    const long ts = tcw.finish();
    DArr<double> T64;
    T64.alloc(std::max<long>(ttot, 1), c.stream);
    DArr<__nv_bfloat16> tmir;
    tmir.alloc((size_t)ts * NSL, c.stream);
    cuda_check(cudaMemsetAsync(tmir.p, 0, tmir.n * sizeof(__nv_bfloat16), c.stream), "memset");
    std::vector<std::vector<int>> tmap(tcw.w.size(), std::vector<int>(nmax / 16 + 1, -1));
    for (size_t k = 0; k < tcw.w.size(); ++k)
      if (tcw.rows[k] > 0)
        for (int h = 16; h <= nmax; h += 16) tmap[k][h / 16] = add_map(tmir, tcw.base[k], ts, tcw.rows[k], tcw.w[k], h);
    // E1 tiles: T block (rows, <= 64 columns) per tile; contractions cut into <= 128 columns
    std::vector<TmTile> e1t;
    std::vector<TmTerm> e1m;
    for (const E1& x : e1x) {
      TmTile tl{};
      tl.t0 = (int)e1m.size();
      tl.m_valid = x.m_valid;
      tl.nvalid = x.nvalid;
      tl.n = pad16(x.nvalid);
      for (size_t si = x.s0; si < x.s1; ++si) {
        const auto& sr = srcs[si];
        const Block& SB = A.blocks[sr[0]];
        const int kdim = left ? SB.rows : SB.cols;
        for (int kc = 0; kc < pad16(kdim); kc += 128)
          e1m.push_back({smap[s_cls[sr[0]]], omap[oc.cls[pad16(kdim)]][tl.n / 16], kc, (int)(s_row[sr[0]] + x.r0), kc,
                         (int)(m_row[sr[1]][sr[2]] + x.c0), std::min(128, pad16(kdim) - kc), NSL << 4, s_exp[sr[0]],
                         m_exp[sr[1]][sr[2]]});
      }
      tl.t1 = (int)e1m.size();
      tl.ldo = x.cols;
      tl.out_off = tpos[x.tix] + (long)x.r0 * x.cols + x.c0;
      e1t.push_back(tl);
    }
    // split of this chunk's T blocks
    std::vector<SplitJob> split2;
    for (size_t tix = 0; tix < tpos.size(); ++tix) {
      if (tpos[tix] < 0) continue;
      const int j = (int)(tix % no), n = (int)((tix / no) % 4);
      const size_t beta = b0 + tix / ((size_t)4 * no);
      const int rows = ob.dim[j], cols = ib.dim[inner_of(beta, n, j)];
      const int w = tcw.w[t_cls[tix]];
      split2.push_back({T64.p + tpos[tix], tmir.p + tcw.base[t_cls[tix]] + t_row[tix] * w, ts, rows, cols, cols, w,
                        pad16(cols), 0, t_exp[tix], 1.0});
    }
    // E2 tiles: every block of every new operator of the chunk, per output class
    std::vector<std::vector<TmTile>> e2t(out.cls.size());
    std::vector<TmTerm> e2m;
    std::vector<std::array<int, 2>> s2;
    for (size_t beta = b0; beta < b1; ++beta) {
      const OpLayout& Lo = out.lay((int)beta);
      const int oc_ = out.st_cls[(int)beta];
      const long obase = (long)(out.op((int)beta) - out.data[oc_].p);
      for (const Block& B : Lo.blocks) {
        s2.clear();
        for (int n = 0; n < 4; ++n) {
          int q, sb;
          if (left) {
            q = Lb.find(Rb.qa[B.rs] - LQA[n], Rb.qb[B.rs] - LQB[n]);
            if (q < 0) continue;
            sb = A.blk(q, n);
            if (sb < 0 || A.blocks[sb].cs != B.rs) continue;
          } else {
            q = Rb.find(Lb.qa[B.rs] + LQA[n], Lb.qb[B.rs] + LQB[n]);
            if (q < 0) continue;
            sb = A.blk(B.rs, n);
            if (sb < 0 || A.blocks[sb].cs != q) continue;
          }
          const size_t tix = ((beta - b0) * 4 + n) * no + B.cs;
          if (tpos[tix] < 0) continue;
          s2.push_back({sb, (int)tix});
          fl += 2.0 * B.rows * B.cols * ib.dim[q];
        }
        if (s2.empty()) continue;
        for (int r0 = 0; r0 < B.rows; r0 += 128)
          for (int c0 = 0; c0 < B.cols; c0 += nmax) {
            TmTile tl{};
            tl.t0 = (int)e2m.size();
            tl.m_valid = std::min(128, B.rows - r0);
            tl.nvalid = std::min(nmax, B.cols - c0);
            tl.n = pad16(tl.nvalid);
            for (const auto& sr : s2) {
              const Block& SB = A.blocks[sr[0]];
              const int kdim = left ? SB.rows : SB.cols;
              for (int kc = 0; kc < pad16(kdim); kc += 128)
                e2m.push_back({smap[s_cls[sr[0]]], tmap[t_cls[(size_t)sr[1]]][tl.n / 16], kc, (int)(s_row[sr[0]] + r0),
                               kc, (int)(t_row[(size_t)sr[1]] + c0), std::min(128, pad16(kdim) - kc), NSL << 4,
                               s_exp[sr[0]], t_exp[(size_t)sr[1]]});
            }
            tl.t1 = (int)e2m.size();
            tl.ldo = B.cols;
            tl.out_off = obase + B.off + (long)r0 * B.cols + c0;
            e2t[(size_t)oc_].push_back(tl);
          }
      }
    }
    // bounds of every output, term and split job before anything runs
    for (const TmTile& tl : e1t)
      if (tl.out_off < 0 || tl.out_off + (long)(tl.m_valid - 1) * tl.ldo + tl.nvalid > (long)T64.n || tl.n > nmax ||
          tl.nvalid > tl.n || tl.t1 <= tl.t0)
        throw Error(ST_ECUDA, "internal: exact stage-1 tile");
    for (size_t ci = 0; ci < e2t.size(); ++ci)
      for (const TmTile& tl : e2t[ci])
        if (tl.out_off < 0 || (size_t)(tl.out_off + (long)(tl.m_valid - 1) * tl.ldo + tl.nvalid) > out.data[ci].n ||
            tl.n > nmax || tl.nvalid > tl.n || tl.t1 <= tl.t0)
          throw Error(ST_ECUDA, "internal: exact stage-2 tile");
    auto check_m = [&](const std::vector<TmTerm>& mm) {
      for (const TmTerm& m : mm)
        if (m.amap < 0 || m.amap + NSL > (int)maps.size() || m.bmap < 0 || m.bmap + NSL > (int)maps.size() ||
            m.k < 16 || m.k % 16 || m.k > 128 || m.ax % 16 || m.ea < 0 || m.ea >= nte || m.eb < 0 || m.eb >= nte ||
            ((m.neg >> 4) & 15) != NSL)
          throw Error(ST_ECUDA, "internal: exact term");
    };
    check_m(e1m);
    check_m(e2m);
    for (const SplitJob& j : split2)
      if (j.rows < 1 || j.cols < 1 || j.expo < nexpo_fixed || j.expo >= nte) throw Error(ST_ECUDA, "internal: split job");
    // run: E1, split T, E2 (one launch per output class of the new operators)
    DArr<CUtensorMap> dmaps;
    dmaps.upload(maps, c.stream);
    DArr<TmTile> d1t;
    DArr<TmTerm> d1m, d2m;
    // copy lists of every launch; each piece reads through one of this update's maps
    // copy lists of every launch (their pieces follow from the terms checked above)
    TmaPlan::Lists dl1;
    dl1.plan(TM_MODE_EXACT_F64, e1t, e1m, c.stream);
    d1t.upload(e1t, c.stream);
    d1m.upload(e1m, c.stream);
    dl1.fill(TM_MODE_EXACT_F64, d1t.p, (int)e1t.size(), d1m.p, c.stream);
    cuda_check(launch_gemm_tma(TM_MODE_EXACT_F64, d1t.p, (int)e1t.size(), d1m.p, dmaps.p, nullptr, nullptr, T64.p, 1, 0,
                               err.p, c.stream, dl1.dev(), expo.p),
               "exact stage 1");
    DArr<SplitJob> dj2;
    dj2.upload(split2, c.stream);
    cuda_check(launch_split_exact(dj2.p, (int)split2.size(), NSL, expo.p, c.stream), "exact split of T");
    d2m.upload(e2m, c.stream);
    std::vector<DArr<TmTile>> d2t(out.cls.size());
    std::vector<TmaPlan::Lists> dl2(out.cls.size());
    for (size_t ci = 0; ci < out.cls.size(); ++ci) {
      if (e2t[ci].empty()) continue;
      dl2[ci].plan(TM_MODE_EXACT_F64, e2t[ci], e2m, c.stream);
      d2t[ci].upload(e2t[ci], c.stream);
      dl2[ci].fill(TM_MODE_EXACT_F64, d2t[ci].p, (int)e2t[ci].size(), d2m.p, c.stream);
      cuda_check(launch_gemm_tma(TM_MODE_EXACT_F64, d2t[ci].p, (int)e2t[ci].size(), d2m.p, dmaps.p, nullptr, nullptr,
                                 out.data[ci].p, 1, 0, err.p, c.stream, dl2[ci].dev(), expo.p),
                 "exact stage 2");
    }
    // the host lists and the chunk's buffers must outlive the launches
    cuda_check(cudaStreamSynchronize(c.stream), "sync");
  }
  c.other_flops_total += fl;
  int h = 0;
  cuda_check(cudaMemcpyAsync(&h, err.p, sizeof(int), cudaMemcpyDeviceToHost, c.stream), "d2h");
  cuda_check(cudaStreamSynchronize(c.stream), "sync");
  if (h) throw Error(ST_ETIMEOUT, "tensor-core GEMM: a bounded wait ran out");
}

// ---------------------------------------------------------------- batched sigma

// Several independent two-site problems (each prepared in tensor-core precision
// on the same device) fused into one launch per stage and chunk: the tile, task
// and term lists are concatenated, so one persistent kernel walks the tiles of
// every problem.  Optionally the whole sequence (conversions, stage launches,
// gathers) is captured once in a CUDA graph and replayed.
struct BatchPlan {
  std::vector<Context*> ctx;
  cudaStream_t stream = nullptr;
  std::vector<TcPlan> stage1, stage2;
  DArr<ConvJob> conv;
  DArr<UnconvJob> unconv;
  int nconv = 0, nunconv = 0;
  long conv_maxel = 0, unconv_maxel = 0;
  DArr<int> err;
  cudaGraph_t graph = nullptr;
  cudaGraphExec_t exec = nullptr;
  long graph_launches = 0, graph_tc_launches = 0;  // kernels in one replay of the graph
  int nsl = 1;                                      // largest slice count of the problems
  double flops = 0;
  ~BatchPlan() {
    if (exec) cudaGraphExecDestroy(exec);
    if (graph) cudaGraphDestroy(graph);
  }
};

static void concat_into(TcPlan& out, const std::vector<const TcPlan*>& parts, cudaStream_t s) {
  std::vector<TcTile> ti;
  std::vector<TcTask> ta;
  std::vector<TcTerm> te;
  std::vector<ZeroJob> zj;
  for (const TcPlan* p : parts) {
    if (p->ntiles && p->htiles.empty()) throw Error(ST_ESTATE, "batched sigma: plan was built without host copies");
    const int toff = (int)ta.size(), eoff = (int)te.size();
    for (TcTask t : p->htasks) {
      t.t0 += eoff;
      t.t1 += eoff;
      ta.push_back(t);
    }
    te.insert(te.end(), p->hterms.begin(), p->hterms.end());
    for (TcTile x : p->htiles) {
      x.task += toff;
      ti.push_back(x);
    }
    zj.insert(zj.end(), p->hzeros.begin(), p->hzeros.end());
    out.zmax = std::max(out.zmax, p->zmax);
  }
  out.tiles.upload(ti, s);
  out.tasks.upload(ta, s);
  out.terms.upload(te, s);
  out.ntiles = (int)ti.size();
  out.nzeros = (int)zj.size();
  out.zeros.upload(zj, s);
  out.hzeros = zj;
  cuda_check(cudaStreamSynchronize(s), "sync");
}

BatchPlan* batch_create(const std::vector<Context*>& ctxs) {
  auto* b = new BatchPlan();
  b->ctx = ctxs;
  b->stream = ctxs[0]->stream;
  size_t nch = 0;
  std::vector<ConvJob> cj;
  std::vector<UnconvJob> uj;
  for (Context* c : ctxs) {
    if (c->prepared < 0 || !c->plan.mx) {
      delete b;
      throw Error(ST_ESTATE,
                  "batched sigma: every context must be prepared in a tensor-core precision of the cp.async plan (1-3)");
    }
    MixedPlan& mx = *c->plan.mx;
    nch = std::max(nch, mx.stage1.size());
    cj.insert(cj.end(), mx.h_psi_jobs.begin(), mx.h_psi_jobs.end());
    uj.insert(uj.end(), mx.h_sig_jobs.begin(), mx.h_sig_jobs.end());
    b->conv_maxel = std::max(b->conv_maxel, mx.psi_maxel);
    b->unconv_maxel = std::max(b->unconv_maxel, mx.sig_maxel);
    b->flops += c->plan.flops;
    b->nsl = std::max(b->nsl, mx.nsl);
  }
  try {
    for (size_t ch = 0; ch < nch; ++ch) {
      std::vector<const TcPlan*> p1, p2;
      for (Context* c : ctxs) {
        MixedPlan& mx = *c->plan.mx;
        if (ch < mx.stage1.size()) {
          p1.push_back(&mx.stage1[ch]);
          p2.push_back(&mx.stage2[ch]);
        }
      }
      b->stage1.emplace_back();
      concat_into(b->stage1.back(), p1, b->stream);
      b->stage2.emplace_back();
      concat_into(b->stage2.back(), p2, b->stream);
    }
    b->conv.upload(cj, b->stream);
    b->nconv = (int)cj.size();
    b->unconv.upload(uj, b->stream);
    b->nunconv = (int)uj.size();
    b->err.alloc(1, b->stream);
    cuda_check(cudaMemsetAsync(b->err.p, 0, sizeof(int), b->stream), "memset");
    cuda_check(cudaStreamSynchronize(b->stream), "sync");
  } catch (...) {
    delete b;
    throw;
  }
  return b;
}

void batch_free(BatchPlan* b) {
  if (b && b->stream) cudaStreamSynchronize(b->stream);
  delete b;
}
double batch_flops(const BatchPlan* b) { return b->flops; }

// the device work of one batched sigma (plan.in -> plan.out of every problem)
static void batch_enqueue(BatchPlan& b) {
  cudaStream_t s = b.stream;
  for (Context* c : b.ctx) {
    MixedPlan& mx = *c->plan.mx;
    cuda_check(cudaMemsetAsync(mx.sig_f.p, 0, mx.sig_total * sizeof(float), s), "memset");
  }
  if (b.nconv) launch_conv(b.conv, b.nconv, b.conv_maxel, s);
  for (size_t i = 0; i < b.stage1.size(); ++i) {
    run_zeros(b.stage1[i], s);
    cuda_check(launch_gemm_bf16_tc(b.stage1[i].tiles.p, b.stage1[i].ntiles, b.stage1[i].tasks.p,
                                   b.stage1[i].terms.p, b.err.p, s, b.nsl),
               "tc stage 1");
    cuda_check(launch_gemm_bf16_tc(b.stage2[i].tiles.p, b.stage2[i].ntiles, b.stage2[i].tasks.p,
                                   b.stage2[i].terms.p, b.err.p, s, b.nsl),
               "tc stage 2");
  }
  if (b.nunconv) launch_unconv(b.unconv.p, b.nunconv, b.unconv_maxel, s);
}

float batch_sigma(BatchPlan& b, const double* const* psi, double* const* sigma, bool use_graph) {
  cudaStream_t s = b.stream;
  for (size_t p = 0; p < b.ctx.size(); ++p) {
    SigmaPlan& pl = b.ctx[p]->plan;
    cuda_check(cudaMemcpyAsync(pl.in.p, psi[p], pl.psi.nnz * sizeof(double), cudaMemcpyDeviceToDevice, s), "d2d");
  }
  cudaEvent_t e0, e1;
  cuda_check(cudaEventCreate(&e0), "event");
  cuda_check(cudaEventCreate(&e1), "event");
  cuda_check(cudaEventRecord(e0, s), "record");
  if (use_graph && b.exec) {
    cuda_check(cudaGraphLaunch(b.exec, s), "graph launch");
    count_launches(b.graph_launches);
    count_tc_launches(b.graph_tc_launches);
  } else {
    batch_enqueue(b);
  }
  cuda_check(cudaEventRecord(e1, s), "record");
  if (use_graph && !b.exec) {
    // captured after one eager pass (which set up every launch attribute); the
    // captured work does not run now, later calls replay it
    const long l0 = launch_count(), t0 = tc_launch_count();
    cuda_check(cudaStreamBeginCapture(s, cudaStreamCaptureModeThreadLocal), "begin capture");
    batch_enqueue(b);
    cuda_check(cudaStreamEndCapture(s, &b.graph), "end capture");
    // captured launches run only when the graph is replayed: count them there
    b.graph_launches = launch_count() - l0;
    b.graph_tc_launches = tc_launch_count() - t0;
    count_launches(-b.graph_launches);
    count_tc_launches(-b.graph_tc_launches);
    cuda_check(cudaGraphInstantiate(&b.exec, b.graph, 0), "graph instantiate");
  }
  for (size_t p = 0; p < b.ctx.size(); ++p) {
    SigmaPlan& pl = b.ctx[p]->plan;
    cuda_check(cudaMemcpyAsync(sigma[p], pl.out.p, pl.psi.nnz * sizeof(double), cudaMemcpyDeviceToDevice, s), "d2d");
  }
  cuda_check(cudaEventSynchronize(e1), "sync");
  float ms = 0;
  cudaEventElapsedTime(&ms, e0, e1);
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  int h = 0;
  cuda_check(cudaMemcpy(&h, b.err.p, sizeof(int), cudaMemcpyDeviceToHost), "d2h");
  if (h) throw Error(ST_ETIMEOUT, "tensor-core GEMM: a bounded wait ran out");
  cuda_check(cudaStreamSynchronize(s), "sync");
  return ms;
}


// ---------------------------------------------------------------- blocking sums on the tensor cores

// out_i = sum_j coef_ij Op_j for the operators Op_j of one class (Sec. "Efficient
// implementation of expectation values": the W contraction with the renormalised
// operators) as one GEMM per class: A = the class's operators transposed into BF16
// slices (element-major, operator index contiguous), B = the coefficient matrix in BF16
// slices, FP32 accumulation, the result gathered into the FP64 outputs.  Three slices
// carry ~24 significant bits, so the sums have about FP32 accuracy.
void combos_tc(Context& c, Env& env, const std::vector<ComboOut>& outs, const std::vector<ComboTerm>& terms,
               const std::vector<int>& out_cls) {
  const int nsl = 3;
  DArr<int> err;
  err.alloc(1, c.stream);
  cuda_check(cudaMemsetAsync(err.p, 0, sizeof(int), c.stream), "memset");
  std::vector<std::vector<size_t>> by_cls(env.cls.size());
  for (size_t i = 0; i < outs.size(); ++i) by_cls[(size_t)out_cls[i]].push_back(i);
  for (size_t cls = 0; cls < env.cls.size(); ++cls) {
    const std::vector<size_t>& mine = by_cls[cls];
    if (mine.empty()) continue;
    const long nnz = env.cls[cls].nnz;
    const int K = env.nslot[cls];
    const int Kp = pad8(K);
    const int S = (int)mine.size();
    if (nnz <= 0 || K <= 0) continue;
    if (nnz > (long)std::numeric_limits<int>::max())
      throw Error(ST_EINVAL, "tensor-core blocking sums: operator class too large");
    const double* base = env.data[cls].p;
    // A: operators transposed, [nnz x Kp] per slice (padding columns zero)
    DArr<__nv_bfloat16> at, bt;
    at.alloc((size_t)nnz * Kp * nsl, c.stream);
    cuda_check(cudaMemsetAsync(at.p, 0, at.n * sizeof(__nv_bfloat16), c.stream), "memset");
    std::vector<ConvJob> jobs;
    jobs.reserve((size_t)K + 1);
    for (int j = 0; j < K; ++j)
      jobs.push_back({base + (long)j * nnz, at.p + j, nnz * Kp, (int)nnz, 1, 1, Kp, nsl, 1.0, 1});
    // B: coefficients [S x Kp] (a repeated operator in one sum adds up)
    std::vector<double> coef((size_t)S * Kp, 0.0);
    for (int sidx = 0; sidx < S; ++sidx) {
      const ComboOut& o = outs[mine[(size_t)sidx]];
      for (int t = o.t0; t < o.t1; ++t) {
        const long d = (long)(terms[(size_t)t].in - base);
        if (d < 0 || d % nnz != 0 || d / nnz >= K)
          throw Error(ST_ECUDA, "internal: blocking-sum term outside its operator class");
        coef[(size_t)sidx * Kp + (size_t)(d / nnz)] += terms[(size_t)t].coef;
      }
    }
    DArr<double> coef_d;
    coef_d.upload(coef, c.stream);
    bt.alloc((size_t)S * Kp * nsl, c.stream);
    jobs.push_back({coef_d.p, bt.p, (long)S * Kp, S, Kp, Kp, Kp, nsl, 1.0, Kp});
    {
      DArr<ConvJob> dj;
      dj.upload(jobs, c.stream);
      launch_conv(dj, (int)jobs.size(), std::max<long>(nnz, (long)S * Kp), c.stream);
    }
    // C^T [S x nnz] in FP32: element (e, i) of the product goes to ct[i * nnz + e]
    DArr<float> ct;
    ct.alloc((size_t)S * nnz, c.stream);
    TcBuilder g;
    TcTask task{};
    task.C = ct.p;
    task.ldc = (int)nnz;
    task.m = (int)nnz;
    task.n = S;
    task.beta = 0;
    task.trans = 1;
    g.begin(task);
    g.term(at.p, nnz * Kp, Kp, bt.p, (long)S * Kp, Kp, K, false, nsl);
    g.end();
    DArr<TcTile> d_tiles;
    DArr<TcTask> d_tasks;
    DArr<TcTerm> d_terms;
    d_tiles.upload(g.tiles, c.stream);
    d_tasks.upload(g.tasks, c.stream);
    d_terms.upload(g.terms, c.stream);
    cuda_check(launch_gemm_bf16_tc(d_tiles.p, (int)g.tiles.size(), d_tasks.p, d_terms.p, err.p, c.stream, nsl),
               "tc blocking sums");
    // gather into the FP64 outputs (a plain copy: one column per job)
    std::vector<UnconvJob> uj;
    uj.reserve((size_t)S);
    for (int sidx = 0; sidx < S; ++sidx)
      uj.push_back({ct.p + (long)sidx * nnz, outs[mine[(size_t)sidx]].out, (int)nnz, 1, 1});
    DArr<UnconvJob> du;
    du.upload(uj, c.stream);
    launch_unconv(du.p, (int)uj.size(), nnz, c.stream);
    cuda_check(cudaStreamSynchronize(c.stream), "sync");
  }
  int h = 0;
  cuda_check(cudaMemcpy(&h, err.p, sizeof(int), cudaMemcpyDeviceToHost), "d2h");
  if (h) throw Error(ST_ETIMEOUT, "tensor-core GEMM: a bounded wait ran out");
}

// ---------------------------------------------------------------- autotuner

TuneChoice autotune_plans(const std::vector<Context*>& ctxs, const std::vector<double>& splits,
                          const std::vector<int>& budgets, int reps, std::vector<double>& ms) {
  if (ctxs.empty() || splits.empty() || budgets.empty() || reps <= 0)
    throw Error(ST_EINVAL, "autotune: empty problem or candidate list");
  for (int b : budgets)
    if (b <= 0) throw Error(ST_EINVAL, "autotune: chunk budgets must be positive");
  const bool batched = ctxs.size() > 1;
  for (Context* c : ctxs) {
    if (c->prepared < 0 || !c->plan.mx)
      throw Error(ST_ESTATE, "autotune: every context must be prepared in a tensor-core precision");
    if (batched && !c->keep_host_plans)
      throw Error(ST_ESTATE, "autotune: tuning a batch needs host copies of the plans (keep_host_plans)");
  }
  // inputs and outputs of the timed calls: zero vectors (the time does not depend on
  // the values), sized for the prepared problems, whose layouts no candidate changes
  std::vector<DArr<double>> in(ctxs.size()), out(ctxs.size());
  std::vector<const double*> pin(ctxs.size());
  std::vector<double*> pout(ctxs.size());
  for (size_t i = 0; i < ctxs.size(); ++i) {
    Context& c = *ctxs[i];
    const size_t n = std::max<size_t>(c.plan.psi.nnz, 1);
    in[i].alloc(n, c.stream);
    out[i].alloc(n, c.stream);
    cuda_check(cudaMemsetAsync(in[i].p, 0, n * sizeof(double), c.stream), "memset");
    cuda_check(cudaStreamSynchronize(c.stream), "sync");
    pin[i] = in[i].p;
    pout[i] = out[i].p;
  }
  auto rebuild = [&](double split, int budget) {
    for (Context* c : ctxs) {
      c->split_tps = split;
      c->chunk_budget_mb = budget;
      build_sigma_plan(*c, c->lt, c->rt, c->prepared, c->plan);
      cuda_check(cudaStreamSynchronize(c->stream), "sync");
    }
  };
  ms.assign(splits.size() * budgets.size(), 0.0);
  size_t best = 0;
  // on an error the contexts get their parameters back and must be prepared again
  std::vector<std::pair<double, int>> saved;
  for (Context* c : ctxs) saved.emplace_back(c->split_tps, c->chunk_budget_mb);
  try {
    for (size_t i = 0; i < splits.size(); ++i)
      for (size_t j = 0; j < budgets.size(); ++j) {
        rebuild(splits[i], budgets[j]);
        double t = 0;
        if (batched) {
          std::unique_ptr<BatchPlan, void (*)(BatchPlan*)> b(batch_create(ctxs), batch_free);
          batch_sigma(*b, pin.data(), pout.data(), true);  // eager pass, then the graph capture
          batch_sigma(*b, pin.data(), pout.data(), true);  // first replay
          for (int r = 0; r < reps; ++r) t += batch_sigma(*b, pin.data(), pout.data(), true);
        } else {
          Context& c = *ctxs[0];
          run_sigma(c, c.plan, pin[0], pout[0]);  // warm-up
          cuda_check(cudaEventRecord(c.ev0, c.stream), "record");
          for (int r = 0; r < reps; ++r) run_sigma(c, c.plan, pin[0], pout[0]);
          cuda_check(cudaEventRecord(c.ev1, c.stream), "record");
          cuda_check(cudaEventSynchronize(c.ev1), "sync");
          if (mixed_error(c, c.plan)) throw Error(ST_ETIMEOUT, "tensor-core GEMM: a bounded wait ran out");
          float e = 0;
          cuda_check(cudaEventElapsedTime(&e, c.ev0, c.ev1), "elapsed");
          t = e;
        }
        const size_t at = i * budgets.size() + j;
        ms[at] = t / reps;
        if (ms[at] < ms[best]) best = at;
      }
    const TuneChoice choice{splits[best / budgets.size()], budgets[best % budgets.size()]};
    rebuild(choice.split_tps, choice.budget_mb);
    return choice;
  } catch (...) {
    for (size_t i = 0; i < ctxs.size(); ++i) {
      ctxs[i]->split_tps = saved[i].first;
      ctxs[i]->chunk_budget_mb = saved[i].second;
      ctxs[i]->prepared = -1;
    }
    throw;
  }
}

}  // namespace gbdmrg
