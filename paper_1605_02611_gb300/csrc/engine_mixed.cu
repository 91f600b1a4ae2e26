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
#include <cmath>
#include <map>

#include "engine.hpp"
#include "kernels_tc.hpp"

namespace gbdmrg {

namespace {

inline int pad8(int x) { return (x + 7) & ~7; }

struct ConvJob {
  const double* src;
  __nv_bfloat16* dst;
  long slice_stride;
  int rows, cols, lds, ldd, nsl;
  double scale;
};

__global__ void conv_kernel(const ConvJob* __restrict__ jobs) {
  const ConvJob jb = jobs[blockIdx.y];
  const long n = (long)jb.rows * jb.ldd;
  for (long e = (long)blockIdx.x * blockDim.x + threadIdx.x; e < n; e += (long)gridDim.x * blockDim.x) {
    const int i = (int)(e / jb.ldd), j = (int)(e % jb.ldd);
    double v = j < jb.cols ? jb.scale * jb.src[(long)i * jb.lds + j] : 0.0;
    __nv_bfloat16* d = jb.dst + (long)i * jb.ldd + j;
    for (int s = 0; s < jb.nsl; ++s) {
      const __nv_bfloat16 h = __double2bfloat16(v);
      d[s * jb.slice_stride] = h;
      v -= (double)__bfloat162float(h);
    }
  }
}

__global__ void f32_to_f64_kernel(const float* __restrict__ a, double* __restrict__ b, long n) {
  for (long e = (long)blockIdx.x * blockDim.x + threadIdx.x; e < n; e += (long)gridDim.x * blockDim.x) b[e] = a[e];
}

void launch_conv(const DArr<ConvJob>& jobs, int njobs, long maxel, cudaStream_t s) {
  for (int o0 = 0; o0 < njobs; o0 += 65535) {
    int no = std::min(65535, njobs - o0);
    long g = std::min<long>(std::max<long>(1, (maxel + 255) / 256), 64);
    conv_kernel<<<dim3((unsigned)g, no), 256, 0, s>>>(jobs.p + o0);
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
};

struct MixedPlan {
  int nsl = 1;
  DArr<__nv_bfloat16> psi_b, X_b, mirror;
  DArr<float> sig_f;
  DArr<ConvJob> psi_jobs;
  int n_psi_jobs = 0;
  long psi_maxel = 0;
  std::vector<TcPlan> stage1, stage2;
  DArr<int> err;
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
  std::map<std::pair<const double*, double>, MirrorRef> mref;
  long mtot = 0;
  std::vector<ConvJob> conv;
  std::vector<std::array<MirrorRef, 16>> lm(mid.size()), rm(mid.size());
  auto mirror_of = [&](const TRef& r, bool left) -> MirrorRef {
    const double a = std::fabs(r.coef);
    const double scale = a == 1.0 ? 1.0 : r.coef;
    auto key = std::make_pair(r.p, scale);
    auto it = mref.find(key);
    MirrorRef m;
    if (it == mref.end()) {
      const OpLayout& L = left ? Lenv.cls[r.cls] : Renv.cls[r.cls];
      const long sz = left ? lsz[r.cls] : rsz[r.cls];
      m.off = mtot;
      m.stride = sz;
      m.boff = left ? &loff[r.cls] : &roff[r.cls];
      mtot += sz * nsl;
      mref[key] = m;
      for (size_t b = 0; b < L.blocks.size(); ++b) {
        const Block& B = L.blocks[b];
        conv.push_back({r.p + B.off, nullptr /*patched*/, sz, B.rows, B.cols, B.cols, pad8(B.cols), nsl, scale});
        conv.back().dst = (__nv_bfloat16*)(intptr_t)(m.off + (*m.boff)[b]);  // offset, patched below
      }
    } else m = it->second;
    m.neg = (a == 1.0 && r.coef < 0);
    return m;
  };
  for (size_t beta = 0; beta < mid.size(); ++beta)
    for (int nn = 0; nn < 16; ++nn) {
      if (lt.ref[beta][nn].p) lm[beta][nn] = mirror_of(lt.ref[beta][nn], true);
      if (rt.ref[beta][nn].p) rm[beta][nn] = mirror_of(rt.ref[beta][nn], false);
    }
  mx->mirror.alloc(std::max<long>(mtot, 8), c.stream);
  for (auto& j : conv) j.dst = mx->mirror.p + (intptr_t)j.dst;
  {
    long maxel = 0;
    for (auto& j : conv) maxel = std::max<long>(maxel, (long)j.rows * j.ldd);
    DArr<ConvJob> dj;
    dj.upload(conv, c.stream);
    if (!conv.empty()) launch_conv(dj, (int)conv.size(), maxel, c.stream);
    cuda_check(cudaStreamSynchronize(c.stream), "sync");
  }
  // ---- psi mirror (padded) and its conversion jobs from plan.in
  std::vector<long> poff(P.blocks.size());
  long ptot = 0;
  for (size_t b = 0; b < P.blocks.size(); ++b) {
    poff[b] = ptot;
    ptot += (long)P.blocks[b].rows * pad8(P.blocks[b].cols);
  }
  mx->psi_b.alloc(std::max<long>(ptot * nsl, 8), c.stream);
  {
    std::vector<ConvJob> pj;
    for (size_t b = 0; b < P.blocks.size(); ++b) {
      const Block& B = P.blocks[b];
      pj.push_back({plan.in.p + B.off, mx->psi_b.p + poff[b], ptot, B.rows, B.cols, B.cols, pad8(B.cols), nsl, 1.0});
      mx->psi_maxel = std::max<long>(mx->psi_maxel, (long)B.rows * pad8(B.cols));
    }
    mx->psi_jobs.upload(pj, c.stream);
    mx->n_psi_jobs = (int)pj.size();
  }
  mx->sig_f.alloc(std::max<long>(P.nnz, 1), c.stream);
  mx->err.alloc(1, c.stream);
  cuda_check(cudaMemsetAsync(mx->err.p, 0, sizeof(int), c.stream), "memset");
  // ---- X^T sizes per beta (padded), chunking
  std::vector<size_t> xsz(mid.size(), 0);
  for (size_t beta = 0; beta < mid.size(); ++beta)
    for (int ql = 0; ql < nL; ++ql)
      for (int n1 = 0; n1 < 4; ++n1)
        for (int n2 = 0; n2 < 4; ++n2) {
          int qr = Rb.find(Lb.qa[ql] + LQA[n1] + LQA[n2] + mid[beta].dna,
                           Lb.qb[ql] + LQB[n1] + LQB[n2] + mid[beta].dnb);
          if (qr >= 0) xsz[beta] += (size_t)Rb.dim[qr] * pad8(Lb.dim[ql]);
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
  for (auto ch : chunks) {
    TcBuilder g1, g2;
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
            const int m = Rb.dim[qr], n = Lb.dim[qlp], ldx = pad8(n);
            TcTask t{};
            t.Cb = mx->X_b.p + xoff;
            t.slice_stride = xstride;
            t.ldcb = ldx;
            t.m = m;
            t.n = n;
            t.nslices = nsl;
            g1.begin(t);
            for (int n2p = 0; n2p < 4; ++n2p) {
              const TRef& r = rt.ref[beta][n2 * 4 + n2p];
              if (!r.p) continue;
              int pb = P.blk(qlp, n1p, n2p);
              if (pb < 0) continue;
              int qrp = P.blocks[pb].cs;
              const OpLayout& Lay = Renv.cls[r.cls];
              int bl = Lay.blk_of_col[qrp];
              if (bl < 0 || Lay.blocks[bl].rs != qr) continue;
              const MirrorRef& mr = rm[beta][n2 * 4 + n2p];
              const int kk = Rb.dim[qrp], ld = pad8(kk);
              g1.term(mir + mr.off + (*mr.boff)[bl], mr.stride, ld, mx->psi_b.p + poff[pb], ptot, ld, kk, mr.neg,
                      nsl);
            }
            if (g1.end()) {
              xp[(qlp * 4 + n1p) * 4 + n2] = (long)xoff;
              xoff += (size_t)m * ldx;
            }
          }
    }
    for (size_t pb = 0; pb < P.blocks.size(); ++pb) {
      const Block& ob = P.blocks[pb];
      int ql = ob.rs, n1 = P.b1[pb], n2 = P.b2[pb];
      TcTask t{};
      t.C = mx->sig_f.p + ob.off;
      t.ldc = ob.cols;
      t.m = ob.rows;
      t.n = ob.cols;
      t.beta = 1;
      g2.begin(t);
      for (size_t beta = ch.first; beta < ch.second; ++beta) {
        const auto& xp = xpos[beta - ch.first];
        for (int n1p = 0; n1p < 4; ++n1p) {
          const TRef& r = lt.ref[beta][n1 * 4 + n1p];
          if (!r.p) continue;
          const OpLayout& Lay = Lenv.cls[r.cls];
          int qlp = Lb.find(Lb.qa[ql] - Lay.da, Lb.qb[ql] - Lay.db);
          if (qlp < 0) continue;
          int bl = Lay.blk_of_col[qlp];
          if (bl < 0 || Lay.blocks[bl].rs != ql) continue;
          long xo = xp[(qlp * 4 + n1p) * 4 + n2];
          if (xo < 0) continue;
          const MirrorRef& mr = lm[beta][n1 * 4 + n1p];
          const int kk = Lb.dim[qlp], ld = pad8(kk);
          g2.term(mir + mr.off + (*mr.boff)[bl], mr.stride, ld, mx->X_b.p + xo, xstride, ld, kk, mr.neg, nsl);
        }
      }
      g2.end();
    }
    mx->stage1.emplace_back();
    mx->stage1.back().tiles.upload(g1.tiles, c.stream);
    mx->stage1.back().tasks.upload(g1.tasks, c.stream);
    mx->stage1.back().terms.upload(g1.terms, c.stream);
    mx->stage1.back().ntiles = (int)g1.tiles.size();
    mx->stage2.emplace_back();
    mx->stage2.back().tiles.upload(g2.tiles, c.stream);
    mx->stage2.back().tasks.upload(g2.tasks, c.stream);
    mx->stage2.back().terms.upload(g2.terms, c.stream);
    mx->stage2.back().ntiles = (int)g2.tiles.size();
    cuda_check(cudaStreamSynchronize(c.stream), "sync");
  }
  plan.flops = count_sigma_flops(c.mpo, k, Lb, Rb);
}

void run_mixed_sigma(Context& c, SigmaPlan& plan, const double* x, double* y) {
  MixedPlan& mx = *plan.mx;
  const size_t n = plan.psi.nnz;
  if (x != plan.in.p) cuda_check(cudaMemcpyAsync(plan.in.p, x, n * sizeof(double), cudaMemcpyDeviceToDevice, c.stream), "d2d");
  if (mx.n_psi_jobs) launch_conv(mx.psi_jobs, mx.n_psi_jobs, mx.psi_maxel, c.stream);
  cuda_check(cudaMemsetAsync(mx.sig_f.p, 0, n * sizeof(float), c.stream), "memset");
  for (size_t i = 0; i < mx.stage1.size(); ++i) {
    auto& s1 = mx.stage1[i];
    auto& s2 = mx.stage2[i];
    cuda_check(launch_gemm_bf16_tc(s1.tiles.p, s1.ntiles, s1.tasks.p, s1.terms.p, mx.err.p, c.stream), "tc stage 1");
    cuda_check(launch_gemm_bf16_tc(s2.tiles.p, s2.ntiles, s2.tasks.p, s2.terms.p, mx.err.p, c.stream), "tc stage 2");
  }
  long g = std::min<long>(std::max<long>(1, ((long)n + 255) / 256), 152 * 16);
  f32_to_f64_kernel<<<(unsigned)g, 256, 0, c.stream>>>(mx.sig_f.p, y, (long)n);
  cuda_check(cudaGetLastError(), "f32->f64");
}

int mixed_error(Context& c, SigmaPlan& plan) {
  int h = 0;
  cuda_check(cudaMemcpyAsync(&h, plan.mx->err.p, sizeof(int), cudaMemcpyDeviceToHost, c.stream), "d2h");
  cuda_check(cudaStreamSynchronize(c.stream), "sync");
  return h;
}

}  // namespace gbdmrg
