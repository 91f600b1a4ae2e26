// extern "C" boundary of the library (declarations and contracts: include/gbdmrg.h).
#include <algorithm>
#include <cmath>
#include <cstring>
#include <exception>
#include <memory>
#include <string>
#include <vector>

#include "../../include/gbdmrg.h"
#include "engine.hpp"
#include "kernels_tc.hpp"
#include "mlp.hpp"

struct gbdmrg_ctx {
  gbdmrg::Context c;
  gbdmrg::SweepStats stats;
};

struct gbdmrg_mlp {
  gbdmrg::Mlp m;
  std::string err;
};

namespace {

template <class F>
gbdmrg_status guard(gbdmrg_ctx* ctx, F&& f) {
  try {
    f();
    if (ctx) ctx->c.last_error.clear();
    return GBDMRG_OK;
  } catch (const gbdmrg::Error& e) {
    if (ctx) ctx->c.last_error = e.what();
    return (gbdmrg_status)e.code;
  } catch (const std::bad_alloc&) {
    if (ctx) ctx->c.last_error = "host allocation failed";
    return GBDMRG_ENOMEM;
  } catch (const std::exception& e) {
    if (ctx) ctx->c.last_error = e.what();
    return GBDMRG_EINVAL;
  } catch (...) {
    if (ctx) ctx->c.last_error = "unknown error";
    return GBDMRG_ECUDA;
  }
}

void check_problem(const gbdmrg_problem* p) {
  using gbdmrg::Error;
  using gbdmrg::ST_EINVAL;
  if (!p || !p->h1 || !p->eri) throw Error(ST_EINVAL, "null problem or integrals");
  const int K = p->K;
  if (K < 1 || K > 128) throw Error(ST_EINVAL, "K must be in [1, 128]");
  if (p->N < 0 || p->N > 2 * K) throw Error(ST_EINVAL, "N must be in [0, 2K]");
  if (((p->N + p->two_sz) & 1) != 0) throw Error(ST_EINVAL, "two_sz must have the parity of N");
  int na = (p->N + p->two_sz) / 2, nb = (p->N - p->two_sz) / 2;
  if (na < 0 || nb < 0 || na > K || nb > K) throw Error(ST_EINVAL, "S_z out of range");
  if (!std::isfinite(p->ecore)) throw Error(ST_EINVAL, "non-finite ecore");
  for (int i = 0; i < K; ++i)
    for (int j = 0; j < K; ++j) {
      double a = p->h1[i * K + j], b = p->h1[j * K + i];
      if (!std::isfinite(a)) throw Error(ST_EINVAL, "non-finite h1");
      if (std::fabs(a - b) > 1e-12 * (1 + std::fabs(a))) throw Error(ST_EINVAL, "h1 not symmetric");
    }
  auto E = [&](int a, int b, int c, int d) { return p->eri[((size_t)(a * K + b) * K + c) * K + d]; };
  for (int a = 0; a < K; ++a)
    for (int b = 0; b < K; ++b)
      for (int c = 0; c < K; ++c)
        for (int d = 0; d < K; ++d) {
          double v = E(a, b, c, d);
          if (!std::isfinite(v)) throw Error(ST_EINVAL, "non-finite eri");
          double tol = 1e-12 * (1 + std::fabs(v));
          if (std::fabs(v - E(b, a, c, d)) > tol || std::fabs(v - E(a, b, d, c)) > tol ||
              std::fabs(v - E(c, d, a, b)) > tol)
            throw Error(ST_EINVAL, "eri not 8-fold symmetric");
        }
}

template <class F>
gbdmrg_status mguard(gbdmrg_mlp* h, F&& f) {
  try {
    f();
    if (h) h->err.clear();
    return GBDMRG_OK;
  } catch (const gbdmrg::Error& e) {
    if (h) h->err = e.what();
    return (gbdmrg_status)e.code;
  } catch (const std::bad_alloc&) {
    if (h) h->err = "host allocation failed";
    return GBDMRG_ENOMEM;
  } catch (const std::exception& e) {
    if (h) h->err = e.what();
    return GBDMRG_EINVAL;
  } catch (...) {
    if (h) h->err = "unknown error";
    return GBDMRG_ECUDA;
  }
}

// device copy of a caller array (host or device) on stream s
template <class T>
const T* to_device(const T* p, size_t n, int32_t on_device, gbdmrg::DArr<T>& tmp, cudaStream_t s) {
  if (on_device) return p;
  tmp.alloc(n, s);
  gbdmrg::cuda_check(cudaMemcpyAsync(tmp.p, p, n * sizeof(T), cudaMemcpyHostToDevice, s), "h2d");
  return tmp.p;
}

double host_norm(const double* dev, size_t n, cudaStream_t s) {
  std::vector<double> h(n);
  gbdmrg::cuda_check(cudaMemcpyAsync(h.data(), dev, n * sizeof(double), cudaMemcpyDeviceToHost, s), "d2h");
  gbdmrg::cuda_check(cudaStreamSynchronize(s), "sync");
  double r = 0;
  for (double v : h) r += v * v;
  return std::sqrt(r);
}

}  // namespace

extern "C" {

gbdmrg_status gbdmrg_create(const gbdmrg_problem* prob, void* stream, gbdmrg_ctx** out) {
  if (!out) return GBDMRG_EINVAL;
  *out = nullptr;
  std::unique_ptr<gbdmrg_ctx> ctx;
  try {
    check_problem(prob);
    ctx.reset(new gbdmrg_ctx());
  } catch (const gbdmrg::Error& e) {
    return (gbdmrg_status)e.code;
  } catch (...) {
    return GBDMRG_ENOMEM;
  }
  gbdmrg_status st = guard(ctx.get(), [&] {
    auto& c = ctx->c;
    c.K = prob->K;
    c.N = prob->N;
    c.two_sz = prob->two_sz;
    c.Na = (prob->N + prob->two_sz) / 2;
    c.Nb = (prob->N - prob->two_sz) / 2;
    c.ecore = prob->ecore;
    const size_t K = prob->K;
    c.h1.assign(prob->h1, prob->h1 + K * K);
    c.eri.assign(prob->eri, prob->eri + K * K * K * K);
    c.stream = (cudaStream_t)stream;
    gbdmrg::ctx_init(c);
  });
  if (st != GBDMRG_OK) return st;
  *out = ctx.release();
  return GBDMRG_OK;
}

void gbdmrg_destroy(gbdmrg_ctx* ctx) { delete ctx; }

const char* gbdmrg_last_error(const gbdmrg_ctx* ctx) { return ctx ? ctx->c.last_error.c_str() : "null context"; }

gbdmrg_status gbdmrg_mpo_build_host(const gbdmrg_problem* prob, int32_t* dims, double* dense) {
  if (!dims) return GBDMRG_EINVAL;
  return guard(nullptr, [&] {
    check_problem(prob);
    gbdmrg::MPO m = gbdmrg::build_mpo(prob->K, prob->h1, prob->eri);
    for (int b = 0; b <= prob->K; ++b) dims[b] = (int32_t)m.bonds[b].size();
    if (dense) {
      if (prob->K > 5) throw gbdmrg::Error(gbdmrg::ST_EINVAL, "dense MPO needs K <= 5");
      std::vector<double> d;
      gbdmrg::mpo_to_dense(m, d);
      std::memcpy(dense, d.data(), d.size() * sizeof(double));
    }
  });
}

gbdmrg_status gbdmrg_mpo_bond_dims(gbdmrg_ctx* ctx, int32_t* dims) {
  if (!ctx || !dims) return GBDMRG_EINVAL;
  return guard(ctx, [&] {
    for (int b = 0; b <= ctx->c.K; ++b) dims[b] = (int32_t)ctx->c.mpo.bonds[b].size();
  });
}

gbdmrg_status gbdmrg_mpo_dense(gbdmrg_ctx* ctx, double* out) {
  if (!ctx || !out) return GBDMRG_EINVAL;
  return guard(ctx, [&] {
    if (ctx->c.K > 5) throw gbdmrg::Error(gbdmrg::ST_EINVAL, "gbdmrg_mpo_dense needs K <= 5");
    std::vector<double> m;
    gbdmrg::mpo_to_dense(ctx->c.mpo, m);
    std::memcpy(out, m.data(), m.size() * sizeof(double));
  });
}

gbdmrg_status gbdmrg_set_mps(gbdmrg_ctx* ctx, int32_t site, int32_t Dl, int32_t Dr, const int32_t* qn_l,
                             const int32_t* qn_r, const double* A) {
  if (!ctx || !qn_l || !qn_r || !A || Dl <= 0 || Dr <= 0) return GBDMRG_EINVAL;
  return guard(ctx, [&] { gbdmrg::set_site_dense(ctx->c, site, Dl, Dr, qn_l, qn_r, A); });
}

gbdmrg_status gbdmrg_get_mps(gbdmrg_ctx* ctx, int32_t site, int32_t* Dl, int32_t* Dr, double* A) {
  if (!ctx || !Dl || !Dr) return GBDMRG_EINVAL;
  return guard(ctx, [&] {
    auto& c = ctx->c;
    if (site < 0 || site >= c.K || !c.site_set[site]) throw gbdmrg::Error(gbdmrg::ST_ESTATE, "site not set");
    *Dl = c.sites[site].L.total;
    *Dr = c.sites[site].R.total;
    if (A) {
      std::vector<double> d;
      gbdmrg::get_site_dense(c, site, d);
      std::memcpy(A, d.data(), d.size() * sizeof(double));
    }
  });
}

gbdmrg_status gbdmrg_get_bond(gbdmrg_ctx* ctx, int32_t bond, int32_t* D, int32_t* qn) {
  if (!ctx || !D) return GBDMRG_EINVAL;
  return guard(ctx, [&] {
    auto& c = ctx->c;
    if (bond < 0 || bond > c.K) throw gbdmrg::Error(gbdmrg::ST_EINVAL, "bond out of range");
    int s = bond < c.K ? bond : c.K - 1;
    if (!c.site_set[s]) throw gbdmrg::Error(gbdmrg::ST_ESTATE, "site not set");
    const gbdmrg::Bond& b = bond < c.K ? c.sites[s].L : c.sites[s].R;
    *D = b.total;
    if (qn)
      for (int i = 0; i < b.nsec(); ++i)
        for (int j = 0; j < b.dim[i]; ++j) {
          qn[2 * (b.off[i] + j)] = b.qa[i];
          qn[2 * (b.off[i] + j) + 1] = b.qb[i];
        }
  });
}

gbdmrg_status gbdmrg_set_precision(gbdmrg_ctx* ctx, int32_t precision) {
  if (!ctx || precision < 0 || precision > 6) return GBDMRG_EINVAL;
  return guard(ctx, [&] {
    ctx->c.precision = precision;
    ctx->c.prepared = -1;
  });
}

gbdmrg_status gbdmrg_set_chunk_budget(gbdmrg_ctx* ctx, int32_t megabytes) {
  if (!ctx || megabytes <= 0) return GBDMRG_EINVAL;
  return guard(ctx, [&] {
    ctx->c.chunk_budget_mb = megabytes;
    ctx->c.prepared = -1;
  });
}

gbdmrg_status gbdmrg_keep_host_plans(gbdmrg_ctx* ctx, int32_t keep) {
  if (!ctx) return GBDMRG_EINVAL;
  return guard(ctx, [&] { ctx->c.keep_host_plans = keep != 0; });
}

struct gbdmrg_batch {
  gbdmrg::BatchPlan* b = nullptr;
  std::string err;
  ~gbdmrg_batch() {
    if (b) gbdmrg::batch_free(b);
  }
};

gbdmrg_status gbdmrg_batch_create(int32_t n, gbdmrg_ctx* const* ctxs, gbdmrg_batch** out) {
  if (!out || n <= 0 || !ctxs) return GBDMRG_EINVAL;
  *out = nullptr;
  for (int i = 0; i < n; ++i)
    if (!ctxs[i]) return GBDMRG_EINVAL;
  try {
    std::vector<gbdmrg::Context*> v;
    for (int i = 0; i < n; ++i) v.push_back(&ctxs[i]->c);
    auto* bt = new gbdmrg_batch();
    try {
      bt->b = gbdmrg::batch_create(v);
    } catch (...) {
      delete bt;
      throw;
    }
    *out = bt;
    return GBDMRG_OK;
  } catch (const gbdmrg::Error& e) {
    ctxs[0]->c.last_error = e.what();
    return (gbdmrg_status)e.code;
  } catch (const std::bad_alloc&) {
    return GBDMRG_ENOMEM;
  } catch (...) {
    return GBDMRG_ECUDA;
  }
}

gbdmrg_status gbdmrg_batch_sigma(gbdmrg_batch* b, const double* const* psi_dev, double* const* sigma_dev,
                                 int32_t use_graph, double* ms, double* flops) {
  if (!b || !b->b || !psi_dev || !sigma_dev) return GBDMRG_EINVAL;
  try {
    float t = gbdmrg::batch_sigma(*b->b, psi_dev, sigma_dev, use_graph != 0);
    if (ms) *ms = t;
    if (flops) *flops = gbdmrg::batch_flops(b->b);
    b->err.clear();
    return GBDMRG_OK;
  } catch (const gbdmrg::Error& e) {
    b->err = e.what();
    return (gbdmrg_status)e.code;
  } catch (...) {
    b->err = "unknown error";
    return GBDMRG_ECUDA;
  }
}

const char* gbdmrg_batch_last_error(const gbdmrg_batch* b) { return b ? b->err.c_str() : "null batch"; }

void gbdmrg_batch_destroy(gbdmrg_batch* b) { delete b; }

gbdmrg_status gbdmrg_set_split(gbdmrg_ctx* ctx, double tiles_per_sm) {
  if (!ctx || !std::isfinite(tiles_per_sm)) return GBDMRG_EINVAL;
  return guard(ctx, [&] { ctx->c.split_tps = tiles_per_sm; });
}

gbdmrg_status gbdmrg_set_tma_budget(gbdmrg_ctx* ctx, int64_t megabytes) {
  if (!ctx || megabytes <= 0) return GBDMRG_EINVAL;
  return guard(ctx, [&] {
    ctx->c.tma_budget_mb = (long)megabytes;
    ctx->c.prepared = -1;
  });
}

gbdmrg_status gbdmrg_set_env_precision(gbdmrg_ctx* ctx, int32_t precision) {
  if (!ctx || (precision != 0 && precision != 2 && precision != 3)) return GBDMRG_EINVAL;
  return guard(ctx, [&] { ctx->c.env_precision = precision; });
}

gbdmrg_status gbdmrg_set_refinement(gbdmrg_ctx* ctx, int32_t precision, int32_t max_iters) {
  if (!ctx || precision < -1 || precision > 6 || max_iters < 1) return GBDMRG_EINVAL;
  return guard(ctx, [&] {
    ctx->c.refine_precision = precision;
    ctx->c.refine_iters = max_iters;
  });
}

gbdmrg_status gbdmrg_plan_stats(gbdmrg_ctx* ctx, double* out) {
  if (!ctx || !out) return GBDMRG_EINVAL;
  return guard(ctx, [&] {
    if (ctx->c.prepared < 0) throw gbdmrg::Error(gbdmrg::ST_ESTATE, "call gbdmrg_prepare first");
    gbdmrg::tma_plan_stats(ctx->c.plan, out);
  });
}

gbdmrg_status gbdmrg_set_stage1_stacked(gbdmrg_ctx* ctx, int32_t stacked) {
  if (!ctx) return GBDMRG_EINVAL;
  return guard(ctx, [&] { ctx->c.stage1_stacked = stacked != 0; });
}

gbdmrg_status gbdmrg_set_tc_combos(gbdmrg_ctx* ctx, int32_t on, int64_t min_terms) {
  if (!ctx || min_terms < 0) return GBDMRG_EINVAL;
  return guard(ctx, [&] {
    ctx->c.tc_combos = on != 0;
    ctx->c.tc_combo_min_terms = (long)min_terms;
  });
}

gbdmrg_status gbdmrg_get_plan_params(gbdmrg_ctx* ctx, double* tiles_per_sm, int32_t* chunk_budget_mb) {
  if (!ctx) return GBDMRG_EINVAL;
  return guard(ctx, [&] {
    if (tiles_per_sm) *tiles_per_sm = ctx->c.split_tps;
    if (chunk_budget_mb) *chunk_budget_mb = ctx->c.chunk_budget_mb;
  });
}

gbdmrg_status gbdmrg_autotune(int32_t n, gbdmrg_ctx* const* ctxs, int32_t reps, const double* splits,
                              int32_t nsplits, const int32_t* budgets_mb, int32_t nbudgets, double* ms,
                              double* best_split, int32_t* best_budget_mb) {
  if (n <= 0 || !ctxs || reps <= 0) return GBDMRG_EINVAL;
  for (int i = 0; i < n; ++i)
    if (!ctxs[i]) return GBDMRG_EINVAL;
  if ((splits && nsplits <= 0) || (budgets_mb && nbudgets <= 0)) return GBDMRG_EINVAL;
  return guard(ctxs[0], [&] {
    std::vector<gbdmrg::Context*> v;
    for (int i = 0; i < n; ++i) v.push_back(&ctxs[i]->c);
    std::vector<double> sp = splits ? std::vector<double>(splits, splits + nsplits)
                                    : std::vector<double>{32, 8, 2, 0.5, 0.125, 0.03125, 0};
    for (double x : sp)
      if (!std::isfinite(x)) throw gbdmrg::Error(gbdmrg::ST_EINVAL, "autotune: non-finite split candidate");
    std::vector<int> bu = budgets_mb ? std::vector<int>(budgets_mb, budgets_mb + nbudgets)
                                     : std::vector<int>{ctxs[0]->c.chunk_budget_mb};
    std::vector<double> t;
    const gbdmrg::TuneChoice best = gbdmrg::autotune_plans(v, sp, bu, reps, t);
    if (ms) std::copy(t.begin(), t.end(), ms);
    if (best_split) *best_split = best.split_tps;
    if (best_budget_mb) *best_budget_mb = best.budget_mb;
  });
}

gbdmrg_status gbdmrg_plan(gbdmrg_ctx* ctx, int32_t k) {
  if (!ctx) return GBDMRG_EINVAL;
  return guard(ctx, [&] {
    auto& c = ctx->c;
    if (k < 0 || k + 1 >= c.K) throw gbdmrg::Error(gbdmrg::ST_EINVAL, "two-site position out of range");
    if (!c.left[k].valid || !c.right[k + 2].valid)
      throw gbdmrg::Error(gbdmrg::ST_ESTATE, "environments of bonds k and k+2 are not built");
    gbdmrg::build_tilde_left(c, c.left[k], k, c.lt, true);
    gbdmrg::build_tilde_right(c, c.right[k + 2], k + 1, c.rt, true);
    gbdmrg::build_sigma_plan(c, c.lt, c.rt, k, c.plan);
    gbdmrg::cuda_check(cudaStreamSynchronize(c.stream), "sync");
    c.prepared = k;
  });
}

gbdmrg_status gbdmrg_prepare(gbdmrg_ctx* ctx, int32_t k) {
  if (!ctx) return GBDMRG_EINVAL;
  return guard(ctx, [&] { gbdmrg::prepare_two_site(ctx->c, k); });
}

gbdmrg_status gbdmrg_psi_layout(gbdmrg_ctx* ctx, int64_t* nblocks, int64_t* nnz, int64_t* blocks) {
  if (!ctx || !nblocks || !nnz) return GBDMRG_EINVAL;
  return guard(ctx, [&] {
    auto& c = ctx->c;
    if (c.prepared < 0) throw gbdmrg::Error(gbdmrg::ST_ESTATE, "call gbdmrg_prepare first");
    const auto& P = c.plan.psi;
    *nblocks = (int64_t)P.blocks.size();
    *nnz = P.nnz;
    if (blocks)
      for (size_t i = 0; i < P.blocks.size(); ++i) {
        const auto& b = P.blocks[i];
        int64_t* r = blocks + 7 * i;
        r[0] = P.L.off[b.rs];
        r[1] = b.rows;
        r[2] = P.b1[i];
        r[3] = P.b2[i];
        r[4] = P.R.off[b.cs];
        r[5] = b.cols;
        r[6] = b.off;
      }
  });
}

gbdmrg_status gbdmrg_sigma(gbdmrg_ctx* ctx, const double* psi, double* sigma, int32_t on_device, double* flops) {
  if (!ctx || !psi || !sigma) return GBDMRG_EINVAL;
  return guard(ctx, [&] {
    auto& c = ctx->c;
    if (c.prepared < 0) throw gbdmrg::Error(gbdmrg::ST_ESTATE, "call gbdmrg_prepare first");
    auto& plan = c.plan;
    const size_t bytes = plan.psi.nnz * sizeof(double);
    if (on_device) {
      gbdmrg::run_sigma(c, plan, psi, sigma);
    } else {
      gbdmrg::cuda_check(cudaMemcpyAsync(plan.in.p, psi, bytes, cudaMemcpyHostToDevice, c.stream), "h2d");
      gbdmrg::run_sigma(c, plan, plan.in.p, plan.out.p);
      gbdmrg::cuda_check(cudaMemcpyAsync(sigma, plan.out.p, bytes, cudaMemcpyDeviceToHost, c.stream), "d2h");
    }
    gbdmrg::cuda_check(cudaStreamSynchronize(c.stream), "sync");
    if (plan.tensor() && gbdmrg::plan_error(c, plan))
      throw gbdmrg::Error(gbdmrg::ST_ETIMEOUT, "tensor-core GEMM: a bounded wait ran out");
    if (flops) *flops = plan.flops;
  });
}

gbdmrg_status gbdmrg_diag(gbdmrg_ctx* ctx, double* diag, int32_t on_device) {
  if (!ctx || !diag) return GBDMRG_EINVAL;
  return guard(ctx, [&] {
    auto& c = ctx->c;
    if (c.prepared < 0) throw gbdmrg::Error(gbdmrg::ST_ESTATE, "call gbdmrg_prepare first");
    const auto& P = c.plan.psi;
    if (on_device) {
      gbdmrg::compute_diag(c, c.lt, c.rt, c.prepared, P, diag);
    } else {
      gbdmrg::DArr<double> d;
      d.alloc(P.nnz, c.stream);
      gbdmrg::compute_diag(c, c.lt, c.rt, c.prepared, P, d.p);
      gbdmrg::cuda_check(cudaMemcpyAsync(diag, d.p, P.nnz * sizeof(double), cudaMemcpyDeviceToHost, c.stream), "d2h");
    }
    gbdmrg::cuda_check(cudaStreamSynchronize(c.stream), "sync");
  });
}

gbdmrg_status gbdmrg_diag_noalloc(gbdmrg_ctx* ctx, double* diag_dev) {
  if (!ctx || !diag_dev) return GBDMRG_EINVAL;
  return guard(ctx, [&] { gbdmrg::compute_diag_noalloc(ctx->c, diag_dev); });
}

gbdmrg_status gbdmrg_sigma_timing(gbdmrg_ctx* ctx, int32_t reps, const double* psi_dev, double* sigma_dev,
                                  double* ms_per_call) {
  if (!ctx || !psi_dev || !sigma_dev || !ms_per_call || reps <= 0) return GBDMRG_EINVAL;
  return guard(ctx, [&] {
    auto& c = ctx->c;
    if (c.prepared < 0) throw gbdmrg::Error(gbdmrg::ST_ESTATE, "call gbdmrg_prepare first");
    cudaEvent_t e0, e1;
    gbdmrg::cuda_check(cudaEventCreate(&e0), "event");
    gbdmrg::cuda_check(cudaEventCreate(&e1), "event");
    gbdmrg::cuda_check(cudaEventRecord(e0, c.stream), "record");
    for (int r = 0; r < reps; ++r) gbdmrg::run_sigma(c, c.plan, psi_dev, sigma_dev);
    gbdmrg::cuda_check(cudaEventRecord(e1, c.stream), "record");
    gbdmrg::cuda_check(cudaEventSynchronize(e1), "sync");
    if (c.plan.tensor() && gbdmrg::plan_error(c, c.plan))
      throw gbdmrg::Error(gbdmrg::ST_ETIMEOUT, "tensor-core GEMM: a bounded wait ran out");
    float ms = 0;
    cudaEventElapsedTime(&ms, e0, e1);
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    *ms_per_call = ms / reps;
  });
}

gbdmrg_status gbdmrg_step(gbdmrg_ctx* ctx, int32_t k, int32_t direction, int32_t M, double dav_tol,
                          int32_t dav_max_iter, const double* psi_in, double* psi_out, int32_t on_device,
                          double* energy, double* discarded, int32_t* iters) {
  if (!ctx || M <= 0 || !(dav_tol > 0) || (direction != 0 && direction != 1)) return GBDMRG_EINVAL;
  return guard(ctx, [&] {
    auto& c = ctx->c;
    if (k < 0 || k + 1 >= c.K) throw gbdmrg::Error(gbdmrg::ST_EINVAL, "two-site position out of range");
    gbdmrg::DavidsonOpts o;
    o.tol = dav_tol;
    o.max_iter = dav_max_iter > 0 ? dav_max_iter : 200;
    gbdmrg::DArr<double> din, dout;
    const double* p0 = nullptr;
    double* p1 = nullptr;
    if (psi_in || psi_out) {
      if (!c.left[k].valid || !c.right[k + 2].valid)
        throw gbdmrg::Error(gbdmrg::ST_ESTATE, "environments of the two-site step are not built");
      gbdmrg::PsiLayout P;
      P.build(c.left[k].bond, c.right[k + 2].bond);
      if (psi_in) {
        if (on_device) p0 = psi_in;
        else {
          din.alloc(P.nnz, c.stream);
          gbdmrg::cuda_check(cudaMemcpyAsync(din.p, psi_in, P.nnz * sizeof(double), cudaMemcpyHostToDevice, c.stream),
                             "h2d");
          p0 = din.p;
        }
      }
      if (psi_out) {
        if (on_device) p1 = psi_out;
        else {
          dout.alloc(P.nnz, c.stream);
          p1 = dout.p;
        }
      }
    }
    int it = 0;
    double dw = 0;
    long nnz = 0;
    double e = gbdmrg::two_site_step(c, k, direction, M, o, false, &it, &dw, p0, p1, &nnz);
    if (psi_out && !on_device)
      gbdmrg::cuda_check(cudaMemcpy(psi_out, dout.p, nnz * sizeof(double), cudaMemcpyDeviceToHost), "d2h");
    if (energy) *energy = e + c.ecore;
    if (discarded) *discarded = dw;
    if (iters) *iters = it;
  });
}

int64_t gbdmrg_kernel_launches(void) { return (int64_t)(gbdmrg::launch_count() + gbdmrg::tc_launch_count()); }

gbdmrg_status gbdmrg_gemm_bf16_selftest(const int64_t* tasks, int32_t ntasks, const int64_t* terms, int32_t nterms,
                                        void* stream) {
  if (!tasks || !terms || ntasks <= 0 || nterms <= 0) return GBDMRG_EINVAL;
  return guard(nullptr, [&] {
    using namespace gbdmrg;
    cudaStream_t st = (cudaStream_t)stream;
    std::vector<TcTask> ta(ntasks);
    std::vector<TcTerm> te(nterms);
    std::vector<TcTile> ti;
    for (int i = 0; i < nterms; ++i) {
      const int64_t* r = terms + 6 * i;
      te[i] = {(const __nv_bfloat16*)r[0], (const __nv_bfloat16*)r[1], 0, 0, (int)r[2], (int)r[3], (int)r[4],
               (int)r[5], 1};
      if ((r[0] | r[1]) & 15 || r[2] % 8 || r[3] % 8 || r[4] <= 0 || r[4] > r[2] || r[4] > r[3])
        throw Error(ST_EINVAL, "bf16 operands must be 16-byte aligned, ld % 8 == 0, 0 < k <= ld");
    }
    for (int i = 0; i < ntasks; ++i) {
      const int64_t* r = tasks + 8 * i;
      ta[i] = {(float*)r[0], nullptr, 0, (int)r[1], 0, (int)r[2], (int)r[3], (int)r[4], 0, (int)r[7], (int)r[5],
               (int)r[6]};
      if (ta[i].t0 < 0 || ta[i].t1 > nterms || ta[i].t0 >= ta[i].t1 || ta[i].m <= 0 || ta[i].n <= 0)
        throw Error(ST_EINVAL, "bad task");
      for (int r0 = 0; r0 < ta[i].m; r0 += TC_TILE_M)
        for (int c0 = 0; c0 < ta[i].n; c0 += TC_TILE_N) ti.push_back({i, r0, c0});
    }
    DArr<TcTask> dta;
    DArr<TcTerm> dte;
    DArr<TcTile> dti;
    DArr<int> derr;
    dta.upload(ta, st);
    dte.upload(te, st);
    dti.upload(ti, st);
    derr.alloc(1, st);
    cuda_check(cudaMemsetAsync(derr.p, 0, sizeof(int), st), "memset");
    cuda_check(launch_gemm_bf16_tc(dti.p, (int)ti.size(), dta.p, dte.p, derr.p, st), "tc gemm launch");
    int herr = 0;
    cuda_check(cudaMemcpyAsync(&herr, derr.p, sizeof(int), cudaMemcpyDeviceToHost, st), "d2h");
    cuda_check(cudaStreamSynchronize(st), "sync");
    if (herr) throw Error(ST_ETIMEOUT, "tensor-core GEMM: a bounded wait ran out");
  });
}

gbdmrg_status gbdmrg_counters(gbdmrg_ctx* ctx, double* sigma_flops, double* sigma_seconds, int64_t* sigma_calls,
                              double* other_flops) {
  if (!ctx) return GBDMRG_EINVAL;
  return guard(ctx, [&] {
    auto& c = ctx->c;
    if (sigma_flops) *sigma_flops = c.sigma_flops_total;
    if (sigma_seconds) *sigma_seconds = c.sigma_time_total;
    if (sigma_calls) *sigma_calls = c.sigma_calls;
    if (other_flops) *other_flops = c.other_flops_total;
  });
}

gbdmrg_status gbdmrg_phase_times(gbdmrg_ctx* ctx, double* seconds) {
  if (!ctx || !seconds) return GBDMRG_EINVAL;
  return guard(ctx, [&] {
    for (int i = 0; i < 8; ++i) seconds[i] = ctx->c.phase_s[i];
  });
}

gbdmrg_status gbdmrg_phase_flops(gbdmrg_ctx* ctx, double* flops) {
  if (!ctx || !flops) return GBDMRG_EINVAL;
  return guard(ctx, [&] {
    for (int i = 0; i < 8; ++i) flops[i] = ctx->c.phase_flops[i];
  });
}

gbdmrg_status gbdmrg_sigma_flops_host(const gbdmrg_problem* prob, int32_t k, int32_t Dl, const int32_t* qn_l,
                                      int32_t Dr, const int32_t* qn_r, double* flops) {
  if (!flops || !qn_l || !qn_r || Dl <= 0 || Dr <= 0) return GBDMRG_EINVAL;
  return guard(nullptr, [&] {
    check_problem(prob);
    if (k < 0 || k + 1 >= prob->K) throw gbdmrg::Error(gbdmrg::ST_EINVAL, "two-site position out of range");
    gbdmrg::MPO m = gbdmrg::build_mpo(prob->K, prob->h1, prob->eri);
    auto bond = [](int D, const int32_t* q) {
      gbdmrg::Bond b;
      int i = 0;
      while (i < D) {
        int j = i;
        while (j < D && q[2 * j] == q[2 * i] && q[2 * j + 1] == q[2 * i + 1]) ++j;
        b.add(q[2 * i], q[2 * i + 1], j - i);
        i = j;
      }
      return b;
    };
    *flops = gbdmrg::count_sigma_flops(m, k, bond(Dl, qn_l), bond(Dr, qn_r));
  });
}

gbdmrg_status gbdmrg_run(gbdmrg_ctx* ctx, const gbdmrg_schedule* s, double* energies, double* discarded) {
  if (!ctx || !s || !energies || s->nsweeps <= 0 || !s->M || !s->dav_tol) return GBDMRG_EINVAL;
  return guard(ctx, [&] {
    for (int i = 0; i < s->nsweeps; ++i) {
      if (s->M[i] <= 0) throw gbdmrg::Error(gbdmrg::ST_EINVAL, "M must be positive");
      if (!(s->dav_tol[i] > 0)) throw gbdmrg::Error(gbdmrg::ST_EINVAL, "dav_tol must be positive");
    }
    if (s->precision < 0 || s->precision > 6) throw gbdmrg::Error(gbdmrg::ST_EINVAL, "precision must be 0 to 6");
    ctx->c.precision = s->precision;
    ctx->stats = gbdmrg::SweepStats();
    gbdmrg::run_sweeps(ctx->c, s->nsweeps, s->M, s->dav_tol, s->dav_max_iter > 0 ? s->dav_max_iter : 200,
                       ctx->stats);
    for (int i = 0; i < s->nsweeps; ++i) {
      energies[i] = ctx->stats.energy[i];
      if (discarded) discarded[i] = ctx->stats.discarded[i];
    }
  });
}

gbdmrg_status gbdmrg_run_stats(gbdmrg_ctx* ctx, double* seconds, double* sigma_flops, double* sigma_seconds,
                               int32_t* iters) {
  if (!ctx) return GBDMRG_EINVAL;
  return guard(ctx, [&] {
    const auto& st = ctx->stats;
    for (size_t i = 0; i < st.energy.size(); ++i) {
      if (seconds) seconds[i] = st.seconds[i];
      if (sigma_flops) sigma_flops[i] = st.sigma_flops[i];
      if (sigma_seconds) sigma_seconds[i] = st.sigma_seconds[i];
      if (iters) iters[i] = st.davidson_iters[i];
    }
  });
}

// ---------------------------------------------------------------- learned preconditioner

int64_t gbdmrg_mlp_nparams(void) { return gbdmrg::MLP_NPARAMS; }

gbdmrg_status gbdmrg_mlp_create(uint64_t seed, void* stream, gbdmrg_mlp** out) {
  if (!out) return GBDMRG_EINVAL;
  *out = nullptr;
  auto* h = new (std::nothrow) gbdmrg_mlp();
  if (!h) return GBDMRG_ENOMEM;
  gbdmrg_status st = mguard(h, [&] { gbdmrg::mlp_init(h->m, seed, (cudaStream_t)stream); });
  if (st != GBDMRG_OK) {
    delete h;
    return st;
  }
  *out = h;
  return GBDMRG_OK;
}

void gbdmrg_mlp_destroy(gbdmrg_mlp* mlp) { delete mlp; }

const char* gbdmrg_mlp_last_error(const gbdmrg_mlp* mlp) { return mlp ? mlp->err.c_str() : "null network"; }

gbdmrg_status gbdmrg_mlp_set_params(gbdmrg_mlp* mlp, const float* params) {
  if (!mlp || !params) return GBDMRG_EINVAL;
  return mguard(mlp, [&] {
    for (long i = 0; i < gbdmrg::MLP_NPARAMS; ++i)
      if (!std::isfinite(params[i])) throw gbdmrg::Error(gbdmrg::ST_EINVAL, "non-finite parameter");
    gbdmrg::mlp_set_params(mlp->m, params);
  });
}

gbdmrg_status gbdmrg_mlp_get_params(gbdmrg_mlp* mlp, float* params) {
  if (!mlp || !params) return GBDMRG_EINVAL;
  return mguard(mlp, [&] { gbdmrg::mlp_get_params(mlp->m, params); });
}

gbdmrg_status gbdmrg_mlp_forward(gbdmrg_mlp* mlp, const float* features, int64_t n, float* g, int32_t inference,
                                 int32_t on_device) {
  if (!mlp || n < 0 || (n > 0 && (!features || !g))) return GBDMRG_EINVAL;
  return mguard(mlp, [&] {
    if (n == 0) return;
    cudaStream_t s = mlp->m.stream;
    gbdmrg::DArr<float> tf, tg;
    const float* F = to_device(features, (size_t)n * gbdmrg::MLP_F, on_device, tf, s);
    float* G = g;
    if (!on_device) {
      tg.alloc(n, s);
      G = tg.p;
    }
    gbdmrg::mlp_forward(mlp->m, F, n, G, inference != 0);
    if (!on_device) gbdmrg::cuda_check(cudaMemcpyAsync(g, G, n * sizeof(float), cudaMemcpyDeviceToHost, s), "d2h");
    gbdmrg::cuda_check(cudaStreamSynchronize(s), "sync");
  });
}

gbdmrg_status gbdmrg_mlp_loss_grad(gbdmrg_mlp* mlp, const float* features, const float* P, const float* T, int64_t n,
                                   int32_t on_device, float* grad, double* loss) {
  if (!mlp || n <= 0 || !features || !P || !T) return GBDMRG_EINVAL;
  return mguard(mlp, [&] {
    cudaStream_t s = mlp->m.stream;
    gbdmrg::DArr<float> tf, tp, tt;
    const float* F = to_device(features, (size_t)n * gbdmrg::MLP_F, on_device, tf, s);
    const float* Pd = to_device(P, n, on_device, tp, s);
    const float* Td = to_device(T, n, on_device, tt, s);
    double L = gbdmrg::mlp_loss_grad(mlp->m, F, Pd, Td, n);
    if (loss) *loss = L;
    if (grad) {
      gbdmrg::cuda_check(
          cudaMemcpyAsync(grad, mlp->m.grad.p, gbdmrg::MLP_NPARAMS * sizeof(float), cudaMemcpyDeviceToHost, s), "d2h");
      gbdmrg::cuda_check(cudaStreamSynchronize(s), "sync");
    }
  });
}

gbdmrg_status gbdmrg_mlp_train(gbdmrg_mlp* mlp, const float* features, const float* P, const float* T, int64_t n,
                               int32_t on_device, int32_t epochs, int32_t batch, float lr, uint64_t seed,
                               double* loss_first, double* loss_last) {
  if (!mlp || n <= 0 || !features || !P || !T || epochs <= 0 || batch <= 0 || !(lr > 0)) return GBDMRG_EINVAL;
  return mguard(mlp, [&] {
    cudaStream_t s = mlp->m.stream;
    gbdmrg::DArr<float> tf, tp, tt;
    const float* F = to_device(features, (size_t)n * gbdmrg::MLP_F, on_device, tf, s);
    const float* Pd = to_device(P, n, on_device, tp, s);
    const float* Td = to_device(T, n, on_device, tt, s);
    gbdmrg::mlp_train(mlp->m, F, Pd, Td, n, epochs, batch, lr, seed, loss_first, loss_last);
  });
}

gbdmrg_status gbdmrg_set_preconditioner(gbdmrg_ctx* ctx, gbdmrg_mlp* mlp) {
  if (!ctx) return GBDMRG_EINVAL;
  return guard(ctx, [&] { ctx->c.mlp = mlp ? &mlp->m : nullptr; });
}

gbdmrg_status gbdmrg_precondition(gbdmrg_ctx* ctx, const double* r, double theta, double* t, int32_t on_device) {
  if (!ctx || !r || !t || !std::isfinite(theta)) return GBDMRG_EINVAL;
  return guard(ctx, [&] {
    auto& c = ctx->c;
    if (c.prepared < 0) throw gbdmrg::Error(gbdmrg::ST_ESTATE, "call gbdmrg_prepare first");
    const auto& P = c.plan.psi;
    const size_t n = P.nnz;
    gbdmrg::DArr<double> tr, tt, d;
    const double* rd = to_device(r, n, on_device, tr, c.stream);
    double* td = t;
    if (!on_device) {
      tt.alloc(n, c.stream);
      td = tt.p;
    }
    d.alloc(n, c.stream);
    gbdmrg::compute_diag(c, c.lt, c.rt, c.prepared, P, d.p);
    const double rn = host_norm(rd, n, c.stream);
    if (!(rn > 0) || !std::isfinite(rn)) throw gbdmrg::Error(gbdmrg::ST_EINVAL, "zero or non-finite residual");
    if (c.mlp) {
      gbdmrg::MlpScratch sc;
      gbdmrg::mlp_scratch_build(sc, c.mlp, P, c.stream);
      gbdmrg::mlp_scratch_set_diag(sc, d.p, c.stream);
      if (!gbdmrg::mlp_precondition(*c.mlp, sc, rd, d.p, theta, rn, td, c.stream))
        throw gbdmrg::Error(gbdmrg::ST_ENOCONV, "learned preconditioner produced a non-finite value");
    } else {
      gbdmrg::launch_precond((long)n, rd, d.p, theta, 1e-8, td, c.stream);
    }
    if (!on_device)
      gbdmrg::cuda_check(cudaMemcpyAsync(t, td, n * sizeof(double), cudaMemcpyDeviceToHost, c.stream), "d2h");
    gbdmrg::cuda_check(cudaStreamSynchronize(c.stream), "sync");
  });
}

gbdmrg_status gbdmrg_make_pairs(gbdmrg_ctx* ctx, const double* x, const double* r, double theta, const double* psi,
                                int64_t ns, uint64_t seed, int32_t on_device, float* features, float* P, float* T,
                                int64_t* idx, int64_t* written) {
  if (!ctx || !x || !r || !psi || ns < 0 || !features || !P || !T || !std::isfinite(theta)) return GBDMRG_EINVAL;
  return guard(ctx, [&] {
    auto& c = ctx->c;
    if (c.prepared < 0) throw gbdmrg::Error(gbdmrg::ST_ESTATE, "call gbdmrg_prepare first");
    const auto& Pl = c.plan.psi;
    const size_t n = Pl.nnz;
    gbdmrg::DArr<double> tx, tr, tp, d;
    const double* xd = to_device(x, n, on_device, tx, c.stream);
    const double* rd = to_device(r, n, on_device, tr, c.stream);
    const double* pd = to_device(psi, n, on_device, tp, c.stream);
    d.alloc(n, c.stream);
    gbdmrg::compute_diag(c, c.lt, c.rt, c.prepared, Pl, d.p);
    const double rn = host_norm(rd, n, c.stream);
    if (!(rn > 0) || !std::isfinite(rn)) throw gbdmrg::Error(gbdmrg::ST_EINVAL, "zero or non-finite residual");
    gbdmrg::MlpScratch sc;
    gbdmrg::mlp_scratch_build(sc, nullptr, Pl, c.stream);
    gbdmrg::mlp_scratch_set_diag(sc, d.p, c.stream);
    gbdmrg::DArr<float> fF, fP, fT;
    gbdmrg::DArr<long> fi;
    float *oF = features, *oP = P, *oT = T;
    long* oi = (long*)idx;
    if (!on_device) {
      fF.alloc((size_t)ns * gbdmrg::MLP_F, c.stream);
      fP.alloc(ns, c.stream);
      fT.alloc(ns, c.stream);
      fi.alloc(ns, c.stream);
      oF = fF.p;
      oP = fP.p;
      oT = fT.p;
      oi = fi.p;
    }
    long w = gbdmrg::mlp_make_pairs(sc, xd, rd, d.p, theta, rn, pd, ns, seed, oF, oP, oT, oi, 0.0, c.stream);
    if (!on_device && w > 0) {
      gbdmrg::cuda_check(cudaMemcpyAsync(features, oF, w * gbdmrg::MLP_F * sizeof(float), cudaMemcpyDeviceToHost,
                                         c.stream), "d2h");
      gbdmrg::cuda_check(cudaMemcpyAsync(P, oP, w * sizeof(float), cudaMemcpyDeviceToHost, c.stream), "d2h");
      gbdmrg::cuda_check(cudaMemcpyAsync(T, oT, w * sizeof(float), cudaMemcpyDeviceToHost, c.stream), "d2h");
      if (idx) gbdmrg::cuda_check(cudaMemcpyAsync(idx, oi, w * sizeof(long), cudaMemcpyDeviceToHost, c.stream), "d2h");
    }
    gbdmrg::cuda_check(cudaStreamSynchronize(c.stream), "sync");
    if (written) *written = w;
  });
}

gbdmrg_status gbdmrg_set_harvest(gbdmrg_ctx* ctx, int64_t capacity, int32_t per_iteration, uint64_t seed) {
  if (!ctx || capacity < 0 || per_iteration < 0) return GBDMRG_EINVAL;
  return guard(ctx, [&] {
    auto& H = ctx->c.harvest;
    H.cap = capacity;
    H.count = 0;
    H.per_iter = per_iteration;
    H.seed = seed;
    H.solves = 0;
    H.F.alloc((size_t)capacity * gbdmrg::MLP_F, ctx->c.stream);
    H.P.alloc(capacity, ctx->c.stream);
    H.T.alloc(capacity, ctx->c.stream);
    gbdmrg::cuda_check(cudaStreamSynchronize(ctx->c.stream), "sync");
  });
}

gbdmrg_status gbdmrg_get_harvest(gbdmrg_ctx* ctx, float* features, float* P, float* T, int64_t* n) {
  if (!ctx || !n) return GBDMRG_EINVAL;
  return guard(ctx, [&] {
    auto& H = ctx->c.harvest;
    *n = H.count;
    if (H.count == 0) return;
    cudaStream_t s = ctx->c.stream;
    if (features)
      gbdmrg::cuda_check(cudaMemcpyAsync(features, H.F.p, H.count * gbdmrg::MLP_F * sizeof(float),
                                         cudaMemcpyDeviceToHost, s), "d2h");
    if (P) gbdmrg::cuda_check(cudaMemcpyAsync(P, H.P.p, H.count * sizeof(float), cudaMemcpyDeviceToHost, s), "d2h");
    if (T) gbdmrg::cuda_check(cudaMemcpyAsync(T, H.T.p, H.count * sizeof(float), cudaMemcpyDeviceToHost, s), "d2h");
    gbdmrg::cuda_check(cudaStreamSynchronize(s), "sync");
  });
}

gbdmrg_status gbdmrg_precond_counters(gbdmrg_ctx* ctx, int64_t* learned, int64_t* fallbacks) {
  if (!ctx) return GBDMRG_EINVAL;
  return guard(ctx, [&] {
    if (learned) *learned = ctx->c.mlp_applied;
    if (fallbacks) *fallbacks = ctx->c.mlp_fallbacks;
  });
}

// ---------------------------------------------------------------- checkpoint

gbdmrg_status gbdmrg_save(gbdmrg_ctx* ctx, const char* path) {
  if (!ctx || !path) return GBDMRG_EINVAL;
  return guard(ctx, [&] { gbdmrg::save_mps(ctx->c, path); });
}

gbdmrg_status gbdmrg_load(gbdmrg_ctx* ctx, const char* path) {
  if (!ctx || !path) return GBDMRG_EINVAL;
  return guard(ctx, [&] { gbdmrg::load_mps(ctx->c, path); });
}

gbdmrg_status gbdmrg_expectation(gbdmrg_ctx* ctx, double* value) {
  if (!ctx || !value) return GBDMRG_EINVAL;
  return guard(ctx, [&] { *value = gbdmrg::expectation(ctx->c); });
}

}  // extern "C"
