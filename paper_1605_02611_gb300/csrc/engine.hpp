// Two-site DMRG engine: quantum-number block layouts, renormalised operators
// (environments), the sigma vector H_eff.psi, Davidson, decimation, sweep.
#pragma once
#include <cuda_runtime.h>
#include <cusolverDn.h>

#include <array>
#include <cstdint>
#include <memory>
#include <stdexcept>
#include <string>
#include <vector>

#include "kernels.hpp"
#include "mpo.hpp"

namespace gbdmrg {

struct Error : std::runtime_error {
  int code;
  Error(int c, const std::string& m) : std::runtime_error(m), code(c) {}
};
enum : int { ST_OK = 0, ST_EINVAL = 1, ST_ENOMEM = 2, ST_ECUDA = 3, ST_ENOCONV = 4, ST_ETIMEOUT = 5,
             ST_EIO = 6, ST_ESMALL = 7, ST_ESTATE = 8 };

void cuda_check(cudaError_t e, const char* what);

// local basis n = n_alpha + 2 n_beta
constexpr int LQA[4] = {0, 1, 0, 1};
constexpr int LQB[4] = {0, 0, 1, 1};

// Sectors of one bond, sorted by (n_alpha, n_beta); labels are particle
// counts of the block left of the bond.
struct Bond {
  std::vector<int> qa, qb, dim, off;
  int total = 0;
  int nsec() const { return (int)dim.size(); }
  int find(int a, int b) const;
  void add(int a, int b, int d);   // append (must keep sorted order)
};

struct Block {
  int rs, cs, rows, cols;
  long off;
};

// Block-sparse operator with quantum-number change (da, db): block (row
// sector, col sector) exists when q_row = q_col + (da, db) and both exist.
struct OpLayout {
  int da = 0, db = 0;
  std::vector<Block> blocks;
  std::vector<int> blk_of_col;
  long nnz = 0;
};
OpLayout make_op_layout(const Bond& b, int da, int db);

// stream-ordered device allocation
void* dev_alloc(size_t bytes, cudaStream_t s);
void dev_free(void* p, cudaStream_t s);

template <class T>
struct DArr {
  T* p = nullptr;
  size_t n = 0;
  cudaStream_t s = nullptr;
  DArr() = default;
  DArr(const DArr&) = delete;
  DArr& operator=(const DArr&) = delete;
  DArr(DArr&& o) noexcept { *this = std::move(o); }
  DArr& operator=(DArr&& o) noexcept {
    if (this != &o) { release(); p = o.p; n = o.n; s = o.s; o.p = nullptr; o.n = 0; }
    return *this;
  }
  ~DArr() { release(); }
  void release() { if (p) dev_free(p, s); p = nullptr; n = 0; }
  void alloc(size_t cnt, cudaStream_t st) {
    release(); s = st; n = cnt;
    if (cnt) p = (T*)dev_alloc(cnt * sizeof(T), st);
  }
  void upload(const std::vector<T>& h, cudaStream_t st) {
    alloc(h.size(), st);
    if (n) cuda_check(cudaMemcpyAsync(p, h.data(), n * sizeof(T), cudaMemcpyHostToDevice, st), "upload");
  }
};

// Renormalised operators of every MPO state at one bond (Eq. renormop).
struct Env {
  Bond bond;
  std::vector<OpLayout> cls;
  std::vector<DArr<double>> data;    // per class [nslot * nnz]
  std::vector<int> nslot;
  std::vector<int> st_cls, st_slot;  // per MPO state at this bond
  bool valid = false;
  double* op(int st) { return data[st_cls[st]].p + (size_t)st_slot[st] * cls[st_cls[st]].nnz; }
  const OpLayout& lay(int st) const { return cls[st_cls[st]]; }
  size_t bytes() const;
};

// MPS site tensor A^{n}_{l r}: blocks (ql, n, qr = ql + q(n)), row-major ql x qr.
struct SiteT {
  Bond L, R;
  std::vector<Block> blocks;
  std::vector<int> bn;
  std::vector<int> lookup;  // [ql*4 + n]
  long nnz = 0;
  DArr<double> d;
  void layout(const Bond& l, const Bond& r);
  int blk(int ql, int n) const { return lookup[ql * 4 + n]; }
};

// Two-site tensor psi[l, n1, n2, r] with ql + q(n1) + q(n2) + shift = qr.
struct PsiLayout {
  Bond L, R;
  int da = 0, db = 0;
  std::vector<Block> blocks;
  std::vector<int> b1, b2;
  std::vector<int> lookup;  // [(ql*4 + n1)*4 + n2]
  long nnz = 0;
  void build(const Bond& l, const Bond& r, int sa = 0, int sb = 0);
  int blk(int ql, int n1, int n2) const { return lookup[(ql * 4 + n1) * 4 + n2]; }
};

// W-contracted operators of one side of a two-site problem:
//   left : Lt[beta][n n'] = sum_alpha W[k]_{alpha beta}[n, n'] L_k[alpha]
//   right: Rt[beta][n n'] = sum_gamma W[k]_{beta gamma}[n, n'] R_{k+1}[gamma]
// Single-term sums reference the environment directly (pointer + coefficient);
// longer sums are materialised once per site (the element-wise blocking with
// integral coefficients, e.g. the a_k (x) a_s sum of Eq. prenormrule).
struct TRef {
  const double* p = nullptr;
  double coef = 0.0;
  int cls = -1;
};
struct Tilde {
  Env* env = nullptr;
  int nmid = 0;
  std::vector<std::array<TRef, 16>> ref;
  DArr<double> combo;
  long combo_flops = 0;
};

// Device-side work list of one grouped GEMM launch.
struct GemmPlan {
  DArr<GemmTile> tiles;
  DArr<GemmTask> tasks;
  DArr<GemmTerm> terms;
  int ntiles = 0;
  double flops = 0;
  void upload(const std::vector<GemmTile>& ti, const std::vector<GemmTask>& ta,
              const std::vector<GemmTerm>& te, cudaStream_t s);
  void run(cudaStream_t s) const;
};
struct GemmBuilder {
  std::vector<GemmTile> tiles;
  std::vector<GemmTask> tasks;
  std::vector<GemmTerm> terms;
  double flops = 0;
  int begin(double* C, int ldc, int m, int n, int beta);  // returns task index
  void term(const double* A, int lda, const double* B, int ldb, int k, int flags, double alpha, int m, int n);
  void end();  // emits tiles of the last task if it has terms (or beta == 0)
  bool empty() const { return tasks.empty(); }
  void clear() { tiles.clear(); tasks.clear(); terms.clear(); flops = 0; }
};

struct MixedPlan;
void mixed_plan_free(MixedPlan* p);
struct MixedDeleter {
  void operator()(MixedPlan* p) const { mixed_plan_free(p); }
};
struct TmaPlan;
void tma_plan_free(TmaPlan* p);
struct TmaDeleter {
  void operator()(TmaPlan* p) const { tma_plan_free(p); }
};

// Work lists of H_eff.psi for one two-site problem: FP64 grouped GEMMs, or
// (mx set) the tensor-core mixed-precision plan of engine_mixed.cu.
struct SigmaPlan {
  PsiLayout psi;
  DArr<double> in, out, X;
  std::vector<GemmPlan> stage1, stage2;
  std::unique_ptr<MixedPlan, MixedDeleter> mx;
  // tensor-core plan with TMA-staged operands (precisions 4-6)
  std::unique_ptr<TmaPlan, TmaDeleter> tm;
  double flops = 0;
  bool tensor() const { return mx != nullptr || tm != nullptr; }
};

struct Context;
struct Mlp;
struct MlpScratch;
struct MlpScratchDeleter {
  void operator()(MlpScratch* p) const;
};

// training pairs collected by Davidson for the learned preconditioner
struct Harvest {
  long cap = 0, count = 0;  // capacity and pairs collected
  int per_iter = 0;         // pairs drawn from each saved Davidson iterate
  uint64_t seed = 0;
  long solves = 0;
  DArr<float> F, P, T;
};

struct SweepStats {
  std::vector<double> energy, discarded, seconds, sigma_flops, sigma_seconds;
  std::vector<int> davidson_iters;
};

struct Context {
  int K = 0, N = 0, two_sz = 0, Na = 0, Nb = 0;
  double ecore = 0.0;
  std::vector<double> h1, eri;
  MPO mpo;
  cudaStream_t stream = nullptr;
  bool own_stream = false;
  cusolverDnHandle_t solver = nullptr;
  std::string last_error;

  std::vector<SiteT> sites;        // MPS tensors (device)
  std::vector<bool> site_set;
  std::vector<Env> left, right;    // left[b]: bond b (sites < b); right[b]: sites >= b

  // state of an explicitly prepared two-site problem (for gbdmrg_sigma / diag)
  int prepared = -1;
  Tilde lt, rt;
  SigmaPlan plan;
  bool have_plan = false;

  // counters: sigma flops / device seconds (CUDA events on the context stream),
  // and the algorithmic flops of every other grouped GEMM (environments, diagonal,
  // decimation)
  double sigma_flops_total = 0, sigma_time_total = 0, other_flops_total = 0;
  long sigma_calls = 0;
  cudaEvent_t ev0 = nullptr, ev1 = nullptr;
  // auxiliary streams/events for the independent per-sector eigenproblems of the decimation
  static constexpr int kAux = 4;
  cudaStream_t aux[kAux] = {nullptr, nullptr, nullptr, nullptr};
  cusolverDnHandle_t aux_solver[kAux] = {nullptr, nullptr, nullptr, nullptr};
  cudaEvent_t aux_ev[kAux + 1] = {nullptr, nullptr, nullptr, nullptr, nullptr};
  // wall seconds per phase of the two-site step (stream-synchronised):
  // 0 W-contracted operators, 1 sigma work lists, 2 diagonal, 3 Davidson,
  // 4 decimation, 5 environment update
  double phase_s[8] = {0, 0, 0, 0, 0, 0, 0, 0};
  double phase_flops[8] = {0, 0, 0, 0, 0, 0, 0, 0};  // algorithmic flops per phase
  int chunk_budget_mb = 2048;
  // stage-2 split-K granularity of tensor-core plans: the term list of an output block
  // is cut into parts of about (k-steps of the whole stage) / (split_tps x 152), i.e.
  // about split_tps tiles per SM; <= 0: no split
  double split_tps = 8.0;
  // stage 1 of the tensor-core sigma with stacked right operands: one task per
  // (bond state, group) whose operand is the W-contracted right operator over all
  // four x four site blocks of the two groups (absent blocks zero)
  bool stage1_stacked = false;
  // blocking sums with at least tc_combo_min_terms terms that feed only the
  // tensor-core sigma and the H_eff diagonal are formed on the tensor cores
  // (three BF16 slices, FP32 accumulation) instead of the FP64 units
  bool tc_combos = true;
  long tc_combo_min_terms = 100000;
  // 0: FP64 grouped GEMMs; 1: tensor cores, one BF16 pass; 2: tensor cores,
  // three BF16 slices (six products, about FP32 accuracy); 3: two BF16 slices
  // (three products); 4, 5, 6: tensor cores on the TMA-staged plan (stage 1 as
  // one dense GEMM per group over the stacked right operators) with one BF16
  // pass, three slices and two slices
  int precision = 0;
  // Davidson refinement of the tensor-core steps: after the solve with the
  // operator of `precision`, its Ritz vector starts a solve with the operator of
  // refine_precision (-1: none), of at most refine_iters iterations
  int refine_precision = -1;
  int refine_iters = 8;
  // environment updates: 0 FP64 grouped GEMMs; 2 tensor cores, three BF16 slices;
  // 3 tensor cores with exactly split operands (FP64-level results)
  int env_precision = 0;
  // X intermediates of the TMA-staged plan per chunk of bond states (MB)
  long tma_budget_mb = 65536;
  // keep host copies of tensor-core work lists (needed to fuse problems into batches)
  bool keep_host_plans = false;
  // learned Davidson preconditioner (not owned; null: diagonal) and its scratch
  Mlp* mlp = nullptr;
  std::unique_ptr<MlpScratch, MlpScratchDeleter> mlp_s;
  Harvest harvest;
  long mlp_applied = 0, mlp_fallbacks = 0;

  ~Context();
};

void ctx_init(Context& c);
void set_site_dense(Context& c, int k, int Dl, int Dr, const int* qn_l, const int* qn_r, const double* A);
void get_site_dense(Context& c, int k, std::vector<double>& A);
// <psi|H|psi>/<psi|psi> (+ ecore) of the current MPS at the prepared position
double expectation(Context& c);
// checkpoint of the MPS (bond sectors and block data of every site) to a file
void save_mps(Context& c, const char* path);
void load_mps(Context& c, const char* path);

void env_boundary_left(Context& c, Env& e);
void env_boundary_right(Context& c, Env& e);
// approx: the sums feed only the tensor-core sigma and the H_eff diagonal, so with
// tc_combos they may be formed on the tensor cores (about FP32 accuracy)
void build_tilde_left(Context& c, Env& L, int site, Tilde& t, bool approx = false);
void build_tilde_right(Context& c, Env& R, int site, Tilde& t, bool approx = false);
// blocking sums out_i = sum_j coef_ij Op_j of one environment on the tensor cores
// (engine_mixed.cu); out_cls[i] is the operator class of output i
void combos_tc(Context& c, Env& env, const std::vector<ComboOut>& outs, const std::vector<ComboTerm>& terms,
               const std::vector<int>& out_cls);
void env_alloc(Context& c, Env& e, const Bond& b, const std::vector<BondState>& st);
// environment update with both grouped GEMMs on the tensor cores, operands in three BF16
// slices (engine_mixed.cu); left = true: L_{k+1} from L_k and A[k], else R_k from R_{k+1}
void env_update_tc(Context& c, Tilde& t, const SiteT& A, int site, Env& out, bool left);
// the same update with exactly split operands: FP64-level results on the tensor cores
// (engine_mixed.cu)
void env_update_exact(Context& c, Tilde& t, const SiteT& A, int site, Env& out, bool left);
void env_update_left(Context& c, Tilde& lt, const SiteT& A, int site, Env& out);
void env_update_right(Context& c, Tilde& rt, const SiteT& B, int site, Env& out);

void build_sigma_plan(Context& c, Tilde& lt, Tilde& rt, int k, SigmaPlan& plan);
void run_sigma(Context& c, SigmaPlan& plan, const double* x, double* y);
void build_mixed_plan(Context& c, Tilde& lt, Tilde& rt, int k, SigmaPlan& plan, int nslices);
void run_mixed_sigma(Context& c, SigmaPlan& plan, const double* x, double* y);
int mixed_error(Context& c, SigmaPlan& plan);
void build_tma_plan(Context& c, Tilde& lt, Tilde& rt, int k, SigmaPlan& plan, int nslices);
void run_tma_sigma(Context& c, SigmaPlan& plan, const double* x, double* y);
// non-zero if a tensor-core launch of the plan reported a bounded wait that ran out
// (reads and clears nothing; synchronises the context stream)
int plan_error(Context& c, SigmaPlan& plan);
// host statistics of a TMA-staged plan: [0] stage-1 tiles, [1] stage-1 K steps,
// [2] stage-2 tiles, [3] stage-2 K steps, [4] executed stage-1 flops, [5] executed
// stage-2 flops, [6] X intermediate bytes, [7] stacked right-operand bytes, [8] chunks
void tma_plan_stats(const SigmaPlan& plan, double* out);

// batched tensor-core sigma over several prepared contexts (engine_mixed.cu)
struct BatchPlan;
BatchPlan* batch_create(const std::vector<Context*>& ctxs);
void batch_free(BatchPlan* b);
double batch_flops(const BatchPlan* b);
float batch_sigma(BatchPlan& b, const double* const* psi, double* const* sigma, bool use_graph);
// Autotuner of the tensor-core plans (engine_mixed.cu): for every candidate (split_tps,
// chunk budget) the plans of the prepared problems are rebuilt and H_eff.psi is timed
// with CUDA events (one context: its own plan; several: one batched launch per stage
// over all of them, replayed from a CUDA graph).  ms[i * budgets.size() + j] receives
// the time per call of (splits[i], budgets[j]); the plans are left built with the
// fastest candidate, which is returned.
struct TuneChoice {
  double split_tps;
  int budget_mb;
};
TuneChoice autotune_plans(const std::vector<Context*>& ctxs, const std::vector<double>& splits,
                          const std::vector<int>& budgets, int reps, std::vector<double>& ms);
void compute_diag(Context& c, Tilde& lt, Tilde& rt, int k, const PsiLayout& P, double* diag);

void prepare_two_site(Context& c, int k);
// compute_diag for the prepared problem with all scratch in a fixed static device
// array (noalloc.cu); no device allocation.
void compute_diag_noalloc(Context& c, double* diag);
size_t noalloc_scratch_bytes();
void make_psi(Context& c, const SiteT& TL, const SiteT& TR, const PsiLayout& P, double* psi);

struct DavidsonOpts {
  double tol = 1e-9;
  int max_iter = 200, max_sub = 24;
  // stop when the residual norm is below 2e-4 |theta| and has not improved by 10 %
  // for this many iterations (used with the tensor-core operator, whose rounding
  // leaves a residual floor; 0 = never)
  int stagnation = 0;
  // residual floor (relative to |theta|) below which the stagnation stop may fire
  double floor = 2e-4;
};
double davidson(Context& c, SigmaPlan& plan, const double* diag, double* psi, const DavidsonOpts& o,
                int* iters);

// decimation of psi at sites (k, k+1); direction 0 = left-move (A[k] = U, A[k+1] = S V^T),
// 1 = right-move (A[k] = U S, A[k+1] = V^T).  Returns discarded weight.
double decimate(Context& c, const PsiLayout& P, const double* psi, int M, int direction, SiteT& left,
                SiteT& right);

// One two-site step at sites (k, k+1) (blocking, solving, decimation of Sec. "The
// DMRG in renormalization group language"); needs left[k] and right[k+2].
// psi0/psi_out (optional, device, packed) override the start vector / receive
// the optimised one.  Returns the Davidson eigenvalue (without ecore).
double two_site_step(Context& c, int k, int dir, int M, const DavidsonOpts& o, bool free_used, int* iters,
                     double* discarded, const double* psi0 = nullptr, double* psi_out = nullptr,
                     long* nnz_out = nullptr);
// Algorithmic flops (sum 2mnk over non-zero blocks) of one sigma at sites
// (k, k+1) for the given bonds k and k+2 -- host only, equals SigmaPlan::flops.
double count_sigma_flops(const MPO& mpo, int k, const Bond& Lb, const Bond& Rb);

void right_canonicalize(Context& c);
void run_sweeps(Context& c, int nsweeps, const int* M, const double* tol, int max_iter, SweepStats& st);

}  // namespace gbdmrg
