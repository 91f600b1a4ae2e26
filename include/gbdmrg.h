/* gbdmrg: two-site ab initio DMRG hot path on one GPU (sm_103a).
 *
 * Problem statement (paper Sec. "MPO representation of quantum chemistry
 * Hamiltonians", Eq. longrangeh): one- and two-electron integrals over K
 * spatial orbitals, N electrons, 2*S_z, bond dimension M and a sweep
 * schedule in; sweep energies, the MPS and discarded weights out.
 *
 * Conventions shared by every call:
 *  - site = spatial orbital k = 0..K-1, local basis n = n_alpha + 2 n_beta
 *    (|0>, |up>, |dn>, |up dn>); Jordan-Wigner order 0a,0b,1a,1b,...;
 *  - a bond index is labelled by the particle numbers (n_alpha, n_beta) of the
 *    block left of the bond; labels are passed as int32 pairs and must be
 *    grouped and sorted ascending by (n_alpha, n_beta);
 *  - dense MPS tensor of site k: float64 A[l][n][r], shape D_k x 4 x D_{k+1},
 *    row-major (Eq. FSMPS); entries outside l + q(n) = r are ignored;
 *  - two-site wavefunctions psi[l][n1][n2][r] for sites (k, k+1) are passed
 *    in the packed block layout reported by gbdmrg_psi_layout;
 *  - all pointers are owned by the caller; inputs are copied during the call;
 *  - a context is not thread-safe; distinct contexts may run concurrently;
 *  - no call aborts the process: errors return a status and the message is
 *    kept per context (gbdmrg_last_error).
 */
#ifndef GBDMRG_H
#define GBDMRG_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef enum {
  GBDMRG_OK = 0,
  GBDMRG_EINVAL = 1,   /* invalid argument (sizes, labels, symmetry, non-finite values) */
  GBDMRG_ENOMEM = 2,   /* device allocation failed */
  GBDMRG_ECUDA = 3,    /* CUDA / cuSOLVER error */
  GBDMRG_ENOCONV = 4,  /* eigen-solver failure */
  GBDMRG_ETIMEOUT = 5, /* a bounded device wait ran out */
  GBDMRG_EIO = 6,      /* file error */
  GBDMRG_ESMALL = 7,   /* caller buffer too small (size written back) */
  GBDMRG_ESTATE = 8    /* call not valid in the current state (e.g. MPS not set) */
} gbdmrg_status;

typedef struct gbdmrg_ctx gbdmrg_ctx;

/* Hamiltonian of Eq. (longrangeh) with spin made explicit:
 *   H = ecore + sum_{pq,s} h1[p*K+q] a+_{ps} a_{qs}
 *             + 1/2 sum_{pqrs,s,t} eri[((p*K+q)*K+r)*K+s] a+_{ps} a+_{rt} a_{st} a_{qs}
 * eri is (pq|rs) in chemists' order (v_pqrs = <pq|sr> = (ps|qr)).  h1 must be
 * symmetric and eri 8-fold symmetric to 1e-12 (else GBDMRG_EINVAL).
 * two_sz = N_alpha - N_beta; it must have the parity of N, 0 <= N <= 2K. */
typedef struct {
  int32_t K, N, two_sz;
  const double* h1;  /* [K*K] host */
  const double* eri; /* [K^4] host */
  double ecore;
} gbdmrg_problem;

/* Create a context on the current CUDA device.  stream: a cudaStream_t to run
 * on (NULL: the library creates its own).  Builds the MPO of Eq. (wproduct)
 * with normal/complementary operators and the switch of the complementary
 * side at K/2 (Sec. "MPO representation ...").  *out owned by the library. */
gbdmrg_status gbdmrg_create(const gbdmrg_problem* prob, void* stream, gbdmrg_ctx** out);
void gbdmrg_destroy(gbdmrg_ctx* ctx);
const char* gbdmrg_last_error(const gbdmrg_ctx* ctx);

/* Host-only (no GPU needed): build the MPO of `prob` and write its bond
 * dimensions dims[K+1] and, if dense != NULL and K <= 5, the MPO contracted
 * to the dense 4^K x 4^K matrix (row-major, Jordan-Wigner basis). */
gbdmrg_status gbdmrg_mpo_build_host(const gbdmrg_problem* prob, int32_t* dims, double* dense);

/* MPO bond dimensions D(k), k = 0..K (Eq. Hpartition: number of terms). dims[K+1]. */
gbdmrg_status gbdmrg_mpo_bond_dims(gbdmrg_ctx* ctx, int32_t* dims);
/* The MPO contracted to a dense 4^K x 4^K matrix (row-major, Jordan-Wigner
 * basis of the conventions above).  Only K <= 5; out has 4^(2K) doubles. */
gbdmrg_status gbdmrg_mpo_dense(gbdmrg_ctx* ctx, double* out);

/* Set the MPS tensor of one site (Eq. FSMPS).  qn_l[2*Dl], qn_r[2*Dr] are the
 * bond labels; A is D_l x 4 x D_r row-major (host).  Bonds of neighbouring
 * sites must agree; bond 0 is one state (0,0), bond K one state (Na,Nb). */
gbdmrg_status gbdmrg_set_mps(gbdmrg_ctx* ctx, int32_t site, int32_t Dl, int32_t Dr, const int32_t* qn_l,
                             const int32_t* qn_r, const double* A);
/* Bond sizes of site k (D_k, D_{k+1}) and, if A != NULL, the dense tensor. */
gbdmrg_status gbdmrg_get_mps(gbdmrg_ctx* ctx, int32_t site, int32_t* Dl, int32_t* Dr, double* A);
/* Labels of bond b (b = 0..K) of the current MPS: *D and, if qn != NULL, qn[2*D]. */
gbdmrg_status gbdmrg_get_bond(gbdmrg_ctx* ctx, int32_t bond, int32_t* D, int32_t* qn);

/* Arithmetic of H_eff.psi for subsequent gbdmrg_prepare / gbdmrg_step calls:
 * 0 = FP64 grouped GEMMs on the FP64 units; 1 = tensor cores (tcgen05), one
 * BF16 pass with FP32 accumulation; 2 = tensor cores, every operand split in
 * three BF16 slices and the six leading slice products accumulated in FP32
 * (about FP32 accuracy); 3 = tensor cores, two BF16 slices per operand and the
 * three leading products (operands to ~2^-16 relative); 4 = tensor cores, one
 * BF16 pass with FP32 accumulation on the TMA-staged work lists (stage 1 of
 * H_eff.psi, X_beta = psi Rt_beta^T of Eq. Hpartition's right factor, as one
 * dense GEMM per quantum-number group of the cut over all bond states, its
 * operands copied by the Tensor Memory Accelerator from a few large matrices;
 * stage 2 as long contractions over the operator terms); 5 and 6 = the same
 * work lists with three and two BF16 slices per operand (as 2 and 3).
 * Environments, Davidson, decimation stay FP64. */
gbdmrg_status gbdmrg_set_precision(gbdmrg_ctx* ctx, int32_t precision);

/* Device memory (MB) for the X intermediates of the precision 4-6 work lists
 * (default 65536): the bond states are processed in chunks whose intermediates
 * fit this budget (each chunk one stage-1 and one stage-2 launch).  Takes effect
 * at the next gbdmrg_prepare / gbdmrg_plan.  EINVAL for megabytes <= 0. */
gbdmrg_status gbdmrg_set_tma_budget(gbdmrg_ctx* ctx, int64_t megabytes);
/* Arithmetic of the environment (renormalised-operator) updates of later
 * gbdmrg_prepare / gbdmrg_step / gbdmrg_run calls (Eqs. leftrenorm/rightrenorm,
 * prenormmatrix/prenormdec): 0 = FP64 grouped GEMMs on the FP64 units (default);
 * 2 = both grouped GEMMs of the update on the tensor cores with every operand in
 * three BF16 slices (six products, FP32 accumulation, intermediates as three
 * BF16 slices of the FP32 results), the new operators stored in FP64 (FP32-level
 * accuracy); 3 = both GEMMs on the tensor cores with exactly split operands: every
 * block scaled by a power of two and split into six 7-bit integer slices (exact in
 * BF16), the slice products of each level summed exactly in the FP32 accumulators
 * and the levels added in two-float registers, stored in FP64 (operands carried to
 * ~2^-42 of each block's largest element; contractions longer than 128 are cut
 * into exact sums of at most 128 products).  EINVAL for any other value. */
gbdmrg_status gbdmrg_set_env_precision(gbdmrg_ctx* ctx, int32_t precision);
/* Refinement of the Davidson solve of every later tensor-core two-site step
 * (gbdmrg_step, gbdmrg_run; not part of the paper, which names no eigensolver):
 * after the solve with the operator of the context's precision, its Ritz vector
 * starts a second Davidson solve with the operator of `precision` (0 FP64 with
 * every W-contracted sum formed again on the FP64 units, or 1-6), whose residual
 * decides convergence and whose eigenvalue the step reports; it takes at most
 * max_iters iterations of the step's budget.  precision -1 turns it off (the
 * default).  EINVAL for precision outside -1..6 or max_iters < 1. */
gbdmrg_status gbdmrg_set_refinement(gbdmrg_ctx* ctx, int32_t precision, int32_t max_iters);
/* Work-list statistics of the prepared precision 4-6 H_eff.psi (zeros for other
 * precisions): out[0] stage-1 tiles, [1] stage-1 64-wide K steps, [2] stage-2
 * tiles, [3] stage-2 K steps, [4] stage-1 and [5] stage-2 tensor-core flops as
 * executed (128-row tiles, blocks padded to 16), [6] bytes of the X
 * intermediates per chunk, [7] bytes of the stacked right operators, [8] chunks. */
gbdmrg_status gbdmrg_plan_stats(gbdmrg_ctx* ctx, double* out);

/* Device memory (MB) for the per-chunk intermediates X_beta of one H_eff.psi
 * (default 2048): the operator terms are processed in chunks whose
 * intermediates fit this budget.  Takes effect at the next gbdmrg_prepare. */
gbdmrg_status gbdmrg_set_chunk_budget(gbdmrg_ctx* ctx, int32_t megabytes);

/* Keep host copies of the tensor-core work lists built by later gbdmrg_prepare
 * calls (needed by gbdmrg_batch_create; costs host memory).  keep: 0 or 1. */
gbdmrg_status gbdmrg_keep_host_plans(gbdmrg_ctx* ctx, int32_t keep);

/* Batched sigma vectors: n independent two-site problems, each a context on the
 * same device prepared (gbdmrg_prepare) in precision 1, 2 or 3 after
 * gbdmrg_keep_host_plans(ctx, 1).  Their H_eff.psi work lists are concatenated
 * so that one persistent tensor-core launch per stage serves every problem (the
 * independent sums over operator terms of Sec. "Perfect parallelism in the sum
 * of operators formulation", taken across problems).  Runs on the stream of
 * ctxs[0].  The contexts must outlive the batch and stay prepared.  Errors of
 * gbdmrg_batch_create are reported through gbdmrg_last_error(ctxs[0]). */
typedef struct gbdmrg_batch gbdmrg_batch;
gbdmrg_status gbdmrg_batch_create(int32_t n, gbdmrg_ctx* const* ctxs, gbdmrg_batch** out);
/* sigma_p = H_eff,p psi_p for every problem p (device pointers, packed layouts of
 * each context).  use_graph != 0: the device work is captured once into a CUDA
 * graph (after one eager pass) and replayed on later calls.  ms (optional):
 * device time of the batched work (CUDA events, excluding the input/output
 * copies); flops (optional): total algorithmic flops of the batch. */
gbdmrg_status gbdmrg_batch_sigma(gbdmrg_batch* b, const double* const* psi_dev, double* const* sigma_dev,
                                 int32_t use_graph, double* ms, double* flops);
const char* gbdmrg_batch_last_error(const gbdmrg_batch* b);
void gbdmrg_batch_destroy(gbdmrg_batch* b);

/* Split-K granularity of the tensor-core work lists built by later
 * gbdmrg_prepare / gbdmrg_plan calls: in the second stage of H_eff.psi the term
 * list of an output block (the sum over operator terms and symmetry blocks of
 * Eq. Hpartition) is cut into parts that add atomically, sized so that the stage
 * has about tiles_per_sm tiles per SM (152 SMs); tiles_per_sm <= 0: never cut.
 * Default 8.  Every value gives the same sigma up to the order of the FP32
 * additions.  EINVAL for a null context or a non-finite value. */
gbdmrg_status gbdmrg_set_split(gbdmrg_ctx* ctx, double tiles_per_sm);
/* Stage-1 decomposition of the tensor-core H_eff.psi for work lists built by
 * later gbdmrg_prepare / gbdmrg_plan calls.  stacked = 0 (default): one task per
 * (bond state, group of psi columns, output sector) with up to four site-block
 * terms.  stacked = 1: one task per (bond state, group) whose operand is the
 * W-contracted right operator over all four x four site blocks of the two groups,
 * built once per work list in BF16 slices with absent blocks zero (fewer, deeper
 * tiles; more memory and more padded products).  Same sigma up to the order of
 * the FP32 additions.  EINVAL for a null context. */
gbdmrg_status gbdmrg_set_stage1_stacked(gbdmrg_ctx* ctx, int32_t stacked);
/* W-contracted operator sums on the tensor cores.  on != 0: a blocking sum of
 * Eq. prenormrule type with at least min_terms terms in total, built for later
 * gbdmrg_prepare / gbdmrg_plan / gbdmrg_step calls in a tensor-core precision,
 * whose results feed only the tensor-core H_eff.psi and the H_eff diagonal (the
 * side that the environment update of the step does not use), is formed as one
 * GEMM per operator class in three BF16 slices with FP32 accumulation (about
 * FP32 accuracy) instead of on the FP64 units.  Default on, min_terms 100000
 * (in practice the sums of the switch site K/2 of larger problems).
 * EINVAL for a null context or a negative min_terms. */
gbdmrg_status gbdmrg_set_tc_combos(gbdmrg_ctx* ctx, int32_t on, int64_t min_terms);
/* Current plan parameters (either pointer may be NULL). */
gbdmrg_status gbdmrg_get_plan_params(gbdmrg_ctx* ctx, double* tiles_per_sm, int32_t* chunk_budget_mb);

/* Autotuner of the tensor-core work lists.  For every candidate pair
 * (splits[i], budgets_mb[j]) (gbdmrg_set_split, gbdmrg_set_chunk_budget) the
 * work lists of the prepared problems are rebuilt and H_eff.psi is timed with
 * CUDA events over reps calls after warm-up: with n == 1 the context's own
 * sigma, with n > 1 the n problems fused into one batched launch per stage and
 * replayed from a CUDA graph (as gbdmrg_batch_sigma; the contexts need
 * gbdmrg_keep_host_plans).  The inputs are zero vectors (the time does not
 * depend on the values).  ms[i * nbudgets + j] (caller-allocated, may be NULL)
 * receives the time per call of each candidate; the contexts are left with the
 * fastest pair, returned in best_split / best_budget_mb (may be NULL), and
 * their work lists rebuilt with it (a batch created earlier must be created
 * again).  splits == NULL: {32, 8, 2, 0.5, 0.125, 0.03125, 0}; budgets_mb ==
 * NULL: the current budget of ctxs[0].  EINVAL for empty lists, non-positive
 * budgets or reps; ESTATE if a context is not prepared in a tensor-core
 * precision.  Errors are reported through gbdmrg_last_error(ctxs[0]); after an
 * error during timing the contexts keep their previous parameters and must be
 * prepared again. */
gbdmrg_status gbdmrg_autotune(int32_t n, gbdmrg_ctx* const* ctxs, int32_t reps, const double* splits,
                              int32_t nsplits, const int32_t* budgets_mb, int32_t nbudgets, double* ms,
                              double* best_split, int32_t* best_budget_mb);

/* Build the renormalised operators (Eq. renormop) of bonds k and k+2 from the
 * current MPS tensors in whatever gauge they are (blocking + decimation,
 * Eqs. prenormmatrix/prenormdec), and the work lists of H_eff for the sites
 * (k, k+1).  Must precede gbdmrg_sigma / gbdmrg_diag / gbdmrg_psi_layout. */
gbdmrg_status gbdmrg_prepare(gbdmrg_ctx* ctx, int32_t k);

/* Rebuild only the work lists of H_eff for sites (k, k+1) (current precision)
 * from the environments the context already holds for bonds k and k+2. */
gbdmrg_status gbdmrg_plan(gbdmrg_ctx* ctx, int32_t k);

/* Packed layout of psi for the prepared sites.  *nblocks and *nnz are always
 * written; if blocks != NULL it receives nblocks rows of 7 int64:
 * (l_offset, l_dim, n1, n2, r_offset, r_dim, offset): the block holds
 * psi[l_offset + i][n1][n2][r_offset + j] at offset + i*r_dim + j. */
gbdmrg_status gbdmrg_psi_layout(gbdmrg_ctx* ctx, int64_t* nblocks, int64_t* nnz, int64_t* blocks);

/* sigma = H_eff psi (the Davidson sigma vector, two-site form of the
 * projected Hamiltonian; Sec. "Efficient implementation of expectation
 * values").  psi, sigma: packed, nnz doubles; on_device != 0 means both are
 * device pointers (on the context's device), else host.  *flops (optional)
 * receives the algorithmic flop count sum 2mnk over non-zero blocks. */
gbdmrg_status gbdmrg_sigma(gbdmrg_ctx* ctx, const double* psi, double* sigma, int32_t on_device, double* flops);
/* Diagonal of H_eff in the packed layout (Davidson preconditioner input). */
gbdmrg_status gbdmrg_diag(gbdmrg_ctx* ctx, double* diag, int32_t on_device);
/* Diagonal of H_eff for the prepared sites, like gbdmrg_diag with on_device = 1,
 * but without allocating any device memory.  The paper has no counterpart: this
 * entry exists for callers that cannot call cudaMalloc/cudaFree at that moment
 * (for example inside a framework whose memory manager owns the device and
 * forbids allocations between its own phases).  Every scratch buffer it needs is
 * carved from one fixed 32 MiB array compiled into the library (held by each GPU
 * that loads the library until the process exits); problems that need more
 * return GBDMRG_EINVAL with the required size in gbdmrg_last_error.  The first
 * call on a device looks up that array's device address (cudaGetSymbolAddress),
 * so make it with the context's device current and before any stream capture.
 * All calls share the one array (and one host staging buffer): calls whose GPU
 * work overlapped would race, even for different GPUs, so each call holds a
 * process-wide lock until its own GPU work has finished (it synchronises the
 * context stream before returning) and calls from several host threads run one
 * after another.  diag_dev: device pointer, nnz doubles of the packed layout.
 * Requires gbdmrg_prepare (which does allocate) beforehand. */
gbdmrg_status gbdmrg_diag_noalloc(gbdmrg_ctx* ctx, double* diag_dev);
/* Average device time (ms) of the sigma work of the last n calls of gbdmrg_sigma
 * with on_device != 0, timed with CUDA events on the context stream. */
gbdmrg_status gbdmrg_sigma_timing(gbdmrg_ctx* ctx, int32_t reps, const double* psi_dev, double* sigma_dev,
                                  double* ms_per_call);

/* One two-site update at sites (k, k+1) with the environments the context
 * holds for bonds k and k+2 (after gbdmrg_prepare(k), or after a previous
 * step): diagonal of H_eff, Davidson solve (at most dav_max_iter iterations,
 * residual norm dav_tol), decimation to at most M states, environment update
 * of bond k+1 (direction 0: site k left-orthonormal, left environment;
 * direction 1: site k+1 right-orthonormal, right environment).  Blocking,
 * solving and decimation of Sec. "The DMRG in renormalization group language".
 * psi_in (optional): start vector in the packed layout of gbdmrg_psi_layout
 * for (k, k+1), else the product of the two current site tensors; psi_out
 * (optional): the optimised packed psi.  Both host or both device pointers
 * (on_device).  energy (optional): eigenvalue + ecore; discarded (optional):
 * discarded weight; iters (optional): Davidson iterations. */
gbdmrg_status gbdmrg_step(gbdmrg_ctx* ctx, int32_t k, int32_t direction, int32_t M, double dav_tol,
                          int32_t dav_max_iter, const double* psi_in, double* psi_out, int32_t on_device,
                          double* energy, double* discarded, int32_t* iters);
/* Cumulative counters of the context: algorithmic sigma flops, sigma device
 * seconds (CUDA events), number of sigma calls, algorithmic flops of all other
 * grouped GEMMs (environment updates, diagonal, decimation).  Any may be NULL. */
gbdmrg_status gbdmrg_counters(gbdmrg_ctx* ctx, double* sigma_flops, double* sigma_seconds, int64_t* sigma_calls,
                              double* other_flops);
/* Cumulative wall seconds of the phases of gbdmrg_step / gbdmrg_run steps
 * (stream-synchronised): [0] W-contracted operators (element-wise blocking
 * sums), [1] work lists of H_eff.psi, [2] diagonal, [3] Davidson, [4]
 * decimation, [5] environment update, [6..7] reserved.  seconds[8]. */
gbdmrg_status gbdmrg_phase_times(gbdmrg_ctx* ctx, double* seconds);
/* Algorithmic flops of the same phases (sums 2mnk of their GEMMs and 2 per
 * multiply-add of the W-contracted sums), accumulated like gbdmrg_phase_times. */
gbdmrg_status gbdmrg_phase_flops(gbdmrg_ctx* ctx, double* flops);

/* Number of CUDA kernel launches issued by this library in this process. */
int64_t gbdmrg_kernel_launches(void);

/* Self-test of the tensor-core grouped block GEMM used by the mixed-precision
 * sigma (tcgen05, BF16 operands, FP32 accumulation).  For every task i:
 *   C_i (+)= sum_{t in [t0_i, t1_i)} (-1)^neg_t A_t B_t^T
 * with C_i fp32 row-major (m_i x n_i, ldc_i), A_t (m_i x k_t) and B_t (n_i x k_t)
 * row-major bf16, 16-byte aligned, leading dimensions multiples of 8; columns
 * are read only up to the first multiple of 8 at or above k_t, and those past
 * k_t must be zero in at least one operand (finite in the other).  All matrix pointers are
 * device pointers; the descriptor arrays are host arrays:
 * tasks[8*i] = (C, ldc, m, n, beta, t0, t1, trans), terms[6*t] = (A, B, lda, ldb, k, neg);
 * trans != 0 stores element (r, c) of the block at C[c * ldc + r].
 * GBDMRG_ETIMEOUT if a bounded wait inside the kernel ran out. */
gbdmrg_status gbdmrg_gemm_bf16_selftest(const int64_t* tasks, int32_t ntasks, const int64_t* terms, int32_t nterms,
                                        void* stream);

/* Host only: algorithmic flop count of one sigma at sites (k, k+1) when bond k
 * has labels qn_l[2*Dl] and bond k+2 has qn_r[2*Dr] (sum 2mnk over non-zero
 * blocks, the count gbdmrg_sigma reports). */
gbdmrg_status gbdmrg_sigma_flops_host(const gbdmrg_problem* prob, int32_t k, int32_t Dl, const int32_t* qn_l,
                                      int32_t Dr, const int32_t* qn_r, double* flops);

/* Sweep schedule (Sec. "The DMRG in renormalization group language"):
 * nsweeps sweeps, sweep s keeps at most M[s] states and converges Davidson
 * to residual norm dav_tol[s].  One sweep = left-to-right over k = 0..K-3
 * then right-to-left over k = K-2..1.  K >= 3. */
typedef struct {
  int32_t nsweeps;
  const int32_t* M;
  const double* dav_tol;
  int32_t dav_max_iter;
  int32_t precision; /* as gbdmrg_set_precision: 0 FP64, 1 BF16 pass, 2 BF16 x3, 3 BF16 x2 slices,
                        4, 5, 6 one pass, three and two slices on the TMA-staged
                        work lists */
} gbdmrg_schedule;

/* Run the sweeps from the current MPS (brought to right-canonical form first).
 * energies[nsweeps]: energy at the last step of each sweep (incl. ecore);
 * discarded[nsweeps]: largest discarded weight of each sweep (may be NULL). */
gbdmrg_status gbdmrg_run(gbdmrg_ctx* ctx, const gbdmrg_schedule* sched, double* energies, double* discarded);
/* Per-sweep statistics of the last run: seconds, sigma flops, sigma seconds,
 * Davidson iterations (each array nsweeps long, any may be NULL). */
gbdmrg_status gbdmrg_run_stats(gbdmrg_ctx* ctx, double* seconds, double* sigma_flops, double* sigma_seconds,
                               int32_t* davidson_iters);

/* Expectation value <psi|H|psi>/<psi|psi> + ecore of the context's Hamiltonian
 * in the current MPS, evaluated at the prepared two-site position (gbdmrg_prepare)
 * as psi . H_eff psi with psi the contraction of sites k, k+1 (Eq. MPSCform, the
 * two-site form; the renormalised operators of Eq. renormop carry the rest of
 * the chain).  The value is exact when the sites left of k are left-orthonormal
 * and those right of k+1 right-orthonormal (as after gbdmrg_run, for k = 0 and
 * k = 1); elsewhere the norm is only approximated by |psi|^2.  An expectation of
 * another operator of the same form (for
 * example a one-body operator: eri = 0) is obtained from a second context with
 * those integrals and the same MPS (gbdmrg_save / gbdmrg_load or gbdmrg_set_mps).
 * GBDMRG_ESTATE without gbdmrg_prepare. */
gbdmrg_status gbdmrg_expectation(gbdmrg_ctx* ctx, double* value);

/* Checkpoint / resume of the MPS (the state a sweep continues from; Sec.
 * "Matrix product states", Eq. FSMPS): every site's bond sectors
 * (n_alpha, n_beta, dimension) and quantum-number block data in FP64, written
 * to a binary file at `path` (host byte order, header "GBDMRGv1", K, N, 2S_z).
 * gbdmrg_save: GBDMRG_ESTATE if a site is not set, GBDMRG_EIO if the file
 * cannot be written.  gbdmrg_load: GBDMRG_EINVAL if K, N or 2S_z differ from
 * the context's problem, GBDMRG_EIO for an unreadable, truncated or
 * inconsistent file; the context's MPS changes only when the whole file is
 * valid.  Environments are rebuilt by the next gbdmrg_prepare / gbdmrg_run. */
gbdmrg_status gbdmrg_save(gbdmrg_ctx* ctx, const char* path);
gbdmrg_status gbdmrg_load(gbdmrg_ctx* ctx, const char* path);

/* ------------------------------------------------------------------------
 * Learned Davidson preconditioner.
 *
 * The paper's solving step (Sec. "The DMRG in renormalization group language")
 * finds the lowest eigenpair of H_eff without naming the eigensolver; the
 * library uses Davidson, whose diagonal preconditioner turns the residual
 * r = H_eff x - theta x into t_i = r_i / (theta - d_i), d = diag(H_eff),
 * |theta - d_i| clamped to >= 1e-8.  The learned preconditioner keeps this form
 * and multiplies element i by (1 + g(f_i)), where g is a 3-layer network
 * (5 -> 256 -> 256 -> 1, GELU, BF16 weights, FP32 accumulation) of the
 * per-element features (n elements, b the quantum-number block of element i,
 * delta_i = d_i - theta):
 *   f0 = r_i sqrt(n)/|r|, f1 = asinh(delta_i), f2 = delta_i/(delta_i^2 + 0.01),
 *   f3 = asinh(rms_b(r) sqrt(n)/|r|), f4 = asinh(mean_b(d) - theta).
 * Parameters, as one float array of gbdmrg_mlp_nparams() entries:
 *   W1[256][5], b1[256], W2[256][256], b2[256], W3[256], b3   (row = output)
 * Training pairs (f, P, T): P = p_i s and T = tau_i s with p the diagonal
 * correction, tau = psi/(x . psi) - x the exact correction of a Ritz vector x
 * towards the converged psi, s = sqrt(n)/|tau|, both clipped to [-100, 100];
 * loss = mean(((1 + g) P - T)^2).  The untrained network (W3 = 0, b3 = 0) is
 * the diagonal preconditioner.
 * ------------------------------------------------------------------------ */
typedef struct gbdmrg_mlp gbdmrg_mlp;
int64_t gbdmrg_mlp_nparams(void);
/* W1 and W2 drawn from N(0, 1/fan_in) with the seed, the rest zero.  stream:
 * a cudaStream_t, or NULL for a stream owned by the network. */
gbdmrg_status gbdmrg_mlp_create(uint64_t seed, void* stream, gbdmrg_mlp** out);
void gbdmrg_mlp_destroy(gbdmrg_mlp* mlp);
const char* gbdmrg_mlp_last_error(const gbdmrg_mlp* mlp);
/* host arrays of gbdmrg_mlp_nparams() floats; set resets the Adam state.
 * GBDMRG_EINVAL on a non-finite parameter. */
gbdmrg_status gbdmrg_mlp_set_params(gbdmrg_mlp* mlp, const float* params);
gbdmrg_status gbdmrg_mlp_get_params(gbdmrg_mlp* mlp, float* params);
/* g for n feature rows features[n][5].  inference = 0: training numerics (FP32,
 * weights rounded to BF16); 1: inference numerics (h1 rounded to BF16, the
 * 256 x 256 layer on the tensor cores).  on_device: pointers are device (1) or
 * host (0) memory. */
gbdmrg_status gbdmrg_mlp_forward(gbdmrg_mlp* mlp, const float* features, int64_t n, float* g, int32_t inference,
                                 int32_t on_device);
/* Loss of n pairs and its gradient (training numerics; grad: host array of
 * gbdmrg_mlp_nparams() floats, may be NULL). */
gbdmrg_status gbdmrg_mlp_loss_grad(gbdmrg_mlp* mlp, const float* features, const float* P, const float* T, int64_t n,
                                   int32_t on_device, float* grad, double* loss);
/* Adam (beta 0.9/0.999, eps 1e-8, step size lr) for `epochs` passes of
 * ceil(n/batch) minibatches drawn with replacement by a counter-based hash of
 * seed.  loss_first / loss_last (may be NULL): mean loss of the first and the
 * last epoch. */
gbdmrg_status gbdmrg_mlp_train(gbdmrg_mlp* mlp, const float* features, const float* P, const float* T, int64_t n,
                               int32_t on_device, int32_t epochs, int32_t batch, float lr, uint64_t seed,
                               double* loss_first, double* loss_last);
/* Davidson of this context uses the network (not owned; must outlive its use),
 * or the diagonal preconditioner when mlp is NULL.  Per iteration the diagonal
 * correction is used instead when the residual norm did not decrease since the
 * previous iteration or the network produced a non-finite value. */
gbdmrg_status gbdmrg_set_preconditioner(gbdmrg_ctx* ctx, gbdmrg_mlp* mlp);
/* The correction t for residual r and Ritz value theta at the prepared
 * two-site problem (packed layout), with the current preconditioner. */
gbdmrg_status gbdmrg_precondition(gbdmrg_ctx* ctx, const double* r, double theta, double* t, int32_t on_device);
/* Training pairs at ns elements drawn by the SplitMix64 hash of (seed + j),
 * j = 0..ns-1, index = hash mod n: features[ns][5], P[ns], T[ns], idx[ns]
 * (idx may be NULL) for Ritz vector x, residual r, Ritz value theta and
 * converged vector psi of the prepared problem.  written = ns, or 0 when
 * x = psi (no correction). */
gbdmrg_status gbdmrg_make_pairs(gbdmrg_ctx* ctx, const double* x, const double* r, double theta, const double* psi,
                                int64_t ns, uint64_t seed, int32_t on_device, float* features, float* P, float* T,
                                int64_t* idx, int64_t* written);
/* Collect up to `capacity` pairs during later Davidson runs of this context:
 * per solve, from the Ritz vectors of iterations 0, 1, 2, 4, 7, 11 and 16
 * (those not yet converged and with |x . psi| >= 0.5), per_iteration pairs
 * each.  Resets the collection. */
gbdmrg_status gbdmrg_set_harvest(gbdmrg_ctx* ctx, int64_t capacity, int32_t per_iteration, uint64_t seed);
/* Number of pairs collected (n) and, for non-NULL host arrays, the pairs. */
gbdmrg_status gbdmrg_get_harvest(gbdmrg_ctx* ctx, float* features, float* P, float* T, int64_t* n);
/* Davidson iterations that used the network, and those that fell back to
 * the diagonal correction, since the context was created. */
gbdmrg_status gbdmrg_precond_counters(gbdmrg_ctx* ctx, int64_t* learned, int64_t* fallbacks);

#ifdef __cplusplus
}
#endif
#endif
