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
 * (about FP32 accuracy).  Environments, Davidson, decimation stay FP64. */
gbdmrg_status gbdmrg_set_precision(gbdmrg_ctx* ctx, int32_t precision);

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
 * (work recorded while a stream is being captured into a CUDA graph, or inside a
 * framework whose memory manager owns the device).  Every scratch buffer it needs
 * is carved from one fixed 32 MiB array compiled into the library (held by each
 * GPU that loads the library until the process exits); problems that need more
 * return GBDMRG_EINVAL with the required size in gbdmrg_last_error.  The first
 * call on a device looks up that array's device address (cudaGetSymbolAddress),
 * so make it with the context's device current and before any stream capture.
 * All calls share the one array: calls that overlap on the GPU (several streams
 * or host threads at once) race.  diag_dev: device pointer, nnz doubles of the
 * packed layout.  Requires gbdmrg_prepare (which does allocate) beforehand. */
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

/* Number of CUDA kernel launches issued by this library in this process. */
int64_t gbdmrg_kernel_launches(void);

/* Self-test of the tensor-core grouped block GEMM used by the mixed-precision
 * sigma (tcgen05, BF16 operands, FP32 accumulation).  For every task i:
 *   C_i (+)= sum_{t in [t0_i, t1_i)} (-1)^neg_t A_t B_t^T
 * with C_i fp32 row-major (m_i x n_i, ldc_i), A_t (m_i x k_t) and B_t (n_i x k_t)
 * row-major bf16, 16-byte aligned, leading dimensions multiples of 8 and zero
 * padding between k_t and the leading dimension.  All matrix pointers are
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
  int32_t precision; /* as gbdmrg_set_precision: 0 FP64, 1 BF16 pass, 2 BF16 x3 slices */
} gbdmrg_schedule;

/* Run the sweeps from the current MPS (brought to right-canonical form first).
 * energies[nsweeps]: energy at the last step of each sweep (incl. ecore);
 * discarded[nsweeps]: largest discarded weight of each sweep (may be NULL). */
gbdmrg_status gbdmrg_run(gbdmrg_ctx* ctx, const gbdmrg_schedule* sched, double* energies, double* discarded);
/* Per-sweep statistics of the last run: seconds, sigma flops, sigma seconds,
 * Davidson iterations (each array nsweeps long, any may be NULL). */
gbdmrg_status gbdmrg_run_stats(gbdmrg_ctx* ctx, double* seconds, double* sigma_flops, double* sigma_seconds,
                               int32_t* davidson_iters);

#ifdef __cplusplus
}
#endif
#endif
