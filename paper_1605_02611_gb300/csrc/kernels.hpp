// Device kernels of the two-site DMRG hot path and their launch wrappers.
#pragma once
#include <cuda_runtime.h>

#include <cstdint>

namespace gbdmrg {

// One contribution C += alpha * op(A) * op(B) to an output block.
//   A: m x k row-major (lda) unless GT_TA: then A is stored k x m (A^T used)
//   B: n x k row-major (ldb)   (C = A B^T)  unless GT_BN: stored k x n (C = A B)
enum : int { GT_TA = 1, GT_BN = 2 };
struct GemmTerm {
  const double* A;
  const double* B;
  int lda, ldb, k, flags;
  double alpha;
};
// One output block: C (m x n, row-major ldc) = beta*C + sum_{t in [t0,t1)} terms
struct GemmTask {
  double* C;
  int ldc, m, n;
  int beta;
  int t0, t1;
};
struct GemmTile {
  int task, r0, c0;
};

constexpr int GEMM_TM = 64, GEMM_TN = 64, GEMM_TK = 16;

// Linear combination of operators with a common block layout:
//   out_j[e] = sum_{t in [c0_j, c1_j)} coef_t * in_t[e],  e < nnz_j
struct ComboOut {
  double* out;
  long nnz;
  int t0, t1;
};
struct ComboTerm {
  const double* in;
  double coef;
};

// Copy of a 2-D sub-block: dst[i*ldd + j] = alpha * src[i*lds + j] (or src[j*lds + i] if trans)
struct CopyJob {
  const double* src;
  double* dst;
  int rows, cols, lds, ldd, trans;
  double alpha;
};

// number of kernel launches issued by this library (all launch wrappers)
long launch_count();
// adds kernel launches made outside this file to the count
void count_launches(long n);

void launch_gemm(const GemmTile* d_tiles, int ntiles, const GemmTask* d_tasks,
                 const GemmTerm* d_terms, cudaStream_t s);
void launch_combo(const ComboOut* d_outs, int nouts, long max_nnz, const ComboTerm* d_terms,
                  cudaStream_t s);
void launch_copy(const CopyJob* d_jobs, int njobs, int max_elems, cudaStream_t s);
void launch_fill(double* p, long n, double v, cudaStream_t s);

// vector ops (FP64, length n)
// y = a x + b y (b == 0: y is only written)
void launch_axpby(long n, double a, const double* x, double b, double* y, cudaStream_t s);
// dots[j] = <V_j, x> for j < m, V row-major [m][n]; result written to d_out[m] (deterministic)
void launch_multidot(const double* V, long ldv, int m, const double* x, long n, double* d_part,
                     int nblk, double* d_out, cudaStream_t s);
// y = sum_j c[j] V_j  (c on device)
void launch_combine_vectors(const double* V, long ldv, int m, const double* d_c, long n, double* y,
                            cudaStream_t s);
// t = r / (theta - diag), |denominator| clamped to >= eps
void launch_precond(long n, const double* r, const double* diag, double theta, double eps,
                    double* t, cudaStream_t s);
// diagonal extraction: out[i * ldo + col] = coef * A[i*(lda+1)]  for i < rows
struct DiagJob {
  const double* A;
  double* out;
  int rows, lda, ldo;
  double coef;
};
void launch_diag_extract(const DiagJob* d_jobs, int njobs, int max_rows, cudaStream_t s);

// Davidson on the device (FP64).  Rayleigh-Ritz: lowest eigenpair of the symmetric
// part of the m x m projected matrix G (m <= 48) by parallel cyclic Jacobi in one
// thread block; eigenvalue to scal[0], eigenvector to y[0..m).  false (nothing
// launched) if m is outside [1, RR_MAX_SUB]
constexpr int RR_MAX_SUB = 48;
bool launch_rr(const double* G, int ldg, int m, double* y, double* scal, cudaStream_t s);
// r = hx - theta x (theta on device)
void launch_resid(long n, const double* hx, const double* x, const double* d_theta, double* r, cudaStream_t s);
// t = r / (theta - diag), theta on device
void launch_precond_dev(long n, const double* r, const double* diag, const double* d_theta, double eps, double* t,
                        cudaStream_t s);
// t -= sum_j c[j] V_j (c on device)
void launch_sub_combine(const double* V, long ldv, int m, const double* d_c, long n, double* t, cudaStream_t s);
// y = x / sqrt(*nrm2)
void launch_scale_rsqrt(long n, const double* x, const double* d_nrm2, double* y, cudaStream_t s);
// G[i][col] = G[col][i] = dots[i], i < m1
void launch_gcol(const double* dots, int m1, double* G, int ld, int col, cudaStream_t s);
// G[0] = theta / xn2
void launch_restart_g(double* G, const double* d_theta, const double* d_xn2, cudaStream_t s);

}  // namespace gbdmrg
