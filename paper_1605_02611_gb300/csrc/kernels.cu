// FP64 kernels of the two-site DMRG hot path (sm_103a).
//
// gemm_f64: grouped block GEMM.  Every output block of the sigma vector, of
// the stage-1 intermediate and of the renormalised operators is one task with
// a list of terms (A, B, alpha); the sum over terms is the concatenation of
// the contraction dimension over operator terms and quantum-number blocks
// (the paper's sum over left-right operator pairs, Eq. Hpartition, and over
// symmetry blocks).  Tasks are output-stationary, so there are no atomics and
// the result is deterministic.
#include "kernels.hpp"

#include <atomic>

namespace gbdmrg {

namespace {

__global__ void __launch_bounds__(256) gemm_f64_kernel(const GemmTile* __restrict__ tiles,
                                                       const GemmTask* __restrict__ tasks,
                                                       const GemmTerm* __restrict__ terms) {
  __shared__ double As[GEMM_TK][GEMM_TM + 1];
  __shared__ double Bs[GEMM_TK][GEMM_TN + 1];
  const GemmTile tl = tiles[blockIdx.x];
  const GemmTask tk = tasks[tl.task];
  const int tid = threadIdx.x;
  const int tx = tid & 15, ty = tid >> 4;
  double acc[4][4];
#pragma unroll
  for (int i = 0; i < 4; ++i)
#pragma unroll
    for (int j = 0; j < 4; ++j) acc[i][j] = 0.0;

  for (int t = tk.t0; t < tk.t1; ++t) {
    const GemmTerm tm = terms[t];
    const bool ta = tm.flags & GT_TA, bn = tm.flags & GT_BN;
    for (int k0 = 0; k0 < tm.k; k0 += GEMM_TK) {
#pragma unroll
      for (int r = 0; r < 4; ++r) {
        const int e = tid + 256 * r;
        int i, kk;
        if (!ta) { i = e >> 4; kk = e & 15; } else { kk = e >> 6; i = e & 63; }
        const int gi = tl.r0 + i, gk = k0 + kk;
        double v = 0.0;
        if (gi < tk.m && gk < tm.k)
          v = tm.alpha * (ta ? tm.A[(long)gk * tm.lda + gi] : tm.A[(long)gi * tm.lda + gk]);
        As[kk][i] = v;
        int j;
        if (!bn) { j = e >> 4; kk = e & 15; } else { kk = e >> 6; j = e & 63; }
        const int gj = tl.c0 + j, gk2 = k0 + kk;
        double w = 0.0;
        if (gj < tk.n && gk2 < tm.k)
          w = bn ? tm.B[(long)gk2 * tm.ldb + gj] : tm.B[(long)gj * tm.ldb + gk2];
        Bs[kk][j] = w;
      }
      __syncthreads();
#pragma unroll
      for (int kk = 0; kk < GEMM_TK; ++kk) {
        double a[4], b[4];
#pragma unroll
        for (int i = 0; i < 4; ++i) a[i] = As[kk][ty + 16 * i];
#pragma unroll
        for (int j = 0; j < 4; ++j) b[j] = Bs[kk][tx + 16 * j];
#pragma unroll
        for (int i = 0; i < 4; ++i)
#pragma unroll
          for (int j = 0; j < 4; ++j) acc[i][j] = fma(a[i], b[j], acc[i][j]);
      }
      __syncthreads();
    }
  }
#pragma unroll
  for (int i = 0; i < 4; ++i) {
    const int gi = tl.r0 + ty + 16 * i;
    if (gi >= tk.m) continue;
#pragma unroll
    for (int j = 0; j < 4; ++j) {
      const int gj = tl.c0 + tx + 16 * j;
      if (gj >= tk.n) continue;
      double* c = tk.C + (long)gi * tk.ldc + gj;
      *c = (tk.beta ? *c : 0.0) + acc[i][j];
    }
  }
}

__global__ void combo_kernel(const ComboOut* __restrict__ outs, const ComboTerm* __restrict__ terms) {
  const ComboOut o = outs[blockIdx.y];
  for (long e = (long)blockIdx.x * blockDim.x + threadIdx.x; e < o.nnz; e += (long)gridDim.x * blockDim.x) {
    double s = 0.0;
    for (int t = o.t0; t < o.t1; ++t) s = fma(terms[t].coef, terms[t].in[e], s);
    o.out[e] = s;
  }
}

__global__ void copy_kernel(const CopyJob* __restrict__ jobs) {
  const CopyJob jb = jobs[blockIdx.y];
  const long n = (long)jb.rows * jb.cols;
  for (long e = (long)blockIdx.x * blockDim.x + threadIdx.x; e < n; e += (long)gridDim.x * blockDim.x) {
    const int i = (int)(e / jb.cols), j = (int)(e % jb.cols);
    const double v = jb.trans ? jb.src[(long)j * jb.lds + i] : jb.src[(long)i * jb.lds + j];
    jb.dst[(long)i * jb.ldd + j] = jb.alpha * v;
  }
}

__global__ void fill_kernel(double* p, long n, double v) {
  for (long e = (long)blockIdx.x * blockDim.x + threadIdx.x; e < n; e += (long)gridDim.x * blockDim.x) p[e] = v;
}

// y = a x + b y; with b == 0 y is not read (it may be uninitialised, and 0 * NaN is NaN)
__global__ void axpby_kernel(long n, double a, const double* __restrict__ x, double b, double* __restrict__ y) {
  if (b == 0.0) {
    for (long e = (long)blockIdx.x * blockDim.x + threadIdx.x; e < n; e += (long)gridDim.x * blockDim.x)
      y[e] = a * x[e];
    return;
  }
  for (long e = (long)blockIdx.x * blockDim.x + threadIdx.x; e < n; e += (long)gridDim.x * blockDim.x)
    y[e] = a * x[e] + b * y[e];
}

__global__ void multidot_part_kernel(const double* __restrict__ V, long ldv, const double* __restrict__ x,
                                     long n, double* __restrict__ part) {
  __shared__ double red[256];
  const int j = blockIdx.y;
  const double* v = V + (long)j * ldv;
  double s = 0.0;
  for (long e = (long)blockIdx.x * blockDim.x + threadIdx.x; e < n; e += (long)gridDim.x * blockDim.x)
    s = fma(v[e], x[e], s);
  red[threadIdx.x] = s;
  __syncthreads();
  for (int w = 128; w > 0; w >>= 1) {
    if ((int)threadIdx.x < w) red[threadIdx.x] += red[threadIdx.x + w];
    __syncthreads();
  }
  if (threadIdx.x == 0) part[(long)j * gridDim.x + blockIdx.x] = red[0];
}

__global__ void multidot_final_kernel(const double* __restrict__ part, int nblk, int m, double* out) {
  const int j = blockIdx.x * blockDim.x + threadIdx.x;
  if (j >= m) return;
  double s = 0.0;
  for (int b = 0; b < nblk; ++b) s += part[(long)j * nblk + b];
  out[j] = s;
}

__global__ void combine_vectors_kernel(const double* __restrict__ V, long ldv, int m,
                                       const double* __restrict__ c, long n, double* __restrict__ y) {
  for (long e = (long)blockIdx.x * blockDim.x + threadIdx.x; e < n; e += (long)gridDim.x * blockDim.x) {
    double s = 0.0;
    for (int j = 0; j < m; ++j) s = fma(c[j], V[(long)j * ldv + e], s);
    y[e] = s;
  }
}

__global__ void precond_kernel(long n, const double* __restrict__ r, const double* __restrict__ d,
                               double theta, double eps, double* __restrict__ t) {
  for (long e = (long)blockIdx.x * blockDim.x + threadIdx.x; e < n; e += (long)gridDim.x * blockDim.x) {
    double den = theta - d[e];
    if (fabs(den) < eps) den = den < 0 ? -eps : eps;
    t[e] = r[e] / den;
  }
}

__global__ void diag_extract_kernel(const DiagJob* __restrict__ jobs) {
  const DiagJob jb = jobs[blockIdx.y];
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < jb.rows; i += gridDim.x * blockDim.x)
    jb.out[(long)i * jb.ldo] = jb.coef * jb.A[(long)i * (jb.lda + 1)];
}

// ---- device-resident Davidson helpers (FP64)

// Lowest eigenpair of the symmetric part of the m x m projected matrix G (row-major,
// leading dimension ldg), by cyclic Jacobi rotations in parallel (round-robin
// ordering: m/2 disjoint rotations per step, each step J^T A J with the rotations
// applied to all columns, then all rows), one thread block.  Writes the eigenvalue
// to scal[0] and its eigenvector to y[0..m).
constexpr int RR_MAX = 48;
__global__ void rr_kernel(const double* __restrict__ G, int ldg, int m, double* __restrict__ y,
                          double* __restrict__ scal) {
  __shared__ double A[RR_MAX][RR_MAX + 1], V[RR_MAX][RR_MAX + 1];
  __shared__ double cs[RR_MAX / 2], sn[RR_MAX / 2];
  __shared__ int pp[RR_MAX / 2], qq[RR_MAX / 2];
  __shared__ double red[256];
  __shared__ int done;
  const int tid = threadIdx.x, nt = blockDim.x;
  const int mp = m + (m & 1);  // even size: index m (if odd) is a dummy that never rotates
  for (int e = tid; e < m * m; e += nt) {
    const int i = e / m, j = e % m;
    A[i][j] = 0.5 * (G[(long)i * ldg + j] + G[(long)j * ldg + i]);
    V[i][j] = i == j ? 1.0 : 0.0;
  }
  __syncthreads();
  for (int sweep = 0; sweep < 60; ++sweep) {
    // off-diagonal and total squared norms
    double off = 0.0, tot = 0.0;
    for (int e = tid; e < m * m; e += nt) {
      const int i = e / m, j = e % m;
      const double a2 = A[i][j] * A[i][j];
      tot += a2;
      if (i != j) off += a2;
    }
    red[tid] = off;
    __syncthreads();
    for (int w = nt / 2; w > 0; w >>= 1) {
      if (tid < w) red[tid] += red[tid + w];
      __syncthreads();
    }
    const double off_s = red[0];
    __syncthreads();
    red[tid] = tot;
    __syncthreads();
    for (int w = nt / 2; w > 0; w >>= 1) {
      if (tid < w) red[tid] += red[tid + w];
      __syncthreads();
    }
    if (tid == 0) done = (off_s <= 1e-30 * red[0] || off_s == 0.0) ? 1 : 0;
    __syncthreads();
    if (done) break;
    for (int step = 0; step < mp - 1; ++step) {
      // round robin: position 0 fixed, the others rotate by one each step
      if (tid < mp / 2) {
        auto at = [&](int pos) { return pos == 0 ? 0 : 1 + (pos - 1 + step) % (mp - 1); };
        int p = at(tid), q = at(mp - 1 - tid);
        if (p > q) { const int t = p; p = q; q = t; }
        double c = 1.0, s = 0.0;
        if (q < m) {
          const double apq = A[p][q];
          if (fabs(apq) >= 1e-300) {
            const double theta = (A[q][q] - A[p][p]) / (2.0 * apq);
            const double t = (theta >= 0 ? 1.0 : -1.0) / (fabs(theta) + sqrt(theta * theta + 1.0));
            c = 1.0 / sqrt(t * t + 1.0);
            s = t * c;
          }
        }
        pp[tid] = p;
        qq[tid] = q < m ? q : p;
        cs[tid] = c;
        sn[tid] = q < m ? s : 0.0;
      }
      __syncthreads();
      // columns p, q of every row (A and V)
      for (int e = tid; e < (mp / 2) * m; e += nt) {
        const int r = e / m, k = e % m;
        const int p = pp[r], q = qq[r];
        if (p == q) continue;
        const double c = cs[r], s = sn[r];
        const double akp = A[k][p], akq = A[k][q];
        A[k][p] = c * akp - s * akq;
        A[k][q] = s * akp + c * akq;
        const double vkp = V[k][p], vkq = V[k][q];
        V[k][p] = c * vkp - s * vkq;
        V[k][q] = s * vkp + c * vkq;
      }
      __syncthreads();
      // rows p, q of every column
      for (int e = tid; e < (mp / 2) * m; e += nt) {
        const int r = e / m, k = e % m;
        const int p = pp[r], q = qq[r];
        if (p == q) continue;
        const double c = cs[r], s = sn[r];
        const double apk = A[p][k], aqk = A[q][k];
        A[p][k] = c * apk - s * aqk;
        A[q][k] = s * apk + c * aqk;
      }
      __syncthreads();
    }
  }
  // lowest eigenvalue (first index on ties, as a stable ascending sort would give)
  if (tid == 0) {
    int best = 0;
    for (int i = 1; i < m; ++i)
      if (A[i][i] < A[best][best]) best = i;
    scal[0] = A[best][best];
    pp[0] = best;
  }
  __syncthreads();
  for (int i = tid; i < m; i += nt) y[i] = V[i][pp[0]];
}

// r = hx - theta x, theta read from the device
__global__ void resid_kernel(long n, const double* __restrict__ hx, const double* __restrict__ x,
                             const double* __restrict__ theta, double* __restrict__ r) {
  const double th = *theta;
  for (long e = (long)blockIdx.x * blockDim.x + threadIdx.x; e < n; e += (long)gridDim.x * blockDim.x)
    r[e] = hx[e] - th * x[e];
}

// t = r / (theta - diag), theta read from the device, |denominator| clamped to >= eps
__global__ void precond_dev_kernel(long n, const double* __restrict__ r, const double* __restrict__ d,
                                   const double* __restrict__ theta, double eps, double* __restrict__ t) {
  const double th = *theta;
  for (long e = (long)blockIdx.x * blockDim.x + threadIdx.x; e < n; e += (long)gridDim.x * blockDim.x) {
    double den = th - d[e];
    if (fabs(den) < eps) den = den < 0 ? -eps : eps;
    t[e] = r[e] / den;
  }
}

// t -= sum_j c[j] V_j
__global__ void sub_combine_kernel(const double* __restrict__ V, long ldv, int m, const double* __restrict__ c,
                                   long n, double* __restrict__ t) {
  for (long e = (long)blockIdx.x * blockDim.x + threadIdx.x; e < n; e += (long)gridDim.x * blockDim.x) {
    double s = 0.0;
    for (int j = 0; j < m; ++j) s = fma(c[j], V[(long)j * ldv + e], s);
    t[e] -= s;
  }
}

// y = x / sqrt(*nrm2) (zero if the norm is zero)
__global__ void scale_rsqrt_kernel(long n, const double* __restrict__ x, const double* __restrict__ nrm2,
                                   double* __restrict__ y) {
  const double v = *nrm2;
  const double f = v > 0.0 ? 1.0 / sqrt(v) : 0.0;
  for (long e = (long)blockIdx.x * blockDim.x + threadIdx.x; e < n; e += (long)gridDim.x * blockDim.x)
    y[e] = f * x[e];
}

// column and row `col` of G from dots[0..m1)
__global__ void gcol_kernel(const double* __restrict__ dots, int m1, double* __restrict__ G, int ld, int col) {
  for (int i = threadIdx.x; i < m1; i += blockDim.x) {
    G[(long)i * ld + col] = dots[i];
    G[(long)col * ld + i] = dots[i];
  }
}

// G[0] = theta / xn2 (the restarted subspace holds the Ritz vector alone)
__global__ void restart_g_kernel(double* __restrict__ G, const double* __restrict__ theta,
                                 const double* __restrict__ xn2) {
  if (threadIdx.x == 0 && blockIdx.x == 0) G[0] = *theta / *xn2;
}

inline int grid_for(long n, int per = 256, int cap = 152 * 16) {
  long g = (n + per - 1) / per;
  if (g < 1) g = 1;
  if (g > cap) g = cap;
  return (int)g;
}

std::atomic<long> g_launches{0};

}  // namespace

long launch_count() { return g_launches.load(); }
void count_launches(long n) { g_launches += n; }

void launch_gemm(const GemmTile* d_tiles, int ntiles, const GemmTask* d_tasks, const GemmTerm* d_terms,
                 cudaStream_t s) {
  if (ntiles <= 0) return;
  ++g_launches;
  gemm_f64_kernel<<<ntiles, 256, 0, s>>>(d_tiles, d_tasks, d_terms);
}

void launch_combo(const ComboOut* d_outs, int nouts, long max_nnz, const ComboTerm* d_terms, cudaStream_t s) {
  if (nouts <= 0 || max_nnz <= 0) return;
  for (int o0 = 0; o0 < nouts; o0 += 65535) {
    int no = nouts - o0 < 65535 ? nouts - o0 : 65535;
    dim3 g(grid_for(max_nnz, 256, 64), no);
    combo_kernel<<<g, 256, 0, s>>>(d_outs + o0, d_terms);
    ++g_launches;
  }
}

void launch_copy(const CopyJob* d_jobs, int njobs, int max_elems, cudaStream_t s) {
  if (njobs <= 0 || max_elems <= 0) return;
  for (int o0 = 0; o0 < njobs; o0 += 65535) {
    int no = njobs - o0 < 65535 ? njobs - o0 : 65535;
    dim3 g(grid_for(max_elems, 256, 64), no);
    copy_kernel<<<g, 256, 0, s>>>(d_jobs + o0);
    ++g_launches;
  }
}

void launch_fill(double* p, long n, double v, cudaStream_t s) {
  if (n <= 0) return;
  ++g_launches;
  fill_kernel<<<grid_for(n), 256, 0, s>>>(p, n, v);
}

void launch_axpby(long n, double a, const double* x, double b, double* y, cudaStream_t s) {
  if (n <= 0) return;
  ++g_launches;
  axpby_kernel<<<grid_for(n), 256, 0, s>>>(n, a, x, b, y);
}

void launch_multidot(const double* V, long ldv, int m, const double* x, long n, double* d_part, int nblk,
                     double* d_out, cudaStream_t s) {
  if (m <= 0) return;
  dim3 g(nblk, m);
  multidot_part_kernel<<<g, 256, 0, s>>>(V, ldv, x, n, d_part);
  multidot_final_kernel<<<(m + 63) / 64, 64, 0, s>>>(d_part, nblk, m, d_out);
  g_launches += 2;
}

void launch_combine_vectors(const double* V, long ldv, int m, const double* d_c, long n, double* y,
                            cudaStream_t s) {
  if (n <= 0) return;
  ++g_launches;
  combine_vectors_kernel<<<grid_for(n), 256, 0, s>>>(V, ldv, m, d_c, n, y);
}

void launch_precond(long n, const double* r, const double* diag, double theta, double eps, double* t,
                    cudaStream_t s) {
  if (n <= 0) return;
  ++g_launches;
  precond_kernel<<<grid_for(n), 256, 0, s>>>(n, r, diag, theta, eps, t);
}

void launch_diag_extract(const DiagJob* d_jobs, int njobs, int max_rows, cudaStream_t s) {
  if (njobs <= 0 || max_rows <= 0) return;
  for (int o0 = 0; o0 < njobs; o0 += 65535) {
    int no = njobs - o0 < 65535 ? njobs - o0 : 65535;
    dim3 g(grid_for(max_rows, 128, 16), no);
    diag_extract_kernel<<<g, 128, 0, s>>>(d_jobs + o0);
    ++g_launches;
  }
}

bool launch_rr(const double* G, int ldg, int m, double* y, double* scal, cudaStream_t s) {
  if (m < 1 || m > RR_MAX) return false;
  ++g_launches;
  rr_kernel<<<1, 256, 0, s>>>(G, ldg, m, y, scal);
  return true;
}

void launch_resid(long n, const double* hx, const double* x, const double* d_theta, double* r, cudaStream_t s) {
  if (n <= 0) return;
  ++g_launches;
  resid_kernel<<<grid_for(n), 256, 0, s>>>(n, hx, x, d_theta, r);
}

void launch_precond_dev(long n, const double* r, const double* diag, const double* d_theta, double eps, double* t,
                        cudaStream_t s) {
  if (n <= 0) return;
  ++g_launches;
  precond_dev_kernel<<<grid_for(n), 256, 0, s>>>(n, r, diag, d_theta, eps, t);
}

void launch_sub_combine(const double* V, long ldv, int m, const double* d_c, long n, double* t, cudaStream_t s) {
  if (n <= 0 || m <= 0) return;
  ++g_launches;
  sub_combine_kernel<<<grid_for(n), 256, 0, s>>>(V, ldv, m, d_c, n, t);
}

void launch_scale_rsqrt(long n, const double* x, const double* d_nrm2, double* y, cudaStream_t s) {
  if (n <= 0) return;
  ++g_launches;
  scale_rsqrt_kernel<<<grid_for(n), 256, 0, s>>>(n, x, d_nrm2, y);
}

void launch_gcol(const double* dots, int m1, double* G, int ld, int col, cudaStream_t s) {
  ++g_launches;
  gcol_kernel<<<1, 64, 0, s>>>(dots, m1, G, ld, col);
}

void launch_restart_g(double* G, const double* d_theta, const double* d_xn2, cudaStream_t s) {
  ++g_launches;
  restart_g_kernel<<<1, 32, 0, s>>>(G, d_theta, d_xn2);
}

}  // namespace gbdmrg
