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

}  // namespace gbdmrg
