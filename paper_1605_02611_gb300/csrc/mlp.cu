// Learned Davidson preconditioner: training (FP32 CUDA cores) and inference
// (BF16 hidden layer on the tensor cores) kernels.  The definitions are stated
// in mlp.hpp.
#include <cuda_bf16.h>

#include <algorithm>
#include <cmath>
#include <random>
#include <vector>

#include "mlp.hpp"

namespace gbdmrg {

namespace {

constexpr double PAIR_CLIP = 100.0;
constexpr double DEN_EPS = 1e-8;

// SplitMix64 finaliser (Steele, Lea & Flood, OOPSLA 2014): a counter-based
// hash used to draw sample indices
__host__ __device__ inline uint64_t splitmix64(uint64_t x) {
  uint64_t z = x + 0x9E3779B97F4A7C15ULL;
  z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ULL;
  z = (z ^ (z >> 27)) * 0x94D049BB133111EBULL;
  return z ^ (z >> 31);
}

__device__ __forceinline__ float gelu_f(float x) { return 0.5f * x * (1.0f + erff(x * 0.70710678118654752f)); }

// d/dx [x Phi(x)] = Phi(x) + x phi(x)
__device__ __forceinline__ float gelu_grad_f(float x) {
  return 0.5f * (1.0f + erff(x * 0.70710678118654752f)) + x * expf(-0.5f * x * x) * 0.39894228040143268f;
}

__device__ __forceinline__ bool is_weight(long p) {
  return p < MLP_OFF_B1 || (p >= MLP_OFF_W2 && p < MLP_OFF_B2) || (p >= MLP_OFF_W3 && p < MLP_OFF_B3);
}

__device__ __forceinline__ void quantize_one(long p, const float* w, float* wq, __nv_bfloat16* w2b) {
  const float x = w[p];
  const __nv_bfloat16 b = __float2bfloat16_rn(x);
  wq[p] = is_weight(p) ? __bfloat162float(b) : x;
  if (p >= MLP_OFF_W2 && p < MLP_OFF_B2) w2b[p - MLP_OFF_W2] = b;
}

__global__ void quantize_kernel(const float* __restrict__ w, float* __restrict__ wq, __nv_bfloat16* __restrict__ w2b) {
  for (long p = (long)blockIdx.x * blockDim.x + threadIdx.x; p < MLP_NPARAMS; p += (long)gridDim.x * blockDim.x)
    quantize_one(p, w, wq, w2b);
}

__global__ void adam_kernel(float* __restrict__ w, const float* __restrict__ g, float* __restrict__ m,
                            float* __restrict__ v, float lr, float b1, float b2, float c1, float c2, float eps,
                            float* __restrict__ wq, __nv_bfloat16* __restrict__ w2b) {
  for (long p = (long)blockIdx.x * blockDim.x + threadIdx.x; p < MLP_NPARAMS; p += (long)gridDim.x * blockDim.x) {
    const float gg = g[p];
    const float mm = b1 * m[p] + (1.0f - b1) * gg;
    const float vv = b2 * v[p] + (1.0f - b2) * gg * gg;
    m[p] = mm;
    v[p] = vv;
    w[p] -= lr * (mm / c1) / (sqrtf(vv / c2) + eps);
    quantize_one(p, w, wq, w2b);
  }
}

// C[i, j] (+)= sum_k A[i*as0 + k*as1] B[k*bs0 + j*bs1]; 64 x 64 tiles, 4 x 4 per thread
__global__ void __launch_bounds__(256) sgemm_kernel(int M, int N, int K, const float* __restrict__ A, long as0,
                                                    long as1, const float* __restrict__ B, long bs0, long bs1,
                                                    float* __restrict__ C, long ldc, int accumulate) {
  __shared__ float As[16][68], Bs[16][68];
  const int tx = threadIdx.x & 15, ty = threadIdx.x >> 4;
  const int i0 = blockIdx.y * 64, j0 = blockIdx.x * 64;
  float acc[4][4];
#pragma unroll
  for (int p = 0; p < 4; ++p)
#pragma unroll
    for (int q = 0; q < 4; ++q) acc[p][q] = 0.f;
  const bool a_kfast = as1 == 1, b_jfast = bs1 == 1;
  for (int k0 = 0; k0 < K; k0 += 16) {
    for (int e = threadIdx.x; e < 1024; e += 256) {
      // map consecutive threads to the operand's unit-stride index
      const int ia = a_kfast ? e >> 4 : e & 63, ka = a_kfast ? e & 15 : e >> 6;
      const int gi = i0 + ia, gk = k0 + ka;
      As[ka][ia] = (gi < M && gk < K) ? A[gi * as0 + gk * as1] : 0.f;
      const int jb = b_jfast ? e & 63 : e >> 4, kb = b_jfast ? e >> 6 : e & 15;
      const int gj = j0 + jb, gkb = k0 + kb;
      Bs[kb][jb] = (gj < N && gkb < K) ? B[gkb * bs0 + gj * bs1] : 0.f;
    }
    __syncthreads();
#pragma unroll
    for (int kk = 0; kk < 16; ++kk) {
      float a[4], b[4];
#pragma unroll
      for (int q = 0; q < 4; ++q) {
        a[q] = As[kk][ty * 4 + q];
        b[q] = Bs[kk][tx * 4 + q];
      }
#pragma unroll
      for (int p = 0; p < 4; ++p)
#pragma unroll
        for (int q = 0; q < 4; ++q) acc[p][q] = fmaf(a[p], b[q], acc[p][q]);
    }
    __syncthreads();
  }
#pragma unroll
  for (int p = 0; p < 4; ++p)
#pragma unroll
    for (int q = 0; q < 4; ++q) {
      const int gi = i0 + ty * 4 + p, gj = j0 + tx * 4 + q;
      if (gi < M && gj < N) {
        float* c = C + gi * ldc + gj;
        *c = accumulate ? *c + acc[p][q] : acc[p][q];
      }
    }
}

void sgemm(int M, int N, int K, const float* A, long as0, long as1, const float* B, long bs0, long bs1, float* C,
           long ldc, int accumulate, cudaStream_t s) {
  if (M <= 0 || N <= 0) return;
  dim3 g((N + 63) / 64, (M + 63) / 64);
  sgemm_kernel<<<g, 256, 0, s>>>(M, N, K, A, as0, as1, B, bs0, bs1, C, ldc, accumulate);
  count_launches(1);
}

// A [rows x 256] += bias; H = gelu(A)
__global__ void bias_gelu_kernel(long rows, float* __restrict__ A, const float* __restrict__ bias,
                                 float* __restrict__ H) {
  const long tot = rows * MLP_H;
  for (long e = (long)blockIdx.x * blockDim.x + threadIdx.x; e < tot; e += (long)gridDim.x * blockDim.x) {
    const float a = A[e] + bias[e & (MLP_H - 1)];
    A[e] = a;
    H[e] = gelu_f(a);
  }
}

// g[s] = b3 + W3 . H2[s, :]  (one warp per sample)
__global__ void out_train_kernel(long rows, const float* __restrict__ H2, const float* __restrict__ wq,
                                 float* __restrict__ g) {
  const int lane = threadIdx.x & 31;
  const long nw = (long)gridDim.x * (blockDim.x >> 5);
  for (long s = (long)blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5); s < rows; s += nw) {
    float acc = 0.f;
#pragma unroll
    for (int q = 0; q < 8; ++q) {
      const int j = q * 32 + lane;
      acc = fmaf(wq[MLP_OFF_W3 + j], H2[s * MLP_H + j], acc);
    }
#pragma unroll
    for (int o = 16; o; o >>= 1) acc += __shfl_xor_sync(0xffffffffu, acc, o);
    if (lane == 0) g[s] = acc + wq[MLP_OFF_B3];
  }
}

// e = (1 + g) P - T; g := dL/dg = 2 e P / B; loss += sum e^2 * scale; grad[b3] += sum dg
__global__ void loss_kernel(long rows, float* __restrict__ g, const float* __restrict__ P, const float* __restrict__ T,
                            double scale, double* __restrict__ loss, float* __restrict__ grad) {
  __shared__ double sl[8];
  __shared__ float sg[8];
  double l = 0.0;
  float gs = 0.f;
  for (long s = (long)blockIdx.x * blockDim.x + threadIdx.x; s < rows; s += (long)gridDim.x * blockDim.x) {
    const float e = (1.0f + g[s]) * P[s] - T[s];
    const float dg = 2.0f * e * P[s] / (float)rows;
    g[s] = dg;
    l += (double)e * e;
    gs += dg;
  }
  for (int o = 16; o; o >>= 1) {
    l += __shfl_xor_sync(0xffffffffu, l, o);
    gs += __shfl_xor_sync(0xffffffffu, gs, o);
  }
  const int w = threadIdx.x >> 5, lane = threadIdx.x & 31;
  if (lane == 0) {
    sl[w] = l;
    sg[w] = gs;
  }
  __syncthreads();
  if (threadIdx.x == 0) {
    double L = 0.0;
    float G = 0.f;
    for (int i = 0; i < (int)(blockDim.x >> 5); ++i) {
      L += sl[i];
      G += sg[i];
    }
    atomicAdd(loss, L * scale);
    atomicAdd(grad + MLP_OFF_B3, G);
  }
}

// out[j] += sum_s w[s] X[s, j] (w may be null: plain column sums); 256 threads = columns
__global__ void colsum_kernel(long rows, const float* __restrict__ X, const float* __restrict__ w,
                              float* __restrict__ out) {
  const int j = threadIdx.x;
  const long per = 256;
  float acc = 0.f;
  for (long s0 = (long)blockIdx.x * per; s0 < rows; s0 += (long)gridDim.x * per) {
    const long s1 = s0 + per < rows ? s0 + per : rows;
    for (long s = s0; s < s1; ++s) acc = fmaf(w ? w[s] : 1.0f, X[s * MLP_H + j], acc);
  }
  atomicAdd(out + j, acc);
}

// dA2[s, j] = dg[s] W3[j] gelu'(A2[s, j])
__global__ void da2_kernel(long rows, const float* __restrict__ dg, const float* __restrict__ wq,
                           const float* __restrict__ A2, float* __restrict__ dA2) {
  const long tot = rows * MLP_H;
  for (long e = (long)blockIdx.x * blockDim.x + threadIdx.x; e < tot; e += (long)gridDim.x * blockDim.x) {
    const int j = (int)(e & (MLP_H - 1));
    dA2[e] = dg[e / MLP_H] * wq[MLP_OFF_W3 + j] * gelu_grad_f(A2[e]);
  }
}

// X *= gelu'(A) element-wise
__global__ void gelu_back_kernel(long tot, float* __restrict__ X, const float* __restrict__ A) {
  for (long e = (long)blockIdx.x * blockDim.x + threadIdx.x; e < tot; e += (long)gridDim.x * blockDim.x)
    X[e] *= gelu_grad_f(A[e]);
}

__global__ void gather_kernel(long B, long n, uint64_t key, const float* __restrict__ F, const float* __restrict__ P,
                              const float* __restrict__ T, float* __restrict__ Fb, float* __restrict__ Pb,
                              float* __restrict__ Tb) {
  for (long s = (long)blockIdx.x * blockDim.x + threadIdx.x; s < B; s += (long)gridDim.x * blockDim.x) {
    const long i = (long)(splitmix64(key + (uint64_t)s) % (uint64_t)n);
#pragma unroll
    for (int k = 0; k < MLP_F; ++k) Fb[s * MLP_F + k] = F[i * MLP_F + k];
    Pb[s] = P[i];
    Tb[s] = T[i];
  }
}

// ------------------------------------------------------------ inference

__device__ void features(long i, const double* __restrict__ r, const double* __restrict__ d, double theta, double rn,
                         long n, const long* __restrict__ boff, int nb, const double* __restrict__ bsum,
                         const double* __restrict__ bmean, float* f) {
  int lo = 0, hi = nb - 1;  // the block b with boff[b] <= i < boff[b + 1]
  while (lo < hi) {
    const int mid = (lo + hi + 1) >> 1;
    if (boff[mid] <= i)
      lo = mid;
    else
      hi = mid - 1;
  }
  const double sqn = sqrt((double)n);
  const double delta = d[i] - theta;
  f[0] = (float)(r[i] * sqn / rn);
  f[1] = (float)asinh(delta);
  f[2] = (float)(delta / (delta * delta + 0.01));
  const double sz = (double)(boff[lo + 1] - boff[lo]);
  f[3] = (float)asinh(sqrt(bsum[lo] / sz) * sqn / rn);
  f[4] = (float)asinh(bmean[lo] - theta);
}

__device__ __forceinline__ double diag_correction(double r, double d, double theta) {
  double den = theta - d;
  if (fabs(den) < DEN_EPS) den = den < 0 ? -DEN_EPS : DEN_EPS;
  return r / den;
}

// layer 1 for elements e0 .. e0+ne-1: h1 = gelu(W1 f + b1) stored in BF16 (one warp per element)
template <bool FROM_F>
__global__ void l1_kernel(long e0, long ne, const float* __restrict__ F, const double* __restrict__ r,
                          const double* __restrict__ d, double theta, double rn, long n, const long* __restrict__ boff,
                          int nb, const double* __restrict__ bsum, const double* __restrict__ bmean,
                          const float* __restrict__ wq, __nv_bfloat16* __restrict__ H1) {
  __shared__ float sw1[MLP_F * MLP_H], sb1[MLP_H];  // sw1[k * 256 + j] = W1[j, k]
  for (int e = threadIdx.x; e < MLP_F * MLP_H; e += blockDim.x) {
    const int j = e / MLP_F, k = e % MLP_F;
    sw1[k * MLP_H + j] = wq[MLP_OFF_W1 + e];
  }
  for (int j = threadIdx.x; j < MLP_H; j += blockDim.x) sb1[j] = wq[MLP_OFF_B1 + j];
  __syncthreads();
  const int lane = threadIdx.x & 31;
  const long nw = (long)gridDim.x * (blockDim.x >> 5);
  for (long e = (long)blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5); e < ne; e += nw) {
    float f[MLP_F];
    if (FROM_F) {
#pragma unroll
      for (int k = 0; k < MLP_F; ++k) f[k] = F[(e0 + e) * MLP_F + k];
    } else {
      features(e0 + e, r, d, theta, rn, n, boff, nb, bsum, bmean, f);
    }
#pragma unroll
    for (int q = 0; q < 8; ++q) {
      const int j = q * 32 + lane;
      float a = sb1[j];
#pragma unroll
      for (int k = 0; k < MLP_F; ++k) a = fmaf(sw1[k * MLP_H + j], f[k], a);
      H1[e * MLP_H + j] = __float2bfloat16_rn(gelu_f(a));
    }
  }
}

// layer 3 from the tensor-core output Z = h1 W2^T: g = W3 . gelu(Z + b2) + b3;
// MODE 0 writes g, MODE 1 writes t = (1 + g) r / (theta - d)
template <int MODE>
__global__ void out_kernel(long e0, long ne, const float* __restrict__ Z, const float* __restrict__ wq,
                           const double* __restrict__ r, const double* __restrict__ d, double theta,
                           double* __restrict__ t, float* __restrict__ g, int* __restrict__ flag) {
  __shared__ float sb2[MLP_H], sw3[MLP_H];
  for (int j = threadIdx.x; j < MLP_H; j += blockDim.x) {
    sb2[j] = wq[MLP_OFF_B2 + j];
    sw3[j] = wq[MLP_OFF_W3 + j];
  }
  __syncthreads();
  const float b3 = wq[MLP_OFF_B3];
  const int lane = threadIdx.x & 31;
  const long nw = (long)gridDim.x * (blockDim.x >> 5);
  for (long e = (long)blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5); e < ne; e += nw) {
    float acc = 0.f;
#pragma unroll
    for (int q = 0; q < 8; ++q) {
      const int j = q * 32 + lane;
      acc = fmaf(sw3[j], gelu_f(Z[e * MLP_H + j] + sb2[j]), acc);
    }
#pragma unroll
    for (int o = 16; o; o >>= 1) acc += __shfl_xor_sync(0xffffffffu, acc, o);
    if (lane == 0) {
      const float gg = acc + b3;
      if (MODE == 0) {
        g[e0 + e] = gg;
      } else {
        const long i = e0 + e;
        if (!isfinite(gg)) atomicExch(flag, 1);
        t[i] = (1.0 + (double)gg) * diag_correction(r[i], d[i], theta);
      }
    }
  }
}

// per block: sum of v^2 (mode 0) or mean of v (mode 1)
__global__ void block_reduce_kernel(const double* __restrict__ v, const long* __restrict__ boff, int nb,
                                    double* __restrict__ out, int mode) {
  __shared__ double sh[8];
  for (int b = blockIdx.x; b < nb; b += gridDim.x) {
    const long o0 = boff[b], o1 = boff[b + 1];
    double s = 0.0;
    for (long e = o0 + threadIdx.x; e < o1; e += blockDim.x) {
      const double x = v[e];
      s += mode == 0 ? x * x : x;
    }
    for (int o = 16; o; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
    if ((threadIdx.x & 31) == 0) sh[threadIdx.x >> 5] = s;
    __syncthreads();
    if (threadIdx.x == 0) {
      double S = 0.0;
      for (int i = 0; i < (int)(blockDim.x >> 5); ++i) S += sh[i];
      out[b] = mode == 0 ? S : (o1 > o0 ? S / (double)(o1 - o0) : 0.0);
    }
    __syncthreads();
  }
}

__global__ void dot_kernel(long n, const double* __restrict__ a, const double* __restrict__ b,
                           double* __restrict__ out) {
  __shared__ double sh[8];
  double s = 0.0;
  for (long e = (long)blockIdx.x * blockDim.x + threadIdx.x; e < n; e += (long)gridDim.x * blockDim.x)
    s += a[e] * b[e];
  for (int o = 16; o; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
  if ((threadIdx.x & 31) == 0) sh[threadIdx.x >> 5] = s;
  __syncthreads();
  if (threadIdx.x == 0) {
    double S = 0.0;
    for (int i = 0; i < (int)(blockDim.x >> 5); ++i) S += sh[i];
    atomicAdd(out, S);
  }
}

__global__ void tau_kernel(long n, const double* __restrict__ psi, double inv_c, const double* __restrict__ x,
                           double* __restrict__ tau) {
  for (long e = (long)blockIdx.x * blockDim.x + threadIdx.x; e < n; e += (long)gridDim.x * blockDim.x)
    tau[e] = psi[e] * inv_c - x[e];
}

__global__ void pairs_kernel(long ns, uint64_t seed, long n, const double* __restrict__ r, const double* __restrict__ d,
                             double theta, double rn, const long* __restrict__ boff, int nb,
                             const double* __restrict__ bsum, const double* __restrict__ bmean,
                             const double* __restrict__ tau, double sc, float* __restrict__ F, float* __restrict__ P,
                             float* __restrict__ T, long* __restrict__ idx) {
  for (long q = (long)blockIdx.x * blockDim.x + threadIdx.x; q < ns; q += (long)gridDim.x * blockDim.x) {
    const long i = (long)(splitmix64(seed + (uint64_t)q) % (uint64_t)n);
    float f[MLP_F];
    features(i, r, d, theta, rn, n, boff, nb, bsum, bmean, f);
#pragma unroll
    for (int k = 0; k < MLP_F; ++k) F[q * MLP_F + k] = f[k];
    P[q] = (float)fmin(PAIR_CLIP, fmax(-PAIR_CLIP, diag_correction(r[i], d[i], theta) * sc));
    T[q] = (float)fmin(PAIR_CLIP, fmax(-PAIR_CLIP, tau[i] * sc));
    if (idx) idx[q] = i;
  }
}

inline int blocks_for(long n, int threads = 256, int cap = 4096) {
  long b = (n + threads - 1) / threads;
  return (int)std::max<long>(1, std::min<long>(b, cap));
}

}  // namespace

// ------------------------------------------------------------ host side

Mlp::~Mlp() {
  // the arrays are freed on the network's stream: release them before it goes
  for (DArr<float>* a : {&w, &wq, &grad, &am, &av, &Fb, &Pb, &Tb, &A1, &H1, &A2, &H2, &G, &dA2, &dH1}) a->release();
  w2b.release();
  err.release();
  acc.release();
  if (stream) cudaStreamSynchronize(stream);
  if (own_stream && stream) cudaStreamDestroy(stream);
}

void MlpScratchDeleter::operator()(MlpScratch* p) const { delete p; }

static void mlp_requantize(Mlp& m) {
  quantize_kernel<<<blocks_for(MLP_NPARAMS), 256, 0, m.stream>>>(m.w.p, m.wq.p, m.w2b.p);
  count_launches(1);
  cuda_check(cudaGetLastError(), "quantize");
}

void mlp_init(Mlp& m, uint64_t seed, cudaStream_t s) {
  if (!s) {
    cuda_check(cudaStreamCreateWithFlags(&m.stream, cudaStreamNonBlocking), "stream create");
    m.own_stream = true;
  } else {
    m.stream = s;
  }
  std::vector<float> h(MLP_NPARAMS, 0.0f);
  std::mt19937_64 rng(seed);
  std::normal_distribution<float> n1(0.0f, 1.0f / std::sqrt((float)MLP_F)), n2(0.0f, 1.0f / std::sqrt((float)MLP_H));
  for (long p = MLP_OFF_W1; p < MLP_OFF_B1; ++p) h[p] = n1(rng);
  for (long p = MLP_OFF_W2; p < MLP_OFF_B2; ++p) h[p] = n2(rng);
  // W3 = 0, b3 = 0: the untrained network is the diagonal preconditioner
  m.w.alloc(MLP_NPARAMS, m.stream);
  m.wq.alloc(MLP_NPARAMS, m.stream);
  m.w2b.alloc((size_t)MLP_H * MLP_H, m.stream);
  m.grad.alloc(MLP_NPARAMS, m.stream);
  m.am.alloc(MLP_NPARAMS, m.stream);
  m.av.alloc(MLP_NPARAMS, m.stream);
  m.err.alloc(1, m.stream);
  m.acc.alloc(4, m.stream);
  cuda_check(cudaMemsetAsync(m.err.p, 0, sizeof(int), m.stream), "memset");
  mlp_set_params(m, h.data());
}

void mlp_set_params(Mlp& m, const float* host) {
  cuda_check(cudaMemcpyAsync(m.w.p, host, MLP_NPARAMS * sizeof(float), cudaMemcpyHostToDevice, m.stream), "h2d");
  cuda_check(cudaMemsetAsync(m.am.p, 0, MLP_NPARAMS * sizeof(float), m.stream), "memset");
  cuda_check(cudaMemsetAsync(m.av.p, 0, MLP_NPARAMS * sizeof(float), m.stream), "memset");
  m.adam_t = 0;
  mlp_requantize(m);
  cuda_check(cudaStreamSynchronize(m.stream), "sync");
}

void mlp_get_params(Mlp& m, float* host) {
  cuda_check(cudaMemcpyAsync(host, m.w.p, MLP_NPARAMS * sizeof(float), cudaMemcpyDeviceToHost, m.stream), "d2h");
  cuda_check(cudaStreamSynchronize(m.stream), "sync");
}

static void ensure_cap(Mlp& m, long B) {
  if (B <= m.cap) return;
  m.cap = B;
  m.Fb.alloc((size_t)B * MLP_F, m.stream);
  m.Pb.alloc(B, m.stream);
  m.Tb.alloc(B, m.stream);
  m.A1.alloc((size_t)B * MLP_H, m.stream);
  m.H1.alloc((size_t)B * MLP_H, m.stream);
  m.A2.alloc((size_t)B * MLP_H, m.stream);
  m.H2.alloc((size_t)B * MLP_H, m.stream);
  m.G.alloc(B, m.stream);
  m.dA2.alloc((size_t)B * MLP_H, m.stream);
  m.dH1.alloc((size_t)B * MLP_H, m.stream);
}

// FP32 forward of the training numerics: A1, H1, A2, H2 and g (into m.G)
static void forward_f32(Mlp& m, const float* F, long B) {
  cudaStream_t s = m.stream;
  const float* wq = m.wq.p;
  sgemm((int)B, MLP_H, MLP_F, F, MLP_F, 1, wq + MLP_OFF_W1, 1, MLP_F, m.A1.p, MLP_H, 0, s);
  bias_gelu_kernel<<<blocks_for(B * MLP_H), 256, 0, s>>>(B, m.A1.p, wq + MLP_OFF_B1, m.H1.p);
  sgemm((int)B, MLP_H, MLP_H, m.H1.p, MLP_H, 1, wq + MLP_OFF_W2, 1, MLP_H, m.A2.p, MLP_H, 0, s);
  bias_gelu_kernel<<<blocks_for(B * MLP_H), 256, 0, s>>>(B, m.A2.p, wq + MLP_OFF_B2, m.H2.p);
  out_train_kernel<<<blocks_for(B * 32), 256, 0, s>>>(B, m.H2.p, wq, m.G.p);
  count_launches(3);
  cuda_check(cudaGetLastError(), "mlp forward");
}

// forward + backward of one batch (already in F, P, T); gradient into m.grad,
// loss * scale added to *loss_acc
static void step_grad(Mlp& m, const float* F, const float* P, const float* T, long B, double scale,
                      double* loss_acc) {
  cudaStream_t s = m.stream;
  const float* wq = m.wq.p;
  float* gr = m.grad.p;
  cuda_check(cudaMemsetAsync(gr, 0, MLP_NPARAMS * sizeof(float), s), "memset");
  forward_f32(m, F, B);
  loss_kernel<<<blocks_for(B, 256, 1024), 256, 0, s>>>(B, m.G.p, P, T, scale, loss_acc, gr);
  const int cs = (int)std::min<long>((B + 255) / 256, 1024);
  colsum_kernel<<<cs, 256, 0, s>>>(B, m.H2.p, m.G.p, gr + MLP_OFF_W3);
  da2_kernel<<<blocks_for(B * MLP_H), 256, 0, s>>>(B, m.G.p, wq, m.A2.p, m.dA2.p);
  colsum_kernel<<<cs, 256, 0, s>>>(B, m.dA2.p, nullptr, gr + MLP_OFF_B2);
  count_launches(4);
  // dW2[j, k] = sum_s dA2[s, j] H1[s, k]
  sgemm(MLP_H, MLP_H, (int)B, m.dA2.p, 1, MLP_H, m.H1.p, MLP_H, 1, gr + MLP_OFF_W2, MLP_H, 0, s);
  // dH1[s, k] = sum_j dA2[s, j] W2[j, k]
  sgemm((int)B, MLP_H, MLP_H, m.dA2.p, MLP_H, 1, wq + MLP_OFF_W2, MLP_H, 1, m.dH1.p, MLP_H, 0, s);
  gelu_back_kernel<<<blocks_for(B * MLP_H), 256, 0, s>>>(B * MLP_H, m.dH1.p, m.A1.p);
  colsum_kernel<<<cs, 256, 0, s>>>(B, m.dH1.p, nullptr, gr + MLP_OFF_B1);
  count_launches(2);
  // dW1[j, k] = sum_s dA1[s, j] F[s, k]
  sgemm(MLP_H, MLP_F, (int)B, m.dH1.p, 1, MLP_H, F, MLP_F, 1, gr + MLP_OFF_W1, MLP_F, 0, s);
  cuda_check(cudaGetLastError(), "mlp backward");
}

double mlp_loss_grad(Mlp& m, const float* F, const float* P, const float* T, long n) {
  if (n <= 0) throw Error(ST_EINVAL, "no samples");
  ensure_cap(m, n);
  cuda_check(cudaMemsetAsync(m.acc.p, 0, sizeof(double), m.stream), "memset");
  step_grad(m, F, P, T, n, 1.0 / (double)n, m.acc.p);
  double L = 0;
  cuda_check(cudaMemcpyAsync(&L, m.acc.p, sizeof(double), cudaMemcpyDeviceToHost, m.stream), "d2h");
  cuda_check(cudaStreamSynchronize(m.stream), "sync");
  return L;
}

void mlp_forward(Mlp& m, const float* F, long n, float* g, bool inference) {
  if (n <= 0) return;
  cudaStream_t s = m.stream;
  if (!inference) {
    ensure_cap(m, n);
    forward_f32(m, F, n);
    cuda_check(cudaMemcpyAsync(g, m.G.p, n * sizeof(float), cudaMemcpyDeviceToDevice, s), "d2d");
    cuda_check(cudaStreamSynchronize(s), "sync");
    return;
  }
  // inference numerics on given features: BF16 h1, tensor-core layer 2
  DArr<__nv_bfloat16> H1;
  DArr<float> Z;
  H1.alloc((size_t)n * MLP_H, s);
  Z.alloc((size_t)n * MLP_H, s);
  std::vector<TcTile> tiles;
  for (long r0 = 0; r0 < n; r0 += TC_TILE_M)
    for (int c0 = 0; c0 < MLP_H; c0 += TC_TILE_N) tiles.push_back({0, (int)r0, c0});
  std::vector<TcTask> tasks(1);
  tasks[0] = {Z.p, nullptr, 0, MLP_H, 0, (int)n, MLP_H, 0, 1, 0, 0, 1};
  std::vector<TcTerm> terms(1);
  terms[0] = {H1.p, m.w2b.p, 0, 0, MLP_H, MLP_H, MLP_H, 0, 1};
  DArr<TcTile> dt;
  DArr<TcTask> dk;
  DArr<TcTerm> dm;
  dt.upload(tiles, s);
  dk.upload(tasks, s);
  dm.upload(terms, s);
  l1_kernel<true><<<blocks_for(n * 32), 256, 0, s>>>(0, n, F, nullptr, nullptr, 0, 1, n, nullptr, 0, nullptr,
                                                     nullptr, m.wq.p, H1.p);
  count_launches(1);
  cuda_check(launch_gemm_bf16_tc(dt.p, (int)tiles.size(), dk.p, dm.p, m.err.p, s), "tc layer 2");
  out_kernel<0><<<blocks_for(n * 32), 256, 0, s>>>(0, n, Z.p, m.wq.p, nullptr, nullptr, 0, nullptr, g, nullptr);
  count_launches(1);
  cuda_check(cudaGetLastError(), "mlp inference");
  int h = 0;
  cuda_check(cudaMemcpyAsync(&h, m.err.p, sizeof(int), cudaMemcpyDeviceToHost, s), "d2h");
  cuda_check(cudaStreamSynchronize(s), "sync");
  if (h) throw Error(ST_ETIMEOUT, "tensor-core GEMM: a bounded wait ran out");
}

void mlp_train(Mlp& m, const float* F, const float* P, const float* T, long n, int epochs, int batch, float lr,
               uint64_t seed, double* first, double* last) {
  if (n <= 0 || epochs <= 0 || batch <= 0) throw Error(ST_EINVAL, "mlp_train: empty data or schedule");
  ensure_cap(m, batch);
  cudaStream_t s = m.stream;
  const long spe = (n + batch - 1) / batch;  // steps per epoch
  cuda_check(cudaMemsetAsync(m.acc.p, 0, 4 * sizeof(double), s), "memset");
  const float b1 = 0.9f, b2 = 0.999f, eps = 1e-8f;
  for (int ep = 0; ep < epochs; ++ep) {
    double* lacc = m.acc.p + (ep == 0 ? 0 : ep == epochs - 1 ? 1 : 2);
    for (long st = 0; st < spe; ++st) {
      const uint64_t key = splitmix64(seed + (uint64_t)(ep * spe + st));
      gather_kernel<<<blocks_for(batch), 256, 0, s>>>(batch, n, key, F, P, T, m.Fb.p, m.Pb.p, m.Tb.p);
      count_launches(1);
      step_grad(m, m.Fb.p, m.Pb.p, m.Tb.p, batch, 1.0 / ((double)batch * (double)spe), lacc);
      ++m.adam_t;
      const float c1 = 1.0f - std::pow(b1, (float)m.adam_t), c2 = 1.0f - std::pow(b2, (float)m.adam_t);
      adam_kernel<<<blocks_for(MLP_NPARAMS), 256, 0, s>>>(m.w.p, m.grad.p, m.am.p, m.av.p, lr, b1, b2, c1, c2, eps,
                                                          m.wq.p, m.w2b.p);
      count_launches(1);
    }
  }
  cuda_check(cudaGetLastError(), "mlp train");
  double h[2];
  cuda_check(cudaMemcpyAsync(h, m.acc.p, 2 * sizeof(double), cudaMemcpyDeviceToHost, s), "d2h");
  cuda_check(cudaStreamSynchronize(s), "sync");
  if (first) *first = h[0];
  if (last) *last = epochs == 1 ? h[0] : h[1];
}

// ------------------------------------------------------------ per-problem scratch

void mlp_scratch_build(MlpScratch& s, const Mlp* m, const PsiLayout& P, cudaStream_t st) {
  s.n = P.nnz;
  s.nb = (int)P.blocks.size();
  std::vector<long> off(s.nb + 1);
  for (int b = 0; b < s.nb; ++b) off[b] = P.blocks[b].off;
  off[s.nb] = P.nnz;
  s.boff.upload(off, st);
  s.bsum.alloc(std::max(1, s.nb), st);
  s.bmean.alloc(std::max(1, s.nb), st);
  s.flag.alloc(1, st);
  if (!m || s.n == 0) {
    cuda_check(cudaStreamSynchronize(st), "sync");
    return;
  }
  s.chunk = std::min<long>(s.n, 1L << 19);
  s.H1.alloc((size_t)s.chunk * MLP_H, st);
  s.Z.alloc((size_t)s.chunk * MLP_H, st);
  const long last = s.n - (s.n - 1) / s.chunk * s.chunk;  // rows of the last chunk
  std::vector<TcTile> tiles;
  for (long r0 = 0; r0 < s.chunk; r0 += TC_TILE_M)
    for (int c0 = 0; c0 < MLP_H; c0 += TC_TILE_N) tiles.push_back({0, (int)r0, c0});
  s.ntiles_full = (int)tiles.size();
  for (long r0 = 0; r0 < last; r0 += TC_TILE_M)
    for (int c0 = 0; c0 < MLP_H; c0 += TC_TILE_N) tiles.push_back({1, (int)r0, c0});
  s.ntiles_last = (int)tiles.size() - s.ntiles_full;
  std::vector<TcTask> tasks(2);
  tasks[0] = {s.Z.p, nullptr, 0, MLP_H, 0, (int)s.chunk, MLP_H, 0, 1, 0, 0, 1};
  tasks[1] = {s.Z.p, nullptr, 0, MLP_H, 0, (int)last, MLP_H, 0, 1, 0, 0, 1};
  std::vector<TcTerm> terms(1);
  terms[0] = {s.H1.p, m->w2b.p, 0, 0, MLP_H, MLP_H, MLP_H, 0, 1};
  s.tiles.upload(tiles, st);
  s.tasks.upload(tasks, st);
  s.terms.upload(terms, st);
  cuda_check(cudaStreamSynchronize(st), "sync");
}

void mlp_scratch_set_diag(MlpScratch& s, const double* d, cudaStream_t st) {
  if (s.nb == 0) return;
  block_reduce_kernel<<<std::min(s.nb, 4096), 256, 0, st>>>(d, s.boff.p, s.nb, s.bmean.p, 1);
  count_launches(1);
  cuda_check(cudaGetLastError(), "block mean");
}

bool mlp_precondition(Mlp& m, MlpScratch& s, const double* r, const double* d, double theta, double rnorm, double* t,
                      cudaStream_t st) {
  if (s.n == 0) return true;
  if (s.chunk == 0) throw Error(ST_ESTATE, "learned preconditioner: scratch built without the network");
  block_reduce_kernel<<<std::min(s.nb, 4096), 256, 0, st>>>(r, s.boff.p, s.nb, s.bsum.p, 0);
  count_launches(1);
  cuda_check(cudaMemsetAsync(s.flag.p, 0, sizeof(int), st), "memset");
  for (long c0 = 0; c0 < s.n; c0 += s.chunk) {
    const long ne = std::min(s.chunk, s.n - c0);
    const bool lastc = c0 + s.chunk >= s.n;
    l1_kernel<false><<<blocks_for(ne * 32), 256, 0, st>>>(c0, ne, nullptr, r, d, theta, rnorm, s.n, s.boff.p, s.nb,
                                                          s.bsum.p, s.bmean.p, m.wq.p, s.H1.p);
    count_launches(1);
    const TcTile* tl = s.tiles.p + (lastc ? s.ntiles_full : 0);
    const int nt = lastc ? s.ntiles_last : s.ntiles_full;
    cuda_check(launch_gemm_bf16_tc(tl, nt, s.tasks.p, s.terms.p, m.err.p, st), "tc layer 2");
    out_kernel<1><<<blocks_for(ne * 32), 256, 0, st>>>(c0, ne, s.Z.p, m.wq.p, r, d, theta, t, nullptr, s.flag.p);
    count_launches(1);
  }
  cuda_check(cudaGetLastError(), "mlp precondition");
  int h[2] = {0, 0};
  cuda_check(cudaMemcpyAsync(&h[0], s.flag.p, sizeof(int), cudaMemcpyDeviceToHost, st), "d2h");
  cuda_check(cudaMemcpyAsync(&h[1], m.err.p, sizeof(int), cudaMemcpyDeviceToHost, st), "d2h");
  cuda_check(cudaStreamSynchronize(st), "sync");
  if (h[1]) throw Error(ST_ETIMEOUT, "tensor-core GEMM: a bounded wait ran out");
  return h[0] == 0;
}

long mlp_make_pairs(MlpScratch& s, const double* x, const double* r, const double* d, double theta, double rnorm,
                    const double* psi, long ns, uint64_t seed, float* F, float* P, float* T, long* idx,
                    double min_overlap, cudaStream_t st) {
  if (ns <= 0 || s.n == 0) return 0;
  if ((long)s.tmp.n < s.n) s.tmp.alloc(s.n, st);
  DArr<double> dd;
  dd.alloc(2, st);
  cuda_check(cudaMemsetAsync(dd.p, 0, 2 * sizeof(double), st), "memset");
  dot_kernel<<<blocks_for(s.n, 256, 1024), 256, 0, st>>>(s.n, x, psi, dd.p);
  count_launches(1);
  double c = 0;
  cuda_check(cudaMemcpyAsync(&c, dd.p, sizeof(double), cudaMemcpyDeviceToHost, st), "d2h");
  cuda_check(cudaStreamSynchronize(st), "sync");
  if (!(std::fabs(c) > 0) || std::fabs(c) < min_overlap) return 0;
  tau_kernel<<<blocks_for(s.n), 256, 0, st>>>(s.n, psi, 1.0 / c, x, s.tmp.p);
  dot_kernel<<<blocks_for(s.n, 256, 1024), 256, 0, st>>>(s.n, s.tmp.p, s.tmp.p, dd.p + 1);
  block_reduce_kernel<<<std::min(s.nb, 4096), 256, 0, st>>>(r, s.boff.p, s.nb, s.bsum.p, 0);
  count_launches(3);
  double tn2 = 0;
  cuda_check(cudaMemcpyAsync(&tn2, dd.p + 1, sizeof(double), cudaMemcpyDeviceToHost, st), "d2h");
  cuda_check(cudaStreamSynchronize(st), "sync");
  if (!(tn2 > 0)) return 0;
  const double sc = std::sqrt((double)s.n) / std::sqrt(tn2);
  pairs_kernel<<<blocks_for(ns), 256, 0, st>>>(ns, seed, s.n, r, d, theta, rnorm, s.boff.p, s.nb, s.bsum.p,
                                               s.bmean.p, s.tmp.p, sc, F, P, T, idx);
  count_launches(1);
  cuda_check(cudaGetLastError(), "pairs");
  cuda_check(cudaStreamSynchronize(st), "sync");
  return ns;
}

}  // namespace gbdmrg
