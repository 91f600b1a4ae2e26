// Tensor-core (tcgen05, sm_103a) grouped block GEMM for the mixed-precision
// sigma vector: BF16 operands, FP32 accumulation in tensor memory.
//
// Same work-list model as the FP64 kernel: one CTA computes one 128 x 128 tile
// of one output block, summing over the block's term list (the concatenation
// of the contraction dimension over operator terms and quantum-number
// blocks).  Operands are K-major ("NT": C = sum_t op(A_t B_t^T)) with leading
// dimensions padded to multiples of 8 elements and zero padding, so every
// 16-byte chunk is aligned.  Ragged quantum-number blocks are staged into
// 128B-swizzled shared memory with 16-byte cp.async copies (zero fill outside
// the block) -- per-block TMA tensor maps would be needed for every one of the
// ~10^5 operand blocks otherwise.  One elected thread issues tcgen05.mma
// (M = 128, N = 128, K = 16 per instruction) into a TMEM accumulator; each
// commit arrives on an mbarrier that releases the smem stage.  Every wait is
// bounded: on timeout the kernel records an error and returns after freeing
// its tensor memory.
#include <cuda_bf16.h>

#include <atomic>
#include <cstdint>

#include "kernels_tc.hpp"

namespace gbdmrg {

namespace {

constexpr int TC_M = 128, TC_N = 128, TC_K = 64, TC_STAGES = 3;
constexpr int TC_TILE_BYTES = TC_M * TC_K * 2;  // 16 KB per operand tile (A and B alike)
constexpr int TC_STAGE_BYTES = 2 * TC_TILE_BYTES;
constexpr int TC_SMEM = TC_STAGES * TC_STAGE_BYTES + 1024;
constexpr int TC_THREADS = 128;
constexpr long TC_WAIT_LIMIT = 1L << 22;

// slice pairs (i, j) with i + j < nsl, largest products first
__constant__ int PAIR_I[6] = {0, 0, 1, 0, 1, 2};
__constant__ int PAIR_J[6] = {0, 1, 0, 2, 1, 0};
__device__ __forceinline__ int npairs(int nsl) { return nsl <= 1 ? 1 : (nsl == 2 ? 3 : 6); }

__device__ __forceinline__ uint32_t smem_u32(const void* p) {
  return (uint32_t)__cvta_generic_to_shared(p);
}

// shared-memory matrix descriptor: K-major, 128-byte swizzle, 8-row groups 1024 B apart
__device__ __forceinline__ uint64_t sdesc(uint32_t saddr) {
  uint64_t d = 0;
  d |= (uint64_t)((saddr >> 4) & 0x3FFFu);
  d |= (uint64_t)1 << 16;             // leading byte offset (unused for swizzled K-major)
  d |= (uint64_t)(1024 >> 4) << 32;   // stride byte offset
  d |= (uint64_t)1 << 46;             // descriptor version
  d |= (uint64_t)2 << 61;             // SWIZZLE_128B
  return d;
}

// instruction descriptor: D f32, A/B bf16, both K-major, M = 128, N = 128
__device__ __forceinline__ uint32_t idesc_bf16(bool negA) {
  uint32_t d = 0;
  d |= 1u << 4;                        // D format f32
  d |= 1u << 7;                        // A format bf16
  d |= 1u << 10;                       // B format bf16
  if (negA) d |= 1u << 13;             // negate A
  d |= (uint32_t)(TC_N >> 3) << 17;
  d |= (uint32_t)(TC_M >> 4) << 24;
  return d;
}

__device__ __forceinline__ void cp_async16(uint32_t dst, const void* src, int bytes) {
  asm volatile("cp.async.cg.shared.global [%0], [%1], 16, %2;\n" ::"r"(dst), "l"(src), "r"(bytes));
}
__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;\n" ::); }
template <int N>
__device__ __forceinline__ void cp_async_wait() {
  asm volatile("cp.async.wait_group %0;\n" ::"n"(N));
}

__device__ __forceinline__ bool mbar_wait(uint32_t bar, uint32_t parity) {
  for (long it = 0; it < TC_WAIT_LIMIT; ++it) {
    uint32_t done;
    asm volatile(
        "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n selp.u32 %0, 1, 0, p;\n}\n"
        : "=r"(done)
        : "r"(bar), "r"(parity)
        : "memory");
    if (done) return true;
  }
  return false;
}

// load one 128 x 64 K-major tile (rows r0.., k0..) of a row-major bf16 matrix with
// `rows` valid rows and leading dimension ld (elements); zero fill outside
__device__ __forceinline__ void load_tile(uint32_t sbase, const __nv_bfloat16* M, int ld, int rows, int r0,
                                          int k0) {
  const int tid = threadIdx.x;
#pragma unroll
  for (int q = 0; q < 8; ++q) {
    const int e = tid + TC_THREADS * q;  // 1024 chunks of 16 B
    const int r = e >> 3, c = e & 7;
    const int gr = r0 + r, gk = k0 + 8 * c;
    const bool ok = gr < rows && gk < ld;
    const __nv_bfloat16* src = ok ? M + (long)gr * ld + gk : M;
    const uint32_t dst = sbase + r * 128 + ((c ^ (r & 7)) << 4);
    cp_async16(dst, src, ok ? 16 : 0);
  }
}

__global__ void __launch_bounds__(TC_THREADS, 1)
    gemm_bf16_tc_kernel(const TcTile* __restrict__ tiles, const TcTask* __restrict__ tasks,
                        const TcTerm* __restrict__ terms, int* __restrict__ err) {
  extern __shared__ uint8_t dsm[];
  __shared__ __align__(8) uint64_t bars[TC_STAGES];
  __shared__ uint32_t tmem_base_sh;
  const uint32_t base = (smem_u32(dsm) + 1023u) & ~1023u;
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  const TcTile tl = tiles[blockIdx.x];
  const TcTask tk = tasks[tl.task];

  if (warp == 0) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;\n" ::"r"(
                     smem_u32(&tmem_base_sh)),
                 "r"(TC_N));
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;\n" ::);
  }
  if (tid == 0) {
    for (int s = 0; s < TC_STAGES; ++s) asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;\n" ::"r"(smem_u32(&bars[s])));
    asm volatile("fence.mbarrier_init.release.cluster;\n" ::);
  }
  asm volatile("tcgen05.fence::before_thread_sync;\n" ::);
  __syncthreads();
  asm volatile("tcgen05.fence::after_thread_sync;\n" ::);
  const uint32_t tmem = tmem_base_sh;

  // total number of 64-wide k-steps over the term list (and slice pairs)
  int S = 0;
  for (int t = tk.t0; t < tk.t1; ++t) S += npairs(terms[t].nsl) * ((terms[t].k + TC_K - 1) / TC_K);

  int lt = tk.t0, lp = 0, lk = 0;  // load cursor (term, slice pair, k offset)
  int mt = tk.t0, mp = 0, mk = 0;  // MMA cursor
  auto adv = [&](int& t, int& p, int& k0) {
    k0 += TC_K;
    if (k0 >= terms[t].k) {
      k0 = 0;
      if (++p >= npairs(terms[t].nsl)) { p = 0; ++t; }
    }
  };
  auto issue_load = [&](int stage) {
    const TcTerm tm = terms[lt];
    const uint32_t sa = base + stage * TC_STAGE_BYTES;
    load_tile(sa, tm.A + PAIR_I[lp] * tm.sA, tm.lda, tk.m, tl.r0, lk);
    load_tile(sa + TC_TILE_BYTES, tm.B + PAIR_J[lp] * tm.sB, tm.ldb, tk.n, tl.c0, lk);
    adv(lt, lp, lk);
  };
  bool ok = true;
  for (int j = 0; j < TC_STAGES - 1; ++j) {
    if (j < S) issue_load(j);
    cp_async_commit();
  }
  for (int i = 0; i < S; ++i) {
    const int s = i % TC_STAGES;
    const int j = i + TC_STAGES - 1;
    if (j < S) {
      const int sj = j % TC_STAGES;
      if (i >= 1 && !mbar_wait(smem_u32(&bars[sj]), (uint32_t)(((i - 1) / TC_STAGES) & 1))) ok = false;
      if (ok) issue_load(sj);
    }
    cp_async_commit();
    cp_async_wait<TC_STAGES - 1>();
    asm volatile("fence.proxy.async.shared::cta;\n" ::: "memory");
    ok = __syncthreads_and(ok);
    if (!ok) break;
    if (tid == 0) {
      asm volatile("tcgen05.fence::after_thread_sync;\n" ::);
      const TcTerm tm = terms[mt];
      const uint32_t id = idesc_bf16(tm.flags & 1);
      const uint32_t sa = base + s * TC_STAGE_BYTES;
#pragma unroll
      for (int kk = 0; kk < TC_K / 16; ++kk) {
        const uint64_t ad = sdesc(sa + kk * 32), bd = sdesc(sa + TC_TILE_BYTES + kk * 32);
        const uint32_t acc = (i > 0 || kk > 0) ? 1u : 0u;
        asm volatile(
            "{\n .reg .pred p;\n setp.ne.b32 p, %4, 0;\n"
            " tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n}\n" ::"r"(tmem),
            "l"(ad), "l"(bd), "r"(id), "r"(acc));
      }
      asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];\n" ::"r"(
          smem_u32(&bars[s])));
    }
    adv(mt, mp, mk);
  }
  // all threads agree on `ok` before the final wait
  __syncthreads();
  ok = __syncthreads_and(ok);
  if (ok && S > 0) ok = mbar_wait(smem_u32(&bars[(S - 1) % TC_STAGES]), (uint32_t)(((S - 1) / TC_STAGES) & 1));
  ok = __syncthreads_and(ok);
  asm volatile("tcgen05.fence::after_thread_sync;\n" ::);
  if (ok) {
    // epilogue: warp w owns TMEM lanes (rows) 32w .. 32w+31
    const int row = tl.r0 + warp * 32 + lane;
    for (int c0 = 0; c0 < TC_N; c0 += 32) {
      uint32_t v[32];
      const uint32_t taddr = tmem + ((uint32_t)(warp * 32) << 16) + (uint32_t)c0;
      asm volatile(
          "tcgen05.ld.sync.aligned.32x32b.x32.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15,"
          "%16,%17,%18,%19,%20,%21,%22,%23,%24,%25,%26,%27,%28,%29,%30,%31}, [%32];\n"
          : "=r"(v[0]), "=r"(v[1]), "=r"(v[2]), "=r"(v[3]), "=r"(v[4]), "=r"(v[5]), "=r"(v[6]), "=r"(v[7]),
            "=r"(v[8]), "=r"(v[9]), "=r"(v[10]), "=r"(v[11]), "=r"(v[12]), "=r"(v[13]), "=r"(v[14]),
            "=r"(v[15]), "=r"(v[16]), "=r"(v[17]), "=r"(v[18]), "=r"(v[19]), "=r"(v[20]), "=r"(v[21]),
            "=r"(v[22]), "=r"(v[23]), "=r"(v[24]), "=r"(v[25]), "=r"(v[26]), "=r"(v[27]), "=r"(v[28]),
            "=r"(v[29]), "=r"(v[30]), "=r"(v[31])
          : "r"(taddr));
      asm volatile("tcgen05.wait::ld.sync.aligned;\n" ::: "memory");
      if (row < tk.m) {
#pragma unroll
        for (int j = 0; j < 32; ++j) {
          const int col = tl.c0 + c0 + j;
          if (col >= tk.n) break;
          float x = __uint_as_float(v[j]);
          if (tk.C) {
            float* cp = tk.C + (long)row * tk.ldc + col;
            if (tk.beta) x += *cp;
            *cp = x;
          }
          if (tk.Cb) {
            __nv_bfloat16 h0 = __float2bfloat16_rn(x);
            tk.Cb[(long)row * tk.ldcb + col] = h0;
            if (tk.nslices > 1) {
              const float r1 = x - __bfloat162float(h0);
              __nv_bfloat16 h1 = __float2bfloat16_rn(r1);
              tk.Cb[tk.slice_stride + (long)row * tk.ldcb + col] = h1;
              if (tk.nslices > 2)
                tk.Cb[2 * tk.slice_stride + (long)row * tk.ldcb + col] =
                    __float2bfloat16_rn(r1 - __bfloat162float(h1));
            }
          }
        }
      }
    }
  } else if (tid == 0) {
    atomicExch(err, 1);
  }
  // let in-flight copies land before the CTA exits, then free the tensor memory
  cp_async_wait<0>();
  asm volatile("tcgen05.fence::before_thread_sync;\n" ::);
  __syncthreads();
  if (warp == 0) asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;\n" ::"r"(tmem), "r"(TC_N));
}

std::atomic<long> g_tc_launches{0};

}  // namespace

long tc_launch_count() { return g_tc_launches.load(); }

cudaError_t launch_gemm_bf16_tc(const TcTile* d_tiles, int ntiles, const TcTask* d_tasks, const TcTerm* d_terms,
                                int* d_err, cudaStream_t s) {
  if (ntiles <= 0) return cudaSuccess;
  static bool attr = false;
  if (!attr) {
    cudaError_t e = cudaFuncSetAttribute(gemm_bf16_tc_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, TC_SMEM);
    if (e != cudaSuccess) return e;
    attr = true;
  }
  ++g_tc_launches;
  gemm_bf16_tc_kernel<<<ntiles, TC_THREADS, TC_SMEM, s>>>(d_tiles, d_tasks, d_terms, d_err);
  return cudaGetLastError();
}

}  // namespace gbdmrg
