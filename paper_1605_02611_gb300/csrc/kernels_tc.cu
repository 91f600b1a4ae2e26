// Tensor-core (tcgen05, sm_103a) grouped block GEMM for the mixed-precision
// sigma vector: BF16 operands, FP32 accumulation in tensor memory.
//
// Same work-list model as the FP64 kernel: an output tile (128 rows x up to 128
// columns) of one output block is the sum over the block's term list (the
// concatenation of the contraction dimension over operator terms and
// quantum-number blocks).  Operands are K-major (C = sum_t A_t B_t^T) with
// leading dimensions padded to multiples of 8 elements and zero padding, so
// every 16-byte chunk is aligned.  The ragged quantum-number blocks are staged
// into 128B-swizzled shared memory with 16-byte cp.async copies (zero fill
// outside the block): one tensor map per operand block would otherwise be
// needed for ~10^5 small blocks.
//
// Persistent and warp-specialised: each CTA walks a strided sequence of tiles.
//   warps 4-7  producers: cp.async into a 3-stage ring; a stage's full barrier
//              completes through cp.async.mbarrier.arrive when the copies land
//              (producers never wait for data); they also publish each stage's
//              MMA parameters in shared memory, so the issuing thread never
//              waits on a global load
//   warp 8     one thread issues tcgen05.mma (M = 128, N = tile width rounded
//              up to 16, K = 16 per instruction; instructions past the
//              term's K are skipped) into one of two TMEM accumulators and
//              commits to the stage's empty barrier / the accumulator's full
//              barrier
//   warps 0-3  epilogue: tcgen05.ld of their 32 TMEM lanes, FP32 store (plain
//              or +=) and/or BF16 slices, row-major or transposed; then
//              release the accumulator
// The two accumulators let the epilogue of one tile overlap the MMAs of the
// next.  Every wait is bounded: on timeout the CTA raises a shared abort flag,
// records an error, drains its copies, frees its tensor memory and returns.
#include <cuda_bf16.h>

#include <atomic>
#include <cstdint>

#include "kernels_tc.hpp"

namespace gbdmrg {

namespace {

constexpr int TC_M = 128, TC_NMAX = 128, TC_K = 64, TC_STAGES = 3;
constexpr int TC_TILE_BYTES = TC_M * TC_K * 2;  // 16 KB per operand tile
// epilogue staging for transposed BF16 stores: per epilogue warp a 32 x 32 block,
// rows padded to 40 elements (80 B) against bank conflicts
constexpr int TC_EPI_LD = 40;
constexpr int TC_EPI_BYTES = 4 * 32 * TC_EPI_LD * 2;

// With three slices a stage holds every BF16 slice of both operands for one
// 64-wide K step, so each loaded slice serves all the slice products it takes
// part in (six products from six tiles instead of twelve), at two stages and
// one CTA per SM.  With one or two slices a stage holds one A and one B slice
// (one slice pair), three stages, two CTAs per SM: measured faster for two
// slices, where reuse saves only a third of the loads but halves the CTAs.
template <int NSL>
struct TcCfg {
  static constexpr bool REUSE = NSL == 3;
  static constexpr int SLOTS = REUSE ? NSL : 1;  // slices of each operand per stage
  static constexpr int STAGES = REUSE ? 2 : 3;
  static constexpr int STAGE_BYTES = SLOTS * 2 * TC_TILE_BYTES;
  static constexpr int SMEM = STAGES * STAGE_BYTES + 1024 + TC_EPI_BYTES;
  static constexpr int CTAS_PER_SM = REUSE ? 1 : 2;
  // one CTA per SM owns all 512 TMEM columns: four accumulators let the MMAs run
  // up to three tiles ahead of the epilogue; two CTAs per SM share them (two each)
  static constexpr int NACC = REUSE ? 4 : 2;
  static constexpr int TMEM_COLS = NACC * TC_NMAX;
};
constexpr int TC_THREADS = 288;
constexpr int TC_PRODUCERS = 128;  // warps 4-7
constexpr int TC_MAXACC = 4;  // tensor-memory accumulators of 128 columns (at most)
constexpr long TC_WAIT_LIMIT = 1L << 24;

// slice pairs (i, j) with i + j < nsl, largest products first
__constant__ int PAIR_I[6] = {0, 0, 1, 0, 1, 2};
__constant__ int PAIR_J[6] = {0, 1, 0, 2, 1, 0};
__device__ __forceinline__ int npairs(int nsl) { return nsl <= 1 ? 1 : (nsl == 2 ? 3 : 6); }

__device__ __forceinline__ uint32_t smem_u32(const void* p) { return (uint32_t)__cvta_generic_to_shared(p); }

// shared-memory matrix descriptor: K-major, 128-byte swizzle, 8-row groups 1024 B apart
__device__ __forceinline__ uint64_t sdesc(uint32_t saddr) {
  uint64_t d = 0;
  d |= (uint64_t)((saddr >> 4) & 0x3FFFu);
  d |= (uint64_t)1 << 16;            // leading byte offset (unused for swizzled K-major)
  d |= (uint64_t)(1024 >> 4) << 32;  // stride byte offset
  d |= (uint64_t)1 << 46;            // descriptor version
  d |= (uint64_t)2 << 61;            // SWIZZLE_128B
  return d;
}

// instruction descriptor: D f32, A/B bf16, both K-major, M = 128, N = n
__device__ __forceinline__ uint32_t idesc_bf16(int n, bool negA) {
  uint32_t d = 0;
  d |= 1u << 4;   // D format f32
  d |= 1u << 7;   // A format bf16
  d |= 1u << 10;  // B format bf16
  if (negA) d |= 1u << 13;
  d |= (uint32_t)(n >> 3) << 17;
  d |= (uint32_t)(TC_M >> 4) << 24;
  return d;
}

__device__ __forceinline__ void cp_async16(uint32_t dst, const void* src, int bytes) {
  asm volatile("cp.async.cg.shared.global [%0], [%1], 16, %2;\n" ::"r"(dst), "l"(src), "r"(bytes));
}
template <int N>
__device__ __forceinline__ void cp_async_wait() {
  asm volatile("cp.async.wait_group %0;\n" ::"n"(N));
}

__device__ __forceinline__ void mbar_init(uint64_t* b, int count) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;\n" ::"r"(smem_u32(b)), "r"(count));
}
__device__ __forceinline__ void mbar_arrive(uint64_t* b) {
  asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];\n" ::"r"(smem_u32(b)) : "memory");
}
// bounded parity wait; gives up when the CTA-wide abort flag is raised
__device__ __forceinline__ bool mbar_wait(uint64_t* b, uint32_t parity, volatile int* abort_flag) {
  const uint32_t a = smem_u32(b);
  for (long it = 0; it < TC_WAIT_LIMIT; ++it) {
    uint32_t done;
    asm volatile(
        "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n selp.u32 %0, 1, 0, p;\n}\n"
        : "=r"(done)
        : "r"(a), "r"(parity)
        : "memory");
    if (done) return true;
    if ((it & 1023) == 1023 && *abort_flag) return false;
  }
  *abort_flag = 1;
  return false;
}

__device__ __forceinline__ int round16(int x) { return (x + 15) & ~15; }

// four FP32 atomic adds in one vector reduction (16-byte aligned address)
__device__ __forceinline__ void red_add_v4(float* p, uint32_t a, uint32_t b, uint32_t c, uint32_t d) {
  asm volatile("red.relaxed.gpu.global.add.v4.f32 [%0], {%1, %2, %3, %4};\n" ::"l"(p), "f"(__uint_as_float(a)),
               "f"(__uint_as_float(b)), "f"(__uint_as_float(c)), "f"(__uint_as_float(d))
               : "memory");
}

// BF16 slice s of x: x = s0 + s1 + s2 + O(2^-24 |x|)
__device__ __forceinline__ __nv_bfloat16 bf16_slice(float x, int s) {
  const __nv_bfloat16 h0 = __float2bfloat16_rn(x);
  if (s == 0) return h0;
  const float r1 = x - __bfloat162float(h0);
  const __nv_bfloat16 h1 = __float2bfloat16_rn(r1);
  if (s == 1) return h1;
  return __float2bfloat16_rn(r1 - __bfloat162float(h1));
}

// `nrows` rows of a 64-K tile (rows r0.., k0..) of a row-major bf16 matrix with
// `rows` valid rows, leading dimension ld and contraction length k; 16-byte
// chunks that start at or beyond k (or ld) are zero-filled without a read, so
// nothing past the block's own padded columns is touched
__device__ __forceinline__ void load_tile(uint32_t sbase, const __nv_bfloat16* M, int ld, int k, int rows, int r0,
                                          int k0, int nrows, int ptid) {
  const int nchunks = nrows * 8;
  const int kend = k < ld ? k : ld;
  for (int e = ptid; e < nchunks; e += TC_PRODUCERS) {
    const int r = e >> 3, c = e & 7;
    const int gr = r0 + r, gk = k0 + 8 * c;
    const bool ok = gr < rows && gk < kend;
    const __nv_bfloat16* src = ok ? M + (long)gr * ld + gk : M;
    cp_async16(sbase + r * 128 + ((c ^ (r & 7)) << 4), src, ok ? 16 : 0);
  }
}

template <int NSL>
__global__ void __launch_bounds__(TC_THREADS, 2)
    gemm_bf16_tc_kernel(const TcTile* __restrict__ tiles, int ntiles, const TcTask* __restrict__ tasks,
                        const TcTerm* __restrict__ terms, int* __restrict__ err) {
  constexpr int S = TcCfg<NSL>::STAGES;
  constexpr int STAGE_BYTES = TcCfg<NSL>::STAGE_BYTES;
  constexpr bool REUSE = TcCfg<NSL>::REUSE;
  constexpr int SLOTS = TcCfg<NSL>::SLOTS;
  extern __shared__ uint8_t dsm[];
  constexpr int NACC = TcCfg<NSL>::NACC;
  __shared__ __align__(8) uint64_t full_b[TC_STAGES], empty_b[TC_STAGES], tfull_b[TC_MAXACC], tempty_b[TC_MAXACC];
  __shared__ uint32_t tmem_base_sh;
  __shared__ int abort_sh;
  // per stage: instruction descriptor, number of K=16 steps, first/last k-step of the tile
  __shared__ uint32_t meta_id[TC_STAGES];
  __shared__ int meta_nk[TC_STAGES], meta_np[TC_STAGES], meta_first[TC_STAGES], meta_last[TC_STAGES];
  const uint32_t base = (smem_u32(dsm) + 1023u) & ~1023u;
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  __nv_bfloat16* const epi = reinterpret_cast<__nv_bfloat16*>(dsm + (base - smem_u32(dsm)) + S * STAGE_BYTES);

  if (warp == 0) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;\n" ::"r"(smem_u32(&tmem_base_sh)),
                 "r"(TcCfg<NSL>::TMEM_COLS));
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;\n" ::);
  }
  if (tid == 32) {
    for (int s = 0; s < S; ++s) {
      mbar_init(&full_b[s], TC_PRODUCERS + 1);  // async copy arrivals + the metadata writer
      mbar_init(&empty_b[s], 1);
    }
    for (int a = 0; a < NACC; ++a) {
      mbar_init(&tfull_b[a], 1);
      mbar_init(&tempty_b[a], 128);
    }
    abort_sh = 0;
    asm volatile("fence.mbarrier_init.release.cluster;\n" ::);
  }
  asm volatile("tcgen05.fence::before_thread_sync;\n" ::);
  __syncthreads();
  asm volatile("tcgen05.fence::after_thread_sync;\n" ::);
  const uint32_t tmem = tmem_base_sh;
  volatile int* abort_flag = &abort_sh;

  if (warp >= 4 && warp < 8) {
    // ---------------- producers
    const int ptid = tid - 128;
    long j = 0;  // k-steps issued
    bool ok = true;
    for (int ti = blockIdx.x; ti < ntiles && ok; ti += gridDim.x) {
      const TcTile tl = tiles[ti];
      const TcTask tk = tasks[tl.task];
      const int nt = min(TC_NMAX, round16(tk.n - tl.c0));
      TcTerm nxt = terms[tk.t0];
      bool first = true;
      for (int t = tk.t0; t < tk.t1 && ok; ++t) {
        const TcTerm tm = nxt;
        if (t + 1 < tk.t1) nxt = terms[t + 1];  // prefetch the next descriptor
        const int ns = tm.nsl < 1 ? 1 : (tm.nsl > NSL ? NSL : tm.nsl);
        const uint32_t id = idesc_bf16(nt, tm.flags & 1);
        const int np = npairs(ns);
        // stage sequence: one per K step (slice reuse) or one per (slice pair, K step)
        for (int p = 0; p < (REUSE ? 1 : np) && ok; ++p)
        for (int k0 = 0; k0 < tm.k; k0 += TC_K) {
          const int s = (int)(j % S);
          if (j >= S && !mbar_wait(&empty_b[s], (uint32_t)(((j / S) - 1) & 1), abort_flag)) {
            ok = false;
            break;
          }
          const uint32_t sa = base + s * STAGE_BYTES;
          if (REUSE) {
            for (int i = 0; i < ns; ++i)
              load_tile(sa + i * TC_TILE_BYTES, tm.A + i * tm.sA, tm.lda, tm.k, tk.m, tl.r0, k0, TC_M, ptid);
            for (int i = 0; i < ns; ++i)
              load_tile(sa + (SLOTS + i) * TC_TILE_BYTES, tm.B + i * tm.sB, tm.ldb, tm.k, tk.n, tl.c0, k0, nt, ptid);
          } else {
            load_tile(sa, tm.A + PAIR_I[p] * tm.sA, tm.lda, tm.k, tk.m, tl.r0, k0, TC_M, ptid);
            load_tile(sa + TC_TILE_BYTES, tm.B + PAIR_J[p] * tm.sB, tm.ldb, tm.k, tk.n, tl.c0, k0, nt, ptid);
          }
          // the full barrier completes when every producer's copies of this stage
          // have landed (asynchronous arrivals) and the parameters are written
          asm volatile("cp.async.mbarrier.arrive.noinc.shared::cta.b64 [%0];\n" ::"r"(smem_u32(&full_b[s]))
                       : "memory");
          if (ptid == 0) {
            meta_id[s] = id;
            meta_nk[s] = min(TC_K / 16, (tm.k - k0 + 15) / 16);
            meta_np[s] = REUSE ? np : 1;
            meta_first[s] = first ? 1 : 0;
            meta_last[s] = (t + 1 == tk.t1 && (REUSE || p + 1 == np) && k0 + TC_K >= tm.k) ? 1 : 0;
            mbar_arrive(&full_b[s]);
          }
          first = false;
          ++j;
        }
      }
    }
    // let every copy land before the CTA can exit
    cp_async_wait<0>();
  } else if (warp == 8) {
    // ---------------- MMA issuer: consumes stages in order, parameters from shared memory
    if (lane == 0) {
      long j = 0;
      int it = 0;
      bool ok = true;
      for (int ti = blockIdx.x; ti < ntiles && ok; ti += gridDim.x, ++it) {
        const int acc = it % NACC;
        if (it >= NACC && !mbar_wait(&tempty_b[acc], (uint32_t)(((it / NACC) - 1) & 1), abort_flag)) {
          ok = false;
          break;
        }
        asm volatile("tcgen05.fence::after_thread_sync;\n" ::);
        const uint32_t dacc = tmem + (uint32_t)(acc * TC_NMAX);
        for (;;) {
          const int s = (int)(j % S);
          if (!mbar_wait(&full_b[s], (uint32_t)((j / S) & 1), abort_flag)) {
            ok = false;
            break;
          }
          // make the producers' cp.async (generic proxy) writes visible to the tensor core (async proxy)
          asm volatile("fence.proxy.async.shared::cta;\n" ::: "memory");
          asm volatile("tcgen05.fence::after_thread_sync;\n" ::);
          const uint32_t id = meta_id[s];
          const int nk = meta_nk[s], np = meta_np[s], first = meta_first[s], last = meta_last[s];
          const uint32_t sa = base + s * STAGE_BYTES;
          for (int p = 0; p < np; ++p) {
            const uint32_t sa_a = sa + (REUSE ? PAIR_I[p] : 0) * TC_TILE_BYTES;
            const uint32_t sa_b = sa + (SLOTS + (REUSE ? PAIR_J[p] : 0)) * TC_TILE_BYTES;
            for (int kk = 0; kk < nk; ++kk) {
              const uint64_t ad = sdesc(sa_a + kk * 32), bd = sdesc(sa_b + kk * 32);
              const uint32_t accum = (first && p == 0 && kk == 0) ? 0u : 1u;
              asm volatile(
                  "{\n .reg .pred p;\n setp.ne.b32 p, %4, 0;\n"
                  " tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n}\n" ::"r"(dacc),
                  "l"(ad), "l"(bd), "r"(id), "r"(accum));
            }
          }
          asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];\n" ::"r"(
              smem_u32(&empty_b[s])));
          ++j;
          if (last) break;
        }
        if (!ok) break;
        asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];\n" ::"r"(
            smem_u32(&tfull_b[acc])));
      }
    }
  } else if (warp < 4) {
    // ---------------- epilogue
    int it = 0;
    for (int ti = blockIdx.x; ti < ntiles; ti += gridDim.x, ++it) {
      const TcTile tl = tiles[ti];
      const TcTask tk = tasks[tl.task];
      const int nt = min(TC_NMAX, round16(tk.n - tl.c0));
      const int acc = it % NACC;
      bool ok = mbar_wait(&tfull_b[acc], (uint32_t)((it / NACC) & 1), abort_flag);
      ok = __all_sync(0xffffffffu, ok);
      if (!ok) break;
      asm volatile("tcgen05.fence::after_thread_sync;\n" ::);
      const int row = tl.r0 + warp * 32 + lane;
      for (int c0 = 0; c0 < nt; c0 += 32) {
        uint32_t v[32];
        const uint32_t taddr = tmem + ((uint32_t)(warp * 32) << 16) + (uint32_t)(acc * TC_NMAX + c0);
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
        const int colb = tl.c0 + c0;          // first column of this 32-column chunk
        const int nv = min(32, tk.n - colb);  // valid columns in it (>= 1)
        if (tk.C && row < tk.m) {
          if (tk.beta == 2 && !tk.trans) {
            // split-K accumulation: vector reductions along the row
            float* cp = tk.C + (long)row * tk.ldc + colb;
            const bool al = (reinterpret_cast<uintptr_t>(cp) & 15) == 0;
#pragma unroll
            for (int q = 0; q < 32; q += 4) {
              if (q >= nv) break;
              if (al && q + 4 <= nv) {
                red_add_v4(cp + q, v[q], v[q + 1], v[q + 2], v[q + 3]);
              } else {
#pragma unroll
                for (int u = 0; u < 4; ++u)
                  if (q + u < nv) atomicAdd(cp + q + u, __uint_as_float(v[q + u]));
              }
            }
          } else {
#pragma unroll
            for (int q = 0; q < 32; ++q) {
              if (q >= nv) break;
              const int col = colb + q;
              float x = __uint_as_float(v[q]);
              float* cp = tk.C + (tk.trans ? (long)col * tk.ldc + row : (long)row * tk.ldc + col);
              if (tk.beta == 2) {
                atomicAdd(cp, x);
              } else {
                if (tk.beta) x += *cp;
                *cp = x;
              }
            }
          }
        }
        if (tk.Cb) {
          if (tk.trans) {
            // transposed BF16 slices through shared memory: lane = row on the way in,
            // lane = column on the way out, 16-byte stores along the output rows
            __nv_bfloat16* st = epi + warp * 32 * TC_EPI_LD;
            const int rbase = tl.r0 + warp * 32;
            const bool full = rbase + 32 <= tk.m;
            for (int sl = 0; sl < tk.nslices; ++sl) {
#pragma unroll
              for (int q = 0; q < 32; ++q) st[q * TC_EPI_LD + lane] = bf16_slice(__uint_as_float(v[q]), sl);
              __syncwarp();
              if (lane < nv && rbase < tk.m) {
                __nv_bfloat16* dst = tk.Cb + (long)sl * tk.slice_stride + (long)(colb + lane) * tk.ldcb + rbase;
                const __nv_bfloat16* src = st + lane * TC_EPI_LD;
                if (full && (reinterpret_cast<uintptr_t>(dst) & 15) == 0) {
#pragma unroll
                  for (int p4 = 0; p4 < 4; ++p4)
                    *reinterpret_cast<uint4*>(dst + 8 * p4) = *reinterpret_cast<const uint4*>(src + 8 * p4);
                } else {
                  for (int r = 0; r < 32 && rbase + r < tk.m; ++r) dst[r] = src[r];
                }
              }
              __syncwarp();
            }
          } else if (row < tk.m) {
#pragma unroll
            for (int q = 0; q < 32; ++q) {
              if (q >= nv) break;
              const long ob = (long)row * tk.ldcb + colb + q;
              const float x = __uint_as_float(v[q]);
              for (int sl = 0; sl < tk.nslices; ++sl) tk.Cb[sl * tk.slice_stride + ob] = bf16_slice(x, sl);
            }
          }
        }
      }
      asm volatile("tcgen05.fence::before_thread_sync;\n" ::);
      mbar_arrive(&tempty_b[acc]);
    }
  }
  asm volatile("tcgen05.fence::before_thread_sync;\n" ::);
  __syncthreads();
  if (tid == 0 && abort_sh) atomicExch(err, 1);
  if (warp == 0) {
    asm volatile("tcgen05.fence::after_thread_sync;\n" ::);
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;\n" ::"r"(tmem),
                 "r"(TcCfg<NSL>::TMEM_COLS));
  }
}

std::atomic<long> g_tc_launches{0};

}  // namespace

long tc_launch_count() { return g_tc_launches.load(); }
void count_tc_launches(long n) { g_tc_launches += n; }

template <int NSL>
static cudaError_t launch_nsl(const TcTile* d_tiles, int ntiles, const TcTask* d_tasks, const TcTerm* d_terms,
                              int* d_err, cudaStream_t s) {
  // one-time set-up per instantiation, thread-safe (function-local static)
  static const int nsm = [] {
    if (cudaFuncSetAttribute(gemm_bf16_tc_kernel<NSL>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                             TcCfg<NSL>::SMEM) != cudaSuccess)
      return -1;
    int dev = 0, n = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&n, cudaDevAttrMultiProcessorCount, dev);
    return n > 0 ? n : 148;
  }();
  if (nsm < 0) return cudaErrorInvalidValue;
  // persistent: one wave of resident CTAs (256 TMEM columns each)
  const int resident = TcCfg<NSL>::CTAS_PER_SM * nsm;
  const int grid = ntiles < resident ? ntiles : resident;
  ++g_tc_launches;
  gemm_bf16_tc_kernel<NSL><<<grid, TC_THREADS, TcCfg<NSL>::SMEM, s>>>(d_tiles, ntiles, d_tasks, d_terms, d_err);
  return cudaGetLastError();
}

cudaError_t launch_gemm_bf16_tc(const TcTile* d_tiles, int ntiles, const TcTask* d_tasks, const TcTerm* d_terms,
                                int* d_err, cudaStream_t s, int nsl) {
  if (ntiles <= 0) return cudaSuccess;
  if (nsl <= 1) return launch_nsl<1>(d_tiles, ntiles, d_tasks, d_terms, d_err, s);
  if (nsl == 2) return launch_nsl<2>(d_tiles, ntiles, d_tasks, d_terms, d_err, s);
  if (nsl == 3) return launch_nsl<3>(d_tiles, ntiles, d_tasks, d_terms, d_err, s);
  return cudaErrorInvalidValue;
}

}  // namespace gbdmrg
