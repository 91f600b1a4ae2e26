// TMA-staged tensor-core grouped GEMM (tcgen05, sm_103a): BF16 operands, FP32
// accumulation in tensor memory.
//
// The operands of the single-pass sigma vector live in a few large row-major
// BF16 matrices (per quantum-number group of the cut: the stacked two-site
// wavefunction Psi_g, the stacked right operators, the X intermediates; one
// matrix for all left-operator blocks), each described by one tensor map.  A
// K step of a tile is then two TMA box copies (A: 128 rows x 64 columns, B: n
// rows x 64 columns, 128-byte swizzle, zero fill outside the matrix) that
// complete on the stage's mbarrier by transaction count: no producer threads
// copy data, and a ragged edge costs nothing but the zero fill.
//
// Persistent and warp-specialised, one CTA per SM (192 KB shared memory ring,
// all 512 tensor-memory columns):
//   warp 0     one thread: waits for a free stage, posts the expected bytes and
//              the stage's MMA parameters, issues the two box copies
//   warp 1     one thread issues tcgen05.mma (M = 128, N = n, K = 16 per
//              instruction; instructions past the term's K are skipped) and
//              commits to the stage's empty barrier / the accumulator's full
//              barrier
//   warps 2-5  epilogue: tcgen05.ld of their 32 tensor-memory lanes; BF16 rows
//              (X intermediates, up to three slices) staged in shared memory and
//              written row by row with coalesced stores to the rows a row map
//              gives, or FP32 vector reductions (sigma^T, several tiles may add
//              into one block) of per-segment partial sums
// Two (store mode, N <= 256) or four (reduce mode, N <= 128) accumulators let
// the epilogue of one tile overlap the MMAs of the next.  Every wait is
// bounded: on timeout the CTA raises a shared abort flag, records an error,
// waits (bounded) for the copies it issued, frees its tensor memory and returns.
#include "kernels_tma.hpp"

#include <cuda_bf16.h>

#include <atomic>
#include <cstdint>
#include <mutex>

namespace gbdmrg {

long tc_launch_count();
void count_tc_launches(long n);

namespace {

constexpr int TM_THREADS = 192;
constexpr int TM_BOX_K = 64;                       // columns per box (128 bytes)
constexpr int TM_A_BYTES = 128 * TM_BOX_K * 2;     // 16 KB
constexpr long TM_WAIT_LIMIT = 1L << 24;

template <int MODE>
struct TmCfg {
  static constexpr bool STORE = MODE == TM_MODE_STORE_BF16;
  static constexpr bool EXACT = MODE == TM_MODE_EXACT_F64;
  // exact mode: 64 columns, so that the two-float sums (128 registers) fit
  static constexpr int NMAX = STORE ? 256 : (EXACT ? 64 : 128);
  static constexpr int NACC = 512 / NMAX;
  static constexpr int B_BYTES = NMAX * TM_BOX_K * 2;
  static constexpr int STAGE_BYTES = TM_A_BYTES + B_BYTES;
  // store mode: each epilogue warp stages its 32 rows in shared memory (rows padded
  // by 16 bytes against bank conflicts) and writes them row by row with coalesced
  // 16-byte stores
  static constexpr int STAGE_LD = NMAX + 8;  // elements per staged row
  static constexpr int STAGING = STORE ? 128 * STAGE_LD * 2 : 0;
  static constexpr int STAGES = STORE ? 3 : (EXACT ? 8 : 6);
  static constexpr int SMEM = STAGES * STAGE_BYTES + STAGING + 1024;
};
constexpr int TM_MAX_STAGES = 8, TM_MAX_ACC = 8;

__device__ __forceinline__ uint32_t smem_u32(const void* p) { return (uint32_t)__cvta_generic_to_shared(p); }

// shared-memory matrix descriptor: K-major, 128-byte swizzle, 8-row groups 1024 B apart
__device__ __forceinline__ uint64_t sdesc(uint32_t saddr) {
  uint64_t d = 0;
  d |= (uint64_t)((saddr >> 4) & 0x3FFFu);
  d |= (uint64_t)1 << 16;
  d |= (uint64_t)(1024 >> 4) << 32;
  d |= (uint64_t)1 << 46;
  d |= (uint64_t)2 << 61;
  return d;
}

// instruction descriptor: D f32, A/B bf16, both K-major, M = 128, N = n
__device__ __forceinline__ uint32_t idesc_bf16(int n, bool negA) {
  uint32_t d = 0;
  d |= 1u << 4;
  d |= 1u << 7;
  d |= 1u << 10;
  if (negA) d |= 1u << 13;
  d |= (uint32_t)(n >> 3) << 17;
  d |= (uint32_t)(128 >> 4) << 24;
  return d;
}

__device__ __forceinline__ void mbar_init(uint64_t* b, int count) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;\n" ::"r"(smem_u32(b)), "r"(count));
}
__device__ __forceinline__ void mbar_arrive(uint64_t* b) {
  asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];\n" ::"r"(smem_u32(b)) : "memory");
}
__device__ __forceinline__ void mbar_arrive_expect_tx(uint64_t* b, uint32_t bytes) {
  asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;\n" ::"r"(smem_u32(b)), "r"(bytes) : "memory");
}
__device__ __forceinline__ bool mbar_test(uint64_t* b, uint32_t parity) {
  uint32_t done;
  asm volatile(
      "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n selp.u32 %0, 1, 0, p;\n}\n"
      : "=r"(done)
      : "r"(smem_u32(b)), "r"(parity)
      : "memory");
  return done != 0;
}
// bounded parity wait; gives up when the CTA-wide abort flag is raised
__device__ __forceinline__ bool mbar_wait(uint64_t* b, uint32_t parity, volatile int* abort_flag) {
  for (long it = 0; it < TM_WAIT_LIMIT; ++it) {
    if (mbar_test(b, parity)) return true;
    if ((it & 1023) == 1023 && *abort_flag) return false;
  }
  *abort_flag = 1;
  return false;
}

__device__ __forceinline__ void tma_load_2d(uint32_t dst, const CUtensorMap* map, int x, int y, uint64_t* bar) {
  asm volatile(
      "cp.async.bulk.tensor.2d.shared::cluster.global.tile.mbarrier::complete_tx::bytes [%0], [%1, {%2, %3}], [%4];\n" ::"r"(
          dst),
      "l"(map), "r"(x), "r"(y), "r"(smem_u32(bar))
      : "memory");
}

__device__ __forceinline__ void red_add_v4(float* p, uint32_t a, uint32_t b, uint32_t c, uint32_t d) {
  asm volatile("red.relaxed.gpu.global.add.v4.f32 [%0], {%1, %2, %3, %4};\n" ::"l"(p), "f"(__uint_as_float(a)),
               "f"(__uint_as_float(b)), "f"(__uint_as_float(c)), "f"(__uint_as_float(d))
               : "memory");
}

// 32 consecutive FP32 columns of this warp's 32 tensor-memory lanes
__device__ __forceinline__ void tmem_ld32(uint32_t taddr, uint32_t (&v)[32]) {
  asm volatile(
      "tcgen05.ld.sync.aligned.32x32b.x32.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15,"
      "%16,%17,%18,%19,%20,%21,%22,%23,%24,%25,%26,%27,%28,%29,%30,%31}, [%32];\n"
      : "=r"(v[0]), "=r"(v[1]), "=r"(v[2]), "=r"(v[3]), "=r"(v[4]), "=r"(v[5]), "=r"(v[6]), "=r"(v[7]),
        "=r"(v[8]), "=r"(v[9]), "=r"(v[10]), "=r"(v[11]), "=r"(v[12]), "=r"(v[13]), "=r"(v[14]), "=r"(v[15]),
        "=r"(v[16]), "=r"(v[17]), "=r"(v[18]), "=r"(v[19]), "=r"(v[20]), "=r"(v[21]), "=r"(v[22]), "=r"(v[23]),
        "=r"(v[24]), "=r"(v[25]), "=r"(v[26]), "=r"(v[27]), "=r"(v[28]), "=r"(v[29]), "=r"(v[30]), "=r"(v[31])
      : "r"(taddr));
  asm volatile("tcgen05.wait::ld.sync.aligned;\n" ::: "memory");
}

__device__ __forceinline__ uint32_t pack_bf16x2(uint32_t lo, uint32_t hi) {
  const __nv_bfloat162 h = __floats2bfloat162_rn(__uint_as_float(lo), __uint_as_float(hi));
  return *reinterpret_cast<const uint32_t*>(&h);
}

template <int MODE>
__global__ void __launch_bounds__(TM_THREADS, 1)
    gemm_tma_kernel(const TmTile* __restrict__ tiles, int ntiles, const TmTerm* __restrict__ terms,
                    const CUtensorMap* __restrict__ maps, const long* __restrict__ rowmap,
                    const int2* __restrict__ cbtab, void* __restrict__ out, int out_slices, long slice_stride,
                    int* __restrict__ err, const int* __restrict__ expo) {
  using Cfg = TmCfg<MODE>;
  constexpr int S = Cfg::STAGES;
  constexpr int STAGE_BYTES = Cfg::STAGE_BYTES;
  constexpr int NACC = Cfg::NACC;
  constexpr int NMAX = Cfg::NMAX;
  constexpr bool STORE = Cfg::STORE;
  constexpr bool EXACT = Cfg::EXACT;
  // reduce mode: a tile's products accumulate in tensor memory for at most
  // TM_SEG_KSTEPS K steps (a segment); the epilogue adds the segments in FP32
  // registers with round-to-nearest, so the rounding toward zero of the tensor-core
  // accumulation acts on short sums only
  constexpr int SEG = STORE ? (1 << 30) : TM_SEG_KSTEPS;
  extern __shared__ uint8_t dsm[];
  __shared__ __align__(8) uint64_t full_b[TM_MAX_STAGES], empty_b[TM_MAX_STAGES], tfull_b[TM_MAX_ACC],
      tempty_b[TM_MAX_ACC];
  __shared__ uint32_t tmem_base_sh;
  __shared__ int abort_sh;
  // per stage: instruction descriptor, K=16 steps, first K step of a segment, last K
  // step of a segment, last K step of the tile
  // (packed into one 64-bit word: low half the instruction descriptor, high half the
  // K=16 steps in bits 0-2 and the flags first / segment end / last in bits 3-5)
  __shared__ uint64_t meta[TM_MAX_STAGES];
  const uint32_t base = (smem_u32(dsm) + 1023u) & ~1023u;
  uint8_t* const base_ptr = dsm + (base - smem_u32(dsm));
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;

  if (warp == 2) {  // an epilogue warp (all lanes take the same path) owns the tensor memory
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;\n" ::"r"(smem_u32(&tmem_base_sh)),
                 "r"(512));
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;\n" ::);
  }
  if (tid == 0) {
    for (int s = 0; s < S; ++s) {
      mbar_init(&full_b[s], 1);  // the producer's arrive (with the expected bytes)
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

  if (warp == 0) {
    // ---------------- TMA producer: the warp loads the term descriptors of a tile 32 at
    // a time (one per lane) and prefetches their tensor maps (every slice's); lane 0
    // issues the copies.  Descriptor loads run ahead of their use: the tile after next
    // and the next tile's first 32 terms while a tile is issued, the next 32 terms of a
    // tile while the current 32 are issued.
    long j = 0;  // K steps issued (lane 0)
    int st = 0;          // stage of the next K step (j % S)
    uint32_t par = 0;    // its round's parity ((j / S) & 1)
    bool wrapped = false;  // j >= S
    bool ok = true;
    const int G = (int)gridDim.x;
    TmTile cur{}, nxt{};
    TmTerm pre{};  // this lane's term of the current tile's first batch
    if ((int)blockIdx.x < ntiles) {
      cur = tiles[blockIdx.x];
      if (lane < min(32, cur.t1 - cur.t0)) pre = terms[cur.t0 + lane];
    }
    if ((int)blockIdx.x + G < ntiles) nxt = tiles[blockIdx.x + G];
    for (int ti = blockIdx.x; ti < ntiles && ok; ti += G) {
      const TmTile tl = cur;
      TmTile nn{};
      if (ti + 2 * G < ntiles) nn = tiles[ti + 2 * G];
      TmTerm pre_next{};
      if (ti + G < ntiles && lane < min(32, nxt.t1 - nxt.t0)) pre_next = terms[nxt.t0 + lane];
      const uint32_t bbytes = (uint32_t)tl.n * TM_BOX_K * 2;
      int seg_pos = 0;  // K steps of the current segment so far
      TmTerm mine = pre, ahead{};
      for (int tb = tl.t0; tb < tl.t1 && ok; tb += 32) {
        const int cnt = min(32, tl.t1 - tb);
        if (tb != tl.t0) mine = ahead;
        if (tb + 32 < tl.t1 && lane < min(32, tl.t1 - tb - 32)) ahead = terms[tb + 32 + lane];
        if (lane < cnt) {
          const int nslp = max(1, (mine.neg >> 4) & 15);
          for (int i = 0; i < nslp; ++i) {
            asm volatile("prefetch.tensormap [%0];\n" ::"l"(maps + mine.amap + i) : "memory");
            asm volatile("prefetch.tensormap [%0];\n" ::"l"(maps + mine.bmap + i) : "memory");
          }
        }
        for (int q = 0; q < cnt && ok; ++q) {
          TmTerm tm;
          tm.amap = __shfl_sync(0xffffffffu, mine.amap, q);
          tm.bmap = __shfl_sync(0xffffffffu, mine.bmap, q);
          tm.ax = __shfl_sync(0xffffffffu, mine.ax, q);
          tm.ay = __shfl_sync(0xffffffffu, mine.ay, q);
          tm.bx = __shfl_sync(0xffffffffu, mine.bx, q);
          tm.by = __shfl_sync(0xffffffffu, mine.by, q);
          tm.k = __shfl_sync(0xffffffffu, mine.k, q);
          tm.neg = __shfl_sync(0xffffffffu, mine.neg, q);
          tm.ea = __shfl_sync(0xffffffffu, mine.ea, q);
          tm.eb = __shfl_sync(0xffffffffu, mine.eb, q);
          if (lane == 0) {
            const uint32_t id = idesc_bf16(tl.n, (tm.neg & 1) != 0);
            const bool last_term = tb + q + 1 == tl.t1;
            // the term stands for all slice pairs (i, j), i + j < nsl, in order of the
            // level l = i + j (slice i of a map is the map index + i); exact mode: one
            // segment per level
            const int nsl = max(1, (tm.neg >> 4) & 15);
            for (int l = 0; l < nsl && ok; ++l)
              for (int i = 0; i <= l && ok; ++i) {
                const CUtensorMap* ma = maps + tm.amap + i;
                const CUtensorMap* mb = maps + tm.bmap + (l - i);
                for (int k0 = 0; k0 < tm.k; k0 += TM_BOX_K) {
                  if (wrapped && !mbar_wait(&empty_b[st], par ^ 1u, abort_flag)) {
                    ok = false;
                    break;
                  }
                  const bool kend = k0 + TM_BOX_K >= tm.k;
                  const bool last = last_term && kend && l + 1 == nsl && i == l;
                  uint32_t fl = (uint32_t)min(TM_BOX_K / 16, (tm.k - k0) / 16);
                  if (EXACT) {
                    fl |= (i == 0 && k0 == 0) ? 8u : 0u;
                    fl |= (i == l && kend) ? 16u : 0u;
                  } else {
                    fl |= seg_pos == 0 ? 8u : 0u;
                    fl |= (last || seg_pos == SEG - 1) ? 16u : 0u;
                  }
                  fl |= last ? 32u : 0u;
                  meta[st] = (uint64_t)id | ((uint64_t)fl << 32);
                  const uint32_t sa = base + st * STAGE_BYTES;
                  mbar_arrive_expect_tx(&full_b[st], TM_A_BYTES + bbytes);
                  tma_load_2d(sa, ma, tm.ax + k0, tm.ay, &full_b[st]);
                  tma_load_2d(sa + TM_A_BYTES, mb, tm.bx + k0, tm.by, &full_b[st]);
                  ++j;
                  if (++seg_pos == SEG) seg_pos = 0;
                  if (++st == S) {
                    st = 0;
                    par ^= 1u;
                    wrapped = true;
                  }
                }
              }
          }
          ok = __shfl_sync(0xffffffffu, ok, 0);
        }
      }
      cur = nxt;
      nxt = nn;
      pre = pre_next;
    }
    if (lane == 0) {
      // every issued copy must land before the CTA may exit: the last (up to S)
      // issued stages complete their full phase when their bytes arrive
      for (long q = j - 1; q >= 0 && q >= j - S; --q) {
        const int s = (int)(q % S);
        for (long it = 0; it < TM_WAIT_LIMIT && !mbar_test(&full_b[s], (uint32_t)((q / S) & 1)); ++it) {
        }
      }
    }
  } else if (warp == 1) {
    // ---------------- MMA issuer (one thread): one accumulator per segment
    if (lane == 0) {
      int st = 0;            // stage of the next K step
      uint32_t par = 0;      // its round's parity
      int sg = 0;  // segments issued
      bool ok = true;
      // shared-memory descriptors of stage 0's operands; stage s and K=16 step kk add
      // (s * STAGE_BYTES + kk * 32) / 16 to the 14-bit address field (no carry: shared
      // addresses stay below 256 KB)
      const uint64_t ad0 = sdesc(base), bd0 = sdesc(base + TM_A_BYTES);
      for (int ti = blockIdx.x; ti < ntiles && ok; ti += gridDim.x) {
        bool tile_done = false;
        while (!tile_done && ok) {
          const int acc = sg % NACC;
          if (sg >= NACC && !mbar_wait(&tempty_b[acc], (uint32_t)(((sg / NACC) - 1) & 1), abort_flag)) {
            ok = false;
            break;
          }
          asm volatile("tcgen05.fence::after_thread_sync;\n" ::);
          const uint32_t dacc = tmem + (uint32_t)(acc * NMAX);
          for (;;) {
            if (!mbar_wait(&full_b[st], par, abort_flag)) {
              ok = false;
              break;
            }
            asm volatile("tcgen05.fence::after_thread_sync;\n" ::);
            const uint64_t mw = meta[st];
            const uint32_t id = (uint32_t)mw, fl = (uint32_t)(mw >> 32);
            const int nk = (int)(fl & 7u);
            const uint64_t off = (uint64_t)((st * STAGE_BYTES) >> 4);
            for (int kk = 0; kk < nk; ++kk) {
              const uint64_t ad = ad0 + off + (uint64_t)(kk * 2), bd = bd0 + off + (uint64_t)(kk * 2);
              const uint32_t accum = ((fl & 8u) && kk == 0) ? 0u : 1u;
              asm volatile(
                  "{\n .reg .pred p;\n setp.ne.b32 p, %4, 0;\n"
                  " tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n}\n" ::"r"(dacc),
                  "l"(ad), "l"(bd), "r"(id), "r"(accum));
            }
            asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];\n" ::"r"(
                smem_u32(&empty_b[st])));
            if (++st == S) {
              st = 0;
              par ^= 1u;
            }
            if (fl & 16u) {
              tile_done = (fl & 32u) != 0;
              break;
            }
          }
          if (!ok) break;
          asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];\n" ::"r"(
              smem_u32(&tfull_b[acc])));
          ++sg;
        }
      }
    }
  } else {
    // ---------------- epilogue (warps 2-5: tensor-memory lanes 32 * (warp % 4) ...)
    const int sub = warp & 3;
    const int r = sub * 32 + lane;  // row of the tile
    __nv_bfloat16* const srow =
        reinterpret_cast<__nv_bfloat16*>(base_ptr + S * STAGE_BYTES) + (STORE ? r * Cfg::STAGE_LD : 0);
    int sg = 0;
    bool ok = true;
    // the next tile's descriptor is loaded one tile ahead; in store mode the row map and
    // column blocks of a tile are read before its accumulator is waited for
    TmTile tl_next{};
    if ((int)blockIdx.x < ntiles) tl_next = tiles[blockIdx.x];
    for (int ti = blockIdx.x; ti < ntiles && ok; ti += gridDim.x) {
      const TmTile tl = tl_next;
      if (ti + (int)gridDim.x < ntiles) tl_next = tiles[ti + gridDim.x];
      if constexpr (STORE) {
        const int acc = sg % NACC;
        const long row_own = rowmap[tl.rowmap_off + r];
        // this lane's 8-column chunk of every row: its column block, base and width
        long lane_base = -1;
        int lane_w = 0;
        if (lane * 8 < tl.n) {
          const long col = tl.out_off + lane * 8;
          for (int e = tl.cb0; e < tl.cb1; ++e) {
            const int2 cb = cbtab[e];
            if (col >= cb.x && col < cb.x + cb.y) {
              lane_base = tl.xbase + tl.xrows * cb.x + (col - cb.x);
              lane_w = cb.y;
            }
          }
        }
        ok = mbar_wait(&tfull_b[acc], (uint32_t)((sg / NACC) & 1), abort_flag);
        ok = __all_sync(0xffffffffu, ok);
        if (!ok) break;
        asm volatile("tcgen05.fence::after_thread_sync;\n" ::);
        __nv_bfloat16* const wrows =
            reinterpret_cast<__nv_bfloat16*>(base_ptr + S * STAGE_BYTES) + sub * 32 * Cfg::STAGE_LD;
        if (out_slices == 1) {
          // one pass: this thread's row into the staging rows of its warp, then the warp
          // writes its 32 rows one after another, each as one contiguous run of 16-byte
          // stores across the lanes (up to 512 bytes per instruction)
#pragma unroll 1
          for (int c0 = 0; c0 < tl.n; c0 += 32) {
            uint32_t v[32];
            tmem_ld32(tmem + ((uint32_t)(sub * 32) << 16) + (uint32_t)(acc * NMAX + c0), v);
#pragma unroll
            for (int u = 0; u < 32; u += 8) {
              uint4 w;
              w.x = pack_bf16x2(v[u], v[u + 1]);
              w.y = pack_bf16x2(v[u + 2], v[u + 3]);
              w.z = pack_bf16x2(v[u + 4], v[u + 5]);
              w.w = pack_bf16x2(v[u + 6], v[u + 7]);
              if (c0 + u < tl.n) *reinterpret_cast<uint4*>(srow + c0 + u) = w;
            }
          }
          __syncwarp();
#pragma unroll 1
          for (int rr = 0; rr < 32; ++rr) {
            const long d = __shfl_sync(0xffffffffu, row_own, rr);
            if (d >= 0 && lane_base >= 0) {
              const uint4 w = *reinterpret_cast<const uint4*>(wrows + rr * Cfg::STAGE_LD + lane * 8);
              *reinterpret_cast<uint4*>(reinterpret_cast<__nv_bfloat16*>(out) + lane_base + d * lane_w) = w;
            }
          }
          __syncwarp();
        } else {
          // two or three slices x = s0 + s1 + s2 from one read of each value, stored
          // directly: per 8 columns one 16-byte store per slice into this row.  The
          // tensor-memory loads (32 columns, one wait) are warp-wide, the stores only for
          // rows that exist; the column block of 8-column chunk c is lane c's (above)
#pragma unroll 1
          for (int c0 = 0; c0 < tl.n; c0 += 32) {
            uint32_t v[32];
            tmem_ld32(tmem + ((uint32_t)(sub * 32) << 16) + (uint32_t)(acc * NMAX + c0), v);
#pragma unroll
            for (int u8 = 0; u8 < 32; u8 += 8) {
              const int ch = (c0 + u8) >> 3;  // < NMAX / 8 <= 32
              const long cb_base = __shfl_sync(0xffffffffu, lane_base, ch);
              const int cb_w = __shfl_sync(0xffffffffu, lane_w, ch);
              if (c0 + u8 >= tl.n) break;
              uint32_t w[3][4];
#pragma unroll
              for (int u = 0; u < 8; u += 2) {
                float a = __uint_as_float(v[u8 + u]), b = __uint_as_float(v[u8 + u + 1]);
#pragma unroll
                for (int sl = 0; sl < 3; ++sl) {
                  const __nv_bfloat162 h = __floats2bfloat162_rn(a, b);
                  w[sl][u / 2] = *reinterpret_cast<const uint32_t*>(&h);
                  a -= __low2float(h);
                  b -= __high2float(h);
                }
              }
              if (cb_base < 0 || row_own < 0) continue;
              __nv_bfloat16* g = reinterpret_cast<__nv_bfloat16*>(out) + cb_base + row_own * cb_w;
#pragma unroll
              for (int sl = 0; sl < 3; ++sl)
                if (sl < out_slices)
                  *reinterpret_cast<uint4*>(g + sl * slice_stride) =
                      make_uint4(w[sl][0], w[sl][1], w[sl][2], w[sl][3]);
            }
          }
        }
        asm volatile("tcgen05.fence::before_thread_sync;\n" ::);
        mbar_arrive(&tempty_b[acc]);
        ++sg;
      } else if constexpr (EXACT) {
        // per segment: its exact integer sums, times 2^(expo[ea] + expo[eb] - 7 (l + 2)),
        // added into two-float sums hi + lo (error-free additions)
        float hi[NMAX], lo[NMAX];
#pragma unroll
        for (int c = 0; c < NMAX; ++c) hi[c] = lo[c] = 0.0f;
        for (int sgi = 0, t = tl.t0; t < tl.t1 && ok; ++sgi) {
          const int flags = terms[t].neg;
          const int nsl = max(1, (flags >> 4) & 15);
          const int lvl = sgi;  // segment sgi of term t: level sgi
          const int e = expo[terms[t].ea] + expo[terms[t].eb] - TM_EXACT_BITS * (lvl + 2);
          if (sgi + 1 == nsl) {
            sgi = -1;
            ++t;
          }
          const int acc = sg % NACC;
          ok = mbar_wait(&tfull_b[acc], (uint32_t)((sg / NACC) & 1), abort_flag);
          ok = __all_sync(0xffffffffu, ok);
          if (!ok) break;
          asm volatile("tcgen05.fence::after_thread_sync;\n" ::);
#pragma unroll
          for (int cc = 0; cc < NMAX / 32; ++cc) {
            uint32_t v[32];
            tmem_ld32(tmem + ((uint32_t)(sub * 32) << 16) + (uint32_t)(acc * NMAX + cc * 32), v);
#pragma unroll
            for (int u = 0; u < 32; ++u) {
              float x = ldexpf(__uint_as_float(v[u]), e);
              if (flags & 1) x = -x;
              const float a = hi[cc * 32 + u];
              const float sum = __fadd_rn(a, x);
              const float bp = __fsub_rn(sum, a);
              const float err = __fadd_rn(__fsub_rn(a, __fsub_rn(sum, bp)), __fsub_rn(x, bp));
              hi[cc * 32 + u] = sum;
              lo[cc * 32 + u] = __fadd_rn(lo[cc * 32 + u], err);
            }
          }
          asm volatile("tcgen05.fence::before_thread_sync;\n" ::);
          mbar_arrive(&tempty_b[acc]);
          ++sg;
        }
        if (!ok) break;
        if (r < tl.m_valid) {
          double* p = reinterpret_cast<double*>(out) + tl.out_off + (long)r * tl.ldo;
#pragma unroll
          for (int c = 0; c < NMAX; ++c)
            if (c < tl.nvalid) p[c] = (double)hi[c] + (double)lo[c];
        }
      } else {
        float run[NMAX / 32][32];  // the tile's running FP32 sum (row r)
        for (int q = 0; q < tl.nseg; ++q, ++sg) {
          const int acc = sg % NACC;
          ok = mbar_wait(&tfull_b[acc], (uint32_t)((sg / NACC) & 1), abort_flag);
          ok = __all_sync(0xffffffffu, ok);
          if (!ok) break;
          asm volatile("tcgen05.fence::after_thread_sync;\n" ::);
#pragma unroll
          for (int cc = 0; cc < NMAX / 32; ++cc) {
            const int c0 = cc * 32;
            if (c0 < tl.n) {
              uint32_t v[32];
              tmem_ld32(tmem + ((uint32_t)(sub * 32) << 16) + (uint32_t)(acc * NMAX + c0), v);
              if (q == 0) {
#pragma unroll
                for (int u = 0; u < 32; ++u) run[cc][u] = __uint_as_float(v[u]);
              } else {
#pragma unroll
                for (int u = 0; u < 32; ++u) run[cc][u] += __uint_as_float(v[u]);
              }
            }
          }
          asm volatile("tcgen05.fence::before_thread_sync;\n" ::);
          mbar_arrive(&tempty_b[acc]);
        }
        if (!ok) break;
        if (r < tl.m_valid) {
          float* p = reinterpret_cast<float*>(out) + tl.out_off + (long)r * tl.ldo;
#pragma unroll
          for (int cc = 0; cc < NMAX / 32; ++cc)
#pragma unroll
            for (int u = 0; u < 32; u += 4) {
              if (cc * 32 + u >= tl.n) break;
              red_add_v4(p + cc * 32 + u, __float_as_uint(run[cc][u]), __float_as_uint(run[cc][u + 1]),
                         __float_as_uint(run[cc][u + 2]), __float_as_uint(run[cc][u + 3]));
            }
        }
      }
    }
  }
  asm volatile("tcgen05.fence::before_thread_sync;\n" ::);
  __syncthreads();
  if (tid == 0 && abort_sh) atomicExch(err, 1);
  if (warp == 2) {
    __syncwarp();
    asm volatile("tcgen05.fence::after_thread_sync;\n" ::);
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;\n" ::"r"(tmem), "r"(512));
  }
}

template <int MODE>
cudaError_t launch_mode(const TmTile* d_tiles, int ntiles, const TmTerm* d_terms, const CUtensorMap* d_maps,
                        const long* d_rowmap, const int2* d_cbtab, void* out, int out_slices, long slice_stride,
                        int* d_err, cudaStream_t s, const int* d_expo) {
  static const int nsm = [] {
    if (cudaFuncSetAttribute(gemm_tma_kernel<MODE>, cudaFuncAttributeMaxDynamicSharedMemorySize, TmCfg<MODE>::SMEM) !=
        cudaSuccess)
      return -1;
    int dev = 0, n = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&n, cudaDevAttrMultiProcessorCount, dev);
    return n > 0 ? n : 148;
  }();
  if (nsm < 0) return cudaErrorInvalidValue;
  const int grid = ntiles < nsm ? ntiles : nsm;
  count_tc_launches(1);
  gemm_tma_kernel<MODE><<<grid, TM_THREADS, TmCfg<MODE>::SMEM, s>>>(d_tiles, ntiles, d_terms, d_maps, d_rowmap,
                                                                     d_cbtab, out, out_slices, slice_stride, d_err,
                                                                     d_expo);
  return cudaGetLastError();
}

// exact splitting: one block of threads per job, warps over rows, lanes over columns.
// The block maximum is taken on the bit patterns (|x| orders like its bits as an
// unsigned integer), so the FP64 units see one multiply per element for the scaling by
// scale * 2^-e (exact: a power of two times the rounding of scale * x) and the split
// v = a + lo into two FP32 values; the 7-bit slices come from a by exact FP32 steps
// (w *= 2^7, q = rint(w), w -= q), and lo joins the remainder after the third slice
// (one FP32 rounding, below 2^-46 of the block's scale).  Slice magnitudes: the first
// <= 128, the fourth <= 72, the others <= 64.
__global__ void split_exact_kernel(const SplitJob* __restrict__ jobs, int nsl, int* __restrict__ expo_out) {
  const SplitJob jb = jobs[blockIdx.x];
  __shared__ unsigned long long red[32];
  __shared__ int e_sh;
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31, nw = blockDim.x >> 5;
  unsigned long long m = 0;
  for (int r = warp; r < jb.rows; r += nw) {
    const double* src = jb.src + (long)r * jb.lds;
    for (int c = lane; c < jb.cols; c += 32) {
      const unsigned long long bits = (unsigned long long)__double_as_longlong(src[c]) & 0x7fffffffffffffffULL;
      m = bits > m ? bits : m;
    }
  }
  for (int o = 16; o > 0; o >>= 1) {
    const unsigned long long t = __shfl_xor_sync(0xffffffffu, m, o);
    m = t > m ? t : m;
  }
  if (lane == 0) red[warp] = m;
  __syncthreads();
  if (threadIdx.x == 0) {
    unsigned long long mm = 0;
    for (int w = 0; w < nw; ++w) mm = red[w] > mm ? red[w] : mm;
    // fl(|scale| * max|x|) bounds every fl(|scale * x|) (rounding is monotone)
    const double mx = fabs(jb.scale) * __longlong_as_double((long long)mm);
    int e = 0;
    if (mx > 0.0) frexp(mx, &e);  // mx = f 2^e with 0.5 <= f < 1: |scale * x| < 2^e
    e_sh = e;
    expo_out[jb.expo] = e;
  }
  __syncthreads();
  const double f = ldexp(jb.scale, -e_sh);
  constexpr float STEP = (float)(1 << TM_EXACT_BITS);
  constexpr float LO_SCALE = (float)(1 << (3 * TM_EXACT_BITS));  // lo at the scale of the remainder after three slices
  for (int r = warp; r < jb.rows; r += nw) {
    const double* src = jb.src + (long)r * jb.lds;
    for (int c = lane; c < jb.wcols; c += 32) {
      const double v = c < jb.cols ? f * src[c] : 0.0;  // |v| < 1
      float w = __double2float_rn(v);
      const float lo = __double2float_rn(v - (double)w);
      __nv_bfloat16* d = jb.trans ? jb.dst + (long)c * jb.ldd + r : jb.dst + (long)r * jb.ldd + c;
      for (int s = 0; s < nsl; ++s) {
        if (s == 3) w += lo * LO_SCALE;
        w *= STEP;
        const float q = rintf(w);  // an integer of at most 128 in magnitude: exact in BF16
        d[(long)s * jb.slice_stride] = __float2bfloat16_rn(q);
        w -= q;
      }
    }
  }
}

using EncodeTiledFn = CUresult (*)(CUtensorMap*, CUtensorMapDataType, cuuint32_t, void*, const cuuint64_t*,
                                   const cuuint64_t*, const cuuint32_t*, const cuuint32_t*, CUtensorMapInterleave,
                                   CUtensorMapSwizzle, CUtensorMapL2promotion, CUtensorMapFloatOOBfill);

EncodeTiledFn encoder() {
  static EncodeTiledFn fn = [] {
    void* p = nullptr;
    cudaDriverEntryPointQueryResult q;
    if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &p, 12000, cudaEnableDefault, &q) != cudaSuccess ||
        q != cudaDriverEntryPointSuccess)
      return (EncodeTiledFn) nullptr;
    return reinterpret_cast<EncodeTiledFn>(p);
  }();
  return fn;
}

}  // namespace

cudaError_t launch_split_exact(const SplitJob* d_jobs, int njobs, int nsl, int* d_expo, cudaStream_t s) {
  if (njobs <= 0) return cudaSuccess;
  if (nsl < 1 || nsl > 6) return cudaErrorInvalidValue;  // the remainder and level-sum bounds hold up to six slices
  count_tc_launches(1);
  split_exact_kernel<<<njobs, 256, 0, s>>>(d_jobs, nsl, d_expo);
  return cudaGetLastError();
}

int tma_max_n(int mode) { return mode == TM_MODE_STORE_BF16 ? 256 : (mode == TM_MODE_EXACT_F64 ? 64 : 128); }

cudaError_t launch_gemm_tma(int mode, const TmTile* d_tiles, int ntiles, const TmTerm* d_terms,
                            const CUtensorMap* d_maps, const long* d_rowmap, const int2* d_cbtab, void* out,
                            int out_slices, long slice_stride, int* d_err, cudaStream_t s, const int* d_expo) {
  if (ntiles <= 0) return cudaSuccess;
  if (out_slices < 1 || out_slices > 3) return cudaErrorInvalidValue;
  if (mode == TM_MODE_STORE_BF16)
    return launch_mode<TM_MODE_STORE_BF16>(d_tiles, ntiles, d_terms, d_maps, d_rowmap, d_cbtab, out, out_slices,
                                           slice_stride, d_err, s, nullptr);
  if (mode == TM_MODE_REDUCE_F32)
    return launch_mode<TM_MODE_REDUCE_F32>(d_tiles, ntiles, d_terms, d_maps, d_rowmap, d_cbtab, out, 1, 0, d_err, s,
                                           nullptr);
  if (mode == TM_MODE_EXACT_F64) {
    if (!d_expo) return cudaErrorInvalidValue;
    return launch_mode<TM_MODE_EXACT_F64>(d_tiles, ntiles, d_terms, d_maps, d_rowmap, d_cbtab, out, 1, 0, d_err, s,
                                          d_expo);
  }
  return cudaErrorInvalidValue;
}

bool encode_bf16_map(CUtensorMap* out, const void* base, uint64_t rows, uint64_t cols, uint64_t ld,
                     uint32_t box_rows) {
  EncodeTiledFn fn = encoder();
  if (!fn || rows == 0 || cols == 0 || (ld * 2) % 16 != 0 || ((uintptr_t)base & 15) != 0 || box_rows == 0 ||
      box_rows > 256)
    return false;
  const cuuint64_t dims[2] = {cols, rows};
  const cuuint64_t strides[1] = {ld * 2};
  const cuuint32_t box[2] = {(cuuint32_t)TM_BOX_K, box_rows};
  const cuuint32_t estr[2] = {1, 1};
  return fn(out, CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, 2, const_cast<void*>(base), dims, strides, box, estr,
            CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_128B, CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
            CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) == CUDA_SUCCESS;
}

}  // namespace gbdmrg
