// TMA-staged tensor-core grouped GEMM (tcgen05, sm_103a): BF16 operands, FP32
// accumulation in tensor memory.
//
// The operands of the sigma vector live in a few large row-major BF16 matrices (per
// quantum-number group of the cut: the stacked two-site wavefunction Psi_g, the stacked
// right operators, the X intermediates; one matrix for all left-operator blocks), each
// described by one tensor map.  A stage of the ring is one or more pieces, each a pair of
// TMA box copies (A: 128 rows, B: n rows; 64 columns with 128-byte swizzle, or in the
// reduce mode up to four 16-column pieces with 32-byte swizzle) that complete on the
// stage's mbarrier by transaction count; zero fill outside the matrix covers ragged edges.
// The tiles' terms are expanded before the launch into per-CTA copy lists (stage word,
// expected bytes, box coordinates: fill_lists_kernel), so the producer does no term
// arithmetic.
//
// Persistent and warp-specialised, one CTA per SM (up to 212 KB of shared memory,
// all 512 tensor-memory columns):
//   warp 0     fetches its CTA's copy lists 32 stages at a time into shared memory
//              (1D bulk copies, double-buffered); per stage lane 0 waits for the ring
//              slot and posts the stage word and the expected bytes, then lane p issues
//              the two box copies of piece p
//   warp 1     one thread issues tcgen05.mma (M = 128, N = n, K = 16 per instruction)
//              and commits to the stage's empty barrier / the accumulator's full
//              barrier
//   warps 2-5  epilogue: tcgen05.ld of their 32 tensor-memory lanes; BF16 rows
//              (X intermediates, up to three slices) written with 16-byte stores to
//              the rows a row map gives, FP32 vector reductions (sigma^T, several
//              tiles may add into one block) of per-segment partial sums, or (exact
//              mode) two-float sums of exact integer segments stored in FP64
// Two (store mode, N <= 256), four (reduce mode, N <= 128) or eight (exact mode, N <=
// 64) accumulators let the epilogue of one tile overlap the MMAs of the next.  Every
// wait is bounded: on timeout the CTA raises a shared abort flag, records an error,
// waits (bounded) for the copies it issued, frees its tensor memory and returns.
#include "kernels_tma.hpp"

#include <cuda_bf16.h>

#include <algorithm>
#include <atomic>
#include <cstdint>
#include <mutex>
#include <thread>

namespace gbdmrg {

long tc_launch_count();
void count_tc_launches(long n);

namespace {

constexpr int TM_THREADS = 192;
constexpr int TM_BOX_K = 64;                       // columns per box (128 bytes)
constexpr int TM_A_BYTES = 128 * TM_BOX_K * 2;     // 16 KB
constexpr int TM_SLOT_A = 128 * TM_PACK_COLS * 2;  // packed mode: one piece of A (or B, n <= 128)
constexpr long TM_WAIT_LIMIT = 1L << 24;
constexpr int TM_REC_BATCH = 32;  // stages of the copy lists fetched per bulk copy

template <int MODE>
struct TmCfg {
  static constexpr bool STORE = MODE == TM_MODE_STORE_BF16;
  static constexpr bool EXACT = MODE == TM_MODE_EXACT_F64;
  // reduce mode: a stage holds up to TM_PACK_SLOTS pieces of 16 columns (32-byte swizzled
  // boxes), from any terms of the tile, one K=16 instruction each
  static constexpr bool PACK = MODE == TM_MODE_REDUCE_F32;
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

// the same for the packed pieces: K-major rows of TM_PACK_COLS columns, swizzled over
// their width (32 columns: 64-byte swizzle, 8-row groups 512 B apart; 16 columns: 32-byte
// swizzle, 256 B apart)
__device__ __forceinline__ uint64_t sdesc_pack(uint32_t saddr) {
  uint64_t d = 0;
  d |= (uint64_t)((saddr >> 4) & 0x3FFFu);
  d |= (uint64_t)1 << 16;
  d |= (uint64_t)((8 * TM_PACK_COLS * 2) >> 4) << 32;
  d |= (uint64_t)1 << 46;
  d |= (uint64_t)(TM_PACK_COLS == 32 ? 4 : 6) << 61;
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

// 1D bulk copy global -> shared (16-byte aligned addresses, size a multiple of 16), completing on bar
__device__ __forceinline__ void bulk_load(uint32_t dst, const void* src, uint32_t bytes, uint64_t* bar) {
  asm volatile("cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];\n" ::"r"(dst),
               "l"(src), "r"(bytes), "r"(smem_u32(bar))
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
                    int* __restrict__ err, const int* __restrict__ expo, const int* __restrict__ cta_stage,
                    const TmStage* __restrict__ stg, const TmPiece* __restrict__ pcs) {
  using Cfg = TmCfg<MODE>;
  constexpr int S = Cfg::STAGES;
  constexpr int STAGE_BYTES = Cfg::STAGE_BYTES;
  constexpr int NACC = Cfg::NACC;
  constexpr int NMAX = Cfg::NMAX;
  constexpr bool STORE = Cfg::STORE;
  constexpr bool EXACT = Cfg::EXACT;
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
  // copy lists of the producer: batches of TM_REC_BATCH stages, double-buffered, each
  // landing by bulk copy on rec_b[buffer]
  constexpr int PCS = Cfg::PACK ? TM_PACK_SLOTS : 1;
  __shared__ __align__(16) TmStage rec_stage[2][TM_REC_BATCH];
  __shared__ __align__(16) TmPiece rec_piece[2][TM_REC_BATCH * PCS];
  __shared__ __align__(8) uint64_t rec_b[2];
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
    mbar_init(&rec_b[0], 1);
    mbar_init(&rec_b[1], 1);
    abort_sh = 0;
    asm volatile("fence.mbarrier_init.release.cluster;\n" ::);
  }
  asm volatile("tcgen05.fence::before_thread_sync;\n" ::);
  __syncthreads();
  asm volatile("tcgen05.fence::after_thread_sync;\n" ::);
  const uint32_t tmem = tmem_base_sh;
  volatile int* abort_flag = &abort_sh;

  if (warp == 0) {
    // ---------------- TMA producer: the CTA's stages from the copy lists, fetched into
    // shared memory TM_REC_BATCH stages at a time by bulk copies one batch ahead.  Per
    // stage lane 0 waits until the ring slot is free and posts the stage word and the
    // expected bytes, then lane p < np issues the two box copies of piece p.
    constexpr int PIECES = PCS;
    constexpr uint32_t A_BOX = 128u * (Cfg::PACK ? TM_PACK_COLS : TM_BOX_K) * 2;
    constexpr unsigned FULL = 0xffffffffu;
    long j = 0;            // stages issued
    int st = 0;            // ring slot of the next one (j % S)
    uint32_t par = 0;      // its round's parity ((j / S) & 1)
    bool wrapped = false;  // j >= S
    bool ok = true;
    const int s_beg = cta_stage[blockIdx.x], s_end = cta_stage[blockIdx.x + 1];
    const int nbatch = (s_end - s_beg + TM_REC_BATCH - 1) / TM_REC_BATCH;
    int fetched = 0;  // record batches whose copies were issued
    auto fetch = [&](int b) {  // lane 0
      const int f0 = s_beg + b * TM_REC_BATCH, n = min(TM_REC_BATCH, s_end - f0);
      const uint32_t hb = (uint32_t)n * sizeof(TmStage), pb = (uint32_t)(n * PIECES) * sizeof(TmPiece);
      asm volatile("fence.proxy.async.shared::cta;\n" ::: "memory");
      mbar_arrive_expect_tx(&rec_b[b & 1], hb + pb);
      bulk_load(smem_u32(&rec_stage[b & 1][0]), stg + f0, hb, &rec_b[b & 1]);
      bulk_load(smem_u32(&rec_piece[b & 1][0]), pcs + (long)f0 * PIECES, pb, &rec_b[b & 1]);
    };
    if (lane == 0 && nbatch > 0) fetch(0);
    fetched = nbatch > 0 ? 1 : 0;
    for (int b = 0; b < nbatch && ok; ++b) {
      __syncwarp();  // the lanes' reads of the buffer batch b + 1 reuses are done
      if (lane == 0) {
        if (b + 1 < nbatch) fetch(b + 1);
        if (!mbar_wait(&rec_b[b & 1], (uint32_t)((b >> 1) & 1), abort_flag)) ok = false;
      }
      if (b + 1 < nbatch) fetched = b + 2;
      ok = __shfl_sync(FULL, ok, 0);
      if (!ok) break;
      const int f0 = s_beg + b * TM_REC_BATCH, n = min(TM_REC_BATCH, s_end - f0);
      for (int i = 0; i < n && ok; ++i) {
        const TmStage h = rec_stage[b & 1][i];
        if (lane == 0) {
          if (wrapped && !mbar_wait(&empty_b[st], par ^ 1u, abort_flag)) ok = false;
          if (ok) {
            meta[st] = h.word;
            mbar_arrive_expect_tx(&full_b[st], h.bytes);
          }
        }
        ok = __shfl_sync(FULL, ok, 0);
        if (!ok) break;
        if (lane < h.np) {
          const TmPiece q = rec_piece[b & 1][i * PIECES + lane];
          const uint32_t sa = base + st * STAGE_BYTES;
          tma_load_2d(sa + lane * A_BOX, maps + q.amap, q.ax, q.ay, &full_b[st]);
          tma_load_2d(sa + PIECES * A_BOX + lane * A_BOX, maps + q.bmap, q.bx, q.by, &full_b[st]);
        }
        ++j;
        if (++st == S) {
          st = 0;
          par ^= 1u;
          wrapped = true;
        }
      }
    }
    if (lane == 0) {
      // every issued copy must land before the CTA may exit: the last (up to S)
      // issued stages complete their full phase when their bytes arrive, and so does
      // the last record batch fetched
      for (long qq = j - 1; qq >= 0 && qq >= j - S; --qq) {
        const int s2 = (int)(qq % S);
        for (long it = 0; it < TM_WAIT_LIMIT && !mbar_test(&full_b[s2], (uint32_t)((qq / S) & 1)); ++it) {
        }
      }
      for (int b = max(0, fetched - 2); b < fetched; ++b)
        for (long it = 0; it < TM_WAIT_LIMIT && !mbar_test(&rec_b[b & 1], (uint32_t)((b >> 1) & 1)); ++it) {
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
      const uint64_t ad0 = Cfg::PACK ? sdesc_pack(base) : sdesc(base);
      const uint64_t bd0 = Cfg::PACK ? sdesc_pack(base + TM_PACK_SLOTS * TM_SLOT_A) : sdesc(base + TM_A_BYTES);
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
            // (packed) slot sl: A at sl * TM_SLOT_A, B at TM_PACK_SLOTS * TM_SLOT_A + sl *
            // TM_SLOT_A of the stage, its K=16 steps 32 bytes apart along the row
            const int nslot = Cfg::PACK ? nk : 1;
            int m = 0;
            for (int sl = 0; sl < nslot; ++sl) {
              const int nks = Cfg::PACK ? (int)((fl >> (12 + 2 * sl)) & 3u) : nk;
              const uint32_t idk = Cfg::PACK ? (id | (((fl >> (8 + sl)) & 1u) << 13)) : id;
              const uint64_t so = Cfg::PACK ? (uint64_t)((sl * TM_SLOT_A) >> 4) : 0;
              for (int kk = 0; kk < nks; ++kk, ++m) {
                const uint64_t ad = ad0 + off + so + (uint64_t)(kk * 2), bd = bd0 + off + so + (uint64_t)(kk * 2);
                const uint32_t accum = ((fl & 8u) && m == 0) ? 0u : 1u;
                asm volatile(
                    "{\n .reg .pred p;\n setp.ne.b32 p, %4, 0;\n"
                    " tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n}\n" ::"r"(dacc),
                    "l"(ad), "l"(bd), "r"(idk), "r"(accum));
              }
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
                        int* d_err, cudaStream_t s, const int* d_expo, const TmListsDev& lists) {
  static const bool attr_ok = cudaFuncSetAttribute(gemm_tma_kernel<MODE>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                                   TmCfg<MODE>::SMEM) == cudaSuccess;
  if (!attr_ok) return cudaErrorInvalidValue;
  // the lists were built for this grid: every CTA's tiles and stages
  if (lists.grid != tma_grid(ntiles) || !lists.cta_stage || !lists.stages || !lists.pieces)
    return cudaErrorInvalidValue;
  count_tc_launches(1);
  gemm_tma_kernel<MODE><<<lists.grid, TM_THREADS, TmCfg<MODE>::SMEM, s>>>(
      d_tiles, ntiles, d_terms, d_maps, d_rowmap, d_cbtab, out, out_slices, slice_stride, d_err, d_expo,
      lists.cta_stage, lists.stages, lists.pieces);
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
int tma_box_cols(int mode) { return mode == TM_MODE_REDUCE_F32 ? TM_PACK_COLS : TM_BOX_K; }

cudaError_t launch_gemm_tma(int mode, const TmTile* d_tiles, int ntiles, const TmTerm* d_terms,
                            const CUtensorMap* d_maps, const long* d_rowmap, const int2* d_cbtab, void* out,
                            int out_slices, long slice_stride, int* d_err, cudaStream_t s, const TmListsDev& lists,
                            const int* d_expo) {
  if (ntiles <= 0) return cudaSuccess;
  if (out_slices < 1 || out_slices > 3) return cudaErrorInvalidValue;
  if (mode == TM_MODE_STORE_BF16)
    return launch_mode<TM_MODE_STORE_BF16>(d_tiles, ntiles, d_terms, d_maps, d_rowmap, d_cbtab, out, out_slices,
                                           slice_stride, d_err, s, nullptr, lists);
  if (mode == TM_MODE_REDUCE_F32)
    return launch_mode<TM_MODE_REDUCE_F32>(d_tiles, ntiles, d_terms, d_maps, d_rowmap, d_cbtab, out, 1, 0, d_err, s,
                                           nullptr, lists);
  if (mode == TM_MODE_EXACT_F64) {
    if (!d_expo || !d_terms) return cudaErrorInvalidValue;
    return launch_mode<TM_MODE_EXACT_F64>(d_tiles, ntiles, d_terms, d_maps, d_rowmap, d_cbtab, out, 1, 0, d_err, s,
                                          d_expo, lists);
  }
  return cudaErrorInvalidValue;
}

int tma_grid(int ntiles) {
  static const int nsm = [] {
    int dev = 0, n = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || cudaDeviceGetAttribute(&n, cudaDevAttrMultiProcessorCount, dev) !=
                                                   cudaSuccess)
      return 148;
    return n > 0 ? n : 148;
  }();
  return ntiles < nsm ? ntiles : nsm;
}

int tma_pieces(int mode) { return mode == TM_MODE_REDUCE_F32 ? TM_PACK_SLOTS : 1; }

namespace {
__host__ __device__ inline long term_pieces(const TmTerm& m, int bc) {
  const int nsl = ((m.neg >> 4) & 15) > 1 ? ((m.neg >> 4) & 15) : 1;
  return (long)((m.k + bc - 1) / bc) * (nsl * (nsl + 1) / 2);
}

// One thread per stage.  It finds its tile (stages in the launch order: sorder[i] has
// the stages from sfirst[i]) and the term of its first piece (tpiece0: a term's first
// piece within its tile), then walks the stage's pieces: a term's pieces are its slice
// pairs (i, j), i + j < nsl, in level order, each its boxes along K.  Segments: store mode
// one per tile; reduce mode TM_SEG_KSTEPS stages each (the products accumulate in tensor
// memory over a segment only and the epilogue adds the segments in FP32 with
// round-to-nearest, so the rounding toward zero of the tensor-core accumulation acts on
// short sums); exact mode one per level of every term.
__global__ void fill_lists_kernel(int mode, const TmTile* __restrict__ tiles, int ntiles,
                                  const TmTerm* __restrict__ terms, const int* __restrict__ tpiece0,
                                  const int* __restrict__ sorder, const long* __restrict__ sfirst, long total,
                                  TmStage* __restrict__ stages, TmPiece* __restrict__ pieces) {
  const long g = (long)blockIdx.x * blockDim.x + threadIdx.x;
  if (g >= total) return;
  const bool pack = mode == TM_MODE_REDUCE_F32, exact = mode == TM_MODE_EXACT_F64;
  const int bc = pack ? TM_PACK_COLS : TM_BOX_K, P = pack ? TM_PACK_SLOTS : 1;
  int lo = 0, hi = ntiles - 1;  // the last tile (in stage order) starting at or before g
  while (lo < hi) {
    const int mid = (lo + hi + 1) >> 1;
    if (sfirst[mid] <= g) lo = mid; else hi = mid - 1;
  }
  const TmTile tl = tiles[sorder[lo]];
  const long sl = g - sfirst[lo];
  const long nst = (lo + 1 < ntiles ? sfirst[lo + 1] : total) - sfirst[lo];
  const long p0 = sl * P;
  int t = tl.t0, th = tl.t1 - 1;  // the last term whose first piece is at or before p0
  while (t < th) {
    const int mid = (t + th + 1) >> 1;
    if (tpiece0[mid] <= p0) t = mid; else th = mid - 1;
  }
  const long tile_pieces = tpiece0[tl.t1 - 1] + term_pieces(terms[tl.t1 - 1], bc);
  const int np = (int)min((long)P, tile_pieces - p0);
  const uint32_t a_box = 128u * bc * 2, b_box = (uint32_t)tl.n * bc * 2;
  const bool last = sl == nst - 1;
  TmTerm m = terms[t];
  long r = p0 - tpiece0[t];
  uint32_t negm = 0, nkm = 0, fl = 0, id = 0;
  for (int slot = 0; slot < np; ++slot, ++r) {
    if (r >= term_pieces(m, bc)) {
      m = terms[++t];
      r = 0;
    }
    const int nsl = max(1, (m.neg >> 4) & 15);
    const int kp = (m.k + bc - 1) / bc;
    int q = (int)(r / kp);
    const int kk = (int)(r - (long)q * kp);
    int l = 0;
    while (q > l) {
      q -= l + 1;
      ++l;
    }
    const int i = q, k0 = kk * bc;
    const int nk = min(bc / 16, (m.k - k0) / 16);
    pieces[g * P + slot] = TmPiece{m.amap + i, m.ax + k0, m.ay, m.bmap + (l - i), m.bx + k0, m.by, 0, 0};
    negm |= (uint32_t)(m.neg & 1) << slot;
    nkm |= (uint32_t)nk << (12 + 2 * slot);
    if (!pack) {
      fl = (uint32_t)nk;
      if (exact) {
        fl |= (i == 0 && kk == 0) ? 8u : 0u;
        fl |= (i == l && kk == kp - 1) ? 16u : 0u;
      } else {
        fl |= sl == 0 ? 8u : 0u;
        fl |= last ? 16u : 0u;
      }
      id = tm_idesc_bf16(tl.n, (m.neg & 1) != 0);
    }
  }
  for (int p = np; p < P; ++p) pieces[g * P + p] = TmPiece{0, 0, 0, 0, 0, 0, 0, 0};
  if (pack) {
    const long seg_pos = sl % TM_SEG_KSTEPS;
    fl = (uint32_t)np | (negm << 8) | nkm;
    fl |= seg_pos == 0 ? 8u : 0u;
    fl |= (last || seg_pos == TM_SEG_KSTEPS - 1) ? 16u : 0u;
    id = tm_idesc_bf16(tl.n, false);
  }
  fl |= last ? 32u : 0u;
  stages[g] = TmStage{(uint64_t)id | ((uint64_t)fl << 32), (uint32_t)np * (a_box + b_box), np};
}
}  // namespace

bool tma_plan_lists(int mode, std::vector<TmTile>& tiles, const std::vector<TmTerm>& terms, TmListPlan& out) {
  const int ntiles = (int)tiles.size();
  const int grid = ntiles > 0 ? tma_grid(ntiles) : 0;
  const int bc = tma_box_cols(mode), P = tma_pieces(mode);
  for (const TmTerm& m : terms)
    if (m.k < 16 || m.k % 16) return false;
  // every term belongs to one tile; its first piece within the tile
  out.tpiece0.assign(terms.size(), -1);
  std::vector<long> tst((size_t)ntiles);
  for (int ti = 0; ti < ntiles; ++ti) {
    const TmTile& tl = tiles[(size_t)ti];
    if (tl.t0 < 0 || tl.t1 <= tl.t0 || tl.t1 > (int)terms.size()) return false;
    long pc = 0;
    for (int t = tl.t0; t < tl.t1; ++t) {
      if (out.tpiece0[(size_t)t] >= 0 || pc >= (1L << 31)) return false;
      out.tpiece0[(size_t)t] = (int)pc;
      pc += term_pieces(terms[(size_t)t], bc);
    }
    tst[(size_t)ti] = (pc + P - 1) / P;
  }
  // stages in launch order: CTA c takes the tiles c, c + grid, ...
  out.grid = grid;
  out.cta_stage.assign((size_t)grid + 1, 0);
  out.sorder.clear();
  out.sfirst.clear();
  long total = 0;
  for (int c = 0; c < grid; ++c) {
    out.cta_stage[(size_t)c] = (int)total;
    for (int ti = c; ti < ntiles; ti += grid) {
      out.sorder.push_back(ti);
      out.sfirst.push_back(total);
      total += tst[(size_t)ti];
    }
    if (total >= (1L << 31) / P) return false;
  }
  out.cta_stage[(size_t)grid] = (int)total;
  out.total = total;
  if (mode == TM_MODE_REDUCE_F32)
    for (int ti = 0; ti < ntiles; ++ti) {
      tiles[(size_t)ti].pad = (int)tst[(size_t)ti];
      tiles[(size_t)ti].nseg = (int)((tst[(size_t)ti] + TM_SEG_KSTEPS - 1) / TM_SEG_KSTEPS);
    }
  return true;
}

cudaError_t launch_fill_lists(int mode, const TmTile* d_tiles, int ntiles, const TmTerm* d_terms, const int* d_tpiece0,
                              const int* d_sorder, const long* d_sfirst, long total, TmStage* d_stages,
                              TmPiece* d_pieces, cudaStream_t s) {
  if (ntiles <= 0 || total <= 0) return cudaSuccess;
  count_tc_launches(1);
  fill_lists_kernel<<<(unsigned)((total + 255) / 256), 256, 0, s>>>(mode, d_tiles, ntiles, d_terms, d_tpiece0, d_sorder,
                                                                    d_sfirst, total, d_stages, d_pieces);
  return cudaGetLastError();
}

bool encode_bf16_map(CUtensorMap* out, const void* base, uint64_t rows, uint64_t cols, uint64_t ld,
                     uint32_t box_rows, uint32_t box_cols) {
  EncodeTiledFn fn = encoder();
  if (!fn || rows == 0 || cols == 0 || (ld * 2) % 16 != 0 || ((uintptr_t)base & 15) != 0 || box_rows == 0 ||
      box_rows > 256 || (box_cols != 16 && box_cols != 32 && box_cols != (uint32_t)TM_BOX_K))
    return false;
  const cuuint64_t dims[2] = {cols, rows};
  const cuuint64_t strides[1] = {ld * 2};
  const cuuint32_t box[2] = {box_cols, box_rows};
  const cuuint32_t estr[2] = {1, 1};
  return fn(out, CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, 2, const_cast<void*>(base), dims, strides, box, estr,
            CU_TENSOR_MAP_INTERLEAVE_NONE,
            box_cols == 16 ? CU_TENSOR_MAP_SWIZZLE_32B
                           : (box_cols == 32 ? CU_TENSOR_MAP_SWIZZLE_64B : CU_TENSOR_MAP_SWIZZLE_128B),
            CU_TENSOR_MAP_L2_PROMOTION_L2_256B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) == CUDA_SUCCESS;
}

}  // namespace gbdmrg
