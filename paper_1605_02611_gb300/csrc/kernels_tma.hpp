// TMA-staged tensor-core grouped GEMM (tcgen05, BF16 in, FP32 accumulate) for
// the single-pass sigma vector of the group-stacked layout.
#pragma once
#include <cuda.h>  // CUtensorMap (type only; the encoder is reached through the runtime)
#include <cuda_bf16.h>
#include <cuda_runtime.h>

#include <cstdint>
#include <vector>

namespace gbdmrg {

// One term of an output tile: C[128 x n] (-)= A[128 x k] B[n x k]^T (neg bit 0), where A is the
// box of rows [ay, ay + 128) and columns [ax, ax + k) of tensor map amap and B the
// rows [by, by + n) and columns [bx, bx + k) of tensor map bmap (both BF16,
// row-major, 128-byte swizzled boxes of 64 columns; rows or columns outside a
// map's extent read as zero).  k is a multiple of 16; columns of a 64-wide box
// past k are loaded but never multiplied.  The B map's box height must be the
// tile's n.
//
// Exact mode (TM_MODE_EXACT_F64): the operands are integer slices (|x| <= 128, exact in
// BF16) of blocks scaled by powers of two, so every product sum is an exact integer in
// the FP32 accumulator.  A term stands for all slice pairs (i, j), i + j < nsl (neg
// bits 4-7; slice i of map m is map m + i), taken level by level: the pairs of level
// l = i + j form one segment, added with weight 2^(expo[ea] + expo[eb] - 7 (l + 2));
// neg bit 0 negates.  k <= 128, so that the sums stay below 2^24.
struct TmTerm {
  int amap, bmap;
  int ax, ay, bx, by;
  int k, neg;
  int ea, eb;
};

// Output tile over the terms [t0, t1).  n: MMA width (multiple of 16, <= the
// kernel's maximum).
//   reduce mode (packed): the tensor maps of the tile's terms have boxes of TM_PACK_COLS
//     columns, and a K step (stage) holds up to TM_PACK_SLOTS consecutive pieces of the
//     tile (a term has ceil(k / TM_PACK_COLS) pieces per slice pair); pad = the tile's
//     stages, ceil(pieces / TM_PACK_SLOTS).
//   store mode (X intermediates, BF16): the output matrix is split by columns into
//     column blocks, each its own row-major submatrix of xrows rows: block e of
//     cbtab[cb0..cb1) = (first column c0, width w) starts at element
//     xbase + xrows * c0 and holds column c at (c - c0) of its rows.  Row r of the
//     tile is row rowmap[rowmap_off + r] of the submatrices (< 0: skipped); its
//     columns are out_off .. out_off + n (every 8-column chunk inside one block).
//   reduce mode (sigma^T, FP32): rows r < m_valid are added (vector reductions) to
//     out + out_off + r * ldo, columns [0, n).
//   nseg (reduce mode): segments of the tile, ceil(stages / TM_SEG_KSTEPS); each segment
//     accumulates in tensor memory on its own and the epilogue adds the segments in FP32.
struct TmTile {
  int t0, t1;
  int n, m_valid;
  int ldo, nseg;
  long out_off;
  long rowmap_off;
  long xbase, xrows;
  int cb0, cb1;
  int nvalid, pad;  // exact mode: valid columns of the output block; reduce mode: pad = pieces
};

//   exact mode (FP64): rows r < m_valid, columns c < nvalid of
//     out + out_off + r * ldo receive the sum of the tile's segments, accumulated in
//     two-float (hi + lo) registers and stored as FP64.
constexpr int TM_MODE_STORE_BF16 = 1, TM_MODE_REDUCE_F32 = 2, TM_MODE_EXACT_F64 = 3;
// bits of the slices of the exact mode
constexpr int TM_EXACT_BITS = 7;
// K steps (stages of up to TM_PACK_SLOTS 16-column pieces) accumulated in tensor memory
// before the reduce-mode epilogue takes the partial sum over
constexpr int TM_SEG_KSTEPS = 16;
constexpr int TM_PACK_SLOTS = 4;  // pieces per stage of the reduce mode
constexpr int TM_PACK_COLS = 16;  // their width (32-byte swizzled boxes), one K=16 instruction each

// Copy lists.  The tiles' terms are expanded on the host into stages, each holding up
// to tma_pieces(mode) pieces (a piece: one A box and one B box, both of tma_box_cols(mode)
// columns; store and exact modes one piece of 64 columns, reduce mode up to
// TM_PACK_SLOTS consecutive pieces of TM_PACK_COLS columns).  A term expands into its slice pairs
// (i, j), i + j < nsl, in the order of the level l = i + j (A map amap + i, B map
// bmap + j), each into its boxes along K.  CTA c of a launch of `grid` CTAs takes the
// tiles c, c + grid, ... and issues the stages [cta_stage[c], cta_stage[c + 1]), stage s
// with the pieces pieces[s * tma_pieces(mode) + p], p < np.
struct TmPiece {  // 32 bytes, so that any run of pieces is a bulk copy of 16-byte multiples
  int amap, ax, ay, bmap, bx, by, pad0, pad1;
};
// word: the stage word the MMA issuer reads, the instruction descriptor (negation of A in
// the store and exact modes) in the low half, in the high half the K=16 instructions
// (store and exact modes; the pieces in the reduce mode) in bits 0-2, flags first of a
// segment (bit 3), end of a segment (4), last stage of the tile (5), and in the reduce
// mode the negation of slot p in bit 8 + p and its K=16 instructions in bits 12 + 2p and
// 13 + 2p.  bytes: the stage's expected copy bytes.
struct TmStage {
  uint64_t word;
  uint32_t bytes;
  int np;
};
struct TmListsDev {  // device copies, kept alive by the caller for the launches
  int grid = 0;
  const int* cta_stage = nullptr;
  const TmStage* stages = nullptr;
  const TmPiece* pieces = nullptr;
};
// host side of a launch's lists: its grid, every CTA's first stage (grid + 1 entries),
// the tiles in stage order (sorder) with their first stages (sfirst), and every term's
// first piece within its tile (tpiece0; a term belongs to one tile)
struct TmListPlan {
  int grid = 0;
  long total = 0;
  std::vector<int> cta_stage;
  std::vector<int> sorder;
  std::vector<long> sfirst;
  std::vector<int> tpiece0;
};

// instruction descriptor of tcgen05.mma kind::f16: D FP32, A and B BF16, both K-major,
// M = 128, N = n; negA negates A
__host__ __device__ inline uint32_t tm_idesc_bf16(int n, bool negA) {
  uint32_t d = 0;
  d |= 1u << 4;
  d |= 1u << 7;
  d |= 1u << 10;
  if (negA) d |= 1u << 13;
  d |= (uint32_t)(n >> 3) << 17;
  d |= (uint32_t)(128 >> 4) << 24;
  return d;
}

// Host: the stage counts of a launch of `mode` over these tiles (for the grid the launch
// will use, tma_grid(tiles.size())); reduce mode: sets every tile's pad (its stages) and
// nseg.  Returns false if a term is malformed (k not a positive multiple of 16), belongs
// to two tiles, or the lists would be too long.
bool tma_plan_lists(int mode, std::vector<TmTile>& tiles, const std::vector<TmTerm>& terms, TmListPlan& out);
// Device: fills the copy lists (stages: total entries, pieces: total * tma_pieces(mode)),
// one thread per stage, from the tiles and terms the plan was made from and the plan's
// tpiece0, sorder and sfirst (all on the device).
cudaError_t launch_fill_lists(int mode, const TmTile* d_tiles, int ntiles, const TmTerm* d_terms, const int* d_tpiece0,
                              const int* d_sorder, const long* d_sfirst, long total, TmStage* d_stages,
                              TmPiece* d_pieces, cudaStream_t s);
// CTAs of a launch over ntiles tiles (min(ntiles, SMs of the current device))
int tma_grid(int ntiles);
int tma_pieces(int mode);

// maps: device array of encoded tensor maps (64-byte aligned).  Store mode:
// out_slices (1-3) BF16 slices x = s0 + s1 + ... of every FP32 result, written
// slice_stride elements apart.  err: set to 1 if a bounded wait ran out (the CTA
// then stops, lets its copies land and frees its tensor memory).  lists: the copy lists
// of these tiles (tma_plan_lists, launch_fill_lists), on the device.  d_terms: read by the exact mode's
// epilogue only.
cudaError_t launch_gemm_tma(int mode, const TmTile* d_tiles, int ntiles, const TmTerm* d_terms,
                            const CUtensorMap* d_maps, const long* d_rowmap, const int2* d_cbtab, void* out,
                            int out_slices, long slice_stride, int* d_err, cudaStream_t s, const TmListsDev& lists,
                            const int* d_expo = nullptr);

// Exact splitting of FP64 blocks for the exact mode: per job, e = the smallest
// exponent with |scale * x| < 2^e over the block, then nsl (1 to 6) integer slices d_s
// with scale * x * 2^-e = sum_s d_s 2^(-7 (s + 1)) (+ remainder below 2^(-7 nsl)), each
// stored exactly as BF16 (|d_0| <= 128, |d_3| <= 72, the others <= 64), nsl slices
// slice_stride elements apart; columns
// [cols, wcols) are zero.  trans: dst[j * ldd + i] holds element (i, j) (rows of
// the source become columns).  expo[job.expo] receives e.
struct SplitJob {
  const double* src;
  __nv_bfloat16* dst;
  long slice_stride;
  int rows, cols, lds, ldd, wcols, trans, expo;
  double scale;
};
cudaError_t launch_split_exact(const SplitJob* d_jobs, int njobs, int nsl, int* d_expo, cudaStream_t s);
// maximum MMA width of a mode (256 for the BF16 store mode, 128 for the reduce mode)
int tma_max_n(int mode);
// box width in columns of the tensor maps a mode reads (TM_PACK_COLS for the reduce mode,
// else 64)
int tma_box_cols(int mode);

// Host: encode a 2D BF16 tensor map over a row-major matrix (rows x cols, leading
// dimension ld elements, ld * 2 a multiple of 16 bytes, base 16-byte aligned), box
// of box_cols columns x box_rows rows: 64, 32 or 16 columns with 128-, 64- or 32-byte
// swizzle.  Returns false on failure.
bool encode_bf16_map(CUtensorMap* out, const void* base, uint64_t rows, uint64_t cols, uint64_t ld,
                     uint32_t box_rows, uint32_t box_cols = 64);

}  // namespace gbdmrg
