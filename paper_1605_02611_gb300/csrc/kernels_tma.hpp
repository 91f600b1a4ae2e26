// TMA-staged tensor-core grouped GEMM (tcgen05, BF16 in, FP32 accumulate) for
// the single-pass sigma vector of the group-stacked layout.
#pragma once
#include <cuda.h>  // CUtensorMap (type only; the encoder is reached through the runtime)
#include <cuda_bf16.h>
#include <cuda_runtime.h>

#include <cstdint>

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
//   store mode (X intermediates, BF16): the output matrix is split by columns into
//     column blocks, each its own row-major submatrix of xrows rows: block e of
//     cbtab[cb0..cb1) = (first column c0, width w) starts at element
//     xbase + xrows * c0 and holds column c at (c - c0) of its rows.  Row r of the
//     tile is row rowmap[rowmap_off + r] of the submatrices (< 0: skipped); its
//     columns are out_off .. out_off + n (every 8-column chunk inside one block).
//   reduce mode (sigma^T, FP32): rows r < m_valid are added (vector reductions) to
//     out + out_off + r * ldo, columns [0, n).
//   nseg (reduce mode): segments of the tile, ceil(K steps / TM_SEG_KSTEPS) with one K
//     step per 64 columns of every term; each segment accumulates in tensor memory
//     on its own and the epilogue adds the segments in FP32.
struct TmTile {
  int t0, t1;
  int n, m_valid;
  int ldo, nseg;
  long out_off;
  long rowmap_off;
  long xbase, xrows;
  int cb0, cb1;
  int nvalid, pad;  // exact mode: valid columns of the output block
};

//   exact mode (FP64): rows r < m_valid, columns c < nvalid of
//     out + out_off + r * ldo receive the sum of the tile's segments, accumulated in
//     two-float (hi + lo) registers and stored as FP64.
constexpr int TM_MODE_STORE_BF16 = 1, TM_MODE_REDUCE_F32 = 2, TM_MODE_EXACT_F64 = 3;
// bits of the slices of the exact mode
constexpr int TM_EXACT_BITS = 7;
// K steps (64 columns each) accumulated in tensor memory before the reduce-mode
// epilogue takes the partial sum over
constexpr int TM_SEG_KSTEPS = 16;

// maps: device array of encoded tensor maps (64-byte aligned).  Store mode:
// out_slices (1-3) BF16 slices x = s0 + s1 + ... of every FP32 result, written
// slice_stride elements apart.  err: set to 1 if a bounded wait ran out (the CTA
// then stops, lets its copies land and frees its tensor memory).
cudaError_t launch_gemm_tma(int mode, const TmTile* d_tiles, int ntiles, const TmTerm* d_terms,
                            const CUtensorMap* d_maps, const long* d_rowmap, const int2* d_cbtab, void* out,
                            int out_slices, long slice_stride, int* d_err, cudaStream_t s,
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

// Host: encode a 2D BF16 tensor map over a row-major matrix (rows x cols, leading
// dimension ld elements, ld * 2 a multiple of 16 bytes, base 16-byte aligned), box
// of 64 columns x box_rows rows, 128-byte swizzle.  Returns false on failure.
bool encode_bf16_map(CUtensorMap* out, const void* base, uint64_t rows, uint64_t cols, uint64_t ld,
                     uint32_t box_rows);

}  // namespace gbdmrg
