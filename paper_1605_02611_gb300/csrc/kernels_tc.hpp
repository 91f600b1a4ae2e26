// Tensor-core grouped block GEMM (tcgen05, BF16 in, FP32 accumulate).
#pragma once
#include <cuda_bf16.h>
#include <cuda_runtime.h>

namespace gbdmrg {

// C[m x n] (+)= sum_t (-1)^{neg_t} A_t[m x k_t] B_t[n x k_t]^T; A, B row-major bf16 with
// leading dimensions (elements) multiples of 8, 16-byte aligned.  Columns are read
// in 16-byte chunks up to the first multiple of 8 at or above k_t (never beyond
// ld); over the columns between k_t and that multiple one operand must be zero
// and the other finite.
// With nsl > 1 the operands are nsl BF16 slices (x = s_0 + s_1 + ...) stored sA / sB
// elements apart, and the term contributes sum_{i + j < nsl} A_i B_j^T.
struct TcTerm {
  const __nv_bfloat16* A;
  const __nv_bfloat16* B;
  long sA, sB;
  int lda, ldb, k, flags;  // flags bit 0: negate
  int nsl;
};
// outputs: C (fp32, optional, += if beta) and/or Cb (bf16, optional): nslices bf16
// slices x = s0 + s1 + s2 written slice_stride elements apart.  trans: element
// (i, j) of the block goes to [j * ld + i] instead of [i * ld + j].  beta == 2:
// FP32 atomic accumulation into C (several tasks may split one block's term list).
struct TcTask {
  float* C;
  __nv_bfloat16* Cb;
  long slice_stride;
  int ldc, ldcb, m, n, beta, nslices, trans, t0, t1;
};
struct TcTile {
  int task, r0, c0;
};
constexpr int TC_TILE_M = 128, TC_TILE_N = 128;

// nsl: the largest slice count of any term in the list (1, 2 or 3)
cudaError_t launch_gemm_bf16_tc(const TcTile* d_tiles, int ntiles, const TcTask* d_tasks, const TcTerm* d_terms,
                                int* d_err, cudaStream_t s, int nsl = 1);
long tc_launch_count();
void count_tc_launches(long n);

}  // namespace gbdmrg
