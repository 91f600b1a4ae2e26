// Learned Davidson preconditioner: a 3-layer GELU network g(f) that rescales the
// diagonal correction element by element, t_i = (1 + g(f_i)) r_i / (theta - d_i).
//
// Features f_i (per element of psi, with quantum-number-block context; n the
// number of elements, b the block of element i, delta_i = d_i - theta):
//   f0 = r_i sqrt(n) / |r|,  f1 = asinh(delta_i),  f2 = delta_i / (delta_i^2 + 0.01),
//   f3 = asinh(rms_b(r) sqrt(n) / |r|),  f4 = asinh(mean_b(d) - theta).
// Network: a1 = W1 f + b1, h1 = gelu(a1); a2 = W2 h1 + b2, h2 = gelu(a2);
// g = W3 . h2 + b3, hidden width 256, gelu(x) = x Phi(x).
//
// Training pairs are generated by the method: for a Ritz vector x_j of a
// Davidson iteration and the converged vector psi, the exact correction with
// unit weight on x_j is tau = psi / (x_j . psi) - x_j.  A pair holds f, P = p s
// and T = tau s (p the diagonal correction, s = sqrt(n) / |tau|, both clipped
// to [-100, 100]); the loss is mean(((1 + g) P - T)^2).
//
// Numerics: training runs in FP32 on the CUDA cores with the weights rounded to
// BF16 in the forward pass (FP32 master copy, straight-through gradient).
// Inference stores h1 in BF16 and runs the 256 x 256 layer on the tensor cores
// (tcgen05, FP32 accumulation); the rest is FP32, the correction FP64.
#pragma once
#include <cuda_bf16.h>
#include <cuda_runtime.h>

#include <cstdint>

#include "engine.hpp"
#include "kernels_tc.hpp"

namespace gbdmrg {

constexpr int MLP_H = 256, MLP_F = 5;
constexpr long MLP_OFF_W1 = 0;
constexpr long MLP_OFF_B1 = MLP_OFF_W1 + (long)MLP_H * MLP_F;
constexpr long MLP_OFF_W2 = MLP_OFF_B1 + MLP_H;
constexpr long MLP_OFF_B2 = MLP_OFF_W2 + (long)MLP_H * MLP_H;
constexpr long MLP_OFF_W3 = MLP_OFF_B2 + MLP_H;
constexpr long MLP_OFF_B3 = MLP_OFF_W3 + MLP_H;
constexpr long MLP_NPARAMS = MLP_OFF_B3 + 1;

struct Mlp {
  cudaStream_t stream = nullptr;
  bool own_stream = false;
  DArr<float> w;                 // FP32 master parameters (flat layout above)
  DArr<float> wq;                // forward copy: weights rounded to BF16, biases exact
  DArr<__nv_bfloat16> w2b;       // W2 in BF16, row = output neuron (tensor-core operand)
  DArr<float> grad, am, av;      // gradient and Adam moments
  long adam_t = 0;
  DArr<int> err;                 // tensor-core kernel wait flag
  // training scratch, sized for `cap` samples
  long cap = 0;
  DArr<float> Fb, Pb, Tb, A1, H1, A2, H2, G, dA2, dH1;
  DArr<double> acc;
  ~Mlp();
};

void mlp_init(Mlp& m, uint64_t seed, cudaStream_t s);
void mlp_set_params(Mlp& m, const float* host);
void mlp_get_params(Mlp& m, float* host);
// forward pass of the training numerics (FP32) or of the inference numerics
// (BF16 h1, tensor-core layer 2) on features F [n x 5] (device) -> g [n] (device)
void mlp_forward(Mlp& m, const float* F, long n, float* g, bool inference);
// loss and gradient (into m.grad) of the samples F, P, T (device); returns the loss
double mlp_loss_grad(Mlp& m, const float* F, const float* P, const float* T, long n);
// Adam on minibatches drawn with replacement (counter-based hash of seed, step,
// sample); mean loss of the first and of the last epoch
void mlp_train(Mlp& m, const float* F, const float* P, const float* T, long n, int epochs, int batch, float lr,
               uint64_t seed, double* first, double* last);

// per-problem scratch of inference and pair generation
struct MlpScratch {
  long n = 0;
  int nb = 0;
  DArr<long> boff;        // nb + 1 block offsets of psi
  DArr<double> bsum;      // per block: sum of r^2
  DArr<double> bmean;     // per block: mean of the diagonal
  long chunk = 0;
  DArr<__nv_bfloat16> H1; // chunk x 256
  DArr<float> Z;          // chunk x 256
  DArr<TcTile> tiles;     // tiles of a full chunk, then those of the last chunk
  DArr<TcTask> tasks;     // [0] full chunk, [1] last chunk
  DArr<TcTerm> terms;     // [0]: H1 x W2^T
  int ntiles_full = 0, ntiles_last = 0;
  DArr<int> flag;
  DArr<double> tmp;       // n: tau for pair generation
};

// m == nullptr: pair generation only (no inference buffers)
void mlp_scratch_build(MlpScratch& s, const Mlp* m, const PsiLayout& P, cudaStream_t st);
// block means of the diagonal (once per diagonal)
void mlp_scratch_set_diag(MlpScratch& s, const double* d, cudaStream_t st);
// t = (1 + g(f)) r / (theta - d); false when a network output was not finite
bool mlp_precondition(Mlp& m, MlpScratch& s, const double* r, const double* d, double theta, double rnorm, double* t,
                      cudaStream_t st);
// training pairs at `ns` elements drawn by a counter-based hash of `seed`:
// features, P, T and the element index (device outputs; idx may be null).
// Returns ns, or 0 (nothing written) when |x . psi| < min_overlap or x = psi.
long mlp_make_pairs(MlpScratch& s, const double* x, const double* r, const double* d, double theta, double rnorm,
                    const double* psi, long ns, uint64_t seed, float* F, float* P, float* T, long* idx,
                    double min_overlap, cudaStream_t st);

}  // namespace gbdmrg
