// Diagonal of H_eff without any device allocation.
//
// Some callers cannot allocate device memory at the time they need the
// preconditioner input: for example code inside a framework whose memory
// manager owns the whole device and forbids cudaMalloc/cudaFree between its
// own phases.  For them this variant of compute_diag keeps every scratch
// buffer it needs (the gathered diagonals of the W-contracted operators and
// the GEMM work lists) in one file-scope device array of fixed size,
// NOALLOC_SCRATCH_BYTES.  The array lives in the module image, so every GPU
// that loads the library holds it until the process exits.
//
// Host code cannot use the array's name as a device address (in host code it
// names a host-side stand-in); the device address is obtained once per device
// with cudaGetSymbolAddress, with that device current, by the first call made
// on that device.  That first call should therefore come before any stream
// capture.  All calls share the one array (and one host staging buffer for the
// work lists) and it keeps the contents of the last call: everything that must
// start at zero is cleared on every call.  Calls whose GPU work overlapped would
// race on the shared array, even calls for different GPUs (they share the host
// staging); a process-wide lock held from staging until the call's own GPU work
// has finished makes calls from several host threads run one after another.
#include <cuda_runtime.h>

#include <algorithm>
#include <cstring>
#include <mutex>
#include <string>

#include "engine.hpp"
#include "kernels.hpp"

namespace gbdmrg {

constexpr size_t NOALLOC_SCRATCH_BYTES = (size_t)32 << 20;  // 32 MiB

static __device__ __align__(256) unsigned char g_noalloc_scratch[NOALLOC_SCRATCH_BYTES];

namespace {

constexpr int kMaxDevices = 64;
std::mutex g_setup_mu;
void* g_scratch_dev[kMaxDevices] = {nullptr};
// held by a call from staging its work lists until its GPU work has finished
std::mutex g_call_mu;

// host staging for the descriptor lists (also fixed size: no host allocation)
unsigned char g_stage[NOALLOC_SCRATCH_BYTES];

void* scratch_address() {
  int dev = 0;
  cuda_check(cudaGetDevice(&dev), "cudaGetDevice");
  if (dev < 0 || dev >= kMaxDevices) throw Error(ST_EINVAL, "device index out of range for the no-allocation scratch");
  std::lock_guard<std::mutex> lk(g_setup_mu);
  if (!g_scratch_dev[dev]) {
    void* p = nullptr;
    cudaError_t e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
    if (e != cudaSuccess || !p)
      throw Error(ST_ECUDA, std::string("cudaGetSymbolAddress of the no-allocation scratch: ") + cudaGetErrorString(e));
    g_scratch_dev[dev] = p;
  }
  return g_scratch_dev[dev];
}

inline size_t align256(size_t x) { return (x + 255) & ~(size_t)255; }

}  // namespace

size_t noalloc_scratch_bytes() { return NOALLOC_SCRATCH_BYTES; }

// Same arithmetic as compute_diag: diag[l n1 n2 r] = sum over the dQ = 0 states beta of
// Lt_beta^{n1 n1}[l, l] * Rt_beta^{n2 n2}[r, r], as one GEMM per psi block with the
// contraction over beta.
void compute_diag_noalloc(Context& c, double* diag) {
  if (c.prepared < 0) throw Error(ST_ESTATE, "call gbdmrg_prepare first");
  const int k = c.prepared;
  Tilde& lt = c.lt;
  Tilde& rt = c.rt;
  const PsiLayout& P = c.plan.psi;
  const auto& mid = c.mpo.bonds[k + 1];
  Env& Lenv = *lt.env;
  Env& Renv = *rt.env;
  const Bond& Lb = Lenv.bond;
  const Bond& Rb = Renv.bond;
  int nz = 0;
  for (size_t beta = 0; beta < mid.size(); ++beta)
    if (mid[beta].dna == 0 && mid[beta].dnb == 0) ++nz;
  // sizes of every region before touching the GPU
  size_t njobs = 0;
  int mx = 0;
  for (size_t beta = 0; beta < mid.size(); ++beta) {
    if (mid[beta].dna != 0 || mid[beta].dnb != 0) continue;
    for (int n = 0; n < 4; ++n) {
      for (int side = 0; side < 2; ++side) {
        const TRef& r = side == 0 ? lt.ref[beta][n * 5] : rt.ref[beta][n * 5];
        if (!r.p) continue;
        const OpLayout& Lay = side == 0 ? Lenv.cls[r.cls] : Renv.cls[r.cls];
        for (const Block& b : Lay.blocks)
          if (b.rs == b.cs) {
            ++njobs;
            mx = std::max(mx, b.rows);
          }
      }
    }
  }
  size_t nblk = P.blocks.size(), ntiles = 0;
  for (const Block& b : P.blocks)
    ntiles += (size_t)((b.rows + GEMM_TM - 1) / GEMM_TM) * ((b.cols + GEMM_TN - 1) / GEMM_TN);
  const size_t dl_bytes = align256((size_t)4 * Lb.total * nz * sizeof(double));
  const size_t dr_bytes = align256((size_t)4 * Rb.total * nz * sizeof(double));
  const size_t jobs_bytes = align256(njobs * sizeof(DiagJob));
  const size_t tile_bytes = align256(ntiles * sizeof(GemmTile));
  const size_t task_bytes = align256(nblk * sizeof(GemmTask));
  const size_t term_bytes = align256(nblk * sizeof(GemmTerm));
  const size_t need = dl_bytes + dr_bytes + jobs_bytes + tile_bytes + task_bytes + term_bytes;
  if (need > NOALLOC_SCRATCH_BYTES)
    throw Error(ST_EINVAL, "problem too large for the no-allocation diagonal: needs " + std::to_string(need) +
                               " bytes of scratch, the fixed scratch holds " +
                               std::to_string(NOALLOC_SCRATCH_BYTES) + " bytes");
  std::lock_guard<std::mutex> call_lock(g_call_mu);
  unsigned char* base = (unsigned char*)scratch_address();
  double* DL = (double*)base;
  double* DR = (double*)(base + dl_bytes);
  unsigned char* dsc = base + dl_bytes + dr_bytes;  // descriptor region (device)
  cuda_check(cudaMemsetAsync(diag, 0, P.nnz * sizeof(double), c.stream), "memset");
  if (nz == 0) {
    cuda_check(cudaStreamSynchronize(c.stream), "sync");
    return;
  }
  cuda_check(cudaMemsetAsync(DL, 0, dl_bytes + dr_bytes, c.stream), "memset");
  // descriptors staged in fixed host memory, copied into the device scratch
  DiagJob* hj = (DiagJob*)g_stage;
  size_t j = 0;
  int z = 0;
  for (size_t beta = 0; beta < mid.size(); ++beta) {
    if (mid[beta].dna != 0 || mid[beta].dnb != 0) continue;
    for (int n = 0; n < 4; ++n) {
      const TRef& rl = lt.ref[beta][n * 5];
      if (rl.p)
        for (const Block& b : Lenv.cls[rl.cls].blocks)
          if (b.rs == b.cs)
            hj[j++] = {rl.p + b.off, DL + ((size_t)n * Lb.total + Lb.off[b.rs]) * nz + z, b.rows, b.cols, nz, rl.coef};
      const TRef& rr = rt.ref[beta][n * 5];
      if (rr.p)
        for (const Block& b : Renv.cls[rr.cls].blocks)
          if (b.rs == b.cs)
            hj[j++] = {rr.p + b.off, DR + ((size_t)n * Rb.total + Rb.off[b.rs]) * nz + z, b.rows, b.cols, nz, rr.coef};
    }
    ++z;
  }
  GemmTile* ht = (GemmTile*)(g_stage + jobs_bytes);
  GemmTask* hk = (GemmTask*)(g_stage + jobs_bytes + tile_bytes);
  GemmTerm* hm = (GemmTerm*)(g_stage + jobs_bytes + tile_bytes + task_bytes);
  size_t t = 0;
  double flops = 0;
  for (size_t pb = 0; pb < nblk; ++pb) {
    const Block& ob = P.blocks[pb];
    const int n1 = P.b1[pb], n2 = P.b2[pb];
    flops += 2.0 * ob.rows * ob.cols * nz;  // counted like compute_diag's grouped GEMM
    hk[pb] = {diag + ob.off, ob.cols, ob.rows, ob.cols, 0, (int)pb, (int)pb + 1};
    hm[pb] = {DL + ((size_t)n1 * Lb.total + Lb.off[ob.rs]) * nz, DR + ((size_t)n2 * Rb.total + Rb.off[ob.cs]) * nz, nz,
              nz, nz, 0, 1.0};
    for (int r0 = 0; r0 < ob.rows; r0 += GEMM_TM)
      for (int c0 = 0; c0 < ob.cols; c0 += GEMM_TN) ht[t++] = {(int)pb, r0, c0};
  }
  const size_t dsc_bytes = jobs_bytes + tile_bytes + task_bytes + term_bytes;
  cuda_check(cudaMemcpyAsync(dsc, g_stage, dsc_bytes, cudaMemcpyHostToDevice, c.stream), "h2d");
  launch_diag_extract((const DiagJob*)dsc, (int)njobs, mx, c.stream);
  cuda_check(cudaGetLastError(), "diag extract");
  launch_gemm((const GemmTile*)(dsc + jobs_bytes), (int)ntiles, (const GemmTask*)(dsc + jobs_bytes + tile_bytes),
              (const GemmTerm*)(dsc + jobs_bytes + tile_bytes + task_bytes), c.stream);
  cuda_check(cudaGetLastError(), "gemm launch");
  // the host staging buffer is reused by the next call: wait for the copy and the kernels
  cuda_check(cudaStreamSynchronize(c.stream), "sync");
  c.other_flops_total += flops;
}

}  // namespace gbdmrg
