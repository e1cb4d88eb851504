// sfs_apply_AH_noalloc: the backward projection x = A^H y for callers that
// cannot allocate device memory at call time.
//
// Who needs it: acquisition or real-time loops that forbid allocation after
// start-up so that every call has the same latency, and host frameworks that
// own all device memory through their own pool and must not see a library
// allocate behind their back.  These callers create the operator once at
// set-up time and afterwards need calls that touch no allocator at all.
//
// sfs_apply_AH keeps its intermediate data (the lateral spectra of the bin
// planes and the adjoint contraction's partial-sum slots) in workspace that
// the operator allocated.  This variant keeps them instead in one file-scope
// __device__ array of fixed size (kNoAllocScratchBytes, 32 MiB), which every
// GPU that loads this library holds until the process exits.  The call
// itself performs no cudaMalloc, cudaFree or other allocating call.
#include <cuda_runtime.h>

#include <mutex>

#include "sfs_internal.h"

namespace sfs {
namespace {

constexpr size_t kNoAllocScratchBytes = SFS_NOALLOC_SCRATCH_BYTES;
constexpr size_t kNoAllocScratchElems = kNoAllocScratchBytes / sizeof(float2);

// Shared by every call on every operator of this device: calls whose device
// work overlaps in time race on it.
static __device__ __align__(256) float2 g_ah_scratch[kNoAllocScratchElems];

// Device address of g_ah_scratch per device ordinal (the host-side symbol is
// only a stand-in and must never be passed to a kernel).
std::mutex g_mu;
float2* g_scratch_dev[64] = {};

int scratch_for_current_device(float2** out) {
  int dev = 0;
  SFS_CUDA(cudaGetDevice(&dev));
  if (dev < 0 || dev >= 64) {
    set_error("device ordinal %d out of range for the static scratch table", dev);
    return SFS_ERR_INVALID_ARG;
  }
  std::lock_guard<std::mutex> lock(g_mu);
  if (!g_scratch_dev[dev]) {
    void* p = nullptr;
    SFS_CUDA(cudaGetSymbolAddress(&p, g_ah_scratch));
    g_scratch_dev[dev] = (float2*)p;
  }
  *out = g_scratch_dev[dev];
  return SFS_OK;
}

}  // namespace
}  // namespace sfs

using namespace sfs;

extern "C" int sfs_apply_AH_noalloc(sfs_operator* op, const void* y_dev, void* x_dev,
                                    void* stream) {
  clear_error();
  if (!op || !y_dev || !x_dev || ((uintptr_t)y_dev & 15u) || ((uintptr_t)x_dev & 15u)) {
    set_error("null or misaligned argument");
    return SFS_ERR_INVALID_ARG;
  }
  // the bin-plane spectra [Up][Ns] followed by the adjoint slots [nslots][azb][64]
  const size_t n_rh = (size_t)op->Up * op->Ns;
  const size_t n_slots = (size_t)op->nslots * op->azb * kKappaTile;
  if (n_rh + n_slots > kNoAllocScratchElems) {
    set_error("sfs_apply_AH_noalloc needs %zu bytes of scratch, the static maximum is %zu "
              "bytes; use sfs_apply_AH for this operator",
              (n_rh + n_slots) * sizeof(float2), kNoAllocScratchBytes);
    return SFS_ERR_INVALID_ARG;
  }
  int prev = -1;
  if (cudaGetDevice(&prev) != cudaSuccess) prev = -1;
  SFS_CUDA(cudaSetDevice(op->geo.d.device));
  float2* scratch = nullptr;
  int rc = scratch_for_current_device(&scratch);
  if (rc == SFS_OK) {
    // The spectra rows of the padding bins U..Up-1 must be zero (the scatter
    // kernel writes only rows 0..U-1 and the contraction reads all Up rows);
    // they are cleared on every call because other operators may have used
    // the array since.  The contraction writes every slot row the consumer
    // reads before it is read.
    float2* rh = scratch;
    float2* gs = scratch + n_rh;
    const PlaneDims d = operator_dims(op);
    cudaStream_t st = (cudaStream_t)stream;
    if (op->Up > op->U) {
      const cudaError_t e = cudaMemsetAsync(rh + (size_t)op->U * op->Ns, 0,
                                            (size_t)(op->Up - op->U) * op->Ns * sizeof(float2), st);
      if (e != cudaSuccess) rc = cuda_fail(e, "clearing padding spectra", __FILE__, __LINE__);
    }
    if (rc == SFS_OK) rc = launch_scatter_fwd(d, (const float2*)y_dev, op->posmap, rh, st);
    if (rc == SFS_OK) rc = launch_contract_adj(d, op->table, rh, gs, op->ws.err, st);
    if (rc == SFS_OK)
      rc = launch_inv_store(d, gs, op->ws.segslot, (float2*)x_dev, nullptr, nullptr, st);
  }
  if (prev >= 0) cudaSetDevice(prev);
  return rc;
}
