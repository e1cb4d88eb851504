// Host-side launch helpers shared by the kernel files of libsfs.
#pragma once

#include <cuda_runtime.h>

#include <utility>

#include "sfs_internal.h"

namespace sfs {

// Raise a kernel's dynamic shared memory limit to what the device allows next
// to the kernel's static shared memory, once per (kernel, device); each
// launch then asks for what it needs.
int ensure_smem_attr_ptr(const void* kernel, int need);

template <typename K>
int ensure_smem_attr(K kernel, int need) {
  return ensure_smem_attr_ptr((const void*)kernel, need);
}

// Programmatic dependent launch is off unless SFS_PDL=1 is set in the
// environment (read once per process).  Measured on GB300 with the graph-
// replayed FISTA loop it was 4-5 % slower than plain stream order with the
// first kernels (vol32 19,955 vs 20,887 iterations/s; vol64 1,593 vs 1,662)
// and is neutral with the current ones (vol64 FP32 2,408 vs 2,404, BF16
// 3,674 vs 3,682), so the kernels keep their pdl_wait / pdl_trigger points
// (no-ops without the launch attribute) but are launched in plain stream
// order by default.
bool pdl_enabled();

// Priority given to the kernels this thread launches through launch_pdl (0:
// none, the stream's own); set while grouped loops are captured, whose
// graphs run with per-node priorities.
int& launch_priority();

// Launch with programmatic stream serialisation (see pdl_wait).
template <typename... KArgs, typename... Args>
int launch_pdl(void (*kernel)(KArgs...), dim3 grid, dim3 block, size_t smem, cudaStream_t st,
               Args&&... args) {
  cudaLaunchAttribute attr[2];
  attr[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
  attr[0].val.programmaticStreamSerializationAllowed = pdl_enabled() ? 1 : 0;
  unsigned n = 1;
  if (launch_priority() != 0) {
    attr[1].id = cudaLaunchAttributePriority;
    attr[1].val.priority = launch_priority();
    n = 2;
  }
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = grid;
  cfg.blockDim = block;
  cfg.dynamicSmemBytes = smem;
  cfg.stream = st;
  cfg.attrs = attr;
  cfg.numAttrs = n;
  SFS_CUDA(cudaLaunchKernelEx(&cfg, kernel, std::forward<Args>(args)...));
  return SFS_OK;
}

// The same for a kernel run as clusters of `cluster_x` CTAs along x
// (grid.x a multiple of cluster_x).
template <typename... KArgs, typename... Args>
int launch_pdl_cluster(void (*kernel)(KArgs...), int cluster_x, dim3 grid, dim3 block, size_t smem,
                       cudaStream_t st, Args&&... args) {
  cudaLaunchAttribute attr[3];
  attr[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
  attr[0].val.programmaticStreamSerializationAllowed = pdl_enabled() ? 1 : 0;
  attr[1].id = cudaLaunchAttributeClusterDimension;
  attr[1].val.clusterDim.x = (unsigned)cluster_x;
  attr[1].val.clusterDim.y = 1;
  attr[1].val.clusterDim.z = 1;
  unsigned n = 2;
  if (launch_priority() != 0) {
    attr[2].id = cudaLaunchAttributePriority;
    attr[2].val.priority = launch_priority();
    n = 3;
  }
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = grid;
  cfg.blockDim = block;
  cfg.dynamicSmemBytes = smem;
  cfg.stream = st;
  cfg.attrs = attr;
  cfg.numAttrs = n;
  SFS_CUDA(cudaLaunchKernelEx(&cfg, kernel, std::forward<Args>(args)...));
  return SFS_OK;
}

}  // namespace sfs
