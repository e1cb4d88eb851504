// Bin-sharded operator and the building blocks of a FISTA solve split over
// several GPUs (one process per GPU).
//
// A = Phi H restricted to the measurements of one run of the kept-bin union
// is A_g (its rows are the (s, m) with idx[s][m] in the run).  The runs
// partition the rows, so A^H (A x - y) = sum_g A_g^H (A_g x - y): every rank
// forms its partial gradient from its own generator-table slice with no
// exchange (the forward needs none either), one all-reduce (sum) of the V
// voxel values per iteration joins them, and the elementwise update of
// Algorithm 1 (soft threshold and momentum) is replicated.  The lateral
// FFT-domain contraction of Theorem 2 / Algorithm 2 is the same per rank;
// only the bins it runs over change.
#include <cuda_runtime.h>
#include <math.h>
#include <stdint.h>
#include <string.h>

#include <algorithm>

#include "sfs_internal.h"

namespace sfs {
namespace {

constexpr int kVecThreads = 256;
constexpr int kVecMaxBlocks = 1216;

int vec_blocks(int n) { return std::max(1, std::min((n + kVecThreads - 1) / kVecThreads, kVecMaxBlocks)); }

// One FISTA update per element (Algorithm 1), the arithmetic of the fused
// update planes: w = gamma - g/L, x_k = tau_thr(w), gamma_{k+1} = x_k +
// beta (x_k - x_{k-1}).  x holds x_{k-1} on entry and x_k on exit, gamma
// holds gamma_k on entry and gamma_{k+1} on exit.
__global__ void __launch_bounds__(kVecThreads) prox_momentum_kernel(int n, float2* __restrict__ x,
                                                                    float2* __restrict__ gamma,
                                                                    const float2* __restrict__ grad,
                                                                    float thr, float invL, float beta) {
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) {
    const float2 g = grad[i];
    const float2 gm = gamma[i];
    const float2 xp = x[i];
    const float2 w = make_float2(fmaf(-g.x, invL, gm.x), fmaf(-g.y, invL, gm.y));
    const float mag = hypotf(w.x, w.y);
    const float sc = mag > thr ? 1.0f - thr / mag : 0.0f;
    const float2 xn = make_float2(w.x * sc, w.y * sc);
    x[i] = xn;
    gamma[i] = make_float2(fmaf(beta, xn.x - xp.x, xn.x), fmaf(beta, xn.y - xp.y, xn.y));
  }
}

__global__ void __launch_bounds__(kVecThreads) scale_kernel(int n, float2* __restrict__ v, float a) {
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) {
    const float2 t = v[i];
    v[i] = make_float2(t.x * a, t.y * a);
  }
}

// max |v_i| as the bit pattern of a non-negative float (ordered like the
// unsigned integers); NaN propagates as the largest pattern.
__global__ void __launch_bounds__(kVecThreads) max_abs_kernel(int n, const float2* __restrict__ v,
                                                              unsigned int* out) {
  __shared__ unsigned int red[kVecThreads / 32];
  unsigned int mx = 0u;
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) {
    const float2 t = v[i];
    const float m = hypotf(t.x, t.y);
    mx = max(mx, isnan(m) ? 0x7fffffffu : __float_as_uint(m));
  }
  for (int off = 16; off > 0; off >>= 1) mx = max(mx, __shfl_xor_sync(0xffffffffu, mx, off));
  if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = mx;
  __syncthreads();
  if (threadIdx.x == 0) {
    for (int w = 1; w < kVecThreads / 32; ++w) mx = max(mx, red[w]);
    atomicMax(out, mx);
  }
}

bool al16(const void* p) { return ((uintptr_t)p & 15u) == 0; }

struct Device {
  int prev = -1;
  bool ok = false;
  explicit Device(int dev) {
    if (cudaGetDevice(&prev) != cudaSuccess) prev = -1;
    ok = cudaSetDevice(dev) == cudaSuccess;
  }
  ~Device() {
    if (prev >= 0) cudaSetDevice(prev);
  }
};

}  // namespace
}  // namespace sfs

using namespace sfs;

extern "C" {

int sfs_shard_run(int U, int nshards, int shard, int32_t* first, int32_t* count) {
  clear_error();
  if (U < 1 || nshards < 1 || shard < 0 || shard >= nshards || !first || !count) {
    set_error("invalid argument");
    return SFS_ERR_INVALID_ARG;
  }
  int f = 0, c = 0;
  shard_run(U, nshards, shard, &f, &c);
  *first = f;
  *count = c;
  return SFS_OK;
}

int sfs_operator_shard(sfs_geometry* g, int M, const int32_t* idx_host, int nshards, int shard,
                       int precision, sfs_operator** out) {
  clear_error();
  if (nshards < 1 || shard < 0 || shard >= nshards || precision < SFS_PREC_FP32 ||
      precision > SFS_PREC_FP16X2) {
    set_error("invalid argument (shard %d of %d, precision %d)", shard, nshards, precision);
    return SFS_ERR_INVALID_ARG;
  }
  return build_operator_shard(g, M, idx_host, precision, nshards, shard, out);
}

int sfs_normal_residual(sfs_operator* op, const void* x_dev, const void* y_dev, void* g_dev,
                        void* stream) {
  clear_error();
  if (!op || !x_dev || !y_dev || !g_dev || !al16(x_dev) || !al16(y_dev) || !al16(g_dev)) {
    set_error("invalid argument");
    return SFS_ERR_INVALID_ARG;
  }
  Device dev(op->geo.d.device);
  if (!dev.ok) {
    set_error("cannot select CUDA device %d", op->geo.d.device);
    return SFS_ERR_CUDA;
  }
  return normal_residual(op, (const float2*)x_dev, (const float2*)y_dev, (float2*)g_dev,
                         (cudaStream_t)stream);
}

int sfs_prox_momentum(int n, void* x_dev, void* gamma_dev, const void* grad_dev, double lambda,
                      double L, double beta, void* stream) {
  clear_error();
  if (n < 0 || !x_dev || !gamma_dev || !grad_dev || !al16(x_dev) || !al16(gamma_dev) ||
      !al16(grad_dev) || !(L > 0) || !(lambda >= 0) || !isfinite(lambda) || !isfinite(beta)) {
    set_error("invalid argument");
    return SFS_ERR_INVALID_ARG;
  }
  if (n == 0) return SFS_OK;
  // thresholds rounded as the fused update planes take them
  const float thr = (float)(lambda / L), invL = (float)(1.0 / L);
  prox_momentum_kernel<<<vec_blocks(n), kVecThreads, 0, (cudaStream_t)stream>>>(
      n, (float2*)x_dev, (float2*)gamma_dev, (const float2*)grad_dev, thr, invL, (float)beta);
  SFS_CUDA(cudaGetLastError());
  return SFS_OK;
}

int sfs_vec_sumsq(sfs_operator* op, const void* v_dev, int n, double* out_host, void* stream) {
  clear_error();
  if (!op || !v_dev || n < 0 || !out_host) {
    set_error("invalid argument");
    return SFS_ERR_INVALID_ARG;
  }
  Device dev(op->geo.d.device);
  cudaStream_t st = (cudaStream_t)stream;
  double* slot = op->ws.red + kRedC;
  SFS_CUDA(cudaMemsetAsync(slot, 0, sizeof(double), st));
  if (n > 0) SFS_TRY(launch_sumsq((const float2*)v_dev, n, slot, st));
  SFS_CUDA(cudaMemcpyAsync(out_host, slot, sizeof(double), cudaMemcpyDeviceToHost, st));
  SFS_CUDA(cudaStreamSynchronize(st));
  return SFS_OK;
}

int sfs_vec_max_abs(sfs_operator* op, const void* v_dev, int n, double* out_host, void* stream) {
  clear_error();
  if (!op || !v_dev || n < 0 || !out_host) {
    set_error("invalid argument");
    return SFS_ERR_INVALID_ARG;
  }
  Device dev(op->geo.d.device);
  cudaStream_t st = (cudaStream_t)stream;
  unsigned int* slot = (unsigned int*)(op->ws.red + kRedC);
  unsigned int h = 0;
  SFS_CUDA(cudaMemsetAsync(slot, 0, sizeof(unsigned int), st));
  if (n > 0) {
    max_abs_kernel<<<vec_blocks(n), kVecThreads, 0, st>>>(n, (const float2*)v_dev, slot);
    SFS_CUDA(cudaGetLastError());
  }
  SFS_CUDA(cudaMemcpyAsync(&h, slot, sizeof(unsigned int), cudaMemcpyDeviceToHost, st));
  SFS_CUDA(cudaStreamSynchronize(st));
  float f;
  memcpy(&f, &h, sizeof f);
  *out_host = (double)f;
  return SFS_OK;
}

int sfs_vec_scale(void* v_dev, int n, double a, void* stream) {
  clear_error();
  if (!v_dev || n < 0 || !isfinite(a)) {
    set_error("invalid argument");
    return SFS_ERR_INVALID_ARG;
  }
  if (n == 0) return SFS_OK;
  scale_kernel<<<vec_blocks(n), kVecThreads, 0, (cudaStream_t)stream>>>(n, (float2*)v_dev, (float)a);
  SFS_CUDA(cudaGetLastError());
  return SFS_OK;
}

int sfs_vec_randn(void* v_dev, int n, uint64_t seed, void* stream) {
  clear_error();
  if (!v_dev || n < 0) {
    set_error("invalid argument");
    return SFS_ERR_INVALID_ARG;
  }
  if (n == 0) return SFS_OK;
  return launch_randn((float2*)v_dev, n, seed, (cudaStream_t)stream);
}

}  // extern "C"
