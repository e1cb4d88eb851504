// FISTA with backtracking (Sec. IV-C, "Backtracking"): no sigma_max, only a
// lower bound L0 = sigma_low^2 and a factor eta > 1 (Beck and Teboulle's
// backtracking rule).  Step k tries L' = eta^i L_{k-1}, i = 0, 1, ..., until
//   F(p_L'(gamma_k)) <= Q_L'(p_L'(gamma_k), gamma_k).
// For f(x) = 1/2 ||A x - y||^2 that test is exact algebra away from
//   ||A d||^2 <= L' ||d||^2,  d = p_L'(gamma_k) - gamma_k,
// since f(p) - f(gamma) - Re<d, grad f(gamma)> = 1/2 ||A d||^2.  The library
// evaluates this form: it needs one forward apply of d per trial and no
// difference of two nearly equal objective values, which FP32 data would
// blur near convergence.  Per iteration: the gradient (forward, residual
// planes, adjoint: the operator's kernels), then per trial the prox kernel
// (p, d and ||d||^2), a forward apply of d with ||A d||^2, and one host
// read of the two sums; the accepted trial ends in the momentum kernel.
// The host reads make this much slower than the graph-replayed loop of
// sfs_fista; the paper notes the cost of the extra applies.
#include <cuda_runtime.h>
#include <math.h>
#include <stdint.h>
#include <string.h>

#include <algorithm>
#include <vector>

#include "sfs_internal.h"

namespace sfs {
namespace {

constexpr int kBtThreads = 256;
constexpr int kBtMaxBlocks = 1024;

// p = tau_thr(gamma - invL g), d = p - gamma; per-CTA partial of ||d||^2.
__global__ void __launch_bounds__(kBtThreads) bt_prox_kernel(int V, const float2* __restrict__ gam,
                                                             const float2* __restrict__ g, float invL, float thr,
                                                             float2* __restrict__ p, float2* __restrict__ dv,
                                                             double* __restrict__ part) {
  double acc = 0.0;
  for (int i = blockIdx.x * kBtThreads + threadIdx.x; i < V; i += gridDim.x * kBtThreads) {
    const float2 gm = gam[i], gr = g[i];
    const float2 w = make_float2(fmaf(-gr.x, invL, gm.x), fmaf(-gr.y, invL, gm.y));
    const float mag = hypotf(w.x, w.y);
    const float sc = mag > thr ? 1.0f - thr / mag : 0.0f;
    const float2 pv = make_float2(w.x * sc, w.y * sc);
    const float2 dd = make_float2(pv.x - gm.x, pv.y - gm.y);
    p[i] = pv;
    dv[i] = dd;
    acc += (double)dd.x * dd.x + (double)dd.y * dd.y;
  }
  __shared__ double red[kBtThreads / 32];
#pragma unroll
  for (int off = 16; off > 0; off >>= 1) acc += __shfl_xor_sync(0xffffffffu, acc, off);
  if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = acc;
  __syncthreads();
  if (threadIdx.x == 0) {
    double v = 0.0;
    for (int w = 0; w < kBtThreads / 32; ++w) v += red[w];
    part[blockIdx.x] = v;
  }
}

// out = sum of n partials, in a fixed order (deterministic)
__global__ void __launch_bounds__(kBtThreads) bt_sum_kernel(const double* __restrict__ part, int n,
                                                            double* __restrict__ out) {
  double acc = 0.0;
  for (int i = threadIdx.x; i < n; i += kBtThreads) acc += part[i];
  __shared__ double red[kBtThreads];
  red[threadIdx.x] = acc;
  __syncthreads();
  for (int h = kBtThreads / 2; h > 0; h >>= 1) {
    if (threadIdx.x < h) red[threadIdx.x] += red[threadIdx.x + h];
    __syncthreads();
  }
  if (threadIdx.x == 0) *out = red[0];
}

// accepted step: gamma = p + beta (p - x), x = p (Algorithm 1's momentum)
__global__ void __launch_bounds__(kBtThreads) bt_momentum_kernel(int V, const float2* __restrict__ p,
                                                                 float2* __restrict__ x, float2* __restrict__ gam,
                                                                 float beta) {
  for (int i = blockIdx.x * kBtThreads + threadIdx.x; i < V; i += gridDim.x * kBtThreads) {
    const float2 pv = p[i], xp = x[i];
    gam[i] = make_float2(fmaf(beta, pv.x - xp.x, pv.x), fmaf(beta, pv.y - xp.y, pv.y));
    x[i] = pv;
  }
}

struct BtBuf {
  void* p = nullptr;
  ~BtBuf() { cudaFree(p); }
};

}  // namespace
}  // namespace sfs

using namespace sfs;

extern "C" int sfs_fista_backtracking(sfs_operator* op, const void* y_dev, double lambda, double L0,
                                      double eta, int iters, void* x_dev, double* L_hist_host,
                                      void* stream) {
  clear_error();
  if (!op || !y_dev || !x_dev || iters < 0 || !(L0 > 0) || !isfinite(L0) || !(eta > 1.0) || !isfinite(eta) ||
      !isfinite(lambda) || ((uintptr_t)y_dev & 15u) || ((uintptr_t)x_dev & 15u)) {
    set_error("invalid argument (need L0 > 0, eta > 1, finite lambda, aligned buffers)");
    return SFS_ERR_INVALID_ARG;
  }
  int prev = -1;
  if (cudaGetDevice(&prev) != cudaSuccess) prev = -1;
  SFS_CUDA(cudaSetDevice(op->geo.d.device));
  struct Restore {
    int dev;
    ~Restore() {
      if (dev >= 0) cudaSetDevice(dev);
    }
  } restore{prev};
  cudaStream_t st = (cudaStream_t)stream;
  const PlaneDims d = operator_dims(op);
  const int V = op->V;
  const int nblk = std::min(kBtMaxBlocks, (V + kBtThreads - 1) / kBtThreads);
  BtBuf bg, bp, bd, bpart, bred;
  SFS_CUDA(cudaMalloc(&bg.p, (size_t)V * sizeof(float2)));
  SFS_CUDA(cudaMalloc(&bp.p, (size_t)V * sizeof(float2)));
  SFS_CUDA(cudaMalloc(&bd.p, (size_t)V * sizeof(float2)));
  SFS_CUDA(cudaMalloc(&bpart.p, (size_t)nblk * sizeof(double)));
  SFS_CUDA(cudaMalloc(&bred.p, 2 * sizeof(double)));
  float2* g = (float2*)bg.p;
  float2* p = (float2*)bp.p;
  float2* dv = (float2*)bd.p;
  double* part = (double*)bpart.p;
  double* red = (double*)bred.p;
  float2* ybuf = op->ws.ybuf;
  SFS_CUDA(cudaMemcpyAsync(ybuf, y_dev, (size_t)op->S * op->M * sizeof(float2), cudaMemcpyDeviceToDevice, st));
  SFS_CUDA(cudaMemsetAsync(op->ws.xk, 0, (size_t)V * sizeof(float2), st));
  SFS_CUDA(cudaMemsetAsync(op->ws.gam, 0, (size_t)V * sizeof(float2), st));
  SFS_TRY(launch_scatter_y_planes(d, ybuf, op->posmap, op->ws.yplane, st));
  // An early exit first reads (and clears) the operator's device error flag:
  // a bounded wait that ran out in a contraction can surface as a
  // non-finite sum, and is then reported as the timeout it was.
  auto early_exit = [&](int rc) -> int {
    int hf = 0;
    if (cudaMemcpyAsync(&hf, op->ws.err, sizeof(int), cudaMemcpyDeviceToHost, st) == cudaSuccess &&
        cudaStreamSynchronize(st) == cudaSuccess && hf) {
      cudaMemset(op->ws.err, 0, sizeof(int));
      set_error("a bounded wait in a contraction kernel timed out");
      return SFS_ERR_TIMEOUT;
    }
    return rc;
  };
  double lam = lambda;
  if (lambda < 0) {  // mu rule: lambda = -lambda ||A^H y||_inf
    unsigned int* bits = (unsigned int*)(op->ws.scal + kLamMax);
    unsigned int hb = 0;
    SFS_CUDA(cudaMemsetAsync(bits, 0, sizeof(unsigned int), st));
    SFS_TRY(launch_scatter_fwd(d, ybuf, op->posmap, op->ws.Rh, st));
    SFS_TRY(launch_contract_adj(d, op->table, op->ws.Rh, op->ws.Gh, op->ws.err, st));
    SFS_TRY(launch_inv_store(d, op->ws.Gh, op->ws.segslot, nullptr, nullptr, bits, st));
    SFS_CUDA(cudaMemcpyAsync(&hb, bits, sizeof(hb), cudaMemcpyDeviceToHost, st));
    SFS_CUDA(cudaStreamSynchronize(st));
    float mx;
    memcpy(&mx, &hb, sizeof(mx));
    if (!isfinite(mx)) {
      set_error("non-finite value reached the lambda rule");
      return early_exit(SFS_ERR_NON_FINITE);
    }
    lam = -lambda * (double)mx;
  }
  double L = L0, t = 1.0;
  const int gridv = nblk;
  for (int k = 0; k < iters; ++k) {
    // gradient g = A^H (A gamma - y)
    SFS_TRY(launch_fwd_planes(d, op->ws.gam, op->ws.Xh, st));
    SFS_TRY(launch_contract_fwd(d, op->table, op->ws.Xh, op->ws.Yh, op->ws.err, st));
    SFS_TRY(launch_inv_resid_fwd(d, op->ws.Yh, op->posmap, op->ws.yplane, op->ws.Rh, nullptr, st));
    SFS_TRY(launch_contract_adj(d, op->table, op->ws.Rh, op->ws.Gh, op->ws.err, st));
    SFS_TRY(launch_inv_store(d, op->ws.Gh, op->ws.segslot, g, nullptr, nullptr, st));
    for (int trial = 0;; ++trial) {
      if (trial > 200 || !isfinite(L)) {
        set_error("backtracking found no step (L = %g)", L);
        return early_exit(SFS_ERR_NOT_CONVERGED);
      }
      bt_prox_kernel<<<gridv, kBtThreads, 0, st>>>(V, op->ws.gam, g, (float)(1.0 / L), (float)(lam / L), p, dv,
                                                   part);
      bt_sum_kernel<<<1, kBtThreads, 0, st>>>(part, nblk, red);
      SFS_CUDA(cudaGetLastError());
      SFS_CUDA(cudaMemsetAsync(red + 1, 0, sizeof(double), st));
      SFS_TRY(launch_fwd_planes(d, dv, op->ws.Xh, st));
      SFS_TRY(launch_contract_fwd(d, op->table, op->ws.Xh, op->ws.Yh, op->ws.err, st));
      SFS_TRY(launch_inv_gather(d, op->ws.Yh, op->posmap, op->ws.vbuf, red + 1, st));
      double h[2];
      SFS_CUDA(cudaMemcpyAsync(h, red, sizeof(h), cudaMemcpyDeviceToHost, st));
      SFS_CUDA(cudaStreamSynchronize(st));
      if (!isfinite(h[0]) || !isfinite(h[1])) {
        set_error("non-finite step in backtracking");
        return early_exit(SFS_ERR_NON_FINITE);
      }
      if (h[1] <= L * h[0]) break;  // ||A d||^2 <= L ||d||^2 (d = 0 passes)
      L *= eta;
    }
    const double tn = 0.5 * (1.0 + sqrt(1.0 + 4.0 * t * t));
    const float beta = (float)((t - 1.0) / tn);
    t = tn;
    bt_momentum_kernel<<<gridv, kBtThreads, 0, st>>>(V, p, op->ws.xk, op->ws.gam, beta);
    SFS_CUDA(cudaGetLastError());
    if (L_hist_host) L_hist_host[k] = L;
  }
  SFS_CUDA(cudaMemcpyAsync(x_dev, op->ws.xk, (size_t)V * sizeof(float2), cudaMemcpyDeviceToDevice, st));
  // contraction timeouts raise the operator's error flag
  int hf = 0;
  SFS_CUDA(cudaMemcpyAsync(&hf, op->ws.err, sizeof(int), cudaMemcpyDeviceToHost, st));
  SFS_CUDA(cudaStreamSynchronize(st));
  if (hf) {
    SFS_CUDA(cudaMemset(op->ws.err, 0, sizeof(int)));
    set_error("a bounded wait in a contraction kernel timed out");
    return SFS_ERR_TIMEOUT;
  }
  return SFS_OK;
}
