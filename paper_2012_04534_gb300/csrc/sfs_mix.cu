// Compressed model with Rademacher mixing, Phi_s = S_s F Sigma_s (Sec. II-B,
// Eq. "compressed_model"; Sigma_s = Diag{xi_s}, xi_s in {-1, 1}^Nt as in
// Sec. III-A's random sampling).
//
// Sigma_s acts on the time samples of A-scan s, so every kept coefficient
// mixes all Nt bins of that A-scan's spectrum B_s (the bins above Nt/2 are
// the negative frequencies of the periodic spectrum, signed bins k - Nt).
// With Xi_s = DFT(xi_s), the product xi_s . b_s has the spectrum
// (1/Nt) Xi_s (*) B_s, so
//   y_s[m] = (1/Nt) sum_k Xi_s[(k_m - k) mod Nt] B_s[k].
// B_s[k] = fs H(f_k) (...) carries the Gaussian pulse spectrum (Sec. VI), so
// the bins more than SFS_MIX_BAND_DB = 140 dB below its peak hold a fraction
// erfc(sqrt(2 ln 1e7)) ~ 1e-15 of its energy; the sum runs over the others
// (sfs_mixing_band, one run of signed bins), a truncation below 1e-7
// relative.  B = A_band x is the data of a band operator that keeps every
// bin of that run at every position (an ordinary sfs_operator on signed
// bins).  So
//   A_mix = Mix o A_band,   A_mix^H = A_band^H o Mix^H,
// with Mix one M x |band| matrix per position, generated on the fly from the
// position's Xi_s (Nt complex numbers) instead of stored.  The kernels here
// are the per-position mixing steps; the band operator's plane and
// contraction kernels do the rest.  FISTA (Algorithm 1) with mixing runs
//   contract_fwd, inv_gather (band data), mix_resid_adj (r = Mix B - y,
//   Mix^H r), scatter_fwd, contract_adj, inv_fista_fwd
// per iteration, captured once per iteration count as a CUDA graph.
#include <cuda_runtime.h>
#include <math.h>
#include <stdint.h>
#include <string.h>

#include <algorithm>
#include <new>
#include <vector>

#include "sfs_internal.h"
#include "sfs_launch.h"

struct sfs_mixing {
  sfs_operator* band = nullptr;  // not owned
  int S = 0, M = 0, U = 0, Nt = 0;
  int32_t* idx = nullptr;   // [S][M] kept bins
  int32_t* bins = nullptr;  // [U] band bins
  float2* Xi = nullptr;     // [S][Nt] DFT of xi_s, times 1/Nt
  float2* yb = nullptr;     // [S][U] band data
  float2* rb = nullptr;     // [S][U] unmixed residual / data
  float2* ybuf = nullptr;   // [S][M] measurements (FISTA)
  float2* vbuf = nullptr;   // [S][M] scratch (power iteration)
  cudaStream_t cs = nullptr;
  struct Graph {
    int iters;
    cudaGraphExec_t exec;
  };
  std::vector<Graph> graphs;
};

namespace sfs {
namespace {

constexpr int kMixThreads = 128;

// Xi[s][k] = (1/Nt) sum_n xi[s][n] e^{-2 pi j k n / Nt}, FP64 sums, one CTA
// per position; twiddles W^j from an FP64 table indexed by (k n) mod Nt.
__global__ void __launch_bounds__(kMixThreads) mix_setup_kernel(int Nt, const int8_t* __restrict__ xi,
                                                                const double2* __restrict__ W,
                                                                float2* __restrict__ Xi) {
  extern __shared__ int8_t xs[];
  const int s = blockIdx.x;
  for (int n = threadIdx.x; n < Nt; n += kMixThreads) xs[n] = xi[(size_t)s * Nt + n];
  __syncthreads();
  for (int k = threadIdx.x; k < Nt; k += kMixThreads) {
    double re = 0.0, im = 0.0;
    long long j = 0;  // (k n) mod Nt
    for (int n = 0; n < Nt; ++n) {
      const double2 w = W[j];
      const double sgn = (double)xs[n];
      re += sgn * w.x;
      im += sgn * w.y;
      j += k;
      if (j >= Nt) j -= Nt;
    }
    Xi[(size_t)s * Nt + k] = make_float2((float)(re / Nt), (float)(im / Nt));
  }
}

__device__ __forceinline__ float2 cmla(float2 acc, float2 a, float2 b) {
  return make_float2(fmaf(a.x, b.x, fmaf(-a.y, b.y, acc.x)), fmaf(a.x, b.y, fmaf(a.y, b.x, acc.y)));
}
__device__ __forceinline__ float2 cmlac(float2 acc, float2 a, float2 b) {  // acc + conj(a) b
  return make_float2(fmaf(a.x, b.x, fmaf(a.y, b.y, acc.x)), fmaf(a.x, b.y, fmaf(-a.y, b.x, acc.y)));
}
__device__ __forceinline__ float2 warp_sum(float2 v) {
#pragma unroll
  for (int off = 16; off > 0; off >>= 1) {
    v.x += __shfl_xor_sync(0xffffffffu, v.x, off);
    v.y += __shfl_xor_sync(0xffffffffu, v.y, off);
  }
  return v;
}

// Shared memory of one position: Xi_s [Nt], band data [U], kept-bin values
// [M], band bins [U], kept bins [M].
size_t mix_smem(int Nt, int U, int M) {
  return (size_t)Nt * 8 + (size_t)U * 8 + (size_t)M * 8 + (size_t)U * 4 + (size_t)M * 4 + 16;
}

struct MixDims {
  int S, M, U, Nt;
};

// One CTA per position s, Mix_s[m][u] = Xi_s[(k_m - k_u) mod Nt] (1/Nt folded
// into Xi).  MODE 0: y[s][m] = sum_u Mix_s[m][u] yb[s][u] (one warp per kept
// bin).  MODE 1: r = Mix_s yb - meas, then rb[s][u] = sum_m conj(Mix_s[m][u])
// r[m] (one warp per band bin).  MODE 2: rb = Mix_s^H meas.
template <int MODE>
__global__ void __launch_bounds__(kMixThreads) mix_kernel(MixDims md, const float2* __restrict__ Xi,
                                                          const int32_t* __restrict__ idx,
                                                          const int32_t* __restrict__ bins,
                                                          const float2* __restrict__ yb,
                                                          const float2* __restrict__ meas,
                                                          float2* __restrict__ y, float2* __restrict__ rb) {
  extern __shared__ unsigned char msm[];
  const int s = blockIdx.x;
  const int Nt = md.Nt, U = md.U, M = md.M;
  float2* xs = (float2*)msm;           // [Nt]
  float2* vb = xs + Nt;                // [U]
  float2* vm = vb + U;                 // [M]
  int32_t* bu = (int32_t*)(vm + M);    // [U]
  int32_t* km = bu + U;                // [M]
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31, nw = kMixThreads / 32;
  for (int k = threadIdx.x; k < Nt; k += kMixThreads) xs[k] = Xi[(size_t)s * Nt + k];
  for (int u = threadIdx.x; u < U; u += kMixThreads) bu[u] = bins[u];
  for (int m = threadIdx.x; m < M; m += kMixThreads) km[m] = idx[(size_t)s * M + m];
  if (MODE == 2) {
    for (int m = threadIdx.x; m < M; m += kMixThreads) vm[m] = meas[(size_t)s * M + m];
  } else {
    for (int u = threadIdx.x; u < U; u += kMixThreads) vb[u] = yb[(size_t)s * U + u];
  }
  __syncthreads();
  if (MODE != 2) {
    for (int m = warp; m < M; m += nw) {
      const int k = km[m];
      float2 acc = make_float2(0.f, 0.f);
      for (int u = lane; u < U; u += 32) {
        int dk = k - bu[u];
        if (dk < 0) dk += Nt;
        acc = cmla(acc, xs[dk], vb[u]);
      }
      acc = warp_sum(acc);
      if (lane == 0) {
        if (MODE == 0) {
          y[(size_t)s * M + m] = acc;
        } else {
          const float2 mv = meas[(size_t)s * M + m];
          vm[m] = make_float2(acc.x - mv.x, acc.y - mv.y);
        }
      }
    }
    if (MODE == 0) return;
    __syncthreads();
  }
  for (int u = warp; u < U; u += nw) {
    const int ku = bu[u];
    float2 acc = make_float2(0.f, 0.f);
    for (int m = lane; m < M; m += 32) {
      int dk = km[m] - ku;
      if (dk < 0) dk += Nt;
      acc = cmlac(acc, xs[dk], vm[m]);
    }
    acc = warp_sum(acc);
    if (lane == 0) rb[(size_t)s * U + u] = acc;
  }
}

template <int MODE>
int launch_mix(const sfs_mixing* mx, const float2* yb, const float2* meas, float2* y, float2* rb,
               cudaStream_t st) {
  const size_t smem = mix_smem(mx->Nt, mx->U, mx->M);
  SFS_TRY(ensure_smem_attr(mix_kernel<MODE>, (int)smem));
  const MixDims md = {mx->S, mx->M, mx->U, mx->Nt};
  mix_kernel<MODE><<<mx->S, kMixThreads, smem, st>>>(md, mx->Xi, mx->idx, mx->bins, yb, meas, y, rb);
  SFS_CUDA(cudaGetLastError());
  return SFS_OK;
}

// band data yb = A_band x
int band_A(sfs_mixing* mx, const float2* x, float2* yb, double* red_sumsq, cudaStream_t st) {
  sfs_operator* op = mx->band;
  const PlaneDims d = operator_dims(op);
  SFS_TRY(launch_fwd_planes(d, x, op->ws.Xh, st));
  SFS_TRY(launch_contract_fwd(d, op->table, op->ws.Xh, op->ws.Yh, op->ws.err, st));
  return launch_inv_gather(d, op->ws.Yh, op->posmap, yb, red_sumsq, st);
}

// x = A_band^H rb (x may be null: reductions only)
int band_AH(sfs_mixing* mx, const float2* rb, float2* x, double* red_sumsq, unsigned int* maxabs,
            cudaStream_t st) {
  sfs_operator* op = mx->band;
  const PlaneDims d = operator_dims(op);
  SFS_TRY(launch_scatter_fwd(d, rb, op->posmap, op->ws.Rh, st));
  SFS_TRY(launch_contract_adj(d, op->table, op->ws.Rh, op->ws.Gh, op->ws.err, st));
  return launch_inv_store(d, op->ws.Gh, op->ws.segslot, x, red_sumsq, maxabs, st);
}

int mixed_fista_loop(sfs_mixing* mx, int iters, cudaStream_t st) {
  sfs_operator* op = mx->band;
  const PlaneDims d = operator_dims(op);
  std::vector<float> beta(iters);
  double t = 1.0;
  for (int k = 0; k < iters; ++k) {
    const double tn = 0.5 * (1.0 + sqrt(1.0 + 4.0 * t * t));
    beta[k] = (float)((t - 1.0) / tn);
    t = tn;
  }
  SFS_TRY(launch_fwd_planes(d, op->ws.gam, op->ws.Xh, st));
  for (int k = 0; k < iters; ++k) {
    SFS_TRY(launch_contract_fwd(d, op->table, op->ws.Xh, op->ws.Yh, op->ws.err, st));
    SFS_TRY(launch_inv_gather(d, op->ws.Yh, op->posmap, mx->yb, nullptr, st));
    SFS_TRY(launch_mix<1>(mx, mx->yb, mx->ybuf, nullptr, mx->rb, st));
    SFS_TRY(launch_scatter_fwd(d, mx->rb, op->posmap, op->ws.Rh, st));
    SFS_TRY(launch_contract_adj(d, op->table, op->ws.Rh, op->ws.Gh, op->ws.err, st));
    SFS_TRY(launch_inv_fista_fwd(d, op->ws.Gh, op->ws.segslot, op->ws.xk, op->ws.gam, op->ws.scal, beta[k],
                                 k + 1 < iters, op->ws.Xh, nullptr, st));
  }
  return SFS_OK;
}

int mixed_graph(sfs_mixing* mx, int iters, cudaGraphExec_t* out) {
  for (auto& g : mx->graphs)
    if (g.iters == iters) {
      *out = g.exec;
      return SFS_OK;
    }
  if (!mx->cs) SFS_CUDA(cudaStreamCreateWithFlags(&mx->cs, cudaStreamNonBlocking));
  SFS_TRY(prepare_kernels(operator_dims(mx->band)));
  SFS_TRY(ensure_smem_attr(mix_kernel<1>, (int)mix_smem(mx->Nt, mx->U, mx->M)));
  SFS_CUDA(cudaStreamBeginCapture(mx->cs, cudaStreamCaptureModeThreadLocal));
  const int rc = mixed_fista_loop(mx, iters, mx->cs);
  cudaGraph_t graph = nullptr;
  const cudaError_t e = cudaStreamEndCapture(mx->cs, &graph);
  if (rc != SFS_OK) {
    if (graph) cudaGraphDestroy(graph);
    return rc;
  }
  if (e != cudaSuccess) return cuda_fail(e, "cudaStreamEndCapture", __FILE__, __LINE__);
  cudaGraphExec_t exec = nullptr;
  const cudaError_t e2 = cudaGraphInstantiate(&exec, graph, 0);
  cudaGraphDestroy(graph);
  if (e2 != cudaSuccess) return cuda_fail(e2, "cudaGraphInstantiate", __FILE__, __LINE__);
  mx->graphs.push_back({iters, exec});
  *out = exec;
  return SFS_OK;
}

void free_mixing(sfs_mixing* mx) {
  if (!mx) return;
  for (auto& g : mx->graphs) cudaGraphExecDestroy(g.exec);
  if (mx->cs) cudaStreamDestroy(mx->cs);
  cudaFree(mx->idx);
  cudaFree(mx->bins);
  cudaFree(mx->Xi);
  cudaFree(mx->yb);
  cudaFree(mx->rb);
  cudaFree(mx->ybuf);
  cudaFree(mx->vbuf);
  delete mx;
}

int check_err(sfs_operator* op, cudaStream_t st) {
  int h = 0;
  SFS_CUDA(cudaMemcpyAsync(&h, op->ws.err, sizeof(int), cudaMemcpyDeviceToHost, st));
  SFS_CUDA(cudaStreamSynchronize(st));
  if (h) {
    SFS_CUDA(cudaMemset(op->ws.err, 0, sizeof(int)));
    set_error(h == 2 ? "non-finite value reached the lambda rule" : "a bounded wait in a contraction kernel timed out");
    return h == 2 ? SFS_ERR_NON_FINITE : SFS_ERR_TIMEOUT;
  }
  return SFS_OK;
}

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

bool al16(const void* p) { return ((uintptr_t)p & 15u) == 0; }

// Signed bins -Nt/2 < k <= Nt/2 with |H(f_k)| >= 10^(-SFS_MIX_BAND_DB / 20)
// max |H|, f_k = k fs / Nt: one run, since |H| falls off monotonically on
// both sides of fc.
void mixing_band(const sfs_geometry* g, int* lo, int* hi) {
  const int kmax = g->d.Nt / 2, kmin = -((g->d.Nt - 1) / 2);
  double peak = 0.0;
  for (int k = kmin; k <= kmax; ++k)
    peak = std::max(peak, pulse_mag((double)k * g->d.fs / g->d.Nt, g->d.fc, g->alpha));
  const double thr = peak * pow(10.0, -SFS_MIX_BAND_DB / 20.0);
  *lo = kmax;
  *hi = kmin;
  for (int k = kmin; k <= kmax; ++k)
    if (pulse_mag((double)k * g->d.fs / g->d.Nt, g->d.fc, g->alpha) >= thr) {
      *lo = std::min(*lo, k);
      *hi = std::max(*hi, k);
    }
}

}  // namespace
}  // namespace sfs

using namespace sfs;

extern "C" {

int sfs_mixing_band(const sfs_geometry* g, int32_t* k_lo, int32_t* k_hi) {
  clear_error();
  if (!g || !k_lo || !k_hi) {
    set_error("null argument");
    return SFS_ERR_INVALID_ARG;
  }
  int lo = 0, hi = 0;
  mixing_band(g, &lo, &hi);
  *k_lo = lo;
  *k_hi = hi;
  return SFS_OK;
}

int sfs_mixing_create(sfs_operator* band, int M, const int32_t* idx_host, const int8_t* xi_host,
                      sfs_mixing** out) {
  clear_error();
  if (!band || !idx_host || !xi_host || !out) {
    set_error("null argument");
    return SFS_ERR_INVALID_ARG;
  }
  *out = nullptr;
  const int S = band->S, U = band->U, Nt = band->geo.d.Nt, kmax = Nt / 2;
  if (band->M != U) {
    set_error("the band operator must keep every bin of its band at every position");
    return SFS_ERR_INVALID_ARG;
  }
  for (int s = 0; s < S; ++s)
    for (int u = 0; u < U; ++u)
      if (band->idx[(size_t)s * U + u] != band->bins[u]) {
        set_error("the band operator must keep every bin of its band at every position");
        return SFS_ERR_INVALID_ARG;
      }
  {
    int lo = 0, hi = 0;
    mixing_band(&band->geo, &lo, &hi);
    const auto first = std::lower_bound(band->bins.begin(), band->bins.end(), lo);
    if (first == band->bins.end() || band->bins.end() - first < hi - lo + 1 || first[hi - lo] != hi) {
      set_error("the band operator must keep every signed bin %d..%d (sfs_mixing_band)", lo, hi);
      return SFS_ERR_INVALID_ARG;
    }
  }
  if (M < 1 || M > kmax + 1 || Nt > 8192) {
    set_error("M = %d out of range 1..%d (Nt <= 8192)", M, kmax + 1);
    return SFS_ERR_INVALID_ARG;
  }
  for (int s = 0; s < S; ++s)
    for (int m = 0; m < M; ++m) {
      const int k = idx_host[(size_t)s * M + m];
      if (k < 0 || k > kmax || (m > 0 && k <= idx_host[(size_t)s * M + m - 1])) {
        set_error("index row %d is not strictly ascending inside 0..%d", s, kmax);
        return SFS_ERR_INVALID_ARG;
      }
    }
  for (size_t i = 0; i < (size_t)S * Nt; ++i)
    if (xi_host[i] != 1 && xi_host[i] != -1) {
      set_error("mixing sequences must hold +1 or -1");
      return SFS_ERR_INVALID_ARG;
    }
  Device dev(band->geo.d.device);
  if (!dev.ok) {
    set_error("cannot select CUDA device %d", band->geo.d.device);
    return SFS_ERR_CUDA;
  }
  sfs_mixing* mx = new (std::nothrow) sfs_mixing;
  if (!mx) {
    set_error("host allocation failed");
    return SFS_ERR_OOM;
  }
  mx->band = band;
  mx->S = S;
  mx->M = M;
  mx->U = U;
  mx->Nt = Nt;
  int8_t* dxi = nullptr;
  double2* dW = nullptr;
  auto fail = [&](int rc) {
    cudaFree(dxi);
    cudaFree(dW);
    free_mixing(mx);
    return rc;
  };
  std::vector<double2> W(Nt);
  for (int j = 0; j < Nt; ++j) W[j] = make_double2(cos(-2.0 * M_PI * j / Nt), sin(-2.0 * M_PI * j / Nt));
  cudaError_t e = cudaSuccess;
  if (e == cudaSuccess) e = cudaMalloc(&mx->idx, (size_t)S * M * 4);
  if (e == cudaSuccess) e = cudaMalloc(&mx->bins, (size_t)U * 4);
  if (e == cudaSuccess) e = cudaMalloc(&mx->Xi, (size_t)S * Nt * 8);
  if (e == cudaSuccess) e = cudaMalloc(&mx->yb, (size_t)S * U * 8);
  if (e == cudaSuccess) e = cudaMalloc(&mx->rb, (size_t)S * U * 8);
  if (e == cudaSuccess) e = cudaMalloc(&mx->ybuf, (size_t)S * M * 8);
  if (e == cudaSuccess) e = cudaMalloc(&mx->vbuf, (size_t)S * M * 8);
  if (e == cudaSuccess) e = cudaMalloc(&dxi, (size_t)S * Nt);
  if (e == cudaSuccess) e = cudaMalloc(&dW, (size_t)Nt * sizeof(double2));
  if (e == cudaSuccess) e = cudaMemcpy(mx->idx, idx_host, (size_t)S * M * 4, cudaMemcpyHostToDevice);
  if (e == cudaSuccess) e = cudaMemcpy(mx->bins, band->bins.data(), (size_t)U * 4, cudaMemcpyHostToDevice);
  if (e == cudaSuccess) e = cudaMemcpy(dxi, xi_host, (size_t)S * Nt, cudaMemcpyHostToDevice);
  if (e == cudaSuccess) e = cudaMemcpy(dW, W.data(), (size_t)Nt * sizeof(double2), cudaMemcpyHostToDevice);
  if (e != cudaSuccess) return fail(cuda_fail(e, "mixing tables", __FILE__, __LINE__));
  mix_setup_kernel<<<S, kMixThreads, Nt>>>(Nt, dxi, dW, mx->Xi);
  e = cudaGetLastError();
  if (e == cudaSuccess) e = cudaDeviceSynchronize();
  if (e != cudaSuccess) return fail(cuda_fail(e, "mixing spectra", __FILE__, __LINE__));
  cudaFree(dxi);
  cudaFree(dW);
  dxi = nullptr;
  dW = nullptr;
  *out = mx;
  return SFS_OK;
}

int sfs_mixing_destroy(sfs_mixing* mx) {
  clear_error();
  if (!mx) return SFS_OK;
  Device dev(mx->band->geo.d.device);
  free_mixing(mx);
  return SFS_OK;
}

int sfs_apply_A_mixed(sfs_mixing* mx, const void* x_dev, void* y_dev, void* stream) {
  clear_error();
  if (!mx || !x_dev || !y_dev || !al16(x_dev) || !al16(y_dev)) {
    set_error("invalid argument");
    return SFS_ERR_INVALID_ARG;
  }
  Device dev(mx->band->geo.d.device);
  cudaStream_t st = (cudaStream_t)stream;
  SFS_TRY(band_A(mx, (const float2*)x_dev, mx->yb, nullptr, st));
  return launch_mix<0>(mx, mx->yb, nullptr, (float2*)y_dev, nullptr, st);
}

int sfs_apply_AH_mixed(sfs_mixing* mx, const void* y_dev, void* x_dev, void* stream) {
  clear_error();
  if (!mx || !x_dev || !y_dev || !al16(x_dev) || !al16(y_dev)) {
    set_error("invalid argument");
    return SFS_ERR_INVALID_ARG;
  }
  Device dev(mx->band->geo.d.device);
  cudaStream_t st = (cudaStream_t)stream;
  SFS_TRY(launch_mix<2>(mx, nullptr, (const float2*)y_dev, nullptr, mx->rb, st));
  return band_AH(mx, mx->rb, (float2*)x_dev, nullptr, nullptr, st);
}

int sfs_lipschitz_mixed(sfs_mixing* mx, int max_iter, double rtol, uint64_t seed, double safety,
                        double* L_out, void* stream) {
  clear_error();
  if (!mx || !L_out || max_iter < 1 || !(rtol >= 0) || !(safety >= 0)) {
    set_error("invalid argument");
    return SFS_ERR_INVALID_ARG;
  }
  Device dev(mx->band->geo.d.device);
  cudaStream_t st = (cudaStream_t)stream;
  sfs_operator* op = mx->band;
  const int V = op->V, SM = mx->S * mx->M;
  float2* v = op->ws.gam;
  float2* w = op->ws.xk;
  double* red = op->ws.red;
  // power iteration on A_mix^H A_mix: est = ||A v||^2 with ||v|| = 1
  SFS_TRY(launch_randn(v, V, seed, st));
  SFS_CUDA(cudaMemsetAsync(red + kRedB, 0, sizeof(double), st));
  SFS_TRY(launch_sumsq(v, V, red + kRedB, st));
  SFS_TRY(launch_scale_by_rnorm(v, V, red + kRedB, st));
  double prev = -1.0, est = 0.0, h = 0.0;
  for (int it = 0; it < max_iter; ++it) {
    SFS_CUDA(cudaMemsetAsync(red, 0, 2 * sizeof(double), st));
    SFS_TRY(band_A(mx, v, mx->yb, nullptr, st));
    SFS_TRY(launch_mix<0>(mx, mx->yb, nullptr, mx->vbuf, nullptr, st));
    SFS_TRY(launch_sumsq(mx->vbuf, SM, red + kRedA, st));
    SFS_TRY(launch_mix<2>(mx, nullptr, mx->vbuf, nullptr, mx->rb, st));
    SFS_TRY(band_AH(mx, mx->rb, w, red + kRedB, nullptr, st));
    SFS_TRY(launch_scale_by_rnorm(w, V, red + kRedB, st));
    std::swap(v, w);
    SFS_CUDA(cudaMemcpyAsync(&h, red + kRedA, sizeof(double), cudaMemcpyDeviceToHost, st));
    SFS_CUDA(cudaStreamSynchronize(st));
    est = h;
    if (!isfinite(est)) {
      set_error("non-finite Rayleigh quotient in power iteration");
      return SFS_ERR_NON_FINITE;
    }
    if (prev > 0 && fabs(est - prev) <= rtol * est) {
      SFS_TRY(check_err(op, st));
      *L_out = est * (1.0 + safety);
      return SFS_OK;
    }
    prev = est;
  }
  SFS_TRY(check_err(op, st));
  *L_out = est * (1.0 + safety);
  set_error("power iteration did not converge in %d iterations", max_iter);
  return SFS_ERR_NOT_CONVERGED;
}

int sfs_fista_mixed(sfs_mixing* mx, const void* y_dev, double lambda, double L, int iters, void* x_dev,
                    void* stream) {
  clear_error();
  if (!mx || !y_dev || !x_dev || iters < 0 || !(L > 0) || !isfinite(lambda) || !al16(y_dev) ||
      !al16(x_dev)) {
    set_error("invalid argument");
    return SFS_ERR_INVALID_ARG;
  }
  Device dev(mx->band->geo.d.device);
  cudaStream_t st = (cudaStream_t)stream;
  sfs_operator* op = mx->band;
  const size_t vbytes = (size_t)op->V * sizeof(float2);
  SFS_CUDA(cudaMemcpyAsync(mx->ybuf, y_dev, (size_t)mx->S * mx->M * sizeof(float2), cudaMemcpyDeviceToDevice,
                           st));
  SFS_CUDA(cudaMemsetAsync(op->ws.xk, 0, vbytes, st));
  SFS_CUDA(cudaMemsetAsync(op->ws.gam, 0, vbytes, st));
  const int use_mu = lambda < 0;
  if (use_mu) {  // lambda = mu ||A_mix^H y||_inf on the device
    unsigned int* bits = (unsigned int*)(op->ws.scal + kLamMax);
    SFS_CUDA(cudaMemsetAsync(bits, 0, sizeof(unsigned int), st));
    SFS_TRY(launch_mix<2>(mx, nullptr, mx->ybuf, nullptr, mx->rb, st));
    SFS_TRY(band_AH(mx, mx->rb, nullptr, nullptr, bits, st));
  }
  SFS_TRY(launch_set_thresholds(op->ws.scal, op->ws.red, use_mu ? 0.0 : lambda, L, use_mu,
                                use_mu ? -lambda : 0.0, op->ws.err, st));
  if (iters > 0) {
    cudaGraphExec_t exec = nullptr;
    SFS_TRY(mixed_graph(mx, iters, &exec));
    SFS_CUDA(cudaGraphLaunch(exec, st));
  }
  SFS_CUDA(cudaMemcpyAsync(x_dev, op->ws.xk, vbytes, cudaMemcpyDeviceToDevice, st));
  return SFS_OK;
}

}  // extern "C"
