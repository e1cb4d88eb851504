// Learned unrolled ISTA: forward, backward, loss and Adam update, all on the
// GPU, for batches of scenes sharing one operator.
//
// The paper reconstructs with ISTA/FISTA (Sec. IV-A, Algorithm 1).  Each
// layer l of the network keeps that iteration's gradient step and complex
// soft threshold, with a learned step eta_l and threshold theta_l, and adds
// a residual 3-D convolutional proximal block:
//   g_l     = A^H (A x_l - y_n)                 (the batched operator kernels)
//   z_l     = x_l - (eta_l / L) g_l,   s_l = tau_{theta_l}(z_l)
//   h_l     = W1_l * [Re s_l, Im s_l] + b1_l    8 channels, 3x3x3, zero padding
//   x_{l+1} = s_l + (W2_l * relu(h_l) + b2_l)   2 channels read as (re, im)
// with x_0 = 0, y_n = y / sigma, sigma = ||A^H y||_inf / L per scene (L the
// operator's Lipschitz constant, so that ||A^H y_n||_inf = L and the layer
// variables are O(1)), and output sigma x_L.  "*" is the cross-correlation
//   (W * u)[o](v) = sum_{i, t} W[o][i][t] u[i](v + t - (1, 1, 1)).
// Convolution weights are used in FP16 (converted to FP32 in shared memory),
// with FP32 accumulation; the master parameters and Adam moments are FP32.
// Flat parameters per layer (876): eta, theta, W1 [8][2][27], b1 [8],
// W2 [2][8][27], b2 [2].
//
// Backward (reverse layer order), with gx the gradient at x_{l+1}:
//   dW2, db2 from gx and relu(h_l);  gh = (W2^T * gx) . [h_l > 0]
//   dW1, db1 from gh and s_l;        gs = gx + W1^T * gh
//   soft threshold: for |z| > theta with u = z/|z|,
//     gz = (1 - theta/|z|) gs + (theta/|z|) u Re(conj(u) gs),
//     dtheta = -sum Re(conj(u) gs)
//   deta = -sum Re(conj(g_l) gz) / L;   gx_prev = gz - (eta_l / L) A^H A gz.
// Weight gradients are reduced in two deterministic passes (per-block
// partial sums, then a fixed-order sum over blocks in FP64).
#include <cuda_fp16.h>
#include <cuda_runtime.h>
#include <stdint.h>

#include <algorithm>
#include <vector>

#include "sfs_internal.h"

namespace sfs {
namespace {

constexpr int kC = 8;             // hidden channels
constexpr int kTaps = 27;         // 3 x 3 x 3
constexpr int kW1 = kC * 2 * kTaps;
constexpr int kW2 = 2 * kC * kTaps;
constexpr int kPerLayer = 2 + kW1 + kC + kW2 + 2;  // 876
constexpr int kOffW1 = 2, kOffB1 = kOffW1 + kW1, kOffW2 = kOffB1 + kC, kOffB2 = kOffW2 + kW2;
constexpr int kThreads = 256;
constexpr int kChunks = 64;       // voxel chunks of the weight-gradient reductions
constexpr int kWAcc = 16 + kC;    // accumulators per (tap, chunk): 16 weights + up to 8 biases

struct Vol {
  int B, Nz, Ny, Nx, V;
};

__device__ __forceinline__ void decompose(int v, const Vol& g, int& z, int& y, int& x) {
  x = v % g.Nx;
  const int r = v / g.Nx;
  y = r % g.Ny;
  z = r / g.Ny;
}

// neighbour v + (dz - 1, dy - 1, dx - 1) (sign +1) or v - (dz - 1, ...) (sign -1); -1 outside
__device__ __forceinline__ int neighbour(int z, int y, int x, int t, int sign, const Vol& g) {
  const int dz = t / 9 - 1, dy = (t / 3) % 3 - 1, dx = t % 3 - 1;
  const int zz = z + sign * dz, yy = y + sign * dy, xx = x + sign * dx;
  if (zz < 0 || zz >= g.Nz || yy < 0 || yy >= g.Ny || xx < 0 || xx >= g.Nx) return -1;
  return (zz * g.Ny + yy) * g.Nx + xx;
}

// y_n = y / sigma_b, sigma_b = max |A^H y_b| / L (the max from the float bits
// in scal; sigma_b = 1 if the max is 0)
__global__ void normalize_kernel(const float2* __restrict__ y, const float* __restrict__ scal,
                                 float2* __restrict__ yn, float* __restrict__ sigma, float invL, int B, int n) {
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < B * n; i += gridDim.x * blockDim.x) {
    const int b = i / n;
    float s = scal[b * kNumFloatScalars + kLamMax] * invL;
    if (!(s > 0.f)) s = 1.f;
    if (i % n == 0) sigma[b] = s;
    const float2 v = y[i];
    yn[i] = make_float2(v.x / s, v.y / s);
  }
}

// z = x - (eta / L) g, s = tau_theta(z)  (x == nullptr: x = 0)
__global__ void shrink_fwd_kernel(const float2* __restrict__ x, const float2* __restrict__ g,
                                  const float* __restrict__ par, float invL, float2* __restrict__ z,
                                  float2* __restrict__ s, int n) {
  const float eta = par[0] * invL, theta = par[1];
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) {
    const float2 xv = x ? x[i] : make_float2(0.f, 0.f);
    const float2 gv = g[i];
    const float2 zv = make_float2(fmaf(-eta, gv.x, xv.x), fmaf(-eta, gv.y, xv.y));
    const float r = hypotf(zv.x, zv.y);
    const float sc = r > theta ? 1.f - theta / r : 0.f;
    z[i] = zv;
    s[i] = make_float2(zv.x * sc, zv.y * sc);
  }
}

// FP16 weights of one layer's convolution to FP32 in shared memory
__device__ __forceinline__ void load_weights(const __half* __restrict__ w16, float* w, int n) {
  for (int i = threadIdx.x; i < n; i += blockDim.x) w[i] = __half2float(w16[i]);
}

// h[b][c][v] = b1[c] + sum_{i, t} W1[c][i][t] s_i(v + t - 1)
__global__ void __launch_bounds__(kThreads) conv1_fwd_kernel(const float2* __restrict__ s,
                                                             const __half* __restrict__ w16,
                                                             const float* __restrict__ par,
                                                             float* __restrict__ h, Vol g) {
  __shared__ float w[kW1];
  load_weights(w16, w, kW1);
  __syncthreads();
  for (int idx = blockIdx.x * blockDim.x + threadIdx.x; idx < g.B * g.V; idx += gridDim.x * blockDim.x) {
    const int b = idx / g.V, v = idx - b * g.V;
    int z, y, x;
    decompose(v, g, z, y, x);
    float acc[kC];
#pragma unroll
    for (int c = 0; c < kC; ++c) acc[c] = par[kOffB1 + c];
    const float2* sb = s + (size_t)b * g.V;
    for (int t = 0; t < kTaps; ++t) {
      const int nv = neighbour(z, y, x, t, 1, g);
      if (nv < 0) continue;
      const float2 sv = __ldg(sb + nv);
#pragma unroll
      for (int c = 0; c < kC; ++c) acc[c] = fmaf(w[(c * 2 + 0) * kTaps + t], sv.x, fmaf(w[(c * 2 + 1) * kTaps + t], sv.y, acc[c]));
    }
#pragma unroll
    for (int c = 0; c < kC; ++c) h[((size_t)b * kC + c) * g.V + v] = acc[c];
  }
}

// x_next = s + (b2 + sum_{c, t} W2[o][c][t] relu(h[c](v + t - 1)))
__global__ void __launch_bounds__(kThreads) conv2_fwd_kernel(const float* __restrict__ h,
                                                             const float2* __restrict__ s,
                                                             const __half* __restrict__ w16,
                                                             const float* __restrict__ par,
                                                             float2* __restrict__ xn, Vol g) {
  __shared__ float w[kW2];
  load_weights(w16, w, kW2);
  __syncthreads();
  for (int idx = blockIdx.x * blockDim.x + threadIdx.x; idx < g.B * g.V; idx += gridDim.x * blockDim.x) {
    const int b = idx / g.V, v = idx - b * g.V;
    int z, y, x;
    decompose(v, g, z, y, x);
    float a0 = par[kOffB2], a1 = par[kOffB2 + 1];
    const float* hb = h + (size_t)b * kC * g.V;
    for (int t = 0; t < kTaps; ++t) {
      const int nv = neighbour(z, y, x, t, 1, g);
      if (nv < 0) continue;
#pragma unroll
      for (int c = 0; c < kC; ++c) {
        const float a = fmaxf(__ldg(hb + (size_t)c * g.V + nv), 0.f);
        a0 = fmaf(w[(0 * kC + c) * kTaps + t], a, a0);
        a1 = fmaf(w[(1 * kC + c) * kTaps + t], a, a1);
      }
    }
    const float2 sv = s[idx];
    xn[idx] = make_float2(sv.x + a0, sv.y + a1);
  }
}

// gh[c](v) = [h[c](v) > 0] sum_{o, t} W2[o][c][t] gx[o](v - t + 1)
__global__ void __launch_bounds__(kThreads) conv2_bwd_kernel(const float2* __restrict__ gx,
                                                             const float* __restrict__ h,
                                                             const __half* __restrict__ w16,
                                                             float* __restrict__ gh, Vol g) {
  __shared__ float w[kW2];
  load_weights(w16, w, kW2);
  __syncthreads();
  for (int idx = blockIdx.x * blockDim.x + threadIdx.x; idx < g.B * g.V; idx += gridDim.x * blockDim.x) {
    const int b = idx / g.V, v = idx - b * g.V;
    int z, y, x;
    decompose(v, g, z, y, x);
    float acc[kC];
#pragma unroll
    for (int c = 0; c < kC; ++c) acc[c] = 0.f;
    const float2* gb = gx + (size_t)b * g.V;
    for (int t = 0; t < kTaps; ++t) {
      const int nv = neighbour(z, y, x, t, -1, g);
      if (nv < 0) continue;
      const float2 gv = __ldg(gb + nv);
#pragma unroll
      for (int c = 0; c < kC; ++c)
        acc[c] = fmaf(w[(0 * kC + c) * kTaps + t], gv.x, fmaf(w[(1 * kC + c) * kTaps + t], gv.y, acc[c]));
    }
#pragma unroll
    for (int c = 0; c < kC; ++c) {
      const size_t o = ((size_t)b * kC + c) * g.V + v;
      gh[o] = h[o] > 0.f ? acc[c] : 0.f;
    }
  }
}

// gs(v) = gx(v) + sum_{c, t} W1[c][i][t] gh[c](v - t + 1)   (i = re, im)
__global__ void __launch_bounds__(kThreads) conv1_bwd_kernel(const float* __restrict__ gh,
                                                             const float2* __restrict__ gx,
                                                             const __half* __restrict__ w16,
                                                             float2* __restrict__ gs, Vol g) {
  __shared__ float w[kW1];
  load_weights(w16, w, kW1);
  __syncthreads();
  for (int idx = blockIdx.x * blockDim.x + threadIdx.x; idx < g.B * g.V; idx += gridDim.x * blockDim.x) {
    const int b = idx / g.V, v = idx - b * g.V;
    int z, y, x;
    decompose(v, g, z, y, x);
    const float2 gv = gx[idx];
    float a0 = gv.x, a1 = gv.y;
    const float* hb = gh + (size_t)b * kC * g.V;
    for (int t = 0; t < kTaps; ++t) {
      const int nv = neighbour(z, y, x, t, -1, g);
      if (nv < 0) continue;
#pragma unroll
      for (int c = 0; c < kC; ++c) {
        const float q = __ldg(hb + (size_t)c * g.V + nv);
        a0 = fmaf(w[(c * 2 + 0) * kTaps + t], q, a0);
        a1 = fmaf(w[(c * 2 + 1) * kTaps + t], q, a1);
      }
    }
    gs[idx] = make_float2(a0, a1);
  }
}

// Block sum of n values per thread into out[0..n) (thread 0 writes).
template <int N>
__device__ __forceinline__ void block_sum(float (&v)[N], float* out) {
  __shared__ float part[kThreads / 32][N];
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
#pragma unroll
  for (int k = 0; k < N; ++k) {
    float a = v[k];
#pragma unroll
    for (int off = 16; off > 0; off >>= 1) a += __shfl_xor_sync(0xffffffffu, a, off);
    if (lane == 0) part[warp][k] = a;
  }
  __syncthreads();
  if (threadIdx.x < N) {
    float a = 0.f;
    for (int w = 0; w < kThreads / 32; ++w) a += part[w][threadIdx.x];
    out[threadIdx.x] = a;
  }
}

// Partial sums of the second convolution's weight gradient (WHICH = 2:
// dW2[o][c][t] = sum gx[o](v) relu(h[c](v + t - 1)), bias sums at the centre
// tap) or of the first (WHICH = 1: dW1[c][i][t] = sum gh[c](v) s_i(v + t - 1)).
// Block (t, chunk) writes part[(t * kChunks + chunk) * kWAcc + k].
template <int WHICH>
__global__ void __launch_bounds__(kThreads) wgrad_kernel(const float2* __restrict__ gx, const float* __restrict__ h,
                                                         const float* __restrict__ gh, const float2* __restrict__ s,
                                                         float* __restrict__ part, Vol g) {
  const int t = blockIdx.x, chunk = blockIdx.y;
  float acc[kWAcc];
#pragma unroll
  for (int k = 0; k < kWAcc; ++k) acc[k] = 0.f;
  const int total = g.B * g.V;
  const int per = (total + kChunks - 1) / kChunks;
  const int i0 = chunk * per, i1 = min(total, i0 + per);
  for (int idx = i0 + threadIdx.x; idx < i1; idx += kThreads) {
    const int b = idx / g.V, v = idx - b * g.V;
    int z, y, x;
    decompose(v, g, z, y, x);
    const int nv = neighbour(z, y, x, t, 1, g);
    if (WHICH == 2) {
      const float2 gv = gx[idx];
      if (nv >= 0) {
        const float* hb = h + (size_t)b * kC * g.V + nv;
#pragma unroll
        for (int c = 0; c < kC; ++c) {
          const float a = fmaxf(hb[(size_t)c * g.V], 0.f);
          acc[c] = fmaf(gv.x, a, acc[c]);
          acc[kC + c] = fmaf(gv.y, a, acc[kC + c]);
        }
      }
      acc[16] += gv.x;
      acc[17] += gv.y;
    } else {
      const float2 sv = nv >= 0 ? s[(size_t)b * g.V + nv] : make_float2(0.f, 0.f);
      const float* gb = gh + (size_t)b * kC * g.V + v;
#pragma unroll
      for (int c = 0; c < kC; ++c) {
        const float q = gb[(size_t)c * g.V];
        acc[2 * c] = fmaf(q, sv.x, acc[2 * c]);
        acc[2 * c + 1] = fmaf(q, sv.y, acc[2 * c + 1]);
        acc[16 + c] += q;
      }
    }
  }
  block_sum<kWAcc>(acc, part + ((size_t)t * kChunks + chunk) * kWAcc);
}

// Sum of the partials over chunks (FP64, fixed order) into the layer's
// gradient slots.  One thread per (t, k).
template <int WHICH>
__global__ void wgrad_reduce_kernel(const float* __restrict__ part, float* __restrict__ grad) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= kTaps * kWAcc) return;
  const int t = i / kWAcc, k = i % kWAcc;
  double a = 0.0;
  for (int ch = 0; ch < kChunks; ++ch) a += part[((size_t)t * kChunks + ch) * kWAcc + k];
  if (WHICH == 2) {
    if (k < 16) grad[kOffW2 + ((k / kC) * kC + (k % kC)) * kTaps + t] = (float)a;  // o = k / 8, c = k % 8
    else if (k < 18 && t == 13) grad[kOffB2 + (k - 16)] = (float)a;
  } else {
    if (k < 16) grad[kOffW1 + ((k / 2) * 2 + (k % 2)) * kTaps + t] = (float)a;     // c = k / 2, i = k % 2
    else if (t == 13) grad[kOffB1 + (k - 16)] = (float)a;
  }
}

// Soft-threshold backward: gz and per-block partials of dtheta, deta.
__global__ void __launch_bounds__(kThreads) shrink_bwd_kernel(const float2* __restrict__ gs,
                                                              const float2* __restrict__ z,
                                                              const float2* __restrict__ gg,
                                                              const float* __restrict__ par,
                                                              float2* __restrict__ gz,
                                                              float* __restrict__ part, int n) {
  const float theta = par[1];
  float acc[2] = {0.f, 0.f};  // dtheta, deta
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) {
    const float2 zv = z[i], gv = gs[i];
    const float r = hypotf(zv.x, zv.y);
    float2 out = make_float2(0.f, 0.f);
    if (r > theta) {
      const float ux = zv.x / r, uy = zv.y / r;
      const float ug = ux * gv.x + uy * gv.y;
      const float a = 1.f - theta / r, bq = theta / r * ug;
      out = make_float2(fmaf(a, gv.x, bq * ux), fmaf(a, gv.y, bq * uy));
      acc[0] -= ug;
    }
    gz[i] = out;
    const float2 g = gg[i];
    acc[1] -= g.x * out.x + g.y * out.y;
  }
  block_sum<2>(acc, part + 2 * blockIdx.x);
}

__global__ void shrink_reduce_kernel(const float* __restrict__ part, int nblocks, double invL,
                                     float* __restrict__ grad) {
  if (threadIdx.x >= 2) return;
  double a = 0.0;
  for (int i = 0; i < nblocks; ++i) a += part[2 * i + threadIdx.x];
  // part[0] = dtheta -> slot 1, part[1] = L deta -> slot 0
  grad[threadIdx.x == 0 ? 1 : 0] = (float)(threadIdx.x == 0 ? a : a * invL);
}

// out = a - (eta / L) q  (eta = par[0])
__global__ void axpy_kernel(const float2* __restrict__ a, const float2* __restrict__ q,
                            const float* __restrict__ par, float invL, float2* __restrict__ out, int n) {
  const float eta = par[0] * invL;
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) {
    const float2 av = a[i], qv = q[i];
    out[i] = make_float2(fmaf(-eta, qv.x, av.x), fmaf(-eta, qv.y, av.y));
  }
}

// out[b][v] = sigma_b in[b][v]
__global__ void scale_kernel(const float2* __restrict__ in, const float* __restrict__ sigma,
                             float2* __restrict__ out, int B, int V) {
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < B * V; i += gridDim.x * blockDim.x) {
    const float s = sigma[i / V];
    const float2 v = in[i];
    out[i] = make_float2(s * v.x, s * v.y);
  }
}

// per-scene sums |x - t|^2 and |t|^2 (blockIdx.y = scene)
__global__ void __launch_bounds__(kThreads) nmse_sums_kernel(const float2* __restrict__ x,
                                                             const float2* __restrict__ t,
                                                             double* __restrict__ sums, int V) {
  const int b = blockIdx.y;
  double a[2] = {0.0, 0.0};
  for (int v = blockIdx.x * blockDim.x + threadIdx.x; v < V; v += gridDim.x * blockDim.x) {
    const float2 xv = x[(size_t)b * V + v], tv = t[(size_t)b * V + v];
    const double dx = (double)xv.x - tv.x, dy = (double)xv.y - tv.y;
    a[0] += dx * dx + dy * dy;
    a[1] += (double)tv.x * tv.x + (double)tv.y * tv.y;
  }
  __shared__ double part[kThreads / 32][2];
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  for (int k = 0; k < 2; ++k) {
    double q = a[k];
    for (int off = 16; off > 0; off >>= 1) q += __shfl_xor_sync(0xffffffffu, q, off);
    if (lane == 0) part[warp][k] = q;
  }
  __syncthreads();
  if (threadIdx.x < 2) {
    double q = 0.0;
    for (int w = 0; w < kThreads / 32; ++w) q += part[w][threadIdx.x];
    atomicAdd(sums + 2 * b + threadIdx.x, q);
  }
}

// grad[b][v] = 2 (x - t) / (B |t_b|^2)
__global__ void nmse_grad_kernel(const float2* __restrict__ x, const float2* __restrict__ t,
                                 const double* __restrict__ sums, float2* __restrict__ grad, int B, int V) {
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < B * V; i += gridDim.x * blockDim.x) {
    const double den = sums[2 * (i / V) + 1];
    const float f = den > 0.0 ? (float)(2.0 / (B * den)) : 0.f;
    const float2 xv = x[i], tv = t[i];
    grad[i] = make_float2(f * (xv.x - tv.x), f * (xv.y - tv.y));
  }
}

// Adam (bias-corrected) on the FP32 parameters (the FP16 weight copies are
// refreshed by weights16_kernel afterwards).
__global__ void adam_kernel(float* __restrict__ p, float* __restrict__ m, float* __restrict__ v,
                            const float* __restrict__ g, int n, float lr,
                            float b1, float b2, float eps, float c1, float c2) {
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) {
    const float gi = g[i];
    const float mi = b1 * m[i] + (1.f - b1) * gi;
    const float vi = b2 * v[i] + (1.f - b2) * gi * gi;
    m[i] = mi;
    v[i] = vi;
    const float pi = p[i] - lr * (mi / c1) / (sqrtf(vi / c2) + eps);
    p[i] = pi;
  }
}

// FP16 copies of the convolution weights: w16[l][0..kW1) = W1_l, [kW1..) = W2_l
__global__ void weights16_kernel(const float* __restrict__ p, __half* __restrict__ w16, int layers) {
  const int n = layers * (kW1 + kW2);
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) {
    const int l = i / (kW1 + kW2), k = i % (kW1 + kW2);
    const float w = k < kW1 ? p[l * kPerLayer + kOffW1 + k] : p[l * kPerLayer + kOffW2 + (k - kW1)];
    w16[i] = __float2half_rn(w);
  }
}

int grid_for(long long n) { return (int)std::max(1LL, std::min((n + kThreads - 1) / kThreads, 152LL * 8)); }

}  // namespace
}  // namespace sfs

using namespace sfs;

struct sfs_lista {
  sfs_operator* op = nullptr;
  double L = 1.0;  // normalisation: ||A^H y_n||_inf = L
  int layers = 0, cap = 0;
  int S = 0, M = 0, U = 0, V = 0, Nz = 0, Ny = 0, Nx = 0;
  float* par = nullptr;     // [layers][876] FP32 master parameters
  float* adam_m = nullptr;  // Adam moments
  float* adam_v = nullptr;
  __half* w16 = nullptr;    // [layers][kW1 + kW2] FP16 convolution weights
  // activations of the last saved forward, [cap] scenes each
  float2* yn = nullptr;      // [cap][S][M]
  float2* yplane = nullptr;  // [cap][U][S]
  float2* zplane = nullptr;  // [cap][U][S] zeros (A^H A)
  float* scal = nullptr;     // [cap][kNumFloatScalars]
  float* sigma = nullptr;    // [cap]
  float2* xs = nullptr;      // [layers + 1][cap][V]  x_0 .. x_L
  float2* gs = nullptr;      // [layers][cap][V]      g_l
  float2* zs = nullptr;      // [layers][cap][V]      z_l
  float2* ss = nullptr;      // [layers][cap][V]      s_l
  float* hs = nullptr;       // [layers][cap][8][V]   h_l
  float2* t0 = nullptr;      // [cap][V] scratch (gradients)
  float2* t1 = nullptr;
  float2* t2 = nullptr;
  float* ghid = nullptr;     // [cap][8][V]
  float* part = nullptr;     // reduction partials
  double* sums = nullptr;    // [cap][2]
  int saved_batch = 0;
};

namespace {

template <typename T>
int alloc(T** p, size_t n) {
  const cudaError_t e = cudaMalloc((void**)p, std::max<size_t>(1, n) * sizeof(T));
  if (e != cudaSuccess) {
    *p = nullptr;
    return cuda_fail(e, "cudaMalloc", __FILE__, __LINE__);
  }
  return SFS_OK;
}

void free_net(sfs_lista* n) {
  void* ptrs[] = {n->par, n->adam_m, n->adam_v, n->w16, n->yn, n->yplane, n->zplane, n->scal,
                  n->sigma, n->xs, n->gs, n->zs, n->ss, n->hs, n->t0, n->t1, n->t2, n->ghid,
                  n->part, n->sums};
  for (void* p : ptrs) cudaFree(p);
  delete n;
}

struct Scope {
  int prev = -1;
  explicit Scope(int dev) {
    if (cudaGetDevice(&prev) != cudaSuccess) prev = -1;
    cudaSetDevice(dev);
  }
  ~Scope() {
    if (prev >= 0) cudaSetDevice(prev);
  }
};

Vol vol_of(const sfs_lista* n, int B) { return Vol{B, n->Nz, n->Ny, n->Nx, n->V}; }

}  // namespace

extern "C" {

int sfs_lista_create(sfs_operator* op, int layers, int max_batch, double L, sfs_lista** out) {
  clear_error();
  if (!op || !out || layers < 1 || layers > 64 || max_batch < 1 || max_batch > SFS_MAX_BATCH ||
      !(L > 0) || !isfinite(L)) {
    set_error("invalid argument (layers 1..64, max_batch 1..%d, L > 0)", SFS_MAX_BATCH);
    return SFS_ERR_INVALID_ARG;
  }
  *out = nullptr;
  Scope scope(operator_device(op));
  sfs_operator_info_t info;
  SFS_TRY(sfs_operator_info(op, &info));
  sfs_lista* n = new (std::nothrow) sfs_lista;
  if (!n) {
    set_error("host allocation failed");
    return SFS_ERR_OOM;
  }
  n->op = op;
  n->L = L;
  n->layers = layers;
  n->cap = max_batch;
  n->S = info.S;
  n->M = info.M;
  n->U = info.U;
  n->V = info.V;
  n->Nz = info.Nz;
  n->Ny = op->geo.d.Ny;
  n->Nx = op->geo.d.Nx;
  const size_t C = max_batch, Vz = info.V, P = (size_t)layers * kPerLayer;
  int rc = SFS_OK;
  auto A = [&](auto** p, size_t cnt) {
    if (rc == SFS_OK) rc = alloc(p, cnt);
  };
  A(&n->par, P);
  A(&n->adam_m, P);
  A(&n->adam_v, P);
  A(&n->w16, (size_t)layers * (kW1 + kW2));
  A(&n->yn, C * info.S * info.M);
  A(&n->yplane, C * info.U * info.S);
  A(&n->zplane, C * info.U * info.S);
  A(&n->scal, C * kNumFloatScalars);
  A(&n->sigma, C);
  A(&n->xs, (layers + 1) * C * Vz);
  A(&n->gs, layers * C * Vz);
  A(&n->zs, layers * C * Vz);
  A(&n->ss, layers * C * Vz);
  A(&n->hs, layers * C * kC * Vz);
  A(&n->t0, C * Vz);
  A(&n->t1, C * Vz);
  A(&n->t2, C * Vz);
  A(&n->ghid, C * kC * Vz);
  A(&n->part, std::max<size_t>((size_t)kTaps * kChunks * kWAcc, 2 * 8192));
  A(&n->sums, 2 * C);
  if (rc == SFS_OK) {
    cudaError_t e = cudaMemset(n->par, 0, P * sizeof(float));
    if (e == cudaSuccess) e = cudaMemset(n->adam_m, 0, P * sizeof(float));
    if (e == cudaSuccess) e = cudaMemset(n->adam_v, 0, P * sizeof(float));
    if (e == cudaSuccess) e = cudaMemset(n->w16, 0, (size_t)layers * (kW1 + kW2) * sizeof(__half));
    if (e == cudaSuccess) e = cudaMemset(n->zplane, 0, C * info.U * info.S * sizeof(float2));
    if (e == cudaSuccess) e = cudaMemset(n->xs, 0, C * Vz * sizeof(float2));  // x_0 = 0
    if (e != cudaSuccess) rc = cuda_fail(e, "initialising the network", __FILE__, __LINE__);
  }
  if (rc == SFS_OK) rc = batch_workspace(op, max_batch);
  if (rc != SFS_OK) {
    free_net(n);
    return rc;
  }
  *out = n;
  return SFS_OK;
}

int sfs_lista_destroy(sfs_lista* net) {
  if (!net) return SFS_OK;
  Scope scope(operator_device(net->op));
  free_net(net);
  return SFS_OK;
}

int sfs_lista_info(const sfs_lista* net, int32_t* layers, int32_t* nparams) {
  clear_error();
  if (!net || !layers || !nparams) {
    set_error("null argument");
    return SFS_ERR_INVALID_ARG;
  }
  *layers = net->layers;
  *nparams = net->layers * kPerLayer;
  return SFS_OK;
}

int sfs_lista_set_params(sfs_lista* net, const float* params_host) {
  clear_error();
  if (!net || !params_host) {
    set_error("null argument");
    return SFS_ERR_INVALID_ARG;
  }
  Scope scope(operator_device(net->op));
  const size_t P = (size_t)net->layers * kPerLayer;
  SFS_CUDA(cudaMemcpy(net->par, params_host, P * sizeof(float), cudaMemcpyHostToDevice));
  SFS_CUDA(cudaMemset(net->adam_m, 0, P * sizeof(float)));
  SFS_CUDA(cudaMemset(net->adam_v, 0, P * sizeof(float)));
  weights16_kernel<<<grid_for((long long)net->layers * (kW1 + kW2)), kThreads>>>(net->par, net->w16, net->layers);
  SFS_CUDA(cudaGetLastError());
  SFS_CUDA(cudaDeviceSynchronize());
  return SFS_OK;
}

int sfs_lista_load_params_dev(sfs_lista* net, const void* params_dev, void* stream) {
  clear_error();
  if (!net || !params_dev || ((uintptr_t)params_dev & 3u)) {
    set_error("invalid argument");
    return SFS_ERR_INVALID_ARG;
  }
  Scope scope(operator_device(net->op));
  cudaStream_t st = (cudaStream_t)stream;
  SFS_CUDA(cudaMemcpyAsync(net->par, params_dev, (size_t)net->layers * kPerLayer * sizeof(float),
                           cudaMemcpyDeviceToDevice, st));
  weights16_kernel<<<grid_for((long long)net->layers * (kW1 + kW2)), kThreads, 0, st>>>(net->par, net->w16,
                                                                                        net->layers);
  SFS_CUDA(cudaGetLastError());
  return SFS_OK;
}

int sfs_lista_get_params(const sfs_lista* net, float* params_host) {
  clear_error();
  if (!net || !params_host) {
    set_error("null argument");
    return SFS_ERR_INVALID_ARG;
  }
  Scope scope(operator_device(net->op));
  SFS_CUDA(cudaMemcpy(params_host, net->par, (size_t)net->layers * kPerLayer * sizeof(float),
                      cudaMemcpyDeviceToHost));
  return SFS_OK;
}

int sfs_lista_forward(sfs_lista* net, int batch, const void* y_dev, void* x_dev, void* stream) {
  clear_error();
  if (!net || !y_dev || !x_dev || batch < 1 || batch > net->cap || ((uintptr_t)y_dev & 15u) ||
      ((uintptr_t)x_dev & 15u)) {
    set_error("invalid argument (batch 1..%d, 16-byte aligned pointers)", net ? net->cap : 0);
    return SFS_ERR_INVALID_ARG;
  }
  Scope scope(operator_device(net->op));
  cudaStream_t st = (cudaStream_t)stream;
  const int B = batch, V = net->V;
  const long long nV = (long long)B * V;
  const Vol g = vol_of(net, B);
  // sigma_b = ||A^H y_b||_inf, y_n = y / sigma, by bin plane
  SFS_CUDA(cudaMemsetAsync(net->scal, 0, (size_t)B * kNumFloatScalars * sizeof(float), st));
  SFS_TRY(batched_maxabs_AH(net->op, B, (const float2*)y_dev, net->scal, st));
  const int ny = net->S * net->M;
  normalize_kernel<<<grid_for((long long)B * ny), kThreads, 0, st>>>((const float2*)y_dev, net->scal, net->yn,
                                                                      net->sigma, (float)(1.0 / net->L), B, ny);
  SFS_CUDA(cudaGetLastError());
  SFS_TRY(batched_scatter_y(net->op, B, net->yn, net->yplane, st));
  for (int l = 0; l < net->layers; ++l) {
    const float* par = net->par + (size_t)l * kPerLayer;
    const __half* w1 = net->w16 + (size_t)l * (kW1 + kW2);
    const __half* w2 = w1 + kW1;
    float2* xl = net->xs + (size_t)l * net->cap * V;
    float2* xn = net->xs + (size_t)(l + 1) * net->cap * V;
    float2* gl = net->gs + (size_t)l * net->cap * V;
    float2* zl = net->zs + (size_t)l * net->cap * V;
    float2* sl = net->ss + (size_t)l * net->cap * V;
    float* hl = net->hs + (size_t)l * net->cap * kC * V;
    SFS_TRY(batched_normal_residual(net->op, B, xl, net->yplane, gl, st));
    shrink_fwd_kernel<<<grid_for(nV), kThreads, 0, st>>>(l == 0 ? nullptr : xl, gl, par, (float)(1.0 / net->L),
                                                          zl, sl, (int)nV);
    conv1_fwd_kernel<<<grid_for(nV), kThreads, 0, st>>>(sl, w1, par, hl, g);
    conv2_fwd_kernel<<<grid_for(nV), kThreads, 0, st>>>(hl, sl, w2, par, xn, g);
    SFS_CUDA(cudaGetLastError());
  }
  scale_kernel<<<grid_for(nV), kThreads, 0, st>>>(net->xs + (size_t)net->layers * net->cap * V, net->sigma,
                                                   (float2*)x_dev, B, V);
  SFS_CUDA(cudaGetLastError());
  net->saved_batch = B;
  return SFS_OK;
}

int sfs_lista_backward(sfs_lista* net, int batch, const void* grad_x_dev, void* grad_params_dev,
                       void* stream) {
  clear_error();
  if (!net || !grad_x_dev || !grad_params_dev || batch != net->saved_batch || batch < 1 ||
      ((uintptr_t)grad_x_dev & 15u) || ((uintptr_t)grad_params_dev & 3u)) {
    set_error("invalid argument (batch must equal the last forward's)");
    return SFS_ERR_INVALID_ARG;
  }
  Scope scope(operator_device(net->op));
  cudaStream_t st = (cudaStream_t)stream;
  const int B = batch, V = net->V;
  const long long nV = (long long)B * V;
  const Vol g = vol_of(net, B);
  float* grad = (float*)grad_params_dev;
  // d/d x_L = sigma d/d x
  float2* gx = net->t0;
  scale_kernel<<<grid_for(nV), kThreads, 0, st>>>((const float2*)grad_x_dev, net->sigma, gx, B, V);
  SFS_CUDA(cudaGetLastError());
  const int sblocks = grid_for(nV);
  for (int l = net->layers - 1; l >= 0; --l) {
    const float* par = net->par + (size_t)l * kPerLayer;
    float* gp = grad + (size_t)l * kPerLayer;
    const __half* w1 = net->w16 + (size_t)l * (kW1 + kW2);
    const __half* w2 = w1 + kW1;
    const float2* gl = net->gs + (size_t)l * net->cap * V;
    const float2* zl = net->zs + (size_t)l * net->cap * V;
    const float2* sl = net->ss + (size_t)l * net->cap * V;
    const float* hl = net->hs + (size_t)l * net->cap * kC * V;
    // second convolution
    wgrad_kernel<2><<<dim3(kTaps, kChunks), kThreads, 0, st>>>(gx, hl, nullptr, nullptr, net->part, g);
    wgrad_reduce_kernel<2><<<(kTaps * kWAcc + 127) / 128, 128, 0, st>>>(net->part, gp);
    conv2_bwd_kernel<<<grid_for(nV), kThreads, 0, st>>>(gx, hl, w2, net->ghid, g);
    // first convolution
    wgrad_kernel<1><<<dim3(kTaps, kChunks), kThreads, 0, st>>>(nullptr, nullptr, net->ghid, sl, net->part, g);
    wgrad_reduce_kernel<1><<<(kTaps * kWAcc + 127) / 128, 128, 0, st>>>(net->part, gp);
    float2* gsv = net->t1;
    conv1_bwd_kernel<<<grid_for(nV), kThreads, 0, st>>>(net->ghid, gx, w1, gsv, g);
    // soft threshold and step
    float2* gz = net->t2;
    shrink_bwd_kernel<<<sblocks, kThreads, 0, st>>>(gsv, zl, gl, par, gz, net->part, (int)nV);
    shrink_reduce_kernel<<<1, 32, 0, st>>>(net->part, sblocks, 1.0 / net->L, gp);
    SFS_CUDA(cudaGetLastError());
    if (l > 0) {
      // gx_prev = gz - eta A^H A gz
      SFS_TRY(batched_normal_residual(net->op, B, gz, net->zplane, net->t1, st));
      axpy_kernel<<<grid_for(nV), kThreads, 0, st>>>(gz, net->t1, par, (float)(1.0 / net->L), gx, (int)nV);
      SFS_CUDA(cudaGetLastError());
    }
  }
  return SFS_OK;
}

int sfs_lista_nmse(sfs_lista* net, int batch, const void* x_dev, const void* xtrue_dev, void* grad_x_dev,
                   double* loss_host, void* stream) {
  clear_error();
  if (!net || !x_dev || !xtrue_dev || !loss_host || batch < 1 || batch > net->cap) {
    set_error("invalid argument");
    return SFS_ERR_INVALID_ARG;
  }
  Scope scope(operator_device(net->op));
  cudaStream_t st = (cudaStream_t)stream;
  const int B = batch, V = net->V;
  SFS_CUDA(cudaMemsetAsync(net->sums, 0, 2 * B * sizeof(double), st));
  nmse_sums_kernel<<<dim3(std::max(1, std::min(64, (V + kThreads - 1) / kThreads)), B), kThreads, 0, st>>>(
      (const float2*)x_dev, (const float2*)xtrue_dev, net->sums, V);
  if (grad_x_dev)
    nmse_grad_kernel<<<grid_for((long long)B * V), kThreads, 0, st>>>(
        (const float2*)x_dev, (const float2*)xtrue_dev, net->sums, (float2*)grad_x_dev, B, V);
  SFS_CUDA(cudaGetLastError());
  std::vector<double> h(2 * B);
  SFS_CUDA(cudaMemcpyAsync(h.data(), net->sums, h.size() * sizeof(double), cudaMemcpyDeviceToHost, st));
  SFS_CUDA(cudaStreamSynchronize(st));
  double l = 0.0;
  for (int b = 0; b < B; ++b) l += h[2 * b + 1] > 0 ? h[2 * b] / h[2 * b + 1] : 0.0;
  *loss_host = l / B;
  return SFS_OK;
}

int sfs_lista_adam(sfs_lista* net, const void* grad_params_dev, float lr, float beta1, float beta2,
                   float eps, int step, void* stream) {
  clear_error();
  if (!net || !grad_params_dev || step < 1 || !(lr > 0.f)) {
    set_error("invalid argument");
    return SFS_ERR_INVALID_ARG;
  }
  Scope scope(operator_device(net->op));
  cudaStream_t st = (cudaStream_t)stream;
  const int P = net->layers * kPerLayer;
  const float c1 = 1.f - powf(beta1, (float)step), c2 = 1.f - powf(beta2, (float)step);
  adam_kernel<<<grid_for(P), kThreads, 0, st>>>(net->par, net->adam_m, net->adam_v, (const float*)grad_params_dev,
                                                 P, lr, beta1, beta2, eps, c1, c2);
  weights16_kernel<<<grid_for((long long)net->layers * (kW1 + kW2)), kThreads, 0, st>>>(net->par, net->w16,
                                                                                        net->layers);
  SFS_CUDA(cudaGetLastError());
  return SFS_OK;
}

}  // extern "C"
