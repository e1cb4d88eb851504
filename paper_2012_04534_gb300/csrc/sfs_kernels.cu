// Device kernels of libsfs (sm_103a).
//
// The forward operator A = S F H (Eq. (10), Sigma = I) is applied through the
// block 2-level Toeplitz structure of H (Theorem 2, Sec. IV-B): for each kept
// bin k and depth z the lateral kernel h_{k,z}[dy, dx] is convolved with the
// voxel plane x_z, the depth planes are summed, and the bin plane is sampled
// at the scan positions that keep bin k.  In the lateral Fourier domain the
// convolutions are products, so one apply is
//   Xh_z      = FFT2(pad(x_z))                       (fwd_planes)
//   Yh_u(kap) = sum_z T[kap][u][z] Xh_z(kap)         (contract_fwd)
//   y[s, m]   = IFFT2(Yh_u)(s) for bins[u] = idx[s,m] (inv_gather)
// and A^H is the same chain transposed (scatter_fwd, contract_adj,
// inv_store).  T holds FFT2 of the generators times 1/(Px Py), so the
// unnormalised forward and inverse FFTs make A and A^H exact adjoints.
// The two contractions stream T and dominate the run time; everything else
// works on single planes held in shared memory.
#include <cuda_runtime.h>
#include <stdint.h>

#include <mutex>
#include <unordered_map>

#include "sfs_fft.cuh"
#include "sfs_internal.h"

namespace sfs {
namespace {

// ---------------------------------------------------------------------------
// Block reductions
// ---------------------------------------------------------------------------
template <int NT>
__device__ __forceinline__ void block_add_double(double v, double* out) {
  __shared__ double part[NT / 32];
#pragma unroll
  for (int off = 16; off > 0; off >>= 1) v += __shfl_xor_sync(0xffffffffu, v, off);
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  if (lane == 0) part[warp] = v;
  __syncthreads();
  if (warp == 0) {
    v = lane < NT / 32 ? part[lane] : 0.0;
#pragma unroll
    for (int off = 16; off > 0; off >>= 1) v += __shfl_xor_sync(0xffffffffu, v, off);
    if (lane == 0) atomicAdd(out, v);
  }
}

template <int NT>
__device__ __forceinline__ void block_max_bits(float v, unsigned int* out) {
  __shared__ float part[NT / 32];
#pragma unroll
  for (int off = 16; off > 0; off >>= 1) v = fmaxf(v, __shfl_xor_sync(0xffffffffu, v, off));
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  if (lane == 0) part[warp] = v;
  __syncthreads();
  if (warp == 0) {
    v = lane < NT / 32 ? part[lane] : 0.0f;
#pragma unroll
    for (int off = 16; off > 0; off >>= 1) v = fmaxf(v, __shfl_xor_sync(0xffffffffu, v, off));
    // non-negative floats order like their bit patterns
    if (lane == 0) atomicMax(out, __float_as_uint(v));
  }
}

// ---------------------------------------------------------------------------
// Generator table: T[kt][u][z][ki] = FFT2(h_{bins[u], z}) / (Px Py)
// ---------------------------------------------------------------------------
// h_{k,z}[d] = fs H(f_k) g(d, z) exp(-j 2 pi f_k (tau(d, z) - t0)) (Eq. (4)),
// with the phase in turns k * Tn(d, z), Tn = (tau - t0) fs / Nt held as a
// float pair (hi + lo).  The product k * hi is split exactly with an FMA,
// its integer part removed exactly, and the small remainder plus k * lo
// added, so the reduced phase keeps ~1e-7 turn accuracy where a plain
// float product of ~100 turns would lose ~1e-5.
template <int P, bool TWO_D>
__global__ void __launch_bounds__(PlaneFFT<P, TWO_D>::NT)
build_table_kernel(PlaneDims d, const float2* __restrict__ tof,
                   const float* __restrict__ gdir, const float* __restrict__ amp,
                   const int32_t* __restrict__ bins, float2* __restrict__ table) {
  using F = PlaneFFT<P, TWO_D>;
  extern __shared__ float2 smem[];
  float2* buf = smem;
  float2* tw = smem + F::ELEMS;
  const int u = blockIdx.x / d.Nz, z = blockIdx.x % d.Nz;
  make_twiddles<P, F::NT>(tw);
  const float kf = (float)bins[u];
  const float a = amp[u];
  constexpr int PY = TWO_D ? P : 1;
  for (int e = threadIdx.x; e < P * PY; e += F::NT) {
    const int py = e / P, px = e % P;
    const int ady = TWO_D ? (py < d.Ny ? py : (py > P - d.Ny ? P - py : -1)) : 0;
    const int adx = px < d.Nx ? px : (px > P - d.Nx ? P - px : -1);
    float2 val = make_float2(0.f, 0.f);
    if (ady >= 0 && adx >= 0) {
      const int ti = (z * d.Ny + ady) * d.Nx + adx;
      const float2 tn = tof[ti];
      const float p = kf * tn.x;
      const float err = fmaf(kf, tn.x, -p);
      const float r = p - rintf(p);
      const float t = r + fmaf(kf, tn.y, err);
      float s, c;
      sincospif(2.0f * t, &s, &c);
      const float m = a * gdir[ti];
      val = make_float2(m * c, -m * s);
    }
    buf[F::sidx(py, px)] = val;
  }
  __syncthreads();
  F::forward(buf, tw, P);
  for (int kap = threadIdx.x; kap < F::NK; kap += F::NT) {
    const size_t o = (((size_t)(kap >> 6) * d.U + u) * d.Nz + z) * kKappaTile + (kap & 63);
    table[o] = buf[F::kidx(kap)];
  }
}

// ---------------------------------------------------------------------------
// Plane kernels (one lateral plane per CTA)
// ---------------------------------------------------------------------------
template <int P, bool TWO_D>
__device__ __forceinline__ void zero_plane(float2* buf) {
  using F = PlaneFFT<P, TWO_D>;
  for (int e = threadIdx.x; e < F::ELEMS; e += F::NT) buf[e] = make_float2(0.f, 0.f);
}

template <int P, bool TWO_D>
__device__ __forceinline__ void load_spectrum(float2* buf, const float2* __restrict__ src) {
  using F = PlaneFFT<P, TWO_D>;
  for (int kap = threadIdx.x; kap < F::NK; kap += F::NT) buf[F::kidx(kap)] = src[kap];
}

template <int P, bool TWO_D>
__device__ __forceinline__ void store_spectrum(const float2* buf, float2* __restrict__ dst) {
  using F = PlaneFFT<P, TWO_D>;
  for (int kap = threadIdx.x; kap < F::NK; kap += F::NT) dst[kap] = buf[F::kidx(kap)];
}

// Zero every slot of the plane outside the Ny x Nx crop window.
template <int P, bool TWO_D>
__device__ __forceinline__ void zero_outside(float2* buf, int Ny, int Nx) {
  using F = PlaneFFT<P, TWO_D>;
  constexpr int PY = TWO_D ? P : 1;
  for (int e = threadIdx.x; e < P * PY; e += F::NT) {
    const int py = e / P, px = e % P;
    if (py >= Ny || px >= Nx) buf[F::sidx(py, px)] = make_float2(0.f, 0.f);
  }
}

// x plane z -> Xh[z] = FFT2(pad(x_z))
template <int P, bool TWO_D>
__global__ void __launch_bounds__(PlaneFFT<P, TWO_D>::NT)
fwd_planes_kernel(PlaneDims d, const float2* __restrict__ x, float2* __restrict__ Xh) {
  using F = PlaneFFT<P, TWO_D>;
  extern __shared__ float2 smem[];
  float2* buf = smem;
  float2* tw = smem + F::ELEMS;
  const int z = blockIdx.x;
  make_twiddles<P, F::NT>(tw);
  zero_plane<P, TWO_D>(buf);
  __syncthreads();
  const float2* xz = x + (size_t)z * d.Ny * d.Nx;
  for (int e = threadIdx.x; e < d.Ny * d.Nx; e += F::NT)
    buf[F::sidx(e / d.Nx, e % d.Nx)] = xz[e];
  __syncthreads();
  F::forward(buf, tw, d.Nx);
  store_spectrum<P, TWO_D>(buf, Xh + (size_t)z * d.Nk);
}

// Yh[u] -> y[s, m] = IFFT2(Yh_u)(s) where bins[u] = idx[s, m]
template <int P, bool TWO_D>
__global__ void __launch_bounds__(PlaneFFT<P, TWO_D>::NT)
inv_gather_kernel(PlaneDims d, const float2* __restrict__ Yh,
                  const int32_t* __restrict__ posmap, float2* __restrict__ y,
                  double* __restrict__ red_sumsq) {
  using F = PlaneFFT<P, TWO_D>;
  extern __shared__ float2 smem[];
  float2* buf = smem;
  float2* tw = smem + F::ELEMS;
  const int u = blockIdx.x;
  make_twiddles<P, F::NT>(tw);
  load_spectrum<P, TWO_D>(buf, Yh + (size_t)u * d.Nk);
  __syncthreads();
  F::inverse(buf, tw, d.Nx);
  double acc = 0.0;
  const int32_t* pm = posmap + (size_t)u * d.S;
  for (int s = threadIdx.x; s < d.S; s += F::NT) {
    const int m = pm[s];
    if (m >= 0) {
      const float2 v = buf[F::sidx(s / d.Nx, s % d.Nx)];
      y[(size_t)s * d.M + m] = v;
      acc += (double)v.x * v.x + (double)v.y * v.y;
    }
  }
  if (red_sumsq) block_add_double<F::NT>(acc, red_sumsq);
}

// Yh[u] -> residual r = (A gamma - y) on bin plane u -> Rh[u] = FFT2(pad(r_u))
template <int P, bool TWO_D>
__global__ void __launch_bounds__(PlaneFFT<P, TWO_D>::NT)
inv_resid_fwd_kernel(PlaneDims d, const float2* __restrict__ Yh,
                     const int32_t* __restrict__ posmap, const float2* __restrict__ yobs,
                     float2* __restrict__ Rh, double* __restrict__ red_sumsq) {
  using F = PlaneFFT<P, TWO_D>;
  extern __shared__ float2 smem[];
  float2* buf = smem;
  float2* tw = smem + F::ELEMS;
  const int u = blockIdx.x;
  make_twiddles<P, F::NT>(tw);
  load_spectrum<P, TWO_D>(buf, Yh + (size_t)u * d.Nk);
  __syncthreads();
  F::inverse(buf, tw, d.Nx);
  double acc = 0.0;
  const int32_t* pm = posmap + (size_t)u * d.S;
  for (int s = threadIdx.x; s < d.S; s += F::NT) {
    const int m = pm[s];
    const int e = F::sidx(s / d.Nx, s % d.Nx);
    float2 r = make_float2(0.f, 0.f);
    if (m >= 0) {
      r = csub(buf[e], yobs[(size_t)s * d.M + m]);
      acc += (double)r.x * r.x + (double)r.y * r.y;
    }
    buf[e] = r;
  }
  zero_outside<P, TWO_D>(buf, d.Ny, d.Nx);
  if (red_sumsq) block_add_double<F::NT>(acc, red_sumsq);
  __syncthreads();
  F::forward(buf, tw, d.Nx);
  store_spectrum<P, TWO_D>(buf, Rh + (size_t)u * d.Nk);
}

// y[s, m] scattered to bin plane u -> Rh[u] = FFT2(pad(.))
template <int P, bool TWO_D>
__global__ void __launch_bounds__(PlaneFFT<P, TWO_D>::NT)
scatter_fwd_kernel(PlaneDims d, const float2* __restrict__ y,
                   const int32_t* __restrict__ posmap, float2* __restrict__ Rh) {
  using F = PlaneFFT<P, TWO_D>;
  extern __shared__ float2 smem[];
  float2* buf = smem;
  float2* tw = smem + F::ELEMS;
  const int u = blockIdx.x;
  make_twiddles<P, F::NT>(tw);
  zero_plane<P, TWO_D>(buf);
  __syncthreads();
  const int32_t* pm = posmap + (size_t)u * d.S;
  for (int s = threadIdx.x; s < d.S; s += F::NT) {
    const int m = pm[s];
    if (m >= 0) buf[F::sidx(s / d.Nx, s % d.Nx)] = y[(size_t)s * d.M + m];
  }
  __syncthreads();
  F::forward(buf, tw, d.Nx);
  store_spectrum<P, TWO_D>(buf, Rh + (size_t)u * d.Nk);
}

// Gh[z] -> x plane z = crop(IFFT2(Gh_z)); optional sum |x|^2 and max |x|.
template <int P, bool TWO_D>
__global__ void __launch_bounds__(PlaneFFT<P, TWO_D>::NT)
inv_store_kernel(PlaneDims d, const float2* __restrict__ Gh, float2* __restrict__ x,
                 double* __restrict__ red_sumsq, unsigned int* __restrict__ maxabs_bits) {
  using F = PlaneFFT<P, TWO_D>;
  extern __shared__ float2 smem[];
  float2* buf = smem;
  float2* tw = smem + F::ELEMS;
  const int z = blockIdx.x;
  make_twiddles<P, F::NT>(tw);
  load_spectrum<P, TWO_D>(buf, Gh + (size_t)z * d.Nk);
  __syncthreads();
  F::inverse(buf, tw, d.Nx);
  double acc = 0.0;
  float mx = 0.f;
  float2* xz = x ? x + (size_t)z * d.Ny * d.Nx : nullptr;
  for (int e = threadIdx.x; e < d.Ny * d.Nx; e += F::NT) {
    const float2 v = buf[F::sidx(e / d.Nx, e % d.Nx)];
    if (xz) xz[e] = v;
    acc += (double)v.x * v.x + (double)v.y * v.y;
    mx = fmaxf(mx, hypotf(v.x, v.y));
  }
  if (red_sumsq) block_add_double<F::NT>(acc, red_sumsq);
  if (maxabs_bits) {
    __syncthreads();
    block_max_bits<F::NT>(mx, maxabs_bits);
  }
}

// Gh[z] (spectrum of A^H(A gamma - y)) -> FISTA step on plane z (Algorithm 1):
//   x_k = tau_{lambda/L}(gamma_k - grad/L), gamma_{k+1} = x_k + beta_k (x_k - x_{k-1})
// then, unless this is the last iteration, Xh[z] = FFT2(pad(gamma_{k+1})).
template <int P, bool TWO_D>
__global__ void __launch_bounds__(PlaneFFT<P, TWO_D>::NT)
inv_fista_fwd_kernel(PlaneDims d, const float2* __restrict__ Gh, float2* __restrict__ xk,
                     float2* __restrict__ gam, const float* __restrict__ scal, float beta,
                     int do_fwd, float2* __restrict__ Xh, double* __restrict__ red_l1) {
  using F = PlaneFFT<P, TWO_D>;
  extern __shared__ float2 smem[];
  float2* buf = smem;
  float2* tw = smem + F::ELEMS;
  const int z = blockIdx.x;
  make_twiddles<P, F::NT>(tw);
  load_spectrum<P, TWO_D>(buf, Gh + (size_t)z * d.Nk);
  __syncthreads();
  F::inverse(buf, tw, d.Nx);
  const float thr = scal[kThr];
  const float invL = scal[kInvL];
  double l1 = 0.0;
  const size_t off = (size_t)z * d.Ny * d.Nx;
  for (int e = threadIdx.x; e < d.Ny * d.Nx; e += F::NT) {
    const int b = F::sidx(e / d.Nx, e % d.Nx);
    const float2 g = buf[b];
    const float2 gm = gam[off + e];
    const float2 xp = xk[off + e];
    const float2 w = make_float2(fmaf(-g.x, invL, gm.x), fmaf(-g.y, invL, gm.y));
    const float mag = hypotf(w.x, w.y);
    const float sc = mag > thr ? 1.0f - thr / mag : 0.0f;
    const float2 xn = make_float2(w.x * sc, w.y * sc);
    const float2 gn = make_float2(fmaf(beta, xn.x - xp.x, xn.x), fmaf(beta, xn.y - xp.y, xn.y));
    xk[off + e] = xn;
    gam[off + e] = gn;
    l1 += (double)(mag > thr ? mag - thr : 0.0f);
    buf[b] = gn;
  }
  if (red_l1) block_add_double<F::NT>(l1, red_l1);
  if (!do_fwd) return;
  zero_outside<P, TWO_D>(buf, d.Ny, d.Nx);
  __syncthreads();
  F::forward(buf, tw, d.Nx);
  store_spectrum<P, TWO_D>(buf, Xh + (size_t)z * d.Nk);
}

// ---------------------------------------------------------------------------
// Depth contractions (the blockwise products of Sec. IV-B restricted to the
// kept bins).  T is tiled by 64 wavenumbers: T[kt][u][z][ki].  A warp lane
// owns the wavenumber pair (2 lane, 2 lane + 1) of the tile, so every table
// load is a coalesced 16-byte vector (512 bytes per warp) and no cross-lane
// reduction is needed: the sums run over z (forward) or u (adjoint) inside
// each lane.  The small spectra (Xh tile or Rh tile) are staged in shared
// memory once per CTA; the table streams from HBM with evict-first loads.
// ---------------------------------------------------------------------------
constexpr int kContractThreads = 256;
constexpr int kContractWarps = kContractThreads / 32;

__device__ __forceinline__ void cmac2(float4& acc, const float4 h, const float4 x) {
  // acc.(x,y) += (h.x + j h.y)(x.x + j x.y); acc.(z,w) likewise
  acc.x = fmaf(h.x, x.x, acc.x); acc.x = fmaf(-h.y, x.y, acc.x);
  acc.y = fmaf(h.x, x.y, acc.y); acc.y = fmaf(h.y, x.x, acc.y);
  acc.z = fmaf(h.z, x.z, acc.z); acc.z = fmaf(-h.w, x.w, acc.z);
  acc.w = fmaf(h.z, x.w, acc.w); acc.w = fmaf(h.w, x.z, acc.w);
}
__device__ __forceinline__ void cmacc2(float4& acc, const float4 h, const float4 r) {
  // acc += conj(h) r for both halves
  acc.x = fmaf(h.x, r.x, acc.x); acc.x = fmaf(h.y, r.y, acc.x);
  acc.y = fmaf(h.x, r.y, acc.y); acc.y = fmaf(-h.y, r.x, acc.y);
  acc.z = fmaf(h.z, r.z, acc.z); acc.z = fmaf(h.w, r.w, acc.z);
  acc.w = fmaf(h.z, r.w, acc.w); acc.w = fmaf(-h.w, r.z, acc.w);
}

// Yh[u][kap] = sum_z T[kt][u][z][ki] Xh[z][kap]
// grid (ceil(U / UC), Nk / 64); each warp owns whole rows u.
template <int UNROLL>
__global__ void __launch_bounds__(kContractThreads)
contract_fwd_kernel(const float4* __restrict__ T, const float4* __restrict__ Xh,
                    float4* __restrict__ Yh, int Nz, int U, int Nk, int UC) {
  extern __shared__ float4 xs[];  // [Nz][32]
  const int kt = blockIdx.y;
  const size_t nk4 = (size_t)Nk / 2;
  for (int i = threadIdx.x; i < Nz * 32; i += kContractThreads)
    xs[i] = Xh[(size_t)(i >> 5) * nk4 + kt * 32 + (i & 31)];
  __syncthreads();
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int u0 = blockIdx.x * UC;
  const int u1 = min(U, u0 + UC);
  for (int u = u0 + warp; u < u1; u += kContractWarps) {
    const float4* row = T + ((size_t)kt * U + u) * Nz * 32 + lane;
    float4 acc = make_float4(0.f, 0.f, 0.f, 0.f);
    int z = 0;
    for (; z + UNROLL <= Nz; z += UNROLL) {
      float4 h[UNROLL];
#pragma unroll
      for (int j = 0; j < UNROLL; ++j) h[j] = __ldcs(row + (size_t)(z + j) * 32);
#pragma unroll
      for (int j = 0; j < UNROLL; ++j) cmac2(acc, h[j], xs[(z + j) * 32 + lane]);
    }
    for (; z < Nz; ++z) cmac2(acc, __ldcs(row + (size_t)z * 32), xs[z * 32 + lane]);
    Yh[(size_t)u * nk4 + kt * 32 + lane] = acc;
  }
}

// Gh[z][kap] = sum_u conj(T[kt][u][z][ki]) Rh[u][kap]
// grid (ceil(Nz / (8 ZW)), Nk / 64); warp w owns depths z0 + w ZW + j.
template <int ZW>
__global__ void __launch_bounds__(kContractThreads)
contract_adj_kernel(const float4* __restrict__ T, const float4* __restrict__ Rh,
                    float4* __restrict__ Gh, int Nz, int U, int Nk) {
  extern __shared__ float4 rs[];  // [U][32]
  const int kt = blockIdx.y;
  const size_t nk4 = (size_t)Nk / 2;
  for (int i = threadIdx.x; i < U * 32; i += kContractThreads)
    rs[i] = Rh[(size_t)(i >> 5) * nk4 + kt * 32 + (i & 31)];
  __syncthreads();
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int z0 = blockIdx.x * (kContractWarps * ZW) + warp * ZW;
  if (z0 >= Nz) return;
  const int nz = min(ZW, Nz - z0);
  float4 acc[ZW];
#pragma unroll
  for (int j = 0; j < ZW; ++j) acc[j] = make_float4(0.f, 0.f, 0.f, 0.f);
  const float4* base = T + ((size_t)kt * U * Nz + z0) * 32 + lane;
  const size_t ustride = (size_t)Nz * 32;
  if (nz == ZW) {
    int u = 0;
    for (; u + 2 <= U; u += 2) {
      float4 h0[ZW], h1[ZW];
#pragma unroll
      for (int j = 0; j < ZW; ++j) h0[j] = __ldcs(base + u * ustride + j * 32);
#pragma unroll
      for (int j = 0; j < ZW; ++j) h1[j] = __ldcs(base + (u + 1) * ustride + j * 32);
      const float4 r0 = rs[u * 32 + lane], r1 = rs[(u + 1) * 32 + lane];
#pragma unroll
      for (int j = 0; j < ZW; ++j) cmacc2(acc[j], h0[j], r0);
#pragma unroll
      for (int j = 0; j < ZW; ++j) cmacc2(acc[j], h1[j], r1);
    }
    for (; u < U; ++u) {
      const float4 r = rs[u * 32 + lane];
#pragma unroll
      for (int j = 0; j < ZW; ++j) cmacc2(acc[j], __ldcs(base + u * ustride + j * 32), r);
    }
  } else {
    for (int u = 0; u < U; ++u) {
      const float4 r = rs[u * 32 + lane];
#pragma unroll
      for (int j = 0; j < ZW; ++j)
        if (j < nz) cmacc2(acc[j], __ldcs(base + u * ustride + j * 32), r);
    }
  }
#pragma unroll
  for (int j = 0; j < ZW; ++j)
    if (j < nz) Gh[(size_t)(z0 + j) * nk4 + kt * 32 + lane] = acc[j];
}

// ---------------------------------------------------------------------------
// Small kernels
// ---------------------------------------------------------------------------
__global__ void set_thresholds_kernel(float* scal, double* red, double lambda, double L,
                                      int use_mu, double mu) {
  double lam = lambda;
  if (use_mu) lam = mu * (double)__uint_as_float(((unsigned int*)scal)[kLamMax]);
  scal[kThr] = (float)(lam / L);
  scal[kInvL] = (float)(1.0 / L);
  red[kNumRed - 1] = lam;
}

__device__ __forceinline__ uint64_t mix64(uint64_t z) {
  z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
  z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
  return z ^ (z >> 31);
}

// complex Gaussian start vector (Box-Muller on hashed counters)
__global__ void randn_kernel(float2* v, int n, uint64_t seed) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  const uint64_t h = mix64(seed + 0x9E3779B97F4A7C15ull * (uint64_t)(i + 1));
  const float u1 = ((float)(h >> 40) + 0.5f) * (1.0f / 16777216.0f);
  const float u2 = (float)((h >> 16) & 0xFFFFFFu) * (1.0f / 16777216.0f);
  const float r = sqrtf(-2.0f * logf(u1));
  float s, c;
  sincospif(2.0f * u2, &s, &c);
  v[i] = make_float2(r * c, r * s);
}

__global__ void sumsq_kernel(const float2* __restrict__ v, int n, double* out) {
  double acc = 0.0;
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) {
    const float2 a = v[i];
    acc += (double)a.x * a.x + (double)a.y * a.y;
  }
  block_add_double<256>(acc, out);
}

__global__ void scale_rnorm_kernel(float2* v, int n, const double* sumsq) {
  const float sc = (float)(1.0 / sqrt(*sumsq));
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) {
    const float2 a = v[i];
    v[i] = make_float2(a.x * sc, a.y * sc);
  }
}

// ---------------------------------------------------------------------------
// Dispatch on the plane size
// ---------------------------------------------------------------------------
// Raise a kernel's dynamic shared memory limit to the device's opt-in maximum
// once per (kernel, device); each launch then asks for what it needs.
int ensure_smem_attr_ptr(const void* kernel, int need) {
  int dev = 0;
  SFS_CUDA(cudaGetDevice(&dev));
  const int optin = max_smem_optin();
  if (need > optin) {
    set_error("kernel needs %d bytes of shared memory, device allows %d", need, optin);
    return SFS_ERR_INVALID_ARG;
  }
  if (need <= 48 * 1024) return SFS_OK;
  static std::mutex mu;
  static std::unordered_map<const void*, uint64_t> done;  // kernel -> device bits
  std::lock_guard<std::mutex> lock(mu);
  uint64_t& bits = done[kernel];
  if (dev < 64 && ((bits >> dev) & 1u)) return SFS_OK;
  SFS_CUDA(cudaFuncSetAttribute(kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, optin));
  if (dev < 64) bits |= (uint64_t)1 << dev;
  return SFS_OK;
}

template <typename K>
int ensure_smem_attr(K kernel, int need) {
  return ensure_smem_attr_ptr((const void*)kernel, need);
}

template <int P, bool TWO_D, typename K, typename... Args>
int launch_plane(K kernel, int nplanes, cudaStream_t st, Args... args) {
  using F = PlaneFFT<P, TWO_D>;
  if (nplanes <= 0) return SFS_OK;
  SFS_TRY(ensure_smem_attr(kernel, F::SMEM));
  kernel<<<nplanes, F::NT, F::SMEM, st>>>(args...);
  SFS_CUDA(cudaGetLastError());
  return SFS_OK;
}

// Calls fn.template operator()<P, TWO_D>() for the plane shape of d.
template <typename Fn>
int dispatch_plane(const PlaneDims& d, Fn&& fn) {
  if (d.Py > 1) {
    switch (d.Px) {
      case 32: return fn.template operator()<32, true>();
      case 64: return fn.template operator()<64, true>();
      case 128: return fn.template operator()<128, true>();
    }
  } else {
    switch (d.Px) {
      case 64: return fn.template operator()<64, false>();
      case 128: return fn.template operator()<128, false>();
      case 256: return fn.template operator()<256, false>();
      case 512: return fn.template operator()<512, false>();
      case 1024: return fn.template operator()<1024, false>();
    }
  }
  set_error("unsupported lateral FFT size %d x %d", d.Px, d.Py);
  return SFS_ERR_INVALID_ARG;
}

}  // namespace

int max_smem_optin() {
  int dev = 0, v = 48 * 1024;
  if (cudaGetDevice(&dev) != cudaSuccess) return v;
  if (cudaDeviceGetAttribute(&v, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev) != cudaSuccess)
    return 48 * 1024;
  return v;
}

int launch_build_table(const PlaneDims& d, const float2* tof, const float* gdir,
                       const float* amp, const int32_t* bins, float2* table,
                       cudaStream_t st) {
  return dispatch_plane(d, [&]<int P, bool TD>() {
    return launch_plane<P, TD>(build_table_kernel<P, TD>, d.U * d.Nz, st, d, tof, gdir,
                               amp, bins, table);
  });
}

int launch_fwd_planes(const PlaneDims& d, const float2* x, float2* Xh, cudaStream_t st) {
  return dispatch_plane(d, [&]<int P, bool TD>() {
    return launch_plane<P, TD>(fwd_planes_kernel<P, TD>, d.Nz, st, d, x, Xh);
  });
}

int launch_inv_gather(const PlaneDims& d, const float2* Yh, const int32_t* posmap,
                      float2* y, double* red_sumsq, cudaStream_t st) {
  return dispatch_plane(d, [&]<int P, bool TD>() {
    return launch_plane<P, TD>(inv_gather_kernel<P, TD>, d.U, st, d, Yh, posmap, y,
                               red_sumsq);
  });
}

int launch_inv_resid_fwd(const PlaneDims& d, const float2* Yh, const int32_t* posmap,
                         const float2* yobs, float2* Rh, double* red_sumsq,
                         cudaStream_t st) {
  return dispatch_plane(d, [&]<int P, bool TD>() {
    return launch_plane<P, TD>(inv_resid_fwd_kernel<P, TD>, d.U, st, d, Yh, posmap, yobs,
                               Rh, red_sumsq);
  });
}

int launch_scatter_fwd(const PlaneDims& d, const float2* y, const int32_t* posmap,
                       float2* Rh, cudaStream_t st) {
  return dispatch_plane(d, [&]<int P, bool TD>() {
    return launch_plane<P, TD>(scatter_fwd_kernel<P, TD>, d.U, st, d, y, posmap, Rh);
  });
}

int launch_inv_store(const PlaneDims& d, const float2* Gh, float2* x, double* red_sumsq,
                     unsigned int* maxabs_bits, cudaStream_t st) {
  return dispatch_plane(d, [&]<int P, bool TD>() {
    return launch_plane<P, TD>(inv_store_kernel<P, TD>, d.Nz, st, d, Gh, x, red_sumsq,
                               maxabs_bits);
  });
}

int launch_inv_fista_fwd(const PlaneDims& d, const float2* Gh, float2* xk, float2* gam,
                         const float* scal, float beta, int do_fwd, float2* Xh,
                         double* red_l1, cudaStream_t st) {
  return dispatch_plane(d, [&]<int P, bool TD>() {
    return launch_plane<P, TD>(inv_fista_fwd_kernel<P, TD>, d.Nz, st, d, Gh, xk, gam, scal,
                               beta, do_fwd, Xh, red_l1);
  });
}

int launch_contract_fwd(const PlaneDims& d, const float2* table, const float2* Xh,
                        float2* Yh, cudaStream_t st) {
  constexpr int UC = 2 * kContractWarps;
  const size_t smem = (size_t)d.Nz * 32 * sizeof(float4);
  SFS_TRY(ensure_smem_attr(contract_fwd_kernel<8>, (int)smem));
  dim3 grid((d.U + UC - 1) / UC, d.Nk / kKappaTile);
  contract_fwd_kernel<8><<<grid, kContractThreads, smem, st>>>(
      (const float4*)table, (const float4*)Xh, (float4*)Yh, d.Nz, d.U, d.Nk, UC);
  SFS_CUDA(cudaGetLastError());
  return SFS_OK;
}

int launch_contract_adj(const PlaneDims& d, const float2* table, const float2* Rh,
                        float2* Gh, cudaStream_t st) {
  constexpr int ZW = 2;
  const size_t smem = (size_t)d.U * 32 * sizeof(float4);
  SFS_TRY(ensure_smem_attr(contract_adj_kernel<ZW>, (int)smem));
  const int zc = kContractWarps * ZW;
  dim3 grid((d.Nz + zc - 1) / zc, d.Nk / kKappaTile);
  contract_adj_kernel<ZW><<<grid, kContractThreads, smem, st>>>(
      (const float4*)table, (const float4*)Rh, (float4*)Gh, d.Nz, d.U, d.Nk);
  SFS_CUDA(cudaGetLastError());
  return SFS_OK;
}

int launch_set_thresholds(float* scal, double* red, double lambda, double L, int use_mu,
                          double mu, cudaStream_t st) {
  set_thresholds_kernel<<<1, 1, 0, st>>>(scal, red, lambda, L, use_mu, mu);
  SFS_CUDA(cudaGetLastError());
  return SFS_OK;
}

int launch_randn(float2* v, int n, uint64_t seed, cudaStream_t st) {
  randn_kernel<<<(n + 255) / 256, 256, 0, st>>>(v, n, seed);
  SFS_CUDA(cudaGetLastError());
  return SFS_OK;
}

int launch_sumsq(const float2* v, int n, double* out, cudaStream_t st) {
  int blocks = (n + 255) / 256;
  if (blocks > 1216) blocks = 1216;
  sumsq_kernel<<<blocks, 256, 0, st>>>(v, n, out);
  SFS_CUDA(cudaGetLastError());
  return SFS_OK;
}

int launch_scale_by_rnorm(float2* v, int n, const double* sumsq, cudaStream_t st) {
  int blocks = (n + 255) / 256;
  if (blocks > 1216) blocks = 1216;
  scale_rnorm_kernel<<<blocks, 256, 0, st>>>(v, n, sumsq);
  SFS_CUDA(cudaGetLastError());
  return SFS_OK;
}

}  // namespace sfs
