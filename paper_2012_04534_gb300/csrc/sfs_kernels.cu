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
#include <cuda_bf16.h>
#include <cuda_fp16.h>
#include <cuda_runtime.h>
#include <stdint.h>
#include <stdlib.h>

#include <algorithm>
#include <mutex>
#include <utility>
#include <unordered_map>

#include "sfs_async.cuh"
#include "sfs_fft.cuh"
#include "sfs_internal.h"
#include "sfs_launch.h"
#include "sfs_planes.cuh"

namespace sfs {
namespace {

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
__global__ void __launch_bounds__(PlaneFFT<P, TWO_D, false>::NT, PlaneFFT<P, TWO_D, false>::MINB)
build_table_kernel(PlaneDims d, const float2* __restrict__ tof,
                   const float* __restrict__ gdir, const float* __restrict__ amp,
                   const int32_t* __restrict__ bins, float2* __restrict__ table) {
  using F = PlaneFFT<P, TWO_D, false>;  // generator planes fill (2 Ny - 1) x (2 Nx - 1)
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
  // FFT2 of the generator is constant on each symmetry orbit of wavenumbers
  // (h depends on dx^2 + dy^2 only); store it once per orbit, at the orbit's
  // representative.  Orbit o lives in slot tile o / E, entry o % E.
  // Depths 2p and 2p + 1 share one 16-byte word (re_2p, re_2p+1, im_2p,
  // im_2p+1): T4[st][u][p][e] with e < E = 64 / GS.
  // The tensor-core contractions use words ((o nzc + z/16) U + u) 8 + ((z%16)/2
  // xor u%8), one orbit's rows per 16-depth block (sfs_tc.cu).
  // The 16-bit tensor-core contractions (sfs_tc16.cu) use rows of 64 values
  // T16[part][o][z/32][u][2 (z%32) + {0: re, 1: im}]: part 0 holds the BF16
  // rounding of the FP32 value v, part 1 (two-part tables) the BF16 rounding
  // of v - part 0.  FP16 tables round v 2^kT (d.tscale) the same way.
  if (d.tc == 2) {
    const int No = d.Ns / d.GS;
    for (int o = threadIdx.x; o < No; o += F::NT) {
      const int rep = d.orbit_rep[o];
      float2 v = rep >= 0 ? buf[F::kidx(rep)] : make_float2(0.f, 0.f);
      const size_t row = ((size_t)o * d.nkb + (z >> 5)) * d.U + u;
      const size_t row1 = (((size_t)No + o) * d.nkb + (z >> 5)) * d.U + u;
      if (d.f16) {
        v = make_float2(v.x * d.tscale, v.y * d.tscale);
        __half2* t16 = (__half2*)table;
        const __half2 hi = __floats2half2_rn(v.x, v.y);
        t16[row * 32 + (z & 31)] = hi;
        if (d.nparts == 2)
          t16[row1 * 32 + (z & 31)] = __floats2half2_rn(v.x - __low2float(hi), v.y - __high2float(hi));
      } else {
        __nv_bfloat162* t16 = (__nv_bfloat162*)table;
        const __nv_bfloat162 hi = __floats2bfloat162_rn(v.x, v.y);
        t16[row * 32 + (z & 31)] = hi;
        if (d.nparts == 2)
          t16[row1 * 32 + (z & 31)] =
              __floats2bfloat162_rn(v.x - __low2float(hi), v.y - __high2float(hi));
      }
    }
    return;
  }
  const int E = kKappaTile / d.GS;
  const int Nzp = (d.Nz + 1) / 2;
  float* tf = (float*)table;
  for (int o = threadIdx.x; o < d.Ns / d.GS; o += F::NT) {
    const int rep = d.orbit_rep[o];
    const float2 v = rep >= 0 ? buf[F::kidx(rep)] : make_float2(0.f, 0.f);
    const size_t w4 = d.tc ? (((size_t)o * d.nzc + (z >> 4)) * d.U + u) * 8 + (((z & 15) >> 1) ^ (u & 7))
                           : (((size_t)(o / E) * d.Up + u) * Nzp + z / 2) * E + (o % E);
    tf[4 * w4 + (z & 1)] = v.x;
    tf[4 * w4 + 2 + (z & 1)] = v.y;
  }
}

// ---------------------------------------------------------------------------
// Plane kernels (one lateral plane per CTA; their steps are in sfs_planes.cuh)
// ---------------------------------------------------------------------------
// x plane z -> Xh[z] = FFT2(pad(x_z))
template <int P, bool TWO_D>
__global__ void __launch_bounds__(PlaneFFT<P, TWO_D>::NT, PlaneFFT<P, TWO_D>::MINB)
fwd_planes_kernel(PlaneDims d, const float2* __restrict__ x, float2* __restrict__ Xh) {
  using F = PlaneFFT<P, TWO_D>;
  {  // scene blockIdx.y of a batched launch
    const long long b = blockIdx.y;
    x += b * d.bs_x;
    Xh += b * d.bs_xh;
  }
  extern __shared__ float2 smem[];
  float2* buf = smem;
  float2* tw = smem + F::ELEMS;
  const int z = blockIdx.x;
  plane_twiddles<P, TWO_D>(tw);
  pdl_wait();
  pdl_trigger();
  zero_plane<P, TWO_D>(buf);
  __syncthreads();
  const float2* xz = x + (size_t)z * d.Ny * d.Nx;
  for (int e = threadIdx.x; e < d.Ny * d.Nx; e += F::NT)
    buf[F::sidx(e / d.Nx, e % d.Nx)] = xz[e];
  __syncthreads();
  forward_store<P, TWO_D>(buf, tw, Xh + (size_t)z * d.Ns, d,
                          d.pm_x ? d.pm_x + blockIdx.y * d.bs_pmx + z : nullptr);
}

// Yh[u] -> y[s, m] = IFFT2(Yh_u)(s) where bins[u] = idx[s, m]
template <int P, bool TWO_D>
__global__ void __launch_bounds__(PlaneFFT<P, TWO_D>::NT, PlaneFFT<P, TWO_D>::MINB)
inv_gather_kernel(PlaneDims d, const float2* __restrict__ Yh,
                  const int32_t* __restrict__ posmap, float2* __restrict__ y,
                  double* __restrict__ red_sumsq) {
  using F = PlaneFFT<P, TWO_D>;
  {  // scene blockIdx.y of a batched launch
    const long long b = blockIdx.y;
    Yh += b * d.bs_yh;
    y += b * d.bs_y;
    if (red_sumsq) red_sumsq += b * d.bs_red;
  }
  extern __shared__ float2 smem[];
  float2* buf = smem;
  float2* tw = smem + F::ELEMS;
  const int u = blockIdx.x;
  plane_twiddles<P, TWO_D>(tw);
  pdl_wait();
  pdl_trigger();
  load_inverse_fwd<P, TWO_D>(buf, tw, Yh, u, d);
  double acc = 0.0;
  const int32_t* pm = posmap + (size_t)u * d.S;
  for (int s = threadIdx.x; s < d.S; s += F::NT) {
    const int m = pm[s];
    if (m >= 0) {
      const float2 v = buf[F::sidx(s / d.Nx, s % d.Nx)];
      y[(size_t)s * d.M + m] = v;
      // FP64 sums only when asked for: the FP64 pipe runs at a small
      // fraction of the FP32 rate, and the iteration loop asks for none
      if (red_sumsq) acc += (double)v.x * v.x + (double)v.y * v.y;
    }
  }
  if (red_sumsq) block_add_double<F::NT>(acc, red_sumsq);
}

// Yh[u] -> residual r = (A gamma - y) on bin plane u -> Rh[u] = FFT2(pad(r_u)).
// yplane[u][s] holds the measurements laid out by bin plane (scatter_y_planes),
// so they load alongside the selection mask instead of after it.
template <int P, bool TWO_D>
__global__ void __launch_bounds__(PlaneFFT<P, TWO_D>::NT, PlaneFFT<P, TWO_D>::MINB)
inv_resid_fwd_kernel(PlaneDims d, const float2* __restrict__ Yh,
                     const int32_t* __restrict__ posmap, const float2* __restrict__ yplane,
                     float2* __restrict__ Rh, double* __restrict__ red_sumsq) {
  extern __shared__ float2 smem[];
  resid_plane_step<P, TWO_D>(d, (int)blockIdx.x, blockIdx.y, smem, Yh, posmap, yplane, Rh, red_sumsq);
}

// y[s, m] scattered to bin plane u -> Rh[u] = FFT2(pad(.))
template <int P, bool TWO_D>
__global__ void __launch_bounds__(PlaneFFT<P, TWO_D>::NT, PlaneFFT<P, TWO_D>::MINB)
scatter_fwd_kernel(PlaneDims d, const float2* __restrict__ y,
                   const int32_t* __restrict__ posmap, float2* __restrict__ Rh) {
  using F = PlaneFFT<P, TWO_D>;
  {  // scene blockIdx.y of a batched launch
    const long long b = blockIdx.y;
    y += b * d.bs_y;
    Rh += b * d.bs_rh;
  }
  extern __shared__ float2 smem[];
  float2* buf = smem;
  float2* tw = smem + F::ELEMS;
  const int u = blockIdx.x;
  plane_twiddles<P, TWO_D>(tw);
  pdl_wait();
  pdl_trigger();
  zero_plane<P, TWO_D>(buf);
  __syncthreads();
  const int32_t* pm = posmap + (size_t)u * d.S;
  for (int s = threadIdx.x; s < d.S; s += F::NT) {
    const int m = pm[s];
    if (m >= 0) buf[F::sidx(s / d.Nx, s % d.Nx)] = y[(size_t)s * d.M + m];
  }
  __syncthreads();
  forward_store<P, TWO_D>(buf, tw, Rh + (size_t)u * d.Ns, d,
                          d.pm_r ? d.pm_r + blockIdx.y * d.bs_pmr + u : nullptr);
}

// Gh[z] -> x plane z = crop(IFFT2(Gh_z)); optional sum |x|^2 and max |x|.
template <int P, bool TWO_D>
__global__ void __launch_bounds__(PlaneFFT<P, TWO_D>::NT, PlaneFFT<P, TWO_D>::MINB)
inv_store_kernel(PlaneDims d, const float2* __restrict__ Gh, const int2* __restrict__ segslot,
                 float2* __restrict__ x, double* __restrict__ red_sumsq,
                 unsigned int* __restrict__ maxabs_bits) {
  using F = PlaneFFT<P, TWO_D>;
  {  // scene blockIdx.y of a batched launch
    const long long b = blockIdx.y;
    Gh += b * d.bs_gh;
    if (x) x += b * d.bs_x;
    if (red_sumsq) red_sumsq += b * d.bs_red;
    if (maxabs_bits) maxabs_bits += b * d.bs_scal;
  }
  extern __shared__ float2 smem[];
  float2* buf = smem;
  float2* tw = smem + F::ELEMS;
  const int z = blockIdx.x;
  plane_twiddles<P, TWO_D>(tw);
  pdl_wait();
  pdl_trigger();
  load_inverse_adj<P, TWO_D>(buf, tw, Gh, segslot, z, d);
  double acc = 0.0;
  float mx = 0.f;
  float2* xz = x ? x + (size_t)z * d.Ny * d.Nx : nullptr;
  for (int e = threadIdx.x; e < d.Ny * d.Nx; e += F::NT) {
    const float2 v = buf[F::sidx(e / d.Nx, e % d.Nx)];
    if (xz) xz[e] = v;
    if (red_sumsq) acc += (double)v.x * v.x + (double)v.y * v.y;
    if (maxabs_bits) mx = nanmax(mx, hypotf(v.x, v.y));
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
// beta_k is *beta_dev when given (a table written on the device by
// fista_betas_kernel), else beta_arg.
template <int P, bool TWO_D>
__global__ void __launch_bounds__(PlaneFFT<P, TWO_D>::NT, PlaneFFT<P, TWO_D>::MINB)
inv_fista_fwd_kernel(PlaneDims d, const float2* __restrict__ Gh,
                     const int2* __restrict__ segslot, float2* __restrict__ xk,
                     float2* __restrict__ gam, const float* __restrict__ scal, float beta_arg,
                     const float* __restrict__ beta_dev, int do_fwd, float2* __restrict__ Xh,
                     double* __restrict__ red_l1) {
  extern __shared__ float2 smem[];
  update_plane_step<P, TWO_D>(d, (int)blockIdx.x, blockIdx.y, smem, Gh, segslot, xk, gam, scal, beta_arg,
                              beta_dev, do_fwd, Xh, red_l1);
}

// ---------------------------------------------------------------------------
// Cluster plane kernels (QUAD planes, P = 128): one cluster of four CTAs per
// plane instead of one CTA.  CTA rank q = 2 py + px of the cluster owns
// quadrant q of the spectrum and rows 16 q .. 16 q + 15 of the 64 x 64
// spatial plane:
//   1. inverse of quadrant q, twiddled: CTA q's share of the cropped inverse
//      (PlaneFFT::inverse_quad), left in its own plane buffer;
//   2. cluster barrier; each CTA adds the four shares of its 16 rows, reading
//      the other CTAs' buffers through distributed shared memory, and applies
//      the row-local step (residual, or FISTA update);
//   3. cluster barrier; each CTA reads the 64 rows of the new spatial plane
//      from the four CTAs' row buffers and runs the forward transform of its
//      own quadrant (PlaneFFT::forward_quad), then stores its slots.
// The forward transform is the one-CTA engine's arithmetic bit for bit (a
// FISTA call resumed from its state, whose first spectra come from
// fwd_planes_kernel, continues an uninterrupted call exactly).  The inverse
// adds the four twiddled quadrant shares in the order 0 + 1 + 2 + 3, where
// the one-CTA engine adds the two quadrants of each py before its pass along
// ky': the two agree to FP32 rounding.  A CTA leaves only after the
// last cluster barrier, so no CTA reads the shared memory of one that has
// exited.  Every CTA of a cluster passes the same barriers (the branches
// around them depend on kernel arguments only).
// ---------------------------------------------------------------------------
constexpr int kQuadCl = 4;                 // CTAs per plane (one per quadrant)
constexpr int kQuadRows = 64 / kQuadCl;    // spatial rows per CTA

__device__ __forceinline__ void cluster_arrive() {
  asm volatile("barrier.cluster.arrive.release.aligned;" ::: "memory");
}
__device__ __forceinline__ void cluster_wait() {
  asm volatile("barrier.cluster.wait.acquire.aligned;" ::: "memory");
}
__device__ __forceinline__ int cluster_rank() {
  unsigned r;
  asm volatile("mov.u32 %0, %%cluster_ctarank;" : "=r"(r));
  return (int)r;
}
// generic address of the same shared-memory location in CTA `rank` of the cluster
template <typename T>
__device__ __forceinline__ T* cluster_map(T* p, int rank) {
  uint64_t out;
  asm volatile("mapa.u64 %0, %1, %2;" : "=l"(out) : "l"((uint64_t)p), "r"(rank));
  return reinterpret_cast<T*>(out);
}

// Shared memory of a cluster plane CTA: plane buffer, twiddles, the 16 x 64
// row buffer, and the per-CTA maxima of the FP16 modes.
template <int P, bool TWO_D>
__host__ __device__ constexpr int quad_cl_smem() {
  return (PlaneFFT<P, TWO_D>::ELEMS + PlaneFFT<P, TWO_D>::NTW + kQuadRows * 64) * 8 + 8 * 4;
}

// After step 1: the four shares of row y, column x, added in quadrant order.
template <int LD>
__device__ __forceinline__ float2 sum_shares(float2* const sh[kQuadCl], int y, int x) {
  const int o = y * LD + x;
  float2 g = sh[0][o];
#pragma unroll
  for (int r = 1; r < kQuadCl; ++r) g = cadd(g, sh[r][o]);
  return g;
}

// Step 3 of the cluster kernels: the spatial column of this thread from the
// row buffers of the cluster, the forward transform of quadrant q and the
// store of its slots (rank 0 also zeroes the padding slots); with pm, the
// plane's largest |Re| or |Im| at *pm.
template <int P, bool TWO_D>
__device__ __forceinline__ void quad_cl_forward_store(float2* buf, const float2* tw, float2* xg, float* mxs,
                                                      int q, float2* __restrict__ dst, const PlaneDims& d,
                                                      float* pm) {
  using F = PlaneFFT<P, TWO_D>;
  const int lane = threadIdx.x & 31, l = lane >> 2;
  const int c = (threadIdx.x >> 5) * 4 + (lane & 3);
  float2 s[8];
#pragma unroll
  for (int j = 0; j < 8; ++j) {
    const int y = l + 8 * j;
    s[j] = cluster_map(xg, y / kQuadRows)[(y % kQuadRows) * 64 + c];
  }
  cluster_arrive();  // this CTA's reads of the row buffers are done
  F::forward_quad(buf, tw, q, s);
  float mx = 0.0f;
  store_quadrant<P, TWO_D>(buf, dst, d, q, mx);
  if (q == 0) store_quadrant<P, TWO_D>(buf, dst, d, 4, mx);
  cluster_wait();
  if (pm) {  // the cluster's maximum, gathered in rank 0's shared memory
    block_max_store<F::NT>(mx, mxs + 4);
    if (threadIdx.x == 0) *cluster_map(mxs + q, 0) = mxs[4];
    cluster_arrive();
    cluster_wait();
    if (q == 0 && threadIdx.x == 0) *pm = fmaxf(fmaxf(mxs[0], mxs[1]), fmaxf(mxs[2], mxs[3]));
  }
}

// inv_resid_fwd_kernel on a cluster of four CTAs per bin plane.
template <int P, bool TWO_D>
__global__ void __launch_bounds__(PlaneFFT<P, TWO_D>::NT, 2)
inv_resid_fwd_cl_kernel(PlaneDims d, const float2* __restrict__ Yh, const int32_t* __restrict__ posmap,
                        const float2* __restrict__ yplane, float2* __restrict__ Rh,
                        double* __restrict__ red_sumsq) {
  using F = PlaneFFT<P, TWO_D>;
  static_assert(F::QUAD, "cluster plane kernels run quadrant planes");
  {  // scene blockIdx.y of a batched launch
    const long long b = blockIdx.y;
    Yh += b * d.bs_yh;
    yplane += b * d.bs_yplane;
    Rh += b * d.bs_rh;
    if (red_sumsq) red_sumsq += b * d.bs_red;
  }
  extern __shared__ float2 smem[];
  float2* buf = smem;
  float2* tw = smem + F::ELEMS;
  float2* xg = tw + F::NTW;
  float* mxs = reinterpret_cast<float*>(xg + kQuadRows * 64);
  const int q = cluster_rank();
  const int u = blockIdx.x / kQuadCl;
  const int lane = threadIdx.x & 31, l = lane >> 2;
  const int c = (threadIdx.x >> 5) * 4 + (lane & 3);
  plane_twiddles<P, TWO_D>(tw);
  pdl_wait();
  pdl_trigger();
  float2 acc[8];
  F::inverse_quad(buf, tw, q, acc, [&](int qq) { load_quadrant_fwd<P, TWO_D>(buf, Yh, u, d, qq); });
#pragma unroll
  for (int k = 0; k < 8; ++k) buf[(l + 8 * k) * F::LD + c] = acc[k];
  cluster_arrive();
  cluster_wait();  // every share is in its CTA's buffer
  float2* sh[kQuadCl];
#pragma unroll
  for (int r = 0; r < kQuadCl; ++r) sh[r] = cluster_map(buf, r);
  const int32_t* pmap = posmap + (size_t)u * d.S;
  const float2* yu = yplane + (size_t)u * d.S;
  double accs = 0.0;
#pragma unroll
  for (int i = 0; i < kQuadRows * 64 / F::NT; ++i) {
    const int e = threadIdx.x + i * F::NT;
    const int y = q * kQuadRows + (e >> 6), x = e & 63;
    const float2 g = sum_shares<F::LD>(sh, y, x);
    float2 r = make_float2(0.f, 0.f);
    if (y < d.Ny && x < d.Nx) {
      const int s = y * d.Nx + x;
      const int m = pmap[s];
      if (m >= 0) {
        r = csub(g, yu[s]);
        if (red_sumsq) accs += (double)r.x * r.x + (double)r.y * r.y;
      }
    }
    xg[e] = r;
  }
  if (red_sumsq) block_add_double<F::NT>(accs, red_sumsq);
  cluster_arrive();
  cluster_wait();  // the row buffers are complete; the shares have been read
  quad_cl_forward_store<P, TWO_D>(buf, tw, xg, mxs, q, Rh + (size_t)u * d.Ns, d,
                                  d.pm_r ? d.pm_r + blockIdx.y * d.bs_pmr + u : nullptr);
}

// inv_fista_fwd_kernel on a cluster of four CTAs per depth plane.
template <int P, bool TWO_D>
__global__ void __launch_bounds__(PlaneFFT<P, TWO_D>::NT, 2)
inv_fista_fwd_cl_kernel(PlaneDims d, const float2* __restrict__ Gh, const int2* __restrict__ segslot,
                        float2* __restrict__ xk, float2* __restrict__ gam, const float* __restrict__ scal,
                        float beta_arg, const float* __restrict__ beta_dev, int do_fwd,
                        float2* __restrict__ Xh, double* __restrict__ red_l1) {
  using F = PlaneFFT<P, TWO_D>;
  static_assert(F::QUAD, "cluster plane kernels run quadrant planes");
  {  // scene blockIdx.y of a batched launch
    const long long b = blockIdx.y;
    Gh += b * d.bs_gh;
    xk += b * d.bs_x;
    gam += b * d.bs_x;
    scal += b * d.bs_scal;
    Xh += b * d.bs_xh;
    if (red_l1) red_l1 += b * d.bs_red;
  }
  extern __shared__ float2 smem[];
  float2* buf = smem;
  float2* tw = smem + F::ELEMS;
  float2* xg = tw + F::NTW;
  float* mxs = reinterpret_cast<float*>(xg + kQuadRows * 64);
  const int q = cluster_rank();
  const int z = blockIdx.x / kQuadCl;
  const int lane = threadIdx.x & 31, l = lane >> 2;
  const int c = (threadIdx.x >> 5) * 4 + (lane & 3);
  plane_twiddles<P, TWO_D>(tw);
  pdl_wait();
  pdl_trigger();
  float2 acc[8];
  F::inverse_quad(buf, tw, q, acc,
                  [&](int qq) { load_quadrant_adj<P, TWO_D>(buf, Gh, segslot, z, d, qq); });
#pragma unroll
  for (int k = 0; k < 8; ++k) buf[(l + 8 * k) * F::LD + c] = acc[k];
  cluster_arrive();
  cluster_wait();  // every share is in its CTA's buffer
  float2* sh[kQuadCl];
#pragma unroll
  for (int r = 0; r < kQuadCl; ++r) sh[r] = cluster_map(buf, r);
  const float thr = scal[kThr];
  const float invL = scal[kInvL];
  const float beta = beta_dev ? *beta_dev : beta_arg;
  const size_t off = (size_t)z * d.Ny * d.Nx;
  double l1 = 0.0;
#pragma unroll
  for (int i = 0; i < kQuadRows * 64 / F::NT; ++i) {
    const int e = threadIdx.x + i * F::NT;
    const int y = q * kQuadRows + (e >> 6), x = e & 63;
    const float2 g = sum_shares<F::LD>(sh, y, x);
    float2 gn = make_float2(0.f, 0.f);
    if (y < d.Ny && x < d.Nx) {
      const size_t v = off + (size_t)y * d.Nx + x;
      const float2 gm = gam[v];
      const float2 xp = xk[v];
      const float2 w = make_float2(fmaf(-g.x, invL, gm.x), fmaf(-g.y, invL, gm.y));
      const float mag = hypotf(w.x, w.y);
      const float sc = mag > thr ? 1.0f - thr / mag : 0.0f;
      const float2 xn = make_float2(w.x * sc, w.y * sc);
      gn = make_float2(fmaf(beta, xn.x - xp.x, xn.x), fmaf(beta, xn.y - xp.y, xn.y));
      xk[v] = xn;
      gam[v] = gn;
      if (red_l1) l1 += (double)(mag > thr ? mag - thr : 0.0f);
    }
    xg[e] = gn;
  }
  if (red_l1) block_add_double<F::NT>(l1, red_l1);
  cluster_arrive();
  cluster_wait();  // the row buffers are complete; the shares have been read
  if (!do_fwd) return;  // kernel argument: the whole cluster leaves here
  quad_cl_forward_store<P, TWO_D>(buf, tw, xg, mxs, q, Xh + (size_t)z * d.Ns, d,
                                  d.pm_x ? d.pm_x + blockIdx.y * d.bs_pmx + z : nullptr);
}

// ---------------------------------------------------------------------------
// Depth contractions (the blockwise products of Sec. IV-B restricted to the
// kept bins).
//
// Folded table.  The lateral kernel h_{k,z}[dy, dx] depends on dx^2 + dy^2
// only, so its FFT2 is the same for every wavenumber of a symmetry orbit
// (sign flips of kx and ky, and kx <-> ky on a square grid).  Spectra are
// kept in slot order, GS slots per orbit (2 line, 4 area, 8 square area,
// padding slots carry zero), and the table stores one entry per orbit.
//
// Depth pairs.  Entries of depths 2p and 2p + 1 are interleaved as one
// 16-byte word (re_2p, re_2p+1, im_2p, im_2p+1): T4[st][u][p][e], e < E =
// 64 / GS, for slot tile st of 64 slots, bin u and depth pair p < Nzp =
// ceil(Nz / 2) (a missing odd depth is zero).  One 16-byte shared-memory
// load serves two depths.  In the adjoints its halves are packed pairs that
// multiply duplicated residual spectra in the packed FP32 FMA (FFMA2, two
// FMAs per instruction), with even- and odd-depth sums kept apart; the
// forward uses scalar FMAs.  Lane l owns the slot pair (2l, 2l + 1), both in
// orbit entry l / (GS / 2).
//
// Waits on the mbarriers are bounded (wait_ns of global time, 2 s unless the
// operator sets another limit); a timeout sets *err, drains the copies
// already issued (again bounded, by a fixed 0.5 s) and ends the warp or CTA.
// With `inject` set (failure-handling tests), the first wait is made on a
// barrier that nothing ever arrives at, so that path runs for real.
// ---------------------------------------------------------------------------
constexpr int kContractWarps = 8;
constexpr int kContractThreads = kContractWarps * 32;
constexpr int kRowsPerWarp = 16;                         // depths (8 pairs)
constexpr int kPairsPerWarp = kRowsPerWarp / 2;
constexpr int kZBlock = kContractWarps * kRowsPerWarp;  // 128 depths
constexpr int kZPairs = kZBlock / 2;                     // 64 pairs
constexpr int kSlots = 3;

// Packed pairs of floats (one 64-bit register pair) and the packed FP32
// arithmetic of sm_100 and later (one FFMA2 does two FMAs).
typedef float2 f2x;
__device__ __forceinline__ f2x pk(float lo, float hi) { return make_float2(lo, hi); }
__device__ __forceinline__ f2x ffma2(f2x a, f2x b, f2x c) { return __ffma2_rn(a, b, c); }
__device__ __forceinline__ f2x fneg2(f2x a) { return make_float2(-a.x, -a.y); }

// Position in the unit sequence (segment-major, bin group fastest), advanced
// without divisions.
struct UnitPos {
  int seg, ug, st, zb;
  __device__ __forceinline__ void init(int unit, int NUG, int nzb) {
    seg = unit / NUG;
    ug = unit - seg * NUG;
    st = seg / nzb;
    zb = seg - st * nzb;
  }
  __device__ __forceinline__ void next(int NUG, int nzb) {
    if (++ug == NUG) {
      ug = 0;
      ++seg;
      if (++zb == nzb) {
        zb = 0;
        ++st;
      }
    }
  }
};

// A lane's spectra of its slot pair at two depths as packed pairs:
// xr = (x_2p.re, x_2p+1.re), xi likewise, for slots a (2 lane) and b.
struct PairX {
  f2x ra, ia, rb, ib;
};
__device__ __forceinline__ PairX load_pair_x(const float4* __restrict__ Xh, size_t ns4, int st,
                                             int lane, int z, int Nz) {
  const float4 lo = z < Nz ? Xh[(size_t)z * ns4 + st * 32 + lane] : make_float4(0.f, 0.f, 0.f, 0.f);
  const float4 hi =
      z + 1 < Nz ? Xh[(size_t)(z + 1) * ns4 + st * 32 + lane] : make_float4(0.f, 0.f, 0.f, 0.f);
  return PairX{pk(lo.x, hi.x), pk(lo.y, hi.y), pk(lo.z, hi.z), pk(lo.w, hi.w)};
}

// Accumulators of a lane's slot pair as packed pairs (adjoint): even depth
// in .x, odd depth in .y.
struct PairAcc {
  f2x ra, ia, rb, ib;
};

// acc += h x for the two slots of a lane at one depth pair (forward), both
// depths summed into one value: a = (re_a, im_a, re_b, im_b), h4 = (re_2p,
// re_2p+1, im_2p, im_2p+1) one table word; real hr xr - hi xi, imag hr xi +
// hi xr.  Scalar FMAs: with the spectra of 8 depth pairs held in registers
// the packed form needs more registers than the 2-CTA budget leaves and
// measured slower.  A packed form that keeps only one bin's sums live (bin
// by bin, FFMA2 over the two depths of a pair, real part as sum hr xr - sum
// hi xi, 122-125 registers, no spills) was slower too: vol64 forward 210.8
// against 160.6 us, vol32 22.5 against 18.4 us.
__device__ __forceinline__ void fwd_mac(float4& a, const float4 h4, const PairX& x) {
  a.x = fmaf(h4.x, x.ra.x, a.x); a.x = fmaf(-h4.z, x.ia.x, a.x);
  a.x = fmaf(h4.y, x.ra.y, a.x); a.x = fmaf(-h4.w, x.ia.y, a.x);
  a.y = fmaf(h4.x, x.ia.x, a.y); a.y = fmaf(h4.z, x.ra.x, a.y);
  a.y = fmaf(h4.y, x.ia.y, a.y); a.y = fmaf(h4.w, x.ra.y, a.y);
  a.z = fmaf(h4.x, x.rb.x, a.z); a.z = fmaf(-h4.z, x.ib.x, a.z);
  a.z = fmaf(h4.y, x.rb.y, a.z); a.z = fmaf(-h4.w, x.ib.y, a.z);
  a.w = fmaf(h4.x, x.ib.x, a.w); a.w = fmaf(h4.z, x.rb.x, a.w);
  a.w = fmaf(h4.y, x.ib.y, a.w); a.w = fmaf(h4.w, x.rb.y, a.w);
}
__device__ __forceinline__ void zero_acc(float4& a) { a = make_float4(0.f, 0.f, 0.f, 0.f); }

// Residual spectra of a lane's slot pair for one bin, duplicated into packed
// pairs for the adjoint: rr = (r.re, r.re), ri = (r.im, r.im) for slots a, b.
struct DupR {
  f2x rra, ria, rrb, rib;
};
__device__ __forceinline__ DupR dup_r(const float4 r) {
  return DupR{pk(r.x, r.x), pk(r.y, r.y), pk(r.z, r.z), pk(r.w, r.w)};
}
// acc += conj(h) r at one depth pair (adjoint): real hr rr + hi ri, imag hr ri - hi rr.
__device__ __forceinline__ void adj_mac(PairAcc& a, const float4 h4, const DupR& r) {
  const f2x hr = pk(h4.x, h4.y), hi = pk(h4.z, h4.w);
  const f2x nhi = fneg2(hi);
  a.ra = ffma2(hr, r.rra, a.ra);
  a.ra = ffma2(hi, r.ria, a.ra);
  a.ia = ffma2(hr, r.ria, a.ia);
  a.ia = ffma2(nhi, r.rra, a.ia);
  a.rb = ffma2(hr, r.rrb, a.rb);
  a.rb = ffma2(hi, r.rib, a.rb);
  a.ib = ffma2(hr, r.rib, a.ib);
  a.ib = ffma2(nhi, r.rrb, a.ib);
}
__device__ __forceinline__ void zero_acc(PairAcc& a) {
  a.ra = a.ia = a.rb = a.ib = make_float2(0.f, 0.f);
}


// Forward contraction.  Up = bins padded to a multiple of UP = GS / 2
// (padding table rows are zero); nunits = (Ns / 64) * nzb * (Up / UP).
// Work is cut into units (st, zb, bin group): UP bins of slot tile st over
// the 128-depth block zb; a persistent CTA (two per SM) takes a contiguous,
// equal share.  The 8 warps meet at one CTA barrier after every unit to add
// their depth partials, so the ring is CTA-wide: stage s holds one unit (UP
// bins x 64 depth pairs x E entries, 32 KB), refilled by one thread right
// after the barrier that frees it, one bulk copy per bin (a bin's pairs of a
// depth block are contiguous) and one mbarrier per stage.  Warp w consumes
// pairs 8 w .. 8 w + 7 and keeps their spectra in registers.  The partials
// alternate between two buffers, so that unit i + 1's partials never
// overwrite unit i's before they are added: one barrier per unit instead of
// two (the second buffer takes the shared memory of a third ring stage;
// measured on vol64, 169.9 -> 160.5 us per launch).
constexpr int kFwdStages = 2;
template <int GS>
__global__ void __launch_bounds__(kContractThreads, kContractCtasPerSm)
contract_fwd_stream(const float4* __restrict__ T4, const float4* __restrict__ Xh,
                    float4* __restrict__ Yp, int Nz, int Up, int Ns, int nzb, int nunits,
                    int* __restrict__ err, uint64_t wait_ns, int inject, int stream_table) {
  constexpr int E = kKappaTile / GS;
  constexpr int UP = GS / 2;
  constexpr int STAGE = UP * kZPairs * E;  // float4 per stage (32 KB)
  extern __shared__ __align__(128) float4 sm4[];
  float4* red0 = sm4;                                     // [2][8][UP][32]
  float4* ring = red0 + 2 * kContractWarps * UP * 32;     // [2][STAGE]
  uint64_t* bars = (uint64_t*)(ring + kFwdStages * STAGE);  // [kFwdStages] + never
  __shared__ int abort_flag;
  const int w = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int NUG = Up / UP;
  const int Nzp = (Nz + 1) / 2;
  const int G = gridDim.x, b = blockIdx.x;
  const int first = (int)(((long long)nunits * b) / G);
  const int n = (int)(((long long)nunits * (b + 1)) / G) - first;
  const uint32_t bar0 = smem_addr(bars);
  const uint32_t never = bar0 + 8u * kFwdStages;  // nothing arrives here
  const int ent = lane / (GS / 2);  // this lane's orbit entry in a row
  if (threadIdx.x == 0) {
    abort_flag = 0;
    for (int k = 0; k <= kFwdStages; ++k) mbar_init(bar0 + 8u * k, 1);
    fence_mbar_init();
  }
  __syncthreads();
  UnitPos ip;
  ip.init(first, NUG, nzb);
  auto issue = [&](int i) {
    const int pairs = min(kZPairs, Nzp - ip.zb * kZPairs);
    const uint32_t bytes = (uint32_t)pairs * (E * 16u);
    const uint32_t bar = bar0 + 8u * (i % kFwdStages);
    float4* stage = ring + (i % kFwdStages) * STAGE;
    const float4* src = T4 + ((size_t)(ip.st * Up + ip.ug * UP) * Nzp + ip.zb * kZPairs) * E;
    fence_proxy_async();
    mbar_expect_tx(bar, bytes * UP);
    const uint64_t pol = stream_table ? l2_evict_first_policy() : 0ull;
#pragma unroll
    for (int q = 0; q < UP; ++q)
      bulk_g2s_table(smem_addr(stage + q * kZPairs * E), src + (size_t)q * Nzp * E, bytes, bar,
                     stream_table != 0, pol);
    ip.next(NUG, nzb);
  };
  if (threadIdx.x == 0)
    for (int i = 0; i < kFwdStages && i < n; ++i) issue(i);
  pdl_wait();  // Xh comes from the predecessor; the table copies above do not
  pdl_trigger();
  const size_t ns4 = (size_t)Ns / 2;
  UnitPos cp;  // unit being computed
  cp.init(first, NUG, nzb);
  PairX xr[kPairsPerWarp];
  int cur_seg = -1, npw = 0;
  bool ok = true;
  int waited = 0;
  for (int i = 0; i < n; ++i, cp.next(NUG, nzb)) {
    if (cp.seg != cur_seg) {  // new (st, zb): this warp's spectra into registers
      cur_seg = cp.seg;
      const int p0 = cp.zb * kZPairs + w * kPairsPerWarp;
      npw = min(kPairsPerWarp, max(0, Nzp - p0));
#pragma unroll
      for (int p = 0; p < kPairsPerWarp; ++p) xr[p] = load_pair_x(Xh, ns4, cp.st, lane, 2 * (p0 + p), Nz);
    }
    float4 acc[UP];
#pragma unroll
    for (int q = 0; q < UP; ++q) zero_acc(acc[q]);
    const bool got = (inject && i == 0)
                         ? mbar_wait_bounded(never, 0, wait_ns)
                         : mbar_wait_bounded(bar0 + 8u * (i % kFwdStages), (i / kFwdStages) & 1,
                                             wait_ns);
    if (!got) {
      ok = false;
      if (lane == 0) {
        atomicExch(err, 1);
        abort_flag = 1;
      }
    } else {
      waited = i + 1;
      const float4* rows = ring + (i % kFwdStages) * STAGE + (size_t)w * kPairsPerWarp * E + ent;
      if (npw == kPairsPerWarp) {
#pragma unroll
        for (int p = 0; p < kPairsPerWarp; ++p)
#pragma unroll
          for (int q = 0; q < UP; ++q) fwd_mac(acc[q], rows[(q * kZPairs + p) * E], xr[p]);
      } else {
#pragma unroll
        for (int p = 0; p < kPairsPerWarp; ++p)
          if (p < npw)
#pragma unroll
            for (int q = 0; q < UP; ++q) fwd_mac(acc[q], rows[(q * kZPairs + p) * E], xr[p]);
      }
    }
    float4* red = red0 + (i & 1) * kContractWarps * UP * 32;
#pragma unroll
    for (int q = 0; q < UP; ++q)
      red[(w * UP + q) * 32 + lane] = acc[q];
    __syncthreads();  // partials written; every warp is done with stage i
    if (abort_flag) ok = false;
    if (ok && threadIdx.x == 0 && i + kFwdStages < n) issue(i + kFwdStages);
    if (w < UP && ok) {  // warp q adds the 8 partials of bin ug*UP + q
      float4 sum = red[w * 32 + lane];
#pragma unroll
      for (int k = 1; k < kContractWarps; ++k) {
        const float4 v = red[(k * UP + w) * 32 + lane];
        sum.x += v.x; sum.y += v.y; sum.z += v.z; sum.w += v.w;
      }
      Yp[((size_t)cp.zb * Up + cp.ug * UP + w) * ns4 + cp.st * 32 + lane] = sum;
    }
    if (!ok) break;
  }
  if (!ok && threadIdx.x == 0) {  // drain the units issued but not waited for
    const int issued = min(n, waited + kFwdStages);
    for (int k = waited; k < issued; ++k)
      mbar_wait_bounded(bar0 + 8u * (k % kFwdStages), (k / kFwdStages) & 1, kDrainNs);
  }
}

// Adjoint contraction with partial sums (used when the segment-aligned
// variant below does not fit): units (st, zb, bin group) as in the forward,
// a contiguous share per CTA; warp w owns depth pairs 8 w .. 8 w + 7 of the
// block and streams its part of every unit (UP bins x 8 pairs x E, 4 KB)
// through its own 3-slot ring, filled by its lane 0 with one bulk copy per
// bin and tracked by one mbarrier per slot (always arrived on, with zero
// bytes when the warp has no pairs, so every slot completes one phase per
// use).  It accumulates Gs[gslot][z][slot % 64] = sum over the CTA's bins of
// conj(T) Rh[u][slot] in registers; a segment (st, zb) split between CTAs
// leaves one partial per CTA in consecutive gslots, which the consumer adds.
template <int GS>
__device__ __forceinline__ void issue_adj_unit(const float4* __restrict__ T4, const UnitPos& p,
                                               int Up, int Nzp, int w, float4* slot,
                                               uint32_t bar, int stream_table) {
  constexpr int E = kKappaTile / GS;
  constexpr int UP = GS / 2;
  const int p0 = p.zb * kZPairs + w * kPairsPerWarp;
  const int np = min(kPairsPerWarp, max(0, Nzp - p0));
  const uint32_t bytes = (uint32_t)np * (E * 16u);
  fence_proxy_async();
  mbar_expect_tx(bar, bytes * UP);
  if (bytes) {
    const float4* src = T4 + ((size_t)(p.st * Up + p.ug * UP) * Nzp + p0) * E;
    const uint64_t pol = stream_table ? l2_evict_first_policy() : 0ull;
#pragma unroll
    for (int q = 0; q < UP; ++q)
      bulk_g2s_table(smem_addr(slot + q * kPairsPerWarp * E), src + (size_t)q * Nzp * E, bytes, bar,
                     stream_table != 0, pol);
  }
}

// Drain the copies this warp has in flight (ring uses [from, to)).
__device__ __forceinline__ void drain_warp(int from, int to, uint32_t bar0) {
  for (int i = from; i < to; ++i)
    mbar_wait_bounded(bar0 + 8u * (i % kSlots), (i / kSlots) & 1, kDrainNs);
}

template <int GS>
__global__ void __launch_bounds__(kContractThreads, kContractCtasPerSm)
contract_adj_stream(const float4* __restrict__ T4, const float4* __restrict__ Rh,
                    float4* __restrict__ Gs, int Nz, int Up, int Ns, int nzb, int nunits,
                    int* __restrict__ err, uint64_t wait_ns, int inject, int stream_table) {
  constexpr int E = kKappaTile / GS;
  constexpr int UP = GS / 2;
  constexpr int SLOT = UP * kPairsPerWarp * E;  // float4 per slot (4 KB)
  extern __shared__ __align__(128) float4 sm4[];
  float4* ring = sm4;
  uint64_t* bars = (uint64_t*)(ring + kContractWarps * kSlots * SLOT);  // [8][4]
  const int w = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int NUG = Up / UP;
  const int Nzp = (Nz + 1) / 2;
  const int G = gridDim.x, b = blockIdx.x;
  const int first = (int)(((long long)nunits * b) / G);
  const int n = (int)(((long long)nunits * (b + 1)) / G) - first;
  float4* my = ring + w * kSlots * SLOT;
  const uint32_t bar0 = smem_addr(bars + w * (kSlots + 1));
  const uint32_t never = bar0 + 8u * kSlots;  // nothing arrives here
  const int ent = lane / (GS / 2);
  if (lane == 0) {
    for (int s = 0; s <= kSlots; ++s) mbar_init(bar0 + 8u * s, 1);
    fence_mbar_init();
  }
  __syncwarp();
  const size_t ns4 = (size_t)Ns / 2;
  UnitPos ip;
  ip.init(first, NUG, nzb);
  int next_issue = 0;
  for (; next_issue < kSlots - 1 && next_issue < n; ++next_issue, ip.next(NUG, nzb))
    if (lane == 0)
      issue_adj_unit<GS>(T4, ip, Up, Nzp, w, my + (next_issue % kSlots) * SLOT,
                         bar0 + 8u * (next_issue % kSlots), stream_table);
  pdl_wait();  // Rh comes from the predecessor; the table copies above do not
  pdl_trigger();
  // Rh rows of the next unit prefetched into registers
  UnitPos rp;
  rp.init(first, NUG, nzb);
  auto load_rh = [&](float4* dst, const UnitPos& q0, bool valid) {
#pragma unroll
    for (int q = 0; q < UP; ++q)
      dst[q] = valid ? Rh[(size_t)(q0.ug * UP + q) * ns4 + q0.st * 32 + lane]
                     : make_float4(0.f, 0.f, 0.f, 0.f);
  };
  float4 rnext[UP];
  load_rh(rnext, rp, n > 0);
  UnitPos cp;
  cp.init(first, NUG, nzb);
  int p0 = cp.zb * kZPairs + w * kPairsPerWarp;
  int npw = min(kPairsPerWarp, max(0, Nzp - p0));
  PairAcc acc[kPairsPerWarp];
#pragma unroll
  for (int p = 0; p < kPairsPerWarp; ++p) zero_acc(acc[p]);
  for (int i = 0; i < n; ++i) {
    if (next_issue < n) {
      if (lane == 0)
        issue_adj_unit<GS>(T4, ip, Up, Nzp, w, my + (next_issue % kSlots) * SLOT,
                           bar0 + 8u * (next_issue % kSlots), stream_table);
      ++next_issue;
      ip.next(NUG, nzb);
    }
    float4 rr[UP];
#pragma unroll
    for (int q = 0; q < UP; ++q) rr[q] = rnext[q];
    rp.next(NUG, nzb);
    load_rh(rnext, rp, i + 1 < n);
    const bool got = (inject && i == 0)
                         ? mbar_wait_bounded(never, 0, wait_ns)
                         : mbar_wait_bounded(bar0 + 8u * (i % kSlots), (i / kSlots) & 1, wait_ns);
    if (!got) {
      if (lane == 0) atomicExch(err, 1);
      drain_warp(i, next_issue, bar0);
      return;
    }
    const float4* slot = my + (i % kSlots) * SLOT + ent;
#pragma unroll
    for (int q = 0; q < UP; ++q) {
      const DupR r = dup_r(rr[q]);
      if (npw == kPairsPerWarp) {
#pragma unroll
        for (int p = 0; p < kPairsPerWarp; ++p) adj_mac(acc[p], slot[(q * kPairsPerWarp + p) * E], r);
      } else {
#pragma unroll
        for (int p = 0; p < kPairsPerWarp; ++p)
          if (p < npw) adj_mac(acc[p], slot[(q * kPairsPerWarp + p) * E], r);
      }
    }
    __syncwarp();
    const int seg = cp.seg;
    cp.next(NUG, nzb);
    if (i + 1 == n || cp.seg != seg) {  // end of this CTA's part of segment seg
      if (npw > 0) {
        float4* dst = Gs + ((size_t)(seg + b) * kZBlock + w * kRowsPerWarp) * 32 + lane;
#pragma unroll
        for (int p = 0; p < kPairsPerWarp; ++p) {
          if (p < npw) {
            const float2 ra = acc[p].ra, ia = acc[p].ia, rb = acc[p].rb, ib = acc[p].ib;
            dst[(2 * p) * 32] = make_float4(ra.x, ia.x, rb.x, ib.x);
            dst[(2 * p + 1) * 32] = make_float4(ra.y, ia.y, rb.y, ib.y);
          }
        }
      }
#pragma unroll
      for (int p = 0; p < kPairsPerWarp; ++p) zero_acc(acc[p]);
      p0 = cp.zb * kZPairs + w * kPairsPerWarp;
      npw = min(kPairsPerWarp, max(0, Nzp - p0));
    }
  }
}

// Segment-aligned adjoint: one CTA per segment (slot tile st, 32-depth block
// zb), all bins, so each output value is summed by exactly one warp and the
// result is dense (Gs[seg][32][64] = Ghat[z][slot] in tile order): no partial
// sums.  Chosen when the number of such segments fits the resident grid.
// Warp w owns depths zb*32 + 4w .. +3 (two depth pairs).  The slot tile's
// residual spectra Rh[.][st] for all bins are staged once in shared memory;
// the table streams through a 2-slot ring per warp, each slot holding 2 GS
// bins x 2 depth pairs (4 KB), filled by cp.async.bulk (one copy per bin,
// issued by one lane per bin) and tracked by one mbarrier per slot.
constexpr int kSegRows = 4;                // depths per warp
constexpr int kSegPairs = kSegRows / 2;    // depth pairs per warp
constexpr int kSegSlots = 2;               // ring slots per warp
template <int GS>
__global__ void __launch_bounds__(kContractThreads, kContractCtasPerSm)
contract_adj_seg(const float4* __restrict__ T4, const float4* __restrict__ Rh,
                 float4* __restrict__ Gs, int Nz, int Up, int Ns, int anzb,
                 int* __restrict__ err, uint64_t wait_ns, int inject) {
  constexpr int E = kKappaTile / GS;
  constexpr int UPA = 2 * GS;                   // bins per ring slot
  constexpr int SLOT = UPA * kSegPairs * E;     // float4 per slot (4 KB)
  extern __shared__ __align__(128) float4 sm4[];
  float4* rtile = sm4;                                          // [Up][32]
  float4* ring = rtile + (size_t)Up * 32;                       // [8][2][SLOT]
  uint64_t* bars = (uint64_t*)(ring + kContractWarps * kSegSlots * SLOT);
  const int w = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int seg = blockIdx.x;
  const int st = seg / anzb, zb = seg - st * anzb;
  const int Nzp = (Nz + 1) / 2;
  const size_t ns4 = (size_t)Ns / 2;
  float4* my = ring + w * kSegSlots * SLOT;
  const uint32_t bar0 = smem_addr(bars + w * (kSegSlots + 1));
  const uint32_t never = bar0 + 8u * kSegSlots;  // nothing arrives here
  if (lane == 0) {
    for (int k = 0; k <= kSegSlots; ++k) mbar_init(bar0 + 8u * k, 1);
    fence_mbar_init();
  }
  __syncthreads();
  const int p0 = zb * (kContractWarps * kSegPairs) + w * kSegPairs;  // first global pair
  const int np = min(kSegPairs, max(0, Nzp - p0));
  const int ent = lane / (GS / 2);
  const int nch = (Up + UPA - 1) / UPA;
  const uint32_t bin_bytes = (uint32_t)np * E * 16u;
  auto issue = [&](int c) {
    const int nb = min(UPA, Up - c * UPA);
    float4* slot = my + (c % kSegSlots) * SLOT;
    const uint32_t bar = bar0 + 8u * (c % kSegSlots);
    if (lane == 0) {
      fence_proxy_async();
      mbar_expect_tx(bar, bin_bytes * nb);
    }
    __syncwarp();
    if (bin_bytes && lane < nb) {
      const float4* src = T4 + ((size_t)(st * Up + c * UPA + lane) * Nzp + p0) * E;
      bulk_g2s(smem_addr(slot + lane * kSegPairs * E), src, bin_bytes, bar);
    }
  };
  for (int c = 0; c < kSegSlots - 1 && c < nch; ++c) issue(c);
  pdl_wait();  // Rh comes from the predecessor; the table copies above do not
  pdl_trigger();
  for (int i = threadIdx.x; i < Up * 32; i += kContractThreads)
    rtile[i] = Rh[(size_t)(i >> 5) * ns4 + st * 32 + (i & 31)];
  __syncthreads();
  PairAcc acc[kSegPairs];
#pragma unroll
  for (int p = 0; p < kSegPairs; ++p) zero_acc(acc[p]);
  for (int c = 0; c < nch; ++c) {
    if (c + kSegSlots - 1 < nch) issue(c + kSegSlots - 1);
    const bool got = (inject && c == 0)
                         ? mbar_wait_bounded(never, 0, wait_ns)
                         : mbar_wait_bounded(bar0 + 8u * (c % kSegSlots), (c / kSegSlots) & 1, wait_ns);
    if (!got) {
      if (lane == 0) atomicExch(err, 1);
      for (int k = c; k < min(nch, c + kSegSlots); ++k)  // drain what was issued
        mbar_wait_bounded(bar0 + 8u * (k % kSegSlots), (k / kSegSlots) & 1, kDrainNs);
      return;
    }
    const float4* slot = my + (c % kSegSlots) * SLOT + ent;
    const int nb = min(UPA, Up - c * UPA);
#pragma unroll
    for (int q = 0; q < UPA; ++q)
      if (q < nb) {
        const DupR r = dup_r(rtile[(c * UPA + q) * 32 + lane]);
        if (np == kSegPairs) {
#pragma unroll
          for (int p = 0; p < kSegPairs; ++p) adj_mac(acc[p], slot[(q * kSegPairs + p) * E], r);
        } else {
#pragma unroll
          for (int p = 0; p < kSegPairs; ++p)
            if (p < np) adj_mac(acc[p], slot[(q * kSegPairs + p) * E], r);
        }
      }
    __syncwarp();
  }
  // rows 4 w .. 4 w + 3 of the segment: depths 2 (p0 + p) and 2 (p0 + p) + 1
  float4* dst = Gs + ((size_t)seg * (kContractWarps * kSegRows) + w * kSegRows) * 32 + lane;
#pragma unroll
  for (int p = 0; p < kSegPairs; ++p) {
    const int z = 2 * (p0 + p);
    const float2 ra = acc[p].ra, ia = acc[p].ia, rb = acc[p].rb, ib = acc[p].ib;
    if (z < Nz) dst[(2 * p) * 32] = make_float4(ra.x, ia.x, rb.x, ib.x);
    if (z + 1 < Nz) dst[(2 * p + 1) * 32] = make_float4(ra.y, ia.y, rb.y, ib.y);
  }
}

// ---------------------------------------------------------------------------
// Small kernels
// ---------------------------------------------------------------------------
__global__ void set_thresholds_kernel(float* scal, double* red, double lambda, double L,
                                      int use_mu, double mu, int* err) {
  double lam = lambda;
  if (use_mu) lam = mu * (double)__uint_as_float(((unsigned int*)scal)[kLamMax]);
  if (!isfinite(lam)) atomicExch(err, 2);  // non-finite data reached the lambda rule
  scal[kThr] = (float)(lam / L);
  scal[kInvL] = (float)(1.0 / L);
  red[kNumRed - 1] = lam;
}

// Thresholds of scene blockIdx.x of a batched FISTA call (scal per scene).
__global__ void set_thresholds_batched_kernel(float* scal, double lambda, double L, int use_mu,
                                              double mu, int* err) {
  float* sc = scal + (size_t)blockIdx.x * kNumFloatScalars;
  double lam = lambda;
  if (use_mu) lam = mu * (double)__uint_as_float(((unsigned int*)sc)[kLamMax]);
  if (!isfinite(lam)) atomicExch(err, 2);
  sc[kThr] = (float)(lam / L);
  sc[kInvL] = (float)(1.0 / L);
}

// y[s][m] -> yplane[u][s] (zero where plane u is not kept at position s)
__global__ void scatter_y_planes_kernel(const float2* __restrict__ y,
                                        const int32_t* __restrict__ posmap,
                                        float2* __restrict__ yplane, int S, int M, int U) {
  // scene blockIdx.y of a batched launch
  y += (size_t)blockIdx.y * S * M;
  yplane += (size_t)blockIdx.y * U * S;
  const size_t n = (size_t)U * S;
  for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < n;
       i += (size_t)gridDim.x * blockDim.x) {
    const int m = posmap[i];
    const size_t s = i % S;
    yplane[i] = m >= 0 ? y[s * M + m] : make_float2(0.f, 0.f);
  }
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
// nplanes planes of each of `batch` scenes (gridDim.y; blockIdx.y = scene)
// QUAD = false: launch shape of the full-plane engine (the table build).
template <int P, bool TWO_D, bool QUAD = true, typename K, typename... Args>
int launch_plane(K kernel, int nplanes, int d_batch, cudaStream_t st, Args... args) {
  using F = PlaneFFT<P, TWO_D, QUAD>;
  if (nplanes <= 0) return SFS_OK;
  SFS_TRY(ensure_smem_attr(kernel, F::SMEM));
  return launch_pdl(kernel, dim3(nplanes, std::max(1, d_batch)), dim3(F::NT), F::SMEM, st, args...);
}

// The cluster version of a plane kernel: kQuadCl CTAs per plane.
template <int P, bool TWO_D, typename K, typename... Args>
int launch_plane_cl(K kernel, int nplanes, int d_batch, cudaStream_t st, Args... args) {
  using F = PlaneFFT<P, TWO_D>;
  if (nplanes <= 0) return SFS_OK;
  constexpr int smem = quad_cl_smem<P, TWO_D>();
  SFS_TRY(ensure_smem_attr(kernel, smem));
  return launch_pdl_cluster(kernel, kQuadCl, dim3(nplanes * kQuadCl, std::max(1, d_batch)), dim3(F::NT),
                            smem, st, args...);
}

// Whether n quadrant planes (planes x scenes of one launch) run as clusters.
// One-CTA planes (two per SM) take about three times as long as a cluster's
// CTA (one quadrant each); the cluster form pays off while its 4 n CTAs fill
// at most three waves of two per SM, i.e. 2 n <= 3 SMs.  Measured on GB300,
// vol64 (152 SMs): 163 bin planes 57.5 -> 53.3 us as clusters, 256 depth
// planes 60.3 -> 73.1 us (four waves), so those stay one CTA per plane.
bool plane_clusters(long long n) {
  static int sms[64] = {0};
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= 64) return false;
  if (sms[dev] == 0) {
    int v = 0;
    if (cudaDeviceGetAttribute(&v, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess || v <= 0) return false;
    sms[dev] = v;
  }
  return 2 * n <= 3LL * sms[dev];
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

int ensure_smem_attr_ptr(const void* kernel, int need) {
  int dev = 0;
  SFS_CUDA(cudaGetDevice(&dev));
  static std::mutex mu;
  static std::unordered_map<const void*, uint64_t> done;  // kernel -> device bits
  std::lock_guard<std::mutex> lock(mu);
  uint64_t& bits = done[kernel];
  if (dev < 64 && ((bits >> dev) & 1u)) return SFS_OK;
  cudaFuncAttributes fa;
  SFS_CUDA(cudaFuncGetAttributes(&fa, kernel));
  const int limit = max_smem_optin() - (int)fa.sharedSizeBytes;
  if (need > limit) {
    set_error("kernel needs %d bytes of dynamic shared memory, device allows %d", need, limit);
    return SFS_ERR_INVALID_ARG;
  }
  if (need > 48 * 1024)
    SFS_CUDA(cudaFuncSetAttribute(kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, limit));
  if (dev < 64) bits |= (uint64_t)1 << dev;  // each kernel always asks the same size
  return SFS_OK;
}

int& launch_priority() {
  static thread_local int prio = 0;
  return prio;
}

bool pdl_enabled() {
  static const bool on = [] {
    const char* v = getenv("SFS_PDL");
    return v && v[0] == '1';
  }();
  return on;
}

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
    return launch_plane<P, TD, false>(build_table_kernel<P, TD>, d.U * d.Nz, 1, st, d, tof, gdir,
                                      amp, bins, table);
  });
}

int launch_fwd_planes(const PlaneDims& d, const float2* x, float2* Xh, cudaStream_t st) {
  return dispatch_plane(d, [&]<int P, bool TD>() {
    return launch_plane<P, TD>(fwd_planes_kernel<P, TD>, d.Nz, d.batch, st, d, x, Xh);
  });
}

int launch_inv_gather(const PlaneDims& d, const float2* Yh, const int32_t* posmap,
                      float2* y, double* red_sumsq, cudaStream_t st) {
  return dispatch_plane(d, [&]<int P, bool TD>() {
    return launch_plane<P, TD>(inv_gather_kernel<P, TD>, d.U, d.batch, st, d, Yh, posmap, y,
                               red_sumsq);
  });
}

int launch_inv_resid_fwd(const PlaneDims& d, const float2* Yh, const int32_t* posmap,
                         const float2* yplane, float2* Rh, double* red_sumsq,
                         cudaStream_t st) {
  return dispatch_plane(d, [&]<int P, bool TD>() {
    if constexpr (PlaneFFT<P, TD>::QUAD) {
      if (plane_clusters((long long)d.U * std::max(1, d.batch)))
        return launch_plane_cl<P, TD>(inv_resid_fwd_cl_kernel<P, TD>, d.U, d.batch, st, d, Yh, posmap,
                                      yplane, Rh, red_sumsq);
    }
    return launch_plane<P, TD>(inv_resid_fwd_kernel<P, TD>, d.U, d.batch, st, d, Yh, posmap, yplane,
                               Rh, red_sumsq);
  });
}

int launch_scatter_fwd(const PlaneDims& d, const float2* y, const int32_t* posmap,
                       float2* Rh, cudaStream_t st) {
  return dispatch_plane(d, [&]<int P, bool TD>() {
    return launch_plane<P, TD>(scatter_fwd_kernel<P, TD>, d.U, d.batch, st, d, y, posmap, Rh);
  });
}

int launch_inv_store(const PlaneDims& d, const float2* Gh, const int2* segslot, float2* x,
                     double* red_sumsq, unsigned int* maxabs_bits, cudaStream_t st) {
  return dispatch_plane(d, [&]<int P, bool TD>() {
    return launch_plane<P, TD>(inv_store_kernel<P, TD>, d.Nz, d.batch, st, d, Gh, segslot, x, red_sumsq,
                               maxabs_bits);
  });
}

int launch_inv_fista_fwd(const PlaneDims& d, const float2* Gh, const int2* segslot, float2* xk,
                         float2* gam, const float* scal, float beta, int do_fwd, float2* Xh,
                         double* red_l1, cudaStream_t st, const float* beta_dev) {
  return dispatch_plane(d, [&]<int P, bool TD>() {
    if constexpr (PlaneFFT<P, TD>::QUAD) {
      if (plane_clusters((long long)d.Nz * std::max(1, d.batch)))
        return launch_plane_cl<P, TD>(inv_fista_fwd_cl_kernel<P, TD>, d.Nz, d.batch, st, d, Gh, segslot,
                                      xk, gam, scal, beta, beta_dev, do_fwd, Xh, red_l1);
    }
    return launch_plane<P, TD>(inv_fista_fwd_kernel<P, TD>, d.Nz, d.batch, st, d, Gh, segslot, xk, gam,
                               scal, beta, beta_dev, do_fwd, Xh, red_l1);
  });
}

// Momentum coefficients of Algorithm 1 in FP64, one thread:
// beta_k = (t_k - 1) / t_{k+1}, t_{k+1} = (1 + sqrt(1 + 4 t_k^2)) / 2 for
// k = 1..iters from t_1 = *t_in (1 when t_in is null); writes t_{iters+1} to
// *t_out and, when cnt is given, adds iters to it.  Every FISTA call of an
// operator runs this same code, so a call resumed from a stored t continues
// the sequence of an uninterrupted call bit for bit.
__global__ void fista_betas_kernel(const double* t_in, int iters, float* __restrict__ beta,
                                   double* t_out, long long* cnt) {
  if (threadIdx.x != 0 || blockIdx.x != 0) return;
  double t = t_in ? *t_in : 1.0;
  for (int k = 0; k < iters; ++k) {
    const double tn = 0.5 * (1.0 + sqrt(1.0 + 4.0 * t * t));
    beta[k] = (float)((t - 1.0) / tn);
    t = tn;
  }
  *t_out = t;
  if (cnt) *cnt += iters;
}

int launch_fista_betas(const double* t_in, int iters, float* beta, double* t_out, long long* cnt,
                       cudaStream_t st) {
  fista_betas_kernel<<<1, 1, 0, st>>>(t_in, iters, beta, t_out, cnt);
  SFS_CUDA(cudaGetLastError());
  return SFS_OK;
}

int contract_units(const PlaneDims& d) {
  return (d.Ns / kKappaTile) * d.nzb * (d.Up / (d.GS / 2));
}


namespace {
// ring slot of the adjoints: (GS / 2) bins x 8 depth pairs (stream) or 2 GS
// bins x 2 depth pairs (segment-aligned), x (64 / GS) entries x 16 bytes = 4 KB
constexpr size_t kRingSlotBytes = 4096;
template <int GS>
size_t contract_fwd_smem() {
  return (size_t)2 * kContractWarps * (GS / 2) * 32 * 16 +
         (size_t)kFwdStages * (GS / 2) * kZPairs * (kKappaTile / GS) * 16 + (kFwdStages + 1) * 8;
}
template <int GS>
size_t contract_adj_smem() {
  return (size_t)kContractWarps * kSlots * kRingSlotBytes + kContractWarps * (kSlots + 1) * 8;
}
template <int GS>
int launch_fwd_gs(const PlaneDims& d, const float2* table, const float2* Xh, float2* Yp,
                  int* err, cudaStream_t st) {
  const size_t smem = contract_fwd_smem<GS>();
  SFS_TRY(ensure_smem_attr(contract_fwd_stream<GS>, (int)smem));
  const int n = contract_units(d);
  const int G = std::min(d.G, n);
  return launch_pdl(contract_fwd_stream<GS>, dim3(G), dim3(kContractThreads), smem, st,
                    (const float4*)table, (const float4*)Xh, (float4*)Yp, d.Nz, d.Up, d.Ns, d.nzb, n,
                    err, d.wait_ns, d.inject, d.stream_table);
}
template <int GS>
int launch_adj_gs(const PlaneDims& d, const float2* table, const float2* Rh, float2* Gs,
                  int* err, cudaStream_t st) {
  const size_t smem = contract_adj_smem<GS>();
  SFS_TRY(ensure_smem_attr(contract_adj_stream<GS>, (int)smem));
  const int n = contract_units(d);
  const int G = std::min(d.G, n);
  return launch_pdl(contract_adj_stream<GS>, dim3(G), dim3(kContractThreads), smem, st,
                    (const float4*)table, (const float4*)Rh, (float4*)Gs, d.Nz, d.Up, d.Ns, d.nzb, n, err, d.wait_ns,
                    d.inject, d.stream_table);
}
}  // namespace

int launch_contract_fwd(const PlaneDims& d, const float2* table, const float2* Xh,
                        float2* Yp, int* err, cudaStream_t st) {
  if (d.tc == 2) return launch_contract_fwd_h(d, Xh, Yp, err, st);
  if (d.batch > 1) {  // one launch per scene
    PlaneDims d1 = d;
    d1.batch = 1;
    for (int b = 0; b < d.batch; ++b)
      SFS_TRY(launch_contract_fwd(d1, table, Xh + b * d.bs_xh, Yp + b * d.bs_yh, err, st));
    return SFS_OK;
  }
  if (d.tc) return launch_contract_fwd_tc(d, table, Xh, Yp, err, st);
  switch (d.GS) {
    case 2: return launch_fwd_gs<2>(d, table, Xh, Yp, err, st);
    case 4: return launch_fwd_gs<4>(d, table, Xh, Yp, err, st);
    case 8: return launch_fwd_gs<8>(d, table, Xh, Yp, err, st);
  }
  set_error("unsupported orbit size %d", d.GS);
  return SFS_ERR_INVALID_ARG;
}

template <int GS>
size_t contract_adj_seg_smem(int Up) {
  return (size_t)Up * 32 * 16 + (size_t)kContractWarps * kSegSlots * kRingSlotBytes +
         kContractWarps * (kSegSlots + 1) * 8;
}
template <int GS>
int launch_adj_seg_gs(const PlaneDims& d, const float2* table, const float2* Rh, float2* Gs,
                      int* err, cudaStream_t st) {
  const size_t smem = contract_adj_seg_smem<GS>(d.Up);
  SFS_TRY(ensure_smem_attr(contract_adj_seg<GS>, (int)smem));
  return launch_pdl(contract_adj_seg<GS>, dim3(d.Ga), dim3(kContractThreads), smem, st,
                    (const float4*)table, (const float4*)Rh, (float4*)Gs, d.Nz, d.Up, d.Ns, d.anzb, err, d.wait_ns,
                    d.inject);
}

size_t adj_seg_smem_bytes(int Up) { return contract_adj_seg_smem<8>(Up); }

int launch_contract_adj(const PlaneDims& d, const float2* table, const float2* Rh,
                        float2* Gs, int* err, cudaStream_t st) {
  if (d.tc == 2) return launch_contract_adj_h(d, Rh, Gs, err, st);
  if (d.batch > 1) {  // one launch per scene
    PlaneDims d1 = d;
    d1.batch = 1;
    for (int b = 0; b < d.batch; ++b)
      SFS_TRY(launch_contract_adj(d1, table, Rh + b * d.bs_rh, Gs + b * d.bs_gh, err, st));
    return SFS_OK;
  }
  if (d.tc) return launch_contract_adj_tc(d, table, Rh, Gs, err, st);
  if (d.adj_seg) {
    switch (d.GS) {
      case 2: return launch_adj_seg_gs<2>(d, table, Rh, Gs, err, st);
      case 4: return launch_adj_seg_gs<4>(d, table, Rh, Gs, err, st);
      case 8: return launch_adj_seg_gs<8>(d, table, Rh, Gs, err, st);
    }
  }
  switch (d.GS) {
    case 2: return launch_adj_gs<2>(d, table, Rh, Gs, err, st);
    case 4: return launch_adj_gs<4>(d, table, Rh, Gs, err, st);
    case 8: return launch_adj_gs<8>(d, table, Rh, Gs, err, st);
  }
  set_error("unsupported orbit size %d", d.GS);
  return SFS_ERR_INVALID_ARG;
}

int prepare_kernels(const PlaneDims& d) {
  SFS_TRY(dispatch_plane(d, [&]<int P, bool TD>() -> int {
    constexpr int sm = PlaneFFT<P, TD>::SMEM;
    SFS_TRY(ensure_smem_attr(build_table_kernel<P, TD>, PlaneFFT<P, TD, false>::SMEM));
    SFS_TRY(ensure_smem_attr(fwd_planes_kernel<P, TD>, sm));
    SFS_TRY(ensure_smem_attr(inv_gather_kernel<P, TD>, sm));
    SFS_TRY(ensure_smem_attr(inv_resid_fwd_kernel<P, TD>, sm));
    SFS_TRY(ensure_smem_attr(scatter_fwd_kernel<P, TD>, sm));
    SFS_TRY(ensure_smem_attr(inv_store_kernel<P, TD>, sm));
    SFS_TRY(ensure_smem_attr(inv_fista_fwd_kernel<P, TD>, sm));
    return SFS_OK;
  }));
  if (d.tc == 2) return prepare_tc16_kernels(d);
  if (d.tc) return prepare_tc_kernels();
  if (d.adj_seg) {
    switch (d.GS) {
      case 2: SFS_TRY(ensure_smem_attr(contract_adj_seg<2>, (int)contract_adj_seg_smem<2>(d.Up))); break;
      case 4: SFS_TRY(ensure_smem_attr(contract_adj_seg<4>, (int)contract_adj_seg_smem<4>(d.Up))); break;
      case 8: SFS_TRY(ensure_smem_attr(contract_adj_seg<8>, (int)contract_adj_seg_smem<8>(d.Up))); break;
    }
  }
  switch (d.GS) {
    case 2:
      SFS_TRY(ensure_smem_attr(contract_fwd_stream<2>, (int)contract_fwd_smem<2>()));
      return ensure_smem_attr(contract_adj_stream<2>, (int)contract_adj_smem<2>());
    case 4:
      SFS_TRY(ensure_smem_attr(contract_fwd_stream<4>, (int)contract_fwd_smem<4>()));
      return ensure_smem_attr(contract_adj_stream<4>, (int)contract_adj_smem<4>());
    case 8:
      SFS_TRY(ensure_smem_attr(contract_fwd_stream<8>, (int)contract_fwd_smem<8>()));
      return ensure_smem_attr(contract_adj_stream<8>, (int)contract_adj_smem<8>());
  }
  set_error("unsupported orbit size %d", d.GS);
  return SFS_ERR_INVALID_ARG;
}

int launch_set_thresholds(float* scal, double* red, double lambda, double L, int use_mu,
                          double mu, int* err, cudaStream_t st) {
  set_thresholds_kernel<<<1, 1, 0, st>>>(scal, red, lambda, L, use_mu, mu, err);
  SFS_CUDA(cudaGetLastError());
  return SFS_OK;
}

int launch_set_thresholds_batched(float* scal, int batch, double lambda, double L, int use_mu,
                                  double mu, int* err, cudaStream_t st) {
  set_thresholds_batched_kernel<<<batch, 1, 0, st>>>(scal, lambda, L, use_mu, mu, err);
  SFS_CUDA(cudaGetLastError());
  return SFS_OK;
}

int launch_scatter_y_planes(const PlaneDims& d, const float2* y, const int32_t* posmap,
                            float2* yplane, cudaStream_t st) {
  const size_t n = (size_t)d.U * d.S;
  size_t blocks = (n + 255) / 256;
  if (blocks > 2432) blocks = 2432;
  scatter_y_planes_kernel<<<dim3((unsigned)blocks, std::max(1, d.batch)), 256, 0, st>>>(y, posmap, yplane,
                                                                                     d.S, d.M, d.U);
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
