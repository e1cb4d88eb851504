// Device code of the lateral plane engine shared by the kernel files of
// libsfs: block reductions, the slot-order loads and stores of lateral
// spectra, and the forward / inverse plane steps of A and A^H (Sec. IV-B,
// Algorithm 2).  Everything lives in an unnamed namespace, so each file that
// includes it compiles its own copy.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include "sfs_async.cuh"
#include "sfs_fft.cuh"
#include "sfs_internal.h"

namespace sfs {
namespace {

// ---------------------------------------------------------------------------
// Block reductions
// ---------------------------------------------------------------------------
template <int NT>
__device__ __forceinline__ void block_add_double(double v, double* out) {
  __shared__ double part_g[2][NT / 32];  // per thread group (at most two per CTA)
  double* part = part_g[group_of<NT>()];
#pragma unroll
  for (int off = 16; off > 0; off >>= 1) v += __shfl_xor_sync(0xffffffffu, v, off);
  const int warp = gtid<NT>() >> 5, lane = threadIdx.x & 31;
  if (lane == 0) part[warp] = v;
  group_sync<NT>();
  if (warp == 0) {
    v = lane < NT / 32 ? part[lane] : 0.0;
#pragma unroll
    for (int off = 16; off > 0; off >>= 1) v += __shfl_xor_sync(0xffffffffu, v, off);
    if (lane == 0) atomicAdd(out, v);
  }
}

// max that keeps a NaN (fmaxf would drop it), so that a non-finite input shows
// up in the reduced value
__device__ __forceinline__ float nanmax(float a, float b) {
  return (a != a) ? a : ((b != b) ? b : fmaxf(a, b));
}

template <int NT>
__device__ __forceinline__ void block_max_bits(float v, unsigned int* out) {
  __shared__ float part_g[2][NT / 32];
  float* part = part_g[group_of<NT>()];
#pragma unroll
  for (int off = 16; off > 0; off >>= 1) v = nanmax(v, __shfl_xor_sync(0xffffffffu, v, off));
  const int warp = gtid<NT>() >> 5, lane = threadIdx.x & 31;
  if (lane == 0) part[warp] = v;
  group_sync<NT>();
  if (warp == 0) {
    v = lane < NT / 32 ? part[lane] : 0.0f;
#pragma unroll
    for (int off = 16; off > 0; off >>= 1) v = nanmax(v, __shfl_xor_sync(0xffffffffu, v, off));
    // non-negative floats order like their bit patterns, and a NaN (positive
    // quiet NaN bits) orders above every finite value
    if (lane == 0) atomicMax(out, __float_as_uint(v != v ? __int_as_float(0x7fc00000) : v));
  }
}

// Block maximum of non-negative v, stored by thread 0 (fmaxf: a NaN input is
// ignored here; it still reaches the output through the values themselves).
template <int NT>
__device__ __forceinline__ void block_max_store(float v, float* out) {
  __shared__ float part_g[2][NT / 32];
  float* part = part_g[group_of<NT>()];
#pragma unroll
  for (int off = 16; off > 0; off >>= 1) v = fmaxf(v, __shfl_xor_sync(0xffffffffu, v, off));
  const int warp = gtid<NT>() >> 5, lane = threadIdx.x & 31;
  if (lane == 0) part[warp] = v;
  group_sync<NT>();
  if (warp == 0) {
    v = lane < NT / 32 ? part[lane] : 0.0f;
#pragma unroll
    for (int off = 16; off > 0; off >>= 1) v = fmaxf(v, __shfl_xor_sync(0xffffffffu, v, off));
    if (lane == 0) *out = v;
  }
}

// ---------------------------------------------------------------------------
// Plane kernels (one lateral plane per CTA)
// ---------------------------------------------------------------------------
template <int P, bool TWO_D>
__device__ __forceinline__ void zero_plane(float2* buf) {
  using F = PlaneFFT<P, TWO_D>;
  for (int e = gtid<F::NT>(); e < F::ELEMS; e += F::NT) buf[e] = make_float2(0.f, 0.f);
}

// Twiddles of the plane engine (QUAD: W_128, then W_64 for the quadrants).
template <int P, bool TWO_D>
__device__ __forceinline__ void plane_twiddles(float2* tw) {
  using F = PlaneFFT<P, TWO_D>;
  make_twiddles<P, F::NT>(tw);
  if constexpr (F::QUAD) make_twiddles<64, F::NT>(tw + P);
}

// QUAD planes: the spectrum moves quadrant by quadrant.  d.quad[0..5] are
// offsets into the entries d.quad + 8: quadrant q = 2 (ky & 1) + (kx & 1)
// owns entries quad[q] .. quad[q + 1], the padding slots quad[4] .. quad[5];
// an entry is (slot << 12) | (kx / 2 * 64 + ky / 2), the quadrant-local
// wavenumber.  Every slot appears once; each quadrant covers its 64 x 64
// local wavenumbers once.  Global loads are issued kQuadBatch deep.
constexpr int kQuadBatch = 8;
constexpr int kQuadBatchAdj = 4;  // its segment lookups hold more registers

template <int P, bool TWO_D>
__device__ __forceinline__ void load_quadrant_fwd(float2* buf, const float2* __restrict__ Yp, int u,
                                                  const PlaneDims& d, int q) {
  using F = PlaneFFT<P, TWO_D>;
  const int32_t* ql = d.quad + 8;
  const float2* src = Yp + (size_t)u * d.Ns;
  const size_t stride = (size_t)d.Up * d.Ns;
  const int i1 = __ldg(d.quad + q + 1);
  for (int i0 = __ldg(d.quad + q) + gtid<F::NT>(); i0 < i1; i0 += kQuadBatch * F::NT) {
    int ent[kQuadBatch];
    float2 v[kQuadBatch];
#pragma unroll
    for (int k = 0; k < kQuadBatch; ++k) {
      const int i = i0 + k * F::NT;
      ent[k] = i < i1 ? __ldg(ql + i) : -1;
    }
#pragma unroll
    for (int k = 0; k < kQuadBatch; ++k) v[k] = ent[k] >= 0 ? src[ent[k] >> 12] : make_float2(0.f, 0.f);
    for (int zb = 1; zb < d.nzb; ++zb)
#pragma unroll
      for (int k = 0; k < kQuadBatch; ++k)
        if (ent[k] >= 0) v[k] = cadd(v[k], src[zb * stride + (ent[k] >> 12)]);
#pragma unroll
    for (int k = 0; k < kQuadBatch; ++k)
      if (ent[k] >= 0) buf[F::qidx(ent[k] & 4095)] = v[k];
  }
}

template <int P, bool TWO_D>
__device__ __forceinline__ void load_quadrant_adj(float2* buf, const float2* __restrict__ Gs,
                                                  const int2* __restrict__ segslot, int z,
                                                  const PlaneDims& d, int q) {
  using F = PlaneFFT<P, TWO_D>;
  const int32_t* ql = d.quad + 8;
  const int zb = z / d.azb, zr = z % d.azb;
  const size_t slot_stride = (size_t)d.azb * 64;
  const int i1 = __ldg(d.quad + q + 1);
  for (int i0 = __ldg(d.quad + q) + gtid<F::NT>(); i0 < i1; i0 += kQuadBatchAdj * F::NT) {
    int ent[kQuadBatchAdj];
    int2 sc[kQuadBatchAdj];
#pragma unroll
    for (int k = 0; k < kQuadBatchAdj; ++k) {
      const int i = i0 + k * F::NT;
      ent[k] = i < i1 ? __ldg(ql + i) : -1;
    }
#pragma unroll
    for (int k = 0; k < kQuadBatchAdj; ++k) {
      const int j = ent[k] >> 12;
      const int seg = (j >> 6) * d.anzb + zb;
      sc[k] = ent[k] < 0 ? make_int2(0, 0) : (d.adj_seg ? make_int2(seg, 1) : __ldg(segslot + seg));
    }
    float2 v[kQuadBatchAdj];
#pragma unroll
    for (int k = 0; k < kQuadBatchAdj; ++k)
      v[k] = sc[k].y > 0 ? Gs[(size_t)sc[k].x * slot_stride + (size_t)zr * 64 + ((ent[k] >> 12) & 63)]
                         : make_float2(0.f, 0.f);
    int more = 0;
#pragma unroll
    for (int k = 0; k < kQuadBatchAdj; ++k) more = max(more, sc[k].y);
    for (int c = 1; c < more; ++c)
#pragma unroll
      for (int k = 0; k < kQuadBatchAdj; ++k)
        if (c < sc[k].y)
          v[k] = cadd(v[k], Gs[(size_t)(sc[k].x + c) * slot_stride + (size_t)zr * 64 + ((ent[k] >> 12) & 63)]);
#pragma unroll
    for (int k = 0; k < kQuadBatchAdj; ++k)
      if (ent[k] >= 0) buf[F::qidx(ent[k] & 4095)] = v[k];
  }
}

// Quadrant q of the spectrum in buf to its slots of dst; mx takes the
// largest |Re| or |Im| stored.  With q = 4, zero to the padding slots.
template <int P, bool TWO_D>
__device__ __forceinline__ void store_quadrant(const float2* buf, float2* __restrict__ dst,
                                               const PlaneDims& d, int q, float& mx) {
  using F = PlaneFFT<P, TWO_D>;
  const int32_t* ql = d.quad + 8;
  const int i1 = __ldg(d.quad + q + 1);
  for (int i0 = __ldg(d.quad + q) + gtid<F::NT>(); i0 < i1; i0 += kQuadBatch * F::NT) {
    int ent[kQuadBatch];
#pragma unroll
    for (int k = 0; k < kQuadBatch; ++k) {
      const int i = i0 + k * F::NT;
      ent[k] = i < i1 ? __ldg(ql + i) : -1;
    }
#pragma unroll
    for (int k = 0; k < kQuadBatch; ++k)
      if (ent[k] >= 0) {
        const float2 v = q < 4 ? buf[F::qidx(ent[k] & 4095)] : make_float2(0.f, 0.f);
        dst[ent[k] >> 12] = v;
        mx = fmaxf(mx, fmaxf(fabsf(v.x), fabsf(v.y)));
      }
  }
}

// Lateral spectra travel between kernels in slot order: slot j holds
// wavenumber slot_kappa[j] (orbit-major, GS slots per symmetry orbit, -1 for
// padding slots, which carry zero).

// The slot loops below run kLoadBatch slots per thread per round and issue
// all independent global loads of a round before using any of them, so that
// several L2 round trips overlap instead of queueing one after another.
constexpr int kLoadBatch = 12;
// 64 x 64 planes (4544 slots on a 32 x 32 scan) run two CTAs per SM at <= 64
// registers a thread: 9 slots per thread still cover 4608 slots in one round.
// 128 x 128 planes run 1024 threads (again <= 64 registers): 6 slots a round.
template <int P, bool TWO_D>
__host__ __device__ constexpr int load_batch() {
  return PlaneFFT<P, TWO_D>::LANES64 ? 9
         : PlaneFFT<P, TWO_D>::NT >= 1024 ? 6
         : (TWO_D && P == 32) ? 4  // 32 x 32 planes: at most 2 slots a thread (about 1,100 slots)
                              : kLoadBatch;
}

// Spectrum of bin plane u from the forward contraction: the sum of its nzb
// depth-block partials Yp[zb][u][slot] (plane stride Up * Ns).
template <int P, bool TWO_D>
__device__ __forceinline__ void load_spectrum_fwd(float2* buf, const float2* __restrict__ Yp,
                                                  int u, const PlaneDims& d) {
  using F = PlaneFFT<P, TWO_D>;
  constexpr int LB = load_batch<P, TWO_D>();
  const float2* src = Yp + (size_t)u * d.Ns;
  const size_t stride = (size_t)d.Up * d.Ns;
  for (int j0 = gtid<F::NT>(); j0 < d.Ns; j0 += LB * F::NT) {
    int kap[LB];
    float2 v[LB];
#pragma unroll
    for (int k = 0; k < LB; ++k) {
      const int j = j0 + k * F::NT;
      kap[k] = j < d.Ns ? __ldg(d.slot_kappa + j) : -1;
      v[k] = j < d.Ns ? src[j] : make_float2(0.f, 0.f);
    }
    for (int zb = 1; zb < d.nzb; ++zb)
#pragma unroll
      for (int k = 0; k < LB; ++k) {
        const int j = j0 + k * F::NT;
        if (j < d.Ns) v[k] = cadd(v[k], src[zb * stride + j]);
      }
#pragma unroll
    for (int k = 0; k < LB; ++k)
      if (kap[k] >= 0) buf[F::kidx(kap[k])] = v[k];
  }
}

// Spectrum of voxel plane z from the adjoint contraction: for each slot tile,
// the sum of the partial results its segment (tile, depth block) left in
// consecutive slots of Gs[slot][azb][64]; segslot[seg] = {first, count}.
template <int P, bool TWO_D>
__device__ __forceinline__ void load_spectrum_adj(float2* buf, const float2* __restrict__ Gs,
                                                  const int2* __restrict__ segslot, int z,
                                                  const PlaneDims& d) {
  using F = PlaneFFT<P, TWO_D>;
  constexpr int LB = load_batch<P, TWO_D>();
  const int zb = z / d.azb, zr = z % d.azb;
  const size_t slot_stride = (size_t)d.azb * 64;
  for (int j0 = gtid<F::NT>(); j0 < d.Ns; j0 += LB * F::NT) {
    int kap[LB];
    int2 sc[LB];
#pragma unroll
    for (int k = 0; k < LB; ++k) {
      const int j = j0 + k * F::NT;
      kap[k] = j < d.Ns ? __ldg(d.slot_kappa + j) : -1;
      // the segment-aligned adjoint leaves one dense result per segment
      const int seg = (j >> 6) * d.anzb + zb;
      sc[k] = j >= d.Ns ? make_int2(0, 0) : (d.adj_seg ? make_int2(seg, 1) : __ldg(segslot + seg));
    }
    float2 v[LB];
#pragma unroll
    for (int k = 0; k < LB; ++k) {
      const int j = j0 + k * F::NT;
      v[k] = sc[k].y > 0 ? Gs[(size_t)sc[k].x * slot_stride + (size_t)zr * 64 + (j & 63)]
                         : make_float2(0.f, 0.f);
    }
    int more = 0;
#pragma unroll
    for (int k = 0; k < LB; ++k) more = max(more, sc[k].y);
    for (int c = 1; c < more; ++c)
#pragma unroll
      for (int k = 0; k < LB; ++k) {
        const int j = j0 + k * F::NT;
        if (c < sc[k].y)
          v[k] = cadd(v[k], Gs[(size_t)(sc[k].x + c) * slot_stride + (size_t)zr * 64 + (j & 63)]);
      }
#pragma unroll
    for (int k = 0; k < LB; ++k)
      if (kap[k] >= 0) buf[F::kidx(kap[k])] = v[k];
  }
}

// Stores the plane's spectrum in slot order; with pm (FP16 modes) also the
// plane's largest |Re| or |Im| at *pm (every thread of the CTA must call).
template <int P, bool TWO_D>
__device__ __forceinline__ void store_spectrum(const float2* buf, float2* __restrict__ dst,
                                               const PlaneDims& d, float* pm = nullptr) {
  using F = PlaneFFT<P, TWO_D>;
  constexpr int LB = load_batch<P, TWO_D>();
  float mx = 0.0f;
  for (int j0 = gtid<F::NT>(); j0 < d.Ns; j0 += LB * F::NT) {
    int kap[LB];
#pragma unroll
    for (int k = 0; k < LB; ++k) {
      const int j = j0 + k * F::NT;
      kap[k] = j < d.Ns ? __ldg(d.slot_kappa + j) : -1;
    }
#pragma unroll
    for (int k = 0; k < LB; ++k) {
      const int j = j0 + k * F::NT;
      if (j < d.Ns) {
        const float2 v = kap[k] >= 0 ? buf[F::kidx(kap[k])] : make_float2(0.f, 0.f);
        dst[j] = v;
        mx = fmaxf(mx, fmaxf(fabsf(v.x), fabsf(v.y)));
      }
    }
  }
  if (pm) block_max_store<F::NT>(mx, pm);
}

// Zero every slot of the plane outside the Ny x Nx crop window (QUAD: of the
// 64 x 64 plane it holds).
template <int P, bool TWO_D>
__device__ __forceinline__ void zero_outside(float2* buf, int Ny, int Nx) {
  using F = PlaneFFT<P, TWO_D>;
  constexpr int PX = F::QUAD ? 64 : P;
  constexpr int PY = F::QUAD ? 64 : (TWO_D ? P : 1);
  for (int e = gtid<F::NT>(); e < PX * PY; e += F::NT) {
    const int py = e / PX, px = e % PX;
    if (py >= Ny || px >= Nx) buf[F::sidx(py, px)] = make_float2(0.f, 0.f);
  }
}

// Forward transform of the spatial plane in buf (zero outside the support)
// and the store of its spectrum to dst in slot order; with pm (FP16 modes)
// also the plane's largest |Re| or |Im| at *pm.  Every thread must call.
template <int P, bool TWO_D>
__device__ __forceinline__ void forward_store(float2* buf, const float2* tw, float2* __restrict__ dst,
                                              const PlaneDims& d, float* pm) {
  using F = PlaneFFT<P, TWO_D>;
  if constexpr (F::QUAD) {
    float mx = 0.0f;
    F::forward_quads(buf, tw, [&](int q) { store_quadrant<P, TWO_D>(buf, dst, d, q, mx); });
    store_quadrant<P, TWO_D>(buf, dst, d, 4, mx);
    if (pm) block_max_store<F::NT>(mx, pm);
  } else {
    F::forward(buf, tw, d.Nx);
    store_spectrum<P, TWO_D>(buf, dst, d, pm);
  }
}

// Spectrum of bin plane u from the forward contraction (Yp) into buf and its
// inverse transform: the natural-layout spatial plane in buf.
template <int P, bool TWO_D>
__device__ __forceinline__ void load_inverse_fwd(float2* buf, const float2* tw, const float2* __restrict__ Yp,
                                                 int u, const PlaneDims& d) {
  using F = PlaneFFT<P, TWO_D>;
  if constexpr (F::QUAD) {
    F::inverse_quads(buf, tw, [&](int q) { load_quadrant_fwd<P, TWO_D>(buf, Yp, u, d, q); });
  } else {
    load_spectrum_fwd<P, TWO_D>(buf, Yp, u, d);
    group_sync<F::NT>();
    F::inverse(buf, tw, d.Nx);
  }
}

// The same for voxel plane z from the adjoint contraction (Gs).
template <int P, bool TWO_D>
__device__ __forceinline__ void load_inverse_adj(float2* buf, const float2* tw, const float2* __restrict__ Gs,
                                                 const int2* __restrict__ segslot, int z, const PlaneDims& d) {
  using F = PlaneFFT<P, TWO_D>;
  if constexpr (F::QUAD) {
    F::inverse_quads(buf, tw, [&](int q) { load_quadrant_adj<P, TWO_D>(buf, Gs, segslot, z, d, q); });
  } else {
    load_spectrum_adj<P, TWO_D>(buf, Gs, segslot, z, d);
    group_sync<F::NT>();
    F::inverse(buf, tw, d.Nx);
  }
}

// Residual step on bin plane u of scene b (batched buffers; b = 0 for one
// scene): Yh[u] -> residual r = (A gamma - y) on the plane -> Rh[u] =
// FFT2(pad(r)).  yplane[u][s] holds the measurements laid out by bin plane,
// so they load alongside the selection mask instead of after it.  Every
// thread of the CTA calls it; smem holds the plane and its twiddles.
template <int P, bool TWO_D>
__device__ __forceinline__ void resid_plane_step(const PlaneDims& d, int u, long long b, float2* smem,
                                                 const float2* __restrict__ Yh,
                                                 const int32_t* __restrict__ posmap,
                                                 const float2* __restrict__ yplane, float2* __restrict__ Rh,
                                                 double* __restrict__ red_sumsq) {
  using F = PlaneFFT<P, TWO_D>;
  Yh += b * d.bs_yh;
  yplane += b * d.bs_yplane;
  Rh += b * d.bs_rh;
  if (red_sumsq) red_sumsq += b * d.bs_red;
  float2* buf = smem;
  float2* tw = smem + F::ELEMS;
  plane_twiddles<P, TWO_D>(tw);
  pdl_wait();
  pdl_trigger();
  load_inverse_fwd<P, TWO_D>(buf, tw, Yh, u, d);
  double acc = 0.0;
  const int32_t* pm = posmap + (size_t)u * d.S;
  const float2* yu = yplane + (size_t)u * d.S;
  for (int s = gtid<F::NT>(); s < d.S; s += F::NT) {
    const int m = pm[s];
    const float2 yv = yu[s];
    const int e = F::sidx(s / d.Nx, s % d.Nx);
    float2 r = make_float2(0.f, 0.f);
    if (m >= 0) {
      r = csub(buf[e], yv);
      if (red_sumsq) acc += (double)r.x * r.x + (double)r.y * r.y;
    }
    buf[e] = r;
  }
  zero_outside<P, TWO_D>(buf, d.Ny, d.Nx);
  if (red_sumsq) block_add_double<F::NT>(acc, red_sumsq);
  group_sync<F::NT>();
  forward_store<P, TWO_D>(buf, tw, Rh + (size_t)u * d.Ns, d, d.pm_r ? d.pm_r + b * d.bs_pmr + u : nullptr);
}

// FISTA step on depth plane z of scene b (Algorithm 1): Gh[z] (spectrum of
// A^H(A gamma - y)) ->
//   x_k = tau_{lambda/L}(gamma_k - grad/L), gamma_{k+1} = x_k + beta_k (x_k - x_{k-1})
// then, with do_fwd (every iteration but the last), Xh[z] =
// FFT2(pad(gamma_{k+1})).  beta_k is *beta_dev when given (a table written
// on the device), else beta_arg.  Every thread of the CTA calls it.
template <int P, bool TWO_D>
__device__ __forceinline__ void update_plane_step(const PlaneDims& d, int z, long long b, float2* smem,
                                                  const float2* __restrict__ Gh,
                                                  const int2* __restrict__ segslot, float2* __restrict__ xk,
                                                  float2* __restrict__ gam, const float* __restrict__ scal,
                                                  float beta_arg, const float* __restrict__ beta_dev,
                                                  int do_fwd, float2* __restrict__ Xh,
                                                  double* __restrict__ red_l1) {
  using F = PlaneFFT<P, TWO_D>;
  Gh += b * d.bs_gh;
  xk += b * d.bs_x;
  gam += b * d.bs_x;
  scal += b * d.bs_scal;
  Xh += b * d.bs_xh;
  if (red_l1) red_l1 += b * d.bs_red;
  float2* buf = smem;
  float2* tw = smem + F::ELEMS;
  plane_twiddles<P, TWO_D>(tw);
  pdl_wait();
  pdl_trigger();
  load_inverse_adj<P, TWO_D>(buf, tw, Gh, segslot, z, d);
  const float thr = scal[kThr];
  const float invL = scal[kInvL];
  const float beta = beta_dev ? *beta_dev : beta_arg;
  double l1 = 0.0;
  const size_t off = (size_t)z * d.Ny * d.Nx;
  for (int e = gtid<F::NT>(); e < d.Ny * d.Nx; e += F::NT) {
    const int bi = F::sidx(e / d.Nx, e % d.Nx);
    const float2 g = buf[bi];
    const float2 gm = gam[off + e];
    const float2 xp = xk[off + e];
    const float2 w = make_float2(fmaf(-g.x, invL, gm.x), fmaf(-g.y, invL, gm.y));
    const float mag = hypotf(w.x, w.y);
    const float sc = mag > thr ? 1.0f - thr / mag : 0.0f;
    const float2 xn = make_float2(w.x * sc, w.y * sc);
    const float2 gn = make_float2(fmaf(beta, xn.x - xp.x, xn.x), fmaf(beta, xn.y - xp.y, xn.y));
    xk[off + e] = xn;
    gam[off + e] = gn;
    if (red_l1) l1 += (double)(mag > thr ? mag - thr : 0.0f);
    buf[bi] = gn;
  }
  if (red_l1) block_add_double<F::NT>(l1, red_l1);
  if (!do_fwd) return;
  zero_outside<P, TWO_D>(buf, d.Ny, d.Nx);
  group_sync<F::NT>();
  forward_store<P, TWO_D>(buf, tw, Xh + (size_t)z * d.Ns, d, d.pm_x ? d.pm_x + b * d.bs_pmx + z : nullptr);
}

}  // namespace
}  // namespace sfs
