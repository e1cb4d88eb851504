// Shared-memory FFT engine for one lateral plane per CTA.
//
// The fast transform of the block 2-level Toeplitz operator (Sec. IV-B,
// Algorithm 2) needs 2-D FFTs of zero-padded Px x Py planes.  Each plane
// fits in one CTA's shared memory (Px = Py <= 128, or a line of <= 4096), so
// a plane is transformed in place: radix-2/4/8 Stockham passes whose
// butterflies are held in registers between two barriers.
//
// 2-D layout: a P x P plane with row stride P + 1 (odd, so that both the
// column passes and the transpose are free of bank conflicts).  The forward
// transform runs column FFTs along y, transposes, and runs column FFTs
// along x; its result is stored transposed, element (kx, ky) at row kx,
// column ky.  The inverse consumes that layout and returns the natural
// [y][x] layout.  Every producer and consumer of lateral spectra in this
// library uses these two routines, so the transposed wavenumber order is
// internal and consistent: kappa = kx * P + ky.
#pragma once

#include <cuda_runtime.h>

namespace sfs {

__device__ __forceinline__ float2 cmul(float2 a, float2 b) {
  return make_float2(fmaf(a.x, b.x, -a.y * b.y), fmaf(a.x, b.y, a.y * b.x));
}
// conj(a) * b
__device__ __forceinline__ float2 cmulc(float2 a, float2 b) {
  return make_float2(fmaf(a.x, b.x, a.y * b.y), fmaf(a.x, b.y, -a.y * b.x));
}
__device__ __forceinline__ float2 cadd(float2 a, float2 b) {
  return make_float2(a.x + b.x, a.y + b.y);
}
__device__ __forceinline__ float2 csub(float2 a, float2 b) {
  return make_float2(a.x - b.x, a.y - b.y);
}
// multiply by -j (forward) or +j (inverse)
template <bool INV>
__device__ __forceinline__ float2 mul_j(float2 a) {
  return INV ? make_float2(-a.y, a.x) : make_float2(a.y, -a.x);
}

// In-register DFT of length R (2, 4 or 8); forward uses e^{-j...}.
template <int R, bool INV>
__device__ __forceinline__ void dft_small(float2* v) {
  if constexpr (R == 2) {
    float2 a = v[0], b = v[1];
    v[0] = cadd(a, b);
    v[1] = csub(a, b);
  } else if constexpr (R == 4) {
    float2 s02 = cadd(v[0], v[2]), d02 = csub(v[0], v[2]);
    float2 s13 = cadd(v[1], v[3]), d13 = mul_j<INV>(csub(v[1], v[3]));
    v[0] = cadd(s02, s13);
    v[2] = csub(s02, s13);
    v[1] = cadd(d02, d13);
    v[3] = csub(d02, d13);
  } else {
    static_assert(R == 8, "radix");
    float2 e[4] = {v[0], v[2], v[4], v[6]};
    float2 o[4] = {v[1], v[3], v[5], v[7]};
    dft_small<4, INV>(e);
    dft_small<4, INV>(o);
    const float h = 0.70710678118654752440f;
    // o[k] *= W8^k, W8 = e^{-j pi/4} (forward) or e^{+j pi/4} (inverse)
    o[1] = INV ? make_float2(h * (o[1].x - o[1].y), h * (o[1].x + o[1].y))
               : make_float2(h * (o[1].x + o[1].y), h * (o[1].y - o[1].x));
    o[2] = mul_j<INV>(o[2]);
    o[3] = INV ? make_float2(-h * (o[3].x + o[3].y), h * (o[3].x - o[3].y))
               : make_float2(h * (o[3].y - o[3].x), -h * (o[3].x + o[3].y));
#pragma unroll
    for (int k = 0; k < 4; ++k) {
      v[k] = cadd(e[k], o[k]);
      v[k + 4] = csub(e[k], o[k]);
    }
  }
}

// Radix for the pass that starts after Ns points are combined.
__host__ __device__ constexpr int pass_radix(int N, int Ns) {
  return (N / Ns) % 8 == 0 ? 8 : ((N / Ns) % 4 == 0 ? 4 : 2);
}

// Thread groups of the plane engine.  A plane is transformed by a group of
// NT threads: the whole CTA of the plane kernels, or one of the equal groups
// of a larger CTA (the persistent solve runs two 512-thread groups, one plane
// each).  gtid<NT>() is the thread's index in its group, group_of<NT>() the
// group, group_sync<NT>() the group's barrier (named barrier 2 or 3;
// barriers 0 and 1 are left to whole-CTA and other uses).
template <int NT>
__device__ __forceinline__ int gtid() {
  static_assert((NT & (NT - 1)) == 0 && NT >= 32, "group size");
  return (int)threadIdx.x & (NT - 1);
}
template <int NT>
__device__ __forceinline__ int group_of() {
  return (int)threadIdx.x / NT;
}
template <int NT>
__device__ __forceinline__ void group_sync() {
  // immediate barrier numbers, so that a kernel reserves only the barriers it uses
  if (threadIdx.x < NT)
    asm volatile("bar.sync 2, %0;" ::"n"(NT) : "memory");
  else
    asm volatile("bar.sync 3, %0;" ::"n"(NT) : "memory");
}

// twiddle table: tw[m] = exp(-2 pi j m / N), m in [0, N)
template <int N, int NT>
__device__ __forceinline__ void make_twiddles(float2* tw) {
  for (int m = gtid<NT>(); m < N; m += NT) {
    float s, c;
    sincospif(-2.0f * (float)m / (float)N, &s, &c);
    tw[m] = make_float2(c, s);
  }
}

// One Stockham pass (radix R, Ns points combined so far) over `count`
// sequences of length N; element n of sequence q lives at buf[q*sd + n*es].
// QFAST: consecutive threads take consecutive sequences (column passes),
// otherwise consecutive butterflies of one sequence (row passes).
template <int N, int R, bool INV, int NT, int MAXB, bool QFAST>
__device__ __forceinline__ void stockham_pass(float2* buf, int count, int es,
                                              int sd, int Ns, const float2* tw) {
  constexpr int NB = N / R;
  float2 v[MAXB][R];
  const int total = count * NB;
#pragma unroll
  for (int i = 0; i < MAXB; ++i) {
    const int b = gtid<NT>() + i * NT;
    if (b < total) {
      const int q = QFAST ? b % count : b / NB;
      const int j = QFAST ? b / count : b % NB;
      const float2* src = buf + q * sd;
#pragma unroll
      for (int r = 0; r < R; ++r) v[i][r] = src[(j + r * NB) * es];
    }
  }
  group_sync<NT>();
#pragma unroll
  for (int i = 0; i < MAXB; ++i) {
    const int b = gtid<NT>() + i * NT;
    if (b < total) {
      const int q = QFAST ? b % count : b / NB;
      const int j = QFAST ? b / count : b % NB;
      const int k = j & (Ns - 1);
      if (Ns > 1) {
        const int step = k * (N / (Ns * R));
#pragma unroll
        for (int r = 1; r < R; ++r) {
          float2 w = tw[step * r];
          if (INV) w.y = -w.y;
          v[i][r] = cmul(v[i][r], w);
        }
      }
      dft_small<R, INV>(v[i]);
      const int base = (j - k) * R + k;
      float2* dst = buf + q * sd;
#pragma unroll
      for (int r = 0; r < R; ++r) dst[(base + r * Ns) * es] = v[i][r];
    }
  }
  group_sync<NT>();
}

// Full FFT of length N on `count` sequences (all passes).
template <int N, bool INV, int NT, int MAXCOUNT, bool QFAST, int Ns = 1>
__device__ __forceinline__ void fft_multi(float2* buf, int count, int es, int sd,
                                          const float2* tw) {
  if constexpr (Ns < N) {
    constexpr int R = pass_radix(N, Ns);
    constexpr int MAXB = (MAXCOUNT * (N / R) + NT - 1) / NT;
    stockham_pass<N, R, INV, NT, MAXB, QFAST>(buf, count, es, sd, Ns, tw);
    fft_multi<N, INV, NT, MAXCOUNT, QFAST, Ns * R>(buf, count, es, sd, tw);
  }
}

// In-place transpose of a P x P plane (row stride LD) through registers.
template <int P, int LD, int NT>
__device__ __forceinline__ void transpose_plane(float2* buf) {
  constexpr int PER = (P * P + NT - 1) / NT;
  float2 v[PER];
#pragma unroll
  for (int i = 0; i < PER; ++i) {
    const int e = gtid<NT>() + i * NT;
    if (e < P * P) v[i] = buf[(e / P) * LD + (e % P)];
  }
  group_sync<NT>();
#pragma unroll
  for (int i = 0; i < PER; ++i) {
    const int e = gtid<NT>() + i * NT;
    if (e < P * P) buf[(e % P) * LD + (e / P)] = v[i];
  }
  group_sync<NT>();
}

// ---------------------------------------------------------------------------
// 64-point FFTs by groups of 8 lanes.  Lane bits 2..4 are the FFT lane l;
// lane l holds x[l + 8 j], j = 0..7.  64 = 8 x 8: an 8-point DFT over j, the
// twiddles W64^(l k1), an 8 x 8 transpose across the 8 lanes (three xor
// shuffle stages), and an 8-point DFT over l leave X[l + 8 k2] in lane l,
// slot k2.  No shared memory and no barrier inside the transform.
// ---------------------------------------------------------------------------
__device__ __forceinline__ void transpose8_lanes(float2 v[8], int l) {
#pragma unroll
  for (int s = 4; s >= 1; s >>= 1) {
    const bool hi = (l & s) != 0;
#pragma unroll
    for (int m = 0; m < 8; ++m) {
      if (m & s) continue;
      // the lane with bit s clear sends v[m ^ s] and receives into it; its
      // partner sends v[m] and receives into v[m]
      const float2 send = hi ? v[m] : v[m ^ s];
      float2 recv;
      recv.x = __shfl_xor_sync(0xffffffffu, send.x, s << 2);
      recv.y = __shfl_xor_sync(0xffffffffu, send.y, s << 2);
      if (hi) v[m] = recv;
      else v[m ^ s] = recv;
    }
  }
}

template <bool INV>
__device__ __forceinline__ void fft64_lanes(float2 v[8], const float2* tw, int l) {
  dft_small<8, INV>(v);
#pragma unroll
  for (int k = 1; k < 8; ++k) {
    float2 w = tw[l * k];
    if (INV) w.y = -w.y;
    v[k] = cmul(v[k], w);
  }
  transpose8_lanes(v, l);
  dft_small<8, INV>(v);
}

// ---------------------------------------------------------------------------
// Plane transforms.  TWO_D: P x P plane, row stride P + 1 (P + 4 for P = 64,
// which the lane-group engine reads and writes without bank conflicts).
// Otherwise a line of P points (Py = 1).
//
// QUAD (P = 128, TWO_D, ALLOW_QUAD): the planes the operator transforms at
// run time have their spatial support inside 64 x 64 (Ny, Nx <= 64; the
// padding to 128 only keeps the circular convolution linear).  For such a
// plane the 128-point DFT splits by output parity into 64-point DFTs of
// pre-twiddled inputs (W = e^{-2 pi j / 128}):
//   S[2 ky' + py][2 kx' + px] = FFT64x64( s[y][x] W^(py y + px x) )[ky'][kx']
// and the inverse, cropped to 64 x 64, is the sum over the four quadrants
// q = (py, px) of W^-(py y + px x) IFFT64x64(S_q)[y][x].  So a 128 x 128
// transform is four 64 x 64 lane-group transforms through one 64 x 68 buffer
// (36 KB with twiddles: two CTAs per SM instead of one), with the spatial
// plane held in registers between quadrants.  The spectrum is then never
// whole in shared memory: loads and stores go quadrant by quadrant
// (sfs_kernels.cu).  The generator table, whose planes fill 127 x 127, is
// built with the full 128 x 128 engine (ALLOW_QUAD = false).
// ---------------------------------------------------------------------------
template <int P, bool TWO_D, bool ALLOW_QUAD = true>
struct PlaneFFT {
  // 64 x 64 planes use the lane-group engine (512 threads = 64 columns x 8);
  // full 128 x 128 planes (one CTA per SM: the plane takes 129 KB) run 1024
  // threads, quadrant planes 512, and 32 x 32 planes 512 as well, so that
  // every plane the operator transforms at run time takes a 512-thread CTA
  static constexpr bool QUAD = ALLOW_QUAD && TWO_D && P == 128;
  static constexpr bool LANES64 = TWO_D && P == 64;
  static constexpr int LD = QUAD ? 68 : (TWO_D ? (LANES64 ? P + 4 : P + 1) : P);
  static constexpr int NT = QUAD ? 512
                                 : (TWO_D ? (P >= 128 ? 1024 : 512)
                                          : (P >= 512 ? 256 : (P >= 128 ? 128 : 64)));
  static constexpr int ELEMS = QUAD ? 64 * LD : (TWO_D ? P * LD : P);  // float2 slots of the plane
  static constexpr int NTW = QUAD ? P + 64 : P;                         // twiddles (W_P, then W_64)
  // plane + twiddles; QUAD planes also hold a second 64 x 68 buffer after
  // the twiddles (aux), for the half-transformed quadrants
  static constexpr int SMEM = (ELEMS + NTW + (QUAD ? ELEMS : 0)) * 8;
  // resident CTAs per SM the plane kernels are compiled for: two 64 x 64
  // (or quadrant) planes per SM (at most 64 registers a thread) so that
  // batched calls, which launch many planes per scene, keep two planes in
  // flight per SM
  static constexpr int MINB = (LANES64 || QUAD) ? 2 : 1;

  // spatial element (iy, ix) of the plane (QUAD: iy, ix < 64)
  __device__ static __forceinline__ int sidx(int iy, int ix) { return TWO_D ? iy * LD + ix : ix; }
  // QUAD: buffer position of local wavenumber (kx', ky') of a quadrant
  __device__ static __forceinline__ int qidx(int local) { return (local >> 6) * LD + (local & 63); }

  // QUAD forward: the spatial plane in buf (natural layout, zero outside the
  // support) -> for q = 0..3 (py = q >> 1, px = q & 1) the quadrant's
  // spectrum S_q[kx'][ky'] at buf[qidx(kx' 64 + ky')], then store(q).  buf
  // and the aux buffer (tw + NTW) are overwritten; store(q) must only read
  // buf.  The pre-twiddle W^(py y + px x) splits into W^(py y), applied
  // before the transform along y, and W^(px x), which commutes with it and
  // is applied before the transform along x; so the two quadrants of one py
  // share their pass along y: 6 lane-group passes per plane instead of 8.
  template <typename Store>
  __device__ static __forceinline__ void forward_quads(float2* buf, const float2* tw, Store&& store) {
    static_assert(QUAD, "quadrant engine");
    const float2* tw64 = tw + P;
    float2* aux = const_cast<float2*>(tw) + NTW;
    const int lane = threadIdx.x & 31, l = lane >> 2;
    const int c = (gtid<NT>() >> 5) * 4 + (lane & 3);
    float2 s[8];
#pragma unroll
    for (int j = 0; j < 8; ++j) s[j] = buf[(l + 8 * j) * LD + c];  // (y = l + 8 j, x = c)
#pragma unroll 1
    for (int py = 0; py < 2; ++py) {
      float2 v[8];
#pragma unroll
      for (int j = 0; j < 8; ++j) v[j] = py ? cmul(s[j], tw[l + 8 * j]) : s[j];
      // along y for column x = c; written transposed to aux: row x, column ky'
      fft64_lanes<false>(v, tw64, l);
      // (the previous py's reads of aux came before the barriers of its last store)
#pragma unroll
      for (int k = 0; k < 8; ++k) aux[c * LD + l + 8 * k] = v[k];
      group_sync<NT>();
#pragma unroll 1
      for (int px = 0; px < 2; ++px) {
        // along x for column ky' = c (rows x = l + 8 j): kx' = l + 8 k at row kx'
#pragma unroll
        for (int j = 0; j < 8; ++j) {
          const float2 t = aux[(l + 8 * j) * LD + c];
          v[j] = px ? cmul(t, tw[l + 8 * j]) : t;
        }
        fft64_lanes<false>(v, tw64, l);
        group_sync<NT>();  // the spatial reads, or the previous quadrant's store, are done
#pragma unroll
        for (int k = 0; k < 8; ++k) buf[(l + 8 * k) * LD + c] = v[k];
        group_sync<NT>();
        store(2 * py + px);
      }
    }
  }

  // QUAD inverse: for q = 0..3, load(q) fills buf[qidx(kx' 64 + ky')] with
  // S_q (every local position); the cropped 64 x 64 result is left in buf in
  // the natural layout (aux is overwritten).  The post-twiddle
  // W^-(py y + px x) splits as in forward_quads: the two quadrants of one py
  // are transformed along kx', twiddled by W^-(px x) and added in aux, and
  // share one pass along ky' (6 lane-group passes per plane instead of 8).
  template <typename Load>
  __device__ static __forceinline__ void inverse_quads(float2* buf, const float2* tw, Load&& load) {
    static_assert(QUAD, "quadrant engine");
    const float2* tw64 = tw + P;
    float2* aux = const_cast<float2*>(tw) + NTW;
    const int lane = threadIdx.x & 31, l = lane >> 2;
    const int c = (gtid<NT>() >> 5) * 4 + (lane & 3);
    float2 acc[8];
#pragma unroll
    for (int k = 0; k < 8; ++k) acc[k] = make_float2(0.f, 0.f);
#pragma unroll 1
    for (int py = 0; py < 2; ++py) {
      float2 v[8];
#pragma unroll 1
      for (int px = 0; px < 2; ++px) {
        group_sync<NT>();  // earlier readers of buf (and, for px = 0, of aux) are done
        load(2 * py + px);
        group_sync<NT>();
        // along kx' for column ky' = c: x = l + 8 k, added transposed into aux
        // (row ky' = c, column x: slots this thread alone writes)
#pragma unroll
        for (int j = 0; j < 8; ++j) v[j] = buf[(l + 8 * j) * LD + c];
        fft64_lanes<true>(v, tw64, l);
#pragma unroll
        for (int k = 0; k < 8; ++k) {
          float2* a = aux + c * LD + l + 8 * k;
          *a = px ? cadd(*a, cmulc(tw[l + 8 * k], v[k])) : v[k];
        }
      }
      group_sync<NT>();  // aux holds both quadrants of this py
      // along ky' for column x = c: y = l + 8 k
#pragma unroll
      for (int j = 0; j < 8; ++j) v[j] = aux[(l + 8 * j) * LD + c];
      fft64_lanes<true>(v, tw64, l);
#pragma unroll
      for (int k = 0; k < 8; ++k) acc[k] = py ? cadd(acc[k], cmulc(tw[l + 8 * k], v[k])) : v[k];
    }
    // the last reads of buf came before the barrier above
#pragma unroll
    for (int k = 0; k < 8; ++k) buf[(l + 8 * k) * LD + c] = acc[k];
    group_sync<NT>();
  }
  // QUAD, one quadrant q (the cluster kernels, one CTA per quadrant):
  // load(q) fills buf[qidx(kx' 64 + ky')] with S_q; on return this thread's
  //   acc[k] = W^-(py y + px x) IFFT64x64(S_q)[y = l + 8 k][x = c],
  // its share of the cropped inverse.  The thread group of column c last
  // touched buf at rows l + 8 k of column c, so acc may be written back there
  // without a barrier.
  template <typename Load>
  __device__ static __forceinline__ void inverse_quad(float2* buf, const float2* tw, int q, float2 acc[8],
                                                      Load&& load) {
    static_assert(QUAD, "quadrant engine");
    const float2* tw64 = tw + P;
    const int lane = threadIdx.x & 31, l = lane >> 2;
    const int c = (gtid<NT>() >> 5) * 4 + (lane & 3);
    const int py = q >> 1, px = q & 1;
    load(q);
    group_sync<NT>();
    float2 v[8];
#pragma unroll
    for (int j = 0; j < 8; ++j) v[j] = buf[(l + 8 * j) * LD + c];
    group_sync<NT>();
    fft64_lanes<true>(v, tw64, l);
#pragma unroll
    for (int k = 0; k < 8; ++k) buf[c * LD + l + 8 * k] = v[k];
    group_sync<NT>();
#pragma unroll
    for (int j = 0; j < 8; ++j) v[j] = buf[(l + 8 * j) * LD + c];
    fft64_lanes<true>(v, tw64, l);
#pragma unroll
    for (int k = 0; k < 8; ++k) acc[k] = q ? cmulc(tw[py * (l + 8 * k) + px * c], v[k]) : v[k];
  }

  // QUAD, one quadrant q: s[j] = spatial value (y = l + 8 j, x = c), zero
  // outside the support -> S_q at buf[qidx(kx' 64 + ky')].  No thread of the
  // CTA may still read buf when this is called.
  __device__ static __forceinline__ void forward_quad(float2* buf, const float2* tw, int q, const float2 s[8]) {
    static_assert(QUAD, "quadrant engine");
    const float2* tw64 = tw + P;
    const int lane = threadIdx.x & 31, l = lane >> 2;
    const int c = (gtid<NT>() >> 5) * 4 + (lane & 3);
    const int py = q >> 1, px = q & 1;
    float2 v[8];
    // the twiddle in two factors, as forward_quads applies it, so that both
    // produce the same spectra bit for bit
#pragma unroll
    for (int j = 0; j < 8; ++j) v[j] = py ? cmul(s[j], tw[l + 8 * j]) : s[j];
    fft64_lanes<false>(v, tw64, l);
#pragma unroll
    for (int k = 0; k < 8; ++k) buf[c * LD + l + 8 * k] = v[k];
    group_sync<NT>();
#pragma unroll
    for (int j = 0; j < 8; ++j) {
      const float2 t = buf[(l + 8 * j) * LD + c];
      v[j] = px ? cmul(t, tw[l + 8 * j]) : t;
    }
    fft64_lanes<false>(v, tw64, l);
#pragma unroll
    for (int k = 0; k < 8; ++k) buf[(l + 8 * k) * LD + c] = v[k];
    group_sync<NT>();
  }

  // wavenumber kappa (transposed order, kappa = kx*P + ky) of the plane
  __device__ static __forceinline__ int kidx(int kappa) {
    return TWO_D ? (kappa / P) * LD + (kappa % P) : kappa;
  }
  static constexpr int NK = TWO_D ? P * P : P;

  // Forward 2-D FFT; only spatial columns ix < ncols may be nonzero.
  __device__ static __forceinline__ void forward(float2* buf, const float2* tw, int ncols) {
    if constexpr (LANES64) {
      const int lane = threadIdx.x & 31, l = lane >> 2;
      const int c = (gtid<NT>() >> 5) * 4 + (lane & 3);
      float2 v[8];
      // along y for column x = c; written transposed: row x, column ky
#pragma unroll
      for (int j = 0; j < 8; ++j)
        v[j] = c < ncols ? buf[(l + 8 * j) * LD + c] : make_float2(0.f, 0.f);
      group_sync<NT>();
      fft64_lanes<false>(v, tw, l);
#pragma unroll
      for (int k = 0; k < 8; ++k) buf[c * LD + l + 8 * k] = v[k];
      group_sync<NT>();
      // along x for column ky = c: result kx = l + 8 k at row kx (own column only)
#pragma unroll
      for (int j = 0; j < 8; ++j) v[j] = buf[(l + 8 * j) * LD + c];
      fft64_lanes<false>(v, tw, l);
#pragma unroll
      for (int k = 0; k < 8; ++k) buf[(l + 8 * k) * LD + c] = v[k];
      group_sync<NT>();
    } else if constexpr (TWO_D) {
      fft_multi<P, false, NT, P, true>(buf, ncols, LD, 1, tw);   // along y
      transpose_plane<P, LD, NT>(buf);
      fft_multi<P, false, NT, P, true>(buf, P, LD, 1, tw);       // along x
    } else {
      fft_multi<P, false, NT, 1, false>(buf, 1, 1, P, tw);
    }
  }
  // Inverse (unnormalised) 2-D FFT; only spatial columns ix < ncols of the
  // result are computed.
  __device__ static __forceinline__ void inverse(float2* buf, const float2* tw, int ncols) {
    if constexpr (LANES64) {
      const int lane = threadIdx.x & 31, l = lane >> 2;
      const int c = (gtid<NT>() >> 5) * 4 + (lane & 3);
      float2 v[8];
      // along kx for column ky = c; written transposed: row ky, column x
#pragma unroll
      for (int j = 0; j < 8; ++j) v[j] = buf[(l + 8 * j) * LD + c];
      group_sync<NT>();
      fft64_lanes<true>(v, tw, l);
#pragma unroll
      for (int k = 0; k < 8; ++k) buf[c * LD + l + 8 * k] = v[k];
      group_sync<NT>();
      // along ky for column x = c: result y = l + 8 k at row y (own column only)
#pragma unroll
      for (int j = 0; j < 8; ++j) v[j] = buf[(l + 8 * j) * LD + c];
      fft64_lanes<true>(v, tw, l);
      if (c < ncols) {
#pragma unroll
        for (int k = 0; k < 8; ++k) buf[(l + 8 * k) * LD + c] = v[k];
      }
      group_sync<NT>();
    } else if constexpr (TWO_D) {
      fft_multi<P, true, NT, P, true>(buf, P, LD, 1, tw);        // kx -> x
      transpose_plane<P, LD, NT>(buf);
      fft_multi<P, true, NT, P, true>(buf, ncols, LD, 1, tw);    // ky -> y
    } else {
      fft_multi<P, true, NT, 1, false>(buf, 1, 1, P, tw);
    }
  }
};

}  // namespace sfs
