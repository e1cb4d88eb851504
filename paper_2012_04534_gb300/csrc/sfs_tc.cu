// Depth contractions on the tensor cores (tcgen05, Blackwell sm_100 family).
//
// The generator table holds one entry per symmetry orbit of wavenumbers
// (the lateral kernel depends on dx^2 + dy^2 only, Eq. (3)), so the GS slots
// of an orbit share T[u][z] (bin u, depth z) and both contractions of
// Sec. IV-B are small dense products per orbit o, n over the orbit's slots:
//   forward  Y[u][n] = sum_z T[u][z] X[z][n]          M = bins,   K = depths
//   adjoint  G[z][n] = sum_u conj(T[u][z]) R[u][n]    M = depths, K = bins
// In real arithmetic with N = 16 columns (8 real parts, then 8 imaginary
// parts; slots GS..7 of each half are zero):
//   forward  [Yr | Yi] = Tr [Xr | Xi] + Ti [-Xi | Xr]
//   adjoint  [Gr | Gi] = Tr^T [Rr | Ri] + Ti^T [Ri | -Rr]
// Each real product runs as three TF32 products, a_hi b_hi + a_hi b_lo +
// a_lo b_hi, where hi is the value cut to 10 mantissa bits and lo the exact
// remainder (read by the tensor core to 10 mantissa bits); the dropped
// a_lo b_lo and the cut of lo leave at most about 2^-19 relative error per
// product (about 2^-21 on average), against 2^-24 per FP32 rounding.
//
// Per CTA (320 threads, two CTAs per SM, 256 TMEM columns each):
//   warp 8           streams table chunks into shared memory (cp.async.bulk,
//                    one mbarrier per stage, 6 stages of 16 KB);
//   warps 0-7        two warpgroups, one per K-step (8 of the 16) of a chunk;
//                    warp w serves the 32-lane quarter w % 4 of TMEM.  They
//                    read their rows of a chunk, split them and store A_hi /
//                    A_lo in TMEM (tcgen05.st), split the chunk's spectra
//                    into the B operand in shared memory (K-major, no
//                    swizzle), and warpgroup 0 reads a unit's accumulator
//                    (tcgen05.ld) once the next unit's first chunk is queued;
//   warp 9           issues tcgen05.mma (kind::tf32, M = 128, N = 16, K = 8)
//                    and commits to mbarriers that free the chunk buffers and
//                    signal the accumulators (two, alternating by unit).
// The copy and MMA warps run their loops with all 32 lanes and issue from
// one elected lane, with the 12 MMAs of a chunk unrolled on descriptors that
// differ from a per-chunk base by constants: issued that way an N = 16 MMA
// takes about 22 cycles, against 100-250 cycles from a lone divergent lane
// that recomputes its operands (measured on GB300).
// Work: units (orbit, 128-row M tile), a contiguous share per persistent CTA;
// a unit runs over K in chunks of 16 (3 chunk buffers in flight).
//
// Table layout (written by the table build): word
//   T4[((o * nzc + zc) * U + u) * 8 + (j ^ (u & 7))]
//     = (re_2p, re_2p+1, im_2p, im_2p+1),  p = 8 zc + j,
// depth blocks of 16 (nzc = ceil(Nz / 16), missing depths zero).  A forward
// chunk (o, zc) is one contiguous block of rows; an adjoint chunk (16 bins)
// is one block of 16 rows per depth block.  The XOR spreads the 8 words of a
// row over the banks so that loaders reading whole rows do not conflict.
//
// Every mbarrier wait is bounded (wait_ns, 2 s by default).  A timeout sets
// the device error flag and a shared abort flag that ends the other roles'
// waits; the copy thread then waits (bounded) for its copies in flight, the
// MMA thread for its MMAs, and warp 0 frees the TMEM before the CTA exits.
#include <cuda_runtime.h>
#include <stdint.h>

#include <algorithm>

#include "sfs_async.cuh"
#include "sfs_tcgen05.cuh"
#include "sfs_internal.h"
#include "sfs_launch.h"

namespace sfs {
namespace {

// ---------------------------------------------------------------------------
// Shared-memory plan of one CTA
// ---------------------------------------------------------------------------
constexpr int kTcLoaderWarps = 8;         // two warpgroups, one per K-step of a chunk
constexpr int kTcCopyWarp = kTcLoaderWarps, kTcMmaWarp = kTcLoaderWarps + 1;
constexpr int kTcThreads = (kTcLoaderWarps + 2) * 32;
constexpr int kTcStages = 6;               // table stages
constexpr int kTcBufs = 3;                 // chunk buffers (A in TMEM, B in smem)
constexpr int kTcStageBytes = 16384;       // 128 rows x 128 B (fwd) or 8 x 16 rows x 128 B (adj)
constexpr int kTcBBytes = 1536;            // B hi (or lo): 3 groups x 8 rows x 16 K x 4 B
constexpr uint32_t kTcCols = 256;          // TMEM columns per CTA
constexpr uint32_t kTcColD = 0;            // accumulators: 2 x 16 columns
constexpr uint32_t kTcColA = 32;           // chunk buffer b: 64 columns at 32 + 64 b
// barriers: stage full / empty, buffer full / empty, accumulator full /
// empty, MMA drain, and one that nothing arrives at (failure-handling tests)
enum TcBar { kSF = 0, kSE = kSF + kTcStages, kBF = kSE + kTcStages, kBE = kBF + kTcBufs,
             kDF = kBE + kTcBufs, kDE = kDF + 2, kDR = kDE + 2, kNV, kNumTcBars };
constexpr int kTcOffB = kTcStages * kTcStageBytes;
constexpr int kTcOffBar = kTcOffB + kTcBufs * 2 * kTcBBytes;
constexpr int kTcOffSlot = kTcOffBar + kNumTcBars * 8;
constexpr int kTcSmemUsed = kTcOffSlot + 16;
// asking for at least 78 KB keeps a third CTA off the SM (its TMEM
// allocation would have to wait for one of the two resident CTAs to end)
constexpr int kTcSmem = kTcSmemUsed > 78 * 1024 ? kTcSmemUsed : 78 * 1024;
static_assert(kTcColA + 64 * kTcBufs <= kTcCols, "TMEM plan");

template <bool FWD>
__global__ void __launch_bounds__(kTcThreads, 2)
contract_tc(const float4* __restrict__ T4, const float2* __restrict__ Sp,
            float2* __restrict__ out, PlaneDims d, int nmt, int nch, int nunits,
            int* __restrict__ err) {
  extern __shared__ __align__(1024) unsigned char tsm[];
  const float4* stages = (const float4*)tsm;
  float* bbuf = (float*)(tsm + kTcOffB);
  uint32_t* tslot = (uint32_t*)(tsm + kTcOffSlot);
  volatile int* abort_flag = (volatile int*)(tsm + kTcOffSlot + 4);
  const uint32_t bar0 = smem_addr(tsm + kTcOffBar);
  auto bar = [&](int k) { return bar0 + 8u * (uint32_t)k; };
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int G = gridDim.x, b = blockIdx.x;
  const int first = (int)(((long long)nunits * b) / G);
  const int items = ((int)(((long long)nunits * (b + 1)) / G) - first) * nch;
  const uint64_t wait_ns = d.wait_ns;

  if (threadIdx.x == 0) {
    *abort_flag = 0;
    for (int k = 0; k < kTcStages; ++k) {
      mbar_init(bar(kSF + k), 1);
      mbar_init(bar(kSE + k), kTcLoaderWarps);
    }
    for (int k = 0; k < kTcBufs; ++k) {
      mbar_init(bar(kBF + k), kTcLoaderWarps);
      mbar_init(bar(kBE + k), 1);
    }
    for (int k = 0; k < 2; ++k) {
      mbar_init(bar(kDF + k), 1);
      mbar_init(bar(kDE + k), 4);
    }
    mbar_init(bar(kDR), 1);
    mbar_init(bar(kNV), 1);
    fence_mbar_init();
  }
  if (warp == 0) {
    tc_alloc(smem_addr(tslot), kTcCols);
    tc_relinquish();
  }
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  const uint32_t tmem = *tslot;

  if (warp == kTcCopyWarp) {
    // ---- copy producer: table chunks into the stages (whole warp) ----
    int issued = 0;
    bool ok = true;
    int k = 0, c = 0;  // local unit, chunk
    int o = first / nmt, mt = first - (first / nmt) * nmt;
    for (int i = 0; i < items; ++i) {
      const int s = i % kTcStages;
      if (i >= kTcStages) {
        const bool got = tc_wait(bar(kSE + s), ((i / kTcStages) + 1) & 1, wait_ns, abort_flag);
        if (!__all_sync(0xffffffffu, got)) {
          ok = false;
          break;
        }
      }
      const uint32_t dst = smem_addr(tsm + s * kTcStageBytes);
      if (FWD) {  // rows 128 mt .. of depth block c
        const uint32_t bytes = (uint32_t)min(128, d.U - 128 * mt) * 128u;
        if (elect_one()) {
          fence_proxy_async();
          mbar_expect_tx(bar(kSF + s), bytes);
          bulk_g2s(dst, T4 + ((size_t)(o * d.nzc + c) * d.U + 128 * mt) * 8, bytes, bar(kSF + s));
        }
      } else {  // rows 16 c .. of the (up to 8) depth blocks of tile mt, one lane each
        const int nblk = min(8, d.nzc - 8 * mt);
        const uint32_t bytes = (uint32_t)min(16, d.U - 16 * c) * 128u;
        if (lane == 0) {
          fence_proxy_async();
          mbar_expect_tx(bar(kSF + s), bytes * nblk);
        }
        __syncwarp();
        if (lane < nblk)
          bulk_g2s(dst + lane * 2048u, T4 + ((size_t)(o * d.nzc + 8 * mt + lane) * d.U + 16 * c) * 8,
                   bytes, bar(kSF + s));
      }
      __syncwarp();
      ++issued;
      if (++c == nch) {
        c = 0;
        ++k;
        if (++mt == nmt) {
          mt = 0;
          ++o;
        }
      }
    }
    if (!ok && lane == 0) {
      *abort_flag = 1;
      atomicExch(err, 1);
    }
    // copies in flight: the latest use of each stage
    for (int i = max(0, issued - kTcStages); i < issued; ++i)
      mbar_wait_bounded(bar(kSF + i % kTcStages), (i / kTcStages) & 1, kDrainNs);
  } else if (warp == kTcMmaWarp) {
    // ---- MMA issuer (whole warp, one elected lane issues) ----
    constexpr uint32_t idesc = idesc_tf32(128, 16);
    // B rows: forward [-Xi; Xr; Xi], adjoint [Rr; Ri; -Rr] (8 rows each);
    // descriptor offsets in 16-byte units
    constexpr uint64_t o1 = FWD ? 32 : 0, o2 = FWD ? 0 : 32;
    const uint64_t dB0 = smem_desc(smem_addr(bbuf), 128, 512);
    bool ok = true;
    int k = 0, c = 0;
    for (int i = 0; i < items; ++i) {
      const int bf = i % kTcBufs;
      bool got = true;
      // accumulator k & 1 is free once unit k - 2 has been read out
      if (c == 0 && k >= 2) got = tc_wait(bar(kDE + (k & 1)), ((k - 2) >> 1) & 1, wait_ns, abort_flag);
      if (got) got = tc_wait(bar(kBF + bf), (i / kTcBufs) & 1, wait_ns, abort_flag);
      if (!__all_sync(0xffffffffu, got)) {
        ok = false;
        break;
      }
      tc_fence_after();
      const uint32_t D = tmem + kTcColD + 16u * (k & 1);
      const uint32_t a = tmem + kTcColA + 64u * bf;  // Ar_hi, Ar_lo, Ai_hi, Ai_lo
      const uint64_t bh = dB0 + (uint64_t)(bf * (2 * kTcBBytes / 16)), bl = bh + kTcBBytes / 16;
      const uint32_t acc0 = c > 0 ? 1u : 0u;
      if (elect_one()) {
        tc_mma(D, a, bh + o1, idesc, acc0);
        tc_mma(D, a, bl + o1, idesc, 1u);
        tc_mma(D, a + 16, bh + o1, idesc, 1u);
        tc_mma(D, a + 32, bh + o2, idesc, 1u);
        tc_mma(D, a + 32, bl + o2, idesc, 1u);
        tc_mma(D, a + 48, bh + o2, idesc, 1u);
        tc_mma(D, a + 8, bh + o1 + 16, idesc, 1u);
        tc_mma(D, a + 8, bl + o1 + 16, idesc, 1u);
        tc_mma(D, a + 24, bh + o1 + 16, idesc, 1u);
        tc_mma(D, a + 40, bh + o2 + 16, idesc, 1u);
        tc_mma(D, a + 40, bl + o2 + 16, idesc, 1u);
        tc_mma(D, a + 56, bh + o2 + 16, idesc, 1u);
        tc_commit(bar(kBE + bf));
        if (c == nch - 1) tc_commit(bar(kDF + (k & 1)));
      }
      __syncwarp();
      if (++c == nch) {
        c = 0;
        ++k;
      }
    }
    if (!ok && lane == 0) {
      *abort_flag = 1;
      atomicExch(err, 1);
    }
    if (elect_one()) tc_commit(bar(kDR));  // all MMAs of this CTA
    __syncwarp();
    mbar_wait_bounded(bar(kDR), 0, kDrainNs);
  } else {
    // ---- loaders: warps 0-7; thread t of a warpgroup owns TMEM lane t ----
    const int g = warp >> 2;  // warpgroup: K-step g (entries 8 g .. 8 g + 7) of each chunk
    const int t = threadIdx.x & 127;
    const uint32_t tl = tmem + ((uint32_t)(32 * (warp & 3)) << 16);
    // this thread's B element (threads 0-63 of each warpgroup): slot nn, K index kk
    const bool has_b = t < 64;
    const int nn = t & 7, kk = (t >> 3) + 8 * g;
    const int boff = (kk >> 2) * 32 + nn * 4 + (kk & 3);
    // Accumulator of local unit k (buffer k & 1) to the output; false if the
    // wait for its MMAs failed.  Warpgroup 0 only.
    auto epilogue = [&](int k, int o, int mt) -> bool {
      const bool dgot = tc_wait(bar(kDF + (k & 1)), (k >> 1) & 1, wait_ns, abort_flag);
      if (!__all_sync(0xffffffffu, dgot)) return false;
      tc_fence_after();
      uint32_t dv[16];
      tc_ld16(tl + kTcColD + 16u * (k & 1), dv);
      tc_wait_ld();
      tc_fence_before();
      __syncwarp();
      if (lane == 0) mbar_arrive(bar(kDE + (k & 1)));
      if (FWD) {
        const int u = 128 * mt + t;
        if (u < d.U) {
          float2* dst = out + (size_t)u * d.Ns + o * d.GS;
#pragma unroll
          for (int q = 0; q < 8; ++q)
            if (q < d.GS) dst[q] = make_float2(__uint_as_float(dv[q]), __uint_as_float(dv[8 + q]));
        }
      } else {
        const int z = 128 * mt + t;
        if (z < d.Nz) {
          const int s0 = o * d.GS;  // the orbit's slots lie in one tile of 64
          float2* dst = out + (((size_t)(s0 >> 6) * d.anzb + (z >> 5)) * 32 + (z & 31)) * 64 + (s0 & 63);
#pragma unroll
          for (int q = 0; q < 8; ++q)
            if (q < d.GS) dst[q] = make_float2(__uint_as_float(dv[q]), __uint_as_float(dv[8 + q]));
        }
      }
      return true;
    };
    bool ok = true;
    int k = 0, c = 0;  // local unit, chunk
    int o = first / nmt, mt = first - (first / nmt) * nmt;
    int po = o, pmt = mt;  // the previous unit
    int s = 0, bf = 0, sph = 0, bph = 0;  // stage, buffer and their use counts' parity
    // Spectra value of this thread's B element in chunk cc of orbit oo (the
    // same for every M tile).  It is loaded one item ahead, so that its L2
    // latency overlaps the previous chunk's work.
    auto load_sv = [&](int oo, int cc) -> float2 {
      float2 v = make_float2(0.f, 0.f);
      if (has_b && nn < d.GS) {
        const int r = 16 * cc + kk;  // depth (forward) or bin (adjoint)
        if (r < (FWD ? d.Nz : d.U)) v = Sp[(size_t)r * d.Ns + oo * d.GS + nn];
      }
      return v;
    };
    pdl_wait();
    float2 sv_next = items > 0 ? load_sv(o, c) : make_float2(0.f, 0.f);
    for (int i = 0; i < items; ++i) {
      const float2 sv = sv_next;
      if (i + 1 < items) {
        const bool wrap = c + 1 == nch;
        sv_next = load_sv(wrap && mt + 1 == nmt ? o + 1 : o, wrap ? 0 : c + 1);
      }
      const bool got = (d.inject && i == 0) ? tc_wait(bar(kNV), 0, wait_ns, abort_flag)
                                            : tc_wait(bar(kSF + s), sph, wait_ns, abort_flag);
      if (!__all_sync(0xffffffffu, got)) {
        ok = false;
        break;
      }
      float ar[8], ai[8];  // K entries 8 g .. 8 g + 7 of this thread's row
      const float4* st4 = stages + s * (kTcStageBytes / 16);
      if (FWD) {
        const bool valid = t < d.U - 128 * mt;
#pragma unroll
        for (int j = 0; j < 4; ++j) {
          const int jj = 4 * g + j;
          const float4 w = valid ? st4[t * 8 + (jj ^ (t & 7))] : make_float4(0.f, 0.f, 0.f, 0.f);
          ar[2 * j] = w.x;
          ar[2 * j + 1] = w.y;
          ai[2 * j] = w.z;
          ai[2 * j + 1] = w.w;
        }
      } else {
        const int nu = min(16, d.U - 16 * c);
        const bool zv = 128 * mt + t < d.Nz;
        const int zcl = t >> 4, j = (t & 15) >> 1;
        const bool odd = t & 1;
#pragma unroll
        for (int ul = 0; ul < 8; ++ul) {
          const int ur = 8 * g + ul;
          const float4 w = (zv && ur < nu) ? st4[(zcl * 16 + ur) * 8 + (j ^ (ur & 7))]
                                           : make_float4(0.f, 0.f, 0.f, 0.f);
          ar[ul] = odd ? w.y : w.x;
          ai[ul] = odd ? w.w : w.z;
        }
      }
      __syncwarp();
      if (lane == 0) mbar_arrive(bar(kSE + s));
      if (i >= kTcBufs) {
        const bool free_ok = tc_wait(bar(kBE + bf), bph ^ 1, wait_ns, abort_flag);
        if (!__all_sync(0xffffffffu, free_ok)) {
          ok = false;
          break;
        }
      }
      if (has_b) {  // B operand element, three row groups, hi and lo
        uint32_t* bh = (uint32_t*)(bbuf + (2 * bf) * (kTcBBytes / 4));
        uint32_t* bl = bh + kTcBBytes / 4;
        const float v0 = FWD ? -sv.y : sv.x, v1 = FWD ? sv.x : sv.y, v2 = FWD ? sv.y : -sv.x;
        uint32_t h0, l0, h1, l1, h2, l2;
        tf32_split(v0, h0, l0);
        tf32_split(v1, h1, l1);
        tf32_split(v2, h2, l2);
        bh[boff] = h0;
        bl[boff] = l0;
        bh[128 + boff] = h1;
        bl[128 + boff] = l1;
        bh[256 + boff] = h2;
        bl[256 + boff] = l2;
        fence_proxy_async();
      }
      {  // this K-step's A columns into TMEM: Ar_hi, Ar_lo, Ai_hi, Ai_lo at +0, 16, 32, 48
        uint32_t h[8], l[8];
        const uint32_t ca = tl + kTcColA + 64u * bf + 8u * g;
#pragma unroll
        for (int q = 0; q < 8; ++q) tf32_split(ar[q], h[q], l[q]);
        tc_st8(ca, h);
        tc_st8(ca + 16, l);
#pragma unroll
        for (int q = 0; q < 8; ++q) tf32_split(ai[q], h[q], l[q]);
        tc_st8(ca + 32, h);
        tc_st8(ca + 48, l);
        tc_wait_st();
      }
      tc_fence_before();
      __syncwarp();
      if (lane == 0) mbar_arrive(bar(kBF + bf));
      // the previous unit's accumulator, now that this unit's first chunk is queued
      if (g == 0 && c == 0 && k >= 1 && !epilogue(k - 1, po, pmt)) {
        ok = false;
        break;
      }
      if (++s == kTcStages) {
        s = 0;
        sph ^= 1;
      }
      if (++bf == kTcBufs) {
        bf = 0;
        bph ^= 1;
      }
      if (++c == nch) {
        c = 0;
        ++k;
        po = o;
        pmt = mt;
        if (++mt == nmt) {
          mt = 0;
          ++o;
        }
      }
    }
    if (g == 0 && ok && items > 0 && !epilogue(k - 1, po, pmt)) ok = false;
    if (!ok && lane == 0) {
      *abort_flag = 1;
      atomicExch(err, 1);
    }
  }
  pdl_trigger();
  tc_fence_before();
  __syncthreads();
  if (warp == 0) {
    tc_fence_after();
    tc_dealloc(tmem, kTcCols);
  }
}

template <bool FWD>
int launch_tc(const PlaneDims& d, const float2* table, const float2* Sp, float2* out, int* err,
              cudaStream_t st) {
  SFS_TRY(ensure_smem_attr(contract_tc<FWD>, kTcSmem));
  const int nmt = FWD ? (d.U + 127) / 128 : (d.Nz + 127) / 128;
  const int nch = FWD ? d.nzc : (d.U + 15) / 16;
  const int nunits = (d.Ns / d.GS) * nmt;
  const int G = std::min(d.G, nunits);
  if (G <= 0) return SFS_OK;
  return launch_pdl(contract_tc<FWD>, dim3(G), dim3(kTcThreads), (size_t)kTcSmem, st,
                    (const float4*)table, Sp, out, d, nmt, nch, nunits, err);
}

}  // namespace

int launch_contract_fwd_tc(const PlaneDims& d, const float2* table, const float2* Xh,
                           float2* Yp, int* err, cudaStream_t st) {
  return launch_tc<true>(d, table, Xh, Yp, err, st);
}

int launch_contract_adj_tc(const PlaneDims& d, const float2* table, const float2* Rh,
                           float2* Gs, int* err, cudaStream_t st) {
  return launch_tc<false>(d, table, Rh, Gs, err, st);
}

int prepare_tc_kernels() {
  SFS_TRY(ensure_smem_attr(contract_tc<true>, kTcSmem));
  return ensure_smem_attr(contract_tc<false>, kTcSmem);
}

}  // namespace sfs
