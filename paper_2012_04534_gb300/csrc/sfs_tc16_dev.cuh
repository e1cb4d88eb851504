// Device code of the 16-bit tensor-core contractions (see sfs_tc16.cu for
// the design): TMA and MMA helpers, the shared-memory plan of a CTA and the
// contraction of a range of units by one CTA.  In an unnamed namespace, so
// each file that includes it compiles its own copy.
#pragma once

#include <cuda.h>
#include <cuda_bf16.h>
#include <cuda_fp16.h>
#include <cuda_runtime.h>
#include <stdint.h>

#include "sfs_async.cuh"
#include "sfs_internal.h"
#include "sfs_tcgen05.cuh"

namespace sfs {
namespace {

// ---------------------------------------------------------------------------
// Device helpers
// ---------------------------------------------------------------------------
__device__ __forceinline__ void tma_load_4d(uint32_t dst, const CUtensorMap* map, int c0, int c1, int c2,
                                            int c3, uint32_t bar) {
  asm volatile(
      "cp.async.bulk.tensor.4d.shared::cluster.global.tile.mbarrier::complete_tx::bytes"
      " [%0], [%1, {%2, %3, %4, %5}], [%6];" ::"r"(dst),
      "l"((uint64_t)map), "r"(c0), "r"(c1), "r"(c2), "r"(c3), "r"(bar)
      : "memory");
}
// The same with an L2 cache policy (evict-first for a table larger than L2).
__device__ __forceinline__ void tma_load_4d_hint(uint32_t dst, const CUtensorMap* map, int c0, int c1, int c2,
                                                 int c3, uint32_t bar, uint64_t policy) {
  asm volatile(
      "cp.async.bulk.tensor.4d.shared::cluster.global.tile.mbarrier::complete_tx::bytes.L2::cache_hint"
      " [%0], [%1, {%2, %3, %4, %5}], [%6], %7;" ::"r"(dst),
      "l"((uint64_t)map), "r"(c0), "r"(c1), "r"(c2), "r"(c3), "r"(bar), "l"(policy)
      : "memory");
}
__device__ __forceinline__ void tma_load_table(uint32_t dst, const CUtensorMap* map, int c0, int c1, int c2,
                                               int c3, uint32_t bar, bool stream, uint64_t policy) {
  if (stream)
    tma_load_4d_hint(dst, map, c0, c1, c2, c3, bar, policy);
  else
    tma_load_4d(dst, map, c0, c1, c2, c3, bar);
}
__device__ __forceinline__ void tma_load_3d(uint32_t dst, const CUtensorMap* map, int c0, int c1, int c2,
                                            uint32_t bar) {
  asm volatile(
      "cp.async.bulk.tensor.3d.shared::cluster.global.tile.mbarrier::complete_tx::bytes"
      " [%0], [%1, {%2, %3, %4}], [%5];" ::"r"(dst),
      "l"((uint64_t)map), "r"(c0), "r"(c1), "r"(c2), "r"(bar)
      : "memory");
}
__device__ __forceinline__ void tma_load_2d(uint32_t dst, const CUtensorMap* map, int c0, int c1,
                                            uint32_t bar) {
  asm volatile(
      "cp.async.bulk.tensor.2d.shared::cluster.global.tile.mbarrier::complete_tx::bytes"
      " [%0], [%1, {%2, %3}], [%4];" ::"r"(dst),
      "l"((uint64_t)map), "r"(c0), "r"(c1), "r"(bar)
      : "memory");
}

// Shared-memory matrix descriptor, 128-byte swizzle (layout type 2),
// descriptor version 1.  K-major: sbo = stride between 8-row groups (lbo
// unused); MN-major: lbo = stride between 64-element column blocks, sbo =
// stride between 8-row K groups.
__device__ __forceinline__ uint64_t desc_sw128(uint32_t addr, uint32_t lbo, uint32_t sbo) {
  return (uint64_t)((addr & 0x3FFFFu) >> 4) | ((uint64_t)((lbo & 0x3FFFFu) >> 4) << 16) |
         ((uint64_t)((sbo & 0x3FFFFu) >> 4) << 32) | ((uint64_t)1 << 46) | ((uint64_t)2 << 61);
}
// Instruction descriptor of kind::f16: D f32, A and B both bf16 (f16 =
// false) or both f16, B K-major, A K-major (forward) or MN-major (adjoint).
__host__ __device__ constexpr uint32_t idesc_16(int M, int N, bool a_mn_major, bool f16) {
  return (1u << 4) | (f16 ? 0u : (1u << 7) | (1u << 10)) | ((a_mn_major ? 1u : 0u) << 15) |
         ((uint32_t)(N >> 3) << 17) | ((uint32_t)(M >> 4) << 24);
}
// D[tmem] (+)= A[smem] * B[smem]^T
__device__ __forceinline__ void mma_bf16_ss(uint32_t d, uint64_t adesc, uint64_t bdesc, uint32_t idesc,
                                            uint32_t accumulate) {
  asm volatile(
      "{\n .reg .pred p;\n setp.ne.b32 p, %4, 0;\n"
      " tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n}" ::"r"(d),
      "l"(adesc), "l"(bdesc), "r"(idesc), "r"(accumulate)
      : "memory");
}

// Two values as a 16-bit pair (low half first): their roundings (lo =
// false) or the roundings of what those leave (lo = true), in FP16 (f16) or
// BF16.
__device__ __forceinline__ uint32_t pair16_part(float v0, float v1, bool lo, bool f16) {
  if (f16) {
    __half2 h = __floats2half2_rn(v0, v1);
    if (lo) h = __floats2half2_rn(v0 - __low2float(h), v1 - __high2float(h));
    return *reinterpret_cast<uint32_t*>(&h);
  }
  __nv_bfloat162 h = __floats2bfloat162_rn(v0, v1);
  if (lo) h = __floats2bfloat162_rn(v0 - __low2float(h), v1 - __high2float(h));
  return *reinterpret_cast<uint32_t*>(&h);
}

// 2^k for -126 <= k <= 127, exactly
__device__ __forceinline__ float pow2f(int k) { return __uint_as_float((uint32_t)(k + 127) << 23); }

// ---------------------------------------------------------------------------
// Shared-memory plan of one CTA
// ---------------------------------------------------------------------------
constexpr int kHThreads = 224;  // warps 0-3 build B and read out, 4 table copies, 5 MMA,
                                // 6 spectra copies
constexpr int kHCopyWarp = 4, kHMmaWarp = 5, kHSpecWarp = 6;
constexpr int kHATile = 16384;  // A tile of one part: 128 rows x 128 B (or 2 x 64 rows)
constexpr int kHBTile = 4096;   // B of one scene: 32 rows (16 hi, 16 lo) x 64 K x 2 B, swizzled
constexpr int kHSTile = 4096;   // spectra tile of one scene: 32 depths x 64 B (fwd), 64 bins x 64 B (adj)

// NB = scenes sharing a table tile (batched calls): B has 32 NB columns, the
// accumulators 2 x 32 NB TMEM columns.  NB = 1 runs two CTAs per SM, NB > 1
// one CTA per SM with deeper rings.
template <int NP, int NB>
struct HPlan {
  // Three rings, each with its own producer: the table ring (kST stages of
  // NP A tiles, filled by TMA), the spectra ring (kSS slots of spectra
  // tiles, filled by TMA, emptied by the builders once read) and the B ring
  // (kSBB slots of B operands, built by the builders, emptied by the MMAs).
  // The spectra ring is deep so that the spectra copies, which queue behind
  // the table stream, land well before the builders need them.
  static constexpr int kCtasPerSm = NB == 1 ? 2 : 1;
  static constexpr int kST = NB == 1 ? (NP == 1 ? 4 : 2) : (NP == 1 ? 6 : 3);
  static constexpr int kSS = NB == 1 ? 8 : 4;
  static constexpr int kSBB = 3;
  static constexpr int kLead = 2;  // the builders read out a unit at chunk kLead of the next
  static constexpr int kTStage = NP * kHATile;
  static constexpr int kBSlot = NB * kHBTile;
  static constexpr int kSSlot = NB * kHSTile;
  static constexpr uint32_t kCols = 64 * NB;           // two accumulators of 32 NB columns
  static constexpr int kOffB = kST * kTStage;          // B ring (1 KB aligned)
  static constexpr int kOffS = kOffB + kSBB * kBSlot;   // spectra ring
  // barriers: table full / empty, spectra full / empty, B built / empty,
  // accumulator full / empty, MMA drain, one that nothing arrives at
  // (failure-handling tests)
  static constexpr int kTF = 0, kTE = kST, kXF = 2 * kST, kXE = kXF + kSS, kBF = kXE + kSS,
                       kBE = kBF + kSBB, kDF = kBE + kSBB, kDE = kDF + 2, kDR = kDE + 2, kNV = kDR + 1,
                       kNumBars = kNV + 1;
  static constexpr int kOffBar = kOffS + kSS * kSSlot;
  // TMEM address (0), abort flag (4), FP16 scales 2^ks of the group's scenes
  // (16 + 4 j) and their inverses (32 + 4 j), per-warp maxima (48 + 16 w + 4 j)
  static constexpr int kOffSlot = kOffBar + kNumBars * 8;
  static constexpr int kSmem = kOffSlot + 128 + 1024;  // + alignment of the base to 1 KB
  static_assert(kSmem <= (NB == 1 ? 115 * 1024 : 227 * 1024), "shared memory plan");
};

// out: output of the group's first scene; scene j of the group writes
// out + j * out_stride if j < nscene.
// Units first .. first + nu - 1 of one contraction (a unit is (orbit, tile
// mt), nch chunks each) by the calling CTA, whose dynamic shared memory
// starts at hsm_raw.  Warps 0-6 take the roles above; further warps of a
// larger CTA only pass the CTA barriers at the start and the end.  The
// tensor memory is freed before it returns.  With `reuse` (a CTA that runs
// it again on other units) the roles also wait for the MMAs' last releases
// of the table stages and B slots, so that no arrival is still on its way,
// and the mbarriers are invalidated before the shared memory is used again.
template <bool FWD, int NP, int NB>
__device__ __forceinline__ void contract_h_run(const CUtensorMap* tab, const CUtensorMap* spec,
                                               float2* __restrict__ out, long long out_stride, int nscene,
                                               const PlaneDims& d, int nmt, int nch, int first, int nu,
                                               const float* __restrict__ pm, int* __restrict__ err,
                                               unsigned char* hsm_raw, bool reuse = false) {
  using Pl = HPlan<NP, NB>;
  constexpr uint32_t kHCols = Pl::kCols;
  constexpr int ST = Pl::kST, SS = Pl::kSS, SBB = Pl::kSBB, LEAD = Pl::kLead;
  // 128-byte-swizzled tiles need 1 KB alignment of the shared-memory address
  unsigned char* hsm = hsm_raw + ((1024u - (smem_addr(hsm_raw) & 1023u)) & 1023u);
  const uint32_t sbase = smem_addr(hsm);
  uint32_t* tslot = (uint32_t*)(hsm + Pl::kOffSlot);
  volatile int* abort_flag = (volatile int*)(hsm + Pl::kOffSlot + 4);
  const uint32_t bar0 = sbase + Pl::kOffBar;
  auto bar = [&](int k) { return bar0 + 8u * (uint32_t)k; };
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int items = nu * nch;
  const uint64_t wait_ns = d.wait_ns;
  const int No = d.Ns / d.GS;
  // item j of this CTA: unit first + j / nch = (orbit o, tile mt), chunk c
  auto item = [&](int j, int& o, int& mt, int& c) {
    const int unit = first + j / nch;
    c = j - (j / nch) * nch;
    o = unit / nmt;
    mt = unit - o * nmt;
  };

  if (threadIdx.x == 0) {
    *abort_flag = 0;
    for (int k = 0; k < ST; ++k) {
      mbar_init(bar(Pl::kTF + k), 1);
      mbar_init(bar(Pl::kTE + k), 1);
    }
    for (int k = 0; k < SS; ++k) {
      mbar_init(bar(Pl::kXF + k), 1);
      mbar_init(bar(Pl::kXE + k), 4);
    }
    for (int k = 0; k < SBB; ++k) {
      mbar_init(bar(Pl::kBF + k), 4);
      mbar_init(bar(Pl::kBE + k), 1);
    }
    for (int k = 0; k < 2; ++k) {
      mbar_init(bar(Pl::kDF + k), 1);
      mbar_init(bar(Pl::kDE + k), 4);
    }
    mbar_init(bar(Pl::kDR), 1);
    mbar_init(bar(Pl::kNV), 1);
    fence_mbar_init();
  }
  if (warp == 0) {
    tc_alloc(smem_addr(tslot), kHCols);
    // a CTA that allocates again later keeps its permit (allocating after
    // relinquishing it is illegal)
    if (!reuse) tc_relinquish();
  }
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  const uint32_t tmem = *tslot;

  if (warp == kHSpecWarp) {
    // ---- spectra producer: the spectra tile of item j into slot j % SS ----
    int issued = 0;
    bool ok = true;
    pdl_wait();  // the spectra come from the previous kernel
    for (int j = 0; j < items; ++j) {
      const int sl = j % SS;
      if (j >= SS) {
        const bool got = tc_wait(bar(Pl::kXE + sl), ((j / SS) + 1) & 1, wait_ns, abort_flag);
        if (!__all_sync(0xffffffffu, got)) {
          ok = false;
          break;
        }
      }
      int o, mt, c;
      item(j, o, mt, c);
      if (elect_one()) {
        const uint32_t fb = bar(Pl::kXF + sl);
        mbar_expect_tx(fb, NB * (FWD ? 2048 : 4096));
        tma_load_3d(sbase + Pl::kOffS + sl * Pl::kSSlot, spec, 2 * o * d.GS, (FWD ? 32 : 64) * c, 0, fb);
      }
      __syncwarp();
      ++issued;
    }
    if (!ok && lane == 0) {
      *abort_flag = 1;
      atomicExch(err, 1);
    }
    for (int j = max(0, issued - SS); j < issued; ++j)
      mbar_wait_bounded(bar(Pl::kXF + j % SS), (j / SS) & 1, kDrainNs);
  } else if (warp == kHCopyWarp) {
    // ---- table producer: the table tile(s) of item i into stage i % ST ----
    int issued = 0;
    bool ok = true;
    for (int i = 0; i < items; ++i) {
      const int s = i % ST;
      if (i >= ST) {
        const bool got = tc_wait(bar(Pl::kTE + s), ((i / ST) + 1) & 1, wait_ns, abort_flag);
        if (!__all_sync(0xffffffffu, got)) {
          ok = false;
          break;
        }
      }
      int o, mt, c;
      item(i, o, mt, c);
      if (elect_one()) {
        const uint32_t dst = sbase + (uint32_t)(s * Pl::kTStage), fb = bar(Pl::kTF + s);
        const bool stream = d.stream_table != 0;
        const uint64_t pol = stream ? l2_evict_first_policy() : 0ull;
        mbar_expect_tx(fb, NP * kHATile);
        if (FWD) {  // bins 128 mt .., depth block c
#pragma unroll
          for (int p = 0; p < NP; ++p)
            tma_load_table(dst + p * kHATile, tab, 0, 128 * mt, c, p * No + o, fb, stream, pol);
        } else {  // bins 64 c .., depth blocks 2 mt and 2 mt + 1
#pragma unroll
          for (int p = 0; p < NP; ++p) {
            tma_load_table(dst + p * kHATile, tab, 0, 64 * c, 2 * mt, p * No + o, fb, stream, pol);
            tma_load_table(dst + p * kHATile + 8192, tab, 0, 64 * c, 2 * mt + 1, p * No + o, fb, stream,
                           pol);
          }
        }
      }
      __syncwarp();
      ++issued;
    }
    if (!ok && lane == 0) {
      *abort_flag = 1;
      atomicExch(err, 1);
    }
    // copies in flight: the latest use of each stage
    for (int i = max(0, issued - ST); i < issued; ++i)
      mbar_wait_bounded(bar(Pl::kTF + i % ST), (i / ST) & 1, kDrainNs);
    // and the MMAs' release of those stages (their commits), so that nothing
    // arrives on a barrier after the barriers are invalidated
    if (reuse && ok)
      for (int i = max(0, issued - ST); i < issued; ++i)
        mbar_wait_bounded(bar(Pl::kTE + i % ST), (i / ST) & 1, kDrainNs);
  } else if (warp == kHMmaWarp) {
    // ---- MMA issuer (whole warp, one elected lane issues) ----
    const uint32_t idesc = d.f16 ? idesc_16(128, 32 * NB, !FWD, true) : idesc_16(128, 32 * NB, !FWD, false);
    bool ok = true;
    int k = 0, c = 0;
    for (int i = 0; i < items; ++i) {
      const int s = i % ST, sl = i % SBB;
      bool got = true;
      // accumulator k & 1 is free once unit k - 2 has been read out
      if (c == 0 && k >= 2) got = tc_wait(bar(Pl::kDE + (k & 1)), ((k - 2) >> 1) & 1, wait_ns, abort_flag);
      if (got) got = tc_wait(bar(Pl::kBF + sl), (i / SBB) & 1, wait_ns, abort_flag);
      if (got) got = tc_wait(bar(Pl::kTF + s), (i / ST) & 1, wait_ns, abort_flag);
      if (!__all_sync(0xffffffffu, got)) {
        ok = false;
        break;
      }
      tc_fence_after();
      const uint32_t D = tmem + 32u * NB * (uint32_t)(k & 1);
      const uint32_t a0 = sbase + (uint32_t)(s * Pl::kTStage);
      const uint32_t b0 = sbase + (uint32_t)(Pl::kOffB + sl * Pl::kBSlot);
      if (elect_one()) {
#pragma unroll
        for (int ks = 0; ks < 4; ++ks)
#pragma unroll
          for (int p = 0; p < NP; ++p) {
            const uint64_t ad = FWD ? desc_sw128(a0 + p * kHATile + 32 * ks, 16, 1024)
                                    : desc_sw128(a0 + p * kHATile + 2048 * ks, 8192, 1024);
            const uint64_t bd = desc_sw128(b0 + 32 * ks, 16, 1024);
            mma_bf16_ss(D, ad, bd, idesc, (c > 0 || ks > 0 || p > 0) ? 1u : 0u);
          }
        tc_commit(bar(Pl::kTE + s));
        tc_commit(bar(Pl::kBE + sl));
        if (c == nch - 1) tc_commit(bar(Pl::kDF + (k & 1)));
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
    if (elect_one()) tc_commit(bar(Pl::kDR));  // all MMAs of this CTA
    __syncwarp();
    mbar_wait_bounded(bar(Pl::kDR), 0, kDrainNs);
  } else if (warp < 4) {
    // ---- B builders and epilogue: warps 0-3, thread t owns TMEM lane t ----
    const int t = threadIdx.x;
    const uint32_t tl = tmem + ((uint32_t)(32 * warp) << 16);
    // this thread's B row n (0-15 hi, 16-31 lo; column n & 15: slot n & 7,
    // re for n & 15 < 8, im otherwise) and K range 16 cq .. 16 cq + 15
    const int n = t >> 2, cq = t & 3;
    const bool lo = n >= 16;
    const int nc = n & 15, sl8 = nc & 7;
    const bool slot_ok = sl8 < d.GS;
    const bool f16 = d.f16 != 0;
    float* scl = (float*)(hsm + Pl::kOffSlot + 16);   // [NB] 2^ks
    float* iscl = (float*)(hsm + Pl::kOffSlot + 32);  // [NB] 2^-ks
    if (f16) {
      // scale of scene j of the group from the per-plane maxima of its spectra
      float* wmax = (float*)(hsm + Pl::kOffSlot + 48);
      const int pm_n = FWD ? d.Nz : d.U;
      const long long pm_stride = FWD ? d.bs_pmx : d.bs_pmr;
      pdl_wait();  // the maxima come from the previous kernel
#pragma unroll
      for (int j = 0; j < NB; ++j) {
        float m = 0.0f;
        if (pm && j < nscene)
          for (int i = t; i < pm_n; i += 128) m = fmaxf(m, pm[j * pm_stride + i]);
#pragma unroll
        for (int off = 16; off > 0; off >>= 1) m = fmaxf(m, __shfl_xor_sync(0xffffffffu, m, off));
        if (lane == 0) wmax[4 * warp + j] = m;
      }
      asm volatile("bar.sync 1, 128;" ::: "memory");
      if (t < NB) {
        const float m = fmaxf(fmaxf(wmax[t], wmax[4 + t]), fmaxf(wmax[8 + t], wmax[12 + t]));
        int ks = 0;
        if (m > 0.0f && m <= 3.4e38f) {  // zero, infinite or NaN maxima keep scale 1
          const int e = (int)((__float_as_uint(m) >> 23) & 0xffu) - 127;  // floor(log2 m), -127 if subnormal
          ks = min(126, max(-126, 13 - e));
        }
        scl[t] = pow2f(ks);
        iscl[t] = pow2f(-ks);
      }
      asm volatile("bar.sync 1, 128;" ::: "memory");
    }
    // accumulator of local unit k to the output; false if the wait for its
    // MMAs failed
    auto epilogue = [&](int k) -> bool {
      int o, mt, c;
      item(k * nch, o, mt, c);
      const bool dgot = tc_wait(bar(Pl::kDF + (k & 1)), (k >> 1) & 1, wait_ns, abort_flag);
      if (!__all_sync(0xffffffffu, dgot)) return false;
      tc_fence_after();
#pragma unroll 1
      for (int j = 0; j < NB; ++j) {
      uint32_t v[32];
      uint32_t(&v0)[16] = *reinterpret_cast<uint32_t(*)[16]>(v);
      uint32_t(&v1)[16] = *reinterpret_cast<uint32_t(*)[16]>(v + 16);
      const uint32_t col = 32u * NB * (uint32_t)(k & 1) + 32u * j;
      tc_ld16(tl + col, v0);
      tc_ld16(tl + col + 16, v1);
      tc_wait_ld();
      if (j == NB - 1) {
        tc_fence_before();
        __syncwarp();
        if (lane == 0) mbar_arrive(bar(Pl::kDE + (k & 1)));
      }
      float e[16];
#pragma unroll
      for (int q = 0; q < 16; ++q) e[q] = __uint_as_float(v[q]) + __uint_as_float(v[16 + q]);
      if (f16) {  // undo 2^ks and 2^kT (two exact multiplies)
        const float is = iscl[j];
#pragma unroll
        for (int q = 0; q < 16; ++q) e[q] = (e[q] * is) * d.tinv;
      }
      float2* outj = out + j * out_stride;
      if (FWD) {
        const int u = 128 * mt + t;
        if (u < d.U && j < nscene) {
          float2* dst = outj + (size_t)u * d.Ns + o * d.GS;
#pragma unroll
          for (int q = 0; q < 8; ++q)
            if (q < d.GS) dst[q] = make_float2(e[q], e[8 + q]);
        }
      } else {
        // lane pair (2 zz, 2 zz + 1) holds the Re and Im table rows of depth zz
        float f[16];
#pragma unroll
        for (int q = 0; q < 16; ++q) f[q] = __shfl_xor_sync(0xffffffffu, e[q], 1);
        const int z = 32 * (2 * mt + (t >> 6)) + ((t & 63) >> 1);
        if ((t & 1) == 0 && z < d.Nz && j < nscene) {
          const int s0 = o * d.GS;  // the orbit's slots lie in one tile of 64
          float2* dst = outj + (((size_t)(s0 >> 6) * d.anzb + (z >> 5)) * 32 + (z & 31)) * 64 + (s0 & 63);
#pragma unroll
          for (int q = 0; q < 8; ++q)
            if (q < d.GS) dst[q] = make_float2(e[q] + f[8 + q], e[8 + q] - f[q]);
        }
      }
      }
      return true;
    };
    // a unit's accumulator is read out while the builders are at chunk ce of
    // the next unit, by when the MMAs of the unit have usually completed
    const int ce = min(LEAD, nch - 1);
    bool ok = true;
    int k = 0, c = 0;  // local unit, chunk
    for (int i = 0; i < items; ++i) {
      const int xs = i % SS, sl = i % SBB;
      bool got = (d.inject && i == 0) ? tc_wait(bar(Pl::kNV), 0, wait_ns, abort_flag)
                                      : tc_wait(bar(Pl::kXF + xs), (i / SS) & 1, wait_ns, abort_flag);
      // the B slot is free once the MMAs of item i - SBB are done
      if (got && i >= SBB) got = tc_wait(bar(Pl::kBE + sl), ((i / SBB) + 1) & 1, wait_ns, abort_flag);
      if (!__all_sync(0xffffffffu, got)) {
        ok = false;
        break;
      }
#pragma unroll 1
      for (int jn = 0; jn < NB; ++jn) {
      const float* sp = (const float*)(hsm + Pl::kOffS + xs * Pl::kSSlot + jn * (FWD ? 2048 : 4096));
      const float sc = f16 ? scl[jn] : 1.0f;
      uint32_t w[8];
#pragma unroll
      for (int j = 0; j < 8; ++j) {
        float v0, v1;
        if (FWD) {  // K index 2 zz + q, zz = 8 cq + j
          const float2 x = *(const float2*)(sp + (8 * cq + j) * 16 + 2 * sl8);
          v0 = nc < 8 ? x.x : x.y;
          v1 = nc < 8 ? -x.y : x.x;
        } else {  // K index = bin 16 cq + 2 j (+1)
          const int ub = 16 * cq + 2 * j, comp = nc < 8 ? 0 : 1;
          v0 = sp[ub * 16 + 2 * sl8 + comp];
          v1 = sp[(ub + 1) * 16 + 2 * sl8 + comp];
        }
        if (!slot_ok) v0 = v1 = 0.f;
        w[j] = pair16_part(v0 * sc, v1 * sc, lo, f16);
      }
      // rows 32 jn .. of the B slot (a multiple of 8, so the swizzle phase is n & 7)
      unsigned char* brow = hsm + Pl::kOffB + sl * Pl::kBSlot + (32 * jn + n) * 128;
      *(uint4*)(brow + (((2 * cq) ^ (n & 7)) << 4)) = make_uint4(w[0], w[1], w[2], w[3]);
      *(uint4*)(brow + (((2 * cq + 1) ^ (n & 7)) << 4)) = make_uint4(w[4], w[5], w[6], w[7]);
      }
      __syncwarp();
      if (lane == 0) mbar_arrive(bar(Pl::kXE + xs));  // spectra slot read
      fence_proxy_async();
      __syncwarp();
      if (lane == 0) mbar_arrive(bar(Pl::kBF + sl));
      if (c == ce && k >= 1 && !epilogue(k - 1)) {
        ok = false;
        break;
      }
      if (++c == nch) {
        c = 0;
        ++k;
      }
    }
    if (ok && items > 0 && !epilogue(k - 1)) ok = false;
    if (!ok && lane == 0) {
      *abort_flag = 1;
      atomicExch(err, 1);
    }
    // the MMAs' release of the last B slots (their commits), as above
    if (reuse && ok)
      for (int i = max(0, items - SBB); i < items; ++i)
        mbar_wait_bounded(bar(Pl::kBE + i % SBB), (i / SBB) & 1, kDrainNs);
  }
  pdl_trigger();
  tc_fence_before();
  __syncthreads();
  if (warp == 0) {
    tc_fence_after();
    tc_dealloc(tmem, kHCols);
  }
  if (reuse) {
    if (threadIdx.x == 0)  // every copy, MMA and release has completed: nothing arrives any more
      for (int k = 0; k < Pl::kNumBars; ++k) mbar_inval(bar(k));
    fence_proxy_async_all();  // whatever uses this shared memory next, through either proxy
    __syncthreads();
  }
}

}  // namespace
}  // namespace sfs
