// Depth contractions on the tensor cores from a 16-bit table (tcgen05
// kind::f16, BF16 or FP16 operands, FP32 accumulation in tensor memory).
//
// The generator table holds one entry per symmetry orbit of wavenumbers
// (the lateral kernel depends on dx^2 + dy^2 only, Eq. (3)), so both
// contractions of Sec. IV-B are small dense products per orbit o, with n
// over the orbit's slots (Theorem 2, Algorithm 2):
//   forward  Y[u][n] = sum_z T[u][z] X[z][n]           M = bins,   K = depths
//   adjoint  G[z][n] = sum_u conj(T[u][z]) R[u][n]     M = depths, K = bins
// The table is stored as rows of 64 16-bit values, one row per (part, orbit,
// 32-depth block kb, bin u): element 2 zz + q is Re (q = 0) or Im (q = 1) of
// T[u][32 kb + zz].  Part 0 is the BF16 rounding of the FP32 table, part 1
// (two-part tables) the BF16 rounding of the remainder.  Such a row is one
// 128-byte line of the 128-byte-swizzled canonical layouts, so bulk tensor
// copies (TMA) bring table tiles from global memory straight into the
// layout the MMA reads: the table never passes through registers.
//
// Forward (K-major A = table tile, rows u, K index k = 2 zz + q):
//   [Yr | Yi][u] = sum_k A[u][k] B[k],  B[2zz] = [Xr | Xi],  B[2zz+1] = [-Xi | Xr]
// Adjoint (MN-major A: the same tile read with M index m = 2 zz + q, K = u;
// two depth blocks side by side give M = 128):
//   D[2zz + q][n] = sum_u T_q[u][z] [Rr | Ri][u][n],
//   Gr = D[2zz][re] + D[2zz+1][im],  Gi = D[2zz][im] - D[2zz+1][re],
// combined in the epilogue between neighbouring TMEM lanes.
// The spectra operand B (8 slots x re/im = 16 columns) is split into BF16
// hi and lo = the BF16 rounding of (value - hi); both are stacked along N
// (N = 32) and summed in the epilogue, so the spectra keep about 16
// significant bits and the table's rounding dominates the error.
// FP16 operands (11 significant bits, but only 2^-24 .. 65504) are scaled by
// powers of two: the table by 2^kT at build, each scene's spectra by 2^ks
// from the largest |Re| or |Im| of its spectra (the per-plane maxima that
// the kernels storing the spectra leave in pm), so that the largest value
// lies in [2^13, 2^14).  The epilogue multiplies by 2^-ks and 2^-kT, which
// is exact; BF16 operands are not scaled.
//
// Per CTA (192 threads, two CTAs per SM, 64 TMEM columns):
//   warp 4     issues the TMA copies of a chunk's table tile(s) into a stage
//              of the table ring (one mbarrier per stage);
//   warp 6     issues the TMA copy of a chunk's spectra tile into a slot of
//              the spectra ring (8 slots, one mbarrier per slot), as far
//              ahead as the slots allow;
//   warps 0-3  build a chunk's B operand (hi and lo) from its spectra tile
//              into a slot of the B ring, and read a unit's accumulator
//              (tcgen05.ld) while building the next unit's third chunk;
//   warp 5     issues the 4 x parts MMAs of a chunk (M = 128, N = 32,
//              K = 16) and commits to the barriers that free the stage and
//              the slot and signal the accumulator (two, alternating by
//              unit).
// Work: units (orbit, bin tile of 128) forward, (orbit, pair of depth
// blocks) adjoint; a contiguous share of units per persistent CTA; a unit
// runs over K in chunks (a 32-depth block forward, 64 bins adjoint).
//
// Every mbarrier wait is bounded (wait_ns).  A timeout sets the device error
// flag and a shared abort flag that ends the other roles' waits; the copy
// warp then waits (bounded) for its copies in flight, the MMA warp for its
// MMAs, and warp 0 frees the tensor memory before the CTA exits.
#include <cuda.h>  // CUtensorMap and its enums (the encoder is fetched at run time)
#include <cuda_bf16.h>
#include <cuda_fp16.h>
#include <cuda_runtime.h>
#include <stdint.h>

#include <algorithm>
#include <mutex>

#include "sfs_async.cuh"
#include "sfs_internal.h"
#include "sfs_launch.h"
#include "sfs_tcgen05.cuh"

namespace sfs {

struct TcMaps {
  CUtensorMap tab_f;  // table, box 64 x 128 rows: forward A tiles
  CUtensorMap tab_a;  // table, box 64 x 64 rows: adjoint A tiles (one depth block)
  CUtensorMap xh;     // X^ c64 [Nz][Ns] as floats, box 16 x 32
  CUtensorMap rh;     // R^ c64 [Up][Ns] as floats, box 16 x 64
  const void* xh_ptr = nullptr;
  const void* rh_ptr = nullptr;
  // map of single-scene residual spectra at one other address (the static
  // scratch of sfs_apply_AH_noalloc), encoded on first use and kept
  CUtensorMap rh_alt;
  const void* rh_alt_ptr = nullptr;
};

void free_tc_maps(TcMaps* m) { delete m; }

namespace {

// ---------------------------------------------------------------------------
// Tensor maps (host)
// ---------------------------------------------------------------------------
using EncodeTiledFn = CUresult (*)(CUtensorMap*, CUtensorMapDataType, cuuint32_t, void*,
                                   const cuuint64_t*, const cuuint64_t*, const cuuint32_t*,
                                   const cuuint32_t*, CUtensorMapInterleave, CUtensorMapSwizzle,
                                   CUtensorMapL2promotion, CUtensorMapFloatOOBfill);

int encoder(EncodeTiledFn* out) {
  static std::once_flag once;
  static EncodeTiledFn fn = nullptr;
  static cudaError_t qerr = cudaSuccess;
  std::call_once(once, [] {
    void* p = nullptr;
    cudaDriverEntryPointQueryResult q = cudaDriverEntryPointSymbolNotFound;
    qerr = cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &p, 12000, cudaEnableDefault, &q);
    if (qerr == cudaSuccess && q == cudaDriverEntryPointSuccess) fn = (EncodeTiledFn)p;
  });
  if (!fn) {
    set_error("cuTensorMapEncodeTiled is not available (%s)", cudaGetErrorString(qerr));
    return SFS_ERR_CUDA;
  }
  *out = fn;
  return SFS_OK;
}

// 16-bit table [parts * No][nkb][U][64], 128-byte swizzle, box 64 x rows;
// rows past U and blocks past nkb read as zero.
int encode_table(CUtensorMap* m, const void* table, int U, int nkb, int planes, int rows, bool f16) {
  EncodeTiledFn enc;
  SFS_TRY(encoder(&enc));
  const cuuint64_t dims[4] = {64, (cuuint64_t)U, (cuuint64_t)nkb, (cuuint64_t)planes};
  const cuuint64_t strides[3] = {128, (cuuint64_t)U * 128, (cuuint64_t)nkb * U * 128};
  const cuuint32_t box[4] = {64, (cuuint32_t)rows, 1, 1};
  const cuuint32_t estr[4] = {1, 1, 1, 1};
  const CUresult r = enc(m, f16 ? CU_TENSOR_MAP_DATA_TYPE_FLOAT16 : CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, 4,
                         const_cast<void*>(table), dims, strides,
                         box, estr, CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_128B,
                         CU_TENSOR_MAP_L2_PROMOTION_L2_256B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
  if (r != CUDA_SUCCESS) {
    set_error("tensor map of the 16-bit table rejected (CUresult %d)", (int)r);
    return SFS_ERR_CUDA;
  }
  return SFS_OK;
}

// Lateral spectra of `scenes` consecutive scenes, c64 [scenes][rows][Ns]
// seen as floats [scenes][rows][2 Ns]; box of 8 slots (16 floats) x
// box_rows x box_scenes, no swizzle; rows past `rows` and scenes past
// `scenes` read as zero.
int encode_spec(CUtensorMap* m, const void* base, int rows, int Ns, int box_rows, int scenes = 1,
                int box_scenes = 1) {
  EncodeTiledFn enc;
  SFS_TRY(encoder(&enc));
  const cuuint64_t dims[3] = {(cuuint64_t)2 * Ns, (cuuint64_t)rows, (cuuint64_t)scenes};
  const cuuint64_t strides[2] = {(cuuint64_t)Ns * 8, (cuuint64_t)rows * Ns * 8};
  const cuuint32_t box[3] = {16, (cuuint32_t)box_rows, (cuuint32_t)box_scenes};
  const cuuint32_t estr[3] = {1, 1, 1};
  const CUresult r = enc(m, CU_TENSOR_MAP_DATA_TYPE_FLOAT32, 3, const_cast<void*>(base), dims, strides, box,
                         estr, CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_NONE,
                         CU_TENSOR_MAP_L2_PROMOTION_L2_128B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
  if (r != CUDA_SUCCESS) {
    set_error("tensor map of the lateral spectra rejected (CUresult %d)", (int)r);
    return SFS_ERR_CUDA;
  }
  return SFS_OK;
}

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
template <bool FWD, int NP, int NB>
__global__ void __launch_bounds__(kHThreads, HPlan<NP, NB>::kCtasPerSm)
contract_h(const __grid_constant__ CUtensorMap tab, const __grid_constant__ CUtensorMap spec,
           float2* __restrict__ out, long long out_stride, int nscene, PlaneDims d, int nmt, int nch,
           int nunits, const float* __restrict__ pm, int* __restrict__ err) {
  using Pl = HPlan<NP, NB>;
  constexpr uint32_t kHCols = Pl::kCols;
  constexpr int ST = Pl::kST, SS = Pl::kSS, SBB = Pl::kSBB, LEAD = Pl::kLead;
  extern __shared__ unsigned char hsm_raw[];
  // 128-byte-swizzled tiles need 1 KB alignment of the shared-memory address
  unsigned char* hsm = hsm_raw + ((1024u - (smem_addr(hsm_raw) & 1023u)) & 1023u);
  const uint32_t sbase = smem_addr(hsm);
  uint32_t* tslot = (uint32_t*)(hsm + Pl::kOffSlot);
  volatile int* abort_flag = (volatile int*)(hsm + Pl::kOffSlot + 4);
  const uint32_t bar0 = sbase + Pl::kOffBar;
  auto bar = [&](int k) { return bar0 + 8u * (uint32_t)k; };
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int G = gridDim.x, b = blockIdx.x;
  const int first = (int)(((long long)nunits * b) / G);
  const int items = ((int)(((long long)nunits * (b + 1)) / G) - first) * nch;
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
    tc_relinquish();
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
        tma_load_3d(sbase + Pl::kOffS + sl * Pl::kSSlot, &spec, 2 * o * d.GS, (FWD ? 32 : 64) * c, 0, fb);
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
            tma_load_table(dst + p * kHATile, &tab, 0, 128 * mt, c, p * No + o, fb, stream, pol);
        } else {  // bins 64 c .., depth blocks 2 mt and 2 mt + 1
#pragma unroll
          for (int p = 0; p < NP; ++p) {
            tma_load_table(dst + p * kHATile, &tab, 0, 64 * c, 2 * mt, p * No + o, fb, stream, pol);
            tma_load_table(dst + p * kHATile + 8192, &tab, 0, 64 * c, 2 * mt + 1, p * No + o, fb, stream,
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
  } else {
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
  }
  pdl_trigger();
  tc_fence_before();
  __syncthreads();
  if (warp == 0) {
    tc_fence_after();
    tc_dealloc(tmem, kHCols);
  }
}

template <bool FWD, int NP, int NB>
int launch_h(const PlaneDims& d, const CUtensorMap& tab, const CUtensorMap& spec, float2* out,
             long long out_stride, int nscene, const float* pm, int* err, cudaStream_t st) {
  using Pl = HPlan<NP, NB>;
  SFS_TRY(ensure_smem_attr(contract_h<FWD, NP, NB>, Pl::kSmem));
  const int No = d.Ns / d.GS;
  const int nmt = FWD ? (d.U + 127) / 128 : (d.nkb + 1) / 2;
  const int nch = FWD ? d.nkb : (d.U + 63) / 64;
  const int nunits = No * nmt;
  // d.G = two CTAs per SM
  const int G = std::min(Pl::kCtasPerSm == 2 ? d.G : d.G / 2, nunits);
  if (G <= 0) return SFS_OK;
  return launch_pdl(contract_h<FWD, NP, NB>, dim3(G), dim3(kHThreads), (size_t)Pl::kSmem, st, tab, spec,
                    out, out_stride, nscene, d, nmt, nch, nunits, pm, err);
}

// Scene group size of a batched call: one table tile serves up to 4 scenes
// (default: 4 from three scenes on), unless tuning fixed it (d.nb).
int group_of(const PlaneDims& d) {
  const int batch = std::max(1, d.batch);
  if (d.nb == 1 || d.nb == 2 || d.nb == 4) return d.nb;
  return batch >= 3 ? 4 : batch;
}

// One contraction launch per group of scenes: spectra of the group from
// `spec_base` (scene stride spec_stride elements, `rows` rows), outputs from
// `out` (scene stride out_stride).
template <bool FWD>
int launch_groups(const PlaneDims& d, const CUtensorMap& tab, const CUtensorMap* cached, const float2* base,
                  long long spec_stride, int rows, int box_rows, float2* out, long long out_stride,
                  int* err, cudaStream_t st) {
  const int B = std::max(1, d.batch), NB = group_of(d);
  for (int g0 = 0; g0 < B; g0 += NB) {
    CUtensorMap local;
    const CUtensorMap* spec = cached;
    if (!spec || B > 1) {
      SFS_TRY(encode_spec(&local, base + g0 * spec_stride, rows, d.Ns, box_rows, B - g0, NB));
      spec = &local;
    }
    float2* o = out + g0 * out_stride;
    const int n = std::min(NB, B - g0);
    // per-plane spectra maxima of the group's first scene (FP16 modes)
    const float* pm0 = FWD ? d.pm_x : d.pm_r;
    const float* pm = pm0 ? pm0 + g0 * (FWD ? d.bs_pmx : d.bs_pmr) : nullptr;
    int rc;
    if (d.nparts == 2) {
      rc = NB == 1 ? launch_h<FWD, 2, 1>(d, tab, *spec, o, out_stride, n, pm, err, st)
         : NB == 2 ? launch_h<FWD, 2, 2>(d, tab, *spec, o, out_stride, n, pm, err, st)
                   : launch_h<FWD, 2, 4>(d, tab, *spec, o, out_stride, n, pm, err, st);
    } else {
      rc = NB == 1 ? launch_h<FWD, 1, 1>(d, tab, *spec, o, out_stride, n, pm, err, st)
         : NB == 2 ? launch_h<FWD, 1, 2>(d, tab, *spec, o, out_stride, n, pm, err, st)
                   : launch_h<FWD, 1, 4>(d, tab, *spec, o, out_stride, n, pm, err, st);
    }
    SFS_TRY(rc);
  }
  return SFS_OK;
}

int check_maps(const PlaneDims& d) {
  if (!d.tmaps || (d.nparts != 1 && d.nparts != 2)) {
    set_error("16-bit contraction without tensor maps");
    return SFS_ERR_INVALID_ARG;
  }
  return SFS_OK;
}

}  // namespace

int tc16_setup(sfs_operator* op) {
  TcMaps* m = new (std::nothrow) TcMaps;
  if (!m) {
    set_error("host allocation failed");
    return SFS_ERR_OOM;
  }
  const int planes = op->nparts * (op->Ns / op->GS);
  int rc = encode_table(&m->tab_f, op->table, op->U, op->nkb, planes, 128, op->f16 != 0);
  if (rc == SFS_OK) rc = encode_table(&m->tab_a, op->table, op->U, op->nkb, planes, 64, op->f16 != 0);
  if (rc == SFS_OK) rc = encode_spec(&m->xh, op->ws.Xh, op->geo.d.Nz, op->Ns, 32);
  if (rc == SFS_OK) rc = encode_spec(&m->rh, op->ws.Rh, op->Up, op->Ns, 64);
  if (rc != SFS_OK) {
    delete m;
    return rc;
  }
  m->xh_ptr = op->ws.Xh;
  m->rh_ptr = op->ws.Rh;
  free_tc_maps(op->tmaps);
  op->tmaps = m;
  return SFS_OK;
}

int launch_contract_fwd_h(const PlaneDims& d, const float2* Xh, float2* Yp, int* err, cudaStream_t st) {
  SFS_TRY(check_maps(d));
  const CUtensorMap* cached = (Xh == d.tmaps->xh_ptr && d.batch <= 1) ? &d.tmaps->xh : nullptr;
  return launch_groups<true>(d, d.tmaps->tab_f, cached, Xh, d.bs_xh, d.Nz, 32, Yp, d.bs_yh, err, st);
}

int launch_contract_adj_h(const PlaneDims& d, const float2* Rh, float2* Gs, int* err, cudaStream_t st) {
  SFS_TRY(check_maps(d));
  // spectra elsewhere than the operator's workspace get a map of their own:
  // a batched workspace per launch, one other single-scene address (the
  // static scratch of sfs_apply_AH_noalloc) once, then from the cache
  const CUtensorMap* cached = nullptr;
  if (d.batch <= 1) {
    if (Rh == d.tmaps->rh_ptr) {
      cached = &d.tmaps->rh;
    } else {
      if (Rh != d.tmaps->rh_alt_ptr) {
        d.tmaps->rh_alt_ptr = nullptr;
        SFS_TRY(encode_spec(&d.tmaps->rh_alt, Rh, d.Up, d.Ns, 64));
        d.tmaps->rh_alt_ptr = Rh;
      }
      cached = &d.tmaps->rh_alt;
    }
  }
  return launch_groups<false>(d, d.tmaps->tab_a, cached, Rh, d.bs_rh, d.Up, 64, Gs, d.bs_gh, err, st);
}

template <int NP, int NB>
int prepare_one() {
  SFS_TRY(ensure_smem_attr(contract_h<true, NP, NB>, HPlan<NP, NB>::kSmem));
  return ensure_smem_attr(contract_h<false, NP, NB>, HPlan<NP, NB>::kSmem);
}

int prepare_tc16_kernels(const PlaneDims& d) {
  const int NB = group_of(d);
  if (d.nparts == 2)
    return NB == 1 ? prepare_one<2, 1>() : NB == 2 ? prepare_one<2, 2>() : prepare_one<2, 4>();
  return NB == 1 ? prepare_one<1, 1>() : NB == 2 ? prepare_one<1, 2>() : prepare_one<1, 4>();
}

}  // namespace sfs
