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
#include "sfs_tc16_dev.cuh"

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


// One CTA's contiguous share of the nunits units.
template <bool FWD, int NP, int NB>
__global__ void __launch_bounds__(kHThreads, HPlan<NP, NB>::kCtasPerSm)
contract_h(const __grid_constant__ CUtensorMap tab, const __grid_constant__ CUtensorMap spec,
           float2* __restrict__ out, long long out_stride, int nscene, PlaneDims d, int nmt, int nch,
           int nunits, const float* __restrict__ pm, int* __restrict__ err) {
  extern __shared__ unsigned char hsm_raw[];
  const int G = gridDim.x, b = blockIdx.x;
  const int first = (int)(((long long)nunits * b) / G);
  const int nu = (int)(((long long)nunits * (b + 1)) / G) - first;
  contract_h_run<FWD, NP, NB>(&tab, &spec, out, out_stride, nscene, d, nmt, nch, first, nu, pm, err, hsm_raw);
}

template <bool FWD, int NP, int NB>
int launch_h(const PlaneDims& d, const CUtensorMap& tab, const CUtensorMap& spec, float2* out,
             long long out_stride, int nscene, const float* pm, int* err, cudaStream_t st) {
  using Pl = HPlan<NP, NB>;
  SFS_TRY(ensure_smem_attr(contract_h<FWD, NP, NB>, Pl::kSmem));
  int nmt = 0, nch = 0, nunits = 0;
  tc16_units(d, FWD, &nmt, &nch, &nunits);
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

void tc16_units(const PlaneDims& d, bool fwd, int* nmt, int* nch, int* nunits) {
  const int No = d.Ns / d.GS;
  *nmt = fwd ? (d.U + 127) / 128 : (d.nkb + 1) / 2;
  *nch = fwd ? d.nkb : (d.U + 63) / 64;
  *nunits = No * *nmt;
}

int tc16_group_of(const PlaneDims& d) { return group_of(d); }

int tc16_table_maps(const sfs_operator* op, CUtensorMap* tab_f, CUtensorMap* tab_a) {
  if (!op->tmaps) {
    set_error("16-bit contraction without tensor maps");
    return SFS_ERR_INVALID_ARG;
  }
  *tab_f = op->tmaps->tab_f;
  *tab_a = op->tmaps->tab_a;
  return SFS_OK;
}

int tc16_encode_spec(CUtensorMap* m, const void* base, int rows, int Ns, int box_rows, int scenes,
                     int box_scenes) {
  return encode_spec(m, base, rows, Ns, box_rows, scenes, box_scenes);
}

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
