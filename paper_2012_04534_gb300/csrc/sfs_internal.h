// Internal declarations of libsfs: operator state and the kernel launchers.
#pragma once

#include <cuda.h>
#include <cuda_runtime.h>
#include <math.h>
#include <stdint.h>

#include <string>
#include <utility>
#include <vector>

#include "../../include/sfs.h"

namespace sfs {

// Thread-local error message behind sfs_last_error().
void set_error(const char* fmt, ...);
void clear_error();

// A CUDA runtime failure: records the message and returns SFS_ERR_CUDA (or
// SFS_ERR_OOM for allocation failures).
int cuda_fail(cudaError_t e, const char* what, const char* file, int line);

#define SFS_CUDA(call)                                                   \
  do {                                                                   \
    cudaError_t e_ = (call);                                             \
    if (e_ != cudaSuccess) return ::sfs::cuda_fail(e_, #call, __FILE__, __LINE__); \
  } while (0)

#define SFS_TRY(call)                 \
  do {                                \
    int rc_ = (call);                 \
    if (rc_ != SFS_OK) return rc_;    \
  } while (0)

// |H(f)| of the pulse h(t) = exp(-alpha^2 t^2 + j 2 pi fc t) (Sec. VI):
// (sqrt(pi) / alpha) exp(-(pi (f - fc) / alpha)^2).
inline double pulse_mag(double f, double fc, double alpha) {
  const double a = M_PI * (f - fc) / alpha;
  return sqrt(M_PI) / alpha * exp(-a * a);
}

// Largest lateral FFT side held in one CTA's shared memory (a 128 x 129
// padded c64 plane is 132 KB).
constexpr int kMaxP2D = 128;
constexpr int kMaxP1D = 4096;
// Lateral wavenumbers per table tile: a warp lane owns two, loaded as float4.
constexpr int kKappaTile = 64;

// Device-side scalars of one operator (one cudaMalloc, see Workspace).
enum ScalarSlot {
  kThr = 0,     // float: soft threshold lambda / L
  kInvL = 1,    // float: 1 / L
  kLamMax = 2,  // float bits (uint): max |A^H y| (atomicMax on the bit pattern)
  kNumFloatScalars = 4
};

// Reduction slots (double) of one operator.
enum RedSlot {
  kRedA = 0,   // scratch sums used by the power iteration
  kRedB = 1,
  kRedC = 2,
  kNumRed = 4
};

// Buffers of batched calls (scenes sharing one operator), `cap` scenes each,
// allocated on first use and grown on demand.
struct BatchWorkspace {
  int cap = 0;
  float2* Xh = nullptr;      // [cap][Nz][Ns]
  float2* Yh = nullptr;      // [cap][nzb][Up][Ns]
  float2* Rh = nullptr;      // [cap][Up][Ns] (rows U..Up-1 zero)
  float2* Gh = nullptr;      // [cap][nslots][azb][64]
  float2* xk = nullptr;      // [cap][V]
  float2* gam = nullptr;     // [cap][V]
  float2* yplane = nullptr;  // [cap][U][S]
  float2* ybuf = nullptr;    // [cap][S][M] measurements copy
  float* scal = nullptr;     // [cap][kNumFloatScalars]
  float* pmx = nullptr;      // [cap][Nz] FP16 modes: max |Re|, |Im| of each X^ plane
  float* pmr = nullptr;      // [cap][Up] FP16 modes: the same of each R^ plane
};

struct Workspace {
  float2* Xh = nullptr;     // [Nz][Ns]   lateral spectra of voxel planes (slot order)
  float2* Yh = nullptr;     // [nzb][Up][Ns] depth-block partials of bin-plane spectra
  float2* Rh = nullptr;     // [Up][Ns]   lateral spectra of residual planes (rows
                            //            U..Up-1 stay zero)
  float2* Gh = nullptr;     // [nslots][128][64] adjoint contraction partials
  int2* segslot = nullptr;  // [nseg] {first slot, slot count} per (tile, depth block)
  int* err = nullptr;       // device flag: a bounded wait in a kernel timed out
  float2* xk = nullptr;     // [V] FISTA iterate x_k
  float2* gam = nullptr;    // [V] FISTA extrapolated point gamma_k
  float2* ybuf = nullptr;   // [S][M] measurements copy
  float2* yplane = nullptr; // [U][S] measurements by bin plane (FISTA residual)
  float2* vbuf = nullptr;   // [S][M] scratch (power iteration)
  float* scal = nullptr;    // kNumFloatScalars floats
  double* red = nullptr;    // kNumRed doubles
  float* pmx = nullptr;     // [Nz] FP16 modes: max |Re|, |Im| of each X^ plane
  float* pmr = nullptr;     // [Up] FP16 modes: the same of each R^ plane
  double* obj = nullptr;    // [2 * obj_cap] objective monitor sums
  int obj_cap = 0;
  float* beta = nullptr;    // [beta_cap] momentum coefficients of the current FISTA call
  int beta_cap = 0;
  int beta_fresh = 0;       // beta[0..beta_fresh) holds the sequence from t_1 = 1
  double* tnext = nullptr;  // t_{k+1} after the current FISTA call (no state buffer given)
};

}  // namespace sfs

struct sfs_geometry {
  sfs_geometry_desc d;  // validated copy, t0 resolved
  double alpha;
  int Px, Py;           // lateral FFT sizes
};

namespace sfs {
// Tensor maps of the 16-bit tensor-core contractions (sfs_tc16.cu); opaque
// elsewhere.
struct TcMaps;
void free_tc_maps(TcMaps* m);
}  // namespace sfs

struct sfs_operator {
  sfs_geometry geo;
  int M = 0, S = 0, V = 0, U = 0, Nk = 0;
  int Ns = 0, GS = 0, No = 0;  // wavenumber slots, slots per orbit, orbits
  int Up = 0;                  // bins padded to a multiple of GS / 2
  int prec = 0;                // sfs_precision of the depth contractions
  int tc = 0;                  // contraction kernels: 0 CUDA cores (sfs_kernels.cu),
                               // 1 tensor cores kind::tf32 (sfs_tc.cu), 2 tensor
                               // cores kind::f16 from a 16-bit table (sfs_tc16.cu)
  int nzc = 0;                 // depth blocks of 16 in the tf32 tensor-core table
  int nkb = 0;                 // depth blocks of 32 in the 16-bit table
  int nparts = 1;              // 16-bit table parts: 1 (value) or 2 (hi, lo)
  int f16 = 0;                 // 16-bit table and spectra operands in FP16 (else BF16)
  int tscale_exp = 0;          // FP16 modes: the table is stored times 2^tscale_exp
  sfs::TcMaps* tmaps = nullptr;  // tensor maps of the 16-bit contractions
  int nzb = 1;                 // depth blocks of <= 128 in the contractions
  int G = 1;                   // persistent CTAs of the contractions
  int nslots = 0;              // adjoint partial-sum slots
  int adj_seg = 0, azb = 128, anzb = 1, Ga = 0;  // adjoint layout (see PlaneDims)
  uint64_t wait_ns = 2000000000ull;              // bounded-wait limit (2 s)
  int stream_table = 0;                          // see PlaneDims::stream_table
  int inject = 0;                                // see PlaneDims::inject
  int k_lo = 0, k_hi = 0;
  double band_db = 0.0;
  // bin shard (sfs_operator_shard): this operator holds the run
  // [shard_first, shard_first + U) of the union of all kept bins, split
  // into nshards runs; its rows are the measurements of those bins
  int nshards = 1, shard = 0, shard_first = 0, U_all = 0;
  std::vector<int32_t> idx;    // [S][M]
  std::vector<int32_t> bins;   // [U] union of kept bins, ascending
  // device data
  float2* table = nullptr;     // one entry per symmetry orbit of wavenumbers per
                               // (bin, depth), includes 1/(Px*Py); depth pairs
                               // interleaved, layout per contraction path
                               // (sfs_kernels.cu / sfs_tc.cu)
  int32_t* slot_kappa = nullptr;  // [Ns]
  int32_t* orbit_rep = nullptr;   // [Ns/GS]
  int32_t* quad = nullptr;        // 128 x 128 planes: [8 + Ns] slots grouped by quadrant
  int32_t* posmap = nullptr;   // [U][S]: m with idx[s][m] == bins[u], else -1
  sfs::Workspace ws;
  // kernel timing (SFS_FISTA_TIME_KERNELS)
  std::vector<cudaEvent_t> ev;
  int ev_used = 0;
  // FISTA iteration loops captured as CUDA graphs, keyed by (iterations,
  // objective monitor on/off, event nodes around each kernel on/off);
  // replayed on the caller's stream
  struct GraphEntry {
    int iters;
    bool with_obj;
    bool timed;
    cudaGraphExec_t exec;
  };
  std::vector<GraphEntry> graphs;
  cudaStream_t capture_stream = nullptr;
  // batched FISTA: workspace and captured loops keyed by (iterations, scenes)
  sfs::BatchWorkspace bws;
  uint64_t uid = 0;      // process-unique operator id (keys of grouped graphs)
  uint64_t bws_gen = 0;  // bumped whenever the batched workspace is reallocated (or retuned)
  std::vector<std::pair<int, int>> batch_tile;  // (batch, scenes per table tile) chosen by tuning
  struct BatchGraphEntry {
    int iters;
    int batch;
    cudaGraphExec_t exec;
  };
  std::vector<BatchGraphEntry> bgraphs;
};

namespace sfs {

// ---- kernel launchers (sfs_kernels.cu) ----

struct PlaneDims {
  int Nx, Ny, Nz, Px, Py, Nk, S, M, U;
  int nzb;  // depth blocks of <= 128 depths in the contractions
  int G;    // persistent CTAs of the contractions (<= SM count)
  int Ns;   // wavenumber slots (orbit-major, a multiple of 64)
  int GS;   // slots per symmetry orbit: 2 (line), 4 (area), 8 (square area)
  int Up;   // bins padded to a multiple of GS / 2 (zero table rows and spectra)
  int tc;   // contraction kernels (see sfs_operator::tc); tc > 0: nzb = 1 and the
            // dense segment-aligned adjoint result
  int nzc;  // depth blocks of 16 of the tf32 tensor-core table
  int prec;    // sfs_precision
  int nkb;     // depth blocks of 32 of the 16-bit table
  int nparts;  // parts of the 16-bit table (1 or 2)
  int f16;     // 16-bit operands are FP16 (scaled by powers of two), else BF16
  float tscale;  // FP16 modes: scale 2^kT of the stored table (1 otherwise)
  float tinv;    // 2^-kT
  // FP16 modes: per-plane maxima of max(|Re|, |Im|) of the spectra, written by
  // the kernels that store X^ (pm_x, [batch][Nz]) and R^ (pm_r, [batch][Up]);
  // null otherwise.  The 16-bit contractions scale each scene's spectra by
  // the power of two that brings its largest value just below 2^14.
  float* pm_x;
  float* pm_r;
  long long bs_pmx;  // per-scene strides of pm_x (Nz) and pm_r (Up)
  long long bs_pmr;
  TcMaps* tmaps;  // host pointer: tensor maps of the 16-bit contractions
  int adj_seg;  // adjoint by segment-aligned CTAs (dense result) instead of partial sums
  int azb;      // depth rows per adjoint segment (32 segment-aligned, 128 otherwise)
  int anzb;     // adjoint depth blocks per slot tile
  int Ga;       // CTAs of the segment-aligned adjoint (= its segment count)
  int stream_table;  // the table exceeds half the L2: its copies are evict-first
  uint64_t wait_ns;  // limit of each bounded mbarrier wait in the contractions
  int inject;        // failure-handling tests: first wait of each warp never completes
  // Scenes sharing this operator processed by one launch (gridDim.y of the
  // plane kernels, blockIdx.y = scene), and the per-scene strides (elements)
  // of the batched buffers; batch = 1 for single-scene calls.
  int batch;
  int nb;               // 16-bit contractions: scenes per table tile (1, 2, 4), 0 = default rule
  long long bs_x;       // x, x_k, gamma: V
  long long bs_xh;      // X^: Nz * Ns
  long long bs_yh;      // forward contraction output: nzb * Up * Ns
  long long bs_rh;      // R^: Up * Ns
  long long bs_gh;      // adjoint contraction output: nslots * azb * 64
  long long bs_y;       // measurements: S * M
  long long bs_yplane;  // measurements by bin plane: U * S
  int bs_scal;          // device scalars (floats) per scene
  int bs_red;           // reduction slots (doubles) per scene
  const int32_t* slot_kappa;  // [Ns] wavenumber of each slot, -1 for padding
  const int32_t* orbit_rep;   // [Ns / GS] representative wavenumber, -1 for padding
  const int32_t* quad;        // 128 x 128 planes: slots by quadrant (sfs_kernels.cu), else null
};

// Resident contraction CTAs per SM (8 warps each); the persistent grid is
// this times the SM count.
constexpr int kContractCtasPerSm = 2;
// Depth block of the contractions and the partial-sum slots of the adjoint.
constexpr int kZBlockRows = 128;
// Units of contraction work: (slot tile, depth block, bin).
int contract_units(const PlaneDims& d);

// Kernel-side dimensions and tables of an operator (sfs_api.cu).
PlaneDims operator_dims(const sfs_operator* op);

// Operator build (sfs_api.cu): the union of the kept bins of idx_host is
// split into nshards contiguous runs of floor-balanced length (run j holds
// positions [j U / n, (j + 1) U / n) of the ascending union); the operator
// keeps run `shard` (nshards = 1: every bin).
int build_operator_shard(sfs_geometry* g, int M, const int32_t* idx_host, int prec, int nshards,
                         int shard, sfs_operator** out);
// First union position and length of run `shard` of U bins in nshards.
void shard_run(int U, int nshards, int shard, int* first, int* count);
// g = A^H (A x - y) on the operator's own rows (single scene, its workspace).
int normal_residual(sfs_operator* op, const float2* x, const float2* y, float2* g, cudaStream_t st);
int check_err_flag_op(sfs_operator* op, cudaStream_t st);

// Table of generators (Theorem 2 / Eq. (4)); tof: float2 [Nz][Ny][Nx]
// (hi, lo) of (tau - t0) fs / Nt in turns per unit bin; gdir: float
// [Nz][Ny][Nx] directivity; amp: float [U] = fs H(f_k) / (Px Py); bins: int [U].
int launch_build_table(const PlaneDims& d, const float2* tof, const float* gdir,
                       const float* amp, const int32_t* bins, float2* table,
                       cudaStream_t st);

// Plane kernels.  Each processes one lateral plane per CTA.
int launch_fwd_planes(const PlaneDims& d, const float2* x, float2* Xh,
                      cudaStream_t st);
int launch_inv_gather(const PlaneDims& d, const float2* Yh, const int32_t* posmap,
                      float2* y, double* red_sumsq, cudaStream_t st);
int launch_inv_resid_fwd(const PlaneDims& d, const float2* Yh, const int32_t* posmap,
                         const float2* yplane, float2* Rh, double* red_sumsq,
                         cudaStream_t st);
// y[s][m] -> yplane[u][s], zero where bin plane u is not kept at position s
int launch_scatter_y_planes(const PlaneDims& d, const float2* y, const int32_t* posmap,
                            float2* yplane, cudaStream_t st);
int launch_scatter_fwd(const PlaneDims& d, const float2* y, const int32_t* posmap,
                       float2* Rh, cudaStream_t st);
int launch_inv_store(const PlaneDims& d, const float2* Gh, const int2* segslot,
                     float2* x, double* red_sumsq, unsigned int* maxabs_bits,
                     cudaStream_t st);
// beta_dev (optional): device pointer to this iteration's beta, else `beta`.
int launch_inv_fista_fwd(const PlaneDims& d, const float2* Gh, const int2* segslot,
                         float2* xk, float2* gam, const float* scal, float beta,
                         int do_fwd, float2* Xh, double* red_l1, cudaStream_t st,
                         const float* beta_dev = nullptr);
// Momentum table beta[0..iters) of Algorithm 1 from t_1 = *t_in (1 if null),
// t_{iters+1} to *t_out, iters added to *cnt (if not null); one thread.
int launch_fista_betas(const double* t_in, int iters, float* beta, double* t_out, long long* cnt,
                       cudaStream_t st);

// Depth contractions over the generator table.  Yp: [nzb][U][Nk] depth-block
// partials; Gs: [slots][128][64] adjoint partials (see segment_slots).  err:
// device int set to 1 when a bounded wait times out.
int launch_contract_fwd(const PlaneDims& d, const float2* table, const float2* Xh,
                        float2* Yp, int* err, cudaStream_t st);
int launch_contract_adj(const PlaneDims& d, const float2* table, const float2* Rh,
                        float2* Gs, int* err, cudaStream_t st);

// The same two contractions on the tensor cores (sfs_tc.cu); used when d.tc.
int launch_contract_fwd_tc(const PlaneDims& d, const float2* table, const float2* Xh,
                           float2* Yp, int* err, cudaStream_t st);
int launch_contract_adj_tc(const PlaneDims& d, const float2* table, const float2* Rh,
                           float2* Gs, int* err, cudaStream_t st);
int prepare_tc_kernels();

// The same two contractions on the tensor cores from the 16-bit table
// (sfs_tc16.cu); used when d.tc == 2.  tc16_setup encodes the tensor maps of
// an operator's table and workspace (once, after the table is allocated).
int tc16_setup(sfs_operator* op);
int launch_contract_fwd_h(const PlaneDims& d, const float2* Xh, float2* Yp, int* err,
                          cudaStream_t st);
int launch_contract_adj_h(const PlaneDims& d, const float2* Rh, float2* Gs, int* err,
                          cudaStream_t st);
int prepare_tc16_kernels(const PlaneDims& d);
// Work units of one 16-bit contraction launch (forward: (orbit, tile of 128
// bins), nch chunks of 32 depths; adjoint: (orbit, pair of 32-depth blocks),
// nch chunks of 64 bins), the scenes a table tile serves, the table's tensor
// maps and the map of a batch's spectra (scene tiles of box_scenes).
void tc16_units(const PlaneDims& d, bool fwd, int* nmt, int* nch, int* nunits);
int tc16_group_of(const PlaneDims& d);
int tc16_table_maps(const sfs_operator* op, CUtensorMap* tab_f, CUtensorMap* tab_a);
int tc16_encode_spec(CUtensorMap* m, const void* base, int rows, int Ns, int box_rows, int scenes,
                     int box_scenes);

// ---- the persistent FISTA loop over groups of scenes (sfs_persist.cu) ----
// persist_build prepares the device plan of `iters` iterations of Algorithm 1
// for the groups (ops[g], dims[g] = the batched dimensions of its scenes) on
// the operators' batched workspaces: 16-bit single-part 2-D operators only.
// persist_launch zeroes the grid barrier and launches the cooperative kernel
// (capturable); the measurements by plane, the thresholds and X^ of gamma_1
// must be in the workspaces first.
struct PersistPlan;
// nb_policy: scenes per table tile of every group, 0 (each group's own
// choice), 1, 2 or 4 (at most what its batch needs).
int persist_build(int ngroups, sfs_operator* const* ops, const PlaneDims* dims, int iters, int nb_policy,
                  PersistPlan** out);
int persist_launch(const PersistPlan* pp, cudaStream_t st);
void persist_free(PersistPlan* pp);
// Time (ms) of the forward-contraction, residual-plane, adjoint-contraction
// and update-plane steps summed over the iterations of the plan's latest run
// (ms8[0..3]), and the mean over CTAs of their busy time in each (ms8[4..7]).
int persist_step_ms(const PersistPlan* pp, double* ms8);

// Batched building blocks (sfs_api.cu) used by the learned network
// (sfs_lista.cu), on the operator's batched workspace:
//   g = A^H (A x - y) for `batch` scenes, y given by bin plane ([batch][U][S];
//   zeros give A^H A x);  scal[b * kNumFloatScalars + kLamMax] = max |A^H y_b|
//   (as float bits, the slots zeroed by the caller);  y -> yplane.
int batch_workspace(sfs_operator* op, int batch);
int batched_normal_residual(sfs_operator* op, int batch, const float2* x, const float2* yplane,
                            float2* g, cudaStream_t st);
int batched_maxabs_AH(sfs_operator* op, int batch, const float2* y, float* scal, cudaStream_t st);
int batched_scatter_y(sfs_operator* op, int batch, const float2* y, float2* yplane, cudaStream_t st);
int operator_device(const sfs_operator* op);

// Small helpers.
int launch_set_thresholds(float* scal, double* red, double lambda, double L,
                          int use_mu, double mu, int* err, cudaStream_t st);
// The same for `batch` scenes: scal + b * kNumFloatScalars (red unused).
int launch_set_thresholds_batched(float* scal, int batch, double lambda, double L, int use_mu,
                                  double mu, int* err, cudaStream_t st);
int launch_randn(float2* v, int n, uint64_t seed, cudaStream_t st);
int launch_sumsq(const float2* v, int n, double* out, cudaStream_t st);
int launch_scale_by_rnorm(float2* v, int n, const double* sumsq, cudaStream_t st);

// Sets the shared-memory attributes of every kernel an operator of shape d
// launches (needed once per device before a stream capture).
int prepare_kernels(const PlaneDims& d);

// Shared memory of the segment-aligned adjoint for Up bins (bytes).
size_t adj_seg_smem_bytes(int Up);

// Opt-in shared memory limit of the current device (bytes).
int max_smem_optin();

}  // namespace sfs
