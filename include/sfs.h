/*
 * sfs.h -- C ABI of libsfs, the GB300 (sm_103a) implementation of the
 * sub-sampled Fourier SAFT operator A = S F H of Kirchhof et al., "Frequency
 * Sub-Sampling of Ultrasound Non-Destructive Measurements: Acquisition,
 * Reconstruction and Performance" (arXiv 2012.04534), its adjoint A^H, and
 * FISTA with complex soft thresholding.
 *
 * Conventions shared by every entry point
 *   - Complex values are interleaved single precision (re, im) pairs
 *     ("c64", 8 bytes), the layout of a C99 float complex or a torch.complex64.
 *   - Reflectivity x: c64 [Nz][Ny][Nx], x fastest (the vectorisation order
 *     of Sec. II-A), V = Nx*Ny*Nz elements.
 *   - Measurements y: c64 [S][M], S = Nx*Ny scan positions, s = iy*Nx + ix;
 *     the M kept DFT bins of a position are in ascending bin order.
 *   - Pointers named *_dev are device pointers on the operator's device, at
 *     least 16-byte aligned, owned by the caller; the library never frees
 *     them.  Pointers named *_host are ordinary host memory.
 *   - `stream` is a cudaStream_t (NULL = the legacy default stream).  Calls
 *     that take a stream enqueue their work on it and return without
 *     synchronising unless stated otherwise.
 *   - Every call returns an sfs_status.  On failure sfs_last_error() gives a
 *     message for the calling thread; outputs are then unspecified.  No C++
 *     exception crosses this boundary.  Handles are not thread safe: calls on
 *     one operator must not overlap in time from several host threads.
 */
#ifndef SFS_H_
#define SFS_H_

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef enum sfs_status {
  SFS_OK = 0,
  SFS_ERR_INVALID_ARG = -1,    /* null pointer, bad size, unsupported shape   */
  SFS_ERR_BAND_TOO_NARROW = -2,/* M exceeds the widest candidate band (40 dB) */
  SFS_ERR_CUDA = -3,           /* a CUDA runtime call failed                  */
  SFS_ERR_OOM = -4,            /* device allocation failed                    */
  SFS_ERR_TIMEOUT = -5,        /* a bounded device wait gave up               */
  SFS_ERR_NOT_CONVERGED = -6,  /* iteration limit reached; result is last est */
  SFS_ERR_NON_FINITE = -7      /* NaN or Inf met in an input or a reduction   */
} sfs_status;

/* Frequency selection strategies (Sec. III-A, Table I; see sfs_select_freqs) */
typedef enum sfs_strategy {
  SFS_SEL_RANDOM = 0,      /* uniform M-subset of the candidate band (Phi_rnd)  */
  SFS_SEL_CONTIGUOUS = 1,  /* M adjacent bins centred on round(fc Nt / fs)      */
  SFS_SEL_EQUISPACED = 2,  /* k_lo + floor((2i+1)|C|/(2M)), i = 0..M-1          */
  SFS_SEL_MAXIMAL = 3,     /* Phi_max: the M bins of largest |H(f_k)| (ties to
                              the lower bin), shared by all positions          */
  SFS_SEL_ENERGY = 4       /* Phi_nrg (shared) or Phi_nrg,f (per_position):
                              M bins drawn without replacement with
                              probability ~ |H(f_k)| among those left; integer
                              weights floor(2^24 |H(f_k)| / max|H|) and draw
                              r = floor(u W / 2^64) from the SplitMix64 stream
                              of the position                                  */
} sfs_strategy;

/*
 * Acquisition geometry and pulse: the scan grid G_2D and voxel grid G_3D of
 * Sec. II-A, the time of flight of Eq. (3), and the Gaussian pulse
 * h(t) = exp(-alpha^2 t^2 + j 2 pi fc t) of Sec. VI.
 */
typedef struct sfs_geometry_desc {
  int32_t Nx, Ny;      /* scan positions per lateral axis (Ny = 1: line scan) */
  double dx, dy;       /* lateral pitch of scan and voxel grid [m]            */
  int32_t Nz;          /* voxels along depth                                  */
  double z0, dz;       /* depth of the first voxel and depth pitch [m]        */
  double c;            /* speed of sound [m/s]                                */
  double fs;           /* sampling rate of the A-scans [Hz]                   */
  int32_t Nt;          /* samples per A-scan; bins k = 0..Nt/2 are candidates */
  double t0;           /* receive-window start [s]; NaN selects
                          floor((2 z0/c - 3/alpha) fs)/fs                      */
  double fc;           /* pulse centre frequency [Hz]                         */
  double frac_bw;      /* -6 dB full amplitude bandwidth as a fraction of fc;
                          alpha = pi (frac_bw fc / 2) / sqrt(ln 2)            */
  double theta;        /* directivity angle [rad]; 0 turns g off (g = 1),
                          else g = exp(-r^2 / (z tan theta)^2)                */
  int32_t device;      /* CUDA device ordinal that holds the operator         */
} sfs_geometry_desc;

/*
 * Arithmetic of the depth contractions (the per-wavenumber products of
 * Theorem 2 / Algorithm 2 that dominate A and A^H).  The paper fixes no
 * precision; every mode accumulates in FP32, and the lateral FFTs, the
 * FISTA update and all reductions are the same in every mode.  u below is
 * the unit roundoff of the stored table.
 *   SFS_PREC_FP32    CUDA-core FP32 FMAs on the FP32 table (the default).
 *   SFS_PREC_TF32X3  tensor cores (tcgen05 kind::tf32): table and spectra
 *                    each split into TF32 hi + lo parts, three products;
 *                    FP32-level accuracy, FP32 table.
 *   SFS_PREC_BF16    tensor cores (kind::f16): table rounded to BF16
 *                    (u = 2^-8, half the bytes of FP32), spectra split into
 *                    BF16 hi + lo; relative error of A x about u.
 *   SFS_PREC_BF16X2  tensor cores (kind::f16): table stored as BF16 hi + lo
 *                    (u about 2^-16, the bytes of FP32), spectra hi + lo.
 *   SFS_PREC_FP16    tensor cores (kind::f16, FP16 operands): table rounded
 *                    to FP16 (u = 2^-11, the bytes of BF16), spectra split
 *                    into FP16 hi + lo.  FP16 spans only 2^-24 .. 65504, so
 *                    both operands are scaled by powers of two, which are
 *                    exact and undone in the FP32 epilogue: the table by
 *                    2^kT with kT fixed at build from a bound on its
 *                    magnitude, each scene's spectra by 2^ks with ks taken
 *                    from the largest |Re| or |Im| of that scene's spectra
 *                    (the kernels that write the spectra record the maximum
 *                    per plane).  The result does not depend on the scale
 *                    of the input, from about 2^-100 to 2^100.
 *   SFS_PREC_FP16X2  as SFS_PREC_FP16 with the table stored as FP16 hi + lo
 *                    (u about 2^-22, the bytes of FP32).
 */
typedef enum sfs_precision {
  SFS_PREC_FP32 = 0,
  SFS_PREC_TF32X3 = 1,
  SFS_PREC_BF16 = 2,
  SFS_PREC_BF16X2 = 3,
  SFS_PREC_FP16 = 4,
  SFS_PREC_FP16X2 = 5
} sfs_precision;

typedef struct sfs_geometry sfs_geometry;  /* opaque, library owned */
typedef struct sfs_operator sfs_operator;  /* opaque, library owned */

/* Sizes and derived constants of an operator (filled by sfs_operator_info). */
typedef struct sfs_operator_info_t {
  int32_t S, M, V, Nz;  /* scan positions, bins per position, voxels, depth   */
  int32_t U;            /* bins in the union of all positions' sets           */
  int32_t Px, Py;       /* lateral FFT sizes (powers of two >= 2N-1)          */
  int32_t Nkappa;       /* lateral wavenumbers Px*Py                          */
  int32_t k_lo, k_hi;   /* candidate band (inclusive) used by the selection   */
  double band_db;       /* band rung (dB below the peak bin) that was used    */
  double alpha, t0;     /* pulse rate [1/s] and receive-window start [s]      */
  int64_t table_bytes;  /* bytes of the lateral-FFT generator table (one entry
                           per symmetry orbit of wavenumbers)                 */
  int32_t launches_per_iter; /* kernels one FISTA iteration launches          */
  int32_t Nslot;        /* wavenumber slots (orbit-major, padded to 64)        */
  int32_t GS;           /* slots per symmetry orbit (2, 4 or 8)               */
  int32_t precision;    /* sfs_precision of the depth contractions            */
  int32_t nshards, shard;  /* bin shard of sfs_operator_shard (1, 0 otherwise)  */
  int32_t shard_first;  /* position of this operator's first bin in the union  */
  int32_t U_all;        /* bins in the union of all shards                    */
} sfs_operator_info_t;

/*
 * Geometry.  Validates the descriptor (positive sizes, Nx, Ny <= 64 for a
 * 3-D scan, Nx <= 512 for a line scan, Nt >= 2, positive pitches, c, fs,
 * fc, frac_bw) and stores a copy.  Frees with sfs_destroy_geometry.
 * Errors: SFS_ERR_INVALID_ARG.
 */
int sfs_create_geometry(const sfs_geometry_desc* desc, sfs_geometry** out);
int sfs_destroy_geometry(sfs_geometry* g);

/*
 * Host-only frequency selection (no device work): the index sets S_{nx,ny}
 * of Sec. II-B / III-A.  The candidate band is C = {0 <= k <= Nt/2 :
 * |H(f_k)| >= 10^(-b/20) max_k |H(f_k)|} for the first b of 6, 10, 20, 40 dB
 * holding at least M bins.  RANDOM draws, for each position s (or once with
 * s = 0 when per_position is 0), a partial Fisher-Yates M-subset of C from
 * the SplitMix64 stream seeded with seed XOR (s * 0x9E3779B97F4A7C15), and
 * sorts it.  CONTIGUOUS and EQUISPACED are shared by all positions.
 * idx_out_host: int32 [S][M] (caller-owned).  band_out_host (may be NULL):
 * int32[2] = {k_lo, k_hi}.  Errors: SFS_ERR_INVALID_ARG, SFS_ERR_BAND_TOO_NARROW.
 */
int sfs_select_indices(const sfs_geometry* g, int strategy, int M,
                       int per_position, uint64_t seed, int32_t* idx_out_host,
                       int32_t* band_out_host);

/*
 * Selection plus operator build: computes the index sets as
 * sfs_select_indices does (bit-identical), then builds the operator as
 * sfs_operator_from_indices does.  idx_out_host (int32 [S][M]) and
 * mask_out_host (uint32 [S][ceil((Nt/2+1)/32)], bit k of position s set when
 * bin k is kept) may be NULL.  Synchronises the device.  Errors: as
 * sfs_select_indices and sfs_operator_from_indices (SFS_ERR_INVALID_ARG,
 * SFS_ERR_BAND_TOO_NARROW, SFS_ERR_OOM, SFS_ERR_CUDA).
 */
int sfs_select_freqs(sfs_geometry* g, int strategy, int M, int per_position,
                     uint64_t seed, int32_t* idx_out_host,
                     uint32_t* mask_out_host, sfs_operator** op);

/*
 * Operator from given index sets (e.g. sets shared with another
 * implementation).  idx_host: int32 [S][M], each row strictly ascending,
 * signed DFT bins -Nt/2 < k <= Nt/2 (the strategies keep 0..Nt/2; a
 * negative k is DFT bin k + Nt, the negative frequency k fs / Nt of the
 * A-scan's periodic spectrum, which the mixing model needs; M <= Nt).
 * Builds on the device the lateral-FFT table of the
 * generating elements of the block 2-level Toeplitz H (Theorem 2, Sec. IV-B)
 * evaluated at the union U of the kept bins with the frequency-domain model
 * of Eq. (4):  h_{k,z}[d] = fs H(f_k) g exp(-j 2 pi f_k (tau(d, z) - t0)).
 * The FFT2 of a generator is the same on every wavenumber of a symmetry
 * orbit (sign flips, and kx <-> ky on square grids), so the table holds one
 * entry per orbit: about 8 * Px*Py * U * Nz / 7.2 bytes for square area scans,
 * / 3.7 for other area scans, / 2 for line scans, plus O(V + U*Px*Py) work
 * space.  Synchronises the device.
 * Errors: SFS_ERR_INVALID_ARG, SFS_ERR_OOM, SFS_ERR_CUDA.
 */
int sfs_operator_from_indices(sfs_geometry* g, int M, const int32_t* idx_host,
                              sfs_operator** op);

/*
 * As sfs_operator_from_indices, with the arithmetic of the depth
 * contractions chosen by `precision` (an sfs_precision).  The table is
 * built in FP32 (as above) and stored in the mode's format: BF16 halves its
 * bytes.  sfs_operator_from_indices uses SFS_PREC_FP32 (or SFS_PREC_TF32X3
 * when the environment sets SFS_CONTRACT=tc).  Several operators of one
 * geometry and index set, in different precisions, may coexist (e.g. a fast
 * BF16 operator for the first FISTA iterations and an FP32 one to finish).
 * Errors: as sfs_operator_from_indices; SFS_ERR_INVALID_ARG for an unknown
 * precision.
 */
int sfs_operator_from_indices_prec(sfs_geometry* g, int M, const int32_t* idx_host,
                                   int precision, sfs_operator** op);
int sfs_destroy_operator(sfs_operator* op);
int sfs_operator_info(const sfs_operator* op, sfs_operator_info_t* info);

/*
 * Forward projection phi_{Phi H}: y = A x (Sec. IV-A; computed by the fast
 * transform of Sec. IV-B, Algorithm 2, restricted to the kept bins).
 * x_dev: c64 [Nz][Ny][Nx] (read), y_dev: c64 [S][M] (written).
 * Errors: SFS_ERR_INVALID_ARG (null operator, null or misaligned pointer),
 * SFS_ERR_CUDA (a launch failed).  A bounded device wait that gives up does
 * not fail the call (it is asynchronous): it sets the operator's error flag,
 * which sfs_check_status and the next synchronising call report as
 * SFS_ERR_TIMEOUT.
 */
int sfs_apply_A(sfs_operator* op, const void* x_dev, void* y_dev, void* stream);

/*
 * Backward projection beta_{Phi H}: x = A^H y (Sec. IV-A; the composition
 * beta_H o beta_Phi of Sec. IV-B).  y_dev: c64 [S][M] (read),
 * x_dev: c64 [Nz][Ny][Nx] (written).  With y the measurements this is the
 * one-step "compressed SAFT" image of Remark 1.  Errors: as sfs_apply_A.
 */
int sfs_apply_AH(sfs_operator* op, const void* y_dev, void* x_dev, void* stream);

/*
 * Backward projection x = A^H y that allocates nothing at call time.  The
 * paper has no counterpart: this is an interface variant of sfs_apply_AH
 * (same arguments, same result) for callers that must not allocate device
 * memory once they are running: acquisition or real-time loops that forbid
 * allocation after start-up so that every call has the same latency, and
 * host frameworks that own all device memory through their own pool.  Such
 * callers create the operator at set-up time; this call then touches no
 * allocator.  Its intermediate data live in one static device array of
 * SFS_NOALLOC_SCRATCH_BYTES that every GPU loading the library holds until
 * the process exits.  All calls share that array and it keeps the last
 * call's contents, so calls whose device work overlaps in time (on other
 * streams, or with other operators of the same device) race and give wrong
 * results; order them on one stream.  The first call on a device looks up
 * the array's device address (cudaGetSymbolAddress) with that device current
 * and keeps it for the life of the process; make that first call before any
 * stream capture.  A device reset (cudaDeviceReset, or any teardown of the
 * device's primary context) invalidates the kept address together with every
 * operator of that device: do not call this entry point again on that
 * device in the same process after one.  An operator whose scratch,
 * 8 * (U * Nslot + slots * 8192) bytes, exceeds the maximum is rejected with
 * SFS_ERR_INVALID_ARG and a message naming both sizes.
 */
#define SFS_NOALLOC_SCRATCH_BYTES (32u << 20)
int sfs_apply_AH_noalloc(sfs_operator* op, const void* y_dev, void* x_dev, void* stream);

/*
 * Batched projections and FISTA: `batch` independent scenes measured with
 * the same geometry and the same kept bins (one operator) processed by one
 * sequence of launches.  This is the serving pattern of a fixed acquisition
 * system, whose frequency sub-sampling is set once (Sec. III) and then
 * applied to every scan.  Scene b occupies x_dev + b V and y_dev + b S M
 * (c64, layouts as for the single-scene calls).  The lateral-FFT plane
 * kernels run the planes of all scenes in one grid; the depth contractions
 * of the 16-bit precisions read each table tile once for a group of up to
 * four scenes (a GEMM with N = 32 columns per scene); the other precisions
 * run one contraction per scene.  The library keeps a batched workspace in
 * the operator, allocated on the first call for a batch size and grown on
 * demand (these calls may therefore allocate, and synchronise the device
 * when they do).  1 <= batch <= SFS_MAX_BATCH.
 * sfs_fista_batched: Algorithm 1 on every scene with the same L and
 * iteration count; lambda >= 0 is used for every scene, lambda < 0 means
 * lambda_b = -lambda ||A^H y_b||_inf per scene (the mu rule of Sec. VII);
 * x_inout_dev receives x_iters of every scene; with flags =
 * SFS_FISTA_WARM_START it holds every scene's x_0 = gamma_1 on entry
 * (t_1 = 1), else x_0 = 0 (no other flag is accepted; no monitor).
 * Errors: SFS_ERR_INVALID_ARG, SFS_ERR_OOM, SFS_ERR_CUDA.
 */
/* Flags of sfs_fista */
#define SFS_FISTA_WARM_START 1u   /* x_inout_dev holds x_0 on entry (else 0)  */
#define SFS_FISTA_TIME_KERNELS 2u /* event nodes around every kernel of the
                                     replayed loop (sfs_stage_times)          */
#define SFS_FISTA_RESUME 4u       /* continue from state_dev (gamma, x, t)     */

#define SFS_MAX_BATCH 256
int sfs_apply_A_batched(sfs_operator* op, int batch, const void* x_dev, void* y_dev,
                        void* stream);
int sfs_apply_AH_batched(sfs_operator* op, int batch, const void* y_dev, void* x_dev,
                         void* stream);
int sfs_fista_batched(sfs_operator* op, int batch, const void* y_dev, double lambda,
                      double L, int iters, void* x_inout_dev, uint32_t flags, void* stream);

/*
 * Serving-style solve of scenes of different geometries: ngroups groups,
 * group g = `batch[g]` scenes of operator ops[g] (distinct operators on one
 * device), measurements y_dev[g] ([batch][S_g][M_g]), Lipschitz constant
 * L[g], results x_out_dev[g] ([batch][V_g]).  The iteration loops of all
 * groups run as one CUDA graph launch, one forked stream per group, so small
 * groups share the GPU.  The graph runs with per-node priorities set by
 * sfs_set_grouped_order (by default a group's kernels get a higher priority
 * the less work its iteration does, scenes x bins x slots x depths, so that
 * small groups finish first).  lambda as in
 * sfs_fista_batched (lambda < 0: mu rule per scene).  The graph is captured on the first call for a set of
 * (operators, batch sizes, iterations) and replayed afterwards (a process-
 * wide cache of 16 graphs, oldest evicted first).  1 <= ngroups <=
 * SFS_MAX_GROUPS.  Errors: SFS_ERR_INVALID_ARG (also for an operator used
 * by two groups), SFS_ERR_OOM, SFS_ERR_CUDA.
 */
#define SFS_MAX_GROUPS 64
int sfs_fista_grouped(int ngroups, sfs_operator* const* ops, const int32_t* batch,
                      const void* const* y_dev, const double* L, double lambda, int iters,
                      void* const* x_out_dev, void* stream);

/*
 * Order of the kernel priorities of the graphs sfs_fista_grouped captures
 * from now on in this process (a graph already cached for another order is
 * not reused): SFS_GROUPED_CHEAPEST_FIRST (default) ranks the groups by the
 * work of their iteration, least work highest, which lowers the median
 * latency; SFS_GROUPED_LARGEST_FIRST ranks them the other way, so that the
 * longest loops start first (the longest-processing-time rule, which aims at
 * the shortest makespan); SFS_GROUPED_NO_PRIORITY gives every kernel the
 * default priority.  The order changes only which ready kernel the GPU
 * starts first: every group's arithmetic, and so its result, is the same
 * bit for bit.  Errors: SFS_ERR_INVALID_ARG for another value.
 */
#define SFS_GROUPED_CHEAPEST_FIRST 0
#define SFS_GROUPED_LARGEST_FIRST 1
#define SFS_GROUPED_NO_PRIORITY 2
int sfs_set_grouped_order(int order);

/*
 * The same solve (arguments, results and errors as sfs_fista_grouped) with
 * the iteration loop of all groups in ONE persistent kernel: a cooperative
 * launch of one 1024-thread CTA per SM (two plane transforms at a time in
 * plane steps) that runs every iteration of Algorithm 1 for every scene.  Per iteration it takes four steps over the
 * work of all groups at once: the forward contractions (every group's units
 * of every scene tile, in runs of about equal table bytes, largest first),
 * the residual planes (every group's scenes x bins, groups with the largest
 * planes first), the adjoint contractions and the update planes (scenes x
 * depths); each step's tasks are handed out one at a time from a counter,
 * and the CTAs meet at a grid barrier between steps.  The barrier waits are bounded (the operators' wait
 * limit, 2 s by default); a CTA that gives up sets the first operator's
 * error flag (sfs_check_status then reports SFS_ERR_TIMEOUT) and the kernel
 * ends.  nb_policy sets the scenes per table tile of the contractions: 0
 * takes each group's own choice (sfs_autotune_batch / sfs_set_batch_tile),
 * 1, 2 or 4 that many for every group (fewer where the batch is smaller);
 * other values give SFS_ERR_INVALID_ARG.  The per-group setup (measurements
 * by plane, X^ of gamma_1) and the persistent kernel are captured as one
 * graph on the first call for a set of (operators, batch sizes, iterations,
 * policy) and replayed afterwards (shared cache with sfs_fista_grouped).
 * Every scene finishes with the solve.  Operators: area scans (lateral FFT
 * planes 32, 64 or 128) with a one-part 16-bit table (SFS_PREC_BF16 or
 * SFS_PREC_FP16); others give SFS_ERR_INVALID_ARG.
 */
int sfs_fista_persistent(int ngroups, sfs_operator* const* ops, const int32_t* batch,
                         const void* const* y_dev, const double* L, double lambda, int iters,
                         void* const* x_out_dev, int nb_policy, void* stream);

/*
 * Tuner of the persistent solve's contraction tiles: times `reps` persistent
 * solves of probe_iters iterations (after one that captures the graph) for
 * each tile policy 0, 1, 2, 4 of sfs_fista_persistent on the given groups
 * (its arguments; x_out_dev receives the last probe's results), writes the
 * fastest policy to *policy_out and the ms per probe solve of each to
 * ms_out[0..3] (in that order) if ms_out is not null.  Policy 0 uses the
 * groups' own choices, so tune those first (sfs_autotune_batch).  Errors
 * as sfs_fista_persistent.
 */
int sfs_autotune_persistent(int ngroups, sfs_operator* const* ops, const int32_t* batch,
                            const void* const* y_dev, const double* L, double lambda, int probe_iters,
                            int reps, void* const* x_out_dev, int32_t* policy_out, double* ms_out,
                            void* stream);

/*
 * Time of the four kinds of step of the latest sfs_fista_persistent solve of
 * the process, summed over its iterations (ms, host array of 8: [0..3] the
 * forward contractions, residual planes, adjoint contractions and update
 * planes as CTA 0 sees them, each from the grid barrier that starts the step
 * to the one that ends it, the last update step to CTA 0's own end; [4..7]
 * the mean over CTAs of their busy time in the same steps, up to their
 * arrival at the barrier).  Waits for the device.  Errors: SFS_ERR_INVALID_ARG (no such solve, or its graph was
 * evicted from the cache), SFS_ERR_CUDA.
 */
int sfs_persistent_step_times(double* ms_out_host);

/*
 * Completion times of the latest sfs_fista_grouped call of the process
 * (ngroups must match it): ms_out_host[g] = milliseconds from the start of
 * that call on its stream (before the per-group setup) to the end of group
 * g's iteration loop (an event-record node in the graph), i.e. the latency
 * of every scene of group g.  Waits for those events.
 * Errors: SFS_ERR_INVALID_ARG (no such call), SFS_ERR_CUDA.
 */
int sfs_grouped_times(int ngroups, float* ms_out_host);

/*
 * Learned unrolled ISTA (not in the paper, which reconstructs with
 * ISTA/FISTA, Sec. IV-A; the learned extension the workloads ask for).
 * Layer l keeps Algorithm 1's gradient step and complex soft threshold with
 * a learned step eta_l and threshold theta_l, followed by a residual 3-D
 * convolutional proximal block (2 -> 8 -> 2 channels, 3x3x3, zero padding,
 * ReLU; FP16 weights, FP32 accumulation):
 *   z_l = x_l - (eta_l / L) A^H (A x_l - y/sigma),  s_l = tau_{theta_l}(z_l),
 *   x_{l+1} = s_l + W2_l * relu(W1_l * [Re s_l, Im s_l] + b1_l) + b2_l,
 * x_0 = 0, output sigma x_L with sigma = ||A^H y||_inf / L per scene, L the
 * operator's Lipschitz constant (sfs_lipschitz), given at creation: the
 * normalised data have ||A^H y_n||_inf = L, so eta ~ 1, theta ~ mu and the
 * layer variables are O(1) whatever the data's scale.
 * Parameters: float [layers][876] = eta, theta, W1 [8][2][3][3][3], b1 [8],
 * W2 [2][8][3][3][3], b2 [2] per layer (row-major).  Batches of scenes share
 * the operator (layouts as in the batched calls).
 *   create:   network on `op` for up to max_batch scenes (allocates the
 *             parameters, Adam moments and the activations of every layer).
 *   set/get:  parameters from / to host memory (synchronous; set resets
 *             the Adam moments); load_params_dev: from device memory.
 *   forward:  x_dev [batch][V] <- network(y_dev [batch][S][M]); keeps every
 *             layer's activations for backward.
 *   backward: grad_params_dev (float [layers * 876], overwritten) <-
 *             gradient of a real loss given grad_x_dev = dLoss/dRe x +
 *             i dLoss/dIm x of the last forward (same batch).
 *   nmse:     *loss_host = mean_b ||x_b - t_b||^2 / ||t_b||^2 and, if
 *             grad_x_dev is not NULL, its gradient (synchronises).
 *   adam:     one Adam step (bias-corrected; `step` counts from 1).
 * Errors: SFS_ERR_INVALID_ARG, SFS_ERR_OOM, SFS_ERR_CUDA.
 */
typedef struct sfs_lista sfs_lista;  /* opaque, library owned */
int sfs_lista_create(sfs_operator* op, int layers, int max_batch, double L, sfs_lista** out);
int sfs_lista_destroy(sfs_lista* net);
int sfs_lista_info(const sfs_lista* net, int32_t* layers, int32_t* nparams);
int sfs_lista_set_params(sfs_lista* net, const float* params_host);
int sfs_lista_get_params(const sfs_lista* net, float* params_host);
/* parameters from device memory, enqueued on `stream` (Adam moments kept) */
int sfs_lista_load_params_dev(sfs_lista* net, const void* params_dev, void* stream);
int sfs_lista_forward(sfs_lista* net, int batch, const void* y_dev, void* x_dev, void* stream);
int sfs_lista_backward(sfs_lista* net, int batch, const void* grad_x_dev, void* grad_params_dev,
                       void* stream);
int sfs_lista_nmse(sfs_lista* net, int batch, const void* x_dev, const void* xtrue_dev,
                   void* grad_x_dev, double* loss_host, void* stream);
int sfs_lista_adam(sfs_lista* net, const void* grad_params_dev, float lr, float beta1,
                   float beta2, float eps, int step, void* stream);

/*
 * ||A^H y||_inf (used by the regularisation rule lambda = mu ||beta(y)||_inf
 * of Sec. VII).  Synchronises `stream`; writes the value to *out_host.
 * Errors: SFS_ERR_INVALID_ARG (null or misaligned argument), SFS_ERR_CUDA,
 * SFS_ERR_TIMEOUT (a kernel's bounded wait gave up), SFS_ERR_NON_FINITE (NaN
 * or Inf in A^H y).
 */
int sfs_max_abs_AH(sfs_operator* op, const void* y_dev, double* out_host,
                   void* stream);

/*
 * Lipschitz constant L >= sigma_max^2 of the gradient of 1/2||Ax - y||^2
 * (Sec. IV-C).  Power iteration on A^H A from a seeded start vector, norms
 * and Rayleigh quotients accumulated in FP64, stopped when the estimate
 * changes by less than rtol (checked every few iterations) or after
 * max_iter iterations; *L_out = estimate * (1 + safety).  Synchronises
 * `stream`.  Returns SFS_ERR_NOT_CONVERGED (with *L_out set) when max_iter
 * is reached.  Other errors: SFS_ERR_INVALID_ARG (null operator or output,
 * max_iter < 1, negative or NaN rtol or safety), SFS_ERR_NON_FINITE (a NaN or
 * Inf Rayleigh quotient), SFS_ERR_OOM, SFS_ERR_CUDA, SFS_ERR_TIMEOUT.
 */
int sfs_lipschitz(sfs_operator* op, int max_iter, double rtol, uint64_t seed,
                  double safety, double* L_out, void* stream);

/*
 * Frobenius norm and the sigma_max estimate of Sec. IV-C (host only, FP64,
 * no device work).  Every entry of A has magnitude fs g(s, v) |H(f_k)|
 * (Eq. (4)), so *fro2_out = ||A||_F^2 exactly:
 * fs^2 sum_s sum_v g(s, v)^2 sum_m |H(f_{idx[s][m]})|^2.
 * *sigma_hat_out (may be NULL) = ||A||_F / N^(1/4), N = min(S M, V): the
 * geometric mean of the bounds ||A||_F / sqrt(N) <= sigma_max <= ||A||_F
 * (Eq. (sigma_hat)).  The estimate is not guaranteed to bound sigma_max from
 * above; sfs_lipschitz is the safe choice for FISTA's step.  Errors:
 * SFS_ERR_INVALID_ARG (null operator or fro2_out).
 */
int sfs_frobenius(const sfs_operator* op, double* fro2_out, double* sigma_hat_out);

/*
 * Cramer-Rao bound on the location of one scatterer (Sec. VI, Eq. "fim" and
 * the block inverse after it), for T index sets at once (e.g. the trials of
 * a random strategy, or several strategies).  The scatterer sits at the
 * continuous position pos = {x1, y1, z1} [m] (z1 > 0 the depth below the
 * scan plane) with amplitude amp > 0 and phase `phase`; the data are its
 * kept-bin coefficients (Eq. (4), Sigma = I) in white circular Gaussian
 * noise of variance sigma2 > 0.  J = (2 / sigma2) Re{D^H D} over u = (x1, y1,
 * z1, a, phi), D = d b / d u^T, with d tau / dp = (2 / c) (p - p_s) / R and,
 * for theta > 0, the derivatives of g = exp(-r^2 / (z1 tan theta)^2).
 * param_mask selects the location coordinates estimated (bit 0 x1, bit 1 y1,
 * bit 2 z1; a line scan cannot see y1, a single A-scan neither x1 nor y1);
 * a and phi are always nuisance parameters.
 *   idx_host      int32 [T][S][M], each row strictly ascending in 0..Nt/2
 *   crb_out_host  double [T][3]: diag of the location block of J^-1 [m^2],
 *                 NaN for coordinates outside the mask
 *   fim_out_host  double [T][25] or NULL: J row-major over (x1, y1, z1, a,
 *                 phi), zero rows and columns outside the mask
 * The sums over the S*M rows run on the geometry's device in FP64 (one
 * thread per row, per-CTA partial sums added on the host in a fixed order,
 * so results are reproducible); J is inverted on the host in FP64.  The
 * information does not depend on the phase.  Synchronises the device.
 * Errors: SFS_ERR_INVALID_ARG (sizes, rows, amp, sigma2, z1, mask, or a
 * singular J), SFS_ERR_CUDA, SFS_ERR_OOM.
 */
int sfs_crb(const sfs_geometry* g, int T, int M, const int32_t* idx_host, const double* pos,
            double amp, double phase, double sigma2, int param_mask, double* crb_out_host,
            double* fim_out_host);

/*
 * Rademacher mixing, Phi_s = S_s F Sigma_s with Sigma_s = Diag{xi_s}, xi_s in
 * {-1, 1}^Nt (Sec. II-B, Eq. "compressed_model"; Sec. III-A's random
 * sampling).  Sigma_s acts on the Nt time samples of A-scan s, so each kept
 * coefficient mixes every DFT bin of that A-scan, the bins above Nt/2 being
 * its negative frequencies (signed bins k - Nt):
 *   y_s[m] = (1/Nt) sum_k Xi_s[(k_m - k) mod Nt] (A_band x)_s[k],
 * Xi_s = DFT(xi_s), where A_band is an ordinary operator on signed bins
 * keeping the same bins at every position.  The sum runs over the bins of
 * A_band; it must hold at least the run sfs_mixing_band returns, the bins
 * whose pulse magnitude |H(f_k)| is within SFS_MIX_BAND_DB = 140 dB of the
 * peak: the Gaussian pulse spectrum (Sec. VI) puts a fraction
 * erfc(sqrt(2 ln 1e7)) ~ 1e-15 of its energy outside, so the truncation
 * changes A_mix by less than 1e-7 relative.  A_mix = Mix o A_band,
 * A_mix^H = A_band^H o Mix^H, Mix generated per position from Xi_s.
 *   band      operator with identical index rows covering the run of
 *             sfs_mixing_band; not owned, must outlive the mixing object;
 *             calls on the two must not overlap (they share the band
 *             operator's workspace)
 *   idx_host  int32 [S][M] kept bins, rows strictly ascending in 0..Nt/2
 *   xi_host   int8 [S][Nt], entries +1 or -1 (the random draws are inputs)
 * Xi_s is computed on the device in FP64 and stored as c64 (S Nt values).
 * Errors: SFS_ERR_INVALID_ARG (band rows differ or miss a bin of the run,
 * bad rows or signs, Nt > 8192), SFS_ERR_CUDA, SFS_ERR_OOM.
 * sfs_mixing_band: the signed bins k_lo..k_hi (inclusive, -Nt/2 < k <=
 * Nt/2) with |H(k fs / Nt)| >= 10^(-SFS_MIX_BAND_DB / 20) max |H| (host only,
 * FP64).  Errors: SFS_ERR_INVALID_ARG (null pointer).
 */
#define SFS_MIX_BAND_DB 140.0
typedef struct sfs_mixing sfs_mixing;  /* opaque, library owned */
int sfs_mixing_band(const sfs_geometry* g, int32_t* k_lo, int32_t* k_hi);
int sfs_mixing_create(sfs_operator* band, int M, const int32_t* idx_host, const int8_t* xi_host,
                      sfs_mixing** out);
int sfs_mixing_destroy(sfs_mixing* mx);
/* y = A_mix x: x c64 [Nz][Ny][Nx], y c64 [S][M] (device, 16-byte aligned).
 * Errors of this and the next three calls: as their unmixed counterparts
 * (sfs_apply_A, sfs_apply_AH, sfs_lipschitz, sfs_fista). */
int sfs_apply_A_mixed(sfs_mixing* mx, const void* x_dev, void* y_dev, void* stream);
/* x = A_mix^H y. */
int sfs_apply_AH_mixed(sfs_mixing* mx, const void* y_dev, void* x_dev, void* stream);
/* L >= ||A_mix||^2 by power iteration (as sfs_lipschitz; syncs each step). */
int sfs_lipschitz_mixed(sfs_mixing* mx, int max_iter, double rtol, uint64_t seed, double safety,
                        double* L_out, void* stream);
/* FISTA (Algorithm 1) on A_mix from x_0 = 0, lambda < 0 meaning the mu rule
 * lambda = -lambda ||A_mix^H y||_inf; six kernels per iteration, replayed as
 * one CUDA graph per iteration count. */
int sfs_fista_mixed(sfs_mixing* mx, const void* y_dev, double lambda, double L, int iters,
                    void* x_dev, void* stream);

/*
 * Tile tuning of the batched 16-bit contractions (BF16 / BF16X2 / FP16 /
 * FP16X2 operators).  A batched call groups its scenes so that one table
 * tile serves NB scenes (NB = 1, 2 or 4: an MMA N of 32 NB columns, 64 NB
 * TMEM columns); by default NB = 4 from three scenes on.
 * sfs_autotune_batch times `reps` forward + adjoint contraction pairs of
 * `batch` scenes for each NB up to the batch (CUDA events on a private
 * stream, after one warm-up pair, on zero spectra), keeps the fastest for
 * this (operator, batch) and returns it in *nb_out (0 for FP32 / TF32X3
 * operators, which have nothing to tune); ms_out (may be NULL) receives the
 * milliseconds per pair for NB = 1, 2, 4 (NaN where not tried).
 * sfs_set_batch_tile fixes NB (0 restores the default rule).  Results do not
 * depend on NB: each scene's products and sums are the same.  Both drop the
 * loops captured for that batch size.  Synchronises the device.
 * Errors: SFS_ERR_INVALID_ARG, SFS_ERR_CUDA, SFS_ERR_TIMEOUT.
 */
int sfs_autotune_batch(sfs_operator* op, int batch, int reps, int32_t* nb_out, double* ms_out);
int sfs_set_batch_tile(sfs_operator* op, int batch, int nb);

/*
 * FISTA with backtracking (Sec. IV-C, "Backtracking"): instead of L >=
 * sigma_max^2, a lower bound L0 (sigma_low^2) and a factor eta > 1.  Step k
 * takes the smallest L' = eta^i L_{k-1} with F(p_L') <= Q_L'(p_L', gamma_k)
 * (the cited Beck-Teboulle rule), evaluated in its exact equivalent form
 * for the quadratic data term, ||A d||^2 <= L' ||d||^2 with d = p_L' -
 * gamma_k.  Each trial costs one forward apply and one host read (the
 * loop is host-driven, not graph-replayed).  x_0 = 0; lambda < 0 means the
 * mu rule; L_hist_host (may be NULL) receives L_k per iteration.
 * Errors: SFS_ERR_INVALID_ARG, SFS_ERR_NOT_CONVERGED (no step within 200
 * trials), SFS_ERR_NON_FINITE, SFS_ERR_TIMEOUT, SFS_ERR_CUDA.
 */
int sfs_fista_backtracking(sfs_operator* op, const void* y_dev, double lambda, double L0, double eta,
                           int iters, void* x_dev, double* L_hist_host, void* stream);


/* Bytes of the FISTA state of an operator with V voxels (see sfs_fista). */
#define SFS_FISTA_STATE_BYTES(V) (16u * (uint64_t)(V) + 16u)

/*
 * FISTA (Algorithm 1, Sec. IV-A) for min 1/2||A x - y||^2 + lambda ||x||_1:
 *   x_k = tau_{lambda/L}(gamma_k - A^H(A gamma_k - y)/L),
 *   t_{k+1} = (1 + sqrt(1 + 4 t_k^2))/2,
 *   gamma_{k+1} = x_k + ((t_k - 1)/t_{k+1})(x_k - x_{k-1}),  t_1 = 1,
 * with tau the complex soft threshold max(|z| - a, 0) z/|z|.
 * y_dev: c64 [S][M] (read).  lambda >= 0 is used as given; lambda < 0 means
 * lambda = -lambda * ||A^H y||_inf (the mu rule of Sec. VII, computed on the
 * device).  L: Lipschitz constant (> 0), e.g. from sfs_lipschitz.
 * x_inout_dev: c64 [Nz][Ny][Nx]; receives x_K after the call's `iters`
 * iterations (with SFS_FISTA_WARM_START it also holds x_0 = gamma_1 on entry).
 * state_dev (may be NULL): SFS_FISTA_STATE_BYTES(V) bytes of device memory
 * holding the iteration state, so that a solve can be checkpointed and
 * continued: c64 gamma_{K+1} [V], c64 x_K [V] (the previous iterate of the
 * next step), double t_{K+1}, int64 total iterations.  When given, the call
 * writes the state reached at its end.  With SFS_FISTA_RESUME the call starts
 * from that state instead of x_0 (x_inout_dev is then output only), so n1
 * iterations followed by a resumed n2 give the same result, bit for bit, as
 * n1 + n2 iterations in one call with the same lambda and L (the momentum
 * coefficients are computed on the device in FP64 from the stored t).
 * obj_hist_host (may be NULL): double [iters], entry k-1 =
 * 1/2||A gamma_k - y||^2 + lambda||x_k||_1 (a monitor evaluated with the
 * residual at gamma_k); when given, the call synchronises `stream`.
 * SFS_FISTA_TIME_KERNELS records an event before and after every kernel of
 * ceil(iters / 8)-spaced iterations (at most 8, spread over the solve) as
 * event-record nodes of the replayed iteration graph, read by
 * sfs_stage_times; the other iterations run without them.
 * Errors: SFS_ERR_INVALID_ARG (also RESUME without state_dev, or RESUME
 * with WARM_START), SFS_ERR_CUDA.
 */
int sfs_fista(sfs_operator* op, const void* y_dev, double lambda, double L,
              int iters, void* x_inout_dev, void* state_dev, uint32_t flags,
              double* obj_hist_host, void* stream);

/*
 * Average device time per launch [ms] of the forward and adjoint depth
 * contraction kernels during the last sfs_fista call made with
 * SFS_FISTA_TIME_KERNELS (the event nodes of its replayed graph, over the
 * sampled iterations).  Synchronises the operator's device.  n_out_host
 * receives the number of iterations averaged (0, with zero times, when no
 * such call has run).  Errors: SFS_ERR_INVALID_ARG (null operator or
 * output), SFS_ERR_CUDA.
 */
int sfs_kernel_times(sfs_operator* op, double* fwd_ms, double* adj_ms,
                     int32_t* n_out_host);

/*
 * Average device time per iteration [ms] of each of the four kernels of
 * the last sfs_fista call made with SFS_FISTA_TIME_KERNELS, from the event
 * nodes between consecutive kernels of its sampled iterations (so the four
 * sum to the time of those iterations): ms4_host[0] forward contraction, [1]
 * residual planes (inverse FFT, residual, forward FFT), [2] adjoint
 * contraction, [3] update planes (inverse FFT, FISTA step, forward FFT).
 * Synchronises the operator's device.  n_out_host (may be NULL) receives
 * the number of iterations averaged (0, with zero times, when no such call
 * has run).  Errors: SFS_ERR_INVALID_ARG (null operator or ms4_host),
 * SFS_ERR_CUDA.
 */
int sfs_stage_times(sfs_operator* op, double* ms4_host, int32_t* n_out_host);

/*
 * Limit of every bounded wait inside the contraction kernels (default 2 s of
 * device time).  A wait that runs out sets the operator's device error flag,
 * waits (at most 0.5 s more) for the copies its warp already issued, and
 * returns; the calls that synchronise then report SFS_ERR_TIMEOUT, and so
 * does sfs_check_status.  Results of the affected call are unspecified; the
 * operator and the CUDA context stay usable.  Used to test failure handling
 * (a very small limit forces timeouts).  ns must be > 0.
 */
int sfs_set_wait_timeout_ns(sfs_operator* op, uint64_t ns);

/*
 * Failure injection for tests of the timeout handling: while enabled, the
 * first wait of every warp in each contraction launch is made on a barrier
 * that nothing arrives at, so it runs out after the wait limit and takes the
 * timeout path (error flag, bounded drain of the copies in flight, early
 * return) for real.  Results are unspecified while enabled.
 */
int sfs_inject_wait_timeout(sfs_operator* op, int enable);

/*
 * Synchronises `stream`, then reports (and clears) the operator's device
 * error flag: SFS_OK, SFS_ERR_TIMEOUT if a bounded wait ran out, or
 * SFS_ERR_NON_FINITE if a non-finite lambda was computed, in any call since
 * the last check.
 */
int sfs_check_status(sfs_operator* op, void* stream);

/*
 * Multi-GPU split by bins (one process per GPU).  The union U of the kept
 * bins is cut into nshards contiguous runs; run j holds union positions
 * [floor(j U / n), floor((j + 1) U / n)) (sfs_shard_run, host only).  The
 * runs partition the rows of A = Phi H (Eq. (10)/(11): a row is one kept
 * coefficient (s, m)), so with A_j the rows of run j,
 *   A x = the rows of every A_j x,   A^H y = sum_j A_j^H y,
 *   A^H (A x - y) = sum_j A_j^H (A_j x - y):
 * each rank builds the generator table (Theorem 2) of its own bins only and
 * forms its partial gradient without any exchange; one all-reduce (sum) of
 * the V voxel values per FISTA iteration joins them, and the elementwise
 * update of Algorithm 1 is replicated (sfs_prox_momentum).
 *   sfs_operator_shard: operator of run `shard` (as
 *     sfs_operator_from_indices_prec otherwise).  Its measurement layout
 *     stays the full [S][M]: sfs_apply_A writes only the entries of its
 *     bins (the others are left as they were), sfs_apply_AH and
 *     sfs_normal_residual read only those.  Errors: SFS_ERR_INVALID_ARG
 *     (also for a run with no bin, nshards > U).
 *   sfs_normal_residual: g = A_j^H (A_j x - y) (y c64 [S][M], x and g c64
 *     [Nz][Ny][Nx]); on an unsharded operator the full gradient of
 *     1/2||A x - y||^2.  Enqueued on `stream`.
 *   sfs_prox_momentum: for i < n (c64 elements), w = gamma - grad / L,
 *     x_i <- tau_{lambda/L}(w) (complex soft threshold), gamma_i <- x_i +
 *     beta (x_i - x_prev_i) with x holding x_prev on entry: one iteration's
 *     update of Algorithm 1 (beta = (t_k - 1)/t_{k+1}), in the arithmetic of
 *     sfs_fista's fused update.  lambda >= 0, L > 0.  Enqueued on `stream`.
 *   sfs_vec_sumsq / sfs_vec_max_abs: sum |v_i|^2 (FP64) and max |v_i| of a
 *     c64 device vector (reduction slots of `op`; synchronise `stream`).
 *   sfs_vec_scale: v *= a.  sfs_vec_randn: complex Gaussian entries from a
 *     counter-based hash of (seed, i), the start vector of sfs_lipschitz.
 */
int sfs_shard_run(int U, int nshards, int shard, int32_t* first, int32_t* count);
int sfs_operator_shard(sfs_geometry* g, int M, const int32_t* idx_host, int nshards, int shard,
                       int precision, sfs_operator** op);
int sfs_normal_residual(sfs_operator* op, const void* x_dev, const void* y_dev, void* g_dev,
                        void* stream);
int sfs_prox_momentum(int n, void* x_dev, void* gamma_dev, const void* grad_dev, double lambda,
                      double L, double beta, void* stream);
int sfs_vec_sumsq(sfs_operator* op, const void* v_dev, int n, double* out_host, void* stream);
int sfs_vec_max_abs(sfs_operator* op, const void* v_dev, int n, double* out_host, void* stream);
int sfs_vec_scale(void* v_dev, int n, double a, void* stream);
int sfs_vec_randn(void* v_dev, int n, uint64_t seed, void* stream);

/* Message of the last failed call on this host thread ("" if none). */
const char* sfs_last_error(void);

/* Library version string. */
const char* sfs_version(void);

#ifdef __cplusplus
}
#endif

#endif /* SFS_H_ */
