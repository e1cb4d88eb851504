// Host side of libsfs: the C ABI of include/sfs.h.
//
// Geometry and pulse constants are computed on the host in FP64 (Sec. II-A,
// Eq. (3); pulse of Sec. VI).  The frequency selection (Sec. III-A) is
// integer work on the host.  Everything on the operator's data path runs in
// the device kernels of sfs_kernels.cu; this file only sizes buffers,
// validates arguments, and enqueues launches on the caller's stream.
#include <cuda_runtime.h>
#include <math.h>
#include <stdarg.h>
#include <stdio.h>
#include <string.h>

#include <algorithm>
#include <atomic>
#include <mutex>
#include <new>
#include <string>
#include <vector>

#include "sfs_internal.h"
#include "sfs_launch.h"

namespace sfs {

static thread_local std::string g_last_error;

void set_error(const char* fmt, ...) {
  char buf[1024];
  va_list ap;
  va_start(ap, fmt);
  vsnprintf(buf, sizeof(buf), fmt, ap);
  va_end(ap);
  g_last_error = buf;
}

void clear_error() { g_last_error.clear(); }

int cuda_fail(cudaError_t e, const char* what, const char* file, int line) {
  set_error("%s failed: %s (%s:%d)", what, cudaGetErrorString(e), file, line);
  cudaGetLastError();  // clear a non-sticky error so later calls do not report it
  return e == cudaErrorMemoryAllocation ? SFS_ERR_OOM : SFS_ERR_CUDA;
}

namespace {

// Sets the operator's device for the scope of an API call and restores the
// caller's current device afterwards.
class DeviceScope {
 public:
  explicit DeviceScope(int dev) {
    if (cudaGetDevice(&prev_) != cudaSuccess) prev_ = -1;
    ok_ = cudaSetDevice(dev) == cudaSuccess;
  }
  ~DeviceScope() {
    if (prev_ >= 0) cudaSetDevice(prev_);
  }
  bool ok() const { return ok_; }

 private:
  int prev_ = -1;
  bool ok_ = false;
};

int next_pow2(int v) {
  int p = 1;
  while (p < v) p <<= 1;
  return p;
}

double pulse_alpha(double fc, double frac_bw) {
  return M_PI * (0.5 * frac_bw * fc) / sqrt(log(2.0));
}

// SplitMix64 (Steele, Lea, Flood 2014): Weyl increment plus the 64-bit mixer.
struct SplitMix64 {
  uint64_t s;
  uint64_t next() {
    s += 0x9E3779B97F4A7C15ull;
    uint64_t z = s;
    z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
    z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
    return z ^ (z >> 31);
  }
};

constexpr double kBandLadderDb[4] = {6.0, 10.0, 20.0, 40.0};

int candidate_band(const sfs_geometry* g, int M, int* k_lo, int* k_hi, double* db) {
  const int nb = g->d.Nt / 2 + 1;
  std::vector<double> mag(nb);
  double peak = 0.0;
  for (int k = 0; k < nb; ++k) {
    mag[k] = pulse_mag((double)k * g->d.fs / g->d.Nt, g->d.fc, g->alpha);
    peak = std::max(peak, mag[k]);
  }
  for (double b : kBandLadderDb) {
    const double thr = peak * pow(10.0, -b / 20.0);
    int lo = -1, hi = -1, n = 0;
    for (int k = 0; k < nb; ++k)
      if (mag[k] >= thr) {
        if (lo < 0) lo = k;
        hi = k;
        ++n;
      }
    if (n >= M) {
      *k_lo = lo;
      *k_hi = hi;
      *db = b;
      return SFS_OK;
    }
  }
  set_error("M = %d exceeds the 40 dB band of the pulse", M);
  return SFS_ERR_BAND_TOO_NARROW;
}

// Relative pulse magnitudes e_k = |H(f_k)| / max |H| = exp(-(pi (f_k - fc) /
// alpha)^2) of the bins k = 0..Nt/2 and the integer weights floor(2^24 e_k)
// of the energy-based draw (Sec. III-A, q_i = |hat h_i| / ||hat h||_1).
void pulse_weights(const sfs_geometry* g, std::vector<double>& e, std::vector<int64_t>& w) {
  const int nb = g->d.Nt / 2 + 1;
  e.resize(nb);
  w.resize(nb);
  for (int k = 0; k < nb; ++k) {
    const double a = M_PI * ((double)k * g->d.fs / g->d.Nt - g->d.fc) / g->alpha;
    e[k] = exp(-a * a);
    w[k] = (int64_t)floor(e[k] * 16777216.0);
  }
}

int select_host(const sfs_geometry* g, int strategy, int M, int per_position, uint64_t seed,
                int32_t* idx, int* k_lo_out, int* k_hi_out, double* db_out) {
  if (M <= 0) {
    set_error("M must be positive (got %d)", M);
    return SFS_ERR_INVALID_ARG;
  }
  int k_lo, k_hi;
  double db;
  const int S = g->d.Nx * g->d.Ny;
  if (strategy == SFS_SEL_MAXIMAL || strategy == SFS_SEL_ENERGY) {
    // Phi_max and Phi_nrg(,f) of Sec. III-A draw from all bins 0..Nt/2
    std::vector<double> e;
    std::vector<int64_t> w;
    pulse_weights(g, e, w);
    const int nb = (int)e.size();
    int nonzero = 0;
    for (int64_t v : w) nonzero += v > 0;
    if (M > (strategy == SFS_SEL_MAXIMAL ? nb : nonzero)) {
      set_error("M = %d exceeds the %d bins that carry pulse energy", M,
                strategy == SFS_SEL_MAXIMAL ? nb : nonzero);
      return SFS_ERR_BAND_TOO_NARROW;
    }
    const int rows = (strategy == SFS_SEL_ENERGY && per_position) ? S : 1;
    for (int s = 0; s < rows; ++s) {
      std::vector<int> pick;
      if (strategy == SFS_SEL_MAXIMAL) {
        std::vector<int> order(nb);
        for (int k = 0; k < nb; ++k) order[k] = k;
        std::stable_sort(order.begin(), order.end(), [&](int a, int b) { return e[a] > e[b]; });
        pick.assign(order.begin(), order.begin() + M);
      } else {
        std::vector<int64_t> ww = w;
        SplitMix64 rng{seed ^ ((uint64_t)s * 0x9E3779B97F4A7C15ull)};
        for (int n = 0; n < M; ++n) {
          uint64_t W = 0;
          for (int64_t v : ww) W += (uint64_t)v;
          const uint64_t r = (uint64_t)(((unsigned __int128)rng.next() * W) >> 64);
          uint64_t c = 0;
          for (int k = 0; k < nb; ++k) {
            c += (uint64_t)ww[k];
            if (c > r) {
              pick.push_back(k);
              ww[k] = 0;
              break;
            }
          }
        }
      }
      std::sort(pick.begin(), pick.end());
      for (int m = 0; m < M; ++m) idx[(size_t)s * M + m] = pick[m];
    }
    for (int s = rows; s < S; ++s) memcpy(idx + (size_t)s * M, idx, sizeof(int32_t) * M);
    // the band is reported when it exists; otherwise the span of the sets
    if (candidate_band(g, M, &k_lo, &k_hi, &db) != SFS_OK) {
      clear_error();
      k_lo = *std::min_element(idx, idx + (size_t)S * M);
      k_hi = *std::max_element(idx, idx + (size_t)S * M);
      db = NAN;
    }
    if (k_lo_out) *k_lo_out = k_lo;
    if (k_hi_out) *k_hi_out = k_hi;
    if (db_out) *db_out = db;
    return SFS_OK;
  }
  SFS_TRY(candidate_band(g, M, &k_lo, &k_hi, &db));
  const int n = k_hi - k_lo + 1;
  switch (strategy) {
    case SFS_SEL_RANDOM: {
      std::vector<int> perm(n);
      const int rows = per_position ? S : 1;
      for (int s = 0; s < rows; ++s) {
        for (int i = 0; i < n; ++i) perm[i] = i;
        SplitMix64 rng{seed ^ ((uint64_t)s * 0x9E3779B97F4A7C15ull)};
        for (int i = 0; i < M; ++i) {
          const uint64_t hi32 = rng.next() >> 32;
          const int j = i + (int)((hi32 * (uint64_t)(n - i)) >> 32);
          std::swap(perm[i], perm[j]);
        }
        std::sort(perm.begin(), perm.begin() + M);
        for (int m = 0; m < M; ++m) idx[(size_t)s * M + m] = k_lo + perm[m];
      }
      if (!per_position)
        for (int s = 1; s < S; ++s) memcpy(idx + (size_t)s * M, idx, sizeof(int32_t) * M);
      break;
    }
    case SFS_SEL_CONTIGUOUS: {
      const int kstar = (int)floor(g->d.fc * g->d.Nt / g->d.fs + 0.5);
      const int start = std::min(std::max(kstar - M / 2, k_lo), k_hi - M + 1);
      for (int s = 0; s < S; ++s)
        for (int m = 0; m < M; ++m) idx[(size_t)s * M + m] = start + m;
      break;
    }
    case SFS_SEL_EQUISPACED: {
      for (int s = 0; s < S; ++s)
        for (int m = 0; m < M; ++m)
          idx[(size_t)s * M + m] = k_lo + (int)(((2LL * m + 1) * n) / (2LL * M));
      break;
    }
    default:
      set_error("unknown selection strategy %d", strategy);
      return SFS_ERR_INVALID_ARG;
  }
  if (k_lo_out) *k_lo_out = k_lo;
  if (k_hi_out) *k_hi_out = k_hi;
  if (db_out) *db_out = db;
  return SFS_OK;
}

template <typename T>
int dev_alloc(T** p, size_t count) {
  *p = nullptr;
  if (count == 0) count = 1;
  SFS_CUDA(cudaMalloc((void**)p, count * sizeof(T)));
  return SFS_OK;
}

// Batched workspace and the loops captured on it.
void free_batch(sfs_operator* op) {
  sfs::BatchWorkspace& w = op->bws;
  for (auto& ge : op->bgraphs) cudaGraphExecDestroy(ge.exec);
  op->bgraphs.clear();
  cudaFree(w.Xh);
  cudaFree(w.Yh);
  cudaFree(w.Rh);
  cudaFree(w.Gh);
  cudaFree(w.xk);
  cudaFree(w.gam);
  cudaFree(w.yplane);
  cudaFree(w.ybuf);
  cudaFree(w.scal);
  cudaFree(w.pmx);
  cudaFree(w.pmr);
  w = sfs::BatchWorkspace();
}

void free_operator(sfs_operator* op) {
  if (!op) return;
  cudaFree(op->table);
  cudaFree(op->posmap);
  cudaFree(op->ws.Xh);
  cudaFree(op->ws.Yh);
  cudaFree(op->ws.Rh);
  cudaFree(op->ws.Gh);
  cudaFree(op->ws.segslot);
  cudaFree(op->slot_kappa);
  cudaFree(op->quad);
  cudaFree(op->orbit_rep);
  cudaFree(op->ws.err);
  cudaFree(op->ws.xk);
  cudaFree(op->ws.gam);
  cudaFree(op->ws.ybuf);
  cudaFree(op->ws.yplane);
  cudaFree(op->ws.vbuf);
  cudaFree(op->ws.scal);
  cudaFree(op->ws.red);
  cudaFree(op->ws.obj);
  cudaFree(op->ws.beta);
  cudaFree(op->ws.tnext);
  cudaFree(op->ws.pmx);
  cudaFree(op->ws.pmr);
  for (cudaEvent_t e : op->ev) cudaEventDestroy(e);
  for (auto& ge : op->graphs) cudaGraphExecDestroy(ge.exec);
  if (op->capture_stream) cudaStreamDestroy(op->capture_stream);
  free_tc_maps(op->tmaps);
  free_batch(op);
  delete op;
}

}  // namespace

PlaneDims operator_dims(const sfs_operator* op) {
  PlaneDims d;
  d.Nx = op->geo.d.Nx;
  d.Ny = op->geo.d.Ny;
  d.Nz = op->geo.d.Nz;
  d.Px = op->geo.Px;
  d.Py = op->geo.Py;
  d.Nk = op->Nk;
  d.S = op->S;
  d.M = op->M;
  d.U = op->U;
  d.nzb = op->nzb;
  d.G = op->G;
  d.Ns = op->Ns;
  d.GS = op->GS;
  d.Up = op->Up;
  d.tc = op->tc;
  d.nzc = op->nzc;
  d.prec = op->prec;
  d.nkb = op->nkb;
  d.nparts = op->nparts;
  d.f16 = op->f16;
  d.tscale = ldexpf(1.0f, op->tscale_exp);
  d.tinv = ldexpf(1.0f, -op->tscale_exp);
  d.pm_x = op->f16 ? op->ws.pmx : nullptr;
  d.pm_r = op->f16 ? op->ws.pmr : nullptr;
  d.bs_pmx = op->geo.d.Nz;
  d.bs_pmr = op->Up;
  d.tmaps = op->tmaps;
  d.adj_seg = op->adj_seg;
  d.azb = op->azb;
  d.anzb = op->anzb;
  d.Ga = op->Ga;
  d.wait_ns = op->wait_ns;
  d.stream_table = op->stream_table;
  d.inject = op->inject;
  d.slot_kappa = op->slot_kappa;
  d.orbit_rep = op->orbit_rep;
  d.quad = op->quad;
  d.batch = 1;
  d.nb = 0;
  d.bs_x = op->V;
  d.bs_xh = (long long)op->geo.d.Nz * op->Ns;
  d.bs_yh = (long long)op->nzb * op->Up * op->Ns;
  d.bs_rh = (long long)op->Up * op->Ns;
  d.bs_gh = (long long)op->nslots * op->azb * kKappaTile;
  d.bs_y = (long long)op->S * op->M;
  d.bs_yplane = (long long)op->U * op->S;
  d.bs_scal = kNumFloatScalars;
  d.bs_red = 0;
  return d;
}

namespace {

PlaneDims dims_of(const sfs_operator* op) { return operator_dims(op); }

// Generator table size in c64 entries.  CUDA-core layout: depth pairs of
// Nz rounded up to even, Up rows per slot tile of 64; tf32 tensor-core
// layout: 16-depth blocks, U rows per orbit; 16-bit layout: per part, orbit
// and 32-depth block, U rows of 64 16-bit values (128 B).
size_t table_c64(const sfs_operator* op) {
  const size_t No = (size_t)(op->Ns / op->GS);
  if (op->tc == 2) return (size_t)op->nparts * No * op->nkb * op->U * 16;  // 128 B per row
  if (op->tc) return No * op->nzc * 16 * op->U;
  return No * op->Up * (size_t)((op->geo.d.Nz + 1) / 2 * 2);
}

bool aligned16(const void* p) { return ((uintptr_t)p & 15u) == 0; }

// y = A x on `st` (x, y device pointers)
int enqueue_A(sfs_operator* op, const float2* x, float2* y, double* red_sumsq, cudaStream_t st) {
  const PlaneDims d = dims_of(op);
  SFS_TRY(launch_fwd_planes(d, x, op->ws.Xh, st));
  SFS_TRY(launch_contract_fwd(d, op->table, op->ws.Xh, op->ws.Yh, op->ws.err, st));
  SFS_TRY(launch_inv_gather(d, op->ws.Yh, op->posmap, y, red_sumsq, st));
  return SFS_OK;
}

// x = A^H y on `st`; x may be null when only the reductions are wanted
int enqueue_AH(sfs_operator* op, const float2* y, float2* x, double* red_sumsq,
               unsigned int* maxabs_bits, cudaStream_t st) {
  const PlaneDims d = dims_of(op);
  SFS_TRY(launch_scatter_fwd(d, y, op->posmap, op->ws.Rh, st));
  SFS_TRY(launch_contract_adj(d, op->table, op->ws.Rh, op->ws.Gh, op->ws.err, st));
  SFS_TRY(launch_inv_store(d, op->ws.Gh, op->ws.segslot, x, red_sumsq, maxabs_bits, st));
  return SFS_OK;
}

int ensure_obj(sfs_operator* op, int iters) {
  if (op->ws.obj_cap >= iters) return SFS_OK;
  // graphs that recorded the old monitor buffer become invalid
  for (auto it = op->graphs.begin(); it != op->graphs.end();) {
    if (it->with_obj) {
      cudaGraphExecDestroy(it->exec);
      it = op->graphs.erase(it);
    } else {
      ++it;
    }
  }
  cudaFree(op->ws.obj);
  op->ws.obj = nullptr;
  op->ws.obj_cap = 0;
  SFS_TRY(dev_alloc(&op->ws.obj, 2 * (size_t)iters));
  op->ws.obj_cap = iters;
  return SFS_OK;
}

// Device momentum table for `iters` iterations (grown on demand; loops
// captured on the old table are dropped) and the t_{k+1} slot.
int ensure_beta(sfs_operator* op, int iters) {
  if (!op->ws.tnext) SFS_TRY(dev_alloc(&op->ws.tnext, 2));
  if (op->ws.beta_cap >= iters) return SFS_OK;
  for (auto& ge : op->graphs) cudaGraphExecDestroy(ge.exec);
  op->graphs.clear();
  cudaFree(op->ws.beta);
  op->ws.beta = nullptr;
  op->ws.beta_cap = 0;
  op->ws.beta_fresh = 0;
  const int cap = std::max(iters, 64);
  SFS_TRY(dev_alloc(&op->ws.beta, (size_t)cap));
  op->ws.beta_cap = cap;
  return SFS_OK;
}

int ensure_events(sfs_operator* op, int n) {
  while ((int)op->ev.size() < n) {
    cudaEvent_t e;
    SFS_CUDA(cudaEventCreate(&e));
    op->ev.push_back(e);
  }
  return SFS_OK;
}

// The FISTA iteration loop (Algorithm 1): X^ of gamma_1, then per iteration
// forward contraction, residual planes (with the adjoint scatter and FFT),
// adjoint contraction, and the update planes that also transform
// gamma_{k+1}.  beta_k = (t_k - 1)/t_{k+1} is read from the device table
// beta_dev (single-scene calls, which may resume from a stored t) or fixed
// by k from t_1 = 1 (batched calls), so the loop can be captured once and
// replayed.  With `timing`, events are recorded before and after each
// kernel of every timing_stride(iters)-th iteration (op->ev[5 i + j] for
// the i-th such iteration, at most kTimedIters of them); inside a stream
// capture they become event-record nodes of the graph, so the per-kernel
// times come from the replayed loop itself, and the other iterations run
// without the few microseconds each event node adds.
// Buffers of one FISTA loop: the operator's workspace (one scene) or the
// batched workspace (d.batch scenes).
struct FistaBufs {
  float2 *ybuf, *yplane, *Xh, *Yh, *Rh, *Gh, *xk, *gam;
  float* scal;
};

constexpr int kTimedIters = 8;
int timing_stride(int iters) { return std::max(1, (iters + kTimedIters - 1) / kTimedIters); }
int timed_iters(int iters) { return iters > 0 ? (iters - 1) / timing_stride(iters) + 1 : 0; }

int enqueue_fista_loop(sfs_operator* op, const PlaneDims& d, const FistaBufs& b, int iters,
                       double* obj, bool timing, cudaStream_t st, const float* beta_dev = nullptr) {
  std::vector<float> beta(iters);
  double t = 1.0;
  for (int k = 0; k < iters; ++k) {
    const double tn = 0.5 * (1.0 + sqrt(1.0 + 4.0 * t * t));
    beta[k] = (float)((t - 1.0) / tn);
    t = tn;
  }
  cudaStreamCaptureStatus cap = cudaStreamCaptureStatusNone;
  if (timing) SFS_CUDA(cudaStreamIsCapturing(st, &cap));
  const unsigned evflags = cap == cudaStreamCaptureStatusActive ? cudaEventRecordExternal : 0u;
  const int stride = timing_stride(iters);
  auto mark = [&](int k, int j) -> int {
    if (timing && k % stride == 0)
      SFS_CUDA(cudaEventRecordWithFlags(op->ev[5 * (k / stride) + j], st, evflags));
    return SFS_OK;
  };
  SFS_TRY(launch_scatter_y_planes(d, b.ybuf, op->posmap, b.yplane, st));
  SFS_TRY(launch_fwd_planes(d, b.gam, b.Xh, st));
  for (int k = 0; k < iters; ++k) {
    SFS_TRY(mark(k, 0));
    SFS_TRY(launch_contract_fwd(d, op->table, b.Xh, b.Yh, op->ws.err, st));
    SFS_TRY(mark(k, 1));
    SFS_TRY(launch_inv_resid_fwd(d, b.Yh, op->posmap, b.yplane, b.Rh, obj ? obj + 2 * k : nullptr, st));
    SFS_TRY(mark(k, 2));
    SFS_TRY(launch_contract_adj(d, op->table, b.Rh, b.Gh, op->ws.err, st));
    SFS_TRY(mark(k, 3));
    SFS_TRY(launch_inv_fista_fwd(d, b.Gh, op->ws.segslot, b.xk, b.gam, b.scal, beta[k], k + 1 < iters,
                                 b.Xh, obj ? obj + 2 * k + 1 : nullptr, st,
                                 beta_dev ? beta_dev + k : nullptr));
    SFS_TRY(mark(k, 4));
  }
  return SFS_OK;
}

int enqueue_fista_iterations(sfs_operator* op, int iters, double* obj, bool timing,
                             cudaStream_t st) {
  const FistaBufs b = {op->ws.ybuf, op->ws.yplane, op->ws.Xh, op->ws.Yh, op->ws.Rh,
                       op->ws.Gh,   op->ws.xk,     op->ws.gam, op->ws.scal};
  return enqueue_fista_loop(op, dims_of(op), b, iters, obj, timing, st, op->ws.beta);
}

// Dimensions of a batched call on `batch` scenes.
PlaneDims batch_dims(const sfs_operator* op, int batch) {
  PlaneDims d = dims_of(op);
  d.batch = batch;
  for (const auto& bt : op->batch_tile)
    if (bt.first == batch) d.nb = bt.second;
  d.pm_x = op->f16 ? op->bws.pmx : nullptr;
  d.pm_r = op->f16 ? op->bws.pmr : nullptr;
  return d;
}

// Batched workspace for at least `batch` scenes (grown on demand; loops
// captured on the old buffers are dropped).
int ensure_batch(sfs_operator* op, int batch) {
  if (op->bws.cap >= batch) return SFS_OK;
  free_batch(op);
  const PlaneDims d = dims_of(op);
  sfs::BatchWorkspace& w = op->bws;
  const size_t B = (size_t)batch;
  int rc = SFS_OK;
  if (rc == SFS_OK) rc = dev_alloc(&w.Xh, B * d.bs_xh);
  if (rc == SFS_OK) rc = dev_alloc(&w.Yh, B * d.bs_yh);
  if (rc == SFS_OK) rc = dev_alloc(&w.Rh, B * d.bs_rh);
  if (rc == SFS_OK) rc = dev_alloc(&w.Gh, B * d.bs_gh);
  if (rc == SFS_OK) rc = dev_alloc(&w.xk, B * d.bs_x);
  if (rc == SFS_OK) rc = dev_alloc(&w.gam, B * d.bs_x);
  if (rc == SFS_OK) rc = dev_alloc(&w.yplane, B * d.bs_yplane);
  if (rc == SFS_OK) rc = dev_alloc(&w.ybuf, B * d.bs_y);
  if (rc == SFS_OK) rc = dev_alloc(&w.scal, B * kNumFloatScalars);
  if (rc == SFS_OK && op->f16) rc = dev_alloc(&w.pmx, B * d.bs_pmx);
  if (rc == SFS_OK && op->f16) rc = dev_alloc(&w.pmr, B * d.bs_pmr);
  if (rc == SFS_OK) {
    // spectra rows of the padding bins U..Up-1 are read by the contractions
    // and never written
    const cudaError_t e = cudaMemset(w.Rh, 0, B * d.bs_rh * sizeof(float2));
    if (e != cudaSuccess) rc = cuda_fail(e, "clearing batched spectra", __FILE__, __LINE__);
  }
  if (rc != SFS_OK) {
    free_batch(op);
    return rc;
  }
  w.cap = batch;
  ++op->bws_gen;
  return SFS_OK;
}

int fista_graph_batched(sfs_operator* op, int iters, int batch, cudaGraphExec_t* out) {
  for (auto& ge : op->bgraphs)
    if (ge.iters == iters && ge.batch == batch) {
      *out = ge.exec;
      return SFS_OK;
    }
  if (!op->capture_stream)
    SFS_CUDA(cudaStreamCreateWithFlags(&op->capture_stream, cudaStreamNonBlocking));
  const PlaneDims d = batch_dims(op, batch);
  SFS_TRY(prepare_kernels(d));
  const sfs::BatchWorkspace& w = op->bws;
  const FistaBufs b = {w.ybuf, w.yplane, w.Xh, w.Yh, w.Rh, w.Gh, w.xk, w.gam, w.scal};
  cudaStream_t cs = op->capture_stream;
  SFS_CUDA(cudaStreamBeginCapture(cs, cudaStreamCaptureModeThreadLocal));
  int rc = enqueue_fista_loop(op, d, b, iters, nullptr, false, cs);
  cudaGraph_t graph = nullptr;
  const cudaError_t e = cudaStreamEndCapture(cs, &graph);
  if (rc != SFS_OK) {
    if (graph) cudaGraphDestroy(graph);
    return rc;
  }
  if (e != cudaSuccess) return cuda_fail(e, "cudaStreamEndCapture", __FILE__, __LINE__);
  cudaGraphExec_t exec = nullptr;
  const cudaError_t e2 = cudaGraphInstantiate(&exec, graph, 0);
  cudaGraphDestroy(graph);
  if (e2 != cudaSuccess) return cuda_fail(e2, "cudaGraphInstantiate", __FILE__, __LINE__);
  op->bgraphs.push_back({iters, batch, exec});
  *out = exec;
  return SFS_OK;
}

// Executable graph of the iteration loop for (iters, monitor, timed),
// captured on the operator's own stream the first time it is needed.  All
// pointers and events it bakes in are operator-owned, so it stays valid for
// the operator's life (or until the momentum or monitor buffer grows).
int fista_graph(sfs_operator* op, int iters, bool with_obj, bool timed, cudaGraphExec_t* out) {
  for (auto& ge : op->graphs)
    if (ge.iters == iters && ge.with_obj == with_obj && ge.timed == timed) {
      *out = ge.exec;
      return SFS_OK;
    }
  if (!op->capture_stream)
    SFS_CUDA(cudaStreamCreateWithFlags(&op->capture_stream, cudaStreamNonBlocking));
  SFS_TRY(prepare_kernels(dims_of(op)));  // function attributes are set outside the capture
  cudaStream_t cs = op->capture_stream;
  SFS_CUDA(cudaStreamBeginCapture(cs, cudaStreamCaptureModeThreadLocal));
  int rc = enqueue_fista_iterations(op, iters, with_obj ? op->ws.obj : nullptr, timed, cs);
  cudaGraph_t graph = nullptr;
  const cudaError_t e = cudaStreamEndCapture(cs, &graph);
  if (rc != SFS_OK) {
    if (graph) cudaGraphDestroy(graph);
    return rc;
  }
  if (e != cudaSuccess) return cuda_fail(e, "cudaStreamEndCapture", __FILE__, __LINE__);
  cudaGraphExec_t exec = nullptr;
  const cudaError_t e2 = cudaGraphInstantiate(&exec, graph, 0);
  cudaGraphDestroy(graph);
  if (e2 != cudaSuccess) return cuda_fail(e2, "cudaGraphInstantiate", __FILE__, __LINE__);
  op->graphs.push_back({iters, with_obj, timed, exec});
  *out = exec;
  return SFS_OK;
}

}  // namespace

// ---- batched building blocks shared with the learned network (sfs_lista.cu) ----
int batch_workspace(sfs_operator* op, int batch) { return ensure_batch(op, batch); }

int batched_normal_residual(sfs_operator* op, int batch, const float2* x, const float2* yplane,
                            float2* g, cudaStream_t st) {
  SFS_TRY(ensure_batch(op, batch));
  const PlaneDims d = batch_dims(op, batch);
  const sfs::BatchWorkspace& w = op->bws;
  SFS_TRY(launch_fwd_planes(d, x, w.Xh, st));
  SFS_TRY(launch_contract_fwd(d, op->table, w.Xh, w.Yh, op->ws.err, st));
  SFS_TRY(launch_inv_resid_fwd(d, w.Yh, op->posmap, yplane, w.Rh, nullptr, st));
  SFS_TRY(launch_contract_adj(d, op->table, w.Rh, w.Gh, op->ws.err, st));
  return launch_inv_store(d, w.Gh, op->ws.segslot, g, nullptr, nullptr, st);
}

int batched_maxabs_AH(sfs_operator* op, int batch, const float2* y, float* scal, cudaStream_t st) {
  SFS_TRY(ensure_batch(op, batch));
  const PlaneDims d = batch_dims(op, batch);
  const sfs::BatchWorkspace& w = op->bws;
  SFS_TRY(launch_scatter_fwd(d, y, op->posmap, w.Rh, st));
  SFS_TRY(launch_contract_adj(d, op->table, w.Rh, w.Gh, op->ws.err, st));
  return launch_inv_store(d, w.Gh, op->ws.segslot, nullptr, nullptr, (unsigned int*)(scal + kLamMax), st);
}

int batched_scatter_y(sfs_operator* op, int batch, const float2* y, float2* yplane, cudaStream_t st) {
  return launch_scatter_y_planes(batch_dims(op, batch), y, op->posmap, yplane, st);
}

int operator_device(const sfs_operator* op) { return op->geo.d.device; }

namespace {

// One executable graph that runs the batched FISTA loops of several
// operators concurrently (one forked stream per group, joined at the end).
// Cached process-wide by (operator ids, workspace generations, batches,
// iterations), at most kGroupedCache graphs, oldest evicted first.
constexpr size_t kGroupedCache = 16;
struct GroupedEntry {
  std::vector<uint64_t> key;
  cudaGraphExec_t exec;
  int device;
  PersistPlan* plan;  // persistent solves: the kernel's plan (owned), else null
};
std::mutex g_grouped_mu;
std::vector<GroupedEntry> g_grouped;
std::vector<cudaStream_t> g_fork_streams;
std::vector<cudaEvent_t> g_fork_events;
cudaStream_t g_grouped_capture = nullptr;
// completion of each group's loop (event-record nodes of the graphs) and the
// start of the latest grouped call, for sfs_grouped_times
std::vector<cudaEvent_t> g_done_events;
cudaEvent_t g_grouped_start = nullptr;
int g_grouped_last_n = 0;
// key of the latest persistent solve's cache entry (sfs_persistent_step_times)
std::vector<uint64_t> g_last_persist_key;
// priority order of the grouped graphs captured next (sfs_set_grouped_order)
std::atomic<int> g_grouped_order{SFS_GROUPED_CHEAPEST_FIRST};

// Adds an entry to the cache (g_grouped_mu held), evicting the oldest.
void cache_grouped(const GroupedEntry& ent) {
  if (g_grouped.size() >= kGroupedCache) {
    cudaGraphExecDestroy(g_grouped.front().exec);
    persist_free(g_grouped.front().plan);
    g_grouped.erase(g_grouped.begin());
  }
  g_grouped.push_back(ent);
}

int grouped_graph(int ngroups, sfs_operator* const* ops, const int32_t* batch, int iters,
                  cudaGraphExec_t* out) {
  const int order_kind = g_grouped_order.load();
  std::vector<uint64_t> key = {(uint64_t)iters, (uint64_t)ngroups | ((uint64_t)order_kind << 48)};
  for (int g = 0; g < ngroups; ++g) {
    key.push_back(ops[g]->uid);
    key.push_back(ops[g]->bws_gen);
    key.push_back((uint64_t)batch[g]);
  }
  int dev = 0;
  SFS_CUDA(cudaGetDevice(&dev));
  std::lock_guard<std::mutex> lock(g_grouped_mu);
  for (auto& e : g_grouped)
    if (e.key == key && e.device == dev) {
      *out = e.exec;
      return SFS_OK;
    }
  if (!g_grouped_capture) SFS_CUDA(cudaStreamCreateWithFlags(&g_grouped_capture, cudaStreamNonBlocking));
  while ((int)g_fork_streams.size() < ngroups) {
    cudaStream_t s2;
    SFS_CUDA(cudaStreamCreateWithFlags(&s2, cudaStreamNonBlocking));
    g_fork_streams.push_back(s2);
  }
  while ((int)g_fork_events.size() < ngroups + 1) {
    cudaEvent_t e2;
    SFS_CUDA(cudaEventCreateWithFlags(&e2, cudaEventDisableTiming));
    g_fork_events.push_back(e2);
  }
  while ((int)g_done_events.size() < ngroups) {
    cudaEvent_t e3;
    SFS_CUDA(cudaEventCreate(&e3));
    g_done_events.push_back(e3);
  }
  for (int g = 0; g < ngroups; ++g) SFS_TRY(prepare_kernels(batch_dims(ops[g], batch[g])));
  // kernel priorities ranked by the work of a group's iteration (scenes x
  // bins x slots x depths): by default the cheaper, the higher, so that small
  // groups finish early instead of with the large ones; or the larger, the
  // higher (longest loops first); or none
  std::vector<int> prio(ngroups, 0);
  if (order_kind != SFS_GROUPED_NO_PRIORITY) {
    int least = 0, greatest = 0;
    SFS_CUDA(cudaDeviceGetStreamPriorityRange(&least, &greatest));
    std::vector<int> order(ngroups);
    for (int g = 0; g < ngroups; ++g) order[g] = g;
    auto cost = [&](int g) {
      const double c = (double)batch[g] * ops[g]->U * ops[g]->Ns * ops[g]->geo.d.Nz;
      return order_kind == SFS_GROUPED_LARGEST_FIRST ? -c : c;
    };
    std::stable_sort(order.begin(), order.end(), [&](int a, int b) { return cost(a) < cost(b); });
    const int levels = least - greatest + 1;
    for (int r = 0; r < ngroups; ++r) {
      const int level = ngroups > 1 ? (r * levels) / ngroups : 0;  // 0 = cheapest
      prio[order[r]] = greatest + level;
    }
  }
  cudaStream_t cs = g_grouped_capture;
  SFS_CUDA(cudaStreamBeginCapture(cs, cudaStreamCaptureModeThreadLocal));
  int rc = SFS_OK;
  cudaError_t e = cudaEventRecord(g_fork_events[ngroups], cs);
  if (e != cudaSuccess) rc = cuda_fail(e, "fork event", __FILE__, __LINE__);
  for (int g = 0; g < ngroups && rc == SFS_OK; ++g) {
    cudaStream_t sg = g_fork_streams[g];
    e = cudaStreamWaitEvent(sg, g_fork_events[ngroups], 0);
    if (e != cudaSuccess) {
      rc = cuda_fail(e, "fork wait", __FILE__, __LINE__);
      break;
    }
    const sfs::BatchWorkspace& w = ops[g]->bws;
    const FistaBufs b = {w.ybuf, w.yplane, w.Xh, w.Yh, w.Rh, w.Gh, w.xk, w.gam, w.scal};
    launch_priority() = prio[g];
    rc = enqueue_fista_loop(ops[g], batch_dims(ops[g], batch[g]), b, iters, nullptr, false, sg);
    launch_priority() = 0;
    if (rc == SFS_OK) {
      e = cudaEventRecordWithFlags(g_done_events[g], sg, cudaEventRecordExternal);
      if (e == cudaSuccess) e = cudaEventRecord(g_fork_events[g], sg);
      if (e == cudaSuccess) e = cudaStreamWaitEvent(cs, g_fork_events[g], 0);
      if (e != cudaSuccess) rc = cuda_fail(e, "join", __FILE__, __LINE__);
    }
  }
  cudaGraph_t graph = nullptr;
  e = cudaStreamEndCapture(cs, &graph);
  if (rc != SFS_OK) {
    if (graph) cudaGraphDestroy(graph);
    return rc;
  }
  if (e != cudaSuccess) return cuda_fail(e, "cudaStreamEndCapture", __FILE__, __LINE__);
  cudaGraphExec_t exec = nullptr;
  e = cudaGraphInstantiateWithFlags(&exec, graph, cudaGraphInstantiateFlagUseNodePriority);
  cudaGraphDestroy(graph);
  if (e != cudaSuccess) return cuda_fail(e, "cudaGraphInstantiate", __FILE__, __LINE__);
  cache_grouped({key, exec, dev, nullptr});
  *out = exec;
  return SFS_OK;
}

// The persistent solve's graph: per group the measurements by plane and X^ of
// gamma_1 (plain launches), then the one cooperative kernel of all
// iterations.  Cached with the grouped graphs (its key starts with a tag).
int persistent_graph(int ngroups, sfs_operator* const* ops, const int32_t* batch, int iters, int nb_policy,
                     cudaGraphExec_t* out) {
  std::vector<uint64_t> key = {(uint64_t)iters, (uint64_t)ngroups | ((uint64_t)(nb_policy + 1) << 40)};
  for (int g = 0; g < ngroups; ++g) {
    key.push_back(ops[g]->uid);
    key.push_back(ops[g]->bws_gen);
    key.push_back((uint64_t)batch[g]);
  }
  int dev = 0;
  SFS_CUDA(cudaGetDevice(&dev));
  std::lock_guard<std::mutex> lock(g_grouped_mu);
  g_last_persist_key = key;
  g_last_persist_key.push_back((uint64_t)dev);
  for (auto& e : g_grouped)
    if (e.key == key && e.device == dev) {
      *out = e.exec;
      return SFS_OK;
    }
  if (!g_grouped_capture) SFS_CUDA(cudaStreamCreateWithFlags(&g_grouped_capture, cudaStreamNonBlocking));
  std::vector<PlaneDims> dims(ngroups);
  for (int g = 0; g < ngroups; ++g) {
    dims[g] = batch_dims(ops[g], batch[g]);
    SFS_TRY(prepare_kernels(dims[g]));
  }
  PersistPlan* plan = nullptr;
  SFS_TRY(persist_build(ngroups, ops, dims.data(), iters, nb_policy, &plan));
  cudaStream_t cs = g_grouped_capture;
  cudaError_t e = cudaStreamBeginCapture(cs, cudaStreamCaptureModeThreadLocal);
  if (e != cudaSuccess) {
    persist_free(plan);
    return cuda_fail(e, "cudaStreamBeginCapture", __FILE__, __LINE__);
  }
  int rc = SFS_OK;
  for (int g = 0; g < ngroups && rc == SFS_OK; ++g) {
    const sfs::BatchWorkspace& w = ops[g]->bws;
    rc = launch_scatter_y_planes(dims[g], w.ybuf, ops[g]->posmap, w.yplane, cs);
    if (rc == SFS_OK) rc = launch_fwd_planes(dims[g], w.gam, w.Xh, cs);
  }
  if (rc == SFS_OK) rc = persist_launch(plan, cs);
  cudaGraph_t graph = nullptr;
  e = cudaStreamEndCapture(cs, &graph);
  if (rc == SFS_OK && e != cudaSuccess) rc = cuda_fail(e, "cudaStreamEndCapture", __FILE__, __LINE__);
  cudaGraphExec_t exec = nullptr;
  if (rc == SFS_OK) {
    e = cudaGraphInstantiate(&exec, graph, 0);
    if (e != cudaSuccess) rc = cuda_fail(e, "cudaGraphInstantiate", __FILE__, __LINE__);
  }
  if (graph) cudaGraphDestroy(graph);
  if (rc != SFS_OK) {
    persist_free(plan);
    return rc;
  }
  cache_grouped({key, exec, dev, plan});
  *out = exec;
  return SFS_OK;
}

// Reads (and clears) the device timeout flag; call only where the stream is
// synchronised anyway.
int check_err_flag(sfs_operator* op, cudaStream_t st) {
  int h = 0;
  SFS_CUDA(cudaMemcpyAsync(&h, op->ws.err, sizeof(int), cudaMemcpyDeviceToHost, st));
  SFS_CUDA(cudaStreamSynchronize(st));
  if (h) {
    SFS_CUDA(cudaMemsetAsync(op->ws.err, 0, sizeof(int), st));
    SFS_CUDA(cudaStreamSynchronize(st));
    if (h == 2) {
      set_error("non-finite value reached the lambda rule");
      return SFS_ERR_NON_FINITE;
    }
    set_error("a bounded wait in a contraction kernel timed out");
    return SFS_ERR_TIMEOUT;
  }
  return SFS_OK;
}

// Slot table of the adjoint contraction: CTA b of G owns units
// [N b / G, N (b+1) / G) of the N = nseg * U units (segment-major, bin
// fastest) and leaves one partial per segment it touches in slot seg + b.
// The CTAs touching a segment are consecutive, so its partials occupy the
// consecutive slots seg + b_first .. seg + b_last.
std::vector<int2> segment_slots(int nseg, int U, int G) {
  const long long N = (long long)nseg * U;
  std::vector<int2> out(nseg);
  int b = 0;
  auto last_of = [&](int bb) { return (N * (bb + 1)) / G; };  // one past CTA bb's range
  for (int seg = 0; seg < nseg; ++seg) {
    const long long r0 = (long long)seg * U, r1 = r0 + U - 1;
    while (last_of(b) <= r0) ++b;
    int be = b;
    while (last_of(be) <= r1) ++be;
    out[seg] = make_int2(seg + b, be - b + 1);
  }
  return out;
}

}  // namespace
}  // namespace sfs

namespace sfs {
void shard_run(int U, int nshards, int shard, int* first, int* count) {
  const long long a = (long long)U * shard / nshards, b = (long long)U * (shard + 1) / nshards;
  *first = (int)a;
  *count = (int)(b - a);
}
}  // namespace sfs

using namespace sfs;

extern "C" {

const char* sfs_last_error(void) { return g_last_error.c_str(); }

const char* sfs_version(void) { return "libsfs 0.1 (sm_103a)"; }

int sfs_create_geometry(const sfs_geometry_desc* desc, sfs_geometry** out) {
  clear_error();
  if (!desc || !out) {
    set_error("null argument");
    return SFS_ERR_INVALID_ARG;
  }
  *out = nullptr;
  const sfs_geometry_desc& d = *desc;
  if (d.Nx < 1 || d.Ny < 1 || d.Nz < 1 || d.Nt < 2) {
    set_error("sizes must be positive (Nx=%d Ny=%d Nz=%d Nt=%d)", d.Nx, d.Ny, d.Nz, d.Nt);
    return SFS_ERR_INVALID_ARG;
  }
  if (!(d.dx > 0) || !(d.dy > 0) || !(d.dz > 0) || !(d.c > 0) || !(d.fs > 0) || !(d.fc > 0) ||
      !(d.frac_bw > 0) || !(d.z0 > 0) || !(d.theta >= 0) || !(d.theta < M_PI / 2)) {
    set_error("physical parameters out of range");
    return SFS_ERR_INVALID_ARG;
  }
  int Px, Py;
  if (d.Ny == 1) {
    Py = 1;
    Px = std::max(64, next_pow2(2 * d.Nx - 1));
    if (Px > 1024) {
      set_error("line scans support Nx <= 512 (got %d)", d.Nx);
      return SFS_ERR_INVALID_ARG;
    }
  } else {
    const int P = std::max(32, next_pow2(2 * std::max(d.Nx, d.Ny) - 1));
    if (P > kMaxP2D) {
      set_error("area scans support Nx, Ny <= 64 (got %d x %d)", d.Nx, d.Ny);
      return SFS_ERR_INVALID_ARG;
    }
    Px = Py = P;
  }
  sfs_geometry* g = new (std::nothrow) sfs_geometry;
  if (!g) {
    set_error("host allocation failed");
    return SFS_ERR_OOM;
  }
  g->d = d;
  g->alpha = pulse_alpha(d.fc, d.frac_bw);
  if (isnan(d.t0)) g->d.t0 = floor((2.0 * d.z0 / d.c - 3.0 / g->alpha) * d.fs) / d.fs;
  g->Px = Px;
  g->Py = Py;
  *out = g;
  return SFS_OK;
}

int sfs_destroy_geometry(sfs_geometry* g) {
  delete g;
  return SFS_OK;
}

int sfs_select_indices(const sfs_geometry* g, int strategy, int M, int per_position,
                       uint64_t seed, int32_t* idx_out_host, int32_t* band_out_host) {
  clear_error();
  if (!g || !idx_out_host) {
    set_error("null argument");
    return SFS_ERR_INVALID_ARG;
  }
  int lo, hi;
  SFS_TRY(select_host(g, strategy, M, per_position, seed, idx_out_host, &lo, &hi, nullptr));
  if (band_out_host) {
    band_out_host[0] = lo;
    band_out_host[1] = hi;
  }
  return SFS_OK;
}

static int build_operator(sfs_geometry* g, int M, const int32_t* idx_host, int prec,
                          sfs_operator** out, int nshards = 1, int shard = 0) {
  if (!g || !idx_host || !out) {
    set_error("null argument");
    return SFS_ERR_INVALID_ARG;
  }
  *out = nullptr;
  const sfs_geometry_desc& d = g->d;
  const int S = d.Nx * d.Ny;
  // signed DFT bins -Nt/2 < k <= Nt/2: bin k + Nt of the A-scan for k < 0
  // (the negative frequencies of its periodic spectrum)
  const int kmax = d.Nt / 2, kmin = -((d.Nt - 1) / 2);
  const int nbins = kmax - kmin + 1;
  if (M <= 0 || M > nbins) {
    set_error("M = %d out of range 1..%d", M, nbins);
    return SFS_ERR_INVALID_ARG;
  }
  for (int s = 0; s < S; ++s)
    for (int m = 0; m < M; ++m) {
      const int k = idx_host[(size_t)s * M + m];
      if (k < kmin || k > kmax || (m > 0 && k <= idx_host[(size_t)s * M + m - 1])) {
        set_error("index row %d is not strictly ascending inside %d..%d", s, kmin, kmax);
        return SFS_ERR_INVALID_ARG;
      }
    }
  sfs_operator* op = new (std::nothrow) sfs_operator;
  if (!op) {
    set_error("host allocation failed");
    return SFS_ERR_OOM;
  }
  op->geo = *g;
  {
    static std::atomic<uint64_t> next_uid{1};
    op->uid = next_uid++;
  }
  op->prec = prec;
  op->tc = prec == SFS_PREC_FP32 ? 0 : (prec == SFS_PREC_TF32X3 ? 1 : 2);
  op->nparts = (prec == SFS_PREC_BF16X2 || prec == SFS_PREC_FP16X2) ? 2 : 1;
  op->f16 = (prec == SFS_PREC_FP16 || prec == SFS_PREC_FP16X2) ? 1 : 0;
  op->M = M;
  op->S = S;
  op->V = S * d.Nz;
  op->Nk = g->Px * g->Py;
  op->idx.assign(idx_host, idx_host + (size_t)S * M);
  std::vector<char> used(nbins, 0);
  for (int32_t k : op->idx) used[k - kmin] = 1;
  std::vector<int32_t> all_bins;
  for (int k = kmin; k <= kmax; ++k)
    if (used[k - kmin]) all_bins.push_back(k);
  // the operator's run of the union (all of it unless sharded)
  int first = 0, count = (int)all_bins.size();
  shard_run((int)all_bins.size(), nshards, shard, &first, &count);
  if (count < 1) {
    set_error("shard %d of %d holds no bin (the union has %d)", shard, nshards, (int)all_bins.size());
    delete op;
    return SFS_ERR_INVALID_ARG;
  }
  op->nshards = nshards;
  op->shard = shard;
  op->shard_first = first;
  op->U_all = (int)all_bins.size();
  std::vector<int> u_of(nbins, -1);  // position of bin k in this operator's bins, at k - kmin
  for (int j = 0; j < count; ++j) {
    u_of[all_bins[first + j] - kmin] = j;
    op->bins.push_back(all_bins[first + j]);
  }
  op->U = (int)op->bins.size();
  // band the strategies would use (reported only)
  if (candidate_band(g, M, &op->k_lo, &op->k_hi, &op->band_db) != SFS_OK) {
    op->k_lo = op->bins.front();
    op->k_hi = op->bins.back();
    op->band_db = NAN;
    clear_error();
  }
  op->nzb = (d.Nz + kZBlockRows - 1) / kZBlockRows;

  // Symmetry orbits of the lateral wavenumbers.  The generators depend on
  // dx^2 + dy^2 only, so their FFT2 is invariant under kx -> -kx, ky -> -ky
  // and, on a square grid with equal pitches and sizes, kx <-> ky.  Spectra
  // are kept orbit-major in GS slots per orbit (padding slots carry -1), and
  // the table holds one entry per orbit.  Wavenumber kappa = kx * Py + ky
  // (the FFT engine's order); for a line scan kappa = kx.
  const bool two_d = g->Py > 1;
  const bool swap = two_d && g->Px == g->Py && d.Nx == d.Ny && d.dx == d.dy;
  op->GS = two_d ? (swap ? 8 : 4) : 2;
  std::vector<int32_t> slot_kappa, orbit_rep;
  {
    const int Px = g->Px, Py = g->Py;
    const int half = std::max(Px, Py) / 2 + 1;
    std::vector<int> orbit_of((size_t)half * half, -1);
    std::vector<std::vector<int>> members;
    for (int kap = 0; kap < Px * Py; ++kap) {
      const int kx = two_d ? kap / Py : kap;
      const int ky = two_d ? kap % Py : 0;
      int ax = std::min(kx, (Px - kx) % Px);
      int ay = two_d ? std::min(ky, (Py - ky) % Py) : 0;
      if (swap && ax > ay) std::swap(ax, ay);
      int& o = orbit_of[(size_t)ax * half + ay];
      if (o < 0) {
        o = (int)members.size();
        members.emplace_back();
      }
      members[o].push_back(kap);
    }
    op->No = (int)members.size();
    op->Up = (op->U + op->GS / 2 - 1) / (op->GS / 2) * (op->GS / 2);
    op->Ns = (op->No * op->GS + kKappaTile - 1) / kKappaTile * kKappaTile;
    slot_kappa.assign(op->Ns, -1);
    orbit_rep.assign(op->Ns / op->GS, -1);
    for (int o = 0; o < op->No; ++o) {
      orbit_rep[o] = members[o][0];
      for (size_t m = 0; m < members[o].size(); ++m) slot_kappa[(size_t)o * op->GS + m] = members[o][m];
    }
  }
  // 128 x 128 planes move their spectra quadrant by quadrant (the output
  // parities (ky & 1, kx & 1) of the 128-point transforms): offsets of the
  // four quadrants and the padding slots, then entries (slot << 12) |
  // (kx / 2 * 64 + ky / 2), slots ascending within each group.
  std::vector<int32_t> quad;
  if (two_d && g->Px == 128) {
    std::vector<int32_t> groups[5];
    for (int j = 0; j < op->Ns; ++j) {
      const int kap = slot_kappa[j];
      if (kap < 0) {
        groups[4].push_back(j << 12);
        continue;
      }
      const int kx = kap / g->Py, ky = kap % g->Py;
      groups[2 * (ky & 1) + (kx & 1)].push_back((j << 12) | ((kx >> 1) * 64 + (ky >> 1)));
    }
    quad.assign(8, 0);
    for (int q = 0; q < 5; ++q) {
      quad[q + 1] = quad[q] + (int32_t)groups[q].size();
      quad.insert(quad.end(), groups[q].begin(), groups[q].end());
    }
  }

  // host FP64 geometry tables: (tau - t0) fs / Nt split into (hi, lo) floats,
  // directivity, per-bin amplitude fs H(f_k) / (Px Py)
  const size_t nt = (size_t)d.Nz * d.Ny * d.Nx;
  std::vector<float2> tof(nt);
  std::vector<float> gdir(nt);
  for (int iz = 0; iz < d.Nz; ++iz) {
    const double z = d.z0 + iz * d.dz;
    for (int ay = 0; ay < d.Ny; ++ay)
      for (int ax = 0; ax < d.Nx; ++ax) {
        const double rx = ax * d.dx, ry = ay * d.dy;
        const double tau = 2.0 / d.c * sqrt(rx * rx + ry * ry + z * z);
        const double tn = (tau - d.t0) * d.fs / d.Nt;
        const float hi = (float)tn;
        const float lo = (float)(tn - (double)hi);
        const size_t i = ((size_t)iz * d.Ny + ay) * d.Nx + ax;
        tof[i] = make_float2(hi, lo);
        double gv = 1.0;
        if (d.theta > 0) {
          const double w = z * tan(d.theta);
          gv = exp(-(rx * rx + ry * ry) / (w * w));
        }
        gdir[i] = (float)gv;
      }
  }
  std::vector<float> amp(op->U);
  for (int u = 0; u < op->U; ++u)
    amp[u] = (float)(d.fs * pulse_mag((double)op->bins[u] * d.fs / d.Nt, d.fc, g->alpha) /
                     ((double)g->Px * g->Py));
  if (op->f16) {
    // FP16 table: every entry of FFT2(h_{k,z}) / (Px Py) is at most the sum
    // of the plane's tap magnitudes, amp[u] * sum over (+-dx, +-dy) of g; the
    // stored table is scaled by 2^kT so that this bound lies in [2^13, 2^14)
    // (FP16 holds up to 65504), kT clamped to +-126.
    double gsum = 0.0;
    for (int iz = 0; iz < d.Nz; ++iz) {
      double acc = 0.0;
      for (int ay = 0; ay < d.Ny; ++ay)
        for (int ax = 0; ax < d.Nx; ++ax)
          acc += (ax ? 2.0 : 1.0) * (ay ? 2.0 : 1.0) * gdir[((size_t)iz * d.Ny + ay) * d.Nx + ax];
      gsum = std::max(gsum, acc);
    }
    double amax = 0.0;
    for (int u = 0; u < op->U; ++u) amax = std::max(amax, (double)fabsf(amp[u]));
    const double bound = amax * gsum;
    op->tscale_exp = bound > 0.0 && isfinite(bound)
                         ? std::min(126, std::max(-126, 13 - (int)floor(log2(bound))))
                         : 0;
  }
  std::vector<int32_t> posmap((size_t)op->U * S, -1);
  for (int s = 0; s < S; ++s)
    for (int m = 0; m < M; ++m) {
      const int u = u_of[op->idx[(size_t)s * M + m] - kmin];
      if (u >= 0) posmap[(size_t)u * S + s] = m;  // rows of other shards stay unmapped
    }

  DeviceScope scope(d.device);
  if (!scope.ok()) {
    set_error("cannot select CUDA device %d", d.device);
    delete op;
    return SFS_ERR_CUDA;
  }
  float2* d_tof = nullptr;
  float* d_gdir = nullptr;
  float* d_amp = nullptr;
  int32_t* d_bins = nullptr;
  auto fail = [&](int rc) {
    cudaFree(d_tof);
    cudaFree(d_gdir);
    cudaFree(d_amp);
    cudaFree(d_bins);
    free_operator(op);
    return rc;
  };
  int rc;
  int sms = 0;
  {
    cudaError_t e0 = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, d.device);
    if (e0 != cudaSuccess) return fail(cuda_fail(e0, "SM count query", __FILE__, __LINE__));
  }
  op->nzc = (d.Nz + 15) / 16;
  op->nkb = (d.Nz + 31) / 32;
  if (op->tc) op->nzb = 1;
  const int nseg = (op->Ns / kKappaTile) * op->nzb;
  const int ngroups = op->Up / (op->GS / 2);
  op->G = op->tc ? sms * kContractCtasPerSm
                 : std::max(1, std::min(sms * kContractCtasPerSm, nseg * ngroups));
  // Adjoint: one CTA per (slot tile, 32-depth block) when those segments fit
  // the resident grid and the tile's spectra fit beside the ring (dense
  // result); otherwise CTAs share segments and leave partial sums.
  const int anzb32 = (d.Nz + 31) / 32;
  const int nseg32 = (op->Ns / kKappaTile) * anzb32;
  std::vector<int2> segslot;
  if (op->tc || (nseg32 <= sms * kContractCtasPerSm &&
                 adj_seg_smem_bytes(op->Up) * kContractCtasPerSm + 2048 <=
                     (size_t)max_smem_optin() + 1024)) {
    op->adj_seg = 1;
    op->azb = 32;
    op->anzb = anzb32;
    op->Ga = nseg32;
    op->nslots = nseg32;
    segslot.resize(nseg32);
    for (int sgi = 0; sgi < nseg32; ++sgi) segslot[sgi] = make_int2(sgi, 1);
  } else {
    op->adj_seg = 0;
    op->azb = kZBlockRows;
    op->anzb = op->nzb;
    op->Ga = 0;
    op->nslots = nseg + op->G - 1;
    segslot = segment_slots(nseg, ngroups, op->G);
  }
  const size_t Ns = op->Ns;
  const size_t table_elems = table_c64(op);
  if ((rc = dev_alloc(&op->table, table_elems)) != SFS_OK) return fail(rc);
  if ((rc = dev_alloc(&op->posmap, posmap.size())) != SFS_OK) return fail(rc);
  if ((rc = dev_alloc(&op->ws.Xh, Ns * d.Nz)) != SFS_OK) return fail(rc);
  if ((rc = dev_alloc(&op->slot_kappa, slot_kappa.size())) != SFS_OK) return fail(rc);
  if ((rc = dev_alloc(&op->orbit_rep, orbit_rep.size())) != SFS_OK) return fail(rc);
  if (!quad.empty() && (rc = dev_alloc(&op->quad, quad.size())) != SFS_OK) return fail(rc);
  if ((rc = dev_alloc(&op->ws.Gh, (size_t)op->nslots * op->azb * kKappaTile)) != SFS_OK)
    return fail(rc);
  if ((rc = dev_alloc(&op->ws.segslot, segslot.size())) != SFS_OK) return fail(rc);
  if ((rc = dev_alloc(&op->ws.err, 1)) != SFS_OK) return fail(rc);
  if ((rc = dev_alloc(&op->ws.Yh, Ns * op->Up * op->nzb)) != SFS_OK) return fail(rc);
  if ((rc = dev_alloc(&op->ws.Rh, Ns * op->Up)) != SFS_OK) return fail(rc);
  if ((rc = dev_alloc(&op->ws.xk, (size_t)op->V)) != SFS_OK) return fail(rc);
  if ((rc = dev_alloc(&op->ws.gam, (size_t)op->V)) != SFS_OK) return fail(rc);
  if ((rc = dev_alloc(&op->ws.ybuf, (size_t)S * M)) != SFS_OK) return fail(rc);
  if ((rc = dev_alloc(&op->ws.yplane, (size_t)op->U * S)) != SFS_OK) return fail(rc);
  if ((rc = dev_alloc(&op->ws.vbuf, (size_t)S * M)) != SFS_OK) return fail(rc);
  if ((rc = dev_alloc(&op->ws.scal, kNumFloatScalars)) != SFS_OK) return fail(rc);
  if ((rc = dev_alloc(&op->ws.red, kNumRed)) != SFS_OK) return fail(rc);
  if (op->f16 && (rc = dev_alloc(&op->ws.pmx, (size_t)d.Nz)) != SFS_OK) return fail(rc);
  if (op->f16 && (rc = dev_alloc(&op->ws.pmr, (size_t)op->Up)) != SFS_OK) return fail(rc);
  if ((rc = dev_alloc(&d_tof, nt)) != SFS_OK) return fail(rc);
  if ((rc = dev_alloc(&d_gdir, nt)) != SFS_OK) return fail(rc);
  if ((rc = dev_alloc(&d_amp, (size_t)op->U)) != SFS_OK) return fail(rc);
  if ((rc = dev_alloc(&d_bins, (size_t)op->U)) != SFS_OK) return fail(rc);
  cudaError_t e = cudaSuccess;
  if (e == cudaSuccess) e = cudaMemcpy(op->posmap, posmap.data(), posmap.size() * 4, cudaMemcpyHostToDevice);
  if (e == cudaSuccess) e = cudaMemcpy(d_tof, tof.data(), nt * sizeof(float2), cudaMemcpyHostToDevice);
  if (e == cudaSuccess) e = cudaMemcpy(d_gdir, gdir.data(), nt * sizeof(float), cudaMemcpyHostToDevice);
  if (e == cudaSuccess) e = cudaMemcpy(d_amp, amp.data(), op->U * sizeof(float), cudaMemcpyHostToDevice);
  if (e == cudaSuccess) e = cudaMemcpy(d_bins, op->bins.data(), op->U * sizeof(int32_t), cudaMemcpyHostToDevice);
  if (e == cudaSuccess) e = cudaMemset(op->ws.scal, 0, kNumFloatScalars * sizeof(float));
  if (e == cudaSuccess) e = cudaMemset(op->ws.red, 0, kNumRed * sizeof(double));
  if (e == cudaSuccess) e = cudaMemset(op->ws.err, 0, sizeof(int));
  {  // a table larger than half the L2 streams from HBM on every launch
    int l2 = 0;
    if (cudaDeviceGetAttribute(&l2, cudaDevAttrL2CacheSize, d.device) != cudaSuccess) l2 = 0;
    op->stream_table = l2 > 0 && (double)table_c64(op) * 8.0 > 0.5 * l2;
  }
  // padding bins U..Up-1: zero table rows and zero residual spectra, never written later
  if (e == cudaSuccess) e = cudaMemset(op->table, 0, table_elems * sizeof(float2));
  if (e == cudaSuccess) e = cudaMemset(op->ws.Rh, 0, Ns * op->Up * sizeof(float2));
  if (e == cudaSuccess)
    e = cudaMemcpy(op->slot_kappa, slot_kappa.data(), slot_kappa.size() * 4, cudaMemcpyHostToDevice);
  if (e == cudaSuccess)
    e = cudaMemcpy(op->orbit_rep, orbit_rep.data(), orbit_rep.size() * 4, cudaMemcpyHostToDevice);
  if (e == cudaSuccess && !quad.empty())
    e = cudaMemcpy(op->quad, quad.data(), quad.size() * 4, cudaMemcpyHostToDevice);
  if (e == cudaSuccess)
    e = cudaMemcpy(op->ws.segslot, segslot.data(), segslot.size() * sizeof(int2),
                   cudaMemcpyHostToDevice);
  if (e != cudaSuccess) return fail(cuda_fail(e, "upload of operator tables", __FILE__, __LINE__));
  const PlaneDims pd = dims_of(op);
  if ((rc = launch_build_table(pd, d_tof, d_gdir, d_amp, d_bins, op->table, 0)) != SFS_OK)
    return fail(rc);
  e = cudaDeviceSynchronize();
  if (e != cudaSuccess) return fail(cuda_fail(e, "generator table build", __FILE__, __LINE__));
  cudaFree(d_tof);
  cudaFree(d_gdir);
  cudaFree(d_amp);
  cudaFree(d_bins);
  d_tof = nullptr;
  d_gdir = nullptr;
  d_amp = nullptr;
  d_bins = nullptr;
  if (op->tc == 2 && (rc = tc16_setup(op)) != SFS_OK) return fail(rc);
  *out = op;
  return SFS_OK;
}

}  // extern "C"

namespace sfs {
int build_operator_shard(sfs_geometry* g, int M, const int32_t* idx_host, int prec, int nshards,
                         int shard, sfs_operator** out) {
  return build_operator(g, M, idx_host, prec, out, nshards, shard);
}

int normal_residual(sfs_operator* op, const float2* x, const float2* y, float2* g, cudaStream_t st) {
  const PlaneDims d = dims_of(op);
  SFS_TRY(launch_scatter_y_planes(d, y, op->posmap, op->ws.yplane, st));
  SFS_TRY(launch_fwd_planes(d, x, op->ws.Xh, st));
  SFS_TRY(launch_contract_fwd(d, op->table, op->ws.Xh, op->ws.Yh, op->ws.err, st));
  SFS_TRY(launch_inv_resid_fwd(d, op->ws.Yh, op->posmap, op->ws.yplane, op->ws.Rh, nullptr, st));
  SFS_TRY(launch_contract_adj(d, op->table, op->ws.Rh, op->ws.Gh, op->ws.err, st));
  return launch_inv_store(d, op->ws.Gh, op->ws.segslot, g, nullptr, nullptr, st);
}

int check_err_flag_op(sfs_operator* op, cudaStream_t st) { return check_err_flag(op, st); }
}  // namespace sfs

extern "C" {

int sfs_operator_from_indices(sfs_geometry* g, int M, const int32_t* idx_host,
                              sfs_operator** out) {
  clear_error();
  // SFS_CONTRACT=tc selects the tf32 tensor-core contractions (read per
  // operator); on the 3-D workloads the CUDA-core kernels are the faster.
  const char* cv = getenv("SFS_CONTRACT");
  const int prec = (cv && strcmp(cv, "tc") == 0) ? SFS_PREC_TF32X3 : SFS_PREC_FP32;
  return build_operator(g, M, idx_host, prec, out);
}

int sfs_operator_from_indices_prec(sfs_geometry* g, int M, const int32_t* idx_host,
                                   int precision, sfs_operator** out) {
  clear_error();
  if (precision < SFS_PREC_FP32 || precision > SFS_PREC_FP16X2) {
    set_error("unknown precision %d", precision);
    return SFS_ERR_INVALID_ARG;
  }
  return build_operator(g, M, idx_host, precision, out);
}

int sfs_select_freqs(sfs_geometry* g, int strategy, int M, int per_position, uint64_t seed,
                     int32_t* idx_out_host, uint32_t* mask_out_host, sfs_operator** op) {
  clear_error();
  if (!g || !op) {
    set_error("null argument");
    return SFS_ERR_INVALID_ARG;
  }
  const int S = g->d.Nx * g->d.Ny;
  std::vector<int32_t> idx((size_t)S * std::max(M, 1));
  SFS_TRY(select_host(g, strategy, M, per_position, seed, idx.data(), nullptr, nullptr, nullptr));
  if (idx_out_host) memcpy(idx_out_host, idx.data(), idx.size() * sizeof(int32_t));
  if (mask_out_host) {
    const int words = (g->d.Nt / 2 + 1 + 31) / 32;
    memset(mask_out_host, 0, sizeof(uint32_t) * (size_t)S * words);
    for (int s = 0; s < S; ++s)
      for (int m = 0; m < M; ++m) {
        const int k = idx[(size_t)s * M + m];
        mask_out_host[(size_t)s * words + k / 32] |= 1u << (k % 32);
      }
  }
  return sfs_operator_from_indices(g, M, idx.data(), op);
}

int sfs_destroy_operator(sfs_operator* op) {
  if (!op) return SFS_OK;
  DeviceScope scope(op->geo.d.device);
  free_operator(op);
  return SFS_OK;
}

int sfs_operator_info(const sfs_operator* op, sfs_operator_info_t* info) {
  clear_error();
  if (!op || !info) {
    set_error("null argument");
    return SFS_ERR_INVALID_ARG;
  }
  info->S = op->S;
  info->M = op->M;
  info->V = op->V;
  info->Nz = op->geo.d.Nz;
  info->U = op->U;
  info->Px = op->geo.Px;
  info->Py = op->geo.Py;
  info->Nkappa = op->Nk;
  info->k_lo = op->k_lo;
  info->k_hi = op->k_hi;
  info->band_db = op->band_db;
  info->alpha = op->geo.alpha;
  info->t0 = op->geo.d.t0;
  info->table_bytes = (int64_t)table_c64(op) * 8;
  info->launches_per_iter = 4;
  info->Nslot = op->Ns;
  info->GS = op->GS;
  info->precision = op->prec;
  info->nshards = op->nshards;
  info->shard = op->shard;
  info->shard_first = op->shard_first;
  info->U_all = op->U_all;
  return SFS_OK;
}

int sfs_apply_A(sfs_operator* op, const void* x_dev, void* y_dev, void* stream) {
  clear_error();
  if (!op || !x_dev || !y_dev || !aligned16(x_dev) || !aligned16(y_dev)) {
    set_error("null or misaligned argument");
    return SFS_ERR_INVALID_ARG;
  }
  DeviceScope scope(op->geo.d.device);
  return enqueue_A(op, (const float2*)x_dev, (float2*)y_dev, nullptr, (cudaStream_t)stream);
}

int sfs_apply_AH(sfs_operator* op, const void* y_dev, void* x_dev, void* stream) {
  clear_error();
  if (!op || !x_dev || !y_dev || !aligned16(x_dev) || !aligned16(y_dev)) {
    set_error("null or misaligned argument");
    return SFS_ERR_INVALID_ARG;
  }
  DeviceScope scope(op->geo.d.device);
  return enqueue_AH(op, (const float2*)y_dev, (float2*)x_dev, nullptr, nullptr,
                    (cudaStream_t)stream);
}

int sfs_frobenius(const sfs_operator* op, double* fro2_out, double* sigma_hat_out) {
  clear_error();
  if (!op || !fro2_out) {
    set_error("null argument");
    return SFS_ERR_INVALID_ARG;
  }
  // |A[(s,m), v]| = fs g(s, v) |H(f_k)|, k = idx[s][m] (Eq. (4)), so
  // ||A||_F^2 = fs^2 sum_s G(s) sum_m |H(f_{idx[s][m]})|^2 with
  // G(s) = sum_v g(s, v)^2.  g depends on the lateral offset and the depth
  // only; G(s) comes from 2-D prefix sums of g^2 over the offsets.
  const sfs_geometry_desc& d = op->geo.d;
  const int Nx = d.Nx, Ny = d.Ny, Nz = d.Nz;
  std::vector<double> G((size_t)Nx * Ny, (double)Nx * Ny * Nz);
  if (d.theta > 0) {
    const int WX = 2 * Nx - 1, WY = 2 * Ny - 1;
    std::fill(G.begin(), G.end(), 0.0);
    std::vector<double> P((size_t)(WY + 1) * (WX + 1));
    for (int iz = 0; iz < Nz; ++iz) {
      const double z = d.z0 + iz * d.dz, w = z * tan(d.theta);
      // P[j][i] = sum of g^2 over offsets (dy, dx) with dy < j - (Ny-1), dx < i - (Nx-1)
      std::fill(P.begin(), P.end(), 0.0);
      for (int j = 0; j < WY; ++j)
        for (int i = 0; i < WX; ++i) {
          const double rx = (i - (Nx - 1)) * d.dx, ry = (j - (Ny - 1)) * d.dy;
          const double gv = exp(-(rx * rx + ry * ry) / (w * w));
          P[(size_t)(j + 1) * (WX + 1) + i + 1] = gv * gv + P[(size_t)j * (WX + 1) + i + 1] +
                                                  P[(size_t)(j + 1) * (WX + 1) + i] - P[(size_t)j * (WX + 1) + i];
        }
      for (int sy = 0; sy < Ny; ++sy)
        for (int sx = 0; sx < Nx; ++sx) {
          // voxel offsets v - s: dx in [-sx, Nx-1-sx], dy in [-sy, Ny-1-sy]
          const int i0 = Nx - 1 - sx, i1 = i0 + Nx, j0 = Ny - 1 - sy, j1 = j0 + Ny;
          G[(size_t)sy * Nx + sx] += P[(size_t)j1 * (WX + 1) + i1] - P[(size_t)j0 * (WX + 1) + i1] -
                                     P[(size_t)j1 * (WX + 1) + i0] + P[(size_t)j0 * (WX + 1) + i0];
        }
    }
  }
  double fro2 = 0.0;
  for (int s = 0; s < op->S; ++s) {
    double h2 = 0.0;
    for (int m = 0; m < op->M; ++m) {
      const int k = op->idx[(size_t)s * op->M + m];
      if (k < op->bins.front() || k > op->bins.back()) continue;  // another shard's row
      const double h = pulse_mag((double)k * d.fs / d.Nt, d.fc, op->geo.alpha);
      h2 += h * h;
    }
    fro2 += G[s] * h2;
  }
  fro2 *= d.fs * d.fs;
  *fro2_out = fro2;
  // Eq. (sigma_hat) of Sec. IV-C: the geometric mean of the bounds
  // ||A||_F / sqrt(N) <= sigma_max <= ||A||_F, N = min(S M, V) (rank bound)
  const double N = std::min((double)op->S * op->M, (double)op->V);
  if (sigma_hat_out) *sigma_hat_out = sqrt(fro2) / pow(N, 0.25);
  return SFS_OK;
}

int sfs_max_abs_AH(sfs_operator* op, const void* y_dev, double* out_host, void* stream) {
  clear_error();
  if (!op || !y_dev || !out_host || !aligned16(y_dev)) {
    set_error("null or misaligned argument");
    return SFS_ERR_INVALID_ARG;
  }
  DeviceScope scope(op->geo.d.device);
  cudaStream_t st = (cudaStream_t)stream;
  unsigned int* bits = (unsigned int*)(op->ws.scal + kLamMax);
  SFS_CUDA(cudaMemsetAsync(bits, 0, sizeof(unsigned int), st));
  SFS_TRY(enqueue_AH(op, (const float2*)y_dev, nullptr, nullptr, bits, st));
  unsigned int hb = 0;
  SFS_CUDA(cudaMemcpyAsync(&hb, bits, sizeof(hb), cudaMemcpyDeviceToHost, st));
  SFS_CUDA(cudaStreamSynchronize(st));
  SFS_TRY(check_err_flag(op, st));
  float f;
  memcpy(&f, &hb, sizeof(f));
  if (!isfinite(f)) {
    set_error("non-finite value in A^H y");
    return SFS_ERR_NON_FINITE;
  }
  *out_host = f;
  return SFS_OK;
}

int sfs_lipschitz(sfs_operator* op, int max_iter, double rtol, uint64_t seed, double safety,
                  double* L_out, void* stream) {
  clear_error();
  if (!op || !L_out || max_iter < 1 || !(rtol >= 0) || !(safety >= 0)) {
    set_error("invalid argument");
    return SFS_ERR_INVALID_ARG;
  }
  DeviceScope scope(op->geo.d.device);
  cudaStream_t st = (cudaStream_t)stream;
  const int V = op->V;
  float2* v = op->ws.gam;
  float2* w = op->ws.xk;
  double* red = op->ws.red;
  // v0: seeded complex Gaussian, normalised
  SFS_TRY(launch_randn(v, V, seed, st));
  SFS_CUDA(cudaMemsetAsync(red + kRedB, 0, sizeof(double), st));
  SFS_TRY(launch_sumsq(v, V, red + kRedB, st));
  SFS_TRY(launch_scale_by_rnorm(v, V, red + kRedB, st));
  // power iteration on A^H A:  est = ||A v||^2, v <- A^H A v / ||A^H A v||
  const int check = 8;
  std::vector<double> hist(check);
  double* d_hist = nullptr;
  SFS_TRY(dev_alloc(&d_hist, check));
  double prev = -1.0, est = 0.0;
  int rc = SFS_ERR_NOT_CONVERGED;
  int it = 0;
  while (it < max_iter) {
    const int n = std::min(check, max_iter - it);
    for (int j = 0; j < n; ++j) {
      cudaMemsetAsync(red, 0, 2 * sizeof(double), st);
      if ((rc = enqueue_A(op, v, op->ws.vbuf, red + kRedA, st)) != SFS_OK) break;
      if ((rc = enqueue_AH(op, op->ws.vbuf, w, red + kRedB, nullptr, st)) != SFS_OK) break;
      if ((rc = launch_scale_by_rnorm(w, V, red + kRedB, st)) != SFS_OK) break;
      cudaMemcpyAsync(d_hist + j, red + kRedA, sizeof(double), cudaMemcpyDeviceToDevice, st);
      std::swap(v, w);
      rc = SFS_ERR_NOT_CONVERGED;
    }
    if (cudaGetLastError() != cudaSuccess && rc == SFS_ERR_NOT_CONVERGED) rc = SFS_ERR_CUDA;
    if (rc != SFS_ERR_NOT_CONVERGED) break;
    cudaError_t e = cudaMemcpyAsync(hist.data(), d_hist, n * sizeof(double), cudaMemcpyDeviceToHost, st);
    if (e == cudaSuccess) e = cudaStreamSynchronize(st);
    if (e != cudaSuccess) {
      rc = cuda_fail(e, "power iteration", __FILE__, __LINE__);
      break;
    }
    bool done = false;
    for (int j = 0; j < n; ++j) {
      est = hist[j];
      if (!isfinite(est)) {
        set_error("non-finite Rayleigh quotient in power iteration");
        rc = SFS_ERR_NON_FINITE;
        done = true;
        break;
      }
      ++it;
      if (prev > 0 && fabs(est - prev) <= rtol * est) {
        rc = SFS_OK;
        done = true;
        break;
      }
      prev = est;
    }
    if (done) break;
  }
  cudaFree(d_hist);
  if (rc == SFS_OK || rc == SFS_ERR_NOT_CONVERGED) {
    const int rc2 = check_err_flag(op, st);
    if (rc2 != SFS_OK) return rc2;
  }
  if (rc == SFS_OK || rc == SFS_ERR_NOT_CONVERGED) {
    *L_out = est * (1.0 + safety);
    if (rc == SFS_ERR_NOT_CONVERGED)
      set_error("power iteration did not reach rtol %g in %d iterations", rtol, max_iter);
  }
  return rc;
}

int sfs_fista(sfs_operator* op, const void* y_dev, double lambda, double L, int iters,
              void* x_inout_dev, void* state_dev, uint32_t flags, double* obj_hist_host,
              void* stream) {
  clear_error();
  const bool resume = (flags & SFS_FISTA_RESUME) != 0;
  if (!op || !y_dev || !x_inout_dev || iters < 0 || !(L > 0) || !isfinite(lambda) ||
      !aligned16(y_dev) || !aligned16(x_inout_dev) || (state_dev && !aligned16(state_dev)) ||
      (resume && !state_dev) || (resume && (flags & SFS_FISTA_WARM_START))) {
    set_error("invalid argument");
    return SFS_ERR_INVALID_ARG;
  }
  DeviceScope scope(op->geo.d.device);
  cudaStream_t st = (cudaStream_t)stream;
  const size_t vbytes = (size_t)op->V * sizeof(float2);
  // state layout: gamma_{k+1} [V], x_k [V] (c64), t_{k+1} (double), k (int64)
  float2* st_gam = state_dev ? (float2*)state_dev : nullptr;
  float2* st_x = state_dev ? st_gam + op->V : nullptr;
  double* st_t = state_dev ? (double*)(st_x + op->V) : nullptr;
  long long* st_k = state_dev ? (long long*)(st_t + 1) : nullptr;
  float2* y = op->ws.ybuf;
  SFS_CUDA(cudaMemcpyAsync(y, y_dev, (size_t)op->S * op->M * sizeof(float2),
                           cudaMemcpyDeviceToDevice, st));
  if (resume) {
    SFS_CUDA(cudaMemcpyAsync(op->ws.gam, st_gam, vbytes, cudaMemcpyDeviceToDevice, st));
    SFS_CUDA(cudaMemcpyAsync(op->ws.xk, st_x, vbytes, cudaMemcpyDeviceToDevice, st));
  } else if (flags & SFS_FISTA_WARM_START) {
    SFS_CUDA(cudaMemcpyAsync(op->ws.xk, x_inout_dev, vbytes, cudaMemcpyDeviceToDevice, st));
    SFS_CUDA(cudaMemcpyAsync(op->ws.gam, x_inout_dev, vbytes, cudaMemcpyDeviceToDevice, st));
  } else {
    SFS_CUDA(cudaMemsetAsync(op->ws.xk, 0, vbytes, st));
    SFS_CUDA(cudaMemsetAsync(op->ws.gam, 0, vbytes, st));
  }
  if (state_dev && !resume) SFS_CUDA(cudaMemsetAsync(st_k, 0, sizeof(long long), st));
  // momentum table of this call, continuing the stored t_k when resuming.
  // A fresh start without a state buffer reuses the table of an earlier
  // fresh start that covers `iters` (the sequence from t_1 = 1 is always the
  // same), which saves a serial FP64 kernel of about 0.8 us per iteration.
  SFS_TRY(ensure_beta(op, std::max(iters, 1)));
  const bool fresh = !resume;
  if (!(fresh && !state_dev && op->ws.beta_fresh >= iters)) {
    SFS_TRY(launch_fista_betas(resume ? st_t : nullptr, iters, op->ws.beta,
                               state_dev ? st_t : op->ws.tnext, state_dev ? st_k : nullptr, st));
    op->ws.beta_fresh = fresh ? iters : 0;
  }
  // thresholds: lambda/L and 1/L, with the mu rule evaluated on the device
  const int use_mu = lambda < 0;
  if (use_mu) {
    unsigned int* bits = (unsigned int*)(op->ws.scal + kLamMax);
    SFS_CUDA(cudaMemsetAsync(bits, 0, sizeof(unsigned int), st));
    SFS_TRY(enqueue_AH(op, y, nullptr, nullptr, bits, st));
  }
  SFS_TRY(launch_set_thresholds(op->ws.scal, op->ws.red, use_mu ? 0.0 : lambda, L, use_mu,
                                use_mu ? -lambda : 0.0, op->ws.err, st));
  double* obj = nullptr;
  if (obj_hist_host && iters > 0) {
    SFS_TRY(ensure_obj(op, iters));
    obj = op->ws.obj;
    SFS_CUDA(cudaMemsetAsync(obj, 0, 2 * sizeof(double) * iters, st));
  }
  const bool timing = (flags & SFS_FISTA_TIME_KERNELS) != 0;
  if (timing) {
    SFS_TRY(ensure_events(op, 5 * timed_iters(iters)));
    op->ev_used = 0;
  }
  if (iters > 0) {
    cudaGraphExec_t exec = nullptr;
    SFS_TRY(fista_graph(op, iters, obj != nullptr, timing, &exec));
    SFS_CUDA(cudaGraphLaunch(exec, st));
  }
  if (timing) op->ev_used = timed_iters(iters);
  SFS_CUDA(cudaMemcpyAsync(x_inout_dev, op->ws.xk, vbytes, cudaMemcpyDeviceToDevice, st));
  if (state_dev) {
    SFS_CUDA(cudaMemcpyAsync(st_gam, op->ws.gam, vbytes, cudaMemcpyDeviceToDevice, st));
    SFS_CUDA(cudaMemcpyAsync(st_x, op->ws.xk, vbytes, cudaMemcpyDeviceToDevice, st));
  }
  if (obj) {
    std::vector<double> h(2 * (size_t)iters);
    double lam = 0.0;
    SFS_CUDA(cudaMemcpyAsync(h.data(), obj, h.size() * sizeof(double), cudaMemcpyDeviceToHost, st));
    SFS_CUDA(cudaMemcpyAsync(&lam, op->ws.red + kNumRed - 1, sizeof(double),
                             cudaMemcpyDeviceToHost, st));
    SFS_CUDA(cudaStreamSynchronize(st));
    SFS_TRY(check_err_flag(op, st));
    for (int k = 0; k < iters; ++k) obj_hist_host[k] = 0.5 * h[2 * k] + lam * h[2 * k + 1];
  }
  return SFS_OK;
}

int sfs_set_wait_timeout_ns(sfs_operator* op, uint64_t ns) {
  clear_error();
  if (!op || ns == 0) {
    set_error("invalid argument");
    return SFS_ERR_INVALID_ARG;
  }
  DeviceScope scope(op->geo.d.device);
  op->wait_ns = ns;
  // captured iteration loops carry the old limit as a kernel argument
  for (auto& ge : op->graphs) cudaGraphExecDestroy(ge.exec);
  op->graphs.clear();
  for (auto& ge : op->bgraphs) cudaGraphExecDestroy(ge.exec);
  op->bgraphs.clear();
  return SFS_OK;
}

int sfs_inject_wait_timeout(sfs_operator* op, int enable) {
  clear_error();
  if (!op) {
    set_error("null argument");
    return SFS_ERR_INVALID_ARG;
  }
  DeviceScope scope(op->geo.d.device);
  op->inject = enable ? 1 : 0;
  for (auto& ge : op->graphs) cudaGraphExecDestroy(ge.exec);
  op->graphs.clear();
  for (auto& ge : op->bgraphs) cudaGraphExecDestroy(ge.exec);
  op->bgraphs.clear();
  return SFS_OK;
}

int sfs_check_status(sfs_operator* op, void* stream) {
  clear_error();
  if (!op) {
    set_error("null argument");
    return SFS_ERR_INVALID_ARG;
  }
  DeviceScope scope(op->geo.d.device);
  return check_err_flag(op, (cudaStream_t)stream);
}

int sfs_stage_times(sfs_operator* op, double* ms4, int32_t* n_out_host) {
  clear_error();
  if (!op || !ms4) {
    set_error("null argument");
    return SFS_ERR_INVALID_ARG;
  }
  DeviceScope scope(op->geo.d.device);
  double acc[4] = {0.0, 0.0, 0.0, 0.0};
  for (int k = 0; k < op->ev_used; ++k) {
    SFS_CUDA(cudaEventSynchronize(op->ev[5 * k + 4]));
    for (int j = 0; j < 4; ++j) {
      float t = 0.f;
      SFS_CUDA(cudaEventElapsedTime(&t, op->ev[5 * k + j], op->ev[5 * k + j + 1]));
      acc[j] += t;
    }
  }
  const int n = op->ev_used;
  for (int j = 0; j < 4; ++j) ms4[j] = n ? acc[j] / n : 0.0;
  if (n_out_host) *n_out_host = n;
  return SFS_OK;
}

int sfs_apply_A_batched(sfs_operator* op, int batch, const void* x_dev, void* y_dev, void* stream) {
  clear_error();
  if (!op || batch < 1 || batch > SFS_MAX_BATCH || !x_dev || !y_dev || !aligned16(x_dev) ||
      !aligned16(y_dev)) {
    set_error("invalid argument (batch must be 1..%d, pointers 16-byte aligned)", SFS_MAX_BATCH);
    return SFS_ERR_INVALID_ARG;
  }
  DeviceScope scope(op->geo.d.device);
  SFS_TRY(ensure_batch(op, batch));
  const PlaneDims d = batch_dims(op, batch);
  cudaStream_t st = (cudaStream_t)stream;
  SFS_TRY(launch_fwd_planes(d, (const float2*)x_dev, op->bws.Xh, st));
  SFS_TRY(launch_contract_fwd(d, op->table, op->bws.Xh, op->bws.Yh, op->ws.err, st));
  return launch_inv_gather(d, op->bws.Yh, op->posmap, (float2*)y_dev, nullptr, st);
}

int sfs_apply_AH_batched(sfs_operator* op, int batch, const void* y_dev, void* x_dev, void* stream) {
  clear_error();
  if (!op || batch < 1 || batch > SFS_MAX_BATCH || !x_dev || !y_dev || !aligned16(x_dev) ||
      !aligned16(y_dev)) {
    set_error("invalid argument (batch must be 1..%d, pointers 16-byte aligned)", SFS_MAX_BATCH);
    return SFS_ERR_INVALID_ARG;
  }
  DeviceScope scope(op->geo.d.device);
  SFS_TRY(ensure_batch(op, batch));
  const PlaneDims d = batch_dims(op, batch);
  cudaStream_t st = (cudaStream_t)stream;
  SFS_TRY(launch_scatter_fwd(d, (const float2*)y_dev, op->posmap, op->bws.Rh, st));
  SFS_TRY(launch_contract_adj(d, op->table, op->bws.Rh, op->bws.Gh, op->ws.err, st));
  return launch_inv_store(d, op->bws.Gh, op->ws.segslot, (float2*)x_dev, nullptr, nullptr, st);
}

int sfs_fista_batched(sfs_operator* op, int batch, const void* y_dev, double lambda, double L,
                      int iters, void* x_out_dev, uint32_t flags, void* stream) {
  clear_error();
  if (!op || batch < 1 || batch > SFS_MAX_BATCH || !y_dev || !x_out_dev || iters < 0 || !(L > 0) ||
      !isfinite(lambda) || !aligned16(y_dev) || !aligned16(x_out_dev) ||
      (flags & ~(uint32_t)SFS_FISTA_WARM_START)) {
    set_error("invalid argument");
    return SFS_ERR_INVALID_ARG;
  }
  DeviceScope scope(op->geo.d.device);
  SFS_TRY(ensure_batch(op, batch));
  const PlaneDims d = batch_dims(op, batch);
  const sfs::BatchWorkspace& w = op->bws;
  cudaStream_t st = (cudaStream_t)stream;
  const size_t B = (size_t)batch;
  SFS_CUDA(cudaMemcpyAsync(w.ybuf, y_dev, B * d.bs_y * sizeof(float2), cudaMemcpyDeviceToDevice, st));
  if (flags & SFS_FISTA_WARM_START) {
    SFS_CUDA(cudaMemcpyAsync(w.xk, x_out_dev, B * d.bs_x * sizeof(float2), cudaMemcpyDeviceToDevice, st));
    SFS_CUDA(cudaMemcpyAsync(w.gam, x_out_dev, B * d.bs_x * sizeof(float2), cudaMemcpyDeviceToDevice, st));
  } else {
    SFS_CUDA(cudaMemsetAsync(w.xk, 0, B * d.bs_x * sizeof(float2), st));
    SFS_CUDA(cudaMemsetAsync(w.gam, 0, B * d.bs_x * sizeof(float2), st));
  }
  const int use_mu = lambda < 0;
  SFS_CUDA(cudaMemsetAsync(w.scal, 0, B * kNumFloatScalars * sizeof(float), st));
  if (use_mu) {  // max |A^H y_b| of every scene, on the device
    SFS_TRY(launch_scatter_fwd(d, w.ybuf, op->posmap, w.Rh, st));
    SFS_TRY(launch_contract_adj(d, op->table, w.Rh, w.Gh, op->ws.err, st));
    SFS_TRY(launch_inv_store(d, w.Gh, op->ws.segslot, nullptr, nullptr,
                             (unsigned int*)(w.scal + kLamMax), st));
  }
  SFS_TRY(launch_set_thresholds_batched(w.scal, batch, use_mu ? 0.0 : lambda, L, use_mu,
                                        use_mu ? -lambda : 0.0, op->ws.err, st));
  if (iters > 0) {
    cudaGraphExec_t exec = nullptr;
    SFS_TRY(fista_graph_batched(op, iters, batch, &exec));
    SFS_CUDA(cudaGraphLaunch(exec, st));
  }
  SFS_CUDA(cudaMemcpyAsync(x_out_dev, w.xk, B * d.bs_x * sizeof(float2), cudaMemcpyDeviceToDevice, st));
  return SFS_OK;
}

namespace {

// Checks the groups of a grouped or persistent solve and prepares each
// group's workspace: measurements, zero state, thresholds (mu rule per
// scene).
int grouped_setup(int ngroups, sfs_operator* const* ops, const int32_t* batch, const void* const* y_dev,
                  const double* L, double lambda, int iters, void* const* x_out_dev, cudaStream_t st) {
  if (ngroups < 1 || ngroups > SFS_MAX_GROUPS || !ops || !batch || !y_dev || !L || !x_out_dev ||
      iters < 0 || !isfinite(lambda)) {
    set_error("invalid argument (1..%d groups)", SFS_MAX_GROUPS);
    return SFS_ERR_INVALID_ARG;
  }
  for (int g = 0; g < ngroups; ++g) {
    if (!ops[g] || batch[g] < 1 || batch[g] > SFS_MAX_BATCH || !(L[g] > 0) || !y_dev[g] || !x_out_dev[g] ||
        !aligned16(y_dev[g]) || !aligned16(x_out_dev[g]) || ops[g]->geo.d.device != ops[0]->geo.d.device) {
      set_error("invalid group %d (operator, batch 1..%d, L > 0, aligned buffers, one device)", g,
                SFS_MAX_BATCH);
      return SFS_ERR_INVALID_ARG;
    }
    for (int h = 0; h < g; ++h)
      if (ops[h] == ops[g]) {
        set_error("groups %d and %d share an operator (its batched workspace)", h, g);
        return SFS_ERR_INVALID_ARG;
      }
  }
  for (int g = 0; g < ngroups; ++g) SFS_TRY(ensure_batch(ops[g], batch[g]));
  {
    std::lock_guard<std::mutex> lock(g_grouped_mu);
    if (!g_grouped_start) SFS_CUDA(cudaEventCreate(&g_grouped_start));
    SFS_CUDA(cudaEventRecord(g_grouped_start, st));
    g_grouped_last_n = 0;
  }
  for (int g = 0; g < ngroups; ++g) {
    sfs_operator* op = ops[g];
    const PlaneDims d = batch_dims(op, batch[g]);
    const sfs::BatchWorkspace& w = op->bws;
    const size_t B = (size_t)batch[g];
    SFS_CUDA(cudaMemcpyAsync(w.ybuf, y_dev[g], B * d.bs_y * sizeof(float2), cudaMemcpyDeviceToDevice, st));
    SFS_CUDA(cudaMemsetAsync(w.xk, 0, B * d.bs_x * sizeof(float2), st));
    SFS_CUDA(cudaMemsetAsync(w.gam, 0, B * d.bs_x * sizeof(float2), st));
    SFS_CUDA(cudaMemsetAsync(w.scal, 0, B * kNumFloatScalars * sizeof(float), st));
    const int use_mu = lambda < 0;
    if (use_mu) {
      SFS_TRY(launch_scatter_fwd(d, w.ybuf, op->posmap, w.Rh, st));
      SFS_TRY(launch_contract_adj(d, op->table, w.Rh, w.Gh, op->ws.err, st));
      SFS_TRY(launch_inv_store(d, w.Gh, op->ws.segslot, nullptr, nullptr, (unsigned int*)(w.scal + kLamMax), st));
    }
    SFS_TRY(launch_set_thresholds_batched(w.scal, batch[g], use_mu ? 0.0 : lambda, L[g], use_mu,
                                          use_mu ? -lambda : 0.0, op->ws.err, st));
  }
  return SFS_OK;
}

int grouped_results(int ngroups, sfs_operator* const* ops, const int32_t* batch, void* const* x_out_dev,
                    cudaStream_t st) {
  for (int g = 0; g < ngroups; ++g) {
    const PlaneDims d = batch_dims(ops[g], batch[g]);
    SFS_CUDA(cudaMemcpyAsync(x_out_dev[g], ops[g]->bws.xk, (size_t)batch[g] * d.bs_x * sizeof(float2),
                             cudaMemcpyDeviceToDevice, st));
  }
  return SFS_OK;
}

}  // namespace

int sfs_set_grouped_order(int order) {
  if (order != SFS_GROUPED_CHEAPEST_FIRST && order != SFS_GROUPED_LARGEST_FIRST &&
      order != SFS_GROUPED_NO_PRIORITY) {
    set_error("grouped order %d (0 cheapest first, 1 largest first, 2 no priority)", order);
    return SFS_ERR_INVALID_ARG;
  }
  g_grouped_order.store(order);
  return SFS_OK;
}

int sfs_fista_grouped(int ngroups, sfs_operator* const* ops, const int32_t* batch,
                      const void* const* y_dev, const double* L, double lambda, int iters,
                      void* const* x_out_dev, void* stream) {
  clear_error();
  if (ngroups < 1 || !ops || !ops[0]) {
    set_error("invalid argument (1..%d groups)", SFS_MAX_GROUPS);
    return SFS_ERR_INVALID_ARG;
  }
  DeviceScope scope(ops[0]->geo.d.device);
  cudaStream_t st = (cudaStream_t)stream;
  SFS_TRY(grouped_setup(ngroups, ops, batch, y_dev, L, lambda, iters, x_out_dev, st));
  if (iters > 0) {
    cudaGraphExec_t exec = nullptr;
    SFS_TRY(grouped_graph(ngroups, ops, batch, iters, &exec));
    SFS_CUDA(cudaGraphLaunch(exec, st));
    std::lock_guard<std::mutex> lock(g_grouped_mu);
    g_grouped_last_n = ngroups;
  }
  return grouped_results(ngroups, ops, batch, x_out_dev, st);
}

int sfs_fista_persistent(int ngroups, sfs_operator* const* ops, const int32_t* batch,
                         const void* const* y_dev, const double* L, double lambda, int iters,
                         void* const* x_out_dev, int nb_policy, void* stream) {
  clear_error();
  if (ngroups < 1 || ngroups > SFS_MAX_GROUPS || !ops ||
      (nb_policy != 0 && nb_policy != 1 && nb_policy != 2 && nb_policy != 4)) {
    set_error("invalid argument (1..%d groups, scenes per table tile 0, 1, 2 or 4)", SFS_MAX_GROUPS);
    return SFS_ERR_INVALID_ARG;
  }
  for (int g = 0; g < ngroups; ++g) {
    const sfs_operator* op = ops[g];
    if (!op || op->tc != 2 || op->nparts != 1 || op->geo.Py == 1 ||
        (op->geo.Px != 32 && op->geo.Px != 64 && op->geo.Px != 128)) {
      set_error("group %d: the persistent solve runs area-scan operators with a one-part 16-bit table "
                "(SFS_PREC_BF16 or SFS_PREC_FP16)", g);
      return SFS_ERR_INVALID_ARG;
    }
  }
  DeviceScope scope(ops[0]->geo.d.device);
  cudaStream_t st = (cudaStream_t)stream;
  SFS_TRY(grouped_setup(ngroups, ops, batch, y_dev, L, lambda, iters, x_out_dev, st));
  if (iters > 0) {
    cudaGraphExec_t exec = nullptr;
    SFS_TRY(persistent_graph(ngroups, ops, batch, iters, nb_policy, &exec));
    SFS_CUDA(cudaGraphLaunch(exec, st));
  }
  return grouped_results(ngroups, ops, batch, x_out_dev, st);
}

int sfs_autotune_persistent(int ngroups, sfs_operator* const* ops, const int32_t* batch,
                            const void* const* y_dev, const double* L, double lambda, int probe_iters,
                            int reps, void* const* x_out_dev, int32_t* policy_out, double* ms_out,
                            void* stream) {
  clear_error();
  if (!policy_out || probe_iters < 1 || reps < 1 || ngroups < 1 || !ops || !ops[0]) {
    set_error("invalid argument");
    return SFS_ERR_INVALID_ARG;
  }
  static const int kPolicies[4] = {0, 1, 2, 4};
  if (ms_out)
    for (int i = 0; i < 4; ++i) ms_out[i] = NAN;
  *policy_out = -1;
  DeviceScope scope(ops[0]->geo.d.device);
  cudaStream_t st = (cudaStream_t)stream;
  cudaEvent_t e0 = nullptr, e1 = nullptr;
  SFS_CUDA(cudaEventCreate(&e0));
  if (cudaEventCreate(&e1) != cudaSuccess) {
    cudaEventDestroy(e0);
    set_error("cudaEventCreate failed");
    return SFS_ERR_CUDA;
  }
  int rc = SFS_OK;
  double best = 0.0;
  for (int i = 0; i < 4 && rc == SFS_OK; ++i) {
    const int pol = kPolicies[i];
    // the first solve builds and captures the plan
    rc = sfs_fista_persistent(ngroups, ops, batch, y_dev, L, lambda, probe_iters, x_out_dev, pol, stream);
    if (rc != SFS_OK) break;
    cudaEventRecord(e0, st);
    for (int k = 0; k < reps && rc == SFS_OK; ++k)
      rc = sfs_fista_persistent(ngroups, ops, batch, y_dev, L, lambda, probe_iters, x_out_dev, pol, stream);
    if (rc != SFS_OK) break;
    cudaEventRecord(e1, st);
    const cudaError_t e = cudaEventSynchronize(e1);
    if (e != cudaSuccess) {
      rc = cuda_fail(e, "tuning run", __FILE__, __LINE__);
      break;
    }
    float ms = 0.f;
    cudaEventElapsedTime(&ms, e0, e1);
    const double per = (double)ms / reps;
    if (ms_out) ms_out[i] = per;
    if (*policy_out < 0 || per < best) {
      *policy_out = pol;
      best = per;
    }
  }
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  SFS_TRY(rc);
  return check_err_flag(ops[0], st);
}

int sfs_persistent_step_times(double* ms_out_host) {
  clear_error();
  if (!ms_out_host) {
    set_error("invalid argument");
    return SFS_ERR_INVALID_ARG;
  }
  std::lock_guard<std::mutex> lock(g_grouped_mu);
  if (g_last_persist_key.empty()) {
    set_error("no persistent solve to report");
    return SFS_ERR_INVALID_ARG;
  }
  std::vector<uint64_t> key(g_last_persist_key.begin(), g_last_persist_key.end() - 1);
  const int dev = (int)g_last_persist_key.back();
  for (auto& e : g_grouped)
    if (e.key == key && e.device == dev && e.plan) {
      DeviceScope scope(dev);
      SFS_CUDA(cudaDeviceSynchronize());
      return persist_step_ms(e.plan, ms_out_host);
    }
  set_error("the latest persistent solve's plan is no longer cached");
  return SFS_ERR_INVALID_ARG;
}

int sfs_grouped_times(int ngroups, float* ms_out_host) {
  clear_error();
  std::lock_guard<std::mutex> lock(g_grouped_mu);
  if (!ms_out_host || ngroups < 1 || ngroups != g_grouped_last_n || !g_grouped_start) {
    set_error("no grouped solve of %d groups to report", ngroups);
    return SFS_ERR_INVALID_ARG;
  }
  for (int g = 0; g < ngroups; ++g) {
    SFS_CUDA(cudaEventSynchronize(g_done_events[g]));
    SFS_CUDA(cudaEventElapsedTime(&ms_out_host[g], g_grouped_start, g_done_events[g]));
  }
  return SFS_OK;
}

int sfs_kernel_times(sfs_operator* op, double* fwd_ms, double* adj_ms, int32_t* n_out_host) {
  clear_error();
  if (!op || !fwd_ms || !adj_ms) {
    set_error("null argument");
    return SFS_ERR_INVALID_ARG;
  }
  double ms4[4];
  SFS_TRY(sfs_stage_times(op, ms4, n_out_host));
  *fwd_ms = ms4[0];
  *adj_ms = ms4[2];
  return SFS_OK;
}


// Scenes per table tile of a batched 16-bit contraction (0: the default
// rule).  Loops captured for this batch size are dropped, and grouped loops
// see a new workspace generation.
static void set_batch_tile(sfs_operator* op, int batch, int nb) {
  for (auto it = op->batch_tile.begin(); it != op->batch_tile.end();)
    it = it->first == batch ? op->batch_tile.erase(it) : it + 1;
  if (nb) op->batch_tile.push_back({batch, nb});
  for (auto it = op->bgraphs.begin(); it != op->bgraphs.end();) {
    if (it->batch == batch) {
      cudaGraphExecDestroy(it->exec);
      it = op->bgraphs.erase(it);
    } else {
      ++it;
    }
  }
  ++op->bws_gen;
}

int sfs_set_batch_tile(sfs_operator* op, int batch, int nb) {
  clear_error();
  if (!op || batch < 1 || batch > SFS_MAX_BATCH || (nb != 0 && nb != 1 && nb != 2 && nb != 4)) {
    set_error("invalid argument");
    return SFS_ERR_INVALID_ARG;
  }
  DeviceScope scope(op->geo.d.device);
  set_batch_tile(op, batch, nb);
  return SFS_OK;
}

int sfs_autotune_batch(sfs_operator* op, int batch, int reps, int32_t* nb_out, double* ms_out) {
  clear_error();
  if (!op || batch < 1 || batch > SFS_MAX_BATCH || reps < 1 || !nb_out) {
    set_error("invalid argument");
    return SFS_ERR_INVALID_ARG;
  }
  if (ms_out) ms_out[0] = ms_out[1] = ms_out[2] = NAN;
  *nb_out = 0;
  if (op->tc != 2) return SFS_OK;  // only the 16-bit contractions share table tiles
  DeviceScope scope(op->geo.d.device);
  SFS_TRY(ensure_batch(op, batch));
  const sfs::BatchWorkspace& w = op->bws;
  PlaneDims d = batch_dims(op, batch);
  // defined inputs (zero spectra; zero maxima give scale 1 in FP16 modes)
  SFS_CUDA(cudaMemset(w.Xh, 0, (size_t)batch * d.bs_xh * sizeof(float2)));
  SFS_CUDA(cudaMemset(w.Rh, 0, (size_t)batch * d.bs_rh * sizeof(float2)));
  if (w.pmx) SFS_CUDA(cudaMemset(w.pmx, 0, (size_t)batch * d.bs_pmx * sizeof(float)));
  if (w.pmr) SFS_CUDA(cudaMemset(w.pmr, 0, (size_t)batch * d.bs_pmr * sizeof(float)));
  cudaStream_t st = nullptr;
  cudaEvent_t e0 = nullptr, e1 = nullptr;
  SFS_CUDA(cudaStreamCreateWithFlags(&st, cudaStreamNonBlocking));
  int rc = SFS_OK;
  double best_ms = 0.0;
  int best = 0;
  const int cand[3] = {1, 2, 4};
  if (cudaEventCreate(&e0) != cudaSuccess || cudaEventCreate(&e1) != cudaSuccess) {
    rc = cuda_fail(cudaGetLastError(), "cudaEventCreate", __FILE__, __LINE__);
  }
  for (int c = 0; c < 3 && rc == SFS_OK; ++c) {
    if (cand[c] > 1 && cand[c] / 2 >= batch) break;  // a tile wider than the batch needs
    d.nb = cand[c];
    if ((rc = prepare_kernels(d)) != SFS_OK) break;
    for (int r = -1; r < reps && rc == SFS_OK; ++r) {  // r = -1: warm-up
      if (r == 0) cudaEventRecord(e0, st);
      rc = launch_contract_fwd(d, op->table, w.Xh, w.Yh, op->ws.err, st);
      if (rc == SFS_OK) rc = launch_contract_adj(d, op->table, w.Rh, w.Gh, op->ws.err, st);
    }
    if (rc != SFS_OK) break;
    cudaEventRecord(e1, st);
    const cudaError_t e = cudaEventSynchronize(e1);
    if (e != cudaSuccess) {
      rc = cuda_fail(e, "tuning run", __FILE__, __LINE__);
      break;
    }
    float ms = 0.f;
    cudaEventElapsedTime(&ms, e0, e1);
    const double per = (double)ms / reps;
    if (ms_out) ms_out[c] = per;
    if (!best || per < best_ms) {
      best = cand[c];
      best_ms = per;
    }
  }
  if (e0) cudaEventDestroy(e0);
  if (e1) cudaEventDestroy(e1);
  cudaStreamDestroy(st);
  SFS_TRY(rc);
  SFS_TRY(check_err_flag(op, nullptr));
  set_batch_tile(op, batch, best);
  *nb_out = best;
  return SFS_OK;
}

}  // extern "C"
