// Cramer-Rao bound on the location of one scatterer (Sec. VI, Eq. "fim").
//
// One scatterer at the continuous position p = (x1, y1, z1) with amplitude
// a e^{j phi} leaves, at kept bin k of scan position s (Eq. (4), Sigma = I),
//   b = a e^{j phi} fs H(f_k) g_s(p) exp(-j 2 pi f_k (tau_s(p) - t0)).
// Every derivative of b is b times a coefficient:
//   d/dp: (d ln g / dp - j w_k d tau / dp),  d/da: 1 / a,  d/dphi: j,
// with w_k = 2 pi f_k, d tau / dp = (2 / c) (p - (x_s, y_s, 0)) / R_s, and for
// g = exp(-r^2 / (z1 tan theta)^2): d ln g / dx1 = -2 (x1 - x_s) / (z1 tan
// theta)^2 (y1 alike), d ln g / dz1 = 2 r^2 / (z1^3 tan^2 theta).  So the
// Slepian-Bangs information J = (2 / sigma^2) Re{D^H D} is a sum over rows of
// |b|^2 Re{conj(c_i) c_j}, which needs no phase at all:
//   (p_i, p_j): dlng_i dlng_j + w^2 dtau_i dtau_j,  (p_i, a): dlng_i / a,
//   (p_i, phi): -w dtau_i,  (a, a): 1 / a^2,  (a, phi): 0,  (phi, phi): 1.
// One thread per row (s, m) of one index set, FP64 throughout; each CTA
// leaves the 15 upper-triangle partial sums of its rows, summed on the host
// in block order (deterministic).  The host then inverts J over the chosen
// parameters (Gauss-Jordan with partial pivoting, FP64) and reports the
// diagonal of its location block.
#include <cuda_runtime.h>
#include <math.h>
#include <stdint.h>
#include <string.h>

#include <utility>
#include <vector>

#include "sfs_internal.h"

namespace sfs {
namespace {

constexpr int kCrbThreads = 256;
constexpr int kTri = 15;  // upper triangle of the 5 x 5 information (x, y, z, a, phi)

struct CrbArgs {
  int Nx, S, M, Nt;
  double dx, dy, c, fs, tan_theta;  // tan_theta = 0: no directivity
  double x1, y1, z1, amp;
};

__global__ void __launch_bounds__(kCrbThreads) crb_partials_kernel(CrbArgs a, const int32_t* __restrict__ idx,
                                                                   const double* __restrict__ fsH,
                                                                   double* __restrict__ part) {
  const int t = blockIdx.y;
  const int r = blockIdx.x * kCrbThreads + threadIdx.x;
  const long long rows = (long long)a.S * a.M;
  double acc[kTri];
#pragma unroll
  for (int i = 0; i < kTri; ++i) acc[i] = 0.0;
  if (r < rows) {
    const int s = r / a.M;
    const int k = idx[(long long)t * rows + r];
    const double xs = (double)(s % a.Nx) * a.dx, ys = (double)(s / a.Nx) * a.dy;
    const double ex = a.x1 - xs, ey = a.y1 - ys;
    const double R = sqrt(ex * ex + ey * ey + a.z1 * a.z1);
    const double w = 2.0 * M_PI * (double)k * a.fs / (double)a.Nt;
    double dl[3] = {0.0, 0.0, 0.0};
    double gsq = 1.0;
    if (a.tan_theta > 0.0) {
      const double wz = a.z1 * a.tan_theta, r2 = ex * ex + ey * ey;
      gsq = exp(-2.0 * r2 / (wz * wz));
      dl[0] = -2.0 * ex / (wz * wz);
      dl[1] = -2.0 * ey / (wz * wz);
      dl[2] = 2.0 * r2 / (a.z1 * wz * wz);
    }
    const double dt[3] = {2.0 / a.c * ex / R, 2.0 / a.c * ey / R, 2.0 / a.c * a.z1 / R};
    const double h = a.amp * fsH[k];
    const double b2 = h * h * gsq;  // |b|^2
    int q = 0;
#pragma unroll
    for (int i = 0; i < 3; ++i) {
#pragma unroll
      for (int j = i; j < 3; ++j) acc[q++] = b2 * (dl[i] * dl[j] + w * w * dt[i] * dt[j]);
      acc[q++] = b2 * dl[i] / a.amp;  // (p_i, a)
      acc[q++] = -b2 * w * dt[i];     // (p_i, phi)
    }
    acc[q++] = b2 / (a.amp * a.amp);  // (a, a)
    acc[q++] = 0.0;                   // (a, phi)
    acc[q++] = b2;                    // (phi, phi)
  }
  __shared__ double red[kTri][kCrbThreads / 32];
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
#pragma unroll
  for (int i = 0; i < kTri; ++i) {
    double v = acc[i];
#pragma unroll
    for (int off = 16; off > 0; off >>= 1) v += __shfl_xor_sync(0xffffffffu, v, off);
    if (lane == 0) red[i][warp] = v;
  }
  __syncthreads();
  if (threadIdx.x < kTri) {
    double v = 0.0;
#pragma unroll
    for (int w = 0; w < kCrbThreads / 32; ++w) v += red[threadIdx.x][w];
    part[((long long)t * gridDim.x + blockIdx.x) * kTri + threadIdx.x] = v;
  }
}

// Order of the 15 sums: for i = x, y, z: (i, j >= i within xyz), (i, a),
// (i, phi); then (a, a), (a, phi), (phi, phi).  Expands to the symmetric 5 x 5.
void unpack(const double* tri, double J[5][5]) {
  int q = 0;
  for (int i = 0; i < 3; ++i) {
    for (int j = i; j < 3; ++j) J[i][j] = J[j][i] = tri[q++];
    J[i][3] = J[3][i] = tri[q++];
    J[i][4] = J[4][i] = tri[q++];
  }
  J[3][3] = tri[q++];
  J[3][4] = J[4][3] = tri[q++];
  J[4][4] = tri[q++];
}

// Inverse of the n x n matrix A (row-major, n <= 5) by Gauss-Jordan with
// partial pivoting; false if a pivot falls below 1e-13 of the largest entry.
bool invert(int n, double* A, double* inv) {
  double big = 0.0;
  for (int i = 0; i < n * n; ++i) big = fmax(big, fabs(A[i]));
  for (int i = 0; i < n; ++i)
    for (int j = 0; j < n; ++j) inv[i * n + j] = i == j ? 1.0 : 0.0;
  for (int col = 0; col < n; ++col) {
    int piv = col;
    for (int r = col + 1; r < n; ++r)
      if (fabs(A[r * n + col]) > fabs(A[piv * n + col])) piv = r;
    if (!(fabs(A[piv * n + col]) > 1e-13 * big)) return false;
    if (piv != col)
      for (int j = 0; j < n; ++j) {
        std::swap(A[piv * n + j], A[col * n + j]);
        std::swap(inv[piv * n + j], inv[col * n + j]);
      }
    const double d = A[col * n + col];
    for (int j = 0; j < n; ++j) {
      A[col * n + j] /= d;
      inv[col * n + j] /= d;
    }
    for (int r = 0; r < n; ++r) {
      if (r == col) continue;
      const double f = A[r * n + col];
      if (f == 0.0) continue;
      for (int j = 0; j < n; ++j) {
        A[r * n + j] -= f * A[col * n + j];
        inv[r * n + j] -= f * inv[col * n + j];
      }
    }
  }
  return true;
}

struct DevBuf {
  void* p = nullptr;
  ~DevBuf() { cudaFree(p); }
};

}  // namespace
}  // namespace sfs

using namespace sfs;

extern "C" int sfs_crb(const sfs_geometry* g, int T, int M, const int32_t* idx_host, const double* pos,
                       double amp, double phase, double sigma2, int param_mask, double* crb_out_host,
                       double* fim_out_host) {
  clear_error();
  (void)phase;  // the information does not depend on the phase (see above)
  if (!g || !idx_host || !pos || !crb_out_host) {
    set_error("null argument");
    return SFS_ERR_INVALID_ARG;
  }
  const sfs_geometry_desc& d = g->d;
  const int S = d.Nx * d.Ny, kmax = d.Nt / 2;
  const long long rows = (long long)S * M;
  if (T < 1 || T > 65535 || M < 1 || M > kmax + 1 || rows * T >= (1ll << 31)) {
    set_error("sizes out of range (T = %d, M = %d)", T, M);
    return SFS_ERR_INVALID_ARG;
  }
  if (!(amp > 0.0) || !(sigma2 > 0.0) || !(pos[2] > 0.0) || !isfinite(pos[0]) || !isfinite(pos[1]) ||
      (param_mask & 7) == 0 || (param_mask & ~7) != 0) {
    set_error("need amp > 0, sigma2 > 0, depth z1 > 0, finite position and a mask of x/y/z bits");
    return SFS_ERR_INVALID_ARG;
  }
  for (long long r = 0; r < rows * T; ++r) {
    const int k = idx_host[r];
    const bool first = (r % M) == 0;
    if (k < 0 || k > kmax || (!first && k <= idx_host[r - 1])) {
      set_error("index row %lld is not strictly ascending inside 0..%d", r / M, kmax);
      return SFS_ERR_INVALID_ARG;
    }
  }
  std::vector<double> fsH(kmax + 1);
  for (int k = 0; k <= kmax; ++k) fsH[k] = d.fs * pulse_mag((double)k * d.fs / d.Nt, d.fc, g->alpha);
  CrbArgs a;
  a.Nx = d.Nx;
  a.S = S;
  a.M = M;
  a.Nt = d.Nt;
  a.dx = d.dx;
  a.dy = d.dy;
  a.c = d.c;
  a.fs = d.fs;
  a.tan_theta = d.theta > 0.0 ? tan(d.theta) : 0.0;
  a.x1 = pos[0];
  a.y1 = pos[1];
  a.z1 = pos[2];
  a.amp = amp;
  const int nblk = (int)((rows + kCrbThreads - 1) / kCrbThreads);
  int prev = -1;
  if (cudaGetDevice(&prev) != cudaSuccess) prev = -1;
  cudaError_t e = cudaSetDevice(d.device);
  if (e != cudaSuccess) return cuda_fail(e, "selecting the geometry's device", __FILE__, __LINE__);
  struct Restore {
    int dev;
    ~Restore() {
      if (dev >= 0) cudaSetDevice(dev);
    }
  } restore{prev};
  DevBuf didx, dH, dpart;
  SFS_CUDA(cudaMalloc(&didx.p, (size_t)rows * T * sizeof(int32_t)));
  SFS_CUDA(cudaMalloc(&dH.p, fsH.size() * sizeof(double)));
  SFS_CUDA(cudaMalloc(&dpart.p, (size_t)T * nblk * kTri * sizeof(double)));
  SFS_CUDA(cudaMemcpy(didx.p, idx_host, (size_t)rows * T * sizeof(int32_t), cudaMemcpyHostToDevice));
  SFS_CUDA(cudaMemcpy(dH.p, fsH.data(), fsH.size() * sizeof(double), cudaMemcpyHostToDevice));
  crb_partials_kernel<<<dim3(nblk, T), kCrbThreads>>>(a, (const int32_t*)didx.p, (const double*)dH.p,
                                                       (double*)dpart.p);
  SFS_CUDA(cudaGetLastError());
  std::vector<double> part((size_t)T * nblk * kTri);
  SFS_CUDA(cudaMemcpy(part.data(), dpart.p, part.size() * sizeof(double), cudaMemcpyDeviceToHost));
  int act[5], n = 0;
  for (int i = 0; i < 3; ++i)
    if (param_mask & (1 << i)) act[n++] = i;
  act[n++] = 3;
  act[n++] = 4;
  for (int t = 0; t < T; ++t) {
    double tri[kTri];
    for (int q = 0; q < kTri; ++q) {
      double v = 0.0;
      for (int b = 0; b < nblk; ++b) v += part[((size_t)t * nblk + b) * kTri + q];
      tri[q] = v * (2.0 / sigma2);
    }
    double J[5][5];
    unpack(tri, J);
    if (fim_out_host) {
      for (int i = 0; i < 5; ++i)
        for (int j = 0; j < 5; ++j) {
          const bool on = (i >= 3 || (param_mask & (1 << i))) && (j >= 3 || (param_mask & (1 << j)));
          fim_out_host[(size_t)t * 25 + i * 5 + j] = on ? J[i][j] : 0.0;
        }
    }
    double A[25], inv[25];
    for (int i = 0; i < n; ++i)
      for (int j = 0; j < n; ++j) A[i * n + j] = J[act[i]][act[j]];
    if (!invert(n, A, inv)) {
      set_error("Fisher information of index set %d is singular for the chosen parameters", t);
      return SFS_ERR_INVALID_ARG;
    }
    for (int i = 0; i < 3; ++i) crb_out_host[(size_t)t * 3 + i] = NAN;
    for (int i = 0; i < n; ++i)
      if (act[i] < 3) crb_out_host[(size_t)t * 3 + act[i]] = inv[i * n + i];
  }
  return SFS_OK;
}
