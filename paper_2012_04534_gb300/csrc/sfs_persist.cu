// The FISTA iteration loop of many scene groups (serving: scenes of different
// scan grids, depths and bin counts) as one persistent kernel.
//
// Algorithm 1 for every scene of every group, iteration k:
//   1. forward contraction of every group's spectra X^ of gamma_k (16-bit
//      tensor-core table, Sec. IV-B / Algorithm 2);
//   2. residual planes: inverse lateral FFT, A gamma_k - y at the kept
//      positions, forward FFT of the residual;
//   3. adjoint contraction of the residual spectra;
//   4. update planes: inverse FFT of the gradient, soft threshold, momentum,
//      forward FFT of gamma_{k+1}.
// One cooperative launch of one 1024-thread CTA per SM runs all iterations:
// its warps 0-6 run the contraction roles in contraction steps, and in plane
// steps its two 512-thread groups each transform their own plane (named
// barriers per group, their own shared memory).
// Each step's work of all groups is one list of tasks handed out one at a
// time from a counter per step: runs of contraction units of every (group,
// scene tile) job of about equal table bytes (a unit's accumulator lives in
// one CTA's tensor memory, so a unit is never split), largest first, or the
// planes of every (group, scene), groups with the largest planes first.  The
// CTAs meet at a grid barrier after each step (a global arrival counter,
// waited on with a time limit: a CTA that gives up sets the error flag and
// the kernel ends).  The contraction and plane steps are the code of the
// standalone kernels (sfs_tc16_dev.cuh, sfs_planes.cuh), so a persistent
// solve computes what the grouped one computes, up to the plane engine
// variant (the cluster plane kernels of sfs_kernels.cu add the inverse
// quadrant shares in another order).
#include <cuda.h>
#include <cuda_runtime.h>
#include <stdint.h>

#include <algorithm>
#include <cmath>
#include <cstring>
#include <new>
#include <vector>

#include "sfs_async.cuh"
#include "sfs_internal.h"
#include "sfs_launch.h"
#include "sfs_planes.cuh"
#include "sfs_tc16_dev.cuh"

namespace sfs {
namespace {

constexpr int kPlaneThreads = 512;                 // one plane group (a plane engine)
constexpr int kPGroups = 2;                         // plane groups per CTA
constexpr int kPThreads = kPGroups * kPlaneThreads;  // warps 0-6 run the contraction roles
// shared memory of one plane group: the largest run-time plane (128 x 128 as
// quadrants), rounded to 128 bytes
constexpr int kPlaneSmem = (PlaneFFT<128, true>::SMEM + 127) / 128 * 128;
static_assert(PlaneFFT<64, true>::SMEM <= kPlaneSmem && PlaneFFT<32, true>::SMEM <= kPlaneSmem,
              "plane group shared memory");

// One group as the kernel reads it (device memory).
struct PGroup {
  PlaneDims d;  // batched dimensions: d.batch scenes, per-scene strides
  float2 *Xh, *Yh, *Rh, *Gh, *xk, *gam;
  const float2* yplane;
  const float* scal;
  const int32_t* posmap;
  const int2* segslot;
  int* err;
  int NB;                       // scenes per table tile
  int nmt_f, nch_f, nmt_a, nch_a;
  int map0;                     // maps[map0], maps[map0 + 1]: table (fwd, adj); then per scene tile
                                // j maps[map0 + 2 + 2 j] (X^), maps[map0 + 3 + 2 j] (R^)
};

struct PPlan {
  int ngroups, njobs, iters;
  const CUtensorMap* maps;
  const int2* job;              // contraction job: {group, scene tile}
  const int4* ctask_f;          // forward contraction tasks {job, first unit, units, -}, largest first
  const int4* ctask_a;          // adjoint contraction tasks
  int nct_f, nct_a;
  const int* porder;            // [ngroups] groups in plane-task order (largest planes first)
  const long long* cum_r;       // [ngroups + 1] cumulative residual planes (scenes x bins), porder
  const long long* cum_u;       // [ngroups + 1] cumulative update planes (scenes x depths), porder
  const float* beta;            // [iters] momentum coefficients from t_1 = 1
  unsigned int* arrivals;       // grid barrier counter, zero at launch
  unsigned int* tasks;          // [4 iters] task counters of the steps, zero at launch
  unsigned long long* step_ns;  // [4] time of each kind of step summed over the iterations (CTA 0's
                                //     view: from one barrier to the next), then [4] the CTAs' busy
                                //     time in each kind of step (before their barrier arrival)
                                //     summed over CTAs and iterations; zero at launch
  int* err;                     // set when a grid barrier wait gives up
  uint64_t wait_ns;
};

// The kernel's parameter: the plan and the groups, read through the
// constant cache (a __grid_constant__ parameter of at most 32 KB).
struct PParams {
  PPlan p;
  PGroup groups[SFS_MAX_GROUPS];
};
static_assert(sizeof(PParams) <= 32000, "kernel parameter size");

__device__ __forceinline__ unsigned int ld_acquire(const unsigned int* p) {
  unsigned int v;
  asm volatile("ld.acquire.gpu.global.u32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
  return v;
}

// Grid barrier number `epoch` (1, 2, ...): every CTA's writes before it are
// visible to every CTA after it, to plain loads and to bulk / tensor copies,
// and the shared memory a step leaves may be rewritten by the next step's
// copies.  False (for the whole CTA) when the wait gave up.
__device__ bool grid_sync(const PPlan& p, unsigned int epoch) {
  __shared__ int ok;
  fence_proxy_async_all();  // this step's accesses, either proxy, before the arrival
  __syncthreads();
  if (threadIdx.x == 0) {
    __threadfence();
    atomicAdd(p.arrivals, 1u);
    const unsigned int target = epoch * gridDim.x;
    int good = 1;
    if (ld_acquire(p.arrivals) < target) {
      const uint64_t t0 = global_ns();
      while (ld_acquire(p.arrivals) < target) {
        if (global_ns() - t0 > p.wait_ns) {
          atomicExch(p.err, 1);
          good = 0;
          break;
        }
        __nanosleep(64);
      }
    }
    __threadfence();
    ok = good;
  }
  __syncthreads();
  fence_proxy_async_all();  // the next step's copies and MMAs after it
  return ok != 0;
}

// The next task of step counter `ctr` for the whole CTA.
__device__ __forceinline__ long long next_task(unsigned int* ctr) {
  __shared__ unsigned int s_task;
  __syncthreads();  // every thread has read the previous value
  if (threadIdx.x == 0) s_task = atomicAdd(ctr, 1u);
  __syncthreads();
  return (long long)s_task;
}

// Step 1 or 3: contraction tasks (a run of units of one job, about the same
// number of table chunks each, largest first) taken one at a time from the
// step's counter.
template <bool FWD>
__device__ __forceinline__ void contract_step(const PParams& prm, int k, unsigned char* smem) {
  const PPlan& p = prm.p;
  const int4* tasks = FWD ? p.ctask_f : p.ctask_a;
  const long long T = FWD ? p.nct_f : p.nct_a;
  unsigned int* ctr = p.tasks + 4 * k + (FWD ? 0 : 2);
  for (long long t = next_task(ctr); t < T; t = next_task(ctr)) {
    const int4 tk = tasks[t];
    const int2 jb = p.job[tk.x];
    const PGroup& g = prm.groups[jb.x];
    const int s0 = jb.y * g.NB;
    const int nscene = min(g.NB, g.d.batch - s0);
    const CUtensorMap* tab = p.maps + g.map0 + (FWD ? 0 : 1);
    const CUtensorMap* spec = p.maps + g.map0 + 2 + 2 * jb.y + (FWD ? 0 : 1);
    float2* out = FWD ? g.Yh + s0 * g.d.bs_yh : g.Gh + s0 * g.d.bs_gh;
    const long long ostride = FWD ? g.d.bs_yh : g.d.bs_gh;
    const float* pm0 = FWD ? g.d.pm_x : g.d.pm_r;
    const float* pm = pm0 ? pm0 + s0 * (FWD ? g.d.bs_pmx : g.d.bs_pmr) : nullptr;
    const int nmt = FWD ? g.nmt_f : g.nmt_a, nch = FWD ? g.nch_f : g.nch_a;
    if (g.NB == 1)
      contract_h_run<FWD, 1, 1>(tab, spec, out, ostride, nscene, g.d, nmt, nch, tk.y, tk.z, pm, g.err, smem,
                                true);
    else if (g.NB == 2)
      contract_h_run<FWD, 1, 2>(tab, spec, out, ostride, nscene, g.d, nmt, nch, tk.y, tk.z, pm, g.err, smem,
                                true);
    else
      contract_h_run<FWD, 1, 4>(tab, spec, out, ostride, nscene, g.d, nmt, nch, tk.y, tk.z, pm, g.err, smem,
                                true);
  }
}

// The position (in porder) of the group of plane task t (cum: cumulative
// plane counts in that order).
__device__ __forceinline__ int group_of_task(const long long* cum, int ngroups, long long t) {
  int g = 0;
  while (g + 1 < ngroups && cum[g + 1] <= t) ++g;
  return g;
}



// The next plane task of step counter `ctr` for this thread's plane group.
__device__ __forceinline__ long long next_group_task(unsigned int* ctr) {
  __shared__ unsigned int s_gtask[kPGroups];
  const int grp = group_of<kPlaneThreads>();
  group_sync<kPlaneThreads>();  // the group has read the previous value
  if (gtid<kPlaneThreads>() == 0) s_gtask[grp] = atomicAdd(ctr, 1u);
  group_sync<kPlaneThreads>();
  return (long long)s_gtask[grp];
}

// The group's dimensions copied to shared memory for one plane task of this
// thread's plane group: the plane steps then read them with shared-memory
// loads instead of holding constant-bank copies in registers.  Called by
// every thread of the plane group.
__device__ __forceinline__ const PlaneDims& stage_dims(const PlaneDims& d) {
  __shared__ __align__(16) PlaneDims sd[kPGroups];
  static_assert(sizeof(PlaneDims) % 4 == 0, "word copy");
  const int grp = group_of<kPlaneThreads>();
  group_sync<kPlaneThreads>();  // earlier readers of sd[grp] are done
  const uint32_t* src = reinterpret_cast<const uint32_t*>(&d);
  uint32_t* dst = reinterpret_cast<uint32_t*>(&sd[grp]);
  for (int i = gtid<kPlaneThreads>(); i < (int)(sizeof(PlaneDims) / 4); i += kPlaneThreads) dst[i] = src[i];
  group_sync<kPlaneThreads>();
  return sd[grp];
}

// The plane steps as separate functions, so that each keeps the register
// allocation of its standalone kernel instead of sharing one with the rest
// of the persistent kernel.
template <int P>
__device__ __noinline__ void resid_plane_call(const PlaneDims& d, int u, long long b, float2* smem,
                                              const PGroup& g) {
  resid_plane_step<P, true>(d, u, b, smem, g.Yh, g.posmap, g.yplane, g.Rh, nullptr);
}
template <int P>
__device__ __noinline__ void update_plane_call(const PlaneDims& d, int z, long long b, float2* smem,
                                               const PGroup& g, float beta, int do_fwd) {
  update_plane_step<P, true>(d, z, b, smem, g.Gh, g.segslot, g.xk, g.gam, g.scal, beta, nullptr, do_fwd, g.Xh,
                             nullptr);
}

// Step 2: residual planes of every (group, scene, bin); each plane group of
// the CTA takes the next task from the step's counter, largest planes first,
// in its own part of the shared memory (smem: that part).
__device__ __forceinline__ void resid_step(const PParams& prm, int k, float2* smem) {
  const PPlan& p = prm.p;
  const long long T = p.cum_r[p.ngroups];
  unsigned int* ctr = p.tasks + 4 * k + 1;
  for (long long t = next_group_task(ctr); t < T; t = next_group_task(ctr)) {
    const int pos = group_of_task(p.cum_r, p.ngroups, t);
    const PGroup& g = prm.groups[p.porder[pos]];
    const PlaneDims& sd = stage_dims(g.d);
    const long long r = t - p.cum_r[pos];
    const long long b = r / sd.U;
    const int u = (int)(r - b * sd.U);
    if (sd.Px == 128)
      resid_plane_call<128>(sd, u, b, smem, g);
    else if (sd.Px == 64)
      resid_plane_call<64>(sd, u, b, smem, g);
    else
      resid_plane_call<32>(sd, u, b, smem, g);
    group_sync<kPlaneThreads>();  // the next plane reuses the shared memory
  }
}

// Step 4: update planes of every (group, scene, depth), taken likewise.
__device__ __forceinline__ void update_step(const PParams& prm, int k, float2* smem) {
  const PPlan& p = prm.p;
  const long long T = p.cum_u[p.ngroups];
  const float beta = p.beta[k];
  const int do_fwd = k + 1 < p.iters;
  unsigned int* ctr = p.tasks + 4 * k + 3;
  for (long long t = next_group_task(ctr); t < T; t = next_group_task(ctr)) {
    const int pos = group_of_task(p.cum_u, p.ngroups, t);
    const PGroup& g = prm.groups[p.porder[pos]];
    const PlaneDims& sd = stage_dims(g.d);
    const long long r = t - p.cum_u[pos];
    const long long b = r / sd.Nz;
    const int z = (int)(r - b * sd.Nz);
    if (sd.Px == 128)
      update_plane_call<128>(sd, z, b, smem, g, beta, do_fwd);
    else if (sd.Px == 64)
      update_plane_call<64>(sd, z, b, smem, g, beta, do_fwd);
    else
      update_plane_call<32>(sd, z, b, smem, g, beta, do_fwd);
    group_sync<kPlaneThreads>();
  }
}

__global__ void __launch_bounds__(kPThreads, 1) fista_persistent_kernel(const __grid_constant__ PParams prm) {
  extern __shared__ __align__(1024) unsigned char psm[];
  const PPlan& p = prm.p;
  unsigned int epoch = 0;
  const bool timer = blockIdx.x == 0 && threadIdx.x == 0;
  uint64_t t = timer ? global_ns() : 0;
  uint64_t busy[4] = {0, 0, 0, 0}, t_step = threadIdx.x == 0 ? global_ns() : 0;
  auto done = [&](int step) {  // thread 0 of every CTA, at the end of its share of a step
    if (threadIdx.x == 0) busy[step] += global_ns() - t_step;
  };
  auto mark = [&](int step) {  // after the barrier that ends a step
    if (threadIdx.x == 0) t_step = global_ns();
    if (timer) {
      p.step_ns[step] += t_step - t;
      t = t_step;
    }
  };
  for (int k = 0; k < p.iters; ++k) {
    contract_step<true>(prm, k, psm);
    done(0);
    if (!grid_sync(p, ++epoch)) return;
    mark(0);
    resid_step(prm, k, reinterpret_cast<float2*>(psm + group_of<kPlaneThreads>() * kPlaneSmem));
    done(1);
    if (!grid_sync(p, ++epoch)) return;
    mark(1);
    contract_step<false>(prm, k, psm);
    done(2);
    if (!grid_sync(p, ++epoch)) return;
    mark(2);
    update_step(prm, k, reinterpret_cast<float2*>(psm + group_of<kPlaneThreads>() * kPlaneSmem));
    done(3);
    if (k + 1 < p.iters && !grid_sync(p, ++epoch)) return;
    mark(3);  // the last update step: CTA 0's own end
  }
  if (threadIdx.x == 0)
    for (int i = 0; i < 4; ++i) atomicAdd(p.step_ns + 4 + i, (unsigned long long)busy[i]);
}

}  // namespace

// Plan of one persistent solve: the kernel parameter (plan and groups) on
// the host, and one device allocation holding the tensor maps, the job and
// task tables, the momentum coefficients and the barrier counter.
struct PersistPlan {
  PParams prm;
  void* blob = nullptr;
  int grid = 0;
  int smem = 0;
  int nb_policy = 0;
  size_t counters_bytes = 0;  // the barrier and task counters zeroed before each launch
};

namespace {

size_t align_up(size_t off, size_t a) { return (off + a - 1) / a * a; }

int plan_smem(int NB) {
  const int c = NB == 1 ? HPlan<1, 1>::kSmem : NB == 2 ? HPlan<1, 2>::kSmem : HPlan<1, 4>::kSmem;
  return std::max(c, kPGroups * kPlaneSmem);
}

}  // namespace

int persist_build(int ngroups, sfs_operator* const* ops, const PlaneDims* dims, int iters, int nb_policy,
                  PersistPlan** out) {
  *out = nullptr;
  if (ngroups < 1 || ngroups > SFS_MAX_GROUPS ||
      (nb_policy != 0 && nb_policy != 1 && nb_policy != 2 && nb_policy != 4)) {
    set_error("1..%d groups, scenes per table tile 0 (each group's own), 1, 2 or 4", SFS_MAX_GROUPS);
    return SFS_ERR_INVALID_ARG;
  }
  PersistPlan* pp = new (std::nothrow) PersistPlan;
  if (!pp) {
    set_error("host allocation failed");
    return SFS_ERR_OOM;
  }
  memset(&pp->prm, 0, sizeof(pp->prm));
  std::vector<CUtensorMap> maps;
  std::vector<int2> jobs;
  std::vector<long long> cum_r(1, 0), cum_u(1, 0);
  std::vector<int2> units_f, units_a;  // per job: {units, chunks per unit}
  int smem = 0;
  int rc = SFS_OK;
  for (int gi = 0; gi < ngroups && rc == SFS_OK; ++gi) {
    const sfs_operator* op = ops[gi];
    const PlaneDims& d = dims[gi];
    PGroup& g = pp->prm.groups[gi];
    g.d = d;
    const sfs::BatchWorkspace& w = op->bws;
    g.Xh = w.Xh;
    g.Yh = w.Yh;
    g.Rh = w.Rh;
    g.Gh = w.Gh;
    g.xk = w.xk;
    g.gam = w.gam;
    g.yplane = w.yplane;
    g.scal = w.scal;
    g.posmap = op->posmap;
    g.segslot = op->ws.segslot;
    g.err = op->ws.err;
    // scenes per table tile: the group's own choice, or the policy's (no
    // wider than the batch needs)
    if (nb_policy == 0) {
      g.NB = tc16_group_of(d);
    } else {
      const int B = std::max(1, d.batch);
      g.NB = std::min(nb_policy, B >= 3 ? 4 : B);
    }
    g.d.nb = g.NB;
    int nunits_f = 0, nunits_a = 0;
    tc16_units(d, true, &g.nmt_f, &g.nch_f, &nunits_f);
    tc16_units(d, false, &g.nmt_a, &g.nch_a, &nunits_a);
    g.map0 = (int)maps.size();
    maps.resize(maps.size() + 2);
    rc = tc16_table_maps(op, &maps[g.map0], &maps[g.map0 + 1]);
    const int B = std::max(1, d.batch);
    for (int s0 = 0, j = 0; s0 < B && rc == SFS_OK; s0 += g.NB, ++j) {
      CUtensorMap mx, mr;
      rc = tc16_encode_spec(&mx, w.Xh + s0 * d.bs_xh, d.Nz, d.Ns, 32, B - s0, g.NB);
      if (rc == SFS_OK) rc = tc16_encode_spec(&mr, w.Rh + s0 * d.bs_rh, d.Up, d.Ns, 64, B - s0, g.NB);
      maps.push_back(mx);
      maps.push_back(mr);
      jobs.push_back(make_int2(gi, j));
      units_f.push_back(make_int2(nunits_f, g.nch_f));
      units_a.push_back(make_int2(nunits_a, g.nch_a));
    }
    smem = std::max(smem, plan_smem(g.NB));
  }
  // plane tasks: groups with the largest planes first, so that the last
  // tasks a step hands out are the short ones
  std::vector<int> porder(ngroups);
  for (int g = 0; g < ngroups; ++g) porder[g] = g;
  std::stable_sort(porder.begin(), porder.end(), [&](int a, int b) { return dims[a].Px > dims[b].Px; });
  for (int i = 0; i < ngroups; ++i) {
    const PlaneDims& d = dims[porder[i]];
    const long long B = std::max(1, d.batch);
    cum_r.push_back(cum_r.back() + B * d.U);
    cum_u.push_back(cum_u.back() + B * d.Nz);
  }
  if (rc != SFS_OK) {
    persist_free(pp);
    return rc;
  }
  // contraction tasks: runs of units of about an eighth of a CTA's share of
  // the step's table chunks, largest first
  int dev = 0, sms = 0, occ = 0;
  {
    cudaError_t e0 = cudaGetDevice(&dev);
    if (e0 == cudaSuccess) e0 = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    if (e0 != cudaSuccess) {
      persist_free(pp);
      return cuda_fail(e0, "SM count", __FILE__, __LINE__);
    }
  }
  auto make_tasks = [&](const std::vector<int2>& units) {
    long long total = 0;
    for (const int2& u : units) total += (long long)u.x * u.y;
    const long long target = std::max(1LL, (total + 8LL * sms - 1) / (8LL * sms));
    std::vector<int4> t;
    for (int j = 0; j < (int)units.size(); ++j) {
      const int upt = (int)std::max(1LL, (target + units[j].y - 1) / units[j].y);
      for (int u0 = 0; u0 < units[j].x; u0 += upt)
        t.push_back(make_int4(j, u0, std::min(upt, units[j].x - u0), 0));
    }
    std::stable_sort(t.begin(), t.end(), [&](const int4& a, const int4& b) {
      return (long long)a.z * units[a.x].y > (long long)b.z * units[b.x].y;
    });
    return t;
  };
  const std::vector<int4> ctf = make_tasks(units_f), cta = make_tasks(units_a);
  std::vector<float> beta(std::max(iters, 1));
  {
    double t = 1.0;
    for (int k = 0; k < iters; ++k) {
      const double tn = 0.5 * (1.0 + sqrt(1.0 + 4.0 * t * t));
      beta[k] = (float)((t - 1.0) / tn);
      t = tn;
    }
  }
  // layout of the device allocation (tensor maps first: 64-byte alignment)
  size_t off = 0;
  const size_t o_maps = off;
  off = align_up(off + sizeof(CUtensorMap) * maps.size(), 64);
  const size_t o_jobs = off;
  off = align_up(off + sizeof(int2) * jobs.size(), 64);
  const size_t o_po = off;
  off = align_up(off + sizeof(int) * porder.size(), 64);
  const size_t o_tf = off;
  off += sizeof(int4) * ctf.size();
  const size_t o_ta = off;
  off += sizeof(int4) * cta.size();
  const size_t o_cr = off;
  off += sizeof(long long) * cum_r.size();
  const size_t o_cu = off;
  off = align_up(off + sizeof(long long) * cum_u.size(), 64);
  const size_t o_beta = off;
  off = align_up(off + sizeof(float) * beta.size(), 64);
  const size_t o_arr = off;  // step times, arrivals, then 2 iters task counters
  const size_t counters = 8 * sizeof(unsigned long long) + sizeof(unsigned int) * (1 + 4 * (size_t)std::max(iters, 1));
  off += align_up(counters, 64);
  std::vector<unsigned char> host(off, 0);
  cudaError_t e = cudaMalloc(&pp->blob, off);
  if (e != cudaSuccess) {
    pp->blob = nullptr;
    persist_free(pp);
    return cuda_fail(e, "persistent plan", __FILE__, __LINE__);
  }
  unsigned char* base = (unsigned char*)pp->blob;
  PPlan& hp = pp->prm.p;
  hp.ngroups = ngroups;
  hp.njobs = (int)jobs.size();
  hp.iters = iters;
  hp.maps = (const CUtensorMap*)(base + o_maps);
  hp.job = (const int2*)(base + o_jobs);
  hp.porder = (const int*)(base + o_po);
  hp.ctask_f = (const int4*)(base + o_tf);
  hp.ctask_a = (const int4*)(base + o_ta);
  hp.nct_f = (int)ctf.size();
  hp.nct_a = (int)cta.size();
  hp.cum_r = (const long long*)(base + o_cr);
  hp.cum_u = (const long long*)(base + o_cu);
  hp.beta = (const float*)(base + o_beta);
  hp.step_ns = (unsigned long long*)(base + o_arr);
  hp.arrivals = (unsigned int*)(hp.step_ns + 8);
  hp.tasks = hp.arrivals + 1;
  hp.err = ops[0]->ws.err;
  hp.wait_ns = ops[0]->wait_ns;
  memcpy(host.data() + o_maps, maps.data(), sizeof(CUtensorMap) * maps.size());
  memcpy(host.data() + o_jobs, jobs.data(), sizeof(int2) * jobs.size());
  memcpy(host.data() + o_po, porder.data(), sizeof(int) * porder.size());
  memcpy(host.data() + o_tf, ctf.data(), sizeof(int4) * ctf.size());
  memcpy(host.data() + o_ta, cta.data(), sizeof(int4) * cta.size());
  memcpy(host.data() + o_cr, cum_r.data(), sizeof(long long) * cum_r.size());
  memcpy(host.data() + o_cu, cum_u.data(), sizeof(long long) * cum_u.size());
  memcpy(host.data() + o_beta, beta.data(), sizeof(float) * beta.size());
  e = cudaMemcpy(pp->blob, host.data(), off, cudaMemcpyHostToDevice);
  if (e != cudaSuccess) {
    persist_free(pp);
    return cuda_fail(e, "persistent plan copy", __FILE__, __LINE__);
  }
  pp->smem = smem;
  pp->nb_policy = nb_policy;
  pp->counters_bytes = counters;
  const void* kern = (const void*)fista_persistent_kernel;
  rc = ensure_smem_attr_ptr(kern, smem);
  if (rc == SFS_OK) {
    e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, kern, kPThreads, smem);
    if (e != cudaSuccess) rc = cuda_fail(e, "persistent kernel occupancy", __FILE__, __LINE__);
  }
  if (rc == SFS_OK && occ < 1) {
    set_error("the persistent kernel does not fit an SM (%d bytes of shared memory)", smem);
    rc = SFS_ERR_INVALID_ARG;
  }
  if (rc != SFS_OK) {
    persist_free(pp);
    return rc;
  }
  pp->grid = sms;
  *out = pp;
  return SFS_OK;
}

int persist_launch(const PersistPlan* pp, cudaStream_t st) {
  SFS_CUDA(cudaMemsetAsync(pp->prm.p.step_ns, 0, pp->counters_bytes, st));
  cudaLaunchAttribute attr[1];
  attr[0].id = cudaLaunchAttributeCooperative;
  attr[0].val.cooperative = 1;
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = dim3(pp->grid);
  cfg.blockDim = dim3(kPThreads);
  cfg.dynamicSmemBytes = (size_t)pp->smem;
  cfg.stream = st;
  cfg.attrs = attr;
  cfg.numAttrs = 1;
  SFS_CUDA(cudaLaunchKernelEx(&cfg, fista_persistent_kernel, pp->prm));
  return SFS_OK;
}

void persist_free(PersistPlan* pp) {
  if (!pp) return;
  if (pp->blob) cudaFree(pp->blob);
  delete pp;
}

int persist_step_ms(const PersistPlan* pp, double* ms8) {
  unsigned long long ns[8];
  SFS_CUDA(cudaMemcpy(ns, pp->prm.p.step_ns, sizeof(ns), cudaMemcpyDeviceToHost));
  for (int i = 0; i < 4; ++i) ms8[i] = (double)ns[i] * 1e-6;
  for (int i = 4; i < 8; ++i) ms8[i] = (double)ns[i] * 1e-6 / std::max(1, pp->grid);
  return SFS_OK;
}

}  // namespace sfs
