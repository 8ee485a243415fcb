// smc_small.cu -- a whole small run in one launch: every segment of a run whose
// tiles are warps (32 particles each), few enough for one CTA or one thread-block
// cluster, runs in one launch, with a CTA or cluster barrier as the checkpoint
// barrier of Algorithm 1 (Section 3.3's loop: propagate, combine, resample,
// repeat) instead of a kernel boundary per segment.
//
// Warp w of CTA r (its rank in the cluster; 0 without one) is tile
// r * (TPB / 32) + w of the run.  Each segment is the wave kernel's work with a
// barrier between the steps that need one:
//   combine   (k > 0) the previous segment's tile records (in global memory,
//             written by every CTA of the cluster) combined by each CTA for
//             itself into exact integer offsets (smc_combine.cuh), the log-Z
//             increment, the resampling decision and the search scalars: the
//             same integers in every CTA, so the same decisions;
//   search    each particle's systematic-resampling ancestor and the fused
//             gather of its state (step_tile's code, with the offsets and tile
//             references in shared memory);
//   segment   blocks to the next checkpoint with per-warp PC-sorted dispatch;
//   epilogue  per warp: its power-of-two reference, integer weights, running
//             sums and tile record (a warp is a tile, so the tile reference is
//             the warp's).
// The segment ends at the cluster barrier (release / acquire at cluster scope:
// the records, running sums and states written before it by any CTA of the
// cluster are visible to every CTA after it); the double-buffered records,
// sums and states of segment k are not written again before the barrier that
// ends segment k + 1, which every CTA reaches only after its reads of them.
// The tiles, their rounding and the combine's integers are those of the wave
// kernel for the same N, so a run gives the same bits here, alone through the
// waves, batched and served.  The barriers are the hardware's (every CTA of a
// cluster is resident at once); nothing spins.
#include <cuda_runtime.h>

#include <mutex>

#include "smc_engine.h"
#include "smc_internal.h"
#include "smc_step.cuh"

namespace smc {

constexpr int kSmallMaxTiles = 32;

__device__ __forceinline__ unsigned cluster_rank() {
  unsigned r;
  asm volatile("mov.u32 %0, %%cluster_ctarank;" : "=r"(r));
  return r;
}

// Every thread of every CTA of the cluster: the writes before it (global and
// shared) are visible to every thread of the cluster after it.
__device__ __forceinline__ void cluster_barrier() {
  asm volatile(
      "barrier.cluster.arrive.release;\n\t"
      "barrier.cluster.wait.acquire;" ::: "memory");
}

// CL: launched as one cluster of ceil(n_tiles / (TPB / 32)) CTAs (else one CTA).
template <class M, int TPB, bool CL>
__global__ void __launch_bounds__(TPB, 1) small_run_kernel(const RunDev* __restrict__ runs) {
  using R = typename M::R;
  constexpr int WPC = TPB / 32;
  static_assert(CL || WPC >= 16, "one CTA holds the whole run");
  __shared__ __align__(16) RunDev sr;
  __shared__ double sh[TPB / 32 + 2 + TPB + 1];
  __shared__ long long sh_O[kSmallMaxTiles + 1];
  __shared__ int sh_ks[kSmallMaxTiles + 1];
  __shared__ unsigned long long shq[5];
  {
    const int* src = reinterpret_cast<const int*>(runs);
    int* dst = reinterpret_cast<int*>(&sr);
    for (int w = threadIdx.x; w < (int)(sizeof(RunDev) / 4); w += TPB) dst[w] = src[w];
  }
  __syncthreads();
  const RunDev& A = sr;
  RunState* rs = A.rs;
  const int N = A.N;
  const bool lead = !CL || cluster_rank() == 0;  // the CTA that closes each segment
  const int t = (CL ? (int)cluster_rank() * WPC : 0) + (int)(threadIdx.x >> 5);
  const int lane = threadIdx.x & 31;
  const int i = t * 32 + lane;  // the tile of this path is 32 particles
  const bool tile_live = t < A.n_tiles;
  const bool valid = tile_live && i < N;
  for (int k = 0;; ++k) {
    const int nb = k & 1, cb = nb ^ 1;
    const StateView Sc = A.state[cb];
    const StateView Sn = A.state[nb];
    typename M::Lane L;
    bool near = false;
    if (k > 0) {
      const Combined c = combine_offsets<TPB>(A.rec[cb], A.n_tiles, sh_O, sh_ks, sh,
                                              A.ess ? A.tq[cb] : nullptr);
      const bool go_on = c.kmax != kDeadTile && c.alive && k < A.max_segments;
      const bool resample = decide_resample(A, c);
      if (lead && threadIdx.x == 0) finish_segment(A, k, c, resample);
      if (!go_on) break;  // the same c in every thread: a uniform exit
      if (resample && threadIdx.x == 0) {
        Q64 d, z0;
        long long tolZ;
        search_scalars(c, N, Unif<double>::first(philox(0u, (uint32_t)(k - 1), 0u, 1u, A.k0, A.k1)),
                       &d, &z0, &tolZ);
        shq[0] = d.hi;
        shq[1] = d.lo;
        shq[2] = z0.hi;
        shq[3] = z0.lo;
        shq[4] = (unsigned long long)tolZ;
      }
      __syncthreads();
      SearchCtx X;
      X.rec = A.rec[cb];
      X.O = sh_O;
      X.ks = sh_ks;
      X.kmax = c.kmax;
      X.G = c.G;
      X.d = Q64{shq[0], shq[1]};
      X.z0 = Q64{shq[2], shq[3]};
      X.tolZ = (long long)shq[4];
      if (valid) {
        const int row = A.record_all ? k - 1 : 0;
        int a = resample ? systematic_search<true>(i, A, X, A.E[cb], &near) : i;
        bool bad = false;
        if (SMC_DEBUG_CHECKS) {
          if (!(a >= 0 && a < N)) {
            debug_record(rs, 1, i);
            a = i;
            bad = true;
          }
          if (M::HAS_STACK) {
            const int spa = Sc.inf_(1, a, N);
            if (!(spa >= 0 && spa <= A.md.lam_stack_cap)) {
              debug_record(rs, 3, i);
              bad = true;
            }
          }
        }
        if (row < A.anc_rows) A.anc[(size_t)row * N + i] = a;
        if (bad) {
          M::init(L);
          L.pc = PC_STOP;
          L.logw = neg_inf<R>();
        } else if (resample) {
          M::gather(L, Sc, Sn, a, i, N, A.md);
        } else {
          M::gather(L, Sc, Sn, i, i, N, A.md);
          L.logw = (R)A.logw[i];
        }
      }
      warp_add_u64(&rs->n_near, near ? 1ull : 0ull);
    } else if (valid) {
      M::init(L);
    }
    if (SMC_DEBUG_CHECKS && valid && !(L.pc == PC_STOP || (L.pc >= 0 && L.pc < M::NB))) {
      debug_record(rs, 2, i);
      L.pc = PC_STOP;
      L.logw = neg_inf<R>();
    }
    Stream s{A.k0, A.k1, (uint32_t)i, (uint32_t)k, 0u, 0u, A.md.tab};
    const bool active = valid && L.pc != PC_STOP;
    const int n_exec = run_segment<M>(L, s, A.md, Sn, i, k, N, active);
    double lw = -INFINITY;
    int alive = 0;
    if (valid) {
      M::store(L, Sn, i, N);
      lw = (double)L.logw;
      A.logw[i] = lw;
      alive = L.pc != PC_STOP;
    }
    warp_add_u64(&rs->n_overflow, active ? (unsigned long long)L.overflow : 0ull);
    warp_add_u64(&rs->n_limit, active ? (unsigned long long)L.limited : 0ull);
    warp_add_u64(&rs->n_draws, valid ? (unsigned long long)s.d : 0ull);
    warp_add_u64(&rs->n_blocks, (unsigned long long)n_exec);
    // the tile's weights: a warp is a tile, so its reference is the warp's
    long long ef = 0;
    const double Mw = warp_max_key(lw);
    const int kt = Mw == -INFINITY ? kDeadTile : tile_exponent(Mw);
    if (valid && kt != kDeadTile) {
      if (kt > -2048 && kt < 2048) {
        ef = weight_fix<54>(lw, ref_q58(kt), A.md.tab);
      } else {
        const double kd = (double)kt;
        const double dd = fma(-kd, kLn2Lo, fma(-kd, kLn2Hi, lw));
        ef = exp_fix54(dd, A.md.tab);
      }
    }
    const long long E = block_incl_scan_i64<32>(ef, nullptr);  // a warp scan
    if (valid) A.E[nb][i] = E;
    if (A.ess) {
      const unsigned long long u = (unsigned long long)ef;
      const long long sq = (long long)((__umul64hi(u, u) << 10) | ((u * u) >> 54));
      const long long Q = block_incl_scan_i64<32>(sq, nullptr);
      if (tile_live && lane == 31) A.tq[nb][t] = Q;
    }
    const int tile_alive = __any_sync(0xffffffffu, alive) ? 1 : 0;
    if (tile_live && lane == 31) {
      TileRec r;
      r.s = E;
      r.k = kt;
      r.alive = tile_alive;
      A.rec[nb][t] = r;
    }
    // the segment's records, running sums and states, for the next combine
    if (CL)
      cluster_barrier();
    else
      __syncthreads();
  }
}

// One CTA: register-light models run up to 32 tiles (1024 threads, 64
// registers a thread); the tree and SEIR models up to 16 (512 threads).
// Cluster: up to 32 tiles for every model, 2 warps a CTA in clusters of up to
// 16 CTAs where the GPU schedules them, else 4 warps a CTA in up to 8.
int small_run_max_tiles(int kind, int launch_mode) {
  if (launch_mode == SMC_LAUNCH_CLUSTER) return kSmallMaxTiles;
  switch (kind) {
    case SMC_MODEL_LG:
    case SMC_MODEL_GEOMETRIC: return 32;
    default: return 16;
  }
}

namespace {
template <class M, int TPB>
cudaError_t launch_cluster(const RunDev* runs, int n_tiles, cudaStream_t st) {
  auto kern = small_run_kernel<M, TPB, true>;
  static std::once_flag once;
  static cudaError_t attr = cudaSuccess;
  std::call_once(once, [&] {
    if (TPB / 32 * 8 < kSmallMaxTiles)
      attr = cudaFuncSetAttribute(kern, cudaFuncAttributeNonPortableClusterSizeAllowed, 1);
  });
  if (attr != cudaSuccess) return attr;
  const unsigned ctas = (unsigned)((n_tiles + TPB / 32 - 1) / (TPB / 32));
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = dim3(ctas, 1, 1);
  cfg.blockDim = dim3(TPB, 1, 1);
  cfg.dynamicSmemBytes = 0;
  cfg.stream = st;
  cudaLaunchAttribute at[1];
  at[0].id = cudaLaunchAttributeClusterDimension;
  at[0].val.clusterDim.x = ctas;
  at[0].val.clusterDim.y = 1;
  at[0].val.clusterDim.z = 1;
  cfg.attrs = at;
  cfg.numAttrs = 1;
  return cudaLaunchKernelEx(&cfg, kern, runs);
}

// Whether the GPU schedules clusters of 16 CTAs of 64 threads (asked once per
// process, for the device current at the first call).
bool wide_clusters() {
  static std::once_flag once;
  static bool wide = false;
  std::call_once(once, [] {
    auto kern = small_run_kernel<LgModel<double>, 64, true>;
    if (cudaFuncSetAttribute(kern, cudaFuncAttributeNonPortableClusterSizeAllowed, 1) != cudaSuccess) {
      cudaGetLastError();
      return;
    }
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3(16, 1, 1);
    cfg.blockDim = dim3(64, 1, 1);
    cudaLaunchAttribute at[1];
    at[0].id = cudaLaunchAttributeClusterDimension;
    at[0].val.clusterDim.x = 16;
    at[0].val.clusterDim.y = 1;
    at[0].val.clusterDim.z = 1;
    cfg.attrs = at;
    cfg.numAttrs = 1;
    int n = 0;
    if (cudaOccupancyMaxActiveClusters(&n, kern, &cfg) != cudaSuccess) {
      cudaGetLastError();
      return;
    }
    wide = n > 0;
  });
  return wide;
}

template <class M>
cudaError_t launch_small_m(int launch_mode, int one_cta_tpb, const RunDev* runs, int n_tiles,
                           cudaStream_t st) {
  if (launch_mode == SMC_LAUNCH_CLUSTER)
    return wide_clusters() ? launch_cluster<M, 64>(runs, n_tiles, st)
                           : launch_cluster<M, 128>(runs, n_tiles, st);
  if (one_cta_tpb == 1024)
    small_run_kernel<M, 1024, false><<<1, 1024, 0, st>>>(runs);
  else
    small_run_kernel<M, 512, false><<<1, 512, 0, st>>>(runs);
  return cudaGetLastError();
}

template <typename R>
cudaError_t launch_small_r(int kind, int launch_mode, const RunDev* runs, int n_tiles,
                           cudaStream_t st) {
  switch (kind) {
    case SMC_MODEL_LG: return launch_small_m<LgModel<R>>(launch_mode, 1024, runs, n_tiles, st);
    case SMC_MODEL_GEOMETRIC: return launch_small_m<GeoModel<R>>(launch_mode, 1024, runs, n_tiles, st);
    case SMC_MODEL_SEIR: return launch_small_m<SeirModel<R>>(launch_mode, 512, runs, n_tiles, st);
    case SMC_MODEL_CRBD:
      return launch_small_m<TreeModel<R, false>>(launch_mode, 512, runs, n_tiles, st);
    case SMC_MODEL_RATESHIFT:
      return launch_small_m<TreeModel<R, true>>(launch_mode, 512, runs, n_tiles, st);
    default: return launch_small_m<TreeDsModel<R>>(launch_mode, 512, runs, n_tiles, st);
  }
}
}  // namespace

cudaError_t launch_small_run(int kind, int precision, int launch_mode, const RunDev* runs,
                             int n_tiles, cudaStream_t st) {
  return precision == SMC_PREC_FP32 ? launch_small_r<float>(kind, launch_mode, runs, n_tiles, st)
                                    : launch_small_r<double>(kind, launch_mode, runs, n_tiles, st);
}

}  // namespace smc
