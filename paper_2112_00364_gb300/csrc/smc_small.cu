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

// The cluster barrier in its two halves: the writes of every thread of the
// cluster before its arrive are visible to every thread after its wait; work
// between the two overlaps the other CTAs' arrival.
__device__ __forceinline__ void cluster_arrive() {
  asm volatile("barrier.cluster.arrive.release;" ::: "memory");
}
__device__ __forceinline__ void cluster_wait() {
  asm volatile("barrier.cluster.wait.acquire;" ::: "memory");
}

// systematic_search for one warp of a small run (tiles of 32 particles): each
// lane's tile from the offsets as there; then, per distinct tile among the
// lanes (one or two, the offsets being non-decreasing), the tile's 32 running
// sums in one load (lane l holds E_{j0+l}) and every lane of that tile finds
// its first j with E_j > F by a binary search over the shuffled values.  The
// same ancestors and near-boundary flags as systematic_search; one dependent
// load of the sums instead of the 8-ary search's two.  Every lane calls it;
// `want` marks the lanes whose offset is searched.
__device__ __forceinline__ int small_search(int i, bool want, const RunDev& A, const SearchCtx& X,
                                            const long long* E, bool* near) {
  constexpr unsigned kAll = 0xffffffffu;
  const int N = A.N, T = A.n_tiles, lane = threadIdx.x & 31;
  int a = i, t = -1;
  bool nr = false, need = false;
  long long F = 0, tolF = 0, Z = 0;
  if (want) {
    const Q64 z = q_add(X.z0, q_mul_u32((unsigned)i, X.d));
    Z = (long long)z.hi;
    int lo = 0, hi = T;  // O_0 = 0 <= z
    while (lo < hi) {
      const int mid = (lo + hi + 1) >> 1;
      if (X.O[mid] <= Z)
        lo = mid;
      else
        hi = mid - 1;
    }
    if (lo >= T) {  // above the last offset (rounding at the top)
      nr = Z - X.O[T] < X.tolZ;
      a = N - 1;
    } else {
      t = lo;
      const int sh = X.kmax - X.ks[t] + X.G;
      F = q_threshold(z, X.O[t], sh);
      tolF = shl_sat(X.tolZ, sh);
      need = true;
    }
  }
  unsigned pending = __ballot_sync(kAll, need);
  while (pending) {
    const int tg = __shfl_sync(kAll, t, __ffs(pending) - 1);
    const int j0 = tg * 32, len = min(32, N - j0);
    const long long e = lane < len ? __ldcg(E + j0 + lane) : 0x7FFFFFFFFFFFFFFFll;
    // pos = #{ l < len : E_{j0+l} <= F } (the sums are non-decreasing)
    int pos = 0;
#pragma unroll
    for (int step = 16; step >= 1; step >>= 1) {
      const long long v = __shfl_sync(kAll, e, pos + step - 1);
      if (v <= F) pos += step;
    }
    const long long e31 = __shfl_sync(kAll, e, 31);
    if (pos == 31 && e31 <= F) pos = 32;
    pos = min(pos, len);
    const long long El = __shfl_sync(kAll, e, min(pos, 31));
    const long long Eb = __shfl_sync(kAll, e, max(pos - 1, 0));
    const bool mine = need && t == tg;
    if (mine) {
      nr = F - (pos > 0 ? Eb : 0ll) < tolF;
      if (pos < len) {
        a = j0 + pos;
        nr = nr || El - F <= tolF;
      } else if (j0 + len < N) {  // the first element of the next tile
        a = j0 + len;
        nr = nr || X.O[tg + 1] - Z <= X.tolZ;
      } else {
        a = N - 1;
      }
    }
    pending &= ~__ballot_sync(kAll, mine);
  }
  *near = nr;
  return a;
}

// The warp's sum of a 64-bit per-lane count, added by lane 0.
__device__ __forceinline__ void warp_add_u64_wide(unsigned long long* dst, unsigned long long v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  if ((threadIdx.x & 31) == 0 && v) atomicAdd(dst, v);
}

// The combine of at most 32 tiles by one warp, lane t holding tile t: the
// integers of combine_offsets (the same k_max, coarsening G, unit totals,
// exact offsets and S, and the effective sample size summed in the same
// order) from warp shuffles, with no CTA barrier.  Writes O[0..nt] (O[nt] = S)
// and ks[0..nt) to the warp's own shared arrays.
__device__ __forceinline__ Combined combine_warp(const TileRec* rec, int nt, const long long* q,
                                                 long long* O, int* ks) {
  constexpr unsigned kAll = 0xffffffffu;
  const int lane = threadIdx.x & 31;
  TileRec r;
  r.s = 0;
  r.k = kDeadTile;
  r.alive = 0;
  if (lane < nt) r = load_rec(rec + lane);
  Combined c;
  c.kmax = __reduce_max_sync(kAll, r.k);
  c.alive = __any_sync(kAll, r.alive) ? 1 : 0;
  c.G = 0;
  c.S = 0;
  c.ess = 0.0;
  if (lane < nt) ks[lane] = r.k;
  if (c.kmax == kDeadTile) {
    __syncwarp();
    return c;
  }
  long long b = lane < nt ? magnitude(r.s, r.k, c.kmax) : 0;
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) b += __shfl_xor_sync(kAll, b, o);
  c.G = (64 - __clzll(b)) + 20 - 62;
  const long long v = lane < nt ? to_run_units(r.s, r.k, c.kmax, c.G) : 0;
  long long inc = v;
#pragma unroll
  for (int o = 1; o < 32; o <<= 1) {
    const long long y = __shfl_up_sync(kAll, inc, o);
    if (lane >= o) inc += y;
  }
  c.S = __shfl_sync(kAll, inc, 31);
  if (lane < nt) O[lane] = inc - v;
  if (lane == 0) O[nt] = c.S;
  if (q) {
    double acc = 0.0;
    if (lane < nt && r.k != kDeadTile) {
      const int d2 = 2 * (c.kmax - r.k);
      if (d2 < 900) acc = acc + (double)__ldcg(q + lane) * pow2i(-54 - d2);
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) acc = acc + __shfl_xor_sync(kAll, acc, o);
    const double sd = (double)c.S * pow2i(c.G - 54);
    c.ess = acc > 0.0 ? (sd * sd) / acc : 0.0;
  }
  __syncwarp();
  return c;
}

// CL: launched as one cluster of ceil(n_tiles / (TPB / 32)) CTAs (else one CTA).
template <class M, int TPB, bool CL>
__global__ void __launch_bounds__(TPB, 1) small_run_kernel(const RunDev* __restrict__ runs) {
  using R = typename M::R;
  constexpr int WPC = TPB / 32;
  static_assert(CL || WPC >= 16, "one CTA holds the whole run");
  __shared__ __align__(16) RunDev sr;
  __shared__ long long sh_O[WPC][kSmallMaxTiles + 1];  // each warp's own offsets
  __shared__ int sh_ks[WPC][kSmallMaxTiles + 1];
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
  const int wid = (int)(threadIdx.x >> 5);
  const int t = (CL ? (int)cluster_rank() * WPC : 0) + wid;
  const int lane = threadIdx.x & 31;
  const int i = t * 32 + lane;  // the tile of this path is 32 particles
  const bool tile_live = t < A.n_tiles;
  const bool valid = tile_live && i < N;
  // segment k - 1's closing (log Z, its records) waits for the barrier that
  // ends segment k, where it overlaps the other CTAs' arrival
  Combined c_close;
  bool resample_close = false;
  double u = 0.0;  // the uniform of the next search, drawn in the barrier's shadow
  // the run's counters, summed per lane over the segments and added once
  unsigned long long n_near = 0, n_overflow = 0, n_limit = 0, n_draws = 0, n_blocks = 0;
  for (int k = 0;; ++k) {
    const int nb = k & 1, cb = nb ^ 1;
    const StateView Sc = A.state[cb];
    const StateView Sn = A.state[nb];
    typename M::Lane L;
    bool near = false;
    if (k > 0) {
      const Combined c = combine_warp(A.rec[cb], A.n_tiles, A.ess ? A.tq[cb] : nullptr,
                                      sh_O[wid], sh_ks[wid]);
      const bool go_on = c.kmax != kDeadTile && c.alive && k < A.max_segments;
      const bool resample = decide_resample(A, c);
      if (!go_on) {  // the same c in every thread: a uniform exit
        if (lead && threadIdx.x == 0) finish_segment(A, k, c, resample);
        break;
      }
      c_close = c;
      resample_close = resample;
      // the run's search scalars by each warp's lane 0, broadcast to its lanes
      unsigned long long q5[5] = {0ull, 0ull, 0ull, 0ull, 0ull};
      if (resample && lane == 0) {
        Q64 d, z0;
        long long tolZ;
        search_scalars(c, N, A.recip_n, u, &d, &z0, &tolZ);
        q5[0] = d.hi;
        q5[1] = d.lo;
        q5[2] = z0.hi;
        q5[3] = z0.lo;
        q5[4] = (unsigned long long)tolZ;
      }
#pragma unroll
      for (int q = 0; q < 5; ++q) q5[q] = __shfl_sync(0xffffffffu, q5[q], 0);
      SearchCtx X;
      X.rec = A.rec[cb];
      X.O = sh_O[wid];
      X.ks = sh_ks[wid];
      X.kmax = c.kmax;
      X.G = c.G;
      X.d = Q64{q5[0], q5[1]};
      X.z0 = Q64{q5[2], q5[3]};
      X.tolZ = (long long)q5[4];
      const int a_s = resample ? small_search(i, valid, A, X, A.E[cb], &near) : i;
      if (valid) {
        const int row = A.record_all ? k - 1 : 0;
        int a = a_s;
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
      n_near += near ? 1ull : 0ull;
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
    n_overflow += active ? (unsigned long long)L.overflow : 0ull;
    n_limit += active ? (unsigned long long)L.limited : 0ull;
    n_draws += valid ? (unsigned long long)s.d : 0ull;
    n_blocks += (unsigned long long)n_exec;
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
    if (CL) cluster_arrive();
    if (k > 0 && lead && threadIdx.x == 0) finish_segment(A, k, c_close, resample_close);
    if (lane == 0) u = Unif<double>::first(philox(0u, (uint32_t)k, 0u, 1u, A.k0, A.k1));
    if (CL)
      cluster_wait();
    else
      __syncthreads();
  }
  warp_add_u64_wide(&rs->n_near, n_near);
  warp_add_u64_wide(&rs->n_overflow, n_overflow);
  warp_add_u64_wide(&rs->n_limit, n_limit);
  warp_add_u64_wide(&rs->n_draws, n_draws);
  warp_add_u64_wide(&rs->n_blocks, n_blocks);
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
