// smc_step.cuh -- one tile of one run for one segment: the body of every
// segment kernel (the wave kernel of smc_engine.cu and the single-CTA kernel of
// smc_small.cu).  Algorithm 1 in the RootPPL loop order of Section 3.3: the
// previous segment's tiles combined into exact integer offsets, the log-Z
// increment and the resampling decision; the systematic search and the
// particle duplication fused into the load; blocks run to the next checkpoint;
// the tile's weights, running sums and record.
#pragma once
#include <cuda_runtime.h>

#include "smc_combine.cuh"
#include "smc_device.cuh"
#include "smc_engine.h"
#include "smc_models.cuh"

#ifndef SMC_DEBUG_CHECKS
#define SMC_DEBUG_CHECKS 0
#endif

namespace smc {

// Checking build: record an out-of-range access (the caller skips it).
__device__ __forceinline__ void debug_record(RunState* rs, int code, long long index) {
  atomicAdd(&rs->dbg_count, 1ull);
  if (atomicCAS(&rs->dbg_code, 0, code) == 0) rs->dbg_index = index;
}

__device__ __forceinline__ void warp_add_u64(unsigned long long* dst, unsigned long long v) {
  v = __reduce_add_sync(0xffffffffu, (unsigned)v);
  if ((threadIdx.x & 31) == 0 && v) atomicAdd(dst, v);
}

// Finish segment k-1 of the run from its combined offsets (one thread):
// log Z += k_max ln 2 + (log S - log N) with S = S_units U, the increment
// record, and the end of the run.  Returns whether segment k runs.
// Whether to resample after checkpoint k-1 (the same in every CTA: c is).
__device__ __forceinline__ bool decide_resample(const RunDev& A, const Combined& c) {
  return !A.ess || c.ess < A.ess_target;
}

__device__ __forceinline__ bool finish_segment(const RunDev& A, int k, const Combined& c,
                                               bool resample) {
  RunState* rs = A.rs;
  if (c.kmax == kDeadTile) {
    rs->log_z = -INFINITY;
    rs->log_z_closed = -INFINITY;
    rs->m = -INFINITY;
    rs->S = 0.0;
    A.incr[k - 1] = -INFINITY;
    rs->status = SMC_EDEGENERATE;
    rs->done = 1;
    rs->n_segments = k;
    return false;
  }
  const double Sd = (double)c.S;
  const double inc = (double)(c.kmax - 54 + c.G) * kLn2 + (tang_log(Sd, A.md.tab) - A.log_n);
  const bool go_on = c.alive && k < A.max_segments;
  // the accumulated weights are closed into log Z when the population is
  // resampled, at the end and at the step limit
  const bool close = !go_on || resample;
  if (close) rs->log_z = rs->log_z + inc;
  if (!(c.alive && k >= A.max_segments)) rs->log_z_closed = rs->log_z;  // not a step-limit closure
  A.incr[k - 1] = close ? inc : 0.0;
  rs->m = (double)c.kmax * kLn2;
  rs->S = Sd * pow2i(c.G - 54);
  rs->n_segments = k;
  if (go_on) {
    A.dec[k - 1] = resample ? 1 : 0;
    rs->n_resamples += resample ? 1 : 0;
    if (A.ess && fabs(c.ess - A.ess_target) <= 1e-9 * A.ess_target) rs->n_ess_near += 1;
  }
  if (!c.alive) {
    rs->done = 1;
  } else if (!go_on) {
    rs->status = SMC_ESTEPLIMIT;
    rs->done = 1;
  }
  return go_on;
}

// What the search of segment k needs about segment k-1's weights.
struct SearchCtx {
  const long long* O;  // offsets in units U, O[T] = S
  const int* ks;       // tile reference exponents (shared memory), or NULL: read the records
  const TileRec* rec;
  int kmax, G;
  Q64 d, z0;           // S / N and u S / N in 64.64 (units U)
  long long tolZ;      // 1e-12 N on the q scale, in units U
};

// The run's search scalars from its combined total (one thread).
__device__ __forceinline__ void search_scalars(const Combined& c, int N, unsigned long long recip_n,
                                               double u, Q64* d, Q64* z0, long long* tolZ) {
  *d = q_ratio((unsigned long long)c.S, (unsigned long long)N, recip_n);
  *z0 = q_scale(frac64(u), *d);
  *tolZ = floor_i64(kBoundaryEps * (double)c.S);
}

// a_i = min{ j : q_j > y } for y = i + u, with q_j = P_j N / S and P_j the
// running sum of the weights; on the P scale in units U the offset is
// z_i = z_0 + i S / N (64.64 fixed point, exact and non-decreasing in i).  The
// tile is t = max{ t : O_t <= z } (N - 1 if z lies above every offset); inside
// it P_j = O_t + E_j 2^-(k_max - k_t + G), so P_j > z <=> E_j > floor((z - O_t)
// 2^(k_max - k_t + G)) (E_j is an integer): one threshold per particle, then an
// 8-ary search with integer compares (three rounds of independent loads for a
// 256-particle tile).  If no element of tile t qualifies, the first element of
// tile t+1 does.  The offset is flagged when it lies within 1e-12 N of q_a or
// q_{a-1}, measured in the same units.  Integer arithmetic only.  kL2: the
// running sums were written by other CTAs of the same launch (a cluster's run),
// so they are read at L2, past this SM's L1.
template <bool kL2>
__device__ __forceinline__ long long load_sum(const long long* p) {
  if (kL2) return __ldcg(p);
  return *p;
}

template <bool kL2 = false>
__device__ __forceinline__ int systematic_search(int i, const RunDev& A, const SearchCtx& X,
                                                 const long long* __restrict__ E, bool* near) {
  const int N = A.N, T = A.n_tiles;
  const Q64 z = q_add(X.z0, q_mul_u32((unsigned)i, X.d));
  const long long Z = (long long)z.hi;
  int lo = 0, hi = T;  // O_0 = 0 <= z
  while (lo < hi) {
    const int mid = (lo + hi + 1) >> 1;
    if (X.O[mid] <= Z)
      lo = mid;
    else
      hi = mid - 1;
  }
  if (lo >= T) {  // above the last offset (rounding at the top)
    *near = Z - X.O[T] < X.tolZ;
    return N - 1;
  }
  const int t = lo;
  const int j0 = t * A.tile, j1 = min(N, j0 + A.tile);
  const int kt = X.ks ? X.ks[t] : load_rec(X.rec + t).k;
  const int sh = X.kmax - kt + X.G;
  const long long F = q_threshold(z, X.O[t], sh);
  const long long tolF = shl_sat(X.tolZ, sh);
  // first j in [j0, j1) with E_j > F
  long long Eb = 0;  // E_{b-1} for the current bracket start b (0 before the tile)
  int b = j0, len = j1 - j0;
  while (len > 8) {
    const int w = (len + 7) >> 3;
    long long v[8];
#pragma unroll
    for (int m = 0; m < 8; ++m) v[m] = load_sum<kL2>(E + b + min((m + 1) * w, len) - 1);
    int m = 8;
#pragma unroll
    for (int q = 7; q >= 0; --q)
      if (v[q] > F) m = q;
    if (m == 8) {  // nothing in the tile qualifies
      Eb = v[7];
      b += len;
      len = 0;
      break;
    }
    if (m > 0) Eb = v[m - 1];
    len = min((m + 1) * w, len) - m * w;
    b += m * w;
  }
  int l = b + len;  // none found yet
  long long El = 0;
  if (len > 0) {
    long long v[8];
#pragma unroll
    for (int m = 0; m < 8; ++m) v[m] = m < len ? load_sum<kL2>(E + b + m) : 0x7FFFFFFFFFFFFFFFll;
    int m = 8;
#pragma unroll
    for (int q = 7; q >= 0; --q)
      if (v[q] > F) m = q;
#pragma unroll
    for (int q = 0; q < 8; ++q) {
      if (q == m) El = v[q];
      if (q < m && q < len) Eb = v[q];
    }
    if (m < len) l = b + m;
  }
  bool nr = F - Eb < tolF;
  int a;
  if (l < j1) {
    a = l;
    nr = nr || El - F <= tolF;
  } else if (j1 < N) {  // the first element of the next tile
    a = j1;
    nr = nr || X.O[t + 1] - Z <= X.tolZ;
  } else {
    a = N - 1;
  }
  *near = nr;
  return a;
}

// One L2 line into this SM's L1 ahead of its use (a hint: nothing waits on it).
__device__ __forceinline__ void prefetch_l1(const void* p) {
  asm volatile("{\n\t.reg .u64 g;\n\tcvta.to.global.u64 g, %0;\n\tprefetch.global.L1 [g];\n\t}"
               :: "l"(p));
}

// The lines of particles [lo, hi) of one array of elements of esz bytes.
template <int TPB>
__device__ __forceinline__ void prefetch_range(const void* base, int lo, int hi, int esz) {
  const char* b = static_cast<const char*>(base) + (size_t)lo * esz;
  const int lines = ((hi - lo) * esz + 127) >> 7;
  for (int j = threadIdx.x; j < lines; j += TPB) prefetch_l1(b + (size_t)j * 128);
}

// Before the offsets are read, pull into L1 what this tile's search and gather
// will most likely need: systematic ancestors of a tile's
// particles lie mostly in the tiles t - 1 .. t + 1, so the previous segment's
// running sums and PSTATE rows of those particles (written by the previous
// wave).  Their loads then overlap the combine instead of following it.
template <class M, int TPB>
__device__ __forceinline__ void prefetch_neighbours(const RunDev& A, int t, int cb) {
  using R = typename M::R;
  const int lo = max(0, (t - 1) * A.tile);
  const int hi = (int)min((long long)A.N, (long long)(t + 2) * A.tile);  // N may be near 2^31
  if (lo >= hi) return;
  const StateView& S = A.state[cb];
  prefetch_range<TPB>(A.E[cb], lo, hi, 8);
#pragma unroll
  for (int f = 0; f < M::N_REAL; ++f) prefetch_range<TPB>(&S.rf<R>(f, 0, A.N), lo, hi, (int)sizeof(R));
#pragma unroll
  for (int f = 0; f < M::N_INT; ++f) prefetch_range<TPB>(&S.inf_(f, 0, A.N), lo, hi, 4);
}

// One tile of one run for segment k (the whole per-CTA body of a wave).
template <class M, int TPB>
__device__ __forceinline__ void step_tile(const RunDev& A, const int t, const int k, double* sh,
                                          int* sh_last, int* sh_kw, long long* sh_O, int* sh_ks) {
  using R = typename M::R;
  RunState* rs = A.rs;
  const int N = A.N;
  const int i = t * A.tile + threadIdx.x;
  const bool valid = (int)threadIdx.x < A.tile && i < N;
  const int nb = k & 1, cb = nb ^ 1;
  const StateView Sc = A.state[cb];
  const StateView Sn = A.state[nb];
  const bool redundant = A.redundant != 0;
  // resuming a snapshot: segment resume_k - 1 loads the population instead of running it
  const bool load = A.resume_k > 0 && k == A.resume_k - 1;
  typename M::Lane L;
  bool near = false;
  Stream s{A.k0, A.k1, (uint32_t)i, (uint32_t)k, 0u, 0u, A.md.tab};
  if (load) {
    if (valid) M::load(L, Sn, SnapView{A.snap_logw, A.snap_real, A.snap_int, A.snap_stack}, i, N, s);
  } else if (k > 0) {
    // (a run combined in every CTA keeps its offsets in shared memory and its
    // combine short: there the prefetch measured no gain)
    if (!redundant) prefetch_neighbours<M, TPB>(A, t, cb);
    SearchCtx X;
    X.rec = A.rec[cb];
    bool resample;
    if (redundant) {
      const Combined c = combine_offsets<TPB>(A.rec[cb], A.n_tiles, sh_O, sh_ks, sh,
                                              A.ess ? A.tq[cb] : nullptr);
      const bool go_on = c.kmax != kDeadTile && c.alive && k < A.max_segments;
      resample = decide_resample(A, c);
      if (t == 0 && threadIdx.x == 0) finish_segment(A, k, c, resample);
      if (!go_on) return;
      // the run's search scalars by one thread, shared through shared memory
      unsigned long long* shq = reinterpret_cast<unsigned long long*>(sh + TPB / 32 + 1);
      if (resample && threadIdx.x == 0) {
        Q64 d, z0;
        long long tolZ;
        search_scalars(c, N, A.recip_n, Unif<double>::first(philox(0u, (uint32_t)(k - 1), 0u, 1u, A.k0, A.k1)),
                       &d, &z0, &tolZ);
        shq[0] = d.hi;
        shq[1] = d.lo;
        shq[2] = z0.hi;
        shq[3] = z0.lo;
        shq[4] = (unsigned long long)tolZ;
      }
      __syncthreads();
      X.O = sh_O;
      X.ks = sh_ks;
      X.kmax = c.kmax;
      X.G = c.G;
      X.d = Q64{shq[0], shq[1]};
      X.z0 = Q64{shq[2], shq[3]};
      X.tolZ = (long long)shq[4];
    } else {
      resample = rs->resample != 0;
      X.O = A.tile_O;
      X.ks = nullptr;
      X.kmax = rs->kmax;
      X.G = rs->G;
      X.d = Q64{rs->d_hi, rs->d_lo};
      X.z0 = Q64{rs->z0_hi, rs->z0_lo};
      X.tolZ = rs->tolZ;
    }
    if (valid) {
      const int row = A.record_all ? k - 1 : 0;
      int a = resample ? systematic_search(i, A, X, A.E[cb], &near) : i;
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
      if (bad) {  // the access is skipped: the particle is killed
        M::init(L);
        L.pc = PC_STOP;
        L.logw = neg_inf<R>();
      } else if (resample) {
        M::gather(L, Sc, Sn, a, i, N, A.md);
      } else {  // not resampled: the particle keeps its state and its accumulated weight
        M::gather(L, Sc, Sn, i, i, N, A.md);
        L.logw = (R)A.logw[i];
      }
    }
    warp_add_u64(&rs->n_near, near ? 1ull : 0ull);
  } else if (valid) {
    M::init(L);
  }
  if (SMC_DEBUG_CHECKS && valid && !(L.pc == PC_STOP || (L.pc >= 0 && L.pc < M::NB))) {
    debug_record(rs, 2, i);  // a block index outside the table: not dispatched
    L.pc = PC_STOP;
    L.logw = neg_inf<R>();
  }
  const bool active = valid && !load && L.pc != PC_STOP;
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
  // work counters: Philox blocks of the model's draw stream and blocks executed
  warp_add_u64(&rs->n_draws, valid ? (unsigned long long)s.d : 0ull);
  warp_add_u64(&rs->n_blocks, (unsigned long long)n_exec);
  // Weights, first per warp as soon as the warp's particles reached the
  // checkpoint (overlapping the tile's slower warps): the warp's max M_w, its
  // power-of-two reference k_w = ceil(M_w / ln 2), and e_j = exp(logw_j - k_w
  // ln 2) 2^54 rounded to an integer on the integer pipes.  Then, after the tile barrier, the tile
  // reference k_t = max k_w, the exact shift of each weight to it, and the
  // tile's integer running sum E_j (the next segment's search keys).
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
  long long ef = 0;
  const double Mw = warp_max_key(lw);
  const int kw = Mw == -INFINITY ? kDeadTile : tile_exponent(Mw);
  if (valid && kw != kDeadTile) {
    // (an FP32 log-weight is exact as a double, so both precisions share the
    // normaliser's integer-pipe exponential)
    if (kw > -2048 && kw < 2048) {
      ef = weight_fix<54>(lw, ref_q58(kw), A.md.tab);  // integer pipes only
    } else {
      const double kd = (double)kw;
      const double d = fma(-kd, kLn2Lo, fma(-kd, kLn2Hi, lw));  // lw - kw ln 2, two-part ln 2
      ef = exp_fix54(d, A.md.tab);
    }
  }
  if (lane == 0) sh_kw[wid] = kw;
  alive = __syncthreads_or(alive);
  int kt = sh_kw[0];
#pragma unroll
  for (int w = 1; w < TPB / 32; ++w) kt = max(kt, sh_kw[w]);
  const int shift = kw == kDeadTile ? 64 : kt - kw;
  if (shift >= 63)
    ef = 0;
  else if (shift > 0)
    ef = (ef + (1ll << (shift - 1))) >> shift;
  const long long E = block_incl_scan_i64<TPB>(ef, reinterpret_cast<long long*>(sh));
  if (valid) A.E[nb][i] = E;
  if (A.ess) {  // the tile's sum of squared weights, units 2^-54 of 2^(2 k_t)
    const unsigned long long u = (unsigned long long)ef;
    const long long sq = (long long)((__umul64hi(u, u) << 10) | ((u * u) >> 54));
    __syncthreads();
    const long long Q = block_incl_scan_i64<TPB>(sq, reinterpret_cast<long long*>(sh));
    if (threadIdx.x == TPB - 1) A.tq[nb][t] = Q;
  }
  if (threadIdx.x == TPB - 1) {
    TileRec r;
    r.s = E;
    r.k = kt;
    r.alive = alive;
    A.rec[nb][t] = r;
  }
  if (redundant) return;  // the next wave combines
  __threadfence();
  __syncthreads();
  if (threadIdx.x == 0) {
    const unsigned prev = atomicAdd(&rs->arrive, 1u);
    *sh_last = (prev == (unsigned)A.n_tiles - 1u);
  }
  __syncthreads();
  if (*sh_last) {  // the run's last tile of segment k: combine for the next wave
    __threadfence();
    const Combined c = combine_offsets<TPB>(A.rec[nb], A.n_tiles, A.tile_O, nullptr, sh,
                                            A.ess ? A.tq[nb] : nullptr);
    if (threadIdx.x == 0) {
      const bool resample = decide_resample(A, c);
      rs->resample = resample ? 1 : 0;
      if (finish_segment(A, k + 1, c, resample) && resample) {
        Q64 d, z0;
        long long tolZ;
        search_scalars(c, N, A.recip_n, Unif<double>::first(philox(0u, (uint32_t)k, 0u, 1u, A.k0, A.k1)), &d,
                       &z0, &tolZ);
        rs->kmax = c.kmax;
        rs->G = c.G;
        rs->d_hi = d.hi;
        rs->d_lo = d.lo;
        rs->z0_hi = z0.hi;
        rs->z0_lo = z0.lo;
        rs->tolZ = tolZ;
      }
      rs->arrive = 0;
    }
  }
}

// One wave: CTA b runs tile cta_map[b].y of run cta_map[b].x, segment
// k = wave - start_wave of that run.
// 768 resident threads per SM (three 256-thread CTAs: the grid sizing of
// tile_for) bounds the kernel to 85 registers per thread.
// KIND 0 dispatches on each run's model; a KIND of SMC_MODEL_* is the kernel of
// waves whose runs all run that model (only its block table is compiled in).
template <typename R, int TPB, int KIND>
__global__ void __launch_bounds__(TPB, (sizeof(R) == 4 ? 1024 : 768) / TPB) wave_kernel(const RunDev* __restrict__ runs,
                                                   const int2* __restrict__ cta_map, unsigned wave) {
  __shared__ __align__(16) RunDev sr;
  __shared__ double sh[TPB / 32 + 2 + TPB + 1];
  __shared__ int sh_last;
  __shared__ int sh_kw[TPB / 32];
  __shared__ long long sh_O[redundant_cap(TPB)];
  __shared__ int sh_ks[redundant_cap(TPB)];
  const int2 rt = cta_map[blockIdx.x];
  {
    const int* src = reinterpret_cast<const int*>(runs + rt.x);
    int* dst = reinterpret_cast<int*>(&sr);
    for (int w = threadIdx.x; w < (int)(sizeof(RunDev) / 4); w += TPB) dst[w] = src[w];
  }
  __syncthreads();
  // Waves are launched with programmatic stream serialisation: the next wave's
  // CTAs may start (and copy their run table, which no kernel writes) while
  // this wave's last CTAs still run; everything below reads what the previous
  // wave wrote, so it waits for that wave's completion first.
  asm volatile("griddepcontrol.launch_dependents;" ::: "memory");
  asm volatile("griddepcontrol.wait;" ::: "memory");
  RunState* rs = sr.rs;
  if (*(volatile int32_t*)&rs->done) return;
  const int k = (int)(wave - sr.start_wave);  // wraps correctly past 2^32 waves
  if (k < 0) return;
  if (KIND == SMC_MODEL_LG) {
    step_tile<LgModel<R>, TPB>(sr, rt.y, k, sh, &sh_last, sh_kw, sh_O, sh_ks);
    return;
  }
  if (KIND == SMC_MODEL_CRBD) {
    step_tile<TreeModel<R, false>, TPB>(sr, rt.y, k, sh, &sh_last, sh_kw, sh_O, sh_ks);
    return;
  }
  switch (sr.md.kind) {
    case SMC_MODEL_LG: step_tile<LgModel<R>, TPB>(sr, rt.y, k, sh, &sh_last, sh_kw, sh_O, sh_ks); break;
    case SMC_MODEL_SEIR: step_tile<SeirModel<R>, TPB>(sr, rt.y, k, sh, &sh_last, sh_kw, sh_O, sh_ks); break;
    case SMC_MODEL_CRBD: step_tile<TreeModel<R, false>, TPB>(sr, rt.y, k, sh, &sh_last, sh_kw, sh_O, sh_ks); break;
    case SMC_MODEL_RATESHIFT: step_tile<TreeModel<R, true>, TPB>(sr, rt.y, k, sh, &sh_last, sh_kw, sh_O, sh_ks); break;
    case SMC_MODEL_CRBD_DS: step_tile<TreeDsModel<R>, TPB>(sr, rt.y, k, sh, &sh_last, sh_kw, sh_O, sh_ks); break;
    default: step_tile<GeoModel<R>, TPB>(sr, rt.y, k, sh, &sh_last, sh_kw, sh_O, sh_ks); break;
  }
}

// One bucket of a wave, launched so that it may begin before the kernel ahead
// of it in the stream has finished (wave_kernel waits for it where it must).
template <typename R, int TPB, int KIND>
cudaError_t launch_pdl(const RunDev* runs, const int2* map, int n, cudaStream_t st, unsigned wave) {
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = dim3((unsigned)n);
  cfg.blockDim = dim3(TPB);
  cfg.dynamicSmemBytes = 0;
  cfg.stream = st;
  cudaLaunchAttribute at[1];
  at[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
  at[0].val.programmaticStreamSerializationAllowed = 1;
  cfg.attrs = at;
  cfg.numAttrs = 1;
  return cudaLaunchKernelEx(&cfg, wave_kernel<R, TPB, KIND>, runs, map, wave);
}

template <typename R, int KIND>
cudaError_t launch_bucket(int b, const RunDev* runs, const int2* map, int n, cudaStream_t st,
                          unsigned wave) {
  switch (b) {
    case 0: return launch_pdl<R, 32, KIND>(runs, map, n, st, wave);
    case 1: return launch_pdl<R, 64, KIND>(runs, map, n, st, wave);
    case 2: return launch_pdl<R, 128, KIND>(runs, map, n, st, wave);
    default: return launch_pdl<R, 256, KIND>(runs, map, n, st, wave);
  }
}

}  // namespace smc
