// smc_engine.cu -- model registration and smc_run: Algorithm 1 (SMC over
// PCFGs) in the RootPPL loop order of Section 3.3, one fused kernel launch
// per segment.
//
// Segment k's kernel, one particle per thread, one tile of TPB particles per CTA:
//   prologue  (k > 0) systematic resampling search for this particle's
//             ancestor a_i = min{ j : q_j > i + u } over the previous
//             segment's weights, then the particle duplication of
//             Section 3.3: the ancestor's SoA fields are read straight into
//             registers (the gather is fused into the load), the pending
//             stack is copied only up to its stack pointer;
//   segment   blocks run until the next checkpoint with per-warp PC-sorted
//             dispatch (smc_models.cuh); draws from Philox counters;
//   epilogue  the tile's FP64 max M_t, e_j = exp(logw_j - M_t) and its
//             inclusive scan E_j (written out for the next segment's search),
//             tile total s_t; the last CTA to finish combines the tiles:
//             m = max M_t, c_t = exp(M_t - m), exclusive tile offsets
//             O_t = sum_{t'<t} c_t' s_t', S = total, log Z += m + (log S - log N),
//             the resampling uniform u_k and r = N / S.
// The running sum used by the next search is P_j = min(O_t + c_t E_j, O_{t+1})
// (the tile offsets are made monotone with a running max, and the clamp keeps
// P monotone across tile seams) and the scaled boundary is q_j = P_j r.  The
// run stops after the segment in which every particle reached b_stop (no
// resampling after it).
//
// Tiles are sized so that the grid is a whole multiple of the SM count times
// the resident CTAs per SM (all CTAs of a segment run in one wave, equally
// loaded), with at most TPB particles per tile.
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <cstring>
#include <new>
#include <vector>

#include "smc_device.cuh"
#include "smc_internal.h"
#include "smc_models.cuh"

namespace smc {

struct RunState {
  double log_z, m, S, r, u, inv_r;
  unsigned long long n_near, n_overflow, n_limit;
  int32_t done, status, n_segments, n_resamples;
  uint32_t arrive;
  int32_t pad_[3];
};

struct StepArgs {
  ModelDev md;
  StateView state[2];
  double* logw;    // [N] log-weights of the latest segment (f64; FP32 values widened)
  double* E[2];    // [N] tile-local inclusive scans, double-buffered by segment parity
  double* tile_M;  // [n_tiles]
  double* tile_s;  // [n_tiles]
  int32_t* tile_alive;
  double* tile_c;     // [n_tiles] written by the combine: exp(M_t - m)
  double* tile_invc;  // [n_tiles] 1 / c_t (0 where c_t = 0)
  double* tile_O;     // [n_tiles + 1] monotone exclusive offsets, O_T >= S
  double* tile_q;     // [n_tiles + 1] O_t * r
  int32_t* anc;       // ancestor rows
  double* incr;       // [max_segments] per-segment log-Z increments
  RunState* rs;
  int N, n_tiles, tile, max_segments, record_all, anc_rows;
  uint32_t k0, k1;
};

// Non-negative doubles order like their bit patterns read as int64, so the
// searches below compare bits on the integer pipes and spend FP64 work only on
// the few boundary values they actually form.
__device__ __forceinline__ long long dbits(double x) { return __double_as_longlong(x); }

// q_j = min(O_t + c_t E_j, O_{t+1}) * r for j in tile t.
__device__ __forceinline__ double q_at(int j, const StepArgs& A, const double* __restrict__ E,
                                       double r) {
  const int t = j / A.tile;
  const double P = fmin(A.tile_O[t] + A.tile_c[t] * E[j], A.tile_O[t + 1]);
  return P * r;
}

// a_i = min{ j : q_j > i + u } (N - 1 if none).  Tile first: t = max{t : O_t r <= y};
// inside the tile the threshold e* = (y / r - O_t) / c_t on E locates the
// candidate, and the exact q_j then fixes it up by +-1 if rounding moved it.
// If no element of tile t qualifies, the first element of tile t+1 does.
// Flags the offset when it lies within 1e-12 N of q_a or q_{a-1}.
__device__ __forceinline__ int systematic_search(int i, const StepArgs& A, const double* E,
                                                 double r, double inv_r, double u, bool* near) {
  const int N = A.N, T = A.n_tiles;
  const double y = (double)i + u;
  const long long yb = dbits(y);
  int lo = 0, hi = T;  // tile_q[0] = 0 <= y
  while (lo < hi) {
    const int mid = (lo + hi + 1) >> 1;
    if (dbits(A.tile_q[mid]) <= yb)
      lo = mid;
    else
      hi = mid - 1;
  }
  int a;
  if (lo >= T) {
    a = N - 1;
  } else {
    const int t = lo;
    const int j0 = t * A.tile, j1 = min(N, j0 + A.tile);
    const long long eb = dbits((y * inv_r - A.tile_O[t]) * A.tile_invc[t]);
    int l = j0, h = j1;  // first j in [j0, j1) with E_j > e*
    while (l < h) {
      const int mid = (l + h) >> 1;
      if (dbits(E[mid]) > eb)
        h = mid;
      else
        l = mid + 1;
    }
    int j = l;
    while (j < j1 && dbits(q_at(j, A, E, r)) <= yb) ++j;
    while (j > j0 && dbits(q_at(j - 1, A, E, r)) > yb) --j;
    a = j < j1 ? j : (j1 < N ? j1 : N - 1);
  }
  const double tol = kBoundaryEps * (double)N;
  bool f = fabs(q_at(a, A, E, r) - y) < tol;
  if (a > 0 && fabs(q_at(a - 1, A, E, r) - y) < tol) f = true;
  *near = f;
  return a;
}

__device__ __forceinline__ void warp_add_u64(unsigned long long* dst, unsigned long long v) {
  v = __reduce_add_sync(0xffffffffu, (unsigned)v);
  if ((threadIdx.x & 31) == 0 && v) atomicAdd(dst, v);
}

// The last CTA of a segment: combine the tile reductions (all FP64).
template <int TPB>
__device__ void combine_tiles(const StepArgs& A, int k, double* sh) {
  RunState* rs = A.rs;
  const int nt = A.n_tiles;
  double* shx = sh + TPB / 32 + 1;  // [TPB + 1] scratch after the block-op area
  double mloc = -INFINITY;
  int alive = 0;
  for (int t = threadIdx.x; t < nt; t += TPB) {
    mloc = fmax(mloc, __ldcg(A.tile_M + t));
    alive |= __ldcg(A.tile_alive + t);
  }
  const double m = block_max<TPB>(mloc, sh);
  alive = __syncthreads_or(alive);
  if (m == -INFINITY) {
    if (threadIdx.x == 0) {
      rs->log_z = -INFINITY;
      rs->m = m;
      rs->S = 0.0;
      A.incr[k] = -INFINITY;
      rs->status = SMC_EDEGENERATE;
      rs->n_segments = k + 1;
      rs->done = 1;
      rs->arrive = 0;
    }
    return;
  }
  // exclusive offsets O_t of v_t = c_t s_t, made monotone by a running max
  double carry = 0.0, omax = 0.0;
  for (int base = 0; base < nt; base += TPB) {
    const int t = base + threadIdx.x;
    double c = 0.0, v = 0.0;
    if (t < nt) {
      const double Mt = __ldcg(A.tile_M + t);
      c = (Mt == -INFINITY) ? 0.0 : exp(Mt - m);
      v = __ldcg(A.tile_s + t) * c;
    }
    const double incl = block_incl_scan<TPB>(v, sh);
    __syncthreads();
    shx[threadIdx.x + 1] = incl;
    __syncthreads();
    const double excl = threadIdx.x ? shx[threadIdx.x] : 0.0;
    const double chunk_total = shx[TPB];
    const double O = block_incl_max<TPB>(fmax(carry + excl, omax), sh);
    if (t < nt) {
      A.tile_c[t] = c;
      A.tile_invc[t] = c > 0.0 ? 1.0 / c : 0.0;
      A.tile_O[t] = O;
    }
    __syncthreads();
    if (threadIdx.x == TPB - 1) shx[0] = O;
    __syncthreads();
    omax = shx[0];
    carry = carry + chunk_total;
    __syncthreads();
  }
  const double S = carry;
  const double r = (double)A.N / S;
  if (threadIdx.x == 0) A.tile_O[nt] = fmax(S, omax);
  __syncthreads();
  for (int t = threadIdx.x; t <= nt; t += TPB) A.tile_q[t] = A.tile_O[t] * r;
  if (threadIdx.x == 0) {
    const double inc = m + (log(S) - log((double)A.N));
    rs->log_z = rs->log_z + inc;
    A.incr[k] = inc;
    rs->m = m;
    rs->S = S;
    rs->n_segments = k + 1;
    if (!alive) {
      rs->done = 1;
    } else if (k + 1 >= A.max_segments) {
      rs->status = SMC_ESTEPLIMIT;
      rs->done = 1;
    } else {
      const Block4 b = philox(0u, (uint32_t)k, 0u, 1u, A.k0, A.k1);
      rs->u = Unif<double>::first(b);
      rs->r = r;
      rs->inv_r = S / (double)A.N;
    }
    rs->arrive = 0;
  }
}

template <class M, int TPB>
__global__ void __launch_bounds__(TPB) step_kernel(const StepArgs A, const int k) {
  using R = typename M::R;
  __shared__ double sh[TPB / 32 + 2 + TPB + 1];
  __shared__ int sh_last;
  RunState* rs = A.rs;
  if (*(volatile int32_t*)&rs->done) return;
  const int N = A.N;
  const int i = blockIdx.x * A.tile + threadIdx.x;
  const bool valid = (int)threadIdx.x < A.tile && i < N;
  const int nb = k & 1, cb = nb ^ 1;
  const StateView Sc = A.state[cb];
  const StateView Sn = A.state[nb];
  typename M::Lane L;
  bool near = false;
  if (valid) {
    if (k == 0) {
      M::init(L);
    } else {
      const double r = rs->r, u = rs->u, inv_r = rs->inv_r;
      const int a = systematic_search(i, A, A.E[cb], r, inv_r, u, &near);
      const int row = A.record_all ? k - 1 : 0;
      if (row < A.anc_rows) A.anc[(size_t)row * N + i] = a;
      M::gather(L, Sc, Sn, a, i, N, A.md);
    }
  }
  if (k > 0) warp_add_u64(&rs->n_near, near ? 1ull : 0ull);
  Stream s{A.k0, A.k1, (uint32_t)i, (uint32_t)k, 0u, 0u};
  const bool active = valid && L.pc != PC_STOP;
  run_segment<M>(L, s, A.md, Sn, i, k, N, active);
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
  // tile reduction (FP64)
  const double Mt = block_max<TPB>(lw, sh);
  const double e = (valid && Mt != -INFINITY) ? exp(lw - Mt) : 0.0;
  const double E = block_incl_scan<TPB>(e, sh);
  if (valid) A.E[nb][i] = E;
  alive = __syncthreads_or(alive);
  if (threadIdx.x == TPB - 1) {
    A.tile_M[blockIdx.x] = Mt;
    A.tile_s[blockIdx.x] = E;
  }
  if (threadIdx.x == 0) A.tile_alive[blockIdx.x] = alive;
  __threadfence();
  __syncthreads();
  if (threadIdx.x == 0) {
    const unsigned prev = atomicAdd(&rs->arrive, 1u);
    sh_last = (prev == (unsigned)gridDim.x - 1u);
  }
  __syncthreads();
  if (sh_last) {
    __threadfence();
    combine_tiles<TPB>(A, k, sh);
  }
}

// Final outputs: real fields widened to f64, int fields, stack rows with
// entries at or above the stack pointer zeroed.
template <typename R>
__global__ void finalize_kernel(StateView S, int N, int n_real, int n_int, int cap, double* real_out,
                                int32_t* int_out, double* stack_out) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= N) return;
  if (real_out)
    for (int f = 0; f < n_real; ++f) real_out[(size_t)f * N + i] = (double)S.rf<R>(f, i, N);
  if (int_out)
    for (int f = 0; f < n_int; ++f) int_out[(size_t)f * N + i] = S.inf_(f, i, N);
  if (stack_out && cap > 0) {
    const int sp = S.inf_(1, i, N);
    for (int r = 0; r < cap; ++r)
      stack_out[(size_t)r * N + i] = r < sp ? (double)S.st<R>(r, i, N) : 0.0;
  }
}

}  // namespace smc

using namespace smc;

// ------------------------------------------------------------------------
// host side
// ------------------------------------------------------------------------
struct smc_model_s {
  smc_model_desc desc;
  ModelDev md;
  int32_t n_real, n_int, stack_cap, n_segments_known;
  void* dev_blob = nullptr;  // observations / tree arrays
  void* ws = nullptr;        // cached workspace
  size_t ws_bytes = 0;
  cudaEvent_t ev0 = nullptr, ev1 = nullptr;
  std::vector<cudaEvent_t> ev_seg;  // per-launch timing pairs (time_kernels)
};

namespace {

#define SMC_ARG(...) __VA_ARGS__
constexpr int kTPB = 256;
constexpr int kMaxAncRows = 4096;
constexpr int kMaxSegments = 1 << 24;

struct Layout {
  size_t real[2], ints[2], stack[2], logw, E[2], tM, ts, talive, tc, tinvc, tO, tq, rs, anc, incr,
      fin_real, fin_int, fin_stack, total;
  int n_tiles, tile, anc_rows, max_segments;
};

// Particles per tile: one wave of equally loaded CTAs when N is small enough,
// full TPB-particle tiles otherwise.
int tile_size(int64_t N, int ctas_per_sm, int n_sms) {
  const int64_t slots = (int64_t)std::max(1, ctas_per_sm) * std::max(1, n_sms);
  int64_t t = (N + slots - 1) / slots;
  if (t < 32) t = std::min<int64_t>(32, N);
  if (t > kTPB) t = kTPB;
  return (int)std::max<int64_t>(1, t);
}

int model_fields(int kind, int* n_real, int* n_int) {
  switch (kind) {
    case SMC_MODEL_LG: *n_real = 1; *n_int = 1; return 0;
    case SMC_MODEL_CRBD: *n_real = 2; *n_int = 1; return 0;
    case SMC_MODEL_RATESHIFT: *n_real = 2; *n_int = 2; return 0;
    case SMC_MODEL_GEOMETRIC: *n_real = 0; *n_int = 2; return 0;
  }
  return -1;
}

Layout make_layout(const smc_model_s* m, const smc_run_cfg* c, int ctas_per_sm, int n_sms) {
  Layout L{};
  const size_t N = (size_t)c->n_particles;
  const size_t rb = c->precision == SMC_PREC_FP32 ? 4 : 8;
  L.tile = tile_size((int64_t)N, ctas_per_sm, n_sms);
  L.n_tiles = (int)((N + L.tile - 1) / L.tile);
  L.max_segments = c->max_segments > 0 ? c->max_segments
                   : (m->n_segments_known > 0 ? m->n_segments_known : (1 << 20));
  const int max_res = std::max(1, L.max_segments - 1);
  // unknown-length models keep at most kMaxAncRows recorded resamplings
  L.anc_rows = c->record_all_ancestors ? (m->n_segments_known > 0 ? max_res : std::min(max_res, kMaxAncRows)) : 1;
  size_t off = 0;
  auto take = [&](size_t bytes) {
    const size_t o = off;
    off = align_up(off + std::max<size_t>(bytes, 1), 256);
    return o;
  };
  for (int b = 0; b < 2; ++b) {
    L.real[b] = take(rb * N * (size_t)m->n_real);
    L.ints[b] = take(4 * N * (size_t)m->n_int);
    L.stack[b] = take(rb * N * (size_t)m->stack_cap);
  }
  L.logw = take(8 * N);
  L.E[0] = take(8 * N);
  L.E[1] = take(8 * N);
  L.tM = take(8 * (size_t)L.n_tiles);
  L.ts = take(8 * (size_t)L.n_tiles);
  L.talive = take(4 * (size_t)L.n_tiles);
  L.tc = take(8 * (size_t)L.n_tiles);
  L.tinvc = take(8 * (size_t)L.n_tiles);
  L.tO = take(8 * (size_t)(L.n_tiles + 1));
  L.tq = take(8 * (size_t)(L.n_tiles + 1));
  L.rs = take(sizeof(RunState));
  L.anc = take(4 * N * (size_t)L.anc_rows);
  L.incr = take(8 * (size_t)L.max_segments);
  L.fin_real = take(8 * N * (size_t)m->n_real);
  L.fin_int = take(4 * N * (size_t)m->n_int);
  L.fin_stack = take(8 * N * (size_t)m->stack_cap);
  L.total = off;
  return L;
}

template <class M>
cudaError_t launch_segment(const StepArgs& A, int k, cudaStream_t st) {
  step_kernel<M, kTPB><<<A.n_tiles, kTPB, 0, st>>>(A, k);
  return cudaGetLastError();
}

template <class M>
int occupancy() {
  int n = 0;
  if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, step_kernel<M, kTPB>, kTPB, 0) != cudaSuccess)
    return 1;
  return std::max(1, n);
}

typedef cudaError_t (*seg_fn)(const StepArgs&, int, cudaStream_t);
struct SegKernel {
  seg_fn launch;
  int (*occ)();
};

SegKernel pick_segment(int kind, int prec) {
  const bool f32 = prec == SMC_PREC_FP32;
#define SMC_SEG(M) SegKernel{launch_segment<M>, occupancy<M>}
  switch (kind) {
    case SMC_MODEL_LG: return f32 ? SMC_SEG(LgModel<float>) : SMC_SEG(LgModel<double>);
    case SMC_MODEL_CRBD:
      return f32 ? SMC_SEG(SMC_ARG(TreeModel<float, false>)) : SMC_SEG(SMC_ARG(TreeModel<double, false>));
    case SMC_MODEL_RATESHIFT:
      return f32 ? SMC_SEG(SMC_ARG(TreeModel<float, true>)) : SMC_SEG(SMC_ARG(TreeModel<double, true>));
    case SMC_MODEL_GEOMETRIC: return f32 ? SMC_SEG(GeoModel<float>) : SMC_SEG(GeoModel<double>);
  }
#undef SMC_SEG
  return SegKernel{nullptr, nullptr};
}

// device properties of the current device, cached per device
int sm_count() {
  static int cached[64] = {0};
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= 64) return 152;
  if (!cached[dev]) {
    int n = 0;
    if (cudaDeviceGetAttribute(&n, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess || n <= 0) n = 152;
    cached[dev] = n;
  }
  return cached[dev];
}

smc_status check_tree(const smc_model_desc* d) {
  const int M = d->n_nodes;
  if (M < 3 || (M & 1) == 0) return set_error(SMC_EINVAL, "n_nodes must be odd and >= 3");
  if (!d->parent || !d->left || !d->right || !d->preorder || !d->age)
    return set_error(SMC_EINVAL, "tree arrays must be non-NULL");
  if (d->parent[0] != -1 || d->preorder[0] != 0)
    return set_error(SMC_EINVAL, "node 0 must be the root and first in preorder");
  std::vector<char> seen(M, 0);
  for (int j = 0; j < M; ++j) {
    const int v = d->preorder[j];
    if (v < 0 || v >= M || seen[v]) return set_error(SMC_EINVAL, "preorder is not a permutation");
    seen[v] = 1;
    const int l = d->left[v], r = d->right[v];
    if ((l < 0) != (r < 0)) return set_error(SMC_EINVAL, "node %d has one child", v);
    if (l >= M || r >= M) return set_error(SMC_EINVAL, "child index out of range");
    if (l >= 0 && (d->parent[l] != v || d->parent[r] != v))
      return set_error(SMC_EINVAL, "parent/child arrays disagree at node %d", v);
    if (l >= 0 && (j + 1 >= M || d->preorder[j + 1] != l))
      return set_error(SMC_EINVAL, "preorder is not left-first at node %d", v);
    if (v != 0) {
      const int p = d->parent[v];
      if (p < 0 || p >= M) return set_error(SMC_EINVAL, "parent out of range");
      if (!(d->age[p] >= d->age[v]) || !(d->age[v] >= 0.0))
        return set_error(SMC_EINVAL, "ages must be >= 0 and not increase towards the tips");
    }
  }
  if (!(d->rho > 0.0 && d->rho <= 1.0)) return set_error(SMC_EINVAL, "rho must be in (0, 1]");
  if (d->depth_cap < 1 || d->depth_cap > SMC_MAX_DEPTH)
    return set_error(SMC_EINVAL, "depth_cap must be in 1..%d", SMC_MAX_DEPTH);
  if (d->call_limit < 1) return set_error(SMC_EINVAL, "call_limit must be >= 1");
  if (d->fixed_rates && !(d->lambda_fixed >= 0.0 && d->mu_fixed >= 0.0))
    return set_error(SMC_EINVAL, "fixed rates must be >= 0");
  if (!d->fixed_rates && !(d->lambda_scale > 0.0 && d->mu_scale > 0.0))
    return set_error(SMC_EINVAL, "prior scales must be > 0");
  if (d->kind == SMC_MODEL_RATESHIFT) {
    if (d->lam_stack_cap < 1) return set_error(SMC_EINVAL, "lam_stack_cap must be >= 1");
    if (!(d->sigma >= 0.0)) return set_error(SMC_EINVAL, "sigma must be >= 0");
  }
  return SMC_OK;
}

}  // namespace

extern "C" smc_status smc_model_register(const smc_model_desc* d, smc_model_t* out) {
  if (!d || !out) return set_error(SMC_EINVAL, "NULL argument");
  *out = nullptr;
  int n_real, n_int;
  if (model_fields(d->kind, &n_real, &n_int)) return set_error(SMC_EINVAL, "unknown model kind");
  size_t blob = 0;
  if (d->kind == SMC_MODEL_LG) {
    if (d->T < 1 || !d->obs) return set_error(SMC_EINVAL, "LG needs T >= 1 observations");
    if (!(d->r_sd > 0.0) || !(d->x0_sd >= 0.0) || !(d->q_sd >= 0.0))
      return set_error(SMC_EINVAL, "LG standard deviations must be >= 0 (r_sd > 0)");
    blob = 8 * (size_t)d->T;
  } else if (d->kind == SMC_MODEL_GEOMETRIC) {
    if (!(d->geo_p >= 0.0 && d->geo_p <= 1.0)) return set_error(SMC_EINVAL, "geo_p in [0,1]");
  } else {
    smc_status st = check_tree(d);
    if (st) return st;
    blob = align_up(4 * (size_t)d->n_nodes, 256) * 3 + align_up(8 * (size_t)d->n_nodes, 256) * 2;
  }
  smc_model_s* m = new (std::nothrow) smc_model_s();
  if (!m) return set_error(SMC_ENOMEM, "host allocation failed");
  m->desc = *d;
  m->n_real = n_real;
  m->n_int = n_int;
  m->stack_cap = d->kind == SMC_MODEL_RATESHIFT ? d->lam_stack_cap : 0;
  ModelDev& md = m->md;
  std::memset(&md, 0, sizeof(md));
  md.kind = d->kind;
  md.T = d->T;
  md.n_nodes = d->n_nodes;
  md.fixed_rates = d->fixed_rates;
  md.depth_cap = d->depth_cap;
  md.call_limit = d->call_limit;
  md.lam_stack_cap = d->lam_stack_cap;
  md.x0_mean = d->x0_mean;
  md.x0_sd = d->x0_sd;
  md.a = d->a;
  md.b = d->b;
  md.q_sd = d->q_sd;
  md.r_sd = d->r_sd;
  md.rho = d->rho;
  md.lambda_fixed = d->lambda_fixed;
  md.mu_fixed = d->mu_fixed;
  md.lambda_scale = d->lambda_scale;
  md.mu_scale = d->mu_scale;
  md.sigma = d->sigma;
  md.geo_p = d->geo_p;
  md.geo_logw = d->geo_logw;
  m->n_segments_known = 0;
  if (d->kind == SMC_MODEL_LG) {
    md.lg_lc = std::log(d->r_sd) + 0.91893853320467274178;
    m->n_segments_known = d->T;
  }
  if (d->kind == SMC_MODEL_CRBD || d->kind == SMC_MODEL_RATESHIFT) {
    const int tips = (d->n_nodes + 1) / 2;
    double lnfact = 0.0;
    for (int i = 2; i <= tips; ++i) lnfact = lnfact + std::log((double)i);
    md.corr = (double)(tips - 1) * kLn2 - lnfact;
    m->n_segments_known = d->n_nodes;
  }
  if (blob) {
    if (d->fixed_mult) blob += align_up(8 * (size_t)d->n_nodes, 256);
    cudaError_t e = cudaMalloc(&m->dev_blob, blob);
    if (e != cudaSuccess) {
      delete m;
      return cuda_fail(e, "cudaMalloc(model data)");
    }
    char* p = (char*)m->dev_blob;
    auto put = [&](const void* src, size_t bytes) -> void* {
      void* dst = p;
      if (cudaMemcpy(dst, src, bytes, cudaMemcpyHostToDevice) != cudaSuccess) return nullptr;
      p += align_up(bytes, 256);
      return dst;
    };
    bool ok = true;
    if (d->kind == SMC_MODEL_LG) {
      ok = (md.obs = (const double*)put(d->obs, 8 * (size_t)d->T)) != nullptr;
    } else {
      const size_t M = d->n_nodes;
      ok = (md.parent = (const int*)put(d->parent, 4 * M)) && (md.left = (const int*)put(d->left, 4 * M)) &&
           (md.preorder = (const int*)put(d->preorder, 4 * M)) && (md.age = (const double*)put(d->age, 8 * M));
      if (ok && d->fixed_mult) ok = (md.fixed_mult = (const double*)put(d->fixed_mult, 8 * M)) != nullptr;
    }
    if (!ok) {
      cudaFree(m->dev_blob);
      delete m;
      return set_error(SMC_ECUDA, "copying model data to the device failed");
    }
  }
  if (cudaEventCreate(&m->ev0) != cudaSuccess || cudaEventCreate(&m->ev1) != cudaSuccess) {
    if (m->dev_blob) cudaFree(m->dev_blob);
    delete m;
    return set_error(SMC_ECUDA, "cudaEventCreate failed");
  }
  *out = m;
  return SMC_OK;
}

extern "C" void smc_model_destroy(smc_model_t m) {
  if (!m) return;
  if (m->ws) cudaFree(m->ws);
  if (m->dev_blob) cudaFree(m->dev_blob);
  if (m->ev0) cudaEventDestroy(m->ev0);
  if (m->ev1) cudaEventDestroy(m->ev1);
  for (cudaEvent_t e : m->ev_seg) cudaEventDestroy(e);
  delete m;
}

extern "C" smc_status smc_model_info(smc_model_t m, int32_t* n_real, int32_t* n_int,
                                     int32_t* stack_cap, int32_t* n_segments) {
  if (!m) return set_error(SMC_EINVAL, "NULL model");
  if (n_real) *n_real = m->n_real;
  if (n_int) *n_int = m->n_int;
  if (stack_cap) *stack_cap = m->stack_cap;
  if (n_segments) *n_segments = m->n_segments_known;
  return SMC_OK;
}

static smc_status check_cfg(const smc_model_s* m, const smc_run_cfg* c) {
  if (!m || !c) return set_error(SMC_EINVAL, "NULL argument");
  if (c->n_particles < 1 || c->n_particles > (int64_t)0x7fffffff - kTPB)
    return set_error(SMC_EINVAL, "n_particles must be in 1..2^31-257");
  if (c->precision != SMC_PREC_FP64 && c->precision != SMC_PREC_FP32)
    return set_error(SMC_EINVAL, "unknown precision");
  if (c->max_segments < 0 || c->max_segments > kMaxSegments)
    return set_error(SMC_EINVAL, "max_segments must be in 0..2^24");
  return SMC_OK;
}

extern "C" smc_status smc_workspace_bytes(smc_model_t m, const smc_run_cfg* c, size_t* bytes) {
  smc_status st = check_cfg(m, c);
  if (st) return st;
  if (!bytes) return set_error(SMC_EINVAL, "NULL bytes");
  const SegKernel sk = pick_segment(m->desc.kind, c->precision);
  *bytes = make_layout(m, c, sk.occ(), sm_count()).total;
  return SMC_OK;
}

extern "C" smc_status smc_run(smc_model_t m, const smc_run_cfg* c, smc_result* r, void* stream) {
  smc_status st = check_cfg(m, c);
  if (st) return st;
  if (!r) return set_error(SMC_EINVAL, "NULL result");
  if (r->where != SMC_MEM_HOST && r->where != SMC_MEM_DEVICE)
    return set_error(SMC_EINVAL, "result.where must be SMC_MEM_HOST or SMC_MEM_DEVICE");
  cudaStream_t cs = (cudaStream_t)stream;
  const SegKernel sk = pick_segment(m->desc.kind, c->precision);
  const Layout Ly = make_layout(m, c, sk.occ(), sm_count());
  char* ws;
  if (c->workspace) {
    if (c->workspace_bytes < Ly.total)
      return set_error(SMC_EINVAL, "workspace too small (%zu < %zu)", c->workspace_bytes, Ly.total);
    ws = (char*)c->workspace;
  } else {
    if (m->ws_bytes < Ly.total) {
      if (m->ws) cudaFree(m->ws);
      m->ws = nullptr;
      m->ws_bytes = 0;
      cudaError_t e = cudaMalloc(&m->ws, Ly.total);
      if (e != cudaSuccess) return set_error(SMC_ENOMEM, "workspace cudaMalloc(%zu): %s", Ly.total, cudaGetErrorString(e));
      m->ws_bytes = Ly.total;
    }
    ws = (char*)m->ws;
  }
  const int N = (int)c->n_particles;
  StepArgs A;
  std::memset(&A, 0, sizeof(A));
  A.md = m->md;
  for (int b = 0; b < 2; ++b) {
    A.state[b].real = ws + Ly.real[b];
    A.state[b].ints = (int32_t*)(ws + Ly.ints[b]);
    A.state[b].stack = ws + Ly.stack[b];
    A.E[b] = (double*)(ws + Ly.E[b]);
  }
  A.logw = (double*)(ws + Ly.logw);
  A.tile_M = (double*)(ws + Ly.tM);
  A.tile_s = (double*)(ws + Ly.ts);
  A.tile_alive = (int32_t*)(ws + Ly.talive);
  A.tile_c = (double*)(ws + Ly.tc);
  A.tile_invc = (double*)(ws + Ly.tinvc);
  A.tile_O = (double*)(ws + Ly.tO);
  A.tile_q = (double*)(ws + Ly.tq);
  A.anc = (int32_t*)(ws + Ly.anc);
  A.incr = (double*)(ws + Ly.incr);
  A.rs = (RunState*)(ws + Ly.rs);
  A.N = N;
  A.n_tiles = Ly.n_tiles;
  A.tile = Ly.tile;
  A.max_segments = Ly.max_segments;
  A.record_all = c->record_all_ancestors ? 1 : 0;
  A.anc_rows = Ly.anc_rows;
  A.k0 = (uint32_t)(c->seed & 0xffffffffu);
  A.k1 = (uint32_t)(c->seed >> 32) ^ c->run_id;
  seg_fn fn = sk.launch;
  SMC_CUDA_TRY(cudaMemsetAsync(A.rs, 0, sizeof(RunState), cs));
  SMC_CUDA_TRY(cudaEventRecord(m->ev0, cs));
  RunState hrs;
  int launched = 0;
  const bool timed = c->time_kernels != 0;
  // one kernel per segment; with time_kernels an event pair brackets each launch
  auto launch = [&](int k) -> smc_status {
    if (timed) {
      while ((int)m->ev_seg.size() < 2 * (launched + 1)) {
        cudaEvent_t e;
        SMC_CUDA_TRY(cudaEventCreate(&e));
        m->ev_seg.push_back(e);
      }
      SMC_CUDA_TRY(cudaEventRecord(m->ev_seg[2 * launched], cs));
    }
    SMC_CUDA_TRY(fn(A, k, cs));
    if (timed) SMC_CUDA_TRY(cudaEventRecord(m->ev_seg[2 * launched + 1], cs));
    ++launched;
    return SMC_OK;
  };
  if (m->n_segments_known > 0 && Ly.max_segments >= m->n_segments_known) {
    for (int k = 0; k < m->n_segments_known; ++k) {
      smc_status ls = launch(k);
      if (ls) return ls;
    }
  } else {
    // segment count unknown (or capped): poll the device termination flag
    const int chunk = 16;
    for (int k0 = 0; k0 < Ly.max_segments; k0 += chunk) {
      const int k1 = std::min(Ly.max_segments, k0 + chunk);
      for (int k = k0; k < k1; ++k) {
        smc_status ls = launch(k);
        if (ls) return ls;
      }
      SMC_CUDA_TRY(cudaMemcpyAsync(&hrs, A.rs, sizeof(RunState), cudaMemcpyDeviceToHost, cs));
      SMC_CUDA_TRY(cudaStreamSynchronize(cs));
      if (hrs.done) break;
    }
  }
  SMC_CUDA_TRY(cudaEventRecord(m->ev1, cs));
  SMC_CUDA_TRY(cudaMemcpyAsync(&hrs, A.rs, sizeof(RunState), cudaMemcpyDeviceToHost, cs));
  SMC_CUDA_TRY(cudaStreamSynchronize(cs));
  if (!hrs.done && hrs.status == 0) hrs.status = SMC_ESTEPLIMIT;
  float ms = 0.f;
  cudaEventElapsedTime(&ms, m->ev0, m->ev1);
  // outputs
  const int fb = (hrs.n_segments - 1) & 1;
  const bool host = r->where == SMC_MEM_HOST;
  double* fin_real = host ? (double*)(ws + Ly.fin_real) : r->real_fields;
  int32_t* fin_int = host ? (int32_t*)(ws + Ly.fin_int) : r->int_fields;
  double* fin_stack = host ? (double*)(ws + Ly.fin_stack) : r->stack;
  if (hrs.n_segments > 0 && (r->real_fields || r->int_fields || r->stack)) {
    const int blocks = (N + 255) / 256;
    if (c->precision == SMC_PREC_FP32)
      finalize_kernel<float><<<blocks, 256, 0, cs>>>(A.state[fb], N, m->n_real, m->n_int, m->stack_cap,
                                                     r->real_fields ? fin_real : nullptr,
                                                     r->int_fields ? fin_int : nullptr,
                                                     r->stack ? fin_stack : nullptr);
    else
      finalize_kernel<double><<<blocks, 256, 0, cs>>>(A.state[fb], N, m->n_real, m->n_int, m->stack_cap,
                                                      r->real_fields ? fin_real : nullptr,
                                                      r->int_fields ? fin_int : nullptr,
                                                      r->stack ? fin_stack : nullptr);
    SMC_CUDA_TRY(cudaGetLastError());
  }
  const cudaMemcpyKind kind = host ? cudaMemcpyDeviceToHost : cudaMemcpyDeviceToDevice;
  if (r->log_z) SMC_CUDA_TRY(cudaMemcpyAsync(r->log_z, &A.rs->log_z, 8, kind, cs));
  if (r->final_logw) SMC_CUDA_TRY(cudaMemcpyAsync(r->final_logw, A.logw, 8 * (size_t)N, kind, cs));
  if (host) {
    if (r->real_fields && m->n_real)
      SMC_CUDA_TRY(cudaMemcpyAsync(r->real_fields, fin_real, 8 * (size_t)N * m->n_real, kind, cs));
    if (r->int_fields && m->n_int)
      SMC_CUDA_TRY(cudaMemcpyAsync(r->int_fields, fin_int, 4 * (size_t)N * m->n_int, kind, cs));
    if (r->stack && m->stack_cap)
      SMC_CUDA_TRY(cudaMemcpyAsync(r->stack, fin_stack, 8 * (size_t)N * m->stack_cap, kind, cs));
  }
  if (r->ancestors && hrs.n_resamples >= 0) {
    const int n_res = std::max(0, hrs.n_segments - 1);
    const int rows = c->record_all_ancestors ? std::min(std::min(n_res, r->ancestors_rows), Ly.anc_rows)
                                             : (n_res > 0 ? 1 : 0);
    if (rows > 0) SMC_CUDA_TRY(cudaMemcpyAsync(r->ancestors, A.anc, 4 * (size_t)N * rows, kind, cs));
  }
  SMC_CUDA_TRY(cudaStreamSynchronize(cs));
  smc_counters& ct = r->counters;
  ct.n_segments = hrs.n_segments;
  ct.n_resamples = std::max(0, hrs.n_segments - 1);
  ct.n_near_boundary = (int64_t)hrs.n_near;
  ct.n_overflow = (int64_t)hrs.n_overflow;
  ct.n_limit = (int64_t)hrs.n_limit;
  ct.device_ms = ms;
  ct.kernel_launches = launched;
  ct.kernel_ms = 0.0;
  if (timed)
    for (int q = 0; q < launched; ++q) {
      float t = 0.f;
      if (cudaEventElapsedTime(&t, m->ev_seg[2 * q], m->ev_seg[2 * q + 1]) == cudaSuccess) ct.kernel_ms += t;
    }
  if (hrs.status == SMC_EDEGENERATE) return set_error(SMC_EDEGENERATE, "all particle weights are zero");
  if (hrs.status == SMC_ESTEPLIMIT) return set_error(SMC_ESTEPLIMIT, "max_segments reached");
  if (hrs.n_overflow || hrs.n_limit) return SMC_WKILLED;
  return SMC_OK;
}
