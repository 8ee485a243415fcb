// smc_prims.cu -- the resampling primitives of Section 3.3 as standalone
// HBM-streaming kernels, the particle-duplication gather, the random-number
// parity hooks, and the library's error plumbing.
//
// smc_resample (parallel systematic resampling, three launches), in the
// segment kernel's integer arithmetic (smc_combine.cuh):
//   1. rs_tile_reduce: per tile of TPB*IT weights, M_t = max, its power-of-two
//      reference k_t = ceil(M_t / ln 2), the weights round(exp(x - k_t ln 2)
//      2^50) on the integer pipes, their exact tile running sums E_j and total
//      (smc_resample keeps the E_j in its workspace for pass 3)
//   2. rs_combine (one CTA): k = max k_t, integer offsets O_t of the totals in
//      the common unit U, S = O_T, out3 = {k ln 2, S U 2^-k, log-Z increment},
//      and the 64.64 fixed-point offsets' scale S / N and start u S / N
//   3. rs_ancestors: per tile, element j owns the offsets z_i = (i + u) S / N
//      in [B_{j-1}, B_j), B_j = min(O_t + E_j 2^-(k - k_t + G), O_{t+1}) (the
//      first element of a tile from the previous tile's last boundary, the last
//      element of the population everything above): the counts c_j = #{ i :
//      z_i < B_j } go to shared memory and the tile's offsets are spread over
//      the threads, each writing a_i = j found by a binary search over the
//      counts.  Every i is written exactly once and a_i = min{ j : P_j > z_i },
//      the segment kernel's rule.
#include <cuda_runtime.h>

#include <cmath>
#include <cstdarg>
#include <cstdio>
#include <cstring>
#include <mutex>

#include "smc_combine.cuh"
#include "smc_device.cuh"
#include "smc_engine.h"
#include "smc_internal.h"

namespace smc {

static thread_local char g_err[512] = "";

smc_status set_error(smc_status status, const char* fmt, ...) {
  va_list ap;
  va_start(ap, fmt);
  vsnprintf(g_err, sizeof(g_err), fmt, ap);
  va_end(ap);
  return status;
}

constexpr int RS_TPB = 256;
constexpr int RS_IT = 16;
constexpr int RS_TILE = RS_TPB * RS_IT;

__device__ __forceinline__ void load_tile(const double* __restrict__ x, int64_t N, int64_t base,
                                          double (&v)[RS_IT]) {
  const int64_t j0 = base + (int64_t)threadIdx.x * RS_IT;
  if (j0 + RS_IT <= N) {
    const double2* p = reinterpret_cast<const double2*>(x + j0);
#pragma unroll
    for (int q = 0; q < RS_IT / 2; ++q) {
      const double2 d = __ldcs(p + q);
      v[2 * q] = d.x;
      v[2 * q + 1] = d.y;
    }
  } else {
#pragma unroll
    for (int q = 0; q < RS_IT; ++q) v[q] = (j0 + q < N) ? x[j0 + q] : -INFINITY;
  }
}

// The search scalars of a population, written by rs_combine.
struct RsScalars {
  unsigned long long d_hi, d_lo, z0_hi, z0_lo;  // S / N and u S / N in 64.64 (units U)
  unsigned long long inv_d;                      // floor(2^64 N / S)
  long long tolZ;                                // 1e-12 N on the q scale, in units U
  int32_t kmax, G, degenerate, pad_;
};

// Weights as 2^-50 fixed-point integers: a tile of 4096 sums below 2^62.
constexpr int kRsBits = 50;

// The tile's weights round(exp(x - k_t ln 2) 2^50) (k_t from the tile max).
__device__ __forceinline__ void tile_weights(const double (&v)[RS_IT], int kt, const MathTab* tab,
                                             long long (&ef)[RS_IT]) {
  if (kt == kDeadTile) {
#pragma unroll
    for (int q = 0; q < RS_IT; ++q) ef[q] = 0;
  } else if (kt > -2048 && kt < 2048) {
    const __int128 K = ref_q58(kt);
#pragma unroll
    for (int q = 0; q < RS_IT; ++q) ef[q] = weight_fix<kRsBits>(v[q], K, tab);
  } else {
    const double kd = (double)kt;
#pragma unroll
    for (int q = 0; q < RS_IT; ++q)
      ef[q] = exp_fix<kRsBits>(fma(-kd, kLn2Lo, fma(-kd, kLn2Hi, v[q])), tab);
  }
}

// The tile's running sums E_j (tile-local, inclusive) of its weights: the
// thread's 16 consecutive weights in sequence, the threads by a block scan.
__device__ __forceinline__ void tile_running_sums(long long (&ef)[RS_IT], long long* sh) {
  long long loc = 0;
#pragma unroll
  for (int q = 0; q < RS_IT; ++q) {
    loc += ef[q];
    ef[q] = loc;
  }
  const long long excl = block_incl_scan_i64<RS_TPB>(loc, sh) - loc;
#pragma unroll
  for (int q = 0; q < RS_IT; ++q) ef[q] += excl;
}

// Pass 1: tile reference, weights and running sums; the tile's record; with
// `ecache` the running sums are kept for pass 3.
__global__ void __launch_bounds__(RS_TPB) rs_tile_reduce(const double* __restrict__ x, int64_t N,
                                                         TileRec* __restrict__ rec,
                                                         long long* __restrict__ ecache,
                                                         const MathTab* tab) {
  __shared__ long long sh[RS_TPB / 32 + 1];
  __shared__ int sh_k;
  double v[RS_IT];
  load_tile(x, N, (int64_t)blockIdx.x * RS_TILE, v);
  long long key = order_key(v[0]);
#pragma unroll
  for (int q = 1; q < RS_IT; ++q) key = max(key, order_key(v[q]));
  const double Mt = block_max_key<RS_TPB>(from_order_key(key), sh);
  if (threadIdx.x == 0) sh_k = Mt == -INFINITY ? kDeadTile : tile_exponent(Mt);
  __syncthreads();
  const int kt = sh_k;
  long long E[RS_IT];
  tile_weights(v, kt, tab, E);
  tile_running_sums(E, sh);
  if (ecache) {
    longlong2* p = reinterpret_cast<longlong2*>(ecache + (int64_t)blockIdx.x * RS_TILE +
                                                threadIdx.x * RS_IT);
#pragma unroll
    for (int q = 0; q < RS_IT / 2; ++q) p[q] = make_longlong2(E[2 * q], E[2 * q + 1]);
  }
  if (threadIdx.x == RS_TPB - 1) {
    TileRec r;
    r.s = E[RS_IT - 1];
    r.k = kt;
    r.alive = 0;
    rec[blockIdx.x] = r;
  }
}

// Single CTA: combine nt tile records.  O has nt + 1 entries (O[nt] = S).
__global__ void __launch_bounds__(RS_TPB) rs_combine(const TileRec* __restrict__ rec, int nt,
                                                     int64_t N, double log_n, double u,
                                                     long long* __restrict__ O, RsScalars* sc,
                                                     double* out3, const MathTab* tab) {
  __shared__ double sh[RS_TPB / 32 + 2 + RS_TPB + 1];
  const Combined c = combine_offsets<RS_TPB>(rec, nt, O, nullptr, sh);
  if (threadIdx.x != 0) return;
  RsScalars s;
  std::memset(&s, 0, sizeof(s));
  if (c.kmax == kDeadTile) {
    out3[0] = -INFINITY;
    out3[1] = 0.0;
    out3[2] = -INFINITY;
    s.degenerate = 1;
    *sc = s;
    return;
  }
  const double Sd = (double)c.S;
  out3[0] = (double)c.kmax * kLn2;
  out3[1] = Sd * pow2i(c.G - kRsBits);
  out3[2] = (double)(c.kmax - kRsBits + c.G) * kLn2 + (tang_log(Sd, tab) - log_n);
  const Q64 d = q_ratio((unsigned long long)c.S, (unsigned long long)N);
  const Q64 z0 = q_scale(frac64(u), d);
  s.d_hi = d.hi;
  s.d_lo = d.lo;
  s.z0_hi = z0.hi;
  s.z0_lo = z0.lo;
  s.inv_d = (unsigned long long)(((unsigned __int128)N << 64) / (unsigned long long)c.S);
  s.tolZ = floor_i64(kBoundaryEps * Sd);
  s.kmax = c.kmax;
  s.G = c.G;
  *sc = s;
}

// O_t + E 2^-sh in 64.64 (E >= 0 a tile running sum), capped at cap
__device__ __forceinline__ Q64 boundary(long long O_t, long long E, int sh, long long cap) {
  Q64 b;
  if (sh <= 0) {  // the run's unit is finer than the tile's: exact
    b.hi = (unsigned long long)(O_t + (E << -sh));
    b.lo = 0;
  } else if (sh < 64) {
    b.hi = (unsigned long long)(O_t + (E >> sh));
    b.lo = (unsigned long long)E << (64 - sh);
  } else {
    b.hi = (unsigned long long)O_t;
    b.lo = sh - 64 < 63 ? ((unsigned long long)E >> (sh - 64)) : 0ull;
  }
  const Q64 c{(unsigned long long)cap, 0ull};
  return q_lt(c, b) ? c : b;
}

// c = min{ i in [0, N] : z_i >= B } with z_i = z0 + i d: an estimate from the
// 0.64 reciprocal of d, then exact integer steps.  Adds to *near the offsets
// c - 1 and c when they lie within tol of B.
__device__ __forceinline__ int64_t count_below(Q64 B, Q64 z0, Q64 d, unsigned long long inv_d,
                                               int64_t N, Q64 tol, unsigned* near) {
  if (!q_lt(z0, B)) {  // z_0 >= B
    if (q_lt(q_sub(z0, B), tol)) ++*near;
    return 0;
  }
  const Q64 diff = q_sub(B, z0);
  int64_t c = (int64_t)min((unsigned long long)N, __umul64hi(diff.hi, inv_d));
  Q64 zc = q_add(z0, q_mul_u32((unsigned)c, d));  // z_c
  while (c < N && q_lt(zc, B)) {
    ++c;
    zc = q_add(zc, d);
  }
  while (c > 0 && !q_lt(q_sub(zc, d), B)) {
    --c;
    zc = q_sub(zc, d);
  }
  // here z_{c-1} < B <= z_c (when those offsets exist)
  if (c > 0 && !q_lt(tol, q_sub(B, q_sub(zc, d)))) ++*near;
  if (c < N && q_lt(q_sub(zc, B), tol)) ++*near;
  return c;
}

// Pass 3: every element's upper boundary B_j and offset count c_j = #{ i :
// z_i < B_j } into shared memory, then the tile's offsets [c_lo, c_end) spread
// over the threads, each finding its element by a binary search over the
// counts.  Element j owns [B_{j-1}, B_j); the first element of a tile starts
// at the previous tile's last boundary, the last element of the population
// owns everything above.
__global__ void __launch_bounds__(RS_TPB) rs_ancestors(
    const double* __restrict__ x, int64_t N, const TileRec* __restrict__ rec,
    const long long* __restrict__ O, const RsScalars* __restrict__ scp,
    const long long* __restrict__ ecache, int32_t* __restrict__ anc, unsigned long long* n_near,
    const MathTab* tab) {
  __shared__ long long sh[RS_TPB / 32 + 1];
  __shared__ int64_t sh_c[RS_TILE + 1];
  const int t = blockIdx.x;
  const int64_t base = (int64_t)t * RS_TILE;
  const int64_t j0 = base + (int64_t)threadIdx.x * RS_IT;
  const RsScalars sc = *scp;
  if (sc.degenerate) {  // every weight zero: identity
    for (int q = 0; q < RS_IT; ++q)
      if (j0 + q < N) anc[j0 + q] = (int32_t)(j0 + q);
    return;
  }
  const TileRec r = rec[t];
  long long E[RS_IT];
  if (ecache) {
    const longlong2* p = reinterpret_cast<const longlong2*>(ecache + j0);
#pragma unroll
    for (int q = 0; q < RS_IT / 2; ++q) {
      const longlong2 w = __ldcs(p + q);
      E[2 * q] = w.x;
      E[2 * q + 1] = w.y;
    }
  } else {
    double v[RS_IT];
    load_tile(x, N, base, v);
    tile_weights(v, r.k, tab, E);
    tile_running_sums(E, sh);
  }
  const Q64 d{sc.d_hi, sc.d_lo}, z0{sc.z0_hi, sc.z0_lo};
  const Q64 tol{(unsigned long long)sc.tolZ, 0ull};
  const long long Ot = O[t], Ot1 = O[t + 1];
  const int sh_t = r.k == kDeadTile ? 1 << 20 : sc.kmax - r.k + sc.G;
  unsigned near = 0;
#pragma unroll
  for (int q = 0; q < RS_IT; ++q) {
    const int64_t j = j0 + q;
    int64_t c = N;
    if (j < N - 1) c = count_below(boundary(Ot, E[q], sh_t, Ot1), z0, d, sc.inv_d, N, tol, &near);
    sh_c[threadIdx.x * RS_IT + q + 1] = c;
  }
  if (threadIdx.x == 0) {
    int64_t c0 = 0;
    if (t > 0) {  // the previous tile's last boundary
      const TileRec rp = rec[t - 1];
      const int shp = rp.k == kDeadTile ? 1 << 20 : sc.kmax - rp.k + sc.G;
      unsigned dummy = 0;
      c0 = count_below(boundary(O[t - 1], rp.s, shp, Ot), z0, d, sc.inv_d, N, tol, &dummy);
    }
    sh_c[0] = c0;
  }
  __syncthreads();
  const int n_el = (int)min((int64_t)RS_TILE, N - base);
  const int64_t c_lo = sh_c[0], c_end = sh_c[n_el];
  for (int64_t i = c_lo + threadIdx.x; i < c_end; i += RS_TPB) {
    int lo = 1, hi = n_el;  // first idx in [1, n_el] with sh_c[idx] > i
    while (lo < hi) {
      const int mid = (lo + hi) >> 1;
      if (sh_c[mid] > i)
        hi = mid;
      else
        lo = mid + 1;
    }
    anc[i] = (int32_t)(base + lo - 1);
  }
  near = __reduce_add_sync(0xffffffffu, near);
  if ((threadIdx.x & 31) == 0 && near) atomicAdd(n_near, (unsigned long long)near);
}

// Particle duplication: dst[f][i] = src[f][anc[i]], 16-byte stores of
// consecutive particles; with sp != NULL row f is copied only if f < sp[anc[i]].
template <typename T, int V>
__global__ void gather_kernel(const T* __restrict__ src, T* __restrict__ dst,
                              const int32_t* __restrict__ anc, const int32_t* __restrict__ sp,
                              int64_t N, int n_fields) {
  const int64_t i0 = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) * V;
  if (i0 >= N) return;
  int32_t a[V];
  int32_t s[V];
#pragma unroll
  for (int q = 0; q < V; ++q) {
    a[q] = (i0 + q < N) ? __ldg(anc + i0 + q) : 0;
    s[q] = sp ? ((i0 + q < N) ? __ldg(sp + a[q]) : 0) : n_fields;
  }
  const bool full = (i0 + V <= N) && ((reinterpret_cast<uintptr_t>(dst) & 15) == 0) && (N % V == 0);
  for (int f = 0; f < n_fields; ++f) {
    const T* sf = src + (size_t)f * N;
    T* df = dst + (size_t)f * N;
    bool all = full;
#pragma unroll
    for (int q = 0; q < V; ++q) all = all && (f < s[q]);
    if (all) {
      union {
        T e[V];
        uint4 u;
      } pk;
#pragma unroll
      for (int q = 0; q < V; ++q) pk.e[q] = __ldg(sf + a[q]);
      *reinterpret_cast<uint4*>(df + i0) = pk.u;
    } else {
#pragma unroll
      for (int q = 0; q < V; ++q)
        if (i0 + q < N && f < s[q]) df[i0 + q] = __ldg(sf + a[q]);
    }
  }
}

__global__ void philox_kernel(const uint32_t* __restrict__ ctr, const uint32_t* __restrict__ key,
                              uint32_t* __restrict__ out, int64_t n) {
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  const Block4 b = philox(ctr[4 * i], ctr[4 * i + 1], ctr[4 * i + 2], ctr[4 * i + 3], key[2 * i],
                          key[2 * i + 1]);
  out[4 * i] = b.w0;
  out[4 * i + 1] = b.w1;
  out[4 * i + 2] = b.w2;
  out[4 * i + 3] = b.w3;
}

template <typename R>
__global__ void sample_kernel(int dist, R p1, R p2, uint32_t k0, uint32_t k1, int64_t n,
                              double* __restrict__ out, int32_t* __restrict__ blocks,
                              const MathTab* tab) {
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  Stream s{k0, k1, (uint32_t)i, 0u, 0u, 0u, tab};
  double v = 0.0;
  switch (dist) {
    case 0: v = (double)uniform01<R>(s); break;
    case 1: v = (double)m_fma(p2, normal01<R>(s), p1); break;
    case 2: v = (double)exponential<R>(s, p1); break;
    case 3: v = (double)gamma1<R>(s, p1); break;
    case 4: v = (double)uniform_ab<R>(s, p1, p2); break;
    case 5: v = bernoulli<R>(s, p1) ? 1.0 : 0.0; break;
    case 6: v = (double)poisson<R>(s, p1); break;
    case 7: v = (double)lognormal<R>(s, p1); break;
    case 8: v = (double)binomial<R>(s, (int)p1, p2); break;
    case 9: v = (double)beta_ab<R>(s, p1, p2); break;
    default: v = (double)gamma_mt<R>(s, p1); break;
  }
  out[i] = v;
  if (blocks) blocks[i] = (int32_t)s.d;
}

__global__ void math_eval_kernel(int fn, const double* __restrict__ x, double* __restrict__ y,
                                 int64_t n, const MathTab* tab) {
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  const double v = x[i];
  const unsigned long long bits = (unsigned long long)__double_as_longlong(v);
  switch (fn) {
    case 0: y[i] = tang_log(v, tab); break;
    case 1: y[i] = tang_exp(v, tab); break;
    case 2: y[i] = log(v); break;
    case 3: y[i] = exp(v); break;
    case 4: y[i] = log_unif53(bits, tab); break;
    case 5: y[i] = tang_log(Unif<double>::from64(bits), tab); break;
    case 6: y[i] = __longlong_as_double(exp_fix54(v, tab)); break;
    default: y[i] = __longlong_as_double(to_fix54(tang_exp(v, tab))); break;
  }
}

}  // namespace smc

using namespace smc;

extern "C" smc_status smc_math_eval(int32_t fn, const double* x, double* y, int64_t n, void* stream) {
  if (!x || !y || n < 0 || fn < 0 || fn > 7) return set_error(SMC_EINVAL, "bad argument");
  if (n == 0) return SMC_OK;
  const MathTab* tab = nullptr;
  smc_status ts = math_table(&tab);
  if (ts) return ts;
  math_eval_kernel<<<(unsigned)((n + 255) / 256), 256, 0, (cudaStream_t)stream>>>(fn, x, y, n, tab);
  SMC_CUDA_TRY(cudaGetLastError());
  return SMC_OK;
}

extern "C" const char* smc_last_error(void) { return g_err; }

extern "C" const char* smc_version(void) { return "gb300-pcfg-smc 0.1 (sm_103a)"; }

namespace smc {
namespace {

struct RsScratch {
  TileRec* rec;       // [nt]
  long long* O;       // [nt + 1]
  RsScalars* sc;
  long long* ecache;  // [nt * RS_TILE] running sums kept from pass 1, or NULL (recomputed)
};

size_t rs_scratch_bytes(int64_t nt, bool cache) {
  return align_up(sizeof(TileRec) * (size_t)nt, 256) + align_up(8 * (size_t)(nt + 1), 256) +
         align_up(sizeof(RsScalars), 256) + (cache ? 8 * (size_t)nt * RS_TILE : 0);
}

RsScratch rs_carve(char* w, int64_t nt, bool cache) {
  RsScratch r;
  r.rec = (TileRec*)w;
  w += align_up(sizeof(TileRec) * (size_t)nt, 256);
  r.O = (long long*)w;
  w += align_up(8 * (size_t)(nt + 1), 256);
  r.sc = (RsScalars*)w;
  w += align_up(sizeof(RsScalars), 256);
  r.ecache = cache ? (long long*)w : nullptr;
  return r;
}

smc_status rs_check(const double* logw, int64_t N, double u, const int32_t* anc, const double* out3,
                    const int64_t* n_near) {
  if (!logw || !anc || !out3 || !n_near) return set_error(SMC_EINVAL, "NULL pointer");
  if (N < 1 || N > 0x7fffffffLL) return set_error(SMC_EINVAL, "N must be in 1..2^31-1");
  if (!(u > 0.0 && u < 1.0)) return set_error(SMC_EINVAL, "u must be in (0,1)");
  if ((reinterpret_cast<uintptr_t>(logw) & 15) != 0)
    return set_error(SMC_EINVAL, "logw must be 16-byte aligned");
  return SMC_OK;
}

smc_status rs_launch(const double* logw, int64_t N, double u, int32_t* ancestors, double* out3,
                     int64_t* n_near, const RsScratch& w, cudaStream_t cs) {
  const MathTab* tab = nullptr;
  smc_status ts = math_table(&tab);
  if (ts) return ts;
  const int nt = (int)((N + RS_TILE - 1) / RS_TILE);
  SMC_CUDA_TRY(cudaMemsetAsync(n_near, 0, sizeof(int64_t), cs));
  rs_tile_reduce<<<nt, RS_TPB, 0, cs>>>(logw, N, w.rec, w.ecache, tab);
  SMC_CUDA_TRY(cudaGetLastError());
  rs_combine<<<1, RS_TPB, 0, cs>>>(w.rec, nt, N, std::log((double)N), u, w.O, w.sc, out3, tab);
  SMC_CUDA_TRY(cudaGetLastError());
  rs_ancestors<<<nt, RS_TPB, 0, cs>>>(logw, N, w.rec, w.O, w.sc, w.ecache, ancestors,
                                      reinterpret_cast<unsigned long long*>(n_near), tab);
  SMC_CUDA_TRY(cudaGetLastError());
  return SMC_OK;
}

}  // namespace
}  // namespace smc

extern "C" size_t smc_resample_workspace_bytes(int64_t N) {
  if (N < 1) return 0;
  return rs_scratch_bytes((N + RS_TILE - 1) / RS_TILE, true);
}

extern "C" smc_status smc_resample(const double* logw, int64_t N, double u, int32_t* ancestors,
                                   double* out3, int64_t* n_near, void* workspace,
                                   size_t workspace_bytes, void* stream) {
  smc_status st = rs_check(logw, N, u, ancestors, out3, n_near);
  if (st) return st;
  if (!workspace) return set_error(SMC_EINVAL, "NULL pointer");
  if (workspace_bytes < smc_resample_workspace_bytes(N))
    return set_error(SMC_EINVAL, "workspace too small");
  if ((reinterpret_cast<uintptr_t>(workspace) & 255) != 0)
    return set_error(SMC_EINVAL, "workspace must be 256-byte aligned");
  return rs_launch(logw, N, u, ancestors, out3, n_near,
                   rs_carve((char*)workspace, (N + RS_TILE - 1) / RS_TILE, true), (cudaStream_t)stream);
}

// ---------------------------------------------------------------------------
// smc_resample_static: smc_resample with its scratch in a fixed device array.
//
// Some callers cannot call cudaMalloc (code whose device memory is owned by
// another framework's pool, paths where an allocation's implicit device-wide
// synchronisation is not allowed, hosts that forbid allocation after start-up).
// For them the per-tile scratch of the three resampling kernels lives in this
// file-scope array, sized for populations of up to SMC_RESAMPLE_STATIC_MAX_N
// particles (4096 tiles): 4096 tile records, 4097 offsets and the search
// scalars in 131,136 bytes that every GPU which loads the library keeps until
// the process exits.  Every call shares the array and it keeps the last call's
// contents; nothing in it has to start at zero (each call writes every entry it
// later reads), but two calls that overlap on the GPU race on it.
constexpr int kStaticTiles = (int)((SMC_RESAMPLE_STATIC_MAX_N + RS_TILE - 1) / RS_TILE);
constexpr int kStaticDoubles = 3 * kStaticTiles + (kStaticTiles + 1) + 7;
static __device__ __align__(256) double g_resample_scratch[kStaticDoubles];
static_assert(sizeof(TileRec) * kStaticTiles % 256 == 0 && (8 * (kStaticTiles + 1) + 255) / 256 * 256 +
                  sizeof(TileRec) * kStaticTiles + 256 <= sizeof(double) * kStaticDoubles,
              "the static scratch holds the tile records, offsets and scalars");

namespace {
std::mutex g_static_mu;
double* g_static_ptr[128] = {nullptr};  // device address of the array, per device

// Once per device, with that device current: resolve the array's device address.
smc_status static_scratch(double** out) {
  int dev = -1;
  SMC_CUDA_TRY(cudaGetDevice(&dev));
  if (dev < 0 || dev >= 128) return set_error(SMC_EINVAL, "device ordinal %d out of range", dev);
  std::lock_guard<std::mutex> lock(g_static_mu);
  if (!g_static_ptr[dev]) {
    void* p = nullptr;
    cudaError_t e = cudaGetSymbolAddress(&p, g_resample_scratch);
    if (e != cudaSuccess) return cuda_fail(e, "cudaGetSymbolAddress(g_resample_scratch)");
    g_static_ptr[dev] = (double*)p;
  }
  *out = g_static_ptr[dev];
  return SMC_OK;
}
}  // namespace

extern "C" smc_status smc_resample_static(const double* logw, int64_t N, double u,
                                          int32_t* ancestors, double* out3, int64_t* n_near,
                                          void* stream) {
  if (!logw || !ancestors || !out3 || !n_near) return set_error(SMC_EINVAL, "NULL pointer");
  if (N < 1) return set_error(SMC_EINVAL, "N must be >= 1");
  if (N > SMC_RESAMPLE_STATIC_MAX_N)
    return set_error(SMC_EINVAL, "N = %lld exceeds the static scratch limit of %lld particles",
                     (long long)N, (long long)SMC_RESAMPLE_STATIC_MAX_N);
  if (!(u > 0.0 && u < 1.0)) return set_error(SMC_EINVAL, "u must be in (0,1)");
  if ((reinterpret_cast<uintptr_t>(logw) & 15) != 0)
    return set_error(SMC_EINVAL, "logw must be 16-byte aligned");
  double* base = nullptr;
  smc_status st = static_scratch(&base);
  if (st) return st;
  return rs_launch(logw, N, u, ancestors, out3, n_near,
                   rs_carve((char*)base, (N + RS_TILE - 1) / RS_TILE, false), (cudaStream_t)stream);
}

extern "C" smc_status smc_gather(const void* src, void* dst, const int32_t* anc, const int32_t* sp,
                                 int64_t N, int32_t n_fields, int32_t elem_bytes, void* stream) {
  if (!src || !dst || !anc) return set_error(SMC_EINVAL, "NULL pointer");
  if (N < 1 || n_fields < 1) return set_error(SMC_EINVAL, "N and n_fields must be >= 1");
  cudaStream_t cs = (cudaStream_t)stream;
  if (elem_bytes == 8) {
    const int64_t threads = (N + 1) / 2;
    gather_kernel<double, 2><<<(unsigned)((threads + 255) / 256), 256, 0, cs>>>(
        (const double*)src, (double*)dst, anc, sp, N, n_fields);
  } else if (elem_bytes == 4) {
    const int64_t threads = (N + 3) / 4;
    gather_kernel<float, 4><<<(unsigned)((threads + 255) / 256), 256, 0, cs>>>(
        (const float*)src, (float*)dst, anc, sp, N, n_fields);
  } else {
    return set_error(SMC_EINVAL, "elem_bytes must be 4 or 8");
  }
  SMC_CUDA_TRY(cudaGetLastError());
  return SMC_OK;
}

extern "C" smc_status smc_philox(const uint32_t* ctr, const uint32_t* key, uint32_t* out, int64_t n,
                                 void* stream) {
  if (!ctr || !key || !out || n < 0) return set_error(SMC_EINVAL, "bad argument");
  if (n == 0) return SMC_OK;
  philox_kernel<<<(unsigned)((n + 255) / 256), 256, 0, (cudaStream_t)stream>>>(ctr, key, out, n);
  SMC_CUDA_TRY(cudaGetLastError());
  return SMC_OK;
}

extern "C" smc_status smc_sample(int32_t dist, int32_t precision, double p1, double p2,
                                 uint64_t seed, uint32_t run_id, int64_t n, double* out,
                                 int32_t* blocks, void* stream) {
  if (!out || n < 0 || dist < 0 || dist > 10) return set_error(SMC_EINVAL, "bad argument");
  if (n == 0) return SMC_OK;
  const uint32_t k0 = (uint32_t)(seed & 0xffffffffu), k1 = (uint32_t)(seed >> 32) ^ run_id;
  const unsigned g = (unsigned)((n + 255) / 256);
  cudaStream_t cs = (cudaStream_t)stream;
  const MathTab* tab = nullptr;
  smc_status ts = math_table(&tab);
  if (ts) return ts;
  if (precision == SMC_PREC_FP64)
    sample_kernel<double><<<g, 256, 0, cs>>>(dist, p1, p2, k0, k1, n, out, blocks, tab);
  else if (precision == SMC_PREC_FP32)
    sample_kernel<float><<<g, 256, 0, cs>>>(dist, (float)p1, (float)p2, k0, k1, n, out, blocks, tab);
  else
    return set_error(SMC_EINVAL, "unknown precision");
  SMC_CUDA_TRY(cudaGetLastError());
  return SMC_OK;
}
