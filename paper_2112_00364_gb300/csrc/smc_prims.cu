// smc_prims.cu -- the resampling primitives of Section 3.3 as standalone
// HBM-streaming kernels, the particle-duplication gather, the random-number
// parity hooks, and the library's error plumbing.
//
// smc_resample (parallel systematic resampling, three launches), in the
// segment kernel's integer arithmetic (smc_combine.cuh):
//   1. rs_tile_reduce: per tile of TPB*IT weights, M_t = max, its power-of-two
//      reference k_t = ceil(M_t / ln 2), the weights round(exp(x - k_t ln 2)
//      2^50) on the integer pipes (two-table exponential), their exact tile
//      running sums E_j and total (smc_resample keeps the E_j in its
//      workspace for pass 3)
//   2. rs_combine (one CTA): k = max k_t, integer offsets O_t of the totals in
//      the common unit U, S = O_T, out3 = {k ln 2, S U 2^-k, log-Z increment},
//      and the scale N / S as a 64-bit mantissa and shift
//   3. rs_ancestors: per tile, element j owns the offsets i + u in
//      [Q_{j-1}, Q_j), Q_j = B_j N / S in 64.64 offset units, with
//      B_j = min(O_t + E_j 2^-(k - k_t + G), O_{t+1}) (the first element of a
//      tile from the previous tile's last boundary, the last element of the
//      population everything above): c_j = #{ i : i + u < Q_j } = ceil(Q_j - u).
//      Each element with a non-empty range marks its first offset in shared
//      memory; an inclusive max-scan over the marks gives every offset its
//      element, written out coalesced.  Every i is written exactly once and
//      a_i = min{ j : Q_j > i + u }, the segment kernel's rule up to the
//      rounding of N / S (below 2^-62 relative, far inside the 1e-12 band).
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

// Tiles of 4096 weights (the tile fixes each weight's rounding to 2^-50 of its
// tile's reference, so its split over threads does not change the results):
// 256 threads of 16 weights each.  (512 threads of 8 measured the same on GB300:
// 258 against 246 us per 2^24 call.)
constexpr int RS_TPB = 256;
constexpr int RS_IT = 16;
constexpr int RS_TILE = RS_TPB * RS_IT;
static_assert(RS_TILE == 4096, "the tile fixes the weights' rounding");

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
// Offsets are counted in fixed point with F = 63 - bitlen(N) fraction bits
// (N 2^F < 2^63): Q = B N / S 2^F for a boundary B in run units.
struct RsScalars {
  unsigned long long rn;  // floor(2^(64+L) N / S), in [2^63, 2^64)
  long long uF;           // floor(u 2^F)
  long long tolF;         // floor(1e-12 N 2^F)
  int32_t L, F, kmax, G, degenerate, pad_;
};

// Weights as 2^-50 fixed-point integers: a tile of 4096 sums below 2^62.
constexpr int kRsBits = 50;

// The two exponential tables of exp_fix_x2 in shared memory.
struct RsExpTab {
  unsigned long long t64[64], t4096[64];
};

__device__ __forceinline__ void stage_exp_tables(RsExpTab& st, const MathTab* tab) {
  if (threadIdx.x < 64) {
    st.t64[threadIdx.x] = tab->exp2_neg64_q63[threadIdx.x];
    st.t4096[threadIdx.x] = tab->exp2_neg4096_q63[threadIdx.x];
  }
}

// The tile's weights round(exp(x - k_t ln 2) 2^50) (k_t from the tile max).
__device__ __forceinline__ void tile_weights(const double (&v)[RS_IT], int kt, const MathTab* tab,
                                             const RsExpTab& st, long long (&ef)[RS_IT]) {
  if (kt == kDeadTile) {
#pragma unroll
    for (int q = 0; q < RS_IT; ++q) ef[q] = 0;
  } else if (kt > -2048 && kt < 2048) {
    const long long K = ref_q52(kt);
#pragma unroll
    for (int q = 0; q < RS_IT; ++q) ef[q] = weight_fix52<kRsBits>(v[q], K, st.t64, st.t4096);
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
  __shared__ RsExpTab st;
  stage_exp_tables(st, tab);
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
  tile_weights(v, kt, tab, st, E);
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

// Single CTA: combine nt tile records.  O has nt + 1 entries (O[nt] = S).  Up
// to RS_STAGE_TILES tiles the records are read once, all at a time, into shared
// memory (k_t and s_t, the offsets then formed in place and written out
// coalesced); beyond, each pass reads them again from L2.
constexpr int RS_COMBINE_TPB = 1024;
constexpr int RS_STAGE_TILES = 4096;
constexpr size_t RS_STAGE_BYTES = 8 * (RS_STAGE_TILES + 1) + 4 * RS_STAGE_TILES;

__global__ void __launch_bounds__(RS_COMBINE_TPB) rs_combine(const TileRec* __restrict__ rec, int nt,
                                                             int64_t N, double log_n, double u,
                                                             long long* __restrict__ O,
                                                             RsScalars* sc, double* out3,
                                                             const MathTab* tab) {
  __shared__ double sh[RS_COMBINE_TPB / 32 + 2 + RS_COMBINE_TPB + 1];
  extern __shared__ __align__(16) unsigned char rs_stage[];
  const bool stage = nt <= RS_STAGE_TILES;
  long long* Ow = stage ? reinterpret_cast<long long*>(rs_stage) : O;
  int* ks = stage ? reinterpret_cast<int*>(rs_stage + 8 * (RS_STAGE_TILES + 1)) : nullptr;
  const Combined c = combine_offsets<RS_COMBINE_TPB>(rec, nt, Ow, ks, sh);
  if (stage) {
    __syncthreads();  // O[nt] from thread 0
    for (int q = threadIdx.x; q <= nt; q += RS_COMBINE_TPB) O[q] = Ow[q];
  }
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
  // N / S = rn 2^-(64+L) with rn in [2^63, 2^64): S in [2^61, 2^62] has sb = 62
  // or 63 bits and N nb bits, so L = sb - nb puts N 2^(64+L) / S in (2^63, 2^65)
  // (the numerator has 64 + sb <= 127 bits); one step down when it is >= 2^64.
  const unsigned long long Su = (unsigned long long)c.S;
  const int sb = 64 - __clzll((long long)Su), nb = 64 - __clzll((long long)N);
  int L = sb - nb;
  unsigned __int128 rn = ((unsigned __int128)N << (64 + L)) / Su;
  if (rn >> 64) {
    L -= 1;
    rn = ((unsigned __int128)N << (64 + L)) / Su;
  }
  s.rn = (unsigned long long)rn;
  s.L = L;
  s.F = 63 - nb;
  s.uF = (long long)(frac64(u) >> (64 - s.F));
  s.tolF = (long long)(kBoundaryEps * (double)N * pow2i(s.F));
  s.kmax = c.kmax;
  s.G = c.G;
  *sc = s;
}

// A tile's boundaries in offset units: Q_j = min(Q(O_t) + E_j 2^-sh N / S 2^F,
// Q(O_{t+1})), Q(O) = floor(O N / S 2^F).  E_j <= s_t, so E_j 2^z with
// z = clz(s_t) keeps 64 bits, and one multiply-high by rn gives
// E_j 2^-sh N / S 2^F = umulhi(E_j 2^z, rn) 2^e, e = F - sh - L - z: within two
// units of 2^-F, monotone in E_j.
struct TileQ {
  long long q0, qcap;
  int z, e;
};

__device__ __forceinline__ long long q_of_offset(long long O, const RsScalars& sc) {
  // 64 + L - F is sb or sb + 1 (62..64): see rs_combine
  return (long long)(((unsigned __int128)(unsigned long long)O * sc.rn) >> (64 + sc.L - sc.F));
}

__device__ __forceinline__ TileQ tile_q(long long O_t, long long O_t1, const TileRec& r,
                                        const RsScalars& sc) {
  TileQ q;
  q.q0 = q_of_offset(O_t, sc);
  q.qcap = q_of_offset(O_t1, sc);
  if (r.k == kDeadTile || r.s <= 0) {
    q.z = 0;
    q.e = -64;  // no contribution
  } else {
    q.z = __clzll(r.s);
    q.e = sc.F - (sc.kmax - r.k + sc.G) - sc.L - q.z;
  }
  return q;
}

__device__ __forceinline__ long long boundary_q(long long E, const TileQ& q, const RsScalars& sc) {
  const unsigned long long m = __umul64hi((unsigned long long)E << q.z, sc.rn);
  unsigned long long c;
  if (q.e >= 0)
    c = q.e < 64 ? (m << q.e) : ~0ull;
  else
    c = q.e > -64 ? (m >> -q.e) : 0ull;
  const unsigned long long room = (unsigned long long)(q.qcap - q.q0);
  return c < room ? q.q0 + (long long)c : q.qcap;
}

// c = #{ i in [0, N) : i + u < Q 2^-F } = ceil((Q - u 2^F) 2^-F), at most N.
// Adds to *near the offsets c - 1 and c when they lie within 1e-12 N of Q.
__device__ __forceinline__ int64_t count_below(long long Q, const RsScalars& sc, int64_t N,
                                               unsigned* near) {
  const long long V = Q - sc.uF;
  if (V < 0) {  // Q below the first offset u
    if (-V < sc.tolF) ++*near;
    return 0;
  }
  const long long one = 1ll << sc.F;
  const long long f = V & (one - 1);
  const int64_t c = min((int64_t)N, (int64_t)(V >> sc.F) + (f != 0 ? 1 : 0));
  // offset c - 1 lies f below Q (a whole unit when f = 0); offset c lies
  // one - f above it (on it when f = 0)
  if (c > 0 && f != 0 && f < sc.tolF) ++*near;
  if (c < N && (f == 0 || one - f < sc.tolF)) ++*near;
  return c;
}

// Pass 3: every element's offset count c_j (above), then the tile's offsets
// [c_lo, c_end) in chunks of RS_TILE: the element j of a non-empty range
// [c_{j-1}, c_j) marks position c_{j-1} with j, an inclusive max-scan over the
// chunk (carrying the previous chunk's last element) gives each offset its
// element, and the chunk is written out coalesced.  The first element of a
// tile starts at the previous tile's last boundary; the last element of the
// population owns everything above.
//
// A slice of a population sharded over ranks runs the same kernel on its own
// tiles: x holds the slice's n_local log-weights, its first tile is tile t0 of
// the population (N = n_total particles), rec and O cover every tile of the
// population, and the ancestors of the offsets its tiles own are written at
// their global offsets; `range` (if not NULL) receives those offsets' range.
__global__ void __launch_bounds__(RS_TPB) rs_ancestors(
    const double* __restrict__ x, int64_t n_local, int t0, int64_t N,
    const TileRec* __restrict__ rec, const long long* __restrict__ O,
    const RsScalars* __restrict__ scp, const long long* __restrict__ ecache,
    int32_t* __restrict__ anc, unsigned long long* n_near, int64_t* range, const MathTab* tab) {
  __shared__ long long sh[RS_TPB / 32 + 1];
  __shared__ int sh_last[RS_TPB + 1];
  __shared__ __align__(16) int sh_m[RS_TILE];
  __shared__ RsExpTab st;
  const int tl = blockIdx.x;         // the slice's tile
  const int t = t0 + tl;             // the population's tile
  const int64_t lbase = (int64_t)tl * RS_TILE, base = (int64_t)t * RS_TILE;
  const int64_t lj0 = lbase + (int64_t)threadIdx.x * RS_IT;
  const int64_t j0 = base + (int64_t)threadIdx.x * RS_IT;
  const RsScalars sc = *scp;
  if (sc.degenerate) {  // every weight zero: identity
    for (int q = 0; q < RS_IT; ++q)
      if (lj0 + q < n_local) anc[j0 + q] = (int32_t)(j0 + q);
    if (range && tl == 0 && threadIdx.x == 0) {
      range[0] = (int64_t)t0 * RS_TILE;
      range[1] = (int64_t)t0 * RS_TILE + n_local;
    }
    return;
  }
  const TileRec r = rec[t];
  long long E[RS_IT];
  if (ecache) {
    const longlong2* p = reinterpret_cast<const longlong2*>(ecache + lj0);
#pragma unroll
    for (int q = 0; q < RS_IT / 2; ++q) {
      const longlong2 w = __ldcs(p + q);
      E[2 * q] = w.x;
      E[2 * q + 1] = w.y;
    }
  } else {
    stage_exp_tables(st, tab);
    __syncthreads();
    double v[RS_IT];
    load_tile(x, n_local, lbase, v);
    tile_weights(v, r.k, tab, st, E);
    tile_running_sums(E, sh);
  }
  const long long Ot = O[t];
  const TileQ tq = tile_q(Ot, O[t + 1], r, sc);
  unsigned near = 0;
  int c[RS_IT];
#pragma unroll
  for (int q = 0; q < RS_IT; ++q) {
    const int64_t j = j0 + q;
    c[q] = (j < N - 1) ? (int)count_below(boundary_q(E[q], tq, sc), sc, N, &near) : (int)N;
  }
  sh_last[threadIdx.x + 1] = c[RS_IT - 1];
  if (threadIdx.x == 0) {
    int64_t c0 = 0;
    if (t > 0) {  // the previous tile's last boundary
      const TileRec rp = rec[t - 1];
      unsigned dummy = 0;
      c0 = count_below(boundary_q(rp.s, tile_q(O[t - 1], Ot, rp, sc), sc), sc, N, &dummy);
    }
    sh_last[0] = (int)c0;
  }
  near = __reduce_add_sync(0xffffffffu, near);
  if ((threadIdx.x & 31) == 0 && near) atomicAdd(n_near, (unsigned long long)near);
  __syncthreads();
  const int c_prev = sh_last[threadIdx.x];  // count below this thread's first element
  const int c_lo = sh_last[0], c_end = sh_last[RS_TPB];
  if (range && threadIdx.x == 0) {
    if (tl == 0) range[0] = c_lo;
    if (tl == (int)gridDim.x - 1) range[1] = c_end;
  }
  const int jl0 = threadIdx.x * RS_IT;       // tile-local index of the first element
  int carry = -1;
  for (int cb = c_lo; cb < c_end; cb += RS_TILE) {
    int4* m4 = reinterpret_cast<int4*>(sh_m);
#pragma unroll
    for (int q = 0; q < RS_IT / 4; ++q) m4[threadIdx.x + q * RS_TPB] = make_int4(-1, -1, -1, -1);
    __syncthreads();
    int lo = c_prev;
#pragma unroll
    for (int q = 0; q < RS_IT; ++q) {
      if (lo < c[q] && lo >= cb && lo - cb < RS_TILE) sh_m[lo - cb] = jl0 + q;
      lo = c[q];
    }
    __syncthreads();
    // inclusive max-scan of the chunk: 16 consecutive marks per thread, then
    // the threads' maxima by a block scan, then the carry
    int m[RS_IT];
    const int4* mp = reinterpret_cast<const int4*>(sh_m + jl0);
#pragma unroll
    for (int q = 0; q < RS_IT / 4; ++q) {
      const int4 w = mp[q];
      m[4 * q] = w.x;
      m[4 * q + 1] = w.y;
      m[4 * q + 2] = w.z;
      m[4 * q + 3] = w.w;
    }
#pragma unroll
    for (int q = 1; q < RS_IT; ++q) m[q] = max(m[q], m[q - 1]);
    const long long run = block_incl_max_i64<RS_TPB>((long long)m[RS_IT - 1], sh);
    sh_last[threadIdx.x + 1] = (int)run;
    __syncthreads();
    // the maximum over the threads before this one and the previous chunks
    const int ex = max(carry, threadIdx.x ? sh_last[threadIdx.x] : -1);
    int4* wp = reinterpret_cast<int4*>(sh_m + jl0);
#pragma unroll
    for (int q = 0; q < RS_IT / 4; ++q)
      wp[q] = make_int4(max(m[4 * q], ex), max(m[4 * q + 1], ex), max(m[4 * q + 2], ex),
                        max(m[4 * q + 3], ex));
    __syncthreads();
    const int n_here = min(RS_TILE, c_end - cb);
    for (int k = threadIdx.x; k < n_here; k += RS_TPB) anc[cb + k] = (int32_t)(base + sh_m[k]);
    carry = max(carry, sh_last[RS_TPB]);
    __syncthreads();
  }
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
    case 10: v = (double)gamma_mt<R>(s, p1); break;
    case 11: v = (double)neg_binomial<R>(s, p1, (R)1.0, p2); break;
    default: v = (double)lomax<R>(s, p1, p2); break;
  }
  out[i] = v;
  if (blocks) blocks[i] = (int32_t)s.d;
}

__global__ void math_eval_kernel(int fn, const double* __restrict__ x, double* __restrict__ y,
                                 int64_t n, const MathTab* tab) {
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  if (fn == 22) {  // pairs (S, N) as 64-bit patterns -> the 64.64 ratio (hi, lo)
    if (i & 1) return;
    const unsigned long long n = (unsigned long long)__double_as_longlong(x[i + 1]);
    const Q64 d = n ? q_ratio((unsigned long long)__double_as_longlong(x[i]), n, ~0ull / n) : Q64{0, 0};
    y[i] = __longlong_as_double((long long)d.hi);
    y[i + 1] = __longlong_as_double((long long)d.lo);
    return;
  }
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
    case 7: y[i] = __longlong_as_double(to_fix54(tang_exp(v, tab))); break;
    case 8:
      y[i] = __longlong_as_double(exp_fix2<54>(v, tab->exp2_neg64_q63, tab->exp2_neg4096_q63));
      break;
    case 9:
      y[i] = __longlong_as_double(
          weight_fix52<50>(v, 0ll, tab->exp2_neg64_q63, tab->exp2_neg4096_q63));
      break;
    case 10: y[i] = exp_neg_int(v, tab); break;
    case 11: y[i] = (double)f32_log((float)v); break;
    case 12: y[i] = (double)f32_exp((float)v); break;
    case 13: y[i] = (double)f32_cos2pi((float)v); break;
    case 14: y[i] = (double)f32_log1p((float)v); break;
    case 15: y[i] = (double)f32_expm1((float)v); break;
    case 16: y[i] = (double)f32_lfact((int)v, tab); break;
    case 17: y[i] = (double)logf((float)v); break;
    case 18: y[i] = (double)expf((float)v); break;
    case 19: y[i] = (double)cospif(2.0f * (float)v); break;
    case 20: y[i] = (double)log1pf((float)v); break;
    default: y[i] = (double)expm1f((float)v); break;
  }
}

}  // namespace smc

using namespace smc;

extern "C" smc_status smc_math_eval(int32_t fn, const double* x, double* y, int64_t n, void* stream) {
  if (!x || !y || n < 0 || fn < 0 || fn > 22) return set_error(SMC_EINVAL, "bad argument");
  if (fn == 22 && (n & 1)) return set_error(SMC_EINVAL, "fn 22 takes pairs: n must be even");
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

// rs_combine with its staging area (above the default 48 KB of dynamic shared
// memory: the opt-in is set once per device).
std::mutex g_combine_mu;
bool g_combine_ready[128];

smc_status launch_rs_combine(const TileRec* rec, int nt, int64_t N, double u, long long* O,
                             RsScalars* sc, double* out3, const MathTab* tab, cudaStream_t cs) {
  int dev = -1;
  SMC_CUDA_TRY(cudaGetDevice(&dev));
  if (dev < 0 || dev >= 128) return set_error(SMC_EINVAL, "device ordinal %d out of range", dev);
  {
    std::lock_guard<std::mutex> lock(g_combine_mu);
    if (!g_combine_ready[dev]) {
      SMC_CUDA_TRY(cudaFuncSetAttribute(rs_combine, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                        (int)RS_STAGE_BYTES));
      g_combine_ready[dev] = true;
    }
  }
  rs_combine<<<1, RS_COMBINE_TPB, RS_STAGE_BYTES, cs>>>(rec, nt, N, std::log((double)N), u, O, sc,
                                                        out3, tab);
  SMC_CUDA_TRY(cudaGetLastError());
  return SMC_OK;
}

smc_status rs_launch(const double* logw, int64_t N, double u, int32_t* ancestors, double* out3,
                     int64_t* n_near, const RsScratch& w, cudaStream_t cs) {
  NvtxRange nv("smc_resample");
  const MathTab* tab = nullptr;
  smc_status ts = math_table(&tab);
  if (ts) return ts;
  const int nt = (int)((N + RS_TILE - 1) / RS_TILE);
  SMC_CUDA_TRY(cudaMemsetAsync(n_near, 0, sizeof(int64_t), cs));
  rs_tile_reduce<<<nt, RS_TPB, 0, cs>>>(logw, N, w.rec, w.ecache, tab);
  SMC_CUDA_TRY(cudaGetLastError());
  if ((ts = launch_rs_combine(w.rec, nt, N, u, w.O, w.sc, out3, tab, cs))) return ts;
  rs_ancestors<<<nt, RS_TPB, 0, cs>>>(logw, N, 0, N, w.rec, w.O, w.sc, w.ecache, ancestors,
                                      reinterpret_cast<unsigned long long*>(n_near), nullptr, tab);
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
// (The math tables are uploaded by math_table() on the first call of the library
// on a device that needs them, which may be this entry point's first call.)
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

// ---------------------------------------------------------------------------
// One population sharded over ranks: the same three kernels, split at the
// exchange of the tile records.  Each rank reduces its own slice (pass 1); once
// every rank holds the records of the whole population in tile order, each runs
// the combine over all of them (the same integers on every rank) and pass 3 on
// its own tiles, with its first tile's index as the offset.
extern "C" size_t smc_shard_records_bytes(int64_t n_local) {
  if (n_local < 1) return 0;
  return sizeof(TileRec) * (size_t)((n_local + RS_TILE - 1) / RS_TILE);
}

extern "C" smc_status smc_shard_reduce(const double* logw, int64_t n_local, void* records,
                                       void* stream) {
  if (!logw || !records) return set_error(SMC_EINVAL, "NULL pointer");
  if (n_local < 1 || n_local > 0x7fffffffLL) return set_error(SMC_EINVAL, "n_local must be in 1..2^31-1");
  if ((reinterpret_cast<uintptr_t>(logw) & 15) != 0)
    return set_error(SMC_EINVAL, "logw must be 16-byte aligned");
  if ((reinterpret_cast<uintptr_t>(records) & 15) != 0)
    return set_error(SMC_EINVAL, "records must be 16-byte aligned");
  const MathTab* tab = nullptr;
  smc_status ts = math_table(&tab);
  if (ts) return ts;
  NvtxRange nv("smc_shard_reduce");
  const int nt = (int)((n_local + RS_TILE - 1) / RS_TILE);
  rs_tile_reduce<<<nt, RS_TPB, 0, (cudaStream_t)stream>>>(logw, n_local, (TileRec*)records, nullptr,
                                                          tab);
  SMC_CUDA_TRY(cudaGetLastError());
  return SMC_OK;
}

extern "C" size_t smc_shard_workspace_bytes(int64_t n_total) {
  if (n_total < 1) return 0;
  const int64_t nt = (n_total + RS_TILE - 1) / RS_TILE;
  return align_up(8 * (size_t)(nt + 1), 256) + align_up(sizeof(RsScalars), 256);
}

extern "C" smc_status smc_shard_ancestors(const double* logw, int64_t n_local, int64_t first,
                                          const void* records_all, int64_t n_total, double u,
                                          int32_t* ancestors, int64_t* range, double* out3,
                                          int64_t* n_near, void* workspace,
                                          size_t workspace_bytes, void* stream) {
  smc_status st = rs_check(logw, n_total, u, ancestors, out3, n_near);
  if (st) return st;
  if (!records_all || !range || !workspace) return set_error(SMC_EINVAL, "NULL pointer");
  if (first < 0 || first % RS_TILE != 0 || n_local < 1 || first + n_local > n_total)
    return set_error(SMC_EINVAL, "the slice must start on a whole tile (%d particles) inside "
                                 "the population", RS_TILE);
  if (first + n_local < n_total && n_local % RS_TILE != 0)
    return set_error(SMC_EINVAL, "every slice but the last holds whole tiles of %d", RS_TILE);
  if (workspace_bytes < smc_shard_workspace_bytes(n_total))
    return set_error(SMC_EINVAL, "workspace too small");
  if ((reinterpret_cast<uintptr_t>(workspace) & 255) != 0)
    return set_error(SMC_EINVAL, "workspace must be 256-byte aligned");
  const MathTab* tab = nullptr;
  if ((st = math_table(&tab))) return st;
  NvtxRange nv("smc_shard_ancestors");
  cudaStream_t cs = (cudaStream_t)stream;
  const int nt_all = (int)((n_total + RS_TILE - 1) / RS_TILE);
  const int nt = (int)((n_local + RS_TILE - 1) / RS_TILE);
  char* w = (char*)workspace;
  long long* O = (long long*)w;
  RsScalars* sc = (RsScalars*)(w + align_up(8 * (size_t)(nt_all + 1), 256));
  const TileRec* rec = (const TileRec*)records_all;
  SMC_CUDA_TRY(cudaMemsetAsync(n_near, 0, sizeof(int64_t), cs));
  if ((st = launch_rs_combine(rec, nt_all, n_total, u, O, sc, out3, tab, cs))) return st;
  rs_ancestors<<<nt, RS_TPB, 0, cs>>>(logw, n_local, (int)(first / RS_TILE), n_total, rec, O, sc,
                                      nullptr, ancestors,
                                      reinterpret_cast<unsigned long long*>(n_near), range, tab);
  SMC_CUDA_TRY(cudaGetLastError());
  return SMC_OK;
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
  if (!out || n < 0 || dist < 0 || dist > 12) return set_error(SMC_EINVAL, "bad argument");
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
