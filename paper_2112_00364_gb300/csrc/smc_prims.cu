// smc_prims.cu -- the resampling primitives of Section 3.3 as standalone
// HBM-streaming kernels, the particle-duplication gather, the random-number
// parity hooks, and the library's error plumbing.
//
// smc_resample (parallel systematic resampling, three launches chained by
// programmatic dependent launch), in the segment kernel's integer arithmetic
// (smc_combine.cuh):
//   1. rs_tile_reduce (persistent): per tile of 4096 weights, the power-of-two
//      reference k_t from the largest high word of its log-weights (k_t ln 2 at
//      least 2^-19 above their maximum), the weights round(exp(x - k_t ln 2)
//      2^50) on the integer pipes (a table of e^(-j/256) in shared memory and
//      a degree-5 polynomial), their exact tile running sums E_j and total;
//      smc_resample keeps each E_j's top 32 bits, normalised by the total's
//      leading zeros, and the exact sum before every 8 elements for pass 3
//   2. rs_combine (one CTA): k = max k_t, integer offsets O_t of the totals in
//      the common unit U, S = O_T, out3 = {k ln 2, S U 2^-k, log-Z increment},
//      and the scale N / S as a 64-bit mantissa and shift
//   3. rs_ancestors: per tile, element j owns the offsets i + u in
//      [Q_{j-1}, Q_j), Q_j = B_j N / S in 64.64 offset units, with
//      B_j = min(O_t + E_j 2^-(k - k_t + G), O_{t+1}) (the first element of a
//      tile from the previous tile's last boundary, the last element of the
//      population everything above): c_j = #{ i : i + u < Q_j } = ceil(Q_j - u),
//      from one 32 x 32-bit product of E_j's top word wherever its error bound
//      decides c_j, exactly otherwise (tile_fast).  Each element with a
//      non-empty range marks its first offset in shared memory; an inclusive
//      max-scan over the marks gives every offset its element, written out
//      coalesced.  Every i is written exactly once and a_i = min{ j : Q_j > i
//      + u }, the segment kernel's rule up to the rounding of N / S (below
//      2^-62 relative, far inside the 1e-12 band).
#include <cuda_runtime.h>

#include <algorithm>
#include <climits>
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
// tile's reference, so its split over threads does not change the results).
// Pass 1 runs 512 threads of 8 weights per tile in persistent CTAs (the
// exponential's table is staged once per CTA); pass 3 runs 256 threads of 16.
constexpr int RS_TPB = 256;
constexpr int RS_IT = 16;
constexpr int RS_TILE = RS_TPB * RS_IT;
static_assert(RS_TILE == 4096, "the tile fixes the weights' rounding");
constexpr int RS1_TPB = 512;
constexpr int RS1_IT = RS_TILE / RS1_TPB;  // 8
constexpr int RS1_WARPS = RS1_TPB / 32;
constexpr size_t RS1_TABLE_BYTES = sizeof(unsigned long long) * kRsExpPad;

template <int IT>
__device__ __forceinline__ void load_run(const double* __restrict__ x, int64_t N, int64_t j0,
                                         double (&v)[IT]) {
  if (j0 + IT <= N) {
    const double2* p = reinterpret_cast<const double2*>(x + j0);
#pragma unroll
    for (int q = 0; q < IT / 2; ++q)  // issued here (a prefetch must not sink to its use)
      asm volatile("ld.global.cs.v2.f64 {%0, %1}, [%2];"
                   : "=d"(v[2 * q]), "=d"(v[2 * q + 1])
                   : "l"(p + q));
  } else {
#pragma unroll
    for (int q = 0; q < IT; ++q) v[q] = (j0 + q < N) ? x[j0 + q] : -INFINITY;
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

// ---- the weight round(e^(x - k_t ln 2) 2^50) on the integer pipes ----
// The argument X = k_t ln 2 - x >= 0 in units of 2^-52: K52 = k_t ln 2 2^52
// (rounded) minus x 2^52 (truncated toward zero) from the bits of x.  For
// |x| < 2^11 the significand m (53 bits) gives x 2^52 = m 2^11 2^-(1034 - e)
// with one right shift by s = 1034 - e >= 1 (zero from s = 64); larger |x|,
// infinities and NaN give X = 2^64 - 1 (weight 0: the caller takes this path
// only for references |k_t| < 2048, so such x lie far below it).
__device__ __forceinline__ unsigned long long rs_arg52(double x, unsigned long long K52) {
  const long long b = __double_as_longlong(x);
  const unsigned hi = (unsigned)((unsigned long long)b >> 32), lo = (unsigned)b;
  const int s = 1034 - (int)((hi >> 20) & 0x7ffu);
  const unsigned mh = (hi & 0xfffffu) | 0x100000u;
  const unsigned Mh = __funnelshift_l(lo, mh, 11), Ml = lo << 11;  // m 2^11, 64 bits
  const unsigned vh = __funnelshift_rc(Mh, 0u, (unsigned)s);       // Mh >> min(s, 32)
  unsigned vl = __funnelshift_rc(Ml, Mh, (unsigned)s);              // (Mh:Ml) >> min(s, 32)
  vl = __funnelshift_rc(vl, 0u, (unsigned)max(s - 32, 0));          // the rest past 32
  const unsigned long long v = ((unsigned long long)vh << 32) | vl;
  const unsigned long long X = b < 0 ? K52 + v : K52 - v;
  return s >= 1 ? X : ~0ull;
}

// round(e^-X 2^50) within one unit of the exact rounding, for X = X52 2^-52
// (X52 unsigned; 0 from X = 36 on).  X = j/256 + r with r < 2^-8:
// e^-X = T_j (1 - q), T_j = round(e^(-j/256) 2^56) from the table `T`, and
// q = 1 - e^-r = r - r^2/2 + r^3/6 - r^4/24 + r^5/120 in units of 2^-64 (the
// dropped r^6/720 is below 2^-57), r^2 from the top 32 bits of r and one cross
// term, the higher powers in 32-bit products; T_j q from three 32 x 32-bit
// products (the low words' product dropped: at most two units of 2^-56 short),
// and the result rounded from 2^-56 to 2^-50.
__device__ __forceinline__ long long rs_weight50(unsigned long long X52,
                                                 const unsigned long long* __restrict__ T) {
  const unsigned xh = (unsigned)(X52 >> 32), xl = (unsigned)X52;
  const unsigned j = min(xh >> 12, (unsigned)kRsExpN);
  const unsigned long long Tj = T[j];
  const unsigned long long r52 = ((unsigned long long)(xh & 0xfffu) << 32) | xl;  // r 2^52
  const unsigned rh = (unsigned)(r52 >> 12), rl = xl & 0xfffu;                     // r 2^40
  const unsigned long long rh2 = (unsigned long long)rh * rh;                      // r^2 2^80
  const unsigned t = (unsigned)(rh2 >> 32);                                         // r^2 2^48
  const unsigned long long a2 = (rh2 >> 17) + __umulhi(rh, rl << 4);  // r^2/2 2^64
  const unsigned long long a3 = ((unsigned long long)__umulhi(t, rh) * 715827883ull) >> 24;
  const unsigned v4 = __umulhi(t, t);                                               // r^4 2^64
  const unsigned a4 = __umulhi(v4, 178956971u);                                     // r^4/24 2^64
  const unsigned a5 = __umulhi(__umulhi(v4, rh), 139810u);                          // r^5/120 2^64
  const unsigned long long q = (r52 << 12) - a2 + a3 - a4 + a5;
  const unsigned Th = (unsigned)(Tj >> 32), Tl = (unsigned)Tj;
  const unsigned qh = (unsigned)(q >> 32), ql = (unsigned)q;
  const unsigned long long mid = (unsigned long long)Th * ql + (unsigned long long)Tl * qh;
  const unsigned long long tq = (unsigned long long)Th * qh + (mid >> 32);
  return (long long)((Tj - tq + 32) >> 6);
}

// A tile's weight of x for its reference exponent kt (K52 = ref_q52(kt)): the
// table exponential for |kt| < 2048, else the general one (a reference that far
// out comes only from log-weights beyond +-1400).
__device__ __forceinline__ long long rs_weight(double x, int kt, unsigned long long K52,
                                               const unsigned long long* __restrict__ T,
                                               const MathTab* tab) {
  if (kt == kDeadTile) return 0;
  if (kt > -2048 && kt < 2048) return rs_weight50(rs_arg52(x, K52), T);
  const double kd = (double)kt;
  return exp_fix<kRsBits>(fma(-kd, kLn2Lo, fma(-kd, kLn2Hi, x)), tab);
}

// Order key of a log-weight's high word: signed comparisons of keys follow the
// order of the values with their low 32 bits cleared.
__device__ __forceinline__ int hi_key(double x) {
  const int h = (int)((unsigned long long)__double_as_longlong(x) >> 32);
  return h ^ ((h >> 31) & 0x7fffffff);
}

// The tile's reference exponent from the largest high-word key: the value of
// that word is within one unit of its last place of the tile's maximum M (above
// it for M < 0, below it for M >= 0), so M_up = that value (+ one unit when it is
// >= 0) bounds M from above and k_t = ceil((M_up + 2^-30) / ln 2) puts every
// log-weight at least 2^-31 below k_t ln 2: X > 0 for every element.
__device__ __forceinline__ int tile_ref_from_key(int key) {
  if (key == hi_key(-INFINITY)) return kDeadTile;
  const int h = key ^ ((key >> 31) & 0x7fffffff);
  const double m = __longlong_as_double((long long)((unsigned long long)(unsigned)h << 32));
  const double mup = h >= 0 ? __longlong_as_double((long long)((unsigned long long)(unsigned)(h + 1) << 32)) : m;
  const double k = ceil((mup + 0x1p-30) * kInvLn2);
  if (!(k > -2147483000.0 && k < 2147483000.0)) return k > 0 ? 2147483000 : -2147483000;
  return (int)k;
}

// The same bound on the integer pipes, for |M| < 2^11 (other maxima: the FP64
// form above; `special` set): A = M_up 2^32 + 2^14 (a margin of 2^-18), and
// k_t = ceil(A / (ln 2 2^32)) from one 64 x 64-bit product with
// C = round(2^32 / ln 2), whose rounding moves the quotient by less than 2^-21:
// k_t ln 2 >= M_up + 2^-19 in every case.
__device__ __forceinline__ int tile_ref_int(int key, bool* special) {
  *special = false;
  if (key == hi_key(-INFINITY)) return kDeadTile;
  const unsigned h = (unsigned)(key ^ ((key >> 31) & 0x7fffffff));
  const int e = (int)((h >> 20) & 0x7ffu);
  if (e >= 1034) {
    *special = true;
    return 0;
  }
  const bool neg = (h >> 31) != 0;
  const unsigned long long m21 =
      (unsigned long long)((h & 0xfffffu) | (e ? 0x100000u : 0u)) + (neg ? 0u : 1u);
  const int sh = e - 1011;  // |M_up| 2^32 = m21 2^(e - 1011)
  const unsigned long long A =
      sh >= 0 ? (m21 << sh) : (sh > -64 ? (m21 >> -sh) : 0ull);
  const long long Am = (neg ? -(long long)A : (long long)A) + (1ll << 14);
  constexpr unsigned long long C = 6196328019ull;  // round(2^32 / ln 2)
  const unsigned long long a = (unsigned long long)(Am < 0 ? -Am : Am);
  const unsigned long long hi = __umul64hi(a, C), lo = a * C;
  return Am >= 0 ? (int)(hi + (lo != 0 ? 1 : 0)) : -(int)hi;
}

// One tile of pass 1 (v: its log-weights; vn receives the next tile's, t + G).
__device__ __forceinline__ void reduce_tile(const double (&v)[RS1_IT], double (&vn)[RS1_IT], int t,
                                            int p, const double* __restrict__ x, int64_t N,
                                            int nt, TileRec* __restrict__ rec,
                                            unsigned* __restrict__ ehi,
                                            long long* __restrict__ pref, const MathTab* tab,
                                            const unsigned long long* rs_T, int (*sh_key)[RS1_WARPS],
                                            long long (*sh_sum)[RS1_WARPS]) {
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
  const int tn = t + gridDim.x;
  if (tn < nt) load_run<RS1_IT>(x, N, (int64_t)tn * RS_TILE + threadIdx.x * RS1_IT, vn);
  int key = hi_key(v[0]);
#pragma unroll
  for (int q = 1; q < RS1_IT; ++q) key = max(key, hi_key(v[q]));
  key = __reduce_max_sync(0xffffffffu, key);
  if (lane == 0) sh_key[p][wid] = key;
  __syncthreads();
  int k2 = lane < RS1_WARPS ? sh_key[p][lane] : INT_MIN;
  k2 = __reduce_max_sync(0xffffffffu, k2);
  bool special;
  int kt = tile_ref_int(k2, &special);
  if (special) kt = tile_ref_from_key(k2);
  long long E[RS1_IT];
  long long loc = 0;
  if (kt > -2048 && kt < 2048) {
    const unsigned long long K52 = (unsigned long long)ref_q52(kt);
#pragma unroll
    for (int q = 0; q < RS1_IT; ++q) {
      loc += rs_weight50(rs_arg52(v[q], K52), rs_T);
      E[q] = loc;
    }
  } else {
#pragma unroll
    for (int q = 0; q < RS1_IT; ++q) {
      loc += rs_weight(v[q], kt, 0ull, rs_T, tab);
      E[q] = loc;
    }
  }
  // the threads' totals: a warp scan, the warps' totals through shared memory
  long long inc = loc;
#pragma unroll
  for (int o = 1; o < 32; o <<= 1) {
    const long long y = __shfl_up_sync(0xffffffffu, inc, o);
    if (lane >= o) inc += y;
  }
  if (lane == 31) sh_sum[p][wid] = inc;
  __syncthreads();
  long long ws = lane < RS1_WARPS ? sh_sum[p][lane] : 0;
#pragma unroll
  for (int o = 1; o < RS1_WARPS; o <<= 1) {
    const long long y = __shfl_up_sync(0xffffffffu, ws, o);
    if (lane >= o) ws += y;
  }
  const long long total = __shfl_sync(0xffffffffu, ws, RS1_WARPS - 1);
  const long long wex = wid ? __shfl_sync(0xffffffffu, ws, wid - 1) : 0;
  const long long ex = wex + inc - loc;  // the running sum before this thread's first element
  if (ehi) {
    // (E_j << z) >> 32 by one funnel shift: a live tile's total is at least
    // 2^49 (its largest weight), so z = clz(s_t) < 32 (pass 3 checks it)
    const unsigned z = total > 0 ? (unsigned)__clzll(total) : 0u;
    unsigned h[RS1_IT];
#pragma unroll
    for (int q = 0; q < RS1_IT; ++q) {
      const unsigned long long e = (unsigned long long)(E[q] + ex);
      h[q] = __funnelshift_l((unsigned)e, (unsigned)(e >> 32), z);
    }
    uint4* dst = reinterpret_cast<uint4*>(ehi + (int64_t)t * RS_TILE + threadIdx.x * RS1_IT);
    dst[0] = make_uint4(h[0], h[1], h[2], h[3]);
    dst[1] = make_uint4(h[4], h[5], h[6], h[7]);
    pref[(int64_t)t * RS1_TPB + threadIdx.x] = ex;
  }
  if (threadIdx.x == 0) {
    TileRec r;
    r.s = total;
    r.k = kt;
    r.alive = 0;
    rec[t] = r;
  }
}

// Pass 1: per tile, the reference k_t, the weights and their running sums; the
// tile's record {s_t, k_t}; with `ehi` (smc_resample) also, per element, the top
// 32 bits of its running sum normalised by the tile total's leading zeros
// (E_j << clz(s_t)) >> 32, and per thread of 8 elements the exact running sum
// before its first element, for pass 3.  Persistent: CTA b takes tiles b, b + G,
// ...; the next tile's log-weights are loaded while this one is processed.
// Launched as a programmatic dependent of the kernel
// before it: the exponential's table is staged first, the log-weights read
// only after that kernel has completed.
__global__ void __launch_bounds__(RS1_TPB, 2)
    rs_tile_reduce(const double* __restrict__ x, int64_t N, int nt, TileRec* __restrict__ rec,
                   unsigned* __restrict__ ehi, long long* __restrict__ pref, const MathTab* tab) {
  extern __shared__ __align__(16) unsigned long long rs_T[];
  __shared__ int sh_key[2][RS1_WARPS];
  __shared__ long long sh_sum[2][RS1_WARPS];
  {
    const ulonglong2* src = reinterpret_cast<const ulonglong2*>(tab->rs_exp_q56);
    ulonglong2* dst = reinterpret_cast<ulonglong2*>(rs_T);
    for (int i = threadIdx.x; i < kRsExpPad / 2; i += RS1_TPB) dst[i] = src[i];
  }
  asm volatile("griddepcontrol.wait;" ::: "memory");
  int t = blockIdx.x;
  double v[RS1_IT];
  if (t < nt) load_run<RS1_IT>(x, N, (int64_t)t * RS_TILE + threadIdx.x * RS1_IT, v);
  __syncthreads();  // the table
  for (int p = 0; t < nt; t += gridDim.x, p ^= 1) {
    double vn[RS1_IT];
    reduce_tile(v, vn, t, p, x, N, nt, rec, ehi, pref, tab, rs_T, sh_key, sh_sum);
#pragma unroll
    for (int q = 0; q < RS1_IT; ++q) v[q] = vn[q];
  }
  asm volatile("griddepcontrol.launch_dependents;" ::: "memory");
}

// Single CTA: combine nt tile records into the offsets O (nt + 1 entries,
// O[nt] = S), the log-Z increment and the search scalars.  Up to 4096 tiles
// (2^24 particles) the records are held in registers (combine_small); beyond,
// combine_offsets reads them from L2 on each of its passes.
constexpr int RS_COMBINE_TPB = 1024;

// The combine of up to 4 x RS_COMBINE_TPB tiles with every record held in
// registers: k_max, the unit exponent G and the exclusive offsets O_t by warp
// reductions and scans around three barriers -- the same integers as
// combine_offsets.
__device__ __forceinline__ Combined combine_small(const TileRec* __restrict__ rec, int nt,
                                                  long long* __restrict__ O, long long* shm,
                                                  int* shk) {
  constexpr int P = 4;
  constexpr unsigned kAll = 0xffffffffu;
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
  TileRec r[P];
  int kl = kDeadTile;
#pragma unroll
  for (int p = 0; p < P; ++p) {
    const int t = threadIdx.x * P + p;
    if (t < nt) {
      r[p] = load_rec(rec + t);
    } else {
      r[p].s = 0;
      r[p].k = kDeadTile;
      r[p].alive = 0;
    }
    kl = max(kl, r[p].k);
  }
  kl = __reduce_max_sync(kAll, kl);
  if (lane == 0) shk[wid] = kl;
  __syncthreads();
  Combined c;
  c.kmax = __reduce_max_sync(kAll, shk[lane]);
  c.alive = 0;
  c.G = 0;
  c.S = 0;
  c.ess = 0.0;
  if (c.kmax == kDeadTile) return c;
  long long bl = 0;
#pragma unroll
  for (int p = 0; p < P; ++p) bl += magnitude(r[p].s, r[p].k, c.kmax);
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) bl += __shfl_xor_sync(kAll, bl, o);
  if (lane == 0) shm[wid] = bl;
  __syncthreads();
  long long bnd = shm[lane];
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) bnd += __shfl_xor_sync(kAll, bnd, o);
  c.G = (64 - __clzll(bnd)) + 20 - 62;
  long long v[P];
  long long tot = 0;
#pragma unroll
  for (int p = 0; p < P; ++p) {
    v[p] = to_run_units(r[p].s, r[p].k, c.kmax, c.G);
    tot += v[p];
  }
  long long inc = tot;
#pragma unroll
  for (int o = 1; o < 32; o <<= 1) {
    const long long y = __shfl_up_sync(kAll, inc, o);
    if (lane >= o) inc += y;
  }
  if (lane == 31) shm[32 + wid] = inc;
  __syncthreads();
  long long ws = shm[32 + lane];
#pragma unroll
  for (int o = 1; o < 32; o <<= 1) {
    const long long y = __shfl_up_sync(kAll, ws, o);
    if (lane >= o) ws += y;
  }
  c.S = __shfl_sync(kAll, ws, 31);
  const long long before = __shfl_sync(kAll, ws, wid > 0 ? wid - 1 : 0);
  long long off = (wid > 0 ? before : 0) + inc - tot;
  long long o4[P];
#pragma unroll
  for (int p = 0; p < P; ++p) {
    o4[p] = off;
    off += v[p];
  }
  if (threadIdx.x * P + P <= nt) {
    longlong2* d = reinterpret_cast<longlong2*>(O + threadIdx.x * P);
    d[0] = make_longlong2(o4[0], o4[1]);
    d[1] = make_longlong2(o4[2], o4[3]);
  } else {
#pragma unroll
    for (int p = 0; p < P; ++p)
      if (threadIdx.x * P + p < nt) O[threadIdx.x * P + p] = o4[p];
  }
  if (threadIdx.x == 0) O[nt] = c.S;
  return c;
}

__global__ void __launch_bounds__(RS_COMBINE_TPB) rs_combine(const TileRec* __restrict__ rec, int nt,
                                                             int64_t N, double log_n, double u,
                                                             long long* __restrict__ O,
                                                             RsScalars* sc, double* out3,
                                                             const MathTab* tab) {
  __shared__ double sh[RS_COMBINE_TPB / 32 + 2 + RS_COMBINE_TPB + 1];
  asm volatile("griddepcontrol.wait;" ::: "memory");  // pass 1's records
  asm volatile("griddepcontrol.launch_dependents;" ::: "memory");
  const Combined c = nt <= 4 * RS_COMBINE_TPB
                         ? combine_small(rec, nt, O, reinterpret_cast<long long*>(sh),
                                         reinterpret_cast<int*>(sh + 64))
                         : combine_offsets<RS_COMBINE_TPB>(rec, nt, O, nullptr, sh);
  // the log-Z increment (thread 0) and the search scalars (thread 32) in parallel
  if (c.kmax == kDeadTile) {
    if (threadIdx.x == 0) {
      out3[0] = -INFINITY;
      out3[1] = 0.0;
      out3[2] = -INFINITY;
      RsScalars s;
      std::memset(&s, 0, sizeof(s));
      s.degenerate = 1;
      *sc = s;
    }
    return;
  }
  if (threadIdx.x == 0) {
    const double Sd = (double)c.S;
    out3[0] = (double)c.kmax * kLn2;
    out3[1] = Sd * pow2i(c.G - kRsBits);
    out3[2] = (double)(c.kmax - kRsBits + c.G) * kLn2 + (tang_log(Sd, tab) - log_n);
  }
  if (threadIdx.x != 32) return;
  RsScalars s;
  std::memset(&s, 0, sizeof(s));
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

// The fast form of a tile's offset counts from the top 32 bits of the
// normalised running sums (E'_hi = (E_j << z) >> 32), in units of 2^-32 offsets
// (R units; F >= 32 since N < 2^31): with P = E'_hi (rn >> 32) the exact
// m = umulhi(E_j << z, rn) lies in [P, P + 2^33 + 1], so the exact
// R = (q0 - uF + m 2^e) 2^(32-F) lies in (R~ - 1, R~ + D) with
// R~ = base + (P >> sR), base = (q0 - uF) >> (F - 32), sR = F - 32 - e and
// D = 3 + ((2^33 + 1) >> sR).  Where R~'s fraction f keeps that interval at least
// the band (tolR >= tolF 2^(32-F)) away from both integers, R~ + D lies below the
// tile's cap (qcap - uF) 2^(32-F) and the integer part I below N, the count is
// I + 1 with no near-boundary offset -- exactly what count_below(boundary_q(E_j))
// gives.  Other elements (about D / 2^32 + 2 tolR / 2^32 of them, and those
// within D of the cap) take the exact path.
struct TileFast {
  long long base, rlim;
  unsigned rnh, lo, span, ilim;
  int sR;
  bool on;
};

__device__ __forceinline__ TileFast tile_fast(const TileQ& q, const TileRec& r,
                                              const RsScalars& sc, int64_t N) {
  TileFast f;
  const int sh = sc.F - 32;
  f.sR = sc.F - 32 - q.e;
  f.rnh = (unsigned)(sc.rn >> 32);
  f.base = (q.q0 - sc.uF) >> sh;
  const long long dl = 3 + (f.sR >= 0 && f.sR < 64 ? (long long)(((1ull << 33) + 1) >> f.sR) : 0);
  const long long tolR = (sc.tolF >> sh) + 1;
  const long long span = (1ll << 32) - dl - 2 * tolR;
  f.rlim = ((q.qcap - sc.uF) >> sh) - dl;  // below it the cap cannot apply
  f.on = r.k != kDeadTile && r.s > 0 && q.z < 32 && f.sR >= 0 && f.sR < 64 && span > 0;
  if (!f.on) f.sR = 0;
  f.lo = (unsigned)(tolR + 1);
  f.span = f.on ? (unsigned)span : 0u;
  f.ilim = f.on ? (unsigned)min((long long)N, 0x7fffffffll) : 0u;
  return f;
}

// The exact running sum E_j of tile-local element jl from pass 1's running sum
// before its 8-element run and the weights of that run up to jl (the same
// integers pass 1 summed; the run's log-weights in one round of loads).
__device__ __noinline__ long long rs_exact_running_sum(const double* __restrict__ x, int64_t N,
                                                       int64_t tbase, int jl, int kt,
                                                       const long long* __restrict__ pref_tile,
                                                       const MathTab* tab) {
  const unsigned long long K52 = (kt > -2048 && kt < 2048) ? (unsigned long long)ref_q52(kt) : 0ull;
  const int r0 = jl & ~(RS1_IT - 1);
  double v[RS1_IT];
  load_run<RS1_IT>(x, N, tbase + r0, v);
  long long E = pref_tile[jl / RS1_IT];
#pragma unroll
  for (int q = 0; q < RS1_IT; ++q)
    if (r0 + q <= jl) E += rs_weight(v[q], kt, K52, tab->rs_exp_q56, tab);
  return E;
}

// Pass 3: every element's offset count c_j (above), then the tile's offsets
// [c_lo, c_end) in chunks of RS_TILE: the element j of a non-empty range
// [c_{j-1}, c_j) marks position c_{j-1} with j, an inclusive max-scan over the
// chunk (carrying the previous chunk's last element) gives each offset its
// element, and the chunk is written out coalesced.  The first element of a
// tile starts at the previous tile's last boundary; the last element of the
// population owns everything above.
//
// FAST (smc_resample): the counts from pass 1's normalised running sums
// (tile_fast), the tiles in reverse order (the last tiles pass 1 wrote are
// still in L2).  Otherwise the weights and running sums are formed again from
// the log-weights (smc_resample_static, the sharded form).
//
// A slice of a population sharded over ranks runs the recomputing form on its
// own tiles: x holds the slice's n_local log-weights, its first tile is tile t0
// of the population (N = n_total particles), rec and O cover every tile of the
// population, and the ancestors of the offsets its tiles own are written at
// their global offsets; `range` (if not NULL) receives those offsets' range.
// The shared slot of chunk position k: four ints of padding after every 32,
// so that the 16-byte reads and writes of the threads' 16 consecutive
// positions (64 bytes apart) fall in different bank groups.
__device__ __forceinline__ int mark_slot(int k) { return k + ((k >> 5) << 2); }

template <bool FAST>
__global__ void __launch_bounds__(RS_TPB, 3) rs_ancestors(
    const double* __restrict__ x, int64_t n_local, int t0, int64_t N,
    const TileRec* __restrict__ rec, const long long* __restrict__ O,
    const RsScalars* __restrict__ scp, const unsigned* __restrict__ ehi,
    const long long* __restrict__ pref, int32_t* __restrict__ anc, unsigned long long* n_near,
    int64_t* range, const MathTab* tab) {
  __shared__ long long sh[RS_TPB / 32 + 1];
  __shared__ int sh_last[RS_TPB + 1];
  __shared__ int sh_wmax[RS_TPB / 32];
  __shared__ __align__(16) int sh_m[RS_TILE + RS_TILE / 8];  // padded: mark_slot()
  asm volatile("griddepcontrol.wait;" ::: "memory");  // the combine's offsets and scalars
  const int tl = FAST ? (int)gridDim.x - 1 - (int)blockIdx.x : (int)blockIdx.x;  // the slice's tile
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
  unsigned h[RS_IT];
  if (FAST) {  // the running sums' loads first, the tile's scalars behind them
    const uint4* p = reinterpret_cast<const uint4*>(ehi + lj0);
#pragma unroll
    for (int q = 0; q < RS_IT / 4; ++q) {
      const uint4 w = __ldcs(p + q);
      h[4 * q] = w.x;
      h[4 * q + 1] = w.y;
      h[4 * q + 2] = w.z;
      h[4 * q + 3] = w.w;
    }
  }
  {  // no offset marked yet (each chunk's write loop clears what it read)
    int4* m4 = reinterpret_cast<int4*>(sh_m);
    for (int q = threadIdx.x; q < (RS_TILE + RS_TILE / 8) / 4; q += RS_TPB)
      m4[q] = make_int4(-1, -1, -1, -1);
  }
  const TileRec r = rec[t];
  const long long Ot = O[t];
  const TileQ tq = tile_q(Ot, O[t + 1], r, sc);
  unsigned near = 0;
  int c[RS_IT];
  if (FAST) {
    const TileFast tf = tile_fast(tq, r, sc, N);
#pragma unroll
    for (int q = 0; q < RS_IT; ++q) {
      const long long R = tf.base + (long long)(((unsigned long long)h[q] * tf.rnh) >> tf.sR);
      const unsigned I = (unsigned)(R >> 32), f = (unsigned)R;
      const int64_t j = j0 + q;
      if (I < tf.ilim && f - tf.lo < tf.span && R < tf.rlim && j < N - 1) {
        c[q] = (int)I + 1;
      } else if (j < N - 1) {
        const int jl = threadIdx.x * RS_IT + q;  // the tile's last running sum is its total
        const long long E = jl == RS_TILE - 1 ? r.s
                                              : rs_exact_running_sum(x, N, base, jl, r.k,
                                                                     pref + (int64_t)t * RS1_TPB, tab);
        c[q] = (int)count_below(boundary_q(E, tq, sc), sc, N, &near);
      } else {
        c[q] = (int)N;
      }
    }
  } else {
    const unsigned long long K52 =
        (r.k > -2048 && r.k < 2048) ? (unsigned long long)ref_q52(r.k) : 0ull;
    double v[RS_IT];
    load_run<RS_IT>(x, n_local, lj0, v);
    long long E[RS_IT];
    long long loc = 0;
#pragma unroll
    for (int q = 0; q < RS_IT; ++q) {
      loc += rs_weight(v[q], r.k, K52, tab->rs_exp_q56, tab);
      E[q] = loc;
    }
    const long long excl = block_incl_scan_i64<RS_TPB>(loc, sh) - loc;
#pragma unroll
    for (int q = 0; q < RS_IT; ++q) {
      const int64_t j = j0 + q;
      c[q] = (j < N - 1) ? (int)count_below(boundary_q(E[q] + excl, tq, sc), sc, N, &near) : (int)N;
    }
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
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
  int carry = -1;
  for (int cb = c_lo; cb < c_end; cb += RS_TILE) {
    int lo = c_prev;
#pragma unroll
    for (int q = 0; q < RS_IT; ++q) {
      if (lo < c[q] && lo >= cb && lo - cb < RS_TILE) sh_m[mark_slot(lo - cb)] = jl0 + q;
      lo = c[q];
    }
    __syncthreads();
    // inclusive max-scan of the chunk: 16 consecutive marks per thread, the
    // threads' maxima by warp scans and the warps' maxima, then the carry
    int m[RS_IT];
    const int4* mp = reinterpret_cast<const int4*>(sh_m + mark_slot(jl0));
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
    int run = m[RS_IT - 1];
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
      const int y = __shfl_up_sync(0xffffffffu, run, o);
      if (lane >= o) run = max(run, y);
    }
    if (lane == 31) sh_wmax[wid] = run;
    __syncthreads();
    int wx = lane < RS_TPB / 32 ? sh_wmax[lane] : -1;
#pragma unroll
    for (int o = 1; o < RS_TPB / 32; o <<= 1) {
      const int y = __shfl_up_sync(0xffffffffu, wx, o);
      if (lane >= o) wx = max(wx, y);
    }
    const int before_warp = __shfl_sync(0xffffffffu, wx, wid > 0 ? wid - 1 : 0);
    const int chunk_max = __shfl_sync(0xffffffffu, wx, RS_TPB / 32 - 1);
    const int before_lane = __shfl_up_sync(0xffffffffu, run, 1);
    // the maximum over the threads before this one and the previous chunks
    const int ex = max(carry, max(wid > 0 ? before_warp : -1, lane > 0 ? before_lane : -1));
    int4* wp = reinterpret_cast<int4*>(sh_m + mark_slot(jl0));
#pragma unroll
    for (int q = 0; q < RS_IT / 4; ++q)
      wp[q] = make_int4(max(m[4 * q], ex), max(m[4 * q + 1], ex), max(m[4 * q + 2], ex),
                        max(m[4 * q + 3], ex));
    __syncthreads();
    const int n_here = min(RS_TILE, c_end - cb);
    for (int k = threadIdx.x; k < n_here; k += RS_TPB) {
      const int m_k = mark_slot(k);
      anc[cb + k] = (int32_t)(base + sh_m[m_k]);
      sh_m[m_k] = -1;
    }
    carry = max(carry, chunk_max);
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
    case 23: y[i] = __longlong_as_double(rs_weight50(rs_arg52(v, 0ull), tab->rs_exp_q56)); break;
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
  if (!x || !y || n < 0 || fn < 0 || fn > 23) return set_error(SMC_EINVAL, "bad argument");
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
  TileRec* rec;     // [nt]
  long long* O;     // [nt + 1]
  RsScalars* sc;
  unsigned* ehi;    // [nt * RS_TILE] pass 1's normalised running sums (top 32 bits), or NULL
  long long* pref;  // [nt * RS1_TPB] pass 1's running sums before each 8-element run, or NULL
};

size_t rs_scratch_bytes(int64_t nt, bool cache) {
  return align_up(sizeof(TileRec) * (size_t)nt, 256) + align_up(8 * (size_t)(nt + 1), 256) +
         align_up(sizeof(RsScalars), 256) +
         (cache ? align_up(4 * (size_t)nt * RS_TILE, 256) + 8 * (size_t)nt * RS1_TPB : 0);
}

RsScratch rs_carve(char* w, int64_t nt, bool cache) {
  RsScratch r;
  r.rec = (TileRec*)w;
  w += align_up(sizeof(TileRec) * (size_t)nt, 256);
  r.O = (long long*)w;
  w += align_up(8 * (size_t)(nt + 1), 256);
  r.sc = (RsScalars*)w;
  w += align_up(sizeof(RsScalars), 256);
  r.ehi = cache ? (unsigned*)w : nullptr;
  if (cache) w += align_up(4 * (size_t)nt * RS_TILE, 256);
  r.pref = cache ? (long long*)w : nullptr;
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

// A launch that may begin before the kernel ahead of it in the stream has
// finished (programmatic stream serialisation): the kernels wait for it
// (griddepcontrol.wait) before they read what it wrote.
template <typename... P, typename... A>
cudaError_t launch_dependent(void (*kernel)(P...), unsigned grid, unsigned block, size_t smem,
                             cudaStream_t st, A... args) {
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = dim3(grid);
  cfg.blockDim = dim3(block);
  cfg.dynamicSmemBytes = smem;
  cfg.stream = st;
  cudaLaunchAttribute at[1];
  at[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
  at[0].val.programmaticStreamSerializationAllowed = 1;
  cfg.attrs = at;
  cfg.numAttrs = 1;
  return cudaLaunchKernelEx(&cfg, kernel, args...);
}

smc_status launch_rs_combine(const TileRec* rec, int nt, int64_t N, double u, long long* O,
                             RsScalars* sc, double* out3, const MathTab* tab, cudaStream_t cs) {
  SMC_CUDA_TRY(launch_dependent(rs_combine, 1, RS_COMBINE_TPB, 0, cs, rec, nt, N,
                                std::log((double)N), u, O, sc, out3, tab));
  return SMC_OK;
}

// Pass 1's persistent grid: as many CTAs as fit on the device at once (the
// exponential's table in dynamic shared memory, opted in once per device),
// at most one per tile.
std::mutex g_reduce_mu;
int g_reduce_ctas[128];

smc_status launch_rs_tile_reduce(const double* logw, int64_t N, TileRec* rec, unsigned* ehi,
                                 long long* pref, const MathTab* tab, cudaStream_t cs) {
  int dev = -1;
  SMC_CUDA_TRY(cudaGetDevice(&dev));
  if (dev < 0 || dev >= 128) return set_error(SMC_EINVAL, "device ordinal %d out of range", dev);
  int grid = 0;
  {
    std::lock_guard<std::mutex> lock(g_reduce_mu);
    if (!g_reduce_ctas[dev]) {
      SMC_CUDA_TRY(cudaFuncSetAttribute(rs_tile_reduce, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                        (int)RS1_TABLE_BYTES));
      int sms = 0, per_sm = 0;
      SMC_CUDA_TRY(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev));
      SMC_CUDA_TRY(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, rs_tile_reduce, RS1_TPB,
                                                                 RS1_TABLE_BYTES));
      g_reduce_ctas[dev] = std::max(1, sms * std::max(1, per_sm));
    }
    grid = g_reduce_ctas[dev];
  }
  const int nt = (int)((N + RS_TILE - 1) / RS_TILE);
  SMC_CUDA_TRY(launch_dependent(rs_tile_reduce, (unsigned)std::min(grid, nt), RS1_TPB,
                                RS1_TABLE_BYTES, cs, logw, N, nt, rec, ehi, pref, tab));
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
  if ((ts = launch_rs_tile_reduce(logw, N, w.rec, w.ehi, w.pref, tab, cs))) return ts;
  if ((ts = launch_rs_combine(w.rec, nt, N, u, w.O, w.sc, out3, tab, cs))) return ts;
  unsigned long long* nn = reinterpret_cast<unsigned long long*>(n_near);
  const unsigned* no_ehi = nullptr;
  const long long* no_pref = nullptr;
  int64_t* no_range = nullptr;
  if (w.ehi)
    SMC_CUDA_TRY(launch_dependent(rs_ancestors<true>, (unsigned)nt, RS_TPB, 0, cs, logw, N, 0, N,
                                  (const TileRec*)w.rec, (const long long*)w.O,
                                  (const RsScalars*)w.sc, (const unsigned*)w.ehi,
                                  (const long long*)w.pref, ancestors, nn, no_range, tab));
  else
    SMC_CUDA_TRY(launch_dependent(rs_ancestors<false>, (unsigned)nt, RS_TPB, 0, cs, logw, N, 0, N,
                                  (const TileRec*)w.rec, (const long long*)w.O,
                                  (const RsScalars*)w.sc, no_ehi, no_pref, ancestors, nn, no_range,
                                  tab));
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
  return launch_rs_tile_reduce(logw, n_local, (TileRec*)records, nullptr, nullptr, tab,
                               (cudaStream_t)stream);
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
  rs_ancestors<false><<<nt, RS_TPB, 0, cs>>>(logw, n_local, (int)(first / RS_TILE), n_total, rec,
                                             O, sc, nullptr, nullptr, ancestors,
                                             reinterpret_cast<unsigned long long*>(n_near), range,
                                             tab);
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
