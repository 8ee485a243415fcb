// smc_combine.cuh -- tile reductions and their combine into offsets
// (Algorithm 1 step 3: the normalising sum and the running sum of the weights
// that systematic resampling searches), in exact integer arithmetic; shared
// by the segment kernel and the standalone resampling kernels.
#pragma once
#include <cstdint>

#include "smc_device.cuh"

namespace smc {

// One tile's reduction of a segment: its running-sum total, the reference
// exponent k (kDeadTile: every weight zero) and
// whether any of its particles is still short of b_stop.  One 16-byte store.
struct __align__(16) TileRec {
  long long s;  // exact, units of 2^-54 of 2^k
  int32_t k, alive;
};

// Runs of fewer tiles than this may combine a segment's tiles in every CTA of
// the next wave (the offsets then live in shared memory); others combine in the
// last CTA of the segment.
__host__ __device__ constexpr int redundant_cap(int tpb) { return 4 * tpb > 512 ? 4 * tpb : 512; }

// A tile record written by another CTA of the previous segment (one 16-byte
// load at L2, past the L1).
__device__ __forceinline__ TileRec load_rec(const TileRec* p) {
  const longlong2 v = __ldcg(reinterpret_cast<const longlong2*>(p));
  TileRec r;
  r.s = v.x;
  r.k = (int32_t)(v.y & 0xffffffffll);
  r.alive = (int32_t)(v.y >> 32);
  return r;
}

// ---------------------------------------------------------------------------
// Offsets.  A tile's record holds its exact running-sum total s_t in units of
// 2^-B of its reference 2^k_t (B = 54 in the segment kernel).  The combine of a
// segment brings every total to the run's reference 2^k_max and one common
// unit U = 2^(k_max - B + G): v_t = round(s_t 2^-(k_max - k_t + G)) (a left
// shift where that exponent is negative).  G is chosen from the totals'
// magnitudes so that S = sum v_t lies in [2^61, 2^62]: the offsets
// O_t = sum_{t' < t} v_t' and S = O_T are then exact integers, non-decreasing
// by construction and the same in whatever order they are summed, and the
// rounding of the totals (at most half a unit each) leaves S within
// n_tiles 2^-62 of the exact sum of the weights.
// ---------------------------------------------------------------------------

// floor(x) as int64 for finite x >= 0 (LLONG_MAX from 2^63 up); -1 for x < 0.
__device__ __forceinline__ long long floor_i64(double x) {
  const long long b = __double_as_longlong(x);
  if ((b & 0x7FFFFFFFFFFFFFFFll) == 0) return 0;
  if (b < 0) return -1;
  const int e = (int)(b >> 52);
  if (e < 1023) return 0;
  if (e >= 1023 + 63) return 0x7FFFFFFFFFFFFFFFll;
  const long long m = (b & 0x000FFFFFFFFFFFFFll) | 0x0010000000000000ll;
  const int sh = e - 1075;  // x = m 2^sh
  return sh >= 0 ? (m << sh) : (m >> -sh);
}

// x 2^sh for x >= 0 (a right shift for sh < 0), saturating at LLONG_MAX
__device__ __forceinline__ long long shl_sat(long long x, int sh) {
  if (x == 0) return 0;
  if (sh < 0) return -sh >= 63 ? 0 : (x >> -sh);
  if (sh >= 63 || x > (0x7FFFFFFFFFFFFFFFll >> sh)) return 0x7FFFFFFFFFFFFFFFll;
  return x << sh;
}

// the tile total in the run's unit U: round(s 2^-(k_max - k_t + G))
__device__ __forceinline__ long long to_run_units(long long s, int kt, int kmax, int G) {
  if (kt == kDeadTile) return 0;
  const int sh = kmax - kt + G;
  if (sh >= 63) return 0;
  if (sh <= 0) return s << -sh;  // G keeps the result below 2^62
  return (s + (1ll << (sh - 1))) >> sh;
}

// a tile's total in units of 2^20 U at G = 0 (truncated; the bound adds one)
__device__ __forceinline__ long long magnitude(long long s, int kt, int kmax) {
  if (kt == kDeadTile) return 0;
  const int sh = kmax - kt + 20;
  return (sh >= 63 ? 0 : (s >> sh)) + 1;
}

struct Combined {
  long long S;  // total in units U
  int kmax, G, alive;
  double ess;   // (sum w)^2 / sum w^2 when the squared sums were given, else 0
};

// Combine n_tiles tile records into the offsets O[0..nt] (O[nt] = S).  With
// `ks` non-NULL the records are first staged in shared memory (k_t into ks,
// s_t into O, which the offsets then overwrite); otherwise they are read from
// `rec` on each pass.  Every thread of the CTA calls it; all integer work.
// With `q` (the tiles' sums of squared weights) non-NULL the effective sample
// size is formed too, in FP64 by the first warp: sum w^2 relative to 2^(2 k_max).
template <int TPB>
__device__ Combined combine_offsets(const TileRec* rec, int nt, long long* O, int* ks, double* sh,
                                    const long long* q = nullptr) {
  constexpr int P = 4;  // consecutive tiles per thread per chunk
  constexpr int W = TPB / 32;
  constexpr unsigned kAll = 0xffffffffu;
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
  // disjoint shared regions, one per reduction, so none needs a barrier before reuse
  int* sk = reinterpret_cast<int*>(sh);                     // [2W] warps' (k max, alive)
  long long* sm = reinterpret_cast<long long*>(sh) + W;     // [W] warps' magnitude sums
  long long* ss = reinterpret_cast<long long*>(sh) + 2 * W;  // [W] warps' unit totals
  double* qs = sh + 3 * W;                                   // [1] effective sample size
  int kl = kDeadTile, al = 0;
  for (int t = threadIdx.x; t < nt; t += TPB) {
    const TileRec r = load_rec(rec + t);
    if (ks) {
      ks[t] = r.k;
      O[t] = r.s;
    }
    kl = max(kl, r.k);
    al |= r.alive;
  }
  kl = __reduce_max_sync(kAll, kl);
  al = (int)__reduce_or_sync(kAll, (unsigned)al);
  if (lane == 0) {
    sk[2 * wid] = kl;
    sk[2 * wid + 1] = al;
  }
  __syncthreads();
  Combined c;
  c.kmax = sk[0];
  c.alive = sk[1];
#pragma unroll
  for (int w = 1; w < W; ++w) {
    c.kmax = max(c.kmax, sk[2 * w]);
    c.alive |= sk[2 * w + 1];
  }
  c.alive = c.alive ? 1 : 0;
  c.G = 0;
  c.S = 0;
  c.ess = 0.0;
  if (c.kmax == kDeadTile) {
    __syncthreads();
    return c;
  }
  // G from b = sum over live tiles of (floor(s_t 2^-(k_max - k_t + 20)) + 1),
  // which lies between the exact sum T of the totals in units of 2^20 U (at
  // G = 0) and T + n_tiles: G = bitlen(b) - 42 gives 2^(41+G) <= b < 2^(42+G),
  // so S = sum v_t is within [2^61 - n_tiles 2^(20-G), 2^62 + n_tiles].  (With
  // ks each thread reads back the tiles it staged itself.)
  long long bl = 0;
  for (int t = threadIdx.x; t < nt; t += TPB) {
    if (ks)
      bl += magnitude(O[t], ks[t], c.kmax);
    else {
      const TileRec r = load_rec(rec + t);
      bl += magnitude(r.s, r.k, c.kmax);
    }
  }
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) bl += __shfl_xor_sync(kAll, bl, o);
  if (lane == 0) sm[wid] = bl;
  __syncthreads();
  long long bnd = sm[0];
#pragma unroll
  for (int w = 1; w < W; ++w) bnd += sm[w];
  c.G = (64 - __clzll(bnd)) + 20 - 62;
  // the totals in units U and their exclusive prefix sums, P consecutive tiles
  // a thread, chunk by chunk
  long long carry = 0;
  for (int base = 0; base < nt; base += TPB * P) {
    long long v[P];
    long long tot = 0;
#pragma unroll
    for (int p = 0; p < P; ++p) {
      const int t = base + threadIdx.x * P + p;
      v[p] = 0;
      if (t < nt) {
        long long st;
        int kt;
        if (ks) {
          st = O[t];
          kt = ks[t];
        } else {
          const TileRec r = load_rec(rec + t);
          st = r.s;
          kt = r.k;
        }
        v[p] = to_run_units(st, kt, c.kmax, c.G);
      }
      tot += v[p];
    }
    long long inc = tot;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
      const long long y = __shfl_up_sync(kAll, inc, o);
      if (lane >= o) inc += y;
    }
    if (lane == 31) ss[wid] = inc;
    __syncthreads();
    long long off = carry + (inc - tot), all = 0;
#pragma unroll
    for (int w = 0; w < W; ++w) {
      const long long x = ss[w];
      if (w < wid) off += x;
      all += x;
    }
#pragma unroll
    for (int p = 0; p < P; ++p) {
      const int t = base + threadIdx.x * P + p;
      if (t < nt) O[t] = off;
      off += v[p];
    }
    carry += all;
    if (base + TPB * P < nt) __syncthreads();  // every thread has read ss
  }
  c.S = carry;
  if (threadIdx.x == 0) O[nt] = carry;
  if (q && wid == 0) {  // sum w^2 relative to 2^(2 k_max), in FP64, by the first warp
    double acc = 0.0;
    for (int t = lane; t < nt; t += 32) {
      const int kt = ks ? ks[t] : load_rec(rec + t).k;
      if (kt != kDeadTile) {
        const int d2 = 2 * (c.kmax - kt);
        if (d2 < 900) acc = acc + (double)__ldcg(q + t) * pow2i(-54 - d2);
      }
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) acc = acc + __shfl_xor_sync(kAll, acc, o);
    if (lane == 0) {
      const double sd = (double)carry * pow2i(c.G - 54);
      qs[0] = acc > 0.0 ? (sd * sd) / acc : 0.0;
    }
  }
  __syncthreads();  // the offsets (and the ESS) for every thread
  if (q) c.ess = qs[0];
  return c;
}

// ---- 64.64 fixed-point positions on the offsets' scale ----
// The systematic offsets i + u scaled to the P scale: z_i = (i + u) S / N in
// units U, as an unsigned integer part and a 2^-64 fraction.  z_i = z_0 + i d
// with d = S / N and z_0 = u d, both truncated once; z_i is then exact and
// non-decreasing in i.
struct Q64 {
  unsigned long long hi, lo;  // hi + lo 2^-64
};

__device__ __forceinline__ Q64 q_add(Q64 a, Q64 b) {
  Q64 r;
  r.lo = a.lo + b.lo;
  r.hi = a.hi + b.hi + (r.lo < a.lo ? 1ull : 0ull);
  return r;
}

// a - b for a >= b
__device__ __forceinline__ Q64 q_sub(Q64 a, Q64 b) {
  Q64 r;
  r.lo = a.lo - b.lo;
  r.hi = a.hi - b.hi - (a.lo < b.lo ? 1ull : 0ull);
  return r;
}

__device__ __forceinline__ bool q_lt(Q64 a, Q64 b) { return a.hi < b.hi || (a.hi == b.hi && a.lo < b.lo); }

// One digit of a long division in base 2^32: floor(num / N) and the remainder
// for num < N 2^32 and 1 <= N < 2^31, from the per-run reciprocal
// R = floor((2^64 - 1) / N).  2^64 / N - R < 2, so num R 2^-64 lies within one
// below num / N (num < 2^63) and its integer part is the digit or one less; one
// correction step makes it exact.  Integer pipes only.
__device__ __forceinline__ unsigned long long div_digit(unsigned long long num, unsigned long long N,
                                                        unsigned long long R,
                                                        unsigned long long* rem) {
  unsigned long long q = __umul64hi(num, R);
  unsigned long long r = num - q * N;
  if (r >= N) {
    q += 1;
    r -= N;
  }
  *rem = r;
  return q;
}

// S / N in 64.64 fixed point, floor(S 2^64 / N) exactly, for S < 2^63 and
// 1 <= N < 2^31: four base-2^32 digits (two of the integer part, two of the
// fraction), no division instruction.  R = floor((2^64 - 1) / N).
__device__ __forceinline__ Q64 q_ratio(unsigned long long S, unsigned long long N,
                                       unsigned long long R) {
  unsigned long long r;
  const unsigned long long q1 = div_digit(S >> 32, N, R, &r);
  const unsigned long long q2 = div_digit((r << 32) | (S & 0xffffffffull), N, R, &r);
  const unsigned long long q3 = div_digit(r << 32, N, R, &r);
  const unsigned long long q4 = div_digit(r << 32, N, R, &r);
  Q64 d;
  d.hi = (q1 << 32) + q2;
  d.lo = (q3 << 32) + q4;
  return d;
}

// floor(u 2^64) for 0 <= u < 1
__device__ __forceinline__ unsigned long long frac64(double u) {
  const long long b = __double_as_longlong(u);
  const int e = (int)(b >> 52);
  if (b <= 0 || e == 0) return 0;
  const unsigned long long m = (unsigned long long)((b & 0x000FFFFFFFFFFFFFll) | 0x0010000000000000ll);
  const int sh = e - 1075 + 64;  // u 2^64 = m 2^sh, sh <= 63 for u < 1
  return sh >= 0 ? (m << sh) : (-sh < 64 ? (m >> -sh) : 0ull);
}

// f d for a 0.64 fraction f and d in 64.64 (truncated)
__device__ __forceinline__ Q64 q_scale(unsigned long long f, Q64 d) {
  Q64 r;
  const unsigned long long a_hi = __umul64hi(f, d.hi), a_lo = f * d.hi;
  r.lo = a_lo + __umul64hi(f, d.lo);
  r.hi = a_hi + (r.lo < a_lo ? 1ull : 0ull);
  return r;
}

// i d (exact, i < 2^32)
__device__ __forceinline__ Q64 q_mul_u32(unsigned i, Q64 d) {
  Q64 r;
  r.lo = (unsigned long long)i * d.lo;
  r.hi = (unsigned long long)i * d.hi + __umul64hi((unsigned long long)i, d.lo);
  return r;
}

// floor((z - O) 2^sh) as int64 for z >= O (saturating), O an integer offset
__device__ __forceinline__ long long q_threshold(Q64 z, long long O, int sh) {
  const unsigned long long ip = z.hi - (unsigned long long)O;
  if (sh < 0) return -sh >= 64 ? 0 : (long long)(ip >> -sh);
  if (sh == 0) return (long long)ip;
  if (sh >= 63 || ip > (0x7FFFFFFFFFFFFFFFull >> sh)) return 0x7FFFFFFFFFFFFFFFll;
  return (long long)((ip << sh) | (z.lo >> (64 - sh)));
}

}  // namespace smc
