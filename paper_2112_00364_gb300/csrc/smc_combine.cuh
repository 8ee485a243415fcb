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
  int* shi = reinterpret_cast<int*>(sh);
  long long* shl = reinterpret_cast<long long*>(sh);
  int kl = kDeadTile, al = 0;
  for (int q = threadIdx.x; q < nt; q += TPB) {
    const TileRec r = load_rec(rec + q);
    if (ks) {
      ks[q] = r.k;
      O[q] = r.s;
    }
    kl = max(kl, r.k);
    al |= r.alive;
  }
  Combined c;
  c.kmax = block_max_int<TPB>(kl, shi);
  c.alive = __syncthreads_or(al);
  c.G = 0;
  c.S = 0;
  c.ess = 0.0;
  if (c.kmax == kDeadTile) return c;
  // G from b = sum over live tiles of (floor(s_t 2^-(k_max - k_t + 20)) + 1),
  // which lies between the exact sum T of the totals in units of 2^20 U (at
  // G = 0) and T + n_tiles: G = bitlen(b) - 42 gives 2^(41+G) <= b < 2^(42+G),
  // so S = sum v_t is within [2^61 - n_tiles 2^(20-G), 2^62 + n_tiles]
  long long bl = 0;
  for (int q = threadIdx.x; q < nt; q += TPB) {
    if (ks)
      bl += magnitude(O[q], ks[q], c.kmax);
    else {
      const TileRec r = load_rec(rec + q);
      bl += magnitude(r.s, r.k, c.kmax);
    }
  }
  const long long bsum = block_incl_scan_i64<TPB>(bl, shl);
  __syncthreads();
  if (threadIdx.x == TPB - 1) shl[0] = bsum;
  __syncthreads();
  const long long bnd = shl[0];
  __syncthreads();
  c.G = (64 - __clzll(bnd)) + 20 - 62;
  long long carry = 0;
  for (int base = 0; base < nt; base += TPB * P) {
    long long v[P];
    long long tot = 0;
#pragma unroll
    for (int q = 0; q < P; ++q) {
      const int t = base + threadIdx.x * P + q;
      v[q] = 0;
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
        v[q] = to_run_units(st, kt, c.kmax, c.G);
      }
      tot += v[q];
    }
    const long long incl = block_incl_scan_i64<TPB>(tot, shl);
    long long off = carry + (incl - tot);
#pragma unroll
    for (int q = 0; q < P; ++q) {
      const int t = base + threadIdx.x * P + q;
      if (t < nt) O[t] = off;
      off += v[q];
    }
    __syncthreads();
    if (threadIdx.x == TPB - 1) shl[0] = incl;
    __syncthreads();
    carry += shl[0];
    __syncthreads();
  }
  c.S = carry;
  if (threadIdx.x == 0) O[nt] = carry;
  if (q) {
    double* qs = sh + TPB / 32 + 1;
    if (threadIdx.x < 32) {
      double acc = 0.0;
      for (int t = threadIdx.x; t < nt; t += 32) {
        const int kt = ks ? ks[t] : load_rec(rec + t).k;
        const int d2 = 2 * (c.kmax - kt);
        if (kt != kDeadTile && d2 < 900) acc = acc + (double)__ldcg(q + t) * pow2i(-54 - d2);
      }
#pragma unroll
      for (int o = 16; o > 0; o >>= 1) acc = acc + __shfl_xor_sync(0xffffffffu, acc, o);
      if (threadIdx.x == 0) {
        const double s = (double)carry * pow2i(c.G - 54);
        qs[0] = acc > 0.0 ? (s * s) / acc : 0.0;
      }
    }
    __syncthreads();
    c.ess = qs[0];
  }
  __syncthreads();
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

// S / N in 64.64 (S < 2^63, N >= 1)
// One digit of a long division in base 2^32: floor(num / N) and the remainder
// for num < N 2^32 and 1 <= N < 2^31.  The FP64 product num (1/N) carries three
// roundings of relative size 2^-53 on a quotient below 2^32, so it lies within
// 2^-19 of num / N and its truncation within one of the digit; one correction
// step each way makes it exact.
__device__ __forceinline__ unsigned long long div_digit(unsigned long long num, long long N,
                                                        double inv, unsigned long long* rem) {
  long long q = (long long)((double)(long long)num * inv);
  long long r = (long long)num - q * N;
  if (r < 0) {
    q -= 1;
    r += N;
  } else if (r >= N) {
    q += 1;
    r -= N;
  }
  *rem = (unsigned long long)r;
  return (unsigned long long)q;
}

// S / N in 64.64 fixed point, floor(S 2^64 / N) exactly, for S < 2^63 and
// 1 <= N < 2^31: four base-2^32 digits (two of the integer part, two of the
// fraction), no 128-bit division.  inv = 1 / N rounded to nearest.
__device__ __forceinline__ Q64 q_ratio(unsigned long long S, unsigned long long N, double inv) {
  const long long n = (long long)N;
  unsigned long long r;
  const unsigned long long q1 = div_digit(S >> 32, n, inv, &r);
  const unsigned long long q2 = div_digit((r << 32) | (S & 0xffffffffull), n, inv, &r);
  const unsigned long long q3 = div_digit(r << 32, n, inv, &r);
  const unsigned long long q4 = div_digit(r << 32, n, inv, &r);
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
