// smc_device.cuh -- device building blocks of the particle-SMC engine:
// counter-based random numbers, the variate recipes used by SAMPLE, the
// table-driven and integer-pipe logarithms and exponentials they and the
// normaliser use (GB300 runs FP64 at 2 DFMA per clock per SM, so the hot path
// does what it can on the integer pipes), and the integer warp / block
// reductions and scans of the normaliser and the search.
//
// Random numbers (Section 3.3 gives each particle its own seed; here the
// generator is counter-based so no per-particle RNG state exists at all):
// Philox4x32-10 (Salmon, Moraes, Dror, Shaw, SC'11), key
// (seed_lo32, seed_hi32 ^ run_id), counter (particle slot n, checkpoint index
// k, draw index d, tag) with tag 0 = model draws, 1 = resampling uniform,
// 2 = rate-shift multipliers.  One 128-bit block per variate.
//
// The library is compiled with -fmad=false: an expression a*b+c below is two
// roundings; a fused multiply-add is always written as fma().
#pragma once
#include <cstdint>
#include <math.h>

namespace smc {

constexpr int PC_STOP = -1;
constexpr double kLn2 = 0.69314718055994530942;
constexpr float kLn2f = 0.693147182f;
constexpr double kTwoPi = 6.28318530717958647692;
constexpr float kTwoPif = 6.28318548f;
constexpr double kBoundaryEps = 1e-12;
constexpr double kInvLn2 = 1.44269504088896340736;
constexpr int kDeadTile = -2147483647 - 1;  // tile whose weights are all zero

// Exact 2^n for n in [-1022, 1023] assembled from bits; 0 below.
__device__ __forceinline__ double pow2i(int n) {
  if (n < -1022) return 0.0;
  return __longlong_as_double((long long)(n + 1023) << 52);
}

// Power-of-two reference of a tile: k = ceil(M / ln 2) (M finite), so that the
// tile's weights exp(logw - k ln 2) are at most ~1 and tiles are rescaled by the
// exact factors 2^(k_t - k_max) instead of exponentials.
__device__ __forceinline__ int tile_exponent(double M) { return (int)ceil(M * kInvLn2); }

struct Block4 {
  uint32_t w0, w1, w2, w3;
};

__host__ __device__ __forceinline__ uint32_t mulhi32(uint32_t a, uint32_t b) {
#ifdef __CUDA_ARCH__
  return __umulhi(a, b);
#else
  return (uint32_t)(((uint64_t)a * (uint64_t)b) >> 32);
#endif
}

// Philox4x32 with 10 rounds: each round multiplies counter words 0 and 2 by
// the two round constants, swaps and xors in the key; the key is bumped by
// the two Weyl constants between rounds.
__host__ __device__ __forceinline__ Block4 philox(uint32_t c0, uint32_t c1, uint32_t c2,
                                                  uint32_t c3, uint32_t k0, uint32_t k1) {
#pragma unroll
  for (int r = 0; r < 10; ++r) {
    if (r > 0) {
      k0 += 0x9E3779B9u;
      k1 += 0xBB67AE85u;
    }
    const uint32_t lo0 = 0xD2511F53u * c0, hi0 = mulhi32(0xD2511F53u, c0);
    const uint32_t lo1 = 0xCD9E8D57u * c2, hi1 = mulhi32(0xCD9E8D57u, c2);
    const uint32_t n0 = hi1 ^ c1 ^ k0;
    const uint32_t n2 = hi0 ^ c3 ^ k1;
    c0 = n0;
    c1 = lo1;
    c2 = n2;
    c3 = lo0;
  }
  return Block4{c0, c1, c2, c3};
}

// ---- table-driven FP64 logarithm and exponential ----
// GB300 executes FP64 at 2 DFMA/clk/SM with ~64 cycles of dependent latency, so
// the length of a dependency chain, not its op count alone, decides how long a
// straggling particle takes.  These follow Tang's table-driven method (ACM TOMS
// 15(2) 1989 for exp, 16(4) 1990 for log): reduce the argument with a small
// table so that a short Taylor polynomial, evaluated in Estrin form, finishes
// the job in ~8 dependent operations.  Both are within ~2 ulp of the correctly
// rounded result; special and extreme arguments go to the library functions.
constexpr int kRsExpN = 36 * 256;      // table points of e^(-j/256), j < kRsExpN
constexpr int kRsExpPad = kRsExpN + 4;  // then zeros (whole 16-byte pairs)
struct MathTab {
  double log_f[192];    // log(j/128), j = 90..181 used
  double inv_f[192];    // 128 / j, j = 90..181 used
  double inv_f52[192];  // (128 / j) 2^-52 (exact scaling of inv_f)
  double inv_f53[192];  // (128 / j) 2^-53
  unsigned long long exp2_neg_q63[128];  // round(2^(-j/128) 2^63)
  unsigned long long inv_f_q62[192];        // round((128 / j) 2^62), j = 90..181 used
  unsigned long long exp2_neg64_q63[64];    // round(2^(-j/64) 2^63)
  unsigned long long exp2_neg4096_q63[64];  // round(2^(-j/4096) 2^63)
  double lfact[32];                      // log k!, k < 32 (sums of logs in order)
  double exp2_j[32];    // 2^(j/32)
  double inv_int[256];  // 1 / k (entry 0 unused)
  // The standalone resampler's exponential: round(e^(-j/256) 2^56) for
  // j < kRsExpN, zero from there on (e^-36 2^50 < 1/2: the weights past it round
  // to zero).
  __align__(16) unsigned long long rs_exp_q56[kRsExpPad];
};

constexpr double kLn2Hi = 0x1.62e42fefa3800p-1;   // ln 2 to 42 bits: e * kLn2Hi exact, |e| < 2^11
constexpr double kLn2Lo = 0x1.ef35793c76730p-45;  // ln 2 - kLn2Hi
constexpr double kLn2by32Hi = 0x1.62e42fefa0000p-6;   // ln 2 / 32 to 37 bits
constexpr double kLn2by32Lo = 0x1.cf79abc9e3b3ap-45;  // ln 2 / 32 - kLn2by32Hi
constexpr double kInvLn2x32 = 0x1.71547652b82fep+5;   // 32 / ln 2

// log x = e ln 2 + log F + log1p(u) with x = 2^e m, m in [sqrt(2)/2, sqrt(2))
// (so that e = 0 around 1), F = j/128 the table point nearest to m (j = 91..181,
// so F = 1 near 1 and log F and log1p(u) never cancel by more than a bit),
// u = (m - F) / F in (-1/180, 1/180); log1p(u) = u - u^2 q(u) with the Taylor
// series of q to degree 6 (truncation < 1e-18 relative).
__device__ __forceinline__ double tang_log_tail(double u, int j, int e, const MathTab* __restrict__ T) {
  const double u2 = u * u;
  const double u4 = u2 * u2;
  const double qa = fma(u, -1.0 / 3.0, 0.5);
  const double qb = fma(u, -0.2, 0.25);
  const double qc = fma(u, -1.0 / 7.0, 1.0 / 6.0);
  const double q = fma(fma(u2, 0.125, qc), u4, fma(qb, u2, qa));
  const double p = fma(-u2, q, u);
  const double de = (double)e;
  const double hi = fma(de, kLn2Hi, __ldg(&T->log_f[j]));
  return hi + fma(de, kLn2Lo, p);
}

__device__ __forceinline__ double tang_log(double x, const MathTab* __restrict__ T) {
  if (!(x >= 0x1p-1022 && x < INFINITY)) return log(x);
  const long long b = __double_as_longlong(x);
  int e = (int)(b >> 52) - 1023;
  double m = __longlong_as_double((b & 0x000FFFFFFFFFFFFFll) | 0x3FF0000000000000ll);
  if (m >= 1.4142135623730951) {
    m = 0.5 * m;  // exact
    e += 1;
  }
  const int j = (int)(m * 128.0 + 0.5);     // nearest table point (both steps exact)
  const double F = (double)j * 0x1p-7;      // exact
  const double u = (m - F) * __ldg(&T->inv_f[j]);  // m - F is exact
  return tang_log_tail(u, j, e, T);
}

// log u for the FP64 uniform u = ((x >> 11) | 1) 2^-53 of 64 random bits x,
// with tang_log's reduction done on the integer pipes: the significand
// n = (x >> 11) | 1 gives the exponent (leading-zero count), the halving test,
// the table point j and the exact difference m - F as an integer, so that
// v = (m - F) / F is one conversion and one product.  log1p(v) = v - v^2 q(v)
// with q(v) = 1/2 - v/3 + v^2 (1/4 - v/5 + v^2 (1/6 - v/7 + v^2/8)) evaluated
// in signed 2^-62 fixed point from v in 2^-64 fixed point (|v| < 2^-7.49; q
// needs only 2^-46.5 relative accuracy, the remaining error being v^2 times
// it), then converted exactly to a double: the FP64 pipe only forms v, v^2,
// v - v^2 q and the e ln 2 + log F combination.  Within 2 ulp of log u.
__device__ __forceinline__ double log_unif53(unsigned long long x, const MathTab* __restrict__ T) {
  const unsigned long long n = (x >> 11) | 1ull;  // u = n 2^-53, n odd, 1 <= n < 2^53
  const int p = 63 - __clzll((long long)n);
  const unsigned long long mb = n << (52 - p);    // significand with its leading 1 at bit 52
  int e = p - 53;
  int j, sh;
  long long diff;
  double rf;
  if (mb >= 0x16A09E667F3BCDull) {  // m >= sqrt(2) (the double 1.4142135623730951): use m / 2
    e += 1;
    j = (int)((mb + (1ull << 45)) >> 46);
    diff = (long long)mb - ((long long)j << 46);  // (m / 2 - j / 128) 2^53
    rf = __ldg(&T->inv_f53[j]);
    sh = 13;  // v 2^64 = diff 2^11 (128 / j)
  } else {
    j = (int)((mb + (1ull << 44)) >> 45);
    diff = (long long)mb - ((long long)j << 45);  // (m - j / 128) 2^52
    rf = __ldg(&T->inv_f52[j]);
    sh = 14;  // v 2^64 = diff 2^12 (128 / j)
  }
  const double v = (double)diff * rf;
  // v in 2^-64 fixed point: |diff| << sh below 2^59, times (128 / j) 2^62, over 2^64
  const unsigned long long ad = (unsigned long long)(diff < 0 ? -diff : diff);
  const long long vm = (long long)__umul64hi(ad << sh, __ldg(&T->inv_f_q62[j]));
  const long long v64 = diff < 0 ? -vm : vm;
  const long long v2 = __mul64hi(v64, v64);  // v^2 2^64
  // coefficients in 2^-62 fixed point
  constexpr long long k2 = 1ll << 61, k3 = 0x1555555555555555ll, k4 = 1ll << 60;
  constexpr long long k5 = 0x0CCCCCCCCCCCCCCDll, k6 = 0x0AAAAAAAAAAAAAABll, k7 = 0x0924924924924925ll;
  const long long c = k6 - __mul64hi(v64, k7) + (v2 >> 5);  // 1/6 - v/7 + v^2/8
  const long long b = k4 - __mul64hi(v64, k5) + __mul64hi(v2, c);
  const long long q = k2 - __mul64hi(v64, k3) + __mul64hi(v2, b);  // in (0.497, 0.503) 2^62
  const double qd = __longlong_as_double(__double_as_longlong(__ll2double_rn(q)) - (62ll << 52));
  const double pl = fma(-(v * v), qd, v);
  const double de = (double)e;
  const double hi = fma(de, kLn2Hi, __ldg(&T->log_f[j]));
  return hi + fma(de, kLn2Lo, pl);
}

// exp x = 2^k 2^(j/32) e^r with n = 32 k + j = round(32 x / ln 2) and
// |r| <= ln 2 / 64; e^r - 1 = r + r^2 (1/2 + r/6 + r^2/24 + r^3/120 + r^4/720).
__device__ __forceinline__ double tang_exp(double x, const MathTab* __restrict__ T) {
  if (!(x > -708.0 && x < 709.0)) return exp(x);
  const double shift = 0x1.8p52;  // adding it leaves round(32 x / ln 2) in the low bits
  const double t = fma(x, kInvLn2x32, shift);
  const int n = (int)(unsigned)__double2loint(t);
  const double nd = t - shift;
  double r = fma(-nd, kLn2by32Hi, x);
  r = fma(-nd, kLn2by32Lo, r);
  const double r2 = r * r;
  const double pa = fma(r, 1.0 / 6.0, 0.5);
  const double pb = fma(r, 1.0 / 120.0, 1.0 / 24.0);
  const double pq = fma(fma(r2, 1.0 / 720.0, pb), r2, pa);
  const double p = fma(r2, pq, r);
  const double s = __ldg(&T->exp2_j[n & 31]);
  return fma(s, p, s) * pow2i(n >> 5);
}

// ---- integer exponential of fixed-point weights ----
// round(e^d 2^B) for d <= 0 (B = 54 for the segment kernel's tiles of at most
// 256 weights, 50 for the standalone resampler's tiles of 4096, so that a
// tile's sum stays below 2^62), the weight of a particle relative to a
// power-of-two reference as a 2^-B fixed-point integer, on the integer pipes
// (only the argument split is FP64).  e^d = 2^-y with y = -d / ln 2 = n + j/128
// + r, r < 2^-7: e^d = 2^-n 2^(-j/128) e^(-r ln 2), the last factor by its
// Taylor series to degree 6 (Horner; all partial sums positive), in 2^-63 fixed
// point with 64-bit multiply-high products.  Within one unit of the exact
// rounding; below e^-38.5 (less than half a unit) it returns 0.  A d slightly
// above 0 (rounding of the reference) is taken as 0.
constexpr unsigned long long kInvLn2Q63 = 0xb8aa3b295c17f0bcull;  // round(2^63 / ln 2)
constexpr unsigned long long kLn2Q64 = 0xb17217f7d1cf79acull;     // round(ln 2 2^64)

__device__ __forceinline__ unsigned long long mulhi64(unsigned long long a, unsigned long long b) {
  return __umul64hi(a, b);
}

// The core from X = -d 2^58 (an unsigned integer, -d < 38.5).
template <int B>
__device__ __forceinline__ long long exp_fix_x(unsigned long long X, const MathTab* __restrict__ T) {
  static_assert(B >= 40 && B <= 54, "fixed-point bits");
  // Y = X / ln 2 in units of 2^-58: floor(X kInvLn2Q63 / 2^63)
  const unsigned long long Y = (mulhi64(X, kInvLn2Q63) << 1) | ((X * kInvLn2Q63) >> 63);
  const int n = (int)(Y >> 58);
  if (n >= B + 1) return 0;  // at most half a unit
  const int j = (int)((Y >> 51) & 127);
  const unsigned long long r = Y & ((1ull << 51) - 1);  // r 2^58, r < 2^-7
  const unsigned long long t2 = mulhi64(r << 5, kLn2Q64) << 1;  // 2 t 2^63 with t = r ln 2
  unsigned long long p = 0x2d82d82d82d82eull;                   // 2^63 / 720
  p = 0x111111111111111ull - mulhi64(t2, p);                     // 2^63 / 120 - t p
  p = 0x555555555555555ull - mulhi64(t2, p);                     // 2^63 / 24
  p = 0x1555555555555555ull - mulhi64(t2, p);                    // 2^63 / 6
  p = 0x4000000000000000ull - mulhi64(t2, p);                    // 2^63 / 2
  p = 0x8000000000000000ull - mulhi64(t2, p);                    // 2^63
  p = 0x8000000000000000ull - mulhi64(t2, p);                    // e^-t 2^63
  const unsigned long long q = mulhi64(p, __ldg(&T->exp2_neg_q63[j])) << 1;  // e^-(j/128 + r) ln 2 2^63
  const int s = 63 - B + n;  // to 2^-B units and the factor 2^-n
  return (long long)((q + (1ull << (s - 1))) >> s);
}

// 2^-(Y 2^-57 - n) in 2^-61 fixed point (in (2^60, 2^61]) for Y = y 2^57 and
// n = floor(y): two 64-entry Q63 tables, T64[j] = 2^(-j/64) and
// T4096[j] = 2^(-j/4096), and a degree-4 polynomial on the remainder
// g < 2^-12 of y: 2^-g = e^-r with r = g ln 2, e^-r = 1 - r + r^2/2 - r^3/6 +
// r^4/24 (truncation below 2^-69), the terms past r in 32-bit products.
// Relative error below 2^-58.
__device__ __forceinline__ unsigned long long exp2_frac_q61(unsigned long long Y,
                                                            const unsigned long long* T64,
                                                            const unsigned long long* T4096) {
  const unsigned long long g = Y & ((1ull << 45) - 1);       // g 2^57, g < 2^-12
  const unsigned long long r = __umul64hi(g << 7, kLn2Q64);  // r 2^64, r < 2^-12.5
  const unsigned rh = (unsigned)(r >> 20);                   // r 2^44, below 2^32
  const unsigned long long r2 = (unsigned long long)rh * rh;  // r^2 2^88
  const unsigned r2h = (unsigned)(r2 >> 32);                  // r^2 2^56, below 2^31
  const unsigned r3 = (unsigned)(((unsigned long long)r2h * rh) >> 37);   // r^3 2^63
  const unsigned r4 = (unsigned)(((unsigned long long)r2h * r2h) >> 49);  // r^4 2^63
  const unsigned long long p =
      0x8000000000000000ull - (r >> 1) + (r2 >> 26) - r3 / 6u + r4 / 24u;  // e^-r 2^63
  const unsigned long long t = __umul64hi(T64[(Y >> 51) & 63], T4096[(Y >> 45) & 63]);  // 2^62
  return __umul64hi(t, p);
}

// The same exponential from the two 64-entry tables (the caller stages them,
// e.g. in shared memory): Y = X / ln 2 = n + j1/64 + j2/4096 + g and
// exp2_frac_q61.  Four 64-bit multiply-highs instead of ten; within one unit
// of the exact rounding for B <= 54.
template <int B>
__device__ __forceinline__ long long exp_fix_x2(unsigned long long X,
                                                const unsigned long long* T64,
                                                const unsigned long long* T4096) {
  static_assert(B >= 40 && B <= 54, "fixed-point bits");
  const unsigned long long Y = __umul64hi(X, kInvLn2Q63);  // X / ln 2 in units of 2^-57
  const int n = (int)(Y >> 57);
  if (n >= B + 1) return 0;  // at most half a unit
  const unsigned long long q = exp2_frac_q61(Y, T64, T4096);  // 2^-(Y 2^-57 - n) 2^61
  const int s = 61 - B + n;                                   // to 2^-B units and 2^-n
  return (long long)((q + (1ull << (s - 1))) >> s);
}

// e^-m as a double for 0 <= m < 64 on the integer pipes: X = m 2^58 from the
// bits of m (truncated, error below 2^-58), Y = X / ln 2, q = exp2_frac_q61,
// then q 2^-(61 + n) with one rounding of q to 53 bits and an exact exponent
// shift: within about 0.6 ulp.  Outside [0, 64) the table exponential.
__device__ __forceinline__ double exp_neg_int(double m, const MathTab* __restrict__ T) {
  if (!(m >= 0.0 && m < 64.0)) return tang_exp(-m, T);
  const long long b = __double_as_longlong(m);
  const int e = (int)(b >> 52);
  if (e == 0) return 1.0;  // m = 0 or subnormal: e^-m rounds to 1
  const unsigned long long mt = (unsigned long long)((b & 0x000FFFFFFFFFFFFFll) | 0x0010000000000000ll);
  const int sh = e - 1017;  // m 2^58 = mt 2^(e - 1075 + 58)
  const unsigned long long X = sh >= 0 ? (mt << sh) : (-sh < 64 ? (mt >> -sh) : 0ull);
  const unsigned long long Y = __umul64hi(X, kInvLn2Q63);
  const int n = (int)(Y >> 57);
  const unsigned long long q = exp2_frac_q61(Y, T->exp2_neg64_q63, T->exp2_neg4096_q63);
  const double dq = __ull2double_rn(q);  // q in (2^60, 2^61]: exact power-of-two shift below
  return __longlong_as_double(__double_as_longlong(dq) - ((long long)(61 + n) << 52));
}

template <int B>
__device__ __forceinline__ long long exp_fix(double d, const MathTab* __restrict__ T) {
  if (!(d > -38.5)) return 0;
  const long long b = __double_as_longlong(-d);
  if (b <= 0) return 1ll << B;  // d >= 0
  const int e = (int)(b >> 52);
  if (e == 0) return 1ll << B;  // |d| below 2^-1022
  const unsigned long long m = (unsigned long long)((b & 0x000FFFFFFFFFFFFFll) | 0x0010000000000000ll);
  const int sh = e - 1017;  // X = -d 2^58 (below 2^64 since -d < 2^6)
  return exp_fix_x<B>(sh >= 0 ? (m << sh) : (-sh < 64 ? (m >> -sh) : 0ull), T);
}

// round(e^d 2^B) for d <= 0 on the two-table exponential
template <int B>
__device__ __forceinline__ long long exp_fix2(double d, const unsigned long long* T64,
                                              const unsigned long long* T4096) {
  if (!(d > -38.5)) return 0;
  const long long b = __double_as_longlong(-d);
  if (b <= 0) return 1ll << B;
  const int e = (int)(b >> 52);
  if (e == 0) return 1ll << B;
  const unsigned long long m = (unsigned long long)((b & 0x000FFFFFFFFFFFFFll) | 0x0010000000000000ll);
  const int sh = e - 1017;
  return exp_fix_x2<B>(sh >= 0 ? (m << sh) : (-sh < 64 ? (m >> -sh) : 0ull), T64, T4096);
}

// ---- the argument k ln 2 - x in 2^-58 fixed point, on the integer pipes ----
// For a power-of-two reference 2^k (|k| < 2^11) and a log-weight x <= k ln 2
// (up to rounding): K = k ln 2 2^58 from ln 2 to 2^-116, and x 2^58 from the
// bits of x, both in 128-bit integers, so X = K - x 2^58 is within two units
// of (k ln 2 - x) 2^58 whatever the magnitudes of k and x.
constexpr unsigned long long kLn2Q116Hi = 0xb17217f7d1cf7ull;               // round(ln 2 2^116) >> 64
constexpr unsigned long long kLn2Q116Lo = 0x9abc9e3b39803f2full;           // its low 64 bits
constexpr unsigned long long kExpCutQ58 = 0x9a00000000000000ull;           // 38.5 2^58

__device__ __forceinline__ __int128 ref_q58(int k) {
  const __int128 l = ((__int128)kLn2Q116Hi << 64) | (__int128)kLn2Q116Lo;
  return ((__int128)k * l) >> 58;
}

// floor-toward-zero of x 2^58 as a signed 128-bit integer (|x| < 2^69)
__device__ __forceinline__ __int128 fix_q58(double x) {
  const long long b = __double_as_longlong(x);
  const int e = (int)((b >> 52) & 0x7ff);
  if (e == 0) return 0;
  const unsigned long long m = (unsigned long long)((b & 0x000FFFFFFFFFFFFFll) | 0x0010000000000000ll);
  const int sh = e - 1017;
  __int128 v;
  if (sh >= 74)
    v = (__int128)1 << 126;
  else if (sh >= 0)
    v = (__int128)m << sh;
  else
    v = -sh < 64 ? (__int128)(m >> -sh) : 0;
  return b < 0 ? -v : v;
}

// round(e^(x - k ln 2) 2^B) for a log-weight x (-inf allowed) and the
// reference K = ref_q58(k), |k| < 2^11: integer pipes only.
template <int B>
__device__ __forceinline__ long long weight_fix(double x, __int128 K, const MathTab* __restrict__ T) {
  if (__double_as_longlong(x) == (long long)0xFFF0000000000000ull) return 0;  // -inf
  __int128 X = K - fix_q58(x);
  if (X < 0) X = 0;  // x above the reference by rounding: weight 1
  if (X >= (__int128)kExpCutQ58) return 0;
  return exp_fix_x<B>((unsigned long long)X, T);
}

// The argument in 2^-52 units, in 64-bit integers: for a reference k with
// |k| < 2048, K52 = round(k ln 2 2^52) (below 2^63) and x 2^52 truncated toward
// zero (exact for |x| >= 1, |x| < 2^11; a log-weight beyond 2^11 in magnitude
// lies more than 38.5 below such a reference, weight 0).  The argument is then
// within 1.5 2^-52 of k ln 2 - x: a relative weight error below 2^-51.
constexpr long long kExpCutQ52 = 0x268000000000000ll;  // 38.5 2^52

__device__ __forceinline__ long long ref_q52(int k) {
  return (long long)((ref_q58(k) + 32) >> 6);
}

template <int B>
__device__ __forceinline__ long long weight_fix52(double x, long long K52,
                                                  const unsigned long long* T64,
                                                  const unsigned long long* T4096) {
  const long long b = __double_as_longlong(x);
  const int e = (int)((b >> 52) & 0x7ff);
  if (e >= 1034) return 0;  // |x| >= 2^11 (or -inf, NaN): far below the reference
  const long long m = (b & 0x000FFFFFFFFFFFFFll) | (e ? 0x0010000000000000ll : 0ll);
  const int sh = e - 1023;  // x 2^52 = m 2^sh
  long long v = sh >= 0 ? (m << sh) : (-sh < 63 ? (m >> -sh) : 0ll);
  if (b < 0) v = -v;
  if (v <= K52 - kExpCutQ52) return 0;
  long long X = K52 - v;
  if (X < 0) X = 0;  // x above the reference by rounding: weight 1
  return exp_fix_x2<B>((unsigned long long)X << 6, T64, T4096);
}

__device__ __forceinline__ long long exp_fix54(double d, const MathTab* __restrict__ T) {
  return exp_fix<54>(d, T);
}

// x / y from a precomputed y_inv ~ 1/y: one residual correction of x * y_inv
// (within an ulp of the correctly rounded quotient).
__device__ __forceinline__ double div_by(double x, double y, double y_inv) {
  const double q = x * y_inv;
  return fma(fma(-q, y, x), y_inv, q);
}

// A particle's draw stream for one segment: counter (n, k, d, tag), d counts
// blocks; `tab` is the device's math table.
struct Stream {
  uint32_t k0, k1, n, k, d, tag;
  const MathTab* tab;
  __device__ __forceinline__ Block4 next() {
    Block4 b = philox(n, k, d, tag, k0, k1);
    d += 1;
    return b;
  }
};

// ---- uniforms: exact odd-integer grids strictly inside (0,1) ----
template <typename R>
struct Unif;
template <>
struct Unif<double> {
  // ((w_hi:w_lo) >> 11) | 1, times 2^-53, assembled from bits on the integer
  // pipes: n = (x >> 11) | 1 is odd with its leading one at bit p (0..52), so
  // n 2^-53 = 1.f 2^(p - 53) exactly, exponent field p + 970 and fraction
  // (n << (52 - p)) without its leading one.  No FP64 operation.
  __device__ __forceinline__ static double from64(uint64_t x) {
    const unsigned long long n = (x >> 11) | 1ull;
    const int p = 63 - __clzll((long long)n);
    const unsigned long long frac = (n << (52 - p)) & 0x000FFFFFFFFFFFFFull;
    return __longlong_as_double((long long)(((unsigned long long)(p + 970) << 52) | frac));
  }
  __device__ __forceinline__ static double first(const Block4& b) {
    return from64(((uint64_t)b.w1 << 32) | b.w0);
  }
  __device__ __forceinline__ static double second(const Block4& b) {
    return from64(((uint64_t)b.w3 << 32) | b.w2);
  }
};
template <>
struct Unif<float> {
  // (w >> 8) | 1, times 2^-24 (24-bit integer: exact in float), w the high word
  // of the FP64 uniform's 64 bits (w1 of the first, w3 of the second): an FP32
  // draw is then the FP64 draw of the same counter to within 2^-24
  __device__ __forceinline__ static float first(const Block4& b) {
    return (float)((b.w1 >> 8) | 1u) * 0x1p-24f;
  }
  __device__ __forceinline__ static float second(const Block4& b) {
    return (float)((b.w3 >> 8) | 1u) * 0x1p-24f;
  }
};

// a > b for non-negative (or +inf) a and b by their bit patterns, which order
// like the values: an integer compare instead of an FP64 one
__device__ __forceinline__ bool gt_nonneg(double a, double b) {
  return __double_as_longlong(a) > __double_as_longlong(b);
}
__device__ __forceinline__ bool gt_nonneg(float a, float b) {
  return __float_as_int(a) > __float_as_int(b);
}

// ---- FP32 elementary functions of the FP32-particle mode ----
// The FP32 mode computes its logarithms, exponentials and the Box-Muller cosine
// with the functions below, written out in single-precision operations (every
// fused multiply-add an explicit fmaf; the library is built with -fmad=false),
// not with CUDA's logf / expf / cosf: every rounding of the mode is then fixed
// by these definitions, so that an implementation elsewhere that performs the
// same operations gets the same bits.  Each follows a textbook method with
// Taylor coefficients rounded to float and is within ~2 ulp of the exact value.
//   log    x = 2^e m, m in [sqrt(2)/2, sqrt(2)], f = m - 1 (exact), s = f / (2 + f):
//          log(1 + f) = 2 atanh(s) = f - s (f - R(s^2)), R(z) = z (2/3 + z (2/5 +
//          z (2/7 + z 2/9))) (the atanh series; |s| <= 0.172), plus e ln 2 with
//          a two-part ln 2 (e ln2_hi exact).
//   exp    n = rint(x / ln 2), r = x - n ln 2 (two-part ln 2), |r| <= ln 2 / 2,
//          e^r = 1 + (r + r^2 (1/2! + r (1/3! + ... + r / 7!))), times 2^n.
//   cos(2 pi u)  4u = q + t exactly (q = rint(4u), |t| <= 1/2), then cos or
//          -/+ sin of t pi/2 by quadrant from their Taylor series in t.
//   log1p  the log core on x itself inside [sqrt(2)/2 - 1, sqrt(2) - 1], else on
//          1 + x with the rounding error of that sum added as c / (1 + x).
//   expm1  the Taylor series of e^x - 1 to x^8/8! for |x| < ln 2 / 2, else
//          2^n expm1(r) + (2^n - 1) with the reduction of exp.
//   log k! the math table's FP64 log k! rounded to float below 32, Stirling's
//          series in float above.
constexpr float kF32Ln2Hi = 0x1.62e4p-1f;     // ln 2 to 15 significant bits: e ln2_hi exact
constexpr float kF32Ln2Lo = 0x1.7f7d1cp-20f;  // ln 2 - kF32Ln2Hi, rounded
constexpr float kF32InvLn2 = 0x1.715476p+0f;
constexpr float kF32Atanh3 = 0x1.555556p-1f, kF32Atanh5 = 0x1.99999ap-2f;  // 2/3, 2/5
constexpr float kF32Atanh7 = 0x1.24924ap-2f, kF32Atanh9 = 0x1.c71c72p-3f;  // 2/7, 2/9
constexpr float kF32Inv2 = 0x1p-1f, kF32Inv6 = 0x1.555556p-3f, kF32Inv24 = 0x1.555556p-5f;
constexpr float kF32Inv120 = 0x1.111112p-7f, kF32Inv720 = 0x1.6c16c2p-10f;
constexpr float kF32Inv5040 = 0x1.a01a02p-13f, kF32Inv40320 = 0x1.a01a02p-16f;
// (pi/2)^n / n! with alternating signs; pi/2 itself as a two-part constant
constexpr float kF32PiO2Hi = 0x1.921fb6p+0f, kF32PiO2Lo = -0x1.777a5cp-25f;
constexpr float kF32S3 = -0x1.4abbcep-1f, kF32S5 = 0x1.466bc6p-4f, kF32S7 = -0x1.32d2ccp-8f,
                kF32S9 = 0x1.507834p-13f;
constexpr float kF32C2 = -0x1.3bd3ccp+0f, kF32C4 = 0x1.03c1f0p-2f, kF32C6 = -0x1.55d3c8p-6f,
                kF32C8 = 0x1.e1f506p-11f, kF32C10 = -0x1.a6d1f2p-16f;
constexpr float kF32HalfLog2Pi = 0x1.d67f1cp-1f;
constexpr float kF32Inv12 = 0x1.555556p-4f, kF32Inv360 = 0x1.6c16c2p-9f,
                kF32Inv1260 = 0x1.a01a02p-11f;

// 2^n as a float for n in [-126, 127]
__device__ __forceinline__ float f32_pow2i(int n) { return __int_as_float((n + 127) << 23); }

// log(1 + f) for f in [sqrt(2)/2 - 1, sqrt(2) - 1]
__device__ __forceinline__ float f32_log1p_core(float f) {
  const float s = f / (2.0f + f);
  const float z = s * s;
  float R = fmaf(z, kF32Atanh9, kF32Atanh7);
  R = fmaf(R, z, kF32Atanh5);
  R = fmaf(R, z, kF32Atanh3);
  R = z * R;
  return f - s * (f - R);
}

// e ln 2 + l
__device__ __forceinline__ float f32_add_eln2(int e, float l) {
  if (e == 0) return l;
  const float fe = (float)e;
  return fe * kF32Ln2Hi + fmaf(fe, kF32Ln2Lo, l);
}

__device__ __forceinline__ float f32_log(float x) {
  if (!(x > 0.0f)) return x == 0.0f ? -INFINITY : __int_as_float(0x7fc00000);
  if (x == INFINITY) return x;
  int ix = __float_as_int(x);
  int e = -127;
  if (ix < 0x00800000) {  // subnormal: scale by 2^24
    ix = __float_as_int(x * 0x1p24f);
    e -= 24;
  }
  const int mb = ix & 0x007fffff;
  e += ix >> 23;
  float m;
  if (mb > 0x3504f3) {  // m above float(sqrt 2): use m / 2
    m = __int_as_float(mb | (126 << 23));
    e += 1;
  } else {
    m = __int_as_float(mb | (127 << 23));
  }
  return f32_add_eln2(e, f32_log1p_core(m - 1.0f));  // m - 1 exact
}

// e^r - 1 - r for |r| <= ln 2 / 2, as r^2 (1/2! + r (1/3! + ... ))
__device__ __forceinline__ float f32_expm1_poly(float r, bool deg8) {
  float q = deg8 ? fmaf(r, kF32Inv40320, kF32Inv5040) : kF32Inv5040;
  q = fmaf(q, r, kF32Inv720);
  q = fmaf(q, r, kF32Inv120);
  q = fmaf(q, r, kF32Inv24);
  q = fmaf(q, r, kF32Inv6);
  q = fmaf(q, r, kF32Inv2);
  return (r * r) * q;
}

__device__ __forceinline__ float f32_exp(float x) {
  if (x != x) return x;
  if (x > 89.0f) return INFINITY;
  if (x < -104.0f) return 0.0f;
  const float nf = rintf(x * kF32InvLn2);
  float r = fmaf(-nf, kF32Ln2Hi, x);
  r = fmaf(-nf, kF32Ln2Lo, r);
  const float y = 1.0f + (r + f32_expm1_poly(r, false));
  const int n = (int)nf;
  if (n >= -126 && n <= 127) return y * f32_pow2i(n);
  if (n > 127) return (y * 2.0f) * f32_pow2i(n - 1);
  return (y * f32_pow2i(n + 100)) * 0x1p-100f;
}

// cos(2 pi u) for u in [0, 1]
__device__ __forceinline__ float f32_cos2pi(float u) {
  const float v = 4.0f * u;
  const float qf = rintf(v);
  const float t = v - qf;  // exact, |t| <= 1/2
  const float z = t * t;
  const int q = (int)qf & 3;
  if (q & 1) {  // -/+ sin(t pi / 2)
    float p = fmaf(z, kF32S9, kF32S7);
    p = fmaf(p, z, kF32S5);
    p = fmaf(p, z, kF32S3);
    const float sn = fmaf(t, kF32PiO2Hi, fmaf(t * z, p, t * kF32PiO2Lo));
    return q == 1 ? -sn : sn;
  }
  float p = fmaf(z, kF32C10, kF32C8);
  p = fmaf(p, z, kF32C6);
  p = fmaf(p, z, kF32C4);
  p = fmaf(p, z, kF32C2);
  const float cs = fmaf(z, p, 1.0f);
  return q == 0 ? cs : -cs;
}

__device__ __forceinline__ float f32_log1p(float x) {
  if (!(x > -1.0f)) return x == -1.0f ? -INFINITY : __int_as_float(0x7fc00000);
  if (x == INFINITY) return x;
  if (x >= -0x1.2bec34p-2f && x <= 0x1.a8279ap-2f) return f32_log1p_core(x);
  const float u = 1.0f + x;
  // the rounding error of 1 + x (exact: the larger operand first), over u
  const float c = (x > 1.0f ? 1.0f - (u - x) : x - (u - 1.0f)) / u;
  const int iu = __float_as_int(u);
  const int mb = iu & 0x007fffff;
  int e = (iu >> 23) - 127;
  float m;
  if (mb > 0x3504f3) {
    m = __int_as_float(mb | (126 << 23));
    e += 1;
  } else {
    m = __int_as_float(mb | (127 << 23));
  }
  return f32_add_eln2(e, f32_log1p_core(m - 1.0f) + c);
}

__device__ __forceinline__ float f32_expm1(float x) {
  if (x != x) return x;
  if (x > 89.0f) return INFINITY;
  if (x < -104.0f) return -1.0f;
  if (fabsf(x) < 0x1.62e430p-2f) return x + f32_expm1_poly(x, true);  // |x| < ln 2 / 2
  const float nf = rintf(x * kF32InvLn2);
  float r = fmaf(-nf, kF32Ln2Hi, x);
  r = fmaf(-nf, kF32Ln2Lo, r);
  const float em = r + f32_expm1_poly(r, true);
  const int n = (int)nf;
  if (n > 127) return (em + 1.0f) * 2.0f * f32_pow2i(n - 1);
  const float two = f32_pow2i(n < -126 ? -126 : n);
  return fmaf(two, em, two - 1.0f);
}

// ---- precision-overloaded math (IEEE library calls in FP64, the functions
// above in FP32; no fast-math) ----
__device__ __forceinline__ double m_log(double x) { return log(x); }
__device__ __forceinline__ float m_log(float x) { return f32_log(x); }
__device__ __forceinline__ double m_sqrt(double x) { return sqrt(x); }
__device__ __forceinline__ float m_sqrt(float x) { return sqrtf(x); }
__device__ __forceinline__ double m_fma(double a, double b, double c) { return fma(a, b, c); }
__device__ __forceinline__ float m_fma(float a, float b, float c) { return fmaf(a, b, c); }
__device__ __forceinline__ double m_floor(double x) { return floor(x); }
__device__ __forceinline__ float m_floor(float x) { return floorf(x); }
__device__ __forceinline__ double m_fabs(double x) { return fabs(x); }
__device__ __forceinline__ float m_fabs(float x) { return fabsf(x); }
// cos(2 pi u), the Box-Muller angle
__device__ __forceinline__ double cos_2pi(double u) { return cos(kTwoPi * u); }
__device__ __forceinline__ float cos_2pi(float u) { return f32_cos2pi(u); }

// Logarithm / exponential used by the samplers: FP64 through the tables,
// FP32 through the single-precision functions above.
__device__ __forceinline__ double lg(double x, const Stream& s) { return tang_log(x, s.tab); }
__device__ __forceinline__ float lg(float x, const Stream&) { return f32_log(x); }
__device__ __forceinline__ double ex(double x, const Stream& s) { return tang_exp(x, s.tab); }
__device__ __forceinline__ float ex(float x, const Stream&) { return f32_exp(x); }

template <typename R>
struct C;
template <>
struct C<double> {
  static constexpr double ln2 = kLn2, two_pi = kTwoPi;
};
template <>
struct C<float> {
  static constexpr float ln2 = kLn2f, two_pi = kTwoPif;
};

template <typename R>
__device__ __forceinline__ R neg_inf() {
  return -(R)INFINITY;
}

// ---- variates (SAMPLE) ----
template <typename R>
__device__ __forceinline__ R uniform01(Stream& s) {
  return Unif<R>::first(s.next());
}

// Box-Muller, cosine branch: sqrt(-2 ln u1) * cos(2 pi u2)
__device__ __forceinline__ double log_first_uniform(const Block4& b, const Stream& s, double) {
  return log_unif53(((unsigned long long)b.w1 << 32) | b.w0, s.tab);
}
__device__ __forceinline__ float log_first_uniform(const Block4& b, const Stream&, float) {
  return f32_log(Unif<float>::first(b));
}

template <typename R>
__device__ __forceinline__ R normal01(Stream& s) {
  const Block4 b = s.next();
  const R u2 = Unif<R>::second(b);
  const R rad = m_sqrt((R)-2.0 * log_first_uniform(b, s, (R)0));
  return rad * cos_2pi(u2);
}

// -ln u of the next uniform (FP64: straight from its random bits)
template <typename R>
__device__ __forceinline__ R neg_log_uniform(Stream& s);
template <>
__device__ __forceinline__ double neg_log_uniform<double>(Stream& s) {
  const Block4 b = s.next();
  return -log_unif53(((unsigned long long)b.w1 << 32) | b.w0, s.tab);
}
template <>
__device__ __forceinline__ float neg_log_uniform<float>(Stream& s) {
  return -f32_log(uniform01<float>(s));
}

// Exponential(rate): -ln(u) / rate
template <typename R>
__device__ __forceinline__ R exponential(Stream& s, R rate) {
  return neg_log_uniform<R>(s) / rate;
}

// Exponential(rate) with a precomputed 1/rate (rate > 0): -ln(u) * (1/rate),
// within an ulp or so of the quotient
__device__ __forceinline__ double exponential_inv(Stream& s, double, double inv_rate) {
  return neg_log_uniform<double>(s) * inv_rate;
}
__device__ __forceinline__ float exponential_inv(Stream& s, float rate, float) {
  return neg_log_uniform<float>(s) / rate;
}

// Gamma(shape 1, scale theta): theta * (-ln u)
template <typename R>
__device__ __forceinline__ R gamma1(Stream& s, R theta) {
  return theta * neg_log_uniform<R>(s);
}

// Uniform(lo, hi): fma(hi - lo, u, lo)
template <typename R>
__device__ __forceinline__ R uniform_ab(Stream& s, R lo, R hi) {
  const R u = uniform01<R>(s);
  return m_fma(hi - lo, u, lo);
}

template <typename R>
__device__ __forceinline__ bool bernoulli(Stream& s, R p) {
  return gt_nonneg(p, uniform01<R>(s));  // u < p; a negative p is never above u
}

// log k! for the Poisson rejection test: FP64 through the library's lgamma,
// FP32 from the math table's FP64 log k! rounded to float below 32 and
// Stirling's series in float operations above (x = k + 1:
// (x - 1/2) log x - x + log(2 pi)/2 + 1/(12x) - 1/(360x^3) + 1/(1260x^5)).
__device__ __forceinline__ float f32_lfact(int k, const MathTab* __restrict__ T) {
  if (k < 32) return (float)__ldg(&T->lfact[k < 0 ? 0 : k]);
  const float x = (float)k + 1.0f;
  const float ix = 1.0f / x, ix2 = ix * ix;
  const float series = ix * (kF32Inv12 - ix2 * (kF32Inv360 - ix2 * kF32Inv1260));
  return (((x - 0.5f) * f32_log(x) - x) + kF32HalfLog2Pi) + series;
}
__device__ __forceinline__ double log_fact(double k, const MathTab*) { return lgamma(k + 1.0); }
__device__ __forceinline__ float log_fact(float k, const MathTab* T) { return f32_lfact((int)k, T); }

// Poisson(mean): sequential-search inversion below 10 (one uniform, at most
// 200 terms); Hormann's transformed rejection with squeeze (PTRS, 1993) from
// 10 up, one block per trial, at most 1000 trials.
template <typename R>
__device__ __noinline__ int poisson(Stream& s, R mean) {
  if (gt_nonneg((R)10.0, mean)) {  // mean >= 0
    const R u = uniform01<R>(s);
    int k = 0;
    R p;
    if constexpr (sizeof(R) == 8)
      p = exp_neg_int(mean, s.tab);  // integer pipes: off the FP64 pipe
    else
      p = f32_exp(-mean);
    R acc = p;
    while (gt_nonneg(u, acc) && k < 200) {
      k += 1;
      if constexpr (sizeof(R) == 8)
        p = p * (mean * __ldg(&s.tab->inv_int[k]));  // mean / k off the chain through p
      else
        p = p * mean / (R)k;
      acc = acc + p;
    }
    return k;
  }
  const R slam = m_sqrt(mean);
  const R loglam = m_log(mean);
  const R b = (R)0.931 + (R)2.53 * slam;
  const R a = (R)-0.059 + (R)0.02483 * b;
  const R invalpha = (R)1.1239 + (R)1.1328 / (b - (R)3.4);
  const R vr = (R)0.9277 - (R)3.6224 / (b - (R)2.0);
  for (int trial = 0; trial < 1000; ++trial) {
    const Block4 blk = s.next();
    const R U = Unif<R>::first(blk) - (R)0.5;
    const R V = Unif<R>::second(blk);
    const R us = (R)0.5 - m_fabs(U);
    const R kr = m_floor(((R)2.0 * a / us + b) * U + mean + (R)0.43);
    if (us >= (R)0.07 && V <= vr) return (int)kr;
    if (kr < (R)0.0 || (us < (R)0.013 && V > us)) continue;
    if (m_log(V) + m_log(invalpha) - m_log(a / (us * us) + b) <=
        -mean + kr * loglam - log_fact(kr, s.tab))
      return (int)kr;
  }
  return (int)m_floor(mean);
}

// LogNormal(0, sigma) = exp(sigma * N(0,1))
template <typename R>
__device__ __forceinline__ R lognormal(Stream& s, R sigma) {
  return ex(sigma * normal01<R>(s), s);
}

// log k!: the table below 32, Stirling's series for log Gamma(k+1) above
// (x = k + 1: (x - 1/2) ln x - x + ln(2 pi)/2 + 1/(12x) - 1/(360x^3) + 1/(1260x^5)).
__device__ __forceinline__ double lfact(int k, const MathTab* __restrict__ T) {
  if (k < 32) return __ldg(&T->lfact[k]);
  const double x = (double)k + 1.0;
  const double ix = 1.0 / x, ix2 = ix * ix;
  const double series = ix * (1.0 / 12.0 - ix2 * (1.0 / 360.0 - ix2 * (1.0 / 1260.0)));
  return (x - 0.5) * tang_log(x, T) - x + 0.91893853320467274178 + series;
}

// Gamma(shape, 1), shape >= 1 (Marsaglia and Tsang 2000): d = shape - 1/3,
// c = 1/sqrt(9d); x ~ N(0,1), v = (1 + c x)^3 (rejected at once if 1 + c x <= 0),
// u ~ U(0,1); accept d v if u < 1 - 0.0331 x^4 or ln u < x^2/2 + d (1 - v + ln v).
template <typename R>
__device__ __noinline__ R gamma_mt(Stream& s, R shape) {
  const R d = shape - (R)1.0 / (R)3.0;
  const R c = (R)1.0 / m_sqrt((R)9.0 * d);
  for (int trial = 0; trial < 1000; ++trial) {
    const R x = normal01<R>(s);
    R v = (R)1.0 + c * x;
    if (v <= (R)0.0) continue;
    v = v * v * v;
    const R u = uniform01<R>(s);
    const R x2 = x * x;
    if (u < (R)1.0 - (R)0.0331 * (x2 * x2)) return d * v;
    if (lg(u, s) < (R)0.5 * x2 + d * ((R)1.0 - v + lg(v, s))) return d * v;
  }
  return d;
}

// Beta(a, b) = X / (X + Y), X ~ Gamma(a), Y ~ Gamma(b) drawn in that order.
template <typename R>
__device__ __forceinline__ R beta_ab(Stream& s, R a, R b) {
  const R x = gamma_mt<R>(s, a);
  const R y = gamma_mt<R>(s, b);
  return x / (x + y);
}

// Binomial(n, p).  With p' = min(p, 1 - p) (the draw for p > 1/2 is n minus
// the draw for 1 - p): n p' < 10: inversion by sequential search from 0 with
// one uniform, f_0 = exp(n ln q), f_{k+1} = f_k (p'/q) (n - k) / (k + 1), at
// most 200 terms; otherwise Hormann's transformed rejection with squeeze
// (BTRS, 1993), one block per trial, acceptance in logs with log k!, at most
// 1000 trials.
template <typename R>
__device__ __noinline__ int binomial(Stream& s, int n, R p) {
  if (n <= 0 || !(p > (R)0.0)) return 0;
  if (!(p < (R)1.0)) return n;
  const bool flip = p > (R)0.5;
  const R pp = flip ? (R)1.0 - p : p;
  const R q = (R)1.0 - pp;
  int k;
  if ((R)n * pp < (R)10.0) {
    const R u = uniform01<R>(s);
    const R r = pp / q;
    R f = ex((R)n * lg(q, s), s);
    R acc = f;
    k = 0;
    while (u > acc && k < n && k < 200) {
      f = f * r * (R)(n - k) / (R)(k + 1);
      k += 1;
      acc = acc + f;
    }
  } else {
    const R spq = m_sqrt((R)n * pp * q);
    const R b = (R)1.15 + (R)2.53 * spq;
    const R a = (R)-0.0873 + (R)0.0248 * b + (R)0.01 * pp;
    const R c = (R)n * pp + (R)0.5;
    const R vr = (R)0.92 - (R)4.2 / b;
    const R alpha = ((R)2.83 + (R)5.1 / b) * spq;
    const R lpq = lg(pp / q, s);
    const int m = (int)m_floor((R)(n + 1) * pp);
    const R h = (R)lfact(m, s.tab) + (R)lfact(n - m, s.tab);
    k = (int)m_floor((R)n * pp);
    for (int trial = 0; trial < 1000; ++trial) {
      const Block4 blk = s.next();
      const R u = Unif<R>::first(blk) - (R)0.5;
      R v = Unif<R>::second(blk);
      const R us = (R)0.5 - m_fabs(u);
      const R kr = m_floor(((R)2.0 * a / us + b) * u + c);
      if (kr < (R)0.0 || kr > (R)n) continue;
      const int kk = (int)kr;
      if (us >= (R)0.07 && v <= vr) {
        k = kk;
        break;
      }
      v = lg(v * alpha / (a / (us * us) + b), s);
      if (v <= h - (R)lfact(kk, s.tab) - (R)lfact(n - kk, s.tab) + (R)(kk - m) * lpq) {
        k = kk;
        break;
      }
    }
  }
  return flip ? n - k : k;
}

// log Binomial(y | z, rho) (-inf for y > z); zero counts contribute nothing.
template <typename R>
__device__ __forceinline__ R binomial_logpmf(int y, int z, R rho, const Stream& s) {
  if (y > z) return neg_inf<R>();
  R lp = (R)(lfact(z, s.tab) - lfact(y, s.tab) - lfact(z - y, s.tab));
  if (y > 0) lp = lp + (R)y * lg(rho, s);
  if (z - y > 0) lp = lp + (R)(z - y) * lg((R)1.0 - rho, s);
  return lp;
}

// ---- predictive draws of the delayed-sampling CRBD (Section 6.3) ----
__device__ __forceinline__ double m_log1p(double x) { return log1p(x); }
__device__ __forceinline__ float m_log1p(float x) { return f32_log1p(x); }
__device__ __forceinline__ double m_expm1(double x) { return expm1(x); }
__device__ __forceinline__ float m_expm1(float x) { return f32_expm1(x); }

// Exponential(mu) with mu ~ Gamma(alpha, rate beta) integrated out (Lomax):
// P(x > t) = (beta / (beta + t))^alpha; by inversion of one uniform,
// x = beta (u^(-1/alpha) - 1) = beta expm1(-ln(u) / alpha).
// x / a for a posterior shape or count a: a product with the table's 1/a when a
// is an integer below 256 (within an ulp of the quotient), else the division
__device__ __forceinline__ double div_shape(double x, double a, const MathTab* __restrict__ T) {
  if (a >= 1.0 && a < 256.0 && a == floor(a)) return x * __ldg(&T->inv_int[(int)a]);
  return x / a;
}
__device__ __forceinline__ float div_shape(float x, float a, const MathTab* __restrict__) {
  return x / a;
}

template <typename R>
__device__ __forceinline__ R lomax(Stream& s, R alpha, R beta) {
  return beta * m_expm1(div_shape(neg_log_uniform<R>(s), alpha, s.tab));
}

// Poisson(lambda tau) with lambda ~ Gamma(alpha, rate beta) integrated out
// (negative binomial, p = beta / (beta + tau), q = tau / (beta + tau)): mean
// alpha tau / beta below 10 by sequential-search inversion of one uniform,
// P(0) = exp(-alpha log1p(tau / beta)), P(n + 1) = P(n) (q (alpha + n) / (n + 1)),
// at most 1000 terms; from 10 up the Gamma-Poisson mixture
// lambda' = Gamma(alpha, 1) / beta (alpha >= 1), then Poisson(lambda' tau).
template <typename R>
__device__ __noinline__ int neg_binomial(Stream& s, R alpha, R beta, R tau) {
  const R r = tau / beta;
  // FP64: one division for the mean and P(0); FP32: the mean as (alpha tau) / beta
  const R mean = sizeof(R) == 8 ? alpha * r : alpha * tau / beta;
  if (mean < (R)10.0) {
    const R u = uniform01<R>(s);
    const R l0 = alpha * m_log1p(r);
    R pk;
    if constexpr (sizeof(R) == 8)
      pk = exp_neg_int(l0, s.tab);  // integer pipes
    else
      pk = f32_exp(-l0);
    R acc = pk;
    if (!gt_nonneg(u, acc)) return 0;  // n = 0: q is not needed
    const R q = tau / (beta + tau);
    int k = 0;
    while (gt_nonneg(u, acc) && k < 1000) {
      pk = pk * div_shape(q * (alpha + (R)k), (R)(k + 1), s.tab);
      acc = acc + pk;
      k += 1;
    }
    return k;
  }
  const R lam = gamma_mt<R>(s, alpha) / beta;
  return poisson<R>(s, lam * tau);
}

// ---- warp / block primitives (integer, deterministic association order) ----
// Block max of an int over TPB threads; every thread gets the result.
template <int TPB>
__device__ __forceinline__ int block_max_int(int v, int* sh) {
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
  v = __reduce_max_sync(0xffffffffu, v);
  __syncthreads();
  if (lane == 0) sh[wid] = v;
  __syncthreads();
  int r = sh[0];
#pragma unroll
  for (int w = 1; w < TPB / 32; ++w) r = max(r, sh[w]);
  return r;
}

// Block inclusive prefix max of int64 keys over TPB threads.  `sh` >= TPB/32
// long longs.  Non-negative doubles order like their bit patterns, so this is
// also the prefix max of such doubles, on the integer pipes.
template <int TPB>
__device__ __forceinline__ long long block_incl_max_i64(long long v, long long* sh) {
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
#pragma unroll
  for (int o = 1; o < 32; o <<= 1) {
    const long long t = __shfl_up_sync(0xffffffffu, v, o);
    if (lane >= o) v = max(v, t);
  }
  if (TPB > 32) {
    __syncthreads();
    if (lane == 31) sh[wid] = v;
    __syncthreads();
    for (int w = 0; w < wid; ++w) v = max(v, sh[w]);
  }
  return v;
}

// Order-preserving int64 key of a double (not NaN): for x >= 0 its bits, for
// x < 0 its bits with the magnitude bits flipped; max of keys = key of max.
__device__ __forceinline__ long long order_key(double x) {
  long long b = __double_as_longlong(x);
  if ((b & 0x7FFFFFFFFFFFFFFFll) > 0x7FF0000000000000ll) b = (long long)0xFFF0000000000000ull;  // NaN as -inf
  return b >= 0 ? b : b ^ 0x7FFFFFFFFFFFFFFFll;
}
__device__ __forceinline__ double from_order_key(long long k) {
  return __longlong_as_double(k >= 0 ? k : k ^ 0x7FFFFFFFFFFFFFFFll);
}

// Warp max of doubles through their order keys (integer shuffles only).
__device__ __forceinline__ double warp_max_key(double x) {
  long long v = order_key(x);
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v = max(v, __shfl_xor_sync(0xffffffffu, v, o));
  return from_order_key(v);
}

// ---- fixed-point weights: w * 2^54 as int64 (tile-local scans) ----
// Weights relative to a tile's power-of-two reference lie in [0, 1], and a
// tile holds at most 256 particles, so its running sums stay below 2^62.
// Integer sums are exact and associative: every order of summation gives the
// same bits, and the running sums are non-decreasing by construction.
constexpr int kFixBits = 54;

// round(x * 2^54) for finite 0 <= x < 2^9 (integer operations only; below
// 2^-55 the result is 0).
__device__ __forceinline__ long long to_fix54(double x) {
  const long long b = __double_as_longlong(x);
  const int e = (int)(b >> 52);  // biased exponent; 0 for zero and subnormals
  if (b <= 0 || e == 0) return 0;
  const long long m = (b & 0x000FFFFFFFFFFFFFll) | 0x0010000000000000ll;  // x = m 2^(e-1075)
  const int sh = e - (1075 - kFixBits);                                     // x 2^54 = m 2^sh
  if (sh >= 0) return m << sh;
  const int rs = -sh;
  if (rs > 54) return 0;
  return (m + (1ll << (rs - 1))) >> rs;
}

// floor(x * 2^54) for any x: -1 below zero, LLONG_MAX from 2^9 up (above every
// tile sum), integer operations only.
__device__ __forceinline__ long long floor_fix54(double x) {
  const long long b = __double_as_longlong(x);
  if ((b & 0x7FFFFFFFFFFFFFFFll) == 0) return 0;  // +-0
  if (b < 0) return -1;
  const int e = (int)(b >> 52);
  if (e == 0) return 0;
  if (e >= 1023 + 9) return 0x7FFFFFFFFFFFFFFFll;
  const long long m = (b & 0x000FFFFFFFFFFFFFll) | 0x0010000000000000ll;
  const int sh = e - (1075 - kFixBits);
  if (sh >= 0) return m << sh;
  const int rs = -sh;
  return rs >= 63 ? 0 : (m >> rs);
}

// Block inclusive scan of int64 over TPB threads (exact).  `sh` >= TPB/32 long longs.
template <int TPB>
__device__ __forceinline__ long long block_incl_scan_i64(long long v, long long* sh) {
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
#pragma unroll
  for (int o = 1; o < 32; o <<= 1) {
    const long long t = __shfl_up_sync(0xffffffffu, v, o);
    if (lane >= o) v += t;
  }
  if (TPB == 32) return v;
  __syncthreads();
  if (lane == 31) sh[wid] = v;
  __syncthreads();
  if (wid == 0) {
    long long t = lane < TPB / 32 ? sh[lane] : 0;
#pragma unroll
    for (int o = 1; o < TPB / 32; o <<= 1) {
      const long long q = __shfl_up_sync(0xffffffffu, t, o);
      if (lane >= o) t += q;
    }
    const long long ex = __shfl_up_sync(0xffffffffu, t, 1);
    if (lane < TPB / 32) sh[lane] = lane ? ex : 0;
  }
  __syncthreads();
  return wid > 0 ? sh[wid] + v : v;
}

// Block max of doubles (no NaN) through their order keys: integer shuffles
// and compares only.  Every thread gets the result.  `sh` >= TPB/32 long longs.
template <int TPB>
__device__ __forceinline__ double block_max_key(double x, long long* sh) {
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
  long long v = order_key(x);
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v = max(v, __shfl_xor_sync(0xffffffffu, v, o));
  if (TPB > 32) {
    __syncthreads();
    if (lane == 0) sh[wid] = v;
    __syncthreads();
    v = sh[0];
#pragma unroll
    for (int w = 1; w < TPB / 32; ++w) v = max(v, sh[w]);
  }
  return from_order_key(v);
}

}  // namespace smc
