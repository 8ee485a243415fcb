/*
 * smc_oracle.c -- CPU oracle for the particle-parallel SMC sweep over a PPL
 * control-flow graph (PCFG), Lunden et al. 2022, Section 3.
 *
 * TEST INFRASTRUCTURE ONLY.  This is the plain, slow, single-threaded
 * restatement against which the CUDA library is checked.  It shares no code
 * with the CUDA path; only tests/, the smoke check and the benchmark's
 * CPU-baseline leg may load it.  Compile with -ffp-contract=off so that every
 * a*b+c below is two roundings unless written as fma().
 *
 * What each part follows:
 *   - Algorithm 1 (SMC over PCFGs) and the RootPPL inference loop of
 *     Section 3.3: init, propagate to the next checkpoint, stop when every
 *     particle is at b_stop, else resample and repeat; sim(b_stop,s) =
 *     (b_stop,s,true).
 *   - Normalising constant: log Z accumulates log((1/N) sum_n w_n) at every
 *     checkpoint (Section 3.3, "normalizing constants").
 *   - ESS-triggered resampling (Section 3.3, adaptive resampling based on the
 *     effective sample size): ESS = (sum w)^2 / sum w^2; the population is
 *     resampled only when ESS < tau N, otherwise the particles keep their
 *     weights, which accumulate until the next resampling, and log Z then
 *     gains log((1/N) sum_n W_n) of the accumulated weights (the paper gives
 *     no formula; this is the standard estimator for it).
 *   - Systematic resampling (Section 3.3): one uniform u per checkpoint,
 *     a_i = min{ j : N P_j / S > i + u }, P_j the running sum of weights.
 *   - Models: the state-space model of Eq. 2 / Fig. 3 (generalised to
 *     x_t = a x_{t-1} + b + q z), the CRBD model of Listing 1, a rate-shift
 *     variant of it, the weighted geometric program of Fig. 2a, the SEIR
 *     vector-borne disease model of Section 6.2 (Listing 2), and the CRBD
 *     model with static delayed sampling of Section 6.3 (lambda and mu kept
 *     as conjugate Gamma posteriors; the paper gives no formulas, the
 *     reading is the standard Gamma-Poisson / Gamma-Exponential conjugacy:
 *     draws from the predictive laws, each followed by its posterior update).
 *
 * Random numbers: counter-based Philox4x32-10 (Salmon et al., SC'11) with
 * key (seed_lo, seed_hi XOR run_id) and counter (particle slot n,
 * checkpoint index k, draw index d, stream tag); one 128-bit block per
 * variate.  Tag 0 = model draws, 1 = resampling uniform, 2 = rate-shift
 * multipliers.  Published definition, implemented here independently.
 */
#include "smc_oracle.h"

#include <math.h>
#include <stdlib.h>
#include <string.h>

#define PC_STOP (-1)

/* ------------------------- Philox4x32-10 ------------------------- */
#define PHILOX_M0 0xD2511F53u
#define PHILOX_M1 0xCD9E8D57u
#define PHILOX_W0 0x9E3779B9u
#define PHILOX_W1 0xBB67AE85u

void orc_philox4x32_10(const uint32_t ctr[4], const uint32_t key[2], uint32_t out[4]) {
  uint32_t c0 = ctr[0], c1 = ctr[1], c2 = ctr[2], c3 = ctr[3];
  uint32_t k0 = key[0], k1 = key[1];
  for (int round = 0; round < 10; round++) {
    if (round > 0) {
      k0 += PHILOX_W0;
      k1 += PHILOX_W1;
    }
    uint64_t p0 = (uint64_t)PHILOX_M0 * (uint64_t)c0;
    uint64_t p1 = (uint64_t)PHILOX_M1 * (uint64_t)c2;
    uint32_t hi0 = (uint32_t)(p0 >> 32), lo0 = (uint32_t)p0;
    uint32_t hi1 = (uint32_t)(p1 >> 32), lo1 = (uint32_t)p1;
    c0 = hi1 ^ c1 ^ k0;
    c1 = lo1;
    c2 = hi0 ^ c3 ^ k1;
    c3 = lo0;
  }
  out[0] = c0;
  out[1] = c1;
  out[2] = c2;
  out[3] = c3;
}

void orc_philox_many(int64_t n, const uint32_t *ctr, const uint32_t *key, uint32_t *out) {
  for (int64_t i = 0; i < n; i++) orc_philox4x32_10(ctr + 4 * i, key + 2 * i, out + 4 * i);
}

static void make_key(uint64_t seed, uint32_t run_id, uint32_t key[2]) {
  key[0] = (uint32_t)(seed & 0xffffffffu);
  key[1] = (uint32_t)(seed >> 32) ^ run_id;
}

typedef struct {
  uint32_t key[2];
  uint32_t n, k, d, tag;
} stream_t;

static void stream_init(stream_t *s, const uint32_t key[2], uint32_t n, uint32_t k, uint32_t tag) {
  s->key[0] = key[0];
  s->key[1] = key[1];
  s->n = n;
  s->k = k;
  s->d = 0;
  s->tag = tag;
}

static void next_block(stream_t *s, uint32_t w[4]) {
  uint32_t c[4] = {s->n, s->k, s->d, s->tag};
  orc_philox4x32_10(c, s->key, w);
  s->d += 1;
}

/* FP64 uniforms: the odd 53-bit integer ((w_hi:w_lo) >> 11) | 1 times 2^-53,
 * exact, strictly inside (0,1).  First uses (w1:w0), second (w3:w2). */
static double u_first_d(const uint32_t w[4]) {
  uint64_t x = ((uint64_t)w[1] << 32) | (uint64_t)w[0];
  return (double)((x >> 11) | 1u) * 0x1p-53;
}
static double u_second_d(const uint32_t w[4]) {
  uint64_t x = ((uint64_t)w[3] << 32) | (uint64_t)w[2];
  return (double)((x >> 11) | 1u) * 0x1p-53;
}
/* FP32 uniforms: the odd 24-bit integer (w >> 8) | 1 times 2^-24, from the high
 * word of the FP64 uniform's 64 bits: first w1, second w3.  An FP32 draw is then
 * the FP64 draw of the same counter to within 2^-24, so that FP32 and FP64 runs
 * of one seed can be compared result by result. */
static float u_first_f(const uint32_t w[4]) { return (float)((w[1] >> 8) | 1u) * 0x1p-24f; }
static float u_second_f(const uint32_t w[4]) { return (float)((w[3] >> 8) | 1u) * 0x1p-24f; }

/* run-level constants computed once in double */
typedef struct {
  double corr;   /* CRBD: (n_tips - 1) ln 2 - ln n_tips! */
  double lg_lc;  /* LG: log(r_sd) + 0.5 log(2 pi) */
} model_consts;

#define LN2_D 0.69314718055994530942
#define HALF_LOG_2PI_D 0.91893853320467274178

static int model_setup(const orc_model *m, model_consts *mc) {
  mc->corr = 0.0;
  mc->lg_lc = 0.0;
  if (m->kind == ORC_LG) {
    if (!m->obs || m->T <= 0 || !(m->r_sd > 0)) return ORC_EINVAL;
    mc->lg_lc = log(m->r_sd) + HALF_LOG_2PI_D;
  } else if (m->kind == ORC_CRBD || m->kind == ORC_RATESHIFT || m->kind == ORC_CRBD_DS) {
    if (m->n_nodes < 3 || !m->parent || !m->left || !m->age || !m->preorder) return ORC_EINVAL;
    if (m->kind == ORC_RATESHIFT && m->lam_stack_cap < 1) return ORC_EINVAL;
    /* delayed sampling integrates the Gamma priors out: no fixed rates */
    if (m->kind == ORC_CRBD_DS && (m->fixed_rates || !(m->lambda_scale > 0) || !(m->mu_scale > 0)))
      return ORC_EINVAL;
    int32_t tips = (m->n_nodes + 1) / 2;
    double lnfact = 0.0;
    for (int32_t i = 2; i <= tips; i++) lnfact = lnfact + log((double)i);
    mc->corr = (double)(tips - 1) * LN2_D - lnfact;
  } else if (m->kind == ORC_SEIR) {
    if (!m->obs || m->T <= 0) return ORC_EINVAL;
  } else if (m->kind != ORC_GEOMETRIC) {
    return ORC_EINVAL;
  }
  return ORC_OK;
}

/* ------------- normaliser and systematic resampling (always FP64) ------------- */

/* m = max_n logw_n; S = sum_n exp(logw_n - m) left to right;
 * increment = m + (log S - log N).  Returns nonzero if every weight is zero. */
static int normaliser(const double *lw, int64_t N, double *m, double *S, double *incr) {
  double mx = -INFINITY;
  for (int64_t i = 0; i < N; i++)
    if (lw[i] > mx) mx = lw[i];
  *m = mx;
  if (mx == -INFINITY) {
    *S = 0.0;
    *incr = -INFINITY;
    return 1;
  }
  double s = 0.0;
  for (int64_t i = 0; i < N; i++) s = s + exp(lw[i] - mx);
  *S = s;
  *incr = mx + (log(s) - log((double)N));
  return 0;
}

/* ESS = (sum_n w_n)^2 / sum_n w_n^2 with w_n = exp(logw_n - m), sums left to right */
static double ess_of(const double *lw, int64_t N, double mx, double S) {
  double q = 0.0;
  for (int64_t i = 0; i < N; i++) {
    const double w = exp(lw[i] - mx);
    q = q + w * w;
  }
  return (S * S) / q;
}

static double resample_uniform(const uint32_t key[2], uint32_t k) {
  uint32_t c[4] = {0u, k, 0u, 1u};
  uint32_t w[4];
  orc_philox4x32_10(c, key, w);
  return u_first_d(w);
}

#define BOUNDARY_EPS 1e-12

/* a_i = min{ j : q_j > i + u } with q_j = P_j * (N / S) and P_j the
 * left-to-right running sum of exp(logw_j - m); if no j qualifies
 * (rounding at the top) a_i = N - 1.  flag[i] = 1 when i + u lies within
 * 1e-12 N of q_{a_i} or of q_{a_i - 1}. */
static void systematic(const double *lw, int64_t N, double u, double mx, double S, int32_t *anc,
                       int32_t *flag) {
  double *q = malloc((size_t)N * sizeof(double));
  double r = (double)N / S;
  double P = 0.0;
  for (int64_t j = 0; j < N; j++) {
    P = P + exp(lw[j] - mx);
    q[j] = P * r;
  }
  const double tol = BOUNDARY_EPS * (double)N;
  int64_t j = 0;
  for (int64_t i = 0; i < N; i++) {
    double y = (double)i + u;
    while (j < N && !(q[j] > y)) j++;
    int64_t a = j < N ? j : N - 1;
    anc[i] = (int32_t)a;
    int f = fabs(q[a] - y) < tol;
    if (a > 0 && fabs(q[a - 1] - y) < tol) f = 1;
    flag[i] = f;
  }
  free(q);
}

int orc_resample(const double *logw, int64_t N, double u, int32_t *anc, int32_t *flag,
                 double *incr, double *m_out, double *S_out) {
  double mx, S, inc;
  if (N <= 0) return ORC_EINVAL;
  int r = normaliser(logw, N, &mx, &S, &inc);
  if (incr) *incr = inc;
  if (m_out) *m_out = mx;
  if (S_out) *S_out = S;
  if (r) return ORC_EDEGENERATE;
  int32_t *f = flag ? flag : malloc((size_t)N * sizeof(int32_t));
  systematic(logw, N, u, mx, S, anc, f);
  if (!flag) free(f);
  return ORC_OK;
}

int orc_n_fields(const orc_model *m, int32_t *n_real, int32_t *n_int, int32_t *stack_cap) {
  *stack_cap = 0;
  switch (m->kind) {
    case ORC_LG: *n_real = 1; *n_int = 1; return ORC_OK;
    case ORC_CRBD: *n_real = 2; *n_int = 1; return ORC_OK;
    case ORC_RATESHIFT: *n_real = 2; *n_int = 2; *stack_cap = m->lam_stack_cap; return ORC_OK;
    case ORC_GEOMETRIC: *n_real = 0; *n_int = 2; return ORC_OK;
    case ORC_SEIR: *n_real = 6; *n_int = 10; return ORC_OK;
    case ORC_CRBD_DS: *n_real = 4; *n_int = 1; return ORC_OK;
  }
  return ORC_EINVAL;
}

/* log k! : exact sums of logs below 32, Stirling's series for log Gamma(k+1)
 * above (x = k + 1: (x - 1/2) ln x - x + ln(2 pi)/2 + 1/(12x) - 1/(360x^3) +
 * 1/(1260x^5), truncation below 1e-13 there). */
static double lfact_table[32];
static int lfact_ready = 0;
static double lfact_d(int64_t k) {
  if (!lfact_ready) {
    double acc = 0.0;
    lfact_table[0] = 0.0;
    for (int i = 1; i < 32; i++) {
      acc = acc + log((double)i);
      lfact_table[i] = acc;
    }
    lfact_ready = 1;
  }
  if (k < 32) return lfact_table[k];
  const double x = (double)k + 1.0;
  const double ix = 1.0 / x, ix2 = ix * ix;
  const double series = ix * (1.0 / 12.0 - ix2 * (1.0 / 360.0 - ix2 * (1.0 / 1260.0)));
  return (x - 0.5) * log(x) - x + HALF_LOG_2PI_D + series;
}

/* --------------- FP32 elementary functions (FP32 mode) ---------------
 * The FP32-particle mode defines its log, exp, cos(2 pi u), log1p and expm1 as
 * the fixed sequences of single-precision operations below (fused
 * multiply-adds only where fmaf is written; the file is compiled with
 * -ffp-contract=off), so that its roundings are specified rather than left to
 * a math library: the GPU library performs the same operations and gets the
 * same bits.  The methods are textbook ones, with Taylor coefficients rounded
 * to float:
 *   log:   x = 2^e m with m in [sqrt(2)/2, sqrt(2)]; f = m - 1 (exact);
 *          log(1 + f) = 2 atanh(f / (2 + f)) = f - s (f - R), s = f / (2 + f),
 *          R = z (2/3 + 2z/5 + 2z^2/7 + 2z^3/9), z = s^2; plus e ln 2, ln 2 in
 *          two parts so that e times the first part is exact.
 *   exp:   x = n ln 2 + r, n = rint(x / ln 2); e^r = 1 + r + r^2 (1/2! + r/3! +
 *          ... + r^5/7!); times 2^n.
 *   cos(2 pi u): 4u = q + t exactly, |t| <= 1/2; cos(2 pi u) is cos(t pi/2),
 *          -sin, -cos or sin of it for q = 0, 1, 2, 3 (mod 4), each from its
 *          Taylor series in t (coefficients (pi/2)^n / n!).
 *   log1p: the log series on x itself when 1 + x lies in [sqrt(2)/2, sqrt(2)],
 *          else the log of u = 1 + x plus the rounding error of that sum over u.
 *   expm1: x + x^2 (1/2! + ... + x^6/8!) for |x| < ln 2 / 2, else
 *          2^n expm1(r) + (2^n - 1).
 *   log k!: lfact_d rounded to float below 32, Stirling's series in float above.
 * The constants are the float roundings of the exact values, as hex literals. */
#define F_LN2_HI 0x1.62e4p-1f
#define F_LN2_LO 0x1.7f7d1cp-20f
#define F_INV_LN2 0x1.715476p+0f

static float f_bits_to_float(uint32_t b) {
  float f;
  memcpy(&f, &b, sizeof f);
  return f;
}
static uint32_t f_float_to_bits(float f) {
  uint32_t b;
  memcpy(&b, &f, sizeof b);
  return b;
}

/* log(1 + f), f in [sqrt(2)/2 - 1, sqrt(2) - 1]: the atanh series */
static float f_log1p_series(float f) {
  const float s = f / (2.0f + f);
  const float z = s * s;
  float R = fmaf(z, 0x1.c71c72p-3f /* 2/9 */, 0x1.24924ap-2f /* 2/7 */);
  R = fmaf(R, z, 0x1.99999ap-2f /* 2/5 */);
  R = fmaf(R, z, 0x1.555556p-1f /* 2/3 */);
  R = z * R;
  return f - s * (f - R);
}

/* e ln 2 + l */
static float f_plus_e_ln2(int32_t e, float l) {
  if (e == 0) return l;
  const float fe = (float)e;
  const float lo = fmaf(fe, F_LN2_LO, l);
  return fe * F_LN2_HI + lo;
}

/* split a positive normal float into 2^e m with m in [sqrt(2)/2, sqrt(2)] */
static float f_split(uint32_t bits, int32_t *e) {
  const uint32_t frac = bits & 0x7fffffu;
  *e = (int32_t)(bits >> 23) - 127;
  if (frac > 0x3504f3u) { /* m above float(sqrt 2): halve it */
    *e += 1;
    return f_bits_to_float(frac | (126u << 23));
  }
  return f_bits_to_float(frac | (127u << 23));
}

static float orc_logf(float x) {
  if (!(x > 0.0f)) return x == 0.0f ? -INFINITY : NAN;
  if (isinf(x)) return x;
  int32_t extra = 0;
  if (x < 0x1p-126f) { /* subnormal */
    x = x * 0x1p24f;
    extra = -24;
  }
  int32_t e;
  const float m = f_split(f_float_to_bits(x), &e);
  return f_plus_e_ln2(e + extra, f_log1p_series(m - 1.0f));
}

/* e^r - 1 - r as r^2 (1/2! + r/3! + ...), up to r^5/7! or, with deg8, r^6/8! */
static float f_exp_tail(float r, int deg8) {
  float q = 0x1.a01a02p-13f; /* 1/7! */
  if (deg8) q = fmaf(r, 0x1.a01a02p-16f /* 1/8! */, q);
  q = fmaf(q, r, 0x1.6c16c2p-10f); /* 1/6! */
  q = fmaf(q, r, 0x1.111112p-7f);  /* 1/5! */
  q = fmaf(q, r, 0x1.555556p-5f);  /* 1/4! */
  q = fmaf(q, r, 0x1.555556p-3f);  /* 1/3! */
  q = fmaf(q, r, 0x1p-1f);         /* 1/2! */
  return (r * r) * q;
}

static float f_pow2(int32_t n) { /* 2^n, n in [-126, 127] */
  return f_bits_to_float((uint32_t)(n + 127) << 23);
}

static float orc_expf(float x) {
  if (isnan(x)) return x;
  if (x > 89.0f) return INFINITY;
  if (x < -104.0f) return 0.0f;
  const float nf = rintf(x * F_INV_LN2);
  float r = fmaf(-nf, F_LN2_HI, x);
  r = fmaf(-nf, F_LN2_LO, r);
  const float y = 1.0f + (r + f_exp_tail(r, 0));
  const int32_t n = (int32_t)nf;
  if (n > 127) return (y * 2.0f) * f_pow2(n - 1);
  if (n < -126) return (y * f_pow2(n + 100)) * 0x1p-100f;
  return y * f_pow2(n);
}

/* cos(2 pi u) for u in [0, 1] */
static float orc_cos2pif(float u) {
  const float v = 4.0f * u;
  const float qf = rintf(v);
  const float t = v - qf;
  const float z = t * t;
  const int32_t quad = (int32_t)qf & 3;
  if (quad == 0 || quad == 2) {
    float c = fmaf(z, -0x1.a6d1f2p-16f, 0x1.e1f506p-11f); /* (pi/2)^10/10!, ^8/8! */
    c = fmaf(c, z, -0x1.55d3c8p-6f);                      /* (pi/2)^6/6! */
    c = fmaf(c, z, 0x1.03c1f0p-2f);                       /* (pi/2)^4/4! */
    c = fmaf(c, z, -0x1.3bd3ccp+0f);                      /* (pi/2)^2/2! */
    const float cv = fmaf(z, c, 1.0f);
    return quad == 0 ? cv : -cv;
  }
  float p = fmaf(z, 0x1.507834p-13f, -0x1.32d2ccp-8f); /* (pi/2)^9/9!, ^7/7! */
  p = fmaf(p, z, 0x1.466bc6p-4f);                      /* (pi/2)^5/5! */
  p = fmaf(p, z, -0x1.4abbcep-1f);                     /* (pi/2)^3/3! */
  /* t pi/2 with pi/2 = 0x1.921fb6p+0 - 0x1.777a5cp-25 */
  const float inner = fmaf(t * z, p, t * -0x1.777a5cp-25f);
  const float sv = fmaf(t, 0x1.921fb6p+0f, inner);
  return quad == 1 ? -sv : sv;
}

static float orc_log1pf(float x) {
  if (!(x > -1.0f)) return x == -1.0f ? -INFINITY : NAN;
  if (isinf(x)) return x;
  if (x >= -0x1.2bec34p-2f && x <= 0x1.a8279ap-2f) return f_log1p_series(x);
  const float u = 1.0f + x;
  float err; /* the rounding error of 1 + x, exact: the larger operand first */
  if (x > 1.0f)
    err = 1.0f - (u - x);
  else
    err = x - (u - 1.0f);
  const float c = err / u;
  int32_t e;
  const float m = f_split(f_float_to_bits(u), &e);
  return f_plus_e_ln2(e, f_log1p_series(m - 1.0f) + c);
}

static float orc_expm1f(float x) {
  if (isnan(x)) return x;
  if (x > 89.0f) return INFINITY;
  if (x < -104.0f) return -1.0f;
  if (fabsf(x) < 0x1.62e430p-2f) return x + f_exp_tail(x, 1);
  const float nf = rintf(x * F_INV_LN2);
  float r = fmaf(-nf, F_LN2_HI, x);
  r = fmaf(-nf, F_LN2_LO, r);
  const float em = r + f_exp_tail(r, 1);
  const int32_t n = (int32_t)nf;
  if (n > 127) return (em + 1.0f) * 2.0f * f_pow2(n - 1);
  const float p2 = f_pow2(n < -126 ? -126 : n);
  return fmaf(p2, em, p2 - 1.0f);
}

static double lfact_d(int64_t k);

static float orc_lfactf(int32_t k) {
  if (k < 32) return (float)lfact_d(k < 0 ? 0 : k);
  const float x = (float)k + 1.0f;
  const float ix = 1.0f / x;
  const float ix2 = ix * ix;
  const float series = ix * (0x1.555556p-4f - ix2 * (0x1.6c16c2p-9f - ix2 * 0x1.a01a02p-11f));
  const float a = (x - 0.5f) * orc_logf(x);
  const float b = a - x;
  const float c = b + 0x1.d67f1cp-1f; /* log(2 pi) / 2 */
  return c + series;
}

/* ------------------ precision instantiations ------------------ */
#define R double
#define SFX(x) x##_d
#define LOGR log
#define EXPR exp
#define LOG1PR log1p
#define EXPM1R expm1
#define SQRTR sqrt
#define FMAR fma
#define FABSR fabs
#define FLOORR floor
#define LFACTR(k) lgamma((k) + 1.0)
#define COS2PIR(u) cos(6.28318530717958647692 * (u))
#define LN2R LN2_D
#include "smc_oracle_prec.inc"
#undef R
#undef SFX
#undef LOGR
#undef EXPR
#undef LOG1PR
#undef EXPM1R
#undef SQRTR
#undef FMAR
#undef FABSR
#undef FLOORR
#undef LFACTR
#undef COS2PIR
#undef LN2R

#define R float
#define SFX(x) x##_f
#define LOGR orc_logf
#define EXPR orc_expf
#define LOG1PR orc_log1pf
#define EXPM1R orc_expm1f
#define SQRTR sqrtf
#define FMAR fmaf
#define FABSR fabsf
#define FLOORR floorf
#define LFACTR(k) orc_lfactf((int32_t)(k))
#define COS2PIR(u) orc_cos2pif(u)
#define LN2R 0.693147182f
#include "smc_oracle_prec.inc"

/* ------------------------- exported ------------------------- */

int orc_sample(int32_t dist, int32_t precision, double p1, double p2, uint64_t seed,
               uint32_t run_id, int64_t n, double *out, int32_t *blocks_used) {
  uint32_t key[2];
  make_key(seed, run_id, key);
  if (precision == ORC_FP64) return sample_d(dist, p1, p2, key, n, out, blocks_used);
  if (precision == ORC_FP32) return sample_f(dist, p1, p2, key, n, out, blocks_used);
  return ORC_EINVAL;
}

int orc_mathf(int32_t fn, const double *x, double *y, int64_t n) {
  for (int64_t i = 0; i < n; i++) {
    const float v = (float)x[i];
    float r;
    switch (fn) {
      case 0: r = orc_logf(v); break;
      case 1: r = orc_expf(v); break;
      case 2: r = orc_cos2pif(v); break;
      case 3: r = orc_log1pf(v); break;
      case 4: r = orc_expm1f(v); break;
      case 5: r = orc_lfactf((int32_t)x[i]); break;
      default: return ORC_EINVAL;
    }
    y[i] = (double)r;
  }
  return ORC_OK;
}

int orc_smc_run(const orc_model *m, const orc_cfg *c, orc_out *o) {
  if (!m || !c || !o || c->N <= 0 || c->N > 0x7fffffff) return ORC_EINVAL;
  if (m->depth_cap < 0 || m->call_limit < 0) return ORC_EINVAL;
  if (c->resume_k < 0) return ORC_EINVAL;
  if (c->resume_k > 0) {
    int32_t n_real, n_int, cap;
    if (orc_n_fields(m, &n_real, &n_int, &cap)) return ORC_EINVAL;
    if (!c->resume_logw || !c->resume_int || (n_real > 0 && !c->resume_real) ||
        (cap > 0 && !c->resume_stack) || c->resume_k > c->max_segments)
      return ORC_EINVAL;
  }
  if (m->precision == ORC_FP64) return smc_run_d(m, c, o);
  if (m->precision == ORC_FP32) return smc_run_f(m, c, o);
  return ORC_EINVAL;
}
