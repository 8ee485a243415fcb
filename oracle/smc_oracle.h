/*
 * smc_oracle.h -- interface of the CPU oracle for the particle-SMC sweep over
 * a PPL control-flow graph (Lunden et al., "Compiling Universal Probabilistic
 * Programming Languages with Efficient Parallel Sequential Monte Carlo
 * Inference", Section 3).
 *
 * TEST INFRASTRUCTURE ONLY.  The oracle is a plain, slow, single-threaded
 * restatement of Algorithm 1 (SMC over PCFGs) and of the models it runs.  It
 * shares no code with the CUDA library.  Only the test suite, the smoke check
 * and the benchmark's CPU-baseline leg may load it; the product path never
 * does.
 */
#ifndef SMC_ORACLE_H
#define SMC_ORACLE_H
#include <stdint.h>

#define ORC_OK 0
#define ORC_EINVAL (-1)
#define ORC_ENOMEM (-2)
#define ORC_EDEGENERATE (-4)
#define ORC_ESTEPLIMIT (-5)

#define ORC_LG 1
#define ORC_CRBD 2
#define ORC_RATESHIFT 3
#define ORC_GEOMETRIC 4
#define ORC_SEIR 5 /* the vector-borne disease SEIR model of Section 6.2 / Listing 2 */
#define ORC_CRBD_DS 6 /* CRBD with lambda and mu integrated out (static delayed sampling, Section 6.3) */

#define ORC_FP64 0
#define ORC_FP32 1 /* FP32 particle arithmetic, FP64 normaliser / scan / log Z */

typedef struct {
  int32_t kind;
  int32_t precision;
  /* linear-Gaussian (Eq. 2 family): x0~N(x0_mean,x0_sd), x=a x+b+N(0,q_sd), y~N(x,r_sd) */
  int32_t T;
  int32_t n_nodes;
  const double *obs;
  double x0_mean, x0_sd, a, b, q_sd, r_sd;
  /* birth-death tree models (Listing 1 and the rate-shift reading) */
  const int32_t *parent, *left, *right, *preorder;
  const double *age;
  double rho;
  double lambda_fixed, mu_fixed;  /* used when fixed_rates != 0 */
  double lambda_scale, mu_scale;  /* Gamma(1, scale) priors otherwise */
  double sigma;                   /* rate-shift log-normal sd */
  const double *fixed_mult;       /* rate-shift: per-node multipliers, or NULL */
  int32_t fixed_rates;
  int32_t depth_cap;              /* hidden-lineage recursion cap (frames) */
  int32_t call_limit;             /* undetected-calls per segment before a kill */
  int32_t lam_stack_cap;          /* rate-shift pending-rate stack capacity */
  /* weighted geometric test program (Fig. 2a) */
  double geo_p, geo_logw;
} orc_model;

typedef struct {
  int64_t N;
  uint64_t seed;
  uint32_t run_id;
  int32_t max_segments;
  const int32_t *follow_anc; /* [n_follow][N] ancestors from another implementation, or NULL */
  int32_t n_follow;
  int32_t pad_;
  /* ESS-triggered resampling: resample at a checkpoint only when ESS < ess_threshold N
   * (0: at every checkpoint) */
  double ess_threshold;
  const int32_t *follow_resampled; /* [n_follow_resampled] another implementation's decisions */
  int32_t n_follow_resampled;
  int32_t pad2_;
  /* Resume from a snapshot (0: a fresh run).  A snapshot is a run stopped by
   * max_segments after resume_k >= 1 segments: its outputs hold the population at
   * checkpoint resume_k - 1 before that checkpoint's resampling decision, in the
   * orc_out layouts below, and resume_log_z is its log_z_closed.  The resumed run
   * takes the decision at checkpoint resume_k - 1 and goes on with segment
   * resume_k, with the same seed and run_id: every draw is the one the
   * uninterrupted run makes, so it ends with the same results bit for bit.
   * max_segments still counts from segment 0. */
  int32_t resume_k;
  int32_t pad3_;
  const double *resume_logw;   /* [N] */
  const double *resume_real;   /* [n_real][N] (NULL when n_real = 0) */
  const int32_t *resume_int;   /* [n_int][N] */
  const double *resume_stack;  /* [lam_stack_cap][N] (rate-shift; else NULL) */
  double resume_log_z;
} orc_cfg;

typedef struct {
  double log_z;
  int64_t n_flagged;        /* resampled particles whose offset lies within 1e-12 N of a boundary */
  int64_t n_flag_mismatch;  /* follow mode: differing ancestors that were flagged */
  int64_t n_hard_mismatch;  /* follow mode: differing ancestors that were not flagged */
  int64_t n_overflow;       /* particles killed by the recursion-depth cap */
  int64_t n_limit;          /* particles killed by the per-segment call limit */
  int64_t n_ess_flagged;    /* ESS decisions within 1e-9 of the threshold */
  int64_t n_dec_flag_mismatch, n_dec_hard_mismatch;  /* follow mode: differing decisions */
  int32_t n_segments;
  int32_t n_resamples;
  /* caller-owned outputs (any may be NULL) */
  double *final_logw;   /* [N] */
  double *real_fields;  /* [n_real][N] (FP32 values widened exactly) */
  int32_t *int_fields;  /* [n_int][N]; field 0 is the block index (pc) */
  double *stack;        /* [lam_stack_cap][N] (rate-shift) */
  int32_t *ancestors;   /* [anc_capacity][N]: row k = the ancestors after checkpoint k
                           (the identity where the population was not resampled) */
  int32_t *resampled;   /* [anc_capacity] 1 where the population was resampled after checkpoint k */
  double *incr;         /* [incr_capacity] per-segment log-Z increments */
  int32_t anc_capacity;
  int32_t incr_capacity;
  /* log Z without the closure made only because the step limit ended the run
   * (equal to log_z otherwise): what a resumed run continues from */
  double log_z_closed;
} orc_out;

#ifdef __cplusplus
extern "C" {
#endif
void orc_philox4x32_10(const uint32_t ctr[4], const uint32_t key[2], uint32_t out[4]);
void orc_philox_many(int64_t n, const uint32_t *ctr, const uint32_t *key, uint32_t *out);
int orc_sample(int32_t dist, int32_t precision, double p1, double p2, uint64_t seed,
               uint32_t run_id, int64_t n, double *out, int32_t *blocks_used);
int orc_resample(const double *logw, int64_t N, double u, int32_t *anc, int32_t *flag,
                 double *incr, double *m_out, double *S_out);
int orc_smc_run(const orc_model *m, const orc_cfg *c, orc_out *o);
/* The FP32 mode's single-precision functions of (float)x[i], widened into y[i]:
 * fn 0 log, 1 exp, 2 cos(2 pi x), 3 log1p, 4 expm1, 5 log k! for k = (int)x[i]. */
int orc_mathf(int32_t fn, const double *x, double *y, int64_t n);
int orc_n_fields(const orc_model *m, int32_t *n_real, int32_t *n_int, int32_t *stack_cap);
#ifdef __cplusplus
}
#endif
#endif
