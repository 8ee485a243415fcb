/*
 * smc.h -- C ABI of the GB300 particle-SMC library.
 *
 * The library runs Sequential Monte Carlo over a PPL control-flow graph
 * (PCFG) as defined in Lunden et al., "Compiling Universal Probabilistic
 * Programming Languages with Efficient Parallel Sequential Monte Carlo
 * Inference" (ESOP 2022): a PCFG is the 6-tuple (B, S, sim, b0, b_stop, L)
 * of Section 3.1; Algorithm 1 (Section 3.2) propagates every particle with
 * sim() until all have reached a checkpoint, then resamples; the RootPPL
 * engine of Section 3.3 stops when every particle is at b_stop, stores the
 * particle state as separate arrays, duplicates particles with a custom
 * aligned copy, resamples systematically and estimates the normalising
 * constant.
 *
 * Conventions for every call:
 *   - Plain C types only; device pointers are CUDA device addresses; a
 *     `stream` argument is a cudaStream_t passed as void* (NULL = the legacy
 *     default stream).
 *   - The return value is an smc_status: 0 = success, < 0 = error (nothing
 *     useful was produced), > 0 = success with a warning.  No call aborts,
 *     traps or throws across the ABI; device-side failures come back as
 *     status words.  smc_last_error() gives a thread-local message for the
 *     last non-zero status of the calling thread.
 *   - The library never frees caller buffers.  Handles are opaque and are
 *     released only by their *_destroy call.
 *   - FP64 is used for the normaliser, the cumulative-weight scan and the
 *     log-Z accumulation in every precision mode.
 */
#ifndef SMC_H
#define SMC_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef int32_t smc_status;
#define SMC_OK 0
#define SMC_EINVAL (-1)       /* bad argument; nothing was launched */
#define SMC_ENOMEM (-2)       /* device or host allocation failed */
#define SMC_ECUDA (-3)        /* a CUDA runtime call failed (see smc_last_error) */
#define SMC_EDEGENERATE (-4)  /* every particle weight became zero; log Z = -inf */
#define SMC_ESTEPLIMIT (-5)   /* max_segments reached before every particle hit b_stop */
#define SMC_ETIMEOUT (-6)     /* a bounded wait gave up (server wait, device barrier) */
#define SMC_EBUSY (-7)        /* resource temporarily unavailable (server shutting down) */
#define SMC_ECANCELLED (-8)   /* the request was cancelled before it finished */
#define SMC_WKILLED 1         /* success; some particles were killed by the recursion-depth
                                 cap, the per-segment call limit or the stack capacity */

/* Built-in block tables (the B, S and sim of Section 3.1).
 *   LG         state-space model of Eq. 2 / Fig. 3, generalised to
 *              x0 ~ N(x0_mean, x0_sd^2), x_t = a x_{t-1} + b + q_sd z, y_t ~ N(x_t, r_sd^2);
 *              blocks: 0 init (jumps to iter without a checkpoint), 1 iter (checkpoint).
 *   CRBD       constant-rate birth-death model of Listing 1 on a fixed tree:
 *              block 0 draws the priors and weights by the correction factor,
 *              block 1 simulates one branch of the left-first preorder, including the
 *              hidden side lineages (simBranch / crbdGoesUndetected / iter) on an
 *              explicit per-particle stack, and weights lnProb1+lnProb2+lnProb3.
 *   RATESHIFT  CRBD with a per-branch LogNormal(0, sigma^2) multiplier on the birth rate,
 *              inherited from the parent branch; pending parent rates are kept on a
 *              PSTATE stack that resampling copies only up to its stack pointer.
 *   GEOMETRIC  the weighted geometric program of Fig. 2a with a checkpoint after each flip.
 * Every model uses b_stop = -1 as its block index. */
#define SMC_MODEL_LG 1
#define SMC_MODEL_CRBD 2
#define SMC_MODEL_RATESHIFT 3
#define SMC_MODEL_GEOMETRIC 4
#define SMC_MODEL_SEIR 5 /* vector-borne disease SEIR (Section 6.2, Listing 2): obs = daily
                            reports (-1: none), T = days; PSTATE ints: block index, hS hE hI
                            hR mS mE mI mR z; reals: hLambda hDelta hGamma mLambda mDelta rho */
#define SMC_MODEL_CRBD_DS 6 /* CRBD with static delayed sampling (Section 6.3): lambda and mu
                             stay Gamma(shape, rate) posteriors updated by conjugacy, every
                             rate-dependent draw from its predictive law (negative binomial
                             counts, Lomax lifetimes); needs the Gamma priors (fixed_rates = 0,
                             lambda_scale, mu_scale > 0); PSTATE reals: a_lambda b_lambda
                             a_mu b_mu; ints: block index */

#define SMC_PREC_FP64 0 /* FP64 particle arithmetic and log-weights */
#define SMC_PREC_FP32 1 /* FP32 particle arithmetic and log-weights; FP64 reductions */

#define SMC_MEM_HOST 0
#define SMC_MEM_DEVICE 1

#define SMC_LAUNCH_AUTO 0
#define SMC_LAUNCH_GRAPH 1
#define SMC_LAUNCH_ONE_CTA 2
#define SMC_LAUNCH_CLUSTER 3
#define SMC_LAUNCH_WAVES 4

#define SMC_MAX_DEPTH 64 /* largest hidden-lineage recursion cap the CRBD blocks accept */
/* Largest particle count of one run: ancestor indices are int32, and a run's
   last tile, rounded up to whole CTAs of at most 256 particles, stays below
   2^31.  smc_run and smc_run_batch return SMC_EINVAL above it. */
#define SMC_MAX_PARTICLES ((((int64_t)1) << 31) - 257)

typedef struct smc_model_s *smc_model_t;

/* Model description.  All pointers are HOST pointers; smc_model_register copies
 * what it needs into device memory owned by the model handle. */
typedef struct {
  int32_t kind;     /* SMC_MODEL_* */
  int32_t T;        /* LG: number of observations (= checkpoints) */
  int32_t n_nodes;  /* tree models: 2 * tips - 1 */
  int32_t fixed_rates;   /* tree models: 1 = use lambda_fixed / mu_fixed, 0 = Gamma priors */
  const double *obs;     /* LG: y_1..y_T, [T] */
  double x0_mean, x0_sd, a, b, q_sd, r_sd; /* LG parameters */
  /* tree arrays, root = node 0: parent[root] = -1, left/right = -1 at tips,
   * age = time before present (tips 0), preorder = left-first node order, root first */
  const int32_t *parent, *left, *right, *preorder;
  const double *age;
  double rho;                      /* sampling fraction */
  double lambda_fixed, mu_fixed;   /* fixed_rates = 1 */
  double lambda_scale, mu_scale;   /* fixed_rates = 0: lambda ~ Gamma(1, lambda_scale),
                                      mu ~ Gamma(1, mu_scale), shape-scale */
  double sigma;                    /* RATESHIFT: log-normal sd of the per-branch multiplier */
  const double *fixed_mult;        /* RATESHIFT: optional per-node multipliers [n_nodes], or NULL */
  int32_t depth_cap;               /* hidden-lineage recursion cap in frames, 1..SMC_MAX_DEPTH */
  int32_t call_limit;              /* undetected-lineage calls per particle per segment */
  int32_t lam_stack_cap;           /* RATESHIFT: pending-rate stack capacity (>= tree need) */
  int32_t pad_;
  double geo_p, geo_logw;          /* GEOMETRIC: heads probability, log weight per heads */
} smc_model_desc;

/* Per-run configuration. */
typedef struct {
  int64_t n_particles;   /* 1 <= N <= SMC_MAX_PARTICLES */
  uint64_t seed;         /* Philox key = (seed_lo32, seed_hi32 XOR run_id) */
  uint32_t run_id;
  int32_t precision;     /* SMC_PREC_* */
  int32_t max_segments;  /* 0 = the model's own segment count (unbounded models: 1 << 20) */
  int32_t record_all_ancestors; /* 1: keep every resampling's ancestors, 0: only the last */
  int32_t time_kernels;  /* 1: time every segment-kernel launch with CUDA events (counters) */
  int32_t launch_mode;   /* how the segments are launched; results are the same bits in
                            every mode:
                            SMC_LAUNCH_AUTO     (0, the default) SMC_LAUNCH_CLUSTER where it
                                                applies (and the GPU launches it), else
                                                SMC_LAUNCH_WAVES;
                            SMC_LAUNCH_WAVES    one launch per segment (wave) and CTA size,
                                                chained by programmatic dependent launch;
                            SMC_LAUNCH_GRAPH    the waves of a known-length run captured in
                                                one CUDA graph (on a stream other than the
                                                legacy default stream; else waves): smc_run
                                                keeps the graph in the model handle and
                                                launches it again while the workspace, N and
                                                precision stay the same, smc_run_batch
                                                captures per call (cfgs[0] decides);
                            SMC_LAUNCH_ONE_CTA  smc_run of a run of 32-particle tiles, at most
                                                32 of them (linear-Gaussian, geometric) or 16
                                                (the others), fresh (not resumed): every
                                                segment in one CTA and one launch, the CTA
                                                barrier as the checkpoint barrier (else
                                                waves);
                            SMC_LAUNCH_CLUSTER  smc_run of a run of 32-particle tiles, at most
                                                32 of them, fresh: every segment in one
                                                launch of one thread-block cluster (2 warps,
                                                i.e. 2 tiles, a CTA in clusters of up to 16
                                                CTAs, or 4 in up to 8 where the GPU does not
                                                schedule 16), the cluster barrier as the
                                                checkpoint barrier (else waves). */
  void *workspace;       /* optional caller-owned device workspace (>= smc_workspace_bytes);
                            NULL = the model handle allocates and caches one */
  size_t workspace_bytes;
  double ess_threshold;  /* adaptive resampling (Section 3.3): 0 = resample after every
                            checkpoint; tau > 0 = resample only when the effective sample
                            size (sum w)^2 / sum w^2 < tau N, otherwise the particles keep
                            their states and accumulated log-weights and the log-Z
                            increment waits for the next resampling or the end */
  /* Resume from a snapshot (smc_run only; resume_k = 0: a fresh run).  Between
   * checkpoints a run is its particles' states and log-weights, the log Z closed so
   * far and its segment index, and every draw comes from a counter, so a run stopped
   * by max_segments after k segments (SMC_ESTEPLIMIT) and resumed from its outputs
   * with the same model, N, seed, run_id, precision and ess_threshold ends exactly
   * as the uninterrupted run.  The snapshot arrays are that run's outputs, in the
   * layouts of smc_result (host or device memory, resume_where); resume_log_z is its
   * counters.log_z_closed.  The resumed run takes the resampling decision at
   * checkpoint k - 1 and goes on with segment k; max_segments still counts from
   * segment 0 (it must be 0 or >= k); its recorded ancestor rows and resampling
   * decisions before checkpoint k - 1 are zero.  Errors: SMC_EINVAL. */
  int32_t resume_k;
  int32_t resume_where;        /* SMC_MEM_HOST or SMC_MEM_DEVICE */
  const double *resume_logw;   /* [N] the snapshot's final_logw */
  const double *resume_real;   /* [n_real][N] its real_fields (NULL when n_real = 0) */
  const int32_t *resume_int;   /* [n_int][N] its int_fields */
  const double *resume_stack;  /* [stack_cap][N] its stack (RATESHIFT; else NULL) */
  double resume_log_z;         /* its counters.log_z_closed */
} smc_run_cfg;

/* Counters of one run (host struct, filled by smc_run before it returns). */
typedef struct {
  int32_t n_segments;       /* segments executed */
  int32_t n_resamples;      /* resampling steps executed */
  int64_t n_near_boundary;  /* resampled offsets within 1e-12 N of a cumulative-weight boundary */
  int64_t n_overflow;       /* particle-segments killed by the depth cap or stack capacity */
  int64_t n_limit;          /* particle-segments killed by the call limit */
  double device_ms;         /* GPU time of the run (CUDA events) */
  double kernel_ms;         /* time_kernels = 1: summed duration of the segment-kernel launches */
  int32_t kernel_launches;  /* segment-kernel launches of the run (one per wave and CTA size) */
  int32_t n_ess_near;       /* ess_threshold > 0: checkpoints whose ESS lay within 1e-9 of tau N */
  smc_status status;        /* this run's own status (0, SMC_WKILLED, SMC_EDEGENERATE,
                               SMC_ESTEPLIMIT) */
  int32_t pad2_;
  int64_t n_draws;          /* Philox blocks drawn by the model's SAMPLE statements, summed over
                               particles and segments (the resampling uniforms not included) */
  int64_t n_blocks;         /* basic-block executions, summed over particles and segments */
  double log_z_closed;      /* log Z without the closure made only because the step limit
                               ended the run (equal to log_z otherwise): what a resumed run
                               continues from */
  /* The checking build of the library (libsmc_debug.so, compiled with
   * SMC_DEBUG_CHECKS) checks every ancestor index against [0, N), every gathered
   * block index against the model's blocks and every gathered stack pointer
   * against the stack capacity; an access found out of range is skipped (the
   * particle is killed) and recorded here.  Always 0 in the release build. */
  int32_t debug_code;       /* first violation: 1 ancestor, 2 block index, 3 stack pointer,
                               4 dispatch; 0 = none */
  int32_t pad3_;
  int64_t debug_index;      /* the particle of the first violation */
  int64_t debug_count;      /* violations found */
} smc_counters;

/* Outputs of one run.  `where` says whether every pointer below is host or
 * device memory.  Any pointer may be NULL (that output is skipped). */
typedef struct {
  int32_t where;             /* SMC_MEM_HOST or SMC_MEM_DEVICE */
  int32_t ancestors_rows;    /* capacity of `ancestors` in rows of N */
  double *log_z;             /* [1] log of the normalising-constant estimate */
  double *final_logw;        /* [N] log-weights after the last segment (not resampled) */
  int32_t *ancestors;        /* [rows][N]: row k = the ancestors after checkpoint k (record_all;
                                the identity where the population was not resampled), or the
                                last checkpoint's in row 0 */
  double *real_fields;       /* [n_real][N] final real state fields, field-major, widened to f64 */
  int32_t *int_fields;       /* [n_int][N] final int fields; field 0 is the block index */
  double *stack;             /* [stack_cap][N] final PSTATE stack (RATESHIFT), entries >= sp are 0 */
  int32_t *resampled;        /* [rows] 1 where the population was resampled after checkpoint k
                                (record_all; else row 0 holds the last checkpoint's) */
  smc_counters counters;     /* filled on return */
} smc_result;

/* ---------------- tiling (the library's one tuned parameter) ----------------
 * A run of N particles is cut into tiles of consecutive particles, one CTA per
 * tile per wave.  The tile size is a function of N alone, from a table of N
 * bands: the band with the smallest n_max >= N gives tiles of
 * clamp(ceil(N / slots), tile_min, tile_max).  Since the tiling fixes how the
 * weights are rounded to their tile's reference, a run gives the same bits
 * alone, batched and served under one table.  The built-in table is data
 * written by the library's autotuner (sweeps of candidate bands timed on a
 * GB300). */
typedef struct {
  int64_t n_max;     /* the band holds runs of N <= n_max (the last band: >= SMC_MAX_PARTICLES) */
  int32_t slots;     /* >= 1 */
  int32_t tile_min;  /* 1 <= tile_min <= tile_max */
  int32_t tile_max;  /* <= 256 */
  int32_t pad_;
} smc_tile_band;

/* Replace the process's tile table (bands sorted by increasing n_max); NULL, 0
 * restores the built-in table.  For tuning: runs in flight keep the tiling they
 * started with; results of runs under different tables differ (within the
 * method's rounding, not bit for bit).  Errors: SMC_EINVAL. */
smc_status smc_set_tile_bands(const smc_tile_band *bands, int32_t n_bands);
/* The current table: up to `cap` bands into `out` (may be NULL), their number
 * into *n_bands.  Errors: SMC_EINVAL. */
smc_status smc_get_tile_bands(smc_tile_band *out, int32_t cap, int32_t *n_bands);
/* The tile size a run of n_particles gets now (0 if n_particles is out of range). */
int32_t smc_tile_size(int64_t n_particles);

/* Register a model: validates `d`, copies observations / tree arrays to device
 * memory owned by the returned handle.  Section 3.1 (the PCFG being run) and
 * Section 3.3 (observations as shared global constant data).
 * Errors: SMC_EINVAL (bad description), SMC_ENOMEM, SMC_ECUDA. */
smc_status smc_model_register(const smc_model_desc *d, smc_model_t *out);

/* Release a model handle and everything it owns.  NULL is ignored.  The caller
 * must ensure no run using the handle is in flight. */
void smc_model_destroy(smc_model_t m);

/* Shape of a model's PSTATE: number of real and int fields, stack capacity and
 * the number of checkpoints a run takes (0 if it is not known in advance). */
smc_status smc_model_info(smc_model_t m, int32_t *n_real, int32_t *n_int, int32_t *stack_cap,
                          int32_t *n_segments);

/* Device workspace a run of `c` on `m` needs, in bytes. */
smc_status smc_workspace_bytes(smc_model_t m, const smc_run_cfg *c, size_t *bytes);

/* Run Algorithm 1 with N particles on model m (Section 3.2) in the RootPPL loop
 * order (Section 3.3): every segment runs one fused CUDA kernel that gathers each
 * particle from its systematic-resampling ancestor, executes blocks until the next
 * checkpoint with per-warp PC-sorted dispatch, and reduces the population's weights
 * (FP64 log-sum-exp and prefix scan); the log-Z increment of every segment is added
 * and resampling stops once every particle is at b_stop.  The call enqueues on
 * `stream` and returns after the stream has completed the run (results valid).
 * A model handle runs one call at a time.
 * Errors: SMC_EINVAL, SMC_ENOMEM, SMC_ECUDA, SMC_EDEGENERATE (log_z = -inf),
 * SMC_ESTEPLIMIT.  Warning: SMC_WKILLED. */
smc_status smc_run(smc_model_t m, const smc_run_cfg *c, smc_result *r, void *stream);

/* Run n_runs independent SMC runs (Algorithm 1 each) in one sequence of waves:
 * every wave advances every unfinished run by one segment, all runs' tiles in the
 * same kernel launches, each run resampled by its own last-arriving CTA, so
 * uneven runs fill the GPU together instead of one after another.  ms[q],
 * cfgs[q], res[q] describe run q exactly as for smc_run (cfg.workspace is
 * ignored: the batch takes stream-ordered device memory for the call and returns
 * it).  Every run must use the same precision.  A run's results are identical
 * to what smc_run gives for the same model and configuration (its tiling
 * depends only on its own N).  Each run's own status is res[q].counters.status.
 * Returns SMC_OK once every run has finished, or a call-level error
 * (SMC_EINVAL, SMC_ENOMEM, SMC_ECUDA) with no results. */
smc_status smc_run_batch(const smc_model_t *ms, const smc_run_cfg *cfgs, smc_result *res,
                         int32_t n_runs, void *stream);

/* ---------------- continuous batching (serving) ----------------
 * A server owns a CUDA stream and a worker thread.  Requests (a model, a run
 * configuration and caller-owned result buffers) are queued by smc_server_submit
 * from any thread; the worker admits queued requests into the set of resident
 * runs whenever the resident-run cap and the device-memory budget allow, and
 * advances every resident run by one segment per wave (the same wave kernels as
 * smc_run_batch), so requests that arrive while others are on the GPU join the
 * running waves instead of waiting for them to finish.  Each run's population
 * stays in device memory across its checkpoints.  A finished run's outputs are
 * copied into its result buffers (stream-ordered; pinned host or device buffers
 * keep the worker from blocking) and its ticket completes.  A request's results
 * are identical to what smc_run gives for the same model and configuration.
 * The model handle and the result buffers must stay valid until the ticket is
 * done.  A request whose result collection fails completes with that error
 * (after every copy already queued into its buffers has ended) while the other
 * requests go on.  Fault injection for tests, on the host: when the environment
 * variable SMC_SERVER_FAIL_TICKET holds a ticket number at smc_server_create,
 * that ticket's retirement fails with SMC_ECUDA after its result copies were
 * queued.  The paper runs one SMC at a time; this layer is the build's serving
 * form of the Section 3.3 engine. */
typedef struct smc_server_s *smc_server_t;

typedef struct {
  int32_t precision;          /* SMC_PREC_*: every request of a server uses it */
  int32_t max_resident_runs;  /* cap on runs resident at once (0 = 4096) */
  int32_t poll_waves;         /* waves launched between looks at the finished runs (0 = 2: the
                                 host's per-look work then overlaps a queued wave; a finished
                                 run is noticed at most poll_waves waves late) */
  int32_t pad_;
} smc_server_cfg;

typedef struct {
  int64_t waves;           /* waves launched */
  int64_t completed;       /* requests finished */
  int64_t particle_steps;  /* particle-steps of finished requests */
  int32_t resident;        /* runs resident now */
  int32_t queued;          /* requests waiting for admission */
  smc_status worker_status;/* 0, or the error that stopped the worker */
  int32_t pad_;
} smc_server_stats_t;

/* Create a server on the current device with a device-memory budget (bytes) for
 * resident runs' workspaces.  Errors: SMC_EINVAL, SMC_ENOMEM, SMC_ECUDA. */
smc_status smc_server_create(size_t device_mem_budget, const smc_server_cfg *cfg,
                             smc_server_t *out);
/* Queue one request; *ticket identifies it.  Errors: SMC_EINVAL (bad arguments or a
 * precision other than the server's), SMC_ENOMEM (the request alone exceeds the
 * budget), SMC_EBUSY (server shutting down).  Never blocks on the GPU. */
smc_status smc_server_submit(smc_server_t s, smc_model_t m, const smc_run_cfg *c, smc_result *r,
                             uint64_t *ticket);
/* *done = 1 once the ticket finished; then returns the run's status. */
smc_status smc_server_poll(smc_server_t s, uint64_t ticket, int32_t *done);
/* Wait at most timeout_s seconds for the ticket (SMC_ETIMEOUT if it is not done);
 * returns the run's status and, if latency_s != NULL, submit-to-done seconds. */
smc_status smc_server_wait(smc_server_t s, uint64_t ticket, double timeout_s, double *latency_s);
/* Cancel a queued or resident request (it completes with SMC_ECANCELLED). */
smc_status smc_server_cancel(smc_server_t s, uint64_t ticket);
smc_status smc_server_stats(smc_server_t s, smc_server_stats_t *out);
/* Finish every queued and resident request, then stop the worker and free everything. */
void smc_server_destroy(smc_server_t s);

/* ---------------- resampling primitives on caller device buffers ----------------
 * These are the normaliser / scan / systematic search / gather of Section 3.3 as
 * standalone HBM-streaming kernels.  All pointers are device pointers. */

/* Scratch bytes smc_resample needs for a population of N: about 5 bytes per
 * particle, kept between its first and third kernel (each running sum's top 32
 * bits after normalising by its tile total's leading zeros, and the exact
 * running sum before every 8 particles), plus the per-tile records and
 * offsets. */
size_t smc_resample_workspace_bytes(int64_t N);

/* Systematic resampling of one population (Section 3.3, parallel systematic
 * resampling): with the power-of-two reference m = k ln 2 (k = max over tiles
 * of the tile's k_t >= ceil(max logw / ln 2), chosen from the log-weights' high
 * words),
 * S = sum exp(logw - m) and P_j the running sum, ancestors[i] = min{ j : P_j (N / S)
 * > i + u } (N - 1 if none); the log-Z increment is m + (log S - log N).  The sums
 * are exact integer sums of the weights rounded to 2^-50 of their tile's
 * power-of-two reference (each within one unit of the exact rounding).  logw [N] f64 in
 * (16-byte aligned), ancestors [N] int32 out, out3 [3] f64 out = {m, S, m + (log S
 * - log N)}, n_near [1] int64 out (offsets within 1e-12 N of a boundary).  u in
 * (0,1).  workspace: device memory of smc_resample_workspace_bytes(N) bytes,
 * 256-byte aligned.  Errors: SMC_EINVAL (N < 1, u outside (0,1), NULL pointer,
 * workspace too small or misaligned), SMC_ECUDA.  An all -inf population gives
 * ancestors = identity and out3 = {-inf, 0, -inf}. */
smc_status smc_resample(const double *logw, int64_t N, double u, int32_t *ancestors,
                        double *out3, int64_t *n_near, void *workspace, size_t workspace_bytes,
                        void *stream);

/* The paper has no counterpart to this entry point: it exists for callers that
 * cannot allocate device memory themselves (code whose device memory belongs to
 * another framework's pool, paths where cudaMalloc's implicit device-wide
 * synchronisation is not allowed, hosts that forbid allocation after start-up).
 * It computes exactly what smc_resample computes, but its tile scratch is a
 * fixed array compiled into the library (131,136 bytes, held on every GPU that
 * loads the library until the process exits) instead of a workspace argument,
 * and it calls no allocating routine.  Limit: N <= SMC_RESAMPLE_STATIC_MAX_N
 * (larger N returns SMC_EINVAL with a message).  The first call on each device
 * resolves the array's device address (cudaGetSymbolAddress, with that device
 * current) and, unless an earlier call of the library on that device did so,
 * uploads the library's math tables with a synchronous cudaMemcpyToSymbol,
 * which waits for the device; so make that first call before any stream
 * capture, on a path where such a wait is allowed.  All calls share
 * the array: calls that overlap on the GPU race and must be serialised by the
 * caller (e.g. one stream).  Arguments, layouts and other errors as for
 * smc_resample; n_near is zeroed on `stream` by the call. */
#define SMC_RESAMPLE_STATIC_MAX_N (((int64_t)1) << 24)
smc_status smc_resample_static(const double *logw, int64_t N, double u, int32_t *ancestors,
                               double *out3, int64_t *n_near, void *stream);

/* ---------------- one population sharded over ranks ----------------
 * Section 3.3's parallel systematic resampling of a population held by several
 * GPUs in consecutive slices: rank r holds particles [first_r, first_r +
 * n_local_r) of n_total, every slice starting on a whole tile of
 * SMC_RESAMPLE_TILE particles and every slice but the last holding whole tiles.
 * The exchange step between the ranks is the tiles' records:
 *   1. every rank: smc_shard_reduce on its slice writes its tiles' records;
 *   2. the ranks exchange the records (an all-gather in rank order: the records
 *      of the whole population in tile order, 16 bytes a tile);
 *   3. every rank: smc_shard_ancestors combines all records (the same integers,
 *      S, log-Z increment and search scalars on every rank) and searches the
 *      offsets its own tiles own, [range[0], range[1]): ancestors[i] for those i
 *      (global particle indices, all inside its slice);
 *   4. the new particle i, owned by the rank whose slice holds index i, copies
 *      the state of particle ancestors[i] from the rank that searched i
 *      (paper_2112_00364_gb300/shard.py exchanges the states).
 * The ancestors, S and the increment are those smc_resample gives for the
 * whole population on one GPU, bit for bit.  All pointers are device pointers. */
#define SMC_RESAMPLE_TILE 4096
/* Bytes of the records of a slice of n_local particles (16 per tile). */
size_t smc_shard_records_bytes(int64_t n_local);
/* Step 1: the tiles' records of a slice (logw [n_local] f64, 16-byte aligned;
 * records [smc_shard_records_bytes(n_local)], 16-byte aligned).
 * Errors: SMC_EINVAL, SMC_ECUDA. */
smc_status smc_shard_reduce(const double *logw, int64_t n_local, void *records, void *stream);
/* Workspace bytes of smc_shard_ancestors for a population of n_total. */
size_t smc_shard_workspace_bytes(int64_t n_total);
/* Step 3: logw [n_local] of the slice starting at particle `first`; records_all
 * [tiles of n_total] in tile order; u in (0,1) the checkpoint's uniform (the same
 * on every rank); ancestors [n_total] int32 (only [range[0], range[1]) written);
 * range [2] int64; out3 [3] f64 = {m, S, log-Z increment} as smc_resample; n_near
 * [1] int64 (this rank's near-boundary offsets, zeroed by the call); workspace of
 * smc_shard_workspace_bytes(n_total), 256-byte aligned.  Errors: SMC_EINVAL (a
 * slice not on whole tiles, bad sizes, NULL), SMC_ECUDA. */
smc_status smc_shard_ancestors(const double *logw, int64_t n_local, int64_t first,
                               const void *records_all, int64_t n_total, double u,
                               int32_t *ancestors, int64_t *range, double *out3, int64_t *n_near,
                               void *workspace, size_t workspace_bytes, void *stream);

/* Particle duplication with a stack-pointer-bounded copy (Section 3.3): for each
 * field f and particle i, dst[f][i] = src[f][anc[i]] (fields field-major, elem_bytes
 * 4 or 8 each); if sp != NULL, stack rows s >= sp[anc[i]] are not copied (they are
 * left as they were in dst).  Arrays: src/dst [n_fields][N], anc [N], sp [N] or NULL.
 * Errors: SMC_EINVAL, SMC_ECUDA. */
smc_status smc_gather(const void *src, void *dst, const int32_t *anc, const int32_t *sp,
                      int64_t N, int32_t n_fields, int32_t elem_bytes, void *stream);

/* ---------------- random-number parity hooks ---------------- */

/* Raw Philox4x32-10 blocks: out[i] = philox(ctr[i], key[i]); ctr [n][4], key [n][2],
 * out [n][4] uint32, device pointers.  Errors: SMC_EINVAL, SMC_ECUDA. */
smc_status smc_philox(const uint32_t *ctr, const uint32_t *key, uint32_t *out, int64_t n,
                      void *stream);

/* n variates of one recipe, variate i drawn from counter (i, 0, d, 0) with d from 0:
 * dist 0 uniform(0,1), 1 normal(p1, p2), 2 exponential(rate p1), 3 gamma(1, scale p1),
 * 4 uniform(p1, p2), 5 bernoulli(p1), 6 poisson(p1), 7 lognormal(0, p1), 8 binomial(n = p1,
 * p = p2), 9 beta(p1, p2), 10 gamma(shape p1 >= 1, scale 1), 11 negative binomial
 * (Poisson(lambda p2) with lambda ~ Gamma(shape p1 >= 1, rate 1) integrated out), 12 Lomax
 * (Exponential(mu) with mu ~ Gamma(shape p1, rate p2) integrated out).
 * out [n] f64 and blocks [n] int32 (Philox blocks consumed, may be NULL) are device
 * pointers.  Errors: SMC_EINVAL, SMC_ECUDA. */
smc_status smc_sample(int32_t dist, int32_t precision, double p1, double p2, uint64_t seed,
                      uint32_t run_id, int64_t n, double *out, int32_t *blocks, void *stream);

/* Device math parity hook: y[i] = f(x[i]) on the GPU for fn 0 = the table-driven
 * FP64 logarithm the samplers use, 1 = the table-driven FP64 exponential, 2 = the
 * CUDA library log, 3 = the CUDA library exp; for fn 4 and 5 x[i] holds 64 random
 * bits b (read as uint64) and y[i] = log u of the FP64 uniform u = ((b >> 11) | 1)
 * 2^-53, 4 = reduced and its log1p polynomial evaluated on the integer pipes (what
 * the samplers use), 5 = the table logarithm of u built as a double; for fn 6 and 7
 * y[i] holds (as int64
 * bits) the fixed-point weight round(e^x[i] 2^54) for x[i] <= 0, 6 = computed
 * on the integer pipes (what the segment kernel uses), 7 = the table exponential
 * rounded to the same grid; fn 8 gives round(e^x[i] 2^54) from the two-table
 * integer exponential, fn 9 round(e^x[i] 2^50) from it with the argument in
 * 2^-52 units; fn 23 gives round(e^x[i] 2^50) as smc_resample forms its weights
 * (the argument in 2^-52 units, a 9216-entry table of e^(-j/256) and a degree-5
 * polynomial); fn 10 gives e^-x[i]
 * (a double, x[i] in [0, 64)) from the same integer exponential, as the Poisson
 * sampler forms it.  fn 11..16 are the FP32 mode's own single-precision
 * functions of x[i] rounded to float (the result widened to f64): 11 log,
 * 12 exp, 13 cos(2 pi x), 14 log1p, 15 expm1, 16 log k! for k = (int)x[i];
 * fn 17..21 are CUDA's logf, expf, cospif(2x), log1pf, expm1f of the same
 * float arguments, for comparison; fn 22 reads pairs (x[2j], x[2j+1]) = (S, N) as
 * 64-bit integer patterns (S < 2^63, 1 <= N < 2^31) and writes (y[2j], y[2j+1]) =
 * floor(S 2^64 / N) as 64.64 fixed point (integer part, fraction bits), the
 * ratio the systematic search scales its offsets by (n even).  x, y [n] f64
 * device pointers.
 * Errors: SMC_EINVAL, SMC_ECUDA. */
smc_status smc_math_eval(int32_t fn, const double *x, double *y, int64_t n, void *stream);

/* Compute-peak probe (the roofline denominators of the arithmetic the path
 * uses; the paper has no counterpart): one launch of 8 x 256-thread CTAs per SM,
 * each thread running 8 independent dependency chains of `iters` steps of one
 * operation: kind 0 = FP64 fused multiply-add, 1 = FP32 fused multiply-add,
 * 2 = FP32 ex2.approx (special function unit), 3 = 32-bit integer multiply-add,
 * 4 = 64-bit unsigned multiply-high.  The caller times the launch (e.g. CUDA
 * events on `stream`); operations = smc_peak_probe_threads() x 8 x iters.
 * sink: device f64 [smc_peak_probe_threads()] (each thread's chain sum, so that
 * nothing is optimised away).  Errors: SMC_EINVAL (kind outside 0..4, iters < 1,
 * NULL sink), SMC_ECUDA. */
int64_t smc_peak_probe_threads(void);
smc_status smc_peak_probe(int32_t kind, int64_t iters, double *sink, void *stream);

/* Thread-local description of the calling thread's last error ("" if none). */
const char *smc_last_error(void);

/* Library version string. */
const char *smc_version(void);

#ifdef __cplusplus
}
#endif
#endif /* SMC_H */
