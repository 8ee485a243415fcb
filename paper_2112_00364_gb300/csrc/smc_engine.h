// smc_engine.h -- structures shared by the run, batch and server paths.
#pragma once
#include <cuda_runtime.h>

#include <cstdint>
#include <vector>

#include "../../include/smc.h"
#include "smc_combine.cuh"
#include "smc_models.cuh"

namespace smc {

constexpr int kMaxAncRows = 4096;
constexpr int kMaxSegments = 1 << 24;
constexpr int kUnboundedSegments = 1 << 20;
constexpr int64_t kMaxParticles = (int64_t)0x7fffffff - 256;

// Per-run device state (one struct per run, in the run's workspace).
struct RunState {
  double log_z, m, S;
  double log_z_closed;  // log Z without a closure made only because the step limit ended the run
  // the next search's scalars when the run combines in one CTA: S / N and
  // u S / N in 64.64 fixed point, and the boundary tolerance (units U)
  unsigned long long d_hi, d_lo, z0_hi, z0_lo;
  long long tolZ;
  unsigned long long n_near, n_overflow, n_limit;
  unsigned long long n_draws, n_blocks;  // Philox blocks drawn by the model, blocks executed
  int32_t done, status, n_segments, n_resamples;
  uint32_t arrive;
  int32_t kmax, G;        // the run's reference exponent and coarsening (one-CTA combine)
  int32_t resample;       // the one-CTA combine's decision for the next wave
  int32_t n_ess_near;     // ESS decisions within 1e-9 of the threshold
  // checking build (SMC_DEBUG_CHECKS): the first out-of-range access found and
  // skipped (code: 1 ancestor, 2 block index, 3 stack pointer, 4 dispatch), its
  // particle, and how many were found
  int32_t dbg_code, dbg_pad;
  long long dbg_index;
  unsigned long long dbg_count;
};

// Everything a CTA needs about its run (copied to shared memory per CTA).
struct RunDev {
  ModelDev md;
  StateView state[2];
  double* logw;       // [N] log-weights of the latest segment (f64; FP32 values widened)
  long long* E[2];    // [N] tile-local running sums of the weights x 2^54 (int64), double-buffered by segment parity
  TileRec* rec[2];    // [n_tiles] tile reductions, double-buffered by segment parity
  long long* tq[2];   // [n_tiles] ESS mode: the tiles' sums of squared weights (units 2^-54 of 2^(2 k_t))
  int32_t* dec;       // [max_segments] 1 where the population was resampled after checkpoint k
  long long* tile_O;  // [n_tiles + 1] offsets in the run's unit, O_T = S (runs combined in one CTA)
  int32_t* anc;       // ancestor rows
  double* incr;       // [max_segments] per-segment log-Z increments
  RunState* rs;
  double log_n;                // log N, computed on the host
  unsigned long long recip_n;  // floor((2^64 - 1) / N), the search scalars' divisor
  double ess_tau;       // 0: resample after every checkpoint; > 0: only when ESS < ess_tau N
  double ess_target;    // ess_tau N
  int N, n_tiles, tile, max_segments, record_all, anc_rows;
  unsigned start_wave;  // wave index of the run's segment 0 (segment k runs in wave start_wave + k)
  int redundant;        // combine a segment's tiles in every CTA of the next wave (else in the last CTA)
  int ess;              // ess_tau > 0 (an integer flag for the kernel's branches)
  uint32_t k0, k1;
  // resume from a snapshot: segment resume_k - 1 loads the population (device copies)
  int resume_k;
  const double* snap_logw;
  const double* snap_real;
  const int32_t* snap_int;
  const double* snap_stack;
};

struct Layout {
  size_t real[2], ints[2], stack[2], logw, E[2], rec[2], tq[2], dec, tO, rs, anc, incr,
      fin_real, fin_int, fin_stack, snap, total;
  int n_tiles, tile, anc_rows, max_segments;
};

// Device addresses of one wave's run table and per-bucket CTA maps.
struct WavePlan {
  const RunDev* runs = nullptr;
  const int2* maps[4] = {nullptr, nullptr, nullptr, nullptr};
  int n_ctas[4] = {0, 0, 0, 0};
  int kind = 0;  // the model of every run of the plan (SMC_MODEL_*), 0 when they differ
};

// An instantiated CUDA graph of a known-length sequence of waves and the wave
// plan it was captured for.
struct GraphCache {
  cudaGraphExec_t exec = nullptr;
  const RunDev* runs = nullptr;
  const int2* maps[4] = {nullptr, nullptr, nullptr, nullptr};
  int n_ctas[4] = {0, 0, 0, 0};
  int precision = -1, waves = 0;
};
void graph_cache_clear(GraphCache* g);

// Device blocks through a small cache of blocks freed by destroyed model
// handles (smc_engine.cu): *got receives the block's size (at least bytes).
cudaError_t block_alloc(void** p, size_t* got, size_t bytes);
void block_free(void* p, size_t bytes, int dev);

// A whole run in one launch (smc_small.cu): for runs of 32-particle tiles, at
// most small_run_max_tiles(kind, launch_mode) of them; launch_mode
// SMC_LAUNCH_ONE_CTA (grid 1) or SMC_LAUNCH_CLUSTER (one thread-block cluster).
int small_run_max_tiles(int kind, int launch_mode);
cudaError_t launch_small_run(int kind, int precision, int launch_mode, const RunDev* runs,
                             int n_tiles, cudaStream_t st);

}  // namespace smc

struct smc_model_s {
  smc_model_desc desc;
  smc::ModelDev md;
  int32_t n_real, n_int, stack_cap, n_segments_known;
  int32_t n_real_state;  // real fields kept in PSTATE (>= n_real; extra ones are internal)
  int dev = 0;                // the device the handle's memory is on
  void* dev_blob = nullptr;  // observations / tree arrays
  size_t blob_bytes = 0;
  void* ws = nullptr;        // cached workspace of smc_run
  size_t ws_bytes = 0;
  cudaEvent_t ev0 = nullptr, ev1 = nullptr;
  std::vector<cudaEvent_t> ev_seg;  // per-launch timing pairs (time_kernels)
  std::vector<char> staging;        // host staging of the run table
  char* pin = nullptr;              // smc_run's pinned copy of it (uploaded without a wait)
  size_t pin_bytes = 0;
  cudaEvent_t pin_ev = nullptr;     // recorded after that upload: the buffer is free again
  smc::GraphCache graph;            // smc_run's captured waves (SMC_LAUNCH_GRAPH)
};

namespace smc {

int model_fields(int kind, int* n_real, int* n_int);
// This device's log / exp tables (filled on first use per device).
smc_status math_table(const MathTab** out);
int tile_for(int64_t N);
int bucket_for(int tile);
// The combine placement of a run (the same results either way): in every CTA
// of the next wave when latency matters (`single`: a run alone, up to
// redundant_cap tiles), else only for runs of at most one tile per thread.
int combine_in_every_cta(int tile, int n_tiles, bool single);
Layout make_layout(const smc_model_s* m, const smc_run_cfg* c);
RunDev make_rundev(const smc_model_s* m, const smc_run_cfg* c, const Layout& Ly, char* ws);
size_t wave_meta_bytes(const std::vector<RunDev>& runs);
smc_status upload_wave(const std::vector<RunDev>& runs, void* meta, cudaStream_t st, WavePlan* W,
                       std::vector<char>* staging, char* pinned = nullptr);
cudaError_t launch_wave(const WavePlan& W, int precision, cudaStream_t st, unsigned wave);
// the waves of a plan whose runs all run the linear-Gaussian or the CRBD model
cudaError_t launch_wave_kind(const WavePlan& W, int precision, cudaStream_t st, unsigned wave);
int uniform_kind(const std::vector<RunDev>& runs);
smc_status collect_run(const smc_model_s* m, const smc_run_cfg* c, const Layout& Ly, char* ws,
                       const RunDev& A, const RunState& hrs, smc_result* r, cudaStream_t cs);
smc_status check_cfg(const smc_model_s* m, const smc_run_cfg* c);
smc_status check_result(const smc_result* r);

}  // namespace smc
