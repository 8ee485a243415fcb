// smc_engine.cu -- model registration, smc_run and smc_run_batch: Algorithm 1
// (SMC over PCFGs) in the RootPPL loop order of Section 3.3.
//
// Execution is organised in waves.  One wave advances every resident run by
// one segment; it is one launch of wave_kernel per block-size bucket.  Each
// CTA of a wave owns one tile (a run and a contiguous slice of its particles,
// one particle per thread):
//   prologue  (segment k > 0) the previous segment's tiles combined into exact
//             integer offsets (in every CTA, or read from the run's last CTA of
//             the previous wave, smc_combine.cuh), log Z increment and the ESS
//             decision; when resampling, the systematic search for each
//             particle's ancestor a_i = min{ j : P_j > z_i } with z_i = (i + u)
//             S / N in 64.64 fixed point, then the particle duplication of
//             Section 3.3: the ancestor's SoA fields are read straight into
//             registers (the gather is fused into the load); a PSTATE stack is
//             copied only up to its stack pointer;
//   segment   blocks run until the next checkpoint with per-warp PC-sorted
//             dispatch (smc_models.cuh); draws from Philox counters;
//   epilogue  per warp, as soon as its particles are done: the warp's max M_w,
//             its power-of-two reference k_w = ceil(M_w / ln 2), and each weight
//             round(exp(logw_j - k_w ln 2) 2^54) on the integer pipes (an FP32
//             log-weight is exact as a double, so both precisions share it);
//             after the tile barrier the tile reference k_t = max k_w, each
//             weight shifted exactly to it, the tile's integer running sums E_j
//             (the next segment's search keys) and its record {total, k_t,
//             alive}; for runs combined in one CTA the run's last CTA to finish
//             forms the offsets for the next wave.
// The combine brings every tile total to the run's reference 2^k_max and a
// common unit with a coarsening G that keeps S in [2^61, 2^62]: the offsets O_t
// and S are exact integers, so the result does not depend on the order of the
// sums.  A run stops after the segment in which every particle reached b_stop
// (no resampling after it); its later CTAs return at once.
//
// A run's tile size depends only on its N (tile = ceil(N / 456) clamped to
// 32..256, 456 = 152 SMs x 3 CTAs), so a run gives the same bits alone and in a
// batch.  The CTA size of a run is the smallest of 32/64/128/256 threads that
// holds its tile; runs of different CTA sizes are launched as separate kernels
// of the same wave.
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <cstring>
#include <iterator>
#include <mutex>
#include <new>
#include <vector>

#include "smc_device.cuh"
#include "smc_engine.h"
#include "smc_internal.h"
#include "smc_models.cuh"
#include "smc_step.cuh"

namespace smc {

// Final outputs: real fields widened to f64, int fields, stack rows with
// entries at or above the stack pointer zeroed.
template <typename R>
__global__ void finalize_kernel(StateView S, int N, int n_real, int n_int, int cap, double* real_out,
                                int32_t* int_out, double* stack_out) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= N) return;
  if (real_out)
    for (int f = 0; f < n_real; ++f) real_out[(size_t)f * N + i] = (double)S.rf<R>(f, i, N);
  if (int_out)
    for (int f = 0; f < n_int; ++f) int_out[(size_t)f * N + i] = S.inf_(f, i, N);
  if (stack_out && cap > 0) {
    const int sp = S.inf_(1, i, N);
    for (int r = 0; r < cap; ++r)
      stack_out[(size_t)r * N + i] = r < sp ? (double)S.st<R>(r, i, N) : 0.0;
  }
}

// ------------------------------------------------------------------------
// host side
// ------------------------------------------------------------------------

__device__ MathTab g_math_tab;

namespace {
std::mutex g_tab_mu;
const MathTab* g_tab_ptr[128] = {nullptr};

// Device blocks kept after the model handle that owned them is destroyed, so
// that registering a model and running it (a caller that builds a model per
// request) reuses a block instead of a cudaMalloc / cudaFree pair, which
// synchronise the device.  Blocks up to 256 MB, 1 GB and 32 blocks in all;
// a failed cudaMalloc frees the device's kept blocks and tries once more.
struct KeptBlock {
  int dev;
  void* p;
  size_t bytes;
};
std::mutex g_kept_mu;
std::vector<KeptBlock> g_kept;
constexpr size_t kKeepMaxBlock = 256ull << 20, kKeepMaxTotal = 1ull << 30, kKeepMaxCount = 32;

void kept_flush(int dev) {
  std::lock_guard<std::mutex> lock(g_kept_mu);
  for (size_t q = 0; q < g_kept.size();) {
    if (g_kept[q].dev == dev) {
      cudaFree(g_kept[q].p);
      g_kept.erase(g_kept.begin() + (long)q);
    } else {
      ++q;
    }
  }
}
}  // namespace

cudaError_t block_alloc(void** p, size_t* got, size_t bytes) {
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return e;
  {
    std::lock_guard<std::mutex> lock(g_kept_mu);
    long best = -1;
    for (size_t q = 0; q < g_kept.size(); ++q) {
      const KeptBlock& b = g_kept[q];
      if (b.dev == dev && b.bytes >= bytes && b.bytes <= 2 * bytes &&
          (best < 0 || b.bytes < g_kept[(size_t)best].bytes))
        best = (long)q;
    }
    if (best >= 0) {
      *p = g_kept[(size_t)best].p;
      *got = g_kept[(size_t)best].bytes;
      g_kept.erase(g_kept.begin() + best);
      return cudaSuccess;
    }
  }
  e = cudaMalloc(p, bytes);
  if (e == cudaErrorMemoryAllocation) {
    cudaGetLastError();
    kept_flush(dev);
    e = cudaMalloc(p, bytes);
  }
  if (e == cudaSuccess) *got = bytes;
  return e;
}

void block_free(void* p, size_t bytes, int dev) {
  if (!p) return;
  if (bytes <= kKeepMaxBlock) {
    std::lock_guard<std::mutex> lock(g_kept_mu);
    size_t total = bytes;
    for (const KeptBlock& b : g_kept) total += b.bytes;
    // make room by freeing the oldest kept blocks of this device
    for (size_t q = 0; q < g_kept.size() && (total > kKeepMaxTotal || g_kept.size() >= kKeepMaxCount);) {
      if (g_kept[q].dev == dev) {
        total -= g_kept[q].bytes;
        cudaFree(g_kept[q].p);
        g_kept.erase(g_kept.begin() + (long)q);
      } else {
        ++q;
      }
    }
    if (total <= kKeepMaxTotal && g_kept.size() < kKeepMaxCount) {
      g_kept.push_back(KeptBlock{dev, p, bytes});
      return;
    }
  }
  cudaFree(p);
}

// The table entries are computed on the host in double (glibc log1p / exp2,
// correctly rounded division) and copied once to each device that uses them.
smc_status math_table(const MathTab** out) {
  int dev = -1;
  SMC_CUDA_TRY(cudaGetDevice(&dev));
  if (dev < 0 || dev >= 128) return set_error(SMC_EINVAL, "device ordinal %d out of range", dev);
  std::lock_guard<std::mutex> lock(g_tab_mu);
  if (!g_tab_ptr[dev]) {
    MathTab h;
    for (int j = 0; j < 192; ++j) {
      h.inv_f_q62[j] = j >= 90 ? (unsigned long long)std::llroundl(std::ldexp(128.0L / j, 62)) : 0ull;
      h.log_f[j] = j ? std::log((double)j / 128.0) : 0.0;
      h.inv_f[j] = j ? 128.0 / (double)j : 0.0;
      h.inv_f52[j] = std::ldexp(h.inv_f[j], -52);
      h.inv_f53[j] = std::ldexp(h.inv_f[j], -53);
    }
    for (int j = 0; j < 32; ++j) h.exp2_j[j] = std::exp2((double)j / 32.0);
    // 2^(-j/m) 2^63 rounded; j = 0 is 2^63 itself, outside the signed range
    auto q63 = [](int j, int m) -> unsigned long long {
      if (j == 0) return 1ull << 63;
      return (unsigned long long)std::llroundl(std::ldexp(std::exp2l(-(long double)j / m), 63));
    };
    for (int j = 0; j < 128; ++j) h.exp2_neg_q63[j] = q63(j, 128);
    for (int j = 0; j < 64; ++j) {
      h.exp2_neg64_q63[j] = q63(j, 64);
      h.exp2_neg4096_q63[j] = q63(j, 4096);
    }
    {
      double acc = 0.0;
      h.lfact[0] = 0.0;
      for (int j = 1; j < 32; ++j) {
        acc = acc + std::log((double)j);
        h.lfact[j] = acc;
      }
    }
    h.inv_int[0] = 0.0;
    for (int k = 1; k < 256; ++k) h.inv_int[k] = 1.0 / (double)k;
    // e^(-j/256) 2^56 from the long-double exponential (64 or more significand
    // bits): within a fraction of a unit of the exact value before rounding
    for (int j = 0; j < kRsExpPad; ++j)
      h.rs_exp_q56[j] = j < kRsExpN ? (unsigned long long)std::llroundl(
                                          std::ldexp(std::exp(-(long double)j / 256.0L), 56))
                                    : 0ull;
    SMC_CUDA_TRY(cudaMemcpyToSymbol(g_math_tab, &h, sizeof(MathTab)));
    void* p = nullptr;
    SMC_CUDA_TRY(cudaGetSymbolAddress(&p, g_math_tab));
    g_tab_ptr[dev] = (const MathTab*)p;
  }
  *out = g_tab_ptr[dev];
  return SMC_OK;
}

void graph_cache_clear(GraphCache* g) {
  if (g->exec) cudaGraphExecDestroy(g->exec);
  *g = GraphCache();
}

int model_fields(int kind, int* n_real, int* n_int) {
  switch (kind) {
    case SMC_MODEL_LG: *n_real = 1; *n_int = 1; return 0;
    case SMC_MODEL_CRBD: *n_real = 2; *n_int = 1; return 0;
    case SMC_MODEL_RATESHIFT: *n_real = 2; *n_int = 2; return 0;
    case SMC_MODEL_GEOMETRIC: *n_real = 0; *n_int = 2; return 0;
    case SMC_MODEL_SEIR: *n_real = 6; *n_int = 10; return 0;
    case SMC_MODEL_CRBD_DS: *n_real = 4; *n_int = 1; return 0;
  }
  return -1;
}

// ---- tiling: a function of N alone, from a table of N bands ----
// The built-in table is data written by the autotuner (autotune.py sweeps the
// candidate rules per band on a GB300 and writes smc_tile_table.inc); a band
// {n_max, slots, tile_min, tile_max} gives a run of N <= n_max particles tiles
// of clamp(ceil(N / slots), tile_min, tile_max) particles.  Because the tile of
// a run depends on its N alone, a run gives the same bits alone, batched and
// served.  smc_set_tile_bands replaces the table for the process (tuning).
namespace {
constexpr smc_tile_band kBuiltinBands[] = {
#include "smc_tile_table.inc"
};
std::mutex g_band_mu;
std::vector<smc_tile_band> g_bands(std::begin(kBuiltinBands), std::end(kBuiltinBands));

smc_status check_bands(const smc_tile_band* b, int n) {
  if (n < 1 || n > 64) return set_error(SMC_EINVAL, "n_bands must be in 1..64");
  for (int i = 0; i < n; ++i) {
    if (b[i].slots < 1) return set_error(SMC_EINVAL, "band %d: slots must be >= 1", i);
    if (b[i].tile_min < 1 || b[i].tile_min > b[i].tile_max || b[i].tile_max > 256)
      return set_error(SMC_EINVAL, "band %d: need 1 <= tile_min <= tile_max <= 256", i);
    if (i > 0 && b[i].n_max <= b[i - 1].n_max)
      return set_error(SMC_EINVAL, "band n_max must increase");
  }
  if (b[n - 1].n_max < kMaxParticles)
    return set_error(SMC_EINVAL, "the last band must reach SMC_MAX_PARTICLES");
  return SMC_OK;
}
}  // namespace

int tile_for(int64_t N) {
  std::lock_guard<std::mutex> lock(g_band_mu);
  const smc_tile_band* b = &g_bands.back();
  for (const smc_tile_band& x : g_bands)
    if (N <= x.n_max) {
      b = &x;
      break;
    }
  int64_t t = (N + b->slots - 1) / b->slots;
  t = std::max<int64_t>(t, b->tile_min);
  t = std::min<int64_t>(t, b->tile_max);
  t = std::min<int64_t>(t, N);
  return (int)std::max<int64_t>(t, 1);
}

int bucket_for(int tile) { return tile <= 32 ? 0 : tile <= 64 ? 1 : tile <= 128 ? 2 : 3; }

int combine_in_every_cta(int tile, int n_tiles, bool single) {
  const int tpb = 32 << bucket_for(tile);
  return single ? (n_tiles < redundant_cap(tpb) ? 1 : 0) : (n_tiles <= tpb ? 1 : 0);
}

int real_state_fields(int kind) {
  int n_real, n_int;
  model_fields(kind, &n_real, &n_int);
  return kind == SMC_MODEL_CRBD ? 3 : n_real;  // CRBD keeps log(lambda) internally
}

Layout make_layout(const smc_model_s* m, const smc_run_cfg* c) {
  Layout L{};
  const size_t N = (size_t)c->n_particles;
  const size_t rb = c->precision == SMC_PREC_FP32 ? 4 : 8;
  L.tile = tile_for((int64_t)N);
  L.n_tiles = (int)((N + L.tile - 1) / L.tile);
  L.max_segments = c->max_segments > 0 ? c->max_segments
                   : (m->n_segments_known > 0 ? m->n_segments_known : kUnboundedSegments);
  const int max_res = std::max(1, L.max_segments - 1);
  // unknown-length models keep at most kMaxAncRows recorded resamplings
  L.anc_rows = c->record_all_ancestors
                   ? (m->n_segments_known > 0 ? max_res : std::min(max_res, kMaxAncRows))
                   : 1;
  size_t off = 0;
  auto take = [&](size_t bytes) {
    const size_t o = off;
    off = align_up(off + std::max<size_t>(bytes, 1), 256);
    return o;
  };
  for (int b = 0; b < 2; ++b) {
    L.real[b] = take(rb * N * (size_t)m->n_real_state);
    L.ints[b] = take(4 * N * (size_t)m->n_int);
    L.stack[b] = take(rb * N * (size_t)m->stack_cap);
  }
  L.logw = take(8 * N);
  L.E[0] = take(8 * N);
  L.E[1] = take(8 * N);
  L.rec[0] = take(sizeof(TileRec) * (size_t)L.n_tiles);
  L.rec[1] = take(sizeof(TileRec) * (size_t)L.n_tiles);
  L.tq[0] = take(8 * (size_t)L.n_tiles);
  L.tq[1] = take(8 * (size_t)L.n_tiles);
  L.dec = take(4 * (size_t)L.max_segments);
  L.tO = take(8 * (size_t)(L.n_tiles + 1));
  L.rs = take(sizeof(RunState));
  L.anc = take(4 * N * (size_t)L.anc_rows);
  L.incr = take(8 * (size_t)L.max_segments);
  L.fin_real = take(8 * N * (size_t)m->n_real);
  L.fin_int = take(4 * N * (size_t)m->n_int);
  L.fin_stack = take(8 * N * (size_t)m->stack_cap);
  // a host snapshot to resume from is copied here
  L.snap = take(c->resume_k > 0 && c->resume_where == SMC_MEM_HOST
                    ? (8 + 8 * (size_t)m->n_real + 8 * (size_t)m->stack_cap) * N + 4 * N * (size_t)m->n_int
                    : 0);
  L.total = off;
  return L;
}

RunDev make_rundev(const smc_model_s* m, const smc_run_cfg* c, const Layout& Ly, char* ws) {
  RunDev A;
  std::memset(&A, 0, sizeof(A));
  const size_t N_ = (size_t)c->n_particles;
  A.md = m->md;
  for (int b = 0; b < 2; ++b) {
    A.state[b].real = ws + Ly.real[b];
    A.state[b].ints = (int32_t*)(ws + Ly.ints[b]);
    A.state[b].stack = ws + Ly.stack[b];
    A.E[b] = (long long*)(ws + Ly.E[b]);
  }
  A.logw = (double*)(ws + Ly.logw);
  A.rec[0] = (TileRec*)(ws + Ly.rec[0]);
  A.rec[1] = (TileRec*)(ws + Ly.rec[1]);
  A.tq[0] = (long long*)(ws + Ly.tq[0]);
  A.tq[1] = (long long*)(ws + Ly.tq[1]);
  A.dec = (int32_t*)(ws + Ly.dec);
  A.ess_tau = c->ess_threshold;
  A.ess = c->ess_threshold > 0.0 ? 1 : 0;
  A.ess_target = c->ess_threshold * (double)c->n_particles;
  A.tile_O = (long long*)(ws + Ly.tO);
  A.anc = (int32_t*)(ws + Ly.anc);
  A.incr = (double*)(ws + Ly.incr);
  A.rs = (RunState*)(ws + Ly.rs);
  A.N = (int)c->n_particles;
  A.log_n = std::log((double)c->n_particles);
  A.recip_n = ~0ull / (unsigned long long)c->n_particles;
  A.n_tiles = Ly.n_tiles;
  A.tile = Ly.tile;
  A.max_segments = Ly.max_segments;
  A.record_all = c->record_all_ancestors ? 1 : 0;
  A.anc_rows = Ly.anc_rows;
  A.k0 = (uint32_t)(c->seed & 0xffffffffu);
  A.k1 = (uint32_t)(c->seed >> 32) ^ c->run_id;
  A.resume_k = c->resume_k;
  if (c->resume_k > 0) {
    if (c->resume_where == SMC_MEM_HOST) {  // the copies made by stage_snapshot
      char* p = ws + Ly.snap;
      A.snap_logw = (const double*)p;
      p += 8 * N_;
      A.snap_real = (const double*)p;
      p += 8 * N_ * (size_t)m->n_real;
      A.snap_stack = (const double*)p;
      p += 8 * N_ * (size_t)m->stack_cap;
      A.snap_int = (const int32_t*)p;
    } else {
      A.snap_logw = c->resume_logw;
      A.snap_real = c->resume_real;
      A.snap_int = c->resume_int;
      A.snap_stack = c->resume_stack;
    }
  }
  return A;
}

cudaError_t launch_wave(const WavePlan& W, int precision, cudaStream_t st, unsigned wave) {
  // waves whose runs all run the linear-Gaussian or the CRBD model launch that
  // model's own kernel (smc_waves_kind.cu); others dispatch per run
  if (W.kind == SMC_MODEL_LG || W.kind == SMC_MODEL_CRBD)
    return launch_wave_kind(W, precision, st, wave);
  for (int b = 0; b < 4; ++b) {
    if (!W.n_ctas[b]) continue;
    cudaError_t e = precision == SMC_PREC_FP32
                        ? launch_bucket<float, 0>(b, W.runs, W.maps[b], W.n_ctas[b], st, wave)
                        : launch_bucket<double, 0>(b, W.runs, W.maps[b], W.n_ctas[b], st, wave);
    if (e != cudaSuccess) return e;
  }
  return cudaSuccess;
}

// The model kind shared by every run of a wave plan (0 when they differ).
int uniform_kind(const std::vector<RunDev>& runs) {
  if (runs.empty()) return 0;
  const int k = runs[0].md.kind;
  for (const RunDev& r : runs)
    if (r.md.kind != k) return 0;
  return k;
}

size_t wave_meta_bytes(const std::vector<RunDev>& runs) {
  size_t n_ctas = 0;
  for (const RunDev& r : runs) n_ctas += (size_t)r.n_tiles;
  return align_up(sizeof(RunDev) * runs.size(), 256) + align_up(sizeof(int2) * n_ctas, 256) + 4 * 256;
}

// Copies the run table and the per-bucket CTA maps to `meta` (device) and
// fills W with their device addresses.
// The run table and CTA maps to device memory at `meta`.  From pageable
// staging the call waits for the copy; from `pinned` (at least
// wave_meta_bytes(runs), not rewritten before the copy has run) it does not.
smc_status upload_wave(const std::vector<RunDev>& runs, void* meta, cudaStream_t st, WavePlan* W,
                       std::vector<char>* staging, char* pinned) {
  const size_t run_bytes = align_up(sizeof(RunDev) * runs.size(), 256);
  std::vector<int2> maps[4];
  for (size_t r = 0; r < runs.size(); ++r) {
    const int b = bucket_for(runs[r].tile);
    for (int t = 0; t < runs[r].n_tiles; ++t) maps[b].push_back(make_int2((int)r, t));
  }
  staging->assign(wave_meta_bytes(runs), 0);
  std::memcpy(staging->data(), runs.data(), sizeof(RunDev) * runs.size());
  size_t off = run_bytes;
  W->runs = (const RunDev*)meta;
  for (int b = 0; b < 4; ++b) {
    W->n_ctas[b] = (int)maps[b].size();
    W->maps[b] = (const int2*)((char*)meta + off);
    if (!maps[b].empty()) std::memcpy(staging->data() + off, maps[b].data(), sizeof(int2) * maps[b].size());
    off = align_up(off + sizeof(int2) * maps[b].size(), 256);
  }
  W->kind = uniform_kind(runs);
  if (pinned) {
    std::memcpy(pinned, staging->data(), off);
    SMC_CUDA_TRY(cudaMemcpyAsync(meta, pinned, off, cudaMemcpyHostToDevice, st));
    return SMC_OK;
  }
  SMC_CUDA_TRY(cudaMemcpyAsync(meta, staging->data(), off, cudaMemcpyHostToDevice, st));
  // the source is pageable host memory: wait for the copy before it can change
  SMC_CUDA_TRY(cudaStreamSynchronize(st));
  return SMC_OK;
}

namespace {

// Whether a graph instantiated earlier launches exactly these waves: the wave
// kernels' arguments are the run-table and CTA-map addresses and the wave
// index, so a graph captured for the same addresses, CTA counts, precision and
// number of waves is reusable once the run table (device memory) is uploaded.
bool graph_matches(const GraphCache* g, const WavePlan& W, int precision, int max_waves) {
  if (!g->exec || g->runs != W.runs || g->precision != precision || g->waves != max_waves)
    return false;
  for (int b = 0; b < 4; ++b)
    if (g->maps[b] != W.maps[b] || g->n_ctas[b] != W.n_ctas[b]) return false;
  return true;
}

// Capture max_waves waves on `st` into a graph and instantiate it into g.
smc_status capture_waves(GraphCache* g, const WavePlan& W, int precision, int max_waves,
                         cudaStream_t st) {
  graph_cache_clear(g);
  SMC_CUDA_TRY(cudaStreamBeginCapture(st, cudaStreamCaptureModeThreadLocal));
  cudaError_t e = cudaSuccess;
  for (int k = 0; k < max_waves && e == cudaSuccess; ++k) e = launch_wave(W, precision, st, (unsigned)k);
  cudaGraph_t graph = nullptr;
  const cudaError_t e2 = cudaStreamEndCapture(st, &graph);
  if (e != cudaSuccess || e2 != cudaSuccess) {
    if (graph) cudaGraphDestroy(graph);
    return cuda_fail(e != cudaSuccess ? e : e2, "capturing the waves in a graph");
  }
  e = cudaGraphInstantiate(&g->exec, graph, 0);
  cudaGraphDestroy(graph);
  if (e != cudaSuccess) {
    g->exec = nullptr;
    return cuda_fail(e, "cudaGraphInstantiate(waves)");
  }
  g->runs = W.runs;
  g->precision = precision;
  g->waves = max_waves;
  for (int b = 0; b < 4; ++b) {
    g->maps[b] = W.maps[b];
    g->n_ctas[b] = W.n_ctas[b];
  }
  return SMC_OK;
}

// Runs waves until every run is done or `max_waves` waves ran.  Known-length
// batches launch exactly max_waves waves without reading anything back (as one
// CUDA graph when `graph` is given and the stream can be captured); otherwise
// the run states are polled every 16 waves.  A run of S segments needs S + 1
// waves: the wave after its last segment combines that segment.
smc_status drive_waves(const WavePlan& W, int precision, const std::vector<RunState*>& states,
                       int max_waves, bool known, cudaStream_t st, std::vector<cudaEvent_t>* evs,
                       bool timed, int* launched, double* kernel_ms, GraphCache* graph = nullptr) {
  *launched = 0;
  *kernel_ms = 0.0;
  timed = timed && evs;
  int kernels_per_wave = 0;
  for (int b = 0; b < 4; ++b) kernels_per_wave += W.n_ctas[b] ? 1 : 0;
  if (known && graph && !timed && st != nullptr && st != cudaStreamLegacy) {
    if (!graph_matches(graph, W, precision, max_waves)) {
      smc_status s = capture_waves(graph, W, precision, max_waves, st);
      if (s) return s;
    }
    SMC_CUDA_TRY(cudaGraphLaunch(graph->exec, st));
    *launched = kernels_per_wave * max_waves;
    return SMC_OK;
  }
  int waves = 0;
  auto one = [&]() -> smc_status {
    if (timed) {
      while ((int)evs->size() < 2 * (waves + 1)) {
        cudaEvent_t e;
        SMC_CUDA_TRY(cudaEventCreate(&e));
        evs->push_back(e);
      }
      SMC_CUDA_TRY(cudaEventRecord((*evs)[2 * waves], st));
    }
    SMC_CUDA_TRY(launch_wave(W, precision, st, (unsigned)waves));
    if (timed) SMC_CUDA_TRY(cudaEventRecord((*evs)[2 * waves + 1], st));
    ++waves;
    *launched += kernels_per_wave;
    return SMC_OK;
  };
  if (known) {
    for (int k = 0; k < max_waves; ++k) {
      smc_status s = one();
      if (s) return s;
    }
  } else {
    const int chunk = 16;
    const size_t n_runs = states.size();
    std::vector<RunState> h(n_runs);
    for (int k0 = 0; k0 < max_waves; k0 += chunk) {
      const int k1 = std::min(max_waves, k0 + chunk);
      for (int k = k0; k < k1; ++k) {
        smc_status s = one();
        if (s) return s;
      }
      for (size_t r = 0; r < n_runs; ++r)
        SMC_CUDA_TRY(cudaMemcpyAsync(&h[r], states[r], sizeof(RunState), cudaMemcpyDeviceToHost, st));
      SMC_CUDA_TRY(cudaStreamSynchronize(st));
      bool all = true;
      for (size_t r = 0; r < n_runs; ++r) all = all && h[r].done;
      if (all) break;
    }
  }
  if (timed) {
    SMC_CUDA_TRY(cudaStreamSynchronize(st));
    for (int q = 0; q < waves; ++q) {
      float t = 0.f;
      if (cudaEventElapsedTime(&t, (*evs)[2 * q], (*evs)[2 * q + 1]) == cudaSuccess) *kernel_ms += t;
    }
  }
  return SMC_OK;
}

smc_status check_tree(const smc_model_desc* d) {
  const int M = d->n_nodes;
  if (M < 3 || (M & 1) == 0) return set_error(SMC_EINVAL, "n_nodes must be odd and >= 3");
  if (!d->parent || !d->left || !d->right || !d->preorder || !d->age)
    return set_error(SMC_EINVAL, "tree arrays must be non-NULL");
  if (d->parent[0] != -1 || d->preorder[0] != 0)
    return set_error(SMC_EINVAL, "node 0 must be the root and first in preorder");
  std::vector<char> seen(M, 0);
  for (int j = 0; j < M; ++j) {
    const int v = d->preorder[j];
    if (v < 0 || v >= M || seen[v]) return set_error(SMC_EINVAL, "preorder is not a permutation");
    seen[v] = 1;
    const int l = d->left[v], r = d->right[v];
    if ((l < 0) != (r < 0)) return set_error(SMC_EINVAL, "node %d has one child", v);
    if (l >= M || r >= M) return set_error(SMC_EINVAL, "child index out of range");
    if (l >= 0 && (d->parent[l] != v || d->parent[r] != v))
      return set_error(SMC_EINVAL, "parent/child arrays disagree at node %d", v);
    if (l >= 0 && (j + 1 >= M || d->preorder[j + 1] != l))
      return set_error(SMC_EINVAL, "preorder is not left-first at node %d", v);
    if (v != 0) {
      const int p = d->parent[v];
      if (p < 0 || p >= M) return set_error(SMC_EINVAL, "parent out of range");
      if (!(d->age[p] >= d->age[v]) || !(d->age[v] >= 0.0))
        return set_error(SMC_EINVAL, "ages must be >= 0 and not increase towards the tips");
    }
  }
  if (!(d->rho > 0.0 && d->rho <= 1.0)) return set_error(SMC_EINVAL, "rho must be in (0, 1]");
  if (d->depth_cap < 1 || d->depth_cap > SMC_MAX_DEPTH)
    return set_error(SMC_EINVAL, "depth_cap must be in 1..%d", SMC_MAX_DEPTH);
  if (d->call_limit < 1) return set_error(SMC_EINVAL, "call_limit must be >= 1");
  if (d->fixed_rates && !(d->lambda_fixed >= 0.0 && d->mu_fixed >= 0.0))
    return set_error(SMC_EINVAL, "fixed rates must be >= 0");
  if (!d->fixed_rates && !(d->lambda_scale > 0.0 && d->mu_scale > 0.0))
    return set_error(SMC_EINVAL, "prior scales must be > 0");
  if (d->kind == SMC_MODEL_RATESHIFT) {
    if (d->lam_stack_cap < 1) return set_error(SMC_EINVAL, "lam_stack_cap must be >= 1");
    if (!(d->sigma >= 0.0)) return set_error(SMC_EINVAL, "sigma must be >= 0");
  }
  return SMC_OK;
}

}  // namespace

// Copies one finished run's outputs into its smc_result and fills its counters.
smc_status collect_run(const smc_model_s* m, const smc_run_cfg* c, const Layout& Ly, char* ws,
                       const RunDev& A, const RunState& hrs, smc_result* r, cudaStream_t cs) {
  const int N = A.N;
  const int fb = (hrs.n_segments - 1) & 1;
  const bool host = r->where == SMC_MEM_HOST;
  double* fin_real = host ? (double*)(ws + Ly.fin_real) : r->real_fields;
  int32_t* fin_int = host ? (int32_t*)(ws + Ly.fin_int) : r->int_fields;
  double* fin_stack = host ? (double*)(ws + Ly.fin_stack) : r->stack;
  if (hrs.n_segments > 0 && (r->real_fields || r->int_fields || r->stack)) {
    const int blocks = (N + 255) / 256;
    if (c->precision == SMC_PREC_FP32)
      finalize_kernel<float><<<blocks, 256, 0, cs>>>(A.state[fb], N, m->n_real, m->n_int, m->stack_cap,
                                                     r->real_fields ? fin_real : nullptr,
                                                     r->int_fields ? fin_int : nullptr,
                                                     r->stack ? fin_stack : nullptr);
    else
      finalize_kernel<double><<<blocks, 256, 0, cs>>>(A.state[fb], N, m->n_real, m->n_int, m->stack_cap,
                                                      r->real_fields ? fin_real : nullptr,
                                                      r->int_fields ? fin_int : nullptr,
                                                      r->stack ? fin_stack : nullptr);
    SMC_CUDA_TRY(cudaGetLastError());
  }
  const cudaMemcpyKind kind = host ? cudaMemcpyDeviceToHost : cudaMemcpyDeviceToDevice;
  if (r->log_z) SMC_CUDA_TRY(cudaMemcpyAsync(r->log_z, &A.rs->log_z, 8, kind, cs));
  if (r->final_logw) SMC_CUDA_TRY(cudaMemcpyAsync(r->final_logw, A.logw, 8 * (size_t)N, kind, cs));
  if (host) {
    if (r->real_fields && m->n_real)
      SMC_CUDA_TRY(cudaMemcpyAsync(r->real_fields, fin_real, 8 * (size_t)N * m->n_real, kind, cs));
    if (r->int_fields && m->n_int)
      SMC_CUDA_TRY(cudaMemcpyAsync(r->int_fields, fin_int, 4 * (size_t)N * m->n_int, kind, cs));
    if (r->stack && m->stack_cap)
      SMC_CUDA_TRY(cudaMemcpyAsync(r->stack, fin_stack, 8 * (size_t)N * m->stack_cap, kind, cs));
  }
  if (r->ancestors) {
    const int n_res = std::max(0, hrs.n_segments - 1);
    const int rows = c->record_all_ancestors ? std::min(std::min(n_res, r->ancestors_rows), Ly.anc_rows)
                                             : (n_res > 0 ? 1 : 0);
    if (rows > 0) SMC_CUDA_TRY(cudaMemcpyAsync(r->ancestors, A.anc, 4 * (size_t)N * rows, kind, cs));
  }
  if (r->resampled) {  // the decisions (record_all: one per checkpoint; else the last one)
    const int n_tr = std::max(0, std::min(hrs.n_segments - 1, Ly.max_segments));
    const int rows = c->record_all_ancestors ? std::min(n_tr, r->ancestors_rows) : (n_tr > 0 ? 1 : 0);
    const int32_t* src = c->record_all_ancestors ? A.dec : A.dec + (n_tr - 1);
    if (rows > 0) SMC_CUDA_TRY(cudaMemcpyAsync(r->resampled, src, 4 * (size_t)rows, kind, cs));
  }
  smc_counters& ct = r->counters;
  ct.n_segments = hrs.n_segments;
  ct.n_resamples = hrs.n_resamples;
  ct.n_ess_near = hrs.n_ess_near;
  ct.n_near_boundary = (int64_t)hrs.n_near;
  ct.n_overflow = (int64_t)hrs.n_overflow;
  ct.n_limit = (int64_t)hrs.n_limit;
  ct.n_draws = (int64_t)hrs.n_draws;
  ct.n_blocks = (int64_t)hrs.n_blocks;
  ct.log_z_closed = hrs.log_z_closed;
  ct.debug_code = hrs.dbg_code;
  ct.debug_index = hrs.dbg_index;
  ct.debug_count = (int64_t)hrs.dbg_count;
  int st = hrs.status;
  if (st == 0 && !hrs.done) st = SMC_ESTEPLIMIT;
  if (st == 0 && (hrs.n_overflow || hrs.n_limit)) st = SMC_WKILLED;
  ct.status = st;
  return SMC_OK;
}

smc_status check_cfg(const smc_model_s* m, const smc_run_cfg* c) {
  if (!m || !c) return set_error(SMC_EINVAL, "NULL argument");
  if (c->n_particles < 1 || c->n_particles > kMaxParticles)
    return set_error(SMC_EINVAL, "n_particles must be in 1..%lld", (long long)kMaxParticles);
  if (c->precision != SMC_PREC_FP64 && c->precision != SMC_PREC_FP32)
    return set_error(SMC_EINVAL, "unknown precision");
  if (c->max_segments < 0 || c->max_segments > kMaxSegments)
    return set_error(SMC_EINVAL, "max_segments must be in 0..2^24");
  if (!(c->ess_threshold >= 0.0 && c->ess_threshold < 1e300))
    return set_error(SMC_EINVAL, "ess_threshold must be finite and >= 0");
  if (c->launch_mode < SMC_LAUNCH_AUTO || c->launch_mode > SMC_LAUNCH_WAVES)
    return set_error(SMC_EINVAL, "unknown launch_mode");
  if (c->resume_k < 0) return set_error(SMC_EINVAL, "resume_k must be >= 0");
  if (c->resume_k > 0) {
    if (c->resume_where != SMC_MEM_HOST && c->resume_where != SMC_MEM_DEVICE)
      return set_error(SMC_EINVAL, "resume_where must be SMC_MEM_HOST or SMC_MEM_DEVICE");
    if (!c->resume_logw || !c->resume_int || (m->n_real > 0 && !c->resume_real) ||
        (m->stack_cap > 0 && !c->resume_stack))
      return set_error(SMC_EINVAL, "a resumed run needs the snapshot's log-weights and fields");
    const int limit = c->max_segments > 0 ? c->max_segments
                      : (m->n_segments_known > 0 ? m->n_segments_known : kUnboundedSegments);
    if (c->resume_k > limit)
      return set_error(SMC_EINVAL, "resume_k %d beyond the run's segment limit %d", c->resume_k, limit);
  }
  return SMC_OK;
}

// Copy a host snapshot into the workspace area the resumed run reads it from.
smc_status stage_snapshot(const smc_model_s* m, const smc_run_cfg* c, const Layout& Ly, char* ws,
                          cudaStream_t cs) {
  if (c->resume_k <= 0 || c->resume_where != SMC_MEM_HOST) return SMC_OK;
  const size_t N = (size_t)c->n_particles;
  char* p = ws + Ly.snap;
  SMC_CUDA_TRY(cudaMemcpyAsync(p, c->resume_logw, 8 * N, cudaMemcpyHostToDevice, cs));
  p += 8 * N;
  if (m->n_real)
    SMC_CUDA_TRY(cudaMemcpyAsync(p, c->resume_real, 8 * N * m->n_real, cudaMemcpyHostToDevice, cs));
  p += 8 * N * (size_t)m->n_real;
  if (m->stack_cap)
    SMC_CUDA_TRY(cudaMemcpyAsync(p, c->resume_stack, 8 * N * m->stack_cap, cudaMemcpyHostToDevice, cs));
  p += 8 * N * (size_t)m->stack_cap;
  SMC_CUDA_TRY(cudaMemcpyAsync(p, c->resume_int, 4 * N * m->n_int, cudaMemcpyHostToDevice, cs));
  return SMC_OK;
}

smc_status check_result(const smc_result* r) {
  if (!r) return set_error(SMC_EINVAL, "NULL result");
  if (r->where != SMC_MEM_HOST && r->where != SMC_MEM_DEVICE)
    return set_error(SMC_EINVAL, "result.where must be SMC_MEM_HOST or SMC_MEM_DEVICE");
  return SMC_OK;
}

}  // namespace smc

using namespace smc;

extern "C" smc_status smc_set_tile_bands(const smc_tile_band* bands, int32_t n_bands) {
  std::vector<smc_tile_band> next;
  if (!bands && n_bands == 0) {
    next.assign(std::begin(kBuiltinBands), std::end(kBuiltinBands));
  } else {
    if (!bands) return set_error(SMC_EINVAL, "NULL bands");
    smc_status st = check_bands(bands, n_bands);
    if (st) return st;
    next.assign(bands, bands + n_bands);
  }
  std::lock_guard<std::mutex> lock(g_band_mu);
  g_bands.swap(next);
  return SMC_OK;
}

extern "C" smc_status smc_get_tile_bands(smc_tile_band* out, int32_t cap, int32_t* n_bands) {
  if (!n_bands) return set_error(SMC_EINVAL, "NULL n_bands");
  std::lock_guard<std::mutex> lock(g_band_mu);
  *n_bands = (int32_t)g_bands.size();
  if (out)
    for (int i = 0; i < (int)g_bands.size() && i < cap; ++i) out[i] = g_bands[i];
  return SMC_OK;
}

extern "C" int32_t smc_tile_size(int64_t n_particles) {
  if (n_particles < 1 || n_particles > kMaxParticles) return 0;
  return tile_for(n_particles);
}

extern "C" smc_status smc_model_register(const smc_model_desc* d, smc_model_t* out) {
  if (!d || !out) return set_error(SMC_EINVAL, "NULL argument");
  *out = nullptr;
  int n_real, n_int;
  if (model_fields(d->kind, &n_real, &n_int)) return set_error(SMC_EINVAL, "unknown model kind");
  size_t blob = 0;
  if (d->kind == SMC_MODEL_LG) {
    if (d->T < 1 || !d->obs) return set_error(SMC_EINVAL, "LG needs T >= 1 observations");
    if (!(d->r_sd > 0.0) || !(d->x0_sd >= 0.0) || !(d->q_sd >= 0.0))
      return set_error(SMC_EINVAL, "LG standard deviations must be >= 0 (r_sd > 0)");
    blob = 8 * (size_t)d->T;
  } else if (d->kind == SMC_MODEL_SEIR) {
    if (d->T < 1 || !d->obs) return set_error(SMC_EINVAL, "SEIR needs T >= 1 days of reports");
    for (int t = 0; t < d->T; ++t)
      if (!(d->obs[t] == -1.0 || (d->obs[t] >= 0.0 && d->obs[t] == std::floor(d->obs[t]) &&
                                  d->obs[t] < 2147483647.0)))
        return set_error(SMC_EINVAL, "SEIR reports must be counts >= 0 or -1 (day %d)", t);
    blob = 8 * (size_t)d->T;
  } else if (d->kind == SMC_MODEL_GEOMETRIC) {
    if (!(d->geo_p >= 0.0 && d->geo_p <= 1.0)) return set_error(SMC_EINVAL, "geo_p in [0,1]");
  } else {
    smc_status st = check_tree(d);
    if (st) return st;
    if (d->kind == SMC_MODEL_CRBD_DS &&
        (d->fixed_rates || !(d->lambda_scale > 0.0) || !(d->mu_scale > 0.0)))
      return set_error(SMC_EINVAL, "delayed-sampling CRBD integrates the Gamma priors out: "
                                   "no fixed rates, lambda_scale and mu_scale > 0");
    blob = align_up(4 * (size_t)d->n_nodes, 256) * 3 + align_up(8 * (size_t)d->n_nodes, 256) * 2 +
           align_up(sizeof(BranchRec) * (size_t)d->n_nodes, 256);
  }
  smc_model_s* m = new (std::nothrow) smc_model_s();
  if (!m) return set_error(SMC_ENOMEM, "host allocation failed");
  m->desc = *d;
  m->n_real = n_real;
  m->n_real_state = real_state_fields(d->kind);
  m->n_int = n_int;
  m->stack_cap = d->kind == SMC_MODEL_RATESHIFT ? d->lam_stack_cap : 0;
  ModelDev& md = m->md;
  std::memset(&md, 0, sizeof(md));
  md.kind = d->kind;
  md.T = d->T;
  md.n_nodes = d->n_nodes;
  md.fixed_rates = d->fixed_rates;
  md.depth_cap = d->depth_cap;
  md.call_limit = d->call_limit;
  md.lam_stack_cap = d->lam_stack_cap;
  md.x0_mean = d->x0_mean;
  md.x0_sd = d->x0_sd;
  md.a = d->a;
  md.b = d->b;
  md.q_sd = d->q_sd;
  md.r_sd = d->r_sd;
  md.rho = d->rho;
  md.lambda_fixed = d->lambda_fixed;
  md.mu_fixed = d->mu_fixed;
  md.lambda_scale = d->lambda_scale;
  md.mu_scale = d->mu_scale;
  md.sigma = d->sigma;
  md.geo_p = d->geo_p;
  md.geo_logw = d->geo_logw;
  md.log_rho = d->rho > 0.0 ? std::log(d->rho) : 0.0;
  {
    const MathTab* tab = nullptr;
    smc_status ts = math_table(&tab);
    if (ts) {
      delete m;
      return ts;
    }
    md.tab = tab;
  }
  m->n_segments_known = 0;
  if (d->kind == SMC_MODEL_LG) {
    md.lg_lc = std::log(d->r_sd) + 0.91893853320467274178;
    m->n_segments_known = d->T;
  }
  if (d->kind == SMC_MODEL_SEIR) m->n_segments_known = d->T;
  if (d->kind == SMC_MODEL_CRBD || d->kind == SMC_MODEL_RATESHIFT || d->kind == SMC_MODEL_CRBD_DS) {
    const int tips = (d->n_nodes + 1) / 2;
    double lnfact = 0.0;
    for (int i = 2; i <= tips; ++i) lnfact = lnfact + std::log((double)i);
    md.corr = (double)(tips - 1) * kLn2 - lnfact;
    m->n_segments_known = d->n_nodes;
  }
  cudaGetDevice(&m->dev);
  if (blob) {
    if (d->fixed_mult) blob += align_up(8 * (size_t)d->n_nodes, 256);
    cudaError_t e = block_alloc(&m->dev_blob, &m->blob_bytes, blob);
    if (e != cudaSuccess) {
      delete m;
      return cuda_fail(e, "cudaMalloc(model data)");
    }
    // the arrays are laid out in a host copy of the block, then copied at once
    std::vector<char> host(blob, 0);
    size_t off = 0;
    auto put = [&](const void* src, size_t bytes) -> void* {
      if (off + bytes > blob) return nullptr;
      std::memcpy(host.data() + off, src, bytes);
      void* dst = (char*)m->dev_blob + off;
      off += align_up(bytes, 256);
      return dst;
    };
    bool ok = true;
    if (d->kind == SMC_MODEL_LG || d->kind == SMC_MODEL_SEIR) {
      ok = (md.obs = (const double*)put(d->obs, 8 * (size_t)d->T)) != nullptr;
    } else {
      const size_t M = d->n_nodes;
      ok = (md.parent = (const int*)put(d->parent, 4 * M)) && (md.left = (const int*)put(d->left, 4 * M)) &&
           (md.preorder = (const int*)put(d->preorder, 4 * M)) && (md.age = (const double*)put(d->age, 8 * M));
      // the branch of each segment k >= 1 in traversal order (entry 0: the root, unused)
      std::vector<BranchRec> br(M);
      for (size_t k = 0; k < M; ++k) {
        BranchRec r{};
        const int v = d->preorder[k];
        r.v = v;
        r.stop = d->age[v];
        if (k > 0) {
          const int pa = d->parent[v];
          r.start = d->age[pa];
          r.flags = (d->left[v] >= 0 ? 1 : 0) | (d->left[pa] == v ? 2 : 0);
        }
        br[k] = r;
      }
      if (ok) ok = (md.branch = (const BranchRec*)put(br.data(), sizeof(BranchRec) * M)) != nullptr;
      if (ok && d->fixed_mult) ok = (md.fixed_mult = (const double*)put(d->fixed_mult, 8 * M)) != nullptr;
    }
    if (ok) ok = cudaMemcpy(m->dev_blob, host.data(), blob, cudaMemcpyHostToDevice) == cudaSuccess;
    if (!ok) {
      block_free(m->dev_blob, m->blob_bytes, m->dev);
      delete m;
      return set_error(SMC_ECUDA, "copying model data to the device failed");
    }
  }
  if (cudaEventCreate(&m->ev0) != cudaSuccess || cudaEventCreate(&m->ev1) != cudaSuccess) {
    block_free(m->dev_blob, m->blob_bytes, m->dev);
    delete m;
    return set_error(SMC_ECUDA, "cudaEventCreate failed");
  }
  *out = m;
  return SMC_OK;
}

extern "C" void smc_model_destroy(smc_model_t m) {
  if (!m) return;
  graph_cache_clear(&m->graph);
  block_free(m->ws, m->ws_bytes, m->dev);
  block_free(m->dev_blob, m->blob_bytes, m->dev);
  if (m->ev0) cudaEventDestroy(m->ev0);
  if (m->ev1) cudaEventDestroy(m->ev1);
  for (cudaEvent_t e : m->ev_seg) cudaEventDestroy(e);
  if (m->pin_ev) {
    cudaEventSynchronize(m->pin_ev);
    cudaEventDestroy(m->pin_ev);
  }
  if (m->pin) cudaFreeHost(m->pin);
  delete m;
}

extern "C" smc_status smc_model_info(smc_model_t m, int32_t* n_real, int32_t* n_int,
                                     int32_t* stack_cap, int32_t* n_segments) {
  if (!m) return set_error(SMC_EINVAL, "NULL model");
  if (n_real) *n_real = m->n_real;
  if (n_int) *n_int = m->n_int;
  if (stack_cap) *stack_cap = m->stack_cap;
  if (n_segments) *n_segments = m->n_segments_known;
  return SMC_OK;
}

extern "C" smc_status smc_workspace_bytes(smc_model_t m, const smc_run_cfg* c, size_t* bytes) {
  smc_status st = check_cfg(m, c);
  if (st) return st;
  if (!bytes) return set_error(SMC_EINVAL, "NULL bytes");
  const Layout Ly = make_layout(m, c);
  std::vector<RunDev> one(1);
  one[0].n_tiles = Ly.n_tiles;
  *bytes = align_up(Ly.total, 256) + wave_meta_bytes(one);
  return SMC_OK;
}

extern "C" smc_status smc_run(smc_model_t m, const smc_run_cfg* c, smc_result* r, void* stream) {
  NvtxRange nv_all("smc_run");
  smc_status st = check_cfg(m, c);
  if (st) return st;
  if ((st = check_result(r))) return st;
  cudaStream_t cs = (cudaStream_t)stream;
  const Layout Ly = make_layout(m, c);
  const size_t meta_off = align_up(Ly.total, 256);
  std::vector<RunDev> runs(1);
  runs[0].n_tiles = Ly.n_tiles;
  const size_t need = meta_off + wave_meta_bytes(runs);
  char* ws;
  if (c->workspace) {
    if (c->workspace_bytes < need)
      return set_error(SMC_EINVAL, "workspace too small (%zu < %zu)", c->workspace_bytes, need);
    ws = (char*)c->workspace;
  } else {
    if (m->ws_bytes < need) {
      graph_cache_clear(&m->graph);  // a captured graph addresses the old workspace
      block_free(m->ws, m->ws_bytes, m->dev);
      m->ws = nullptr;
      m->ws_bytes = 0;
      cudaError_t e = block_alloc(&m->ws, &m->ws_bytes, need);
      if (e != cudaSuccess) {
        m->ws_bytes = 0;
        return set_error(SMC_ENOMEM, "workspace cudaMalloc(%zu): %s", need, cudaGetErrorString(e));
      }
    }
    ws = (char*)m->ws;
  }
  runs[0] = make_rundev(m, c, Ly, ws);
  runs[0].redundant = combine_in_every_cta(Ly.tile, Ly.n_tiles, true);
  // a resumed run's first wave is its segment resume_k - 1 (the snapshot's load)
  const int skip = c->resume_k > 0 ? c->resume_k - 1 : 0;
  runs[0].start_wave = (unsigned)(-skip);
  WavePlan W;
  SMC_CUDA_TRY(cudaMemsetAsync(runs[0].rs, 0, sizeof(RunState), cs));
  if (c->resume_k > 0) {
    const double lz[1] = {c->resume_log_z};
    SMC_CUDA_TRY(cudaMemcpyAsync(&runs[0].rs->log_z, lz, 8, cudaMemcpyHostToDevice, cs));
    SMC_CUDA_TRY(cudaMemcpyAsync(&runs[0].rs->log_z_closed, lz, 8, cudaMemcpyHostToDevice, cs));
    SMC_CUDA_TRY(cudaStreamSynchronize(cs));  // the pageable sources above are locals
    if ((st = stage_snapshot(m, c, Ly, ws, cs))) return st;
    // the rows before checkpoint resume_k - 1 belong to the run that made the snapshot
    if (c->record_all_ancestors && skip > 0) {
      const size_t rows = std::min<size_t>((size_t)skip, (size_t)Ly.anc_rows);
      SMC_CUDA_TRY(cudaMemsetAsync(runs[0].anc, 0, 4 * (size_t)c->n_particles * rows, cs));
      SMC_CUDA_TRY(cudaMemsetAsync(runs[0].dec, 0, 4 * (size_t)skip, cs));
    }
  }
  // the run table through the handle's pinned buffer (no wait for the copy),
  // once the previous call's upload from it has run
  if (m->pin_ev) SMC_CUDA_TRY(cudaEventSynchronize(m->pin_ev));
  const size_t meta_bytes = wave_meta_bytes(runs);
  if (m->pin_bytes < meta_bytes) {
    if (m->pin) cudaFreeHost(m->pin);
    m->pin = nullptr;
    m->pin_bytes = 0;
    if (cudaMallocHost(&m->pin, meta_bytes) == cudaSuccess)
      m->pin_bytes = meta_bytes;
    else
      cudaGetLastError();  // pageable staging instead
  }
  if (m->pin && !m->pin_ev) SMC_CUDA_TRY(cudaEventCreateWithFlags(&m->pin_ev, cudaEventDisableTiming));
  if ((st = upload_wave(runs, ws + meta_off, cs, &W, &m->staging, m->pin))) return st;
  if (m->pin) SMC_CUDA_TRY(cudaEventRecord(m->pin_ev, cs));
  SMC_CUDA_TRY(cudaEventRecord(m->ev0, cs));
  const bool known = m->n_segments_known > 0 && Ly.max_segments >= m->n_segments_known;
  int launched = 0;
  double kms = 0.0;
  std::vector<RunState*> states{runs[0].rs};
  NvtxRange nv_waves("smc_run/waves");
  // a small run (32-particle tiles, few enough for one CTA or one cluster) runs
  // every segment in one launch: the same tiles and integers as the waves
  const int one = c->launch_mode == SMC_LAUNCH_AUTO ? SMC_LAUNCH_CLUSTER : c->launch_mode;
  const bool small = (one == SMC_LAUNCH_ONE_CTA || one == SMC_LAUNCH_CLUSTER) &&
                     c->resume_k == 0 && !c->time_kernels && Ly.tile == 32 &&
                     Ly.n_tiles <= small_run_max_tiles(m->desc.kind, one);
  bool waves = !small;
  if (small) {
    const cudaError_t e = launch_small_run(m->desc.kind, c->precision, one, W.runs, Ly.n_tiles, cs);
    if (e != cudaSuccess && c->launch_mode == SMC_LAUNCH_AUTO) {
      cudaGetLastError();  // a cluster the GPU cannot place: the waves instead
      waves = true;
    } else {
      SMC_CUDA_TRY(e);
      launched = 1;
    }
  }
  if (waves) {
    st = drive_waves(W, c->precision, states,
                     (known ? m->n_segments_known : Ly.max_segments) + 1 - skip, known, cs,
                     &m->ev_seg, c->time_kernels != 0, &launched, &kms,
                     c->launch_mode == SMC_LAUNCH_GRAPH ? &m->graph : nullptr);
    if (st) return st;
  }
  SMC_CUDA_TRY(cudaEventRecord(m->ev1, cs));
  RunState hrs;
  SMC_CUDA_TRY(cudaMemcpyAsync(&hrs, runs[0].rs, sizeof(RunState), cudaMemcpyDeviceToHost, cs));
  SMC_CUDA_TRY(cudaStreamSynchronize(cs));
  NvtxRange nv_collect("smc_run/collect");
  float ms = 0.f;
  cudaEventElapsedTime(&ms, m->ev0, m->ev1);
  if ((st = collect_run(m, c, Ly, ws, runs[0], hrs, r, cs))) return st;
  SMC_CUDA_TRY(cudaStreamSynchronize(cs));
  r->counters.device_ms = ms;
  r->counters.kernel_launches = launched;
  r->counters.kernel_ms = kms;
  const int rs_status = r->counters.status;
  if (rs_status == SMC_EDEGENERATE) return set_error(SMC_EDEGENERATE, "all particle weights are zero");
  if (rs_status == SMC_ESTEPLIMIT) return set_error(SMC_ESTEPLIMIT, "max_segments reached");
  return rs_status;
}

extern "C" smc_status smc_run_batch(const smc_model_t* ms, const smc_run_cfg* cfgs, smc_result* res,
                                    int32_t n_runs, void* stream) {
  NvtxRange nv_all("smc_run_batch");
  if (!ms || !cfgs || !res || n_runs < 1) return set_error(SMC_EINVAL, "bad batch arguments");
  smc_status st;
  const int prec = cfgs[0].precision;
  for (int q = 0; q < n_runs; ++q) {
    if ((st = check_cfg(ms[q], &cfgs[q]))) return st;
    if ((st = check_result(&res[q]))) return st;
    if (cfgs[q].precision != prec) return set_error(SMC_EINVAL, "a batch must use one precision");
    if (cfgs[q].resume_k != 0) return set_error(SMC_EINVAL, "resume is for smc_run only");
  }
  cudaStream_t cs = (cudaStream_t)stream;
  std::vector<Layout> lys(n_runs);
  std::vector<size_t> offs(n_runs);
  std::vector<RunDev> runs(n_runs);
  size_t total = 0;
  int max_waves = 0;
  bool known = true;
  for (int q = 0; q < n_runs; ++q) {
    lys[q] = make_layout(ms[q], &cfgs[q]);
    offs[q] = total;
    total = align_up(total + lys[q].total, 256);
    const bool kq = ms[q]->n_segments_known > 0 && lys[q].max_segments >= ms[q]->n_segments_known;
    known = known && kq;
    max_waves = std::max(max_waves, kq ? ms[q]->n_segments_known : lys[q].max_segments);
    runs[q].n_tiles = lys[q].n_tiles;
  }
  const size_t meta_off = total;
  total += wave_meta_bytes(runs);
  void* ws = nullptr;
  {
    cudaError_t e = cudaMallocAsync(&ws, total, cs);
    if (e != cudaSuccess)
      return set_error(SMC_ENOMEM, "batch workspace cudaMallocAsync(%zu): %s", total, cudaGetErrorString(e));
  }
  struct Free {
    void* p;
    cudaStream_t s;
    ~Free() {
      if (p) cudaFreeAsync(p, s);
    }
  } guard{ws, cs};
  std::vector<RunState*> states(n_runs);
  for (int q = 0; q < n_runs; ++q) {
    runs[q] = make_rundev(ms[q], &cfgs[q], lys[q], (char*)ws + offs[q]);
    runs[q].redundant = combine_in_every_cta(lys[q].tile, lys[q].n_tiles, n_runs == 1);
    states[q] = runs[q].rs;
    SMC_CUDA_TRY(cudaMemsetAsync(runs[q].rs, 0, sizeof(RunState), cs));
  }
  WavePlan W;
  std::vector<char> staging;
  if ((st = upload_wave(runs, (char*)ws + meta_off, cs, &W, &staging))) return st;
  cudaEvent_t e0, e1;
  SMC_CUDA_TRY(cudaEventCreate(&e0));
  SMC_CUDA_TRY(cudaEventCreate(&e1));
  SMC_CUDA_TRY(cudaEventRecord(e0, cs));
  int launched = 0;
  double kms = 0.0;
  GraphCache graph;
  st = drive_waves(W, prec, states, max_waves + 1, known, cs, nullptr, false, &launched, &kms,
                   cfgs[0].launch_mode == SMC_LAUNCH_GRAPH ? &graph : nullptr);
  if (st) {
    graph_cache_clear(&graph);
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    return st;
  }
  SMC_CUDA_TRY(cudaEventRecord(e1, cs));
  std::vector<RunState> h(n_runs);
  for (int q = 0; q < n_runs; ++q)
    SMC_CUDA_TRY(cudaMemcpyAsync(&h[q], states[q], sizeof(RunState), cudaMemcpyDeviceToHost, cs));
  const cudaError_t se = cudaStreamSynchronize(cs);
  graph_cache_clear(&graph);  // its launch has completed
  if (se != cudaSuccess) return cuda_fail(se, "cudaStreamSynchronize(batch)");
  float msec = 0.f;
  cudaEventElapsedTime(&msec, e0, e1);
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  for (int q = 0; q < n_runs; ++q) {
    if ((st = collect_run(ms[q], &cfgs[q], lys[q], (char*)ws + offs[q], runs[q], h[q], &res[q], cs)))
      return st;
    res[q].counters.device_ms = msec;
    res[q].counters.kernel_launches = launched;
    res[q].counters.kernel_ms = 0.0;
  }
  SMC_CUDA_TRY(cudaStreamSynchronize(cs));
  return SMC_OK;
}
