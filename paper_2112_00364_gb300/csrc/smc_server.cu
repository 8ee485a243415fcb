// smc_server.cu -- continuous batching of SMC requests on one GPU.
//
// A worker thread owns a CUDA stream and repeats:
//   1. admit queued requests while the resident-run cap and the device-memory
//      budget allow (each admitted run gets its workspace from the stream-ordered
//      pool and a zeroed run state, so it starts at segment 0 in the next wave);
//   2. launch poll_waves waves (default 2): every resident run advances one
//      segment per wave (the same wave kernels as smc_run_batch, over the
//      current run table), so the host's work of step 3 overlaps a queued wave;
//   3. gather the resident runs' done flags into pinned memory and, one poll
//      behind (so the GPU always has the next waves queued), retire the finished
//      runs: their outputs are copied into the callers' result buffers on the
//      stream, an event marks them complete, and their workspace goes back to the
//      pool after the copies.
// Because a run's arithmetic depends only on its own model, N, seed and run_id
// (tiling is a function of N), a request's results equal those of smc_run,
// whatever else is resident.  All waits are bounded.
#include <cuda_runtime.h>

#include <algorithm>
#include <atomic>
#include <chrono>
#include <condition_variable>
#include <cstdlib>
#include <cstring>
#include <deque>
#include <mutex>
#include <new>
#include <thread>
#include <unordered_map>
#include <unordered_set>
#include <vector>

#include "smc_engine.h"
#include "smc_internal.h"

namespace smc {

// Snapshot of a run's state after a wave: everything retiring it needs.
struct RunFlags {
  unsigned long long n_near, n_overflow, n_limit, n_draws, n_blocks;
  double log_z_closed;
  long long dbg_index;
  unsigned long long dbg_count;
  int32_t dbg_code;
  int32_t done, status, n_segments, n_resamples, n_ess_near;
};

__global__ void gather_flags_kernel(const RunDev* __restrict__ runs, int n, RunFlags* out) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  const RunState* rs = runs[i].rs;
  RunFlags f;
  f.done = *(volatile const int32_t*)&rs->done;
  f.status = rs->status;
  f.n_segments = rs->n_segments;
  f.n_resamples = rs->n_resamples;
  f.n_ess_near = rs->n_ess_near;
  f.n_near = rs->n_near;
  f.n_overflow = rs->n_overflow;
  f.n_limit = rs->n_limit;
  f.n_draws = rs->n_draws;
  f.n_blocks = rs->n_blocks;
  f.log_z_closed = rs->log_z_closed;
  f.dbg_code = rs->dbg_code;
  f.dbg_index = rs->dbg_index;
  f.dbg_count = rs->dbg_count;
  out[i] = f;
}

namespace {

enum TicketState { T_QUEUED = 0, T_RESIDENT = 1, T_COMPLETING = 2, T_DONE = 3, T_FAILED = 4 };

struct Request {
  uint64_t ticket;
  smc_model_s* model;
  smc_run_cfg cfg;
  smc_result* result;
  Layout ly;
  size_t bytes;
  char* ws = nullptr;
  RunDev dev;
  cudaEvent_t done_ev = nullptr;
  double t_submit = 0.0;
  bool cancel = false;  // queued: written and read under the server mutex; resident: worker only
};

double now_s() {
  return std::chrono::duration<double>(std::chrono::steady_clock::now().time_since_epoch()).count();
}

}  // namespace

struct Server {
  smc_server_cfg cfg;
  size_t budget;
  int device = 0;
  cudaStream_t stream = nullptr;
  std::thread worker;
  std::mutex mu;
  std::condition_variable cv_work, cv_done;
  bool stop = false;
  std::deque<Request*> queue;
  std::unordered_map<uint64_t, int> state;  // ticket -> TicketState
  // cancellations of resident runs, handed to the worker under `mu` (the
  // resident list itself belongs to the worker thread alone)
  std::unordered_set<uint64_t> cancel_req;
  std::unordered_map<uint64_t, int> final_status;
  std::unordered_map<uint64_t, double> latency;
  uint64_t next_ticket = 1;
  // worker-owned
  std::vector<Request*> resident;
  std::vector<Request*> completing;
  size_t in_use = 0;
  void* meta = nullptr;          // device run table + CTA maps
  size_t meta_bytes = 0;
  char* pinned_meta = nullptr;   // host staging of the table
  size_t pinned_meta_bytes = 0;
  cudaEvent_t meta_ev = nullptr; // last table upload consumed
  RunFlags* flags_dev = nullptr;
  RunFlags* flags_host[2] = {nullptr, nullptr};
  cudaEvent_t flags_ev[2] = {nullptr, nullptr};
  // tickets of the runs whose flags a snapshot holds, in table order (tickets,
  // not pointers: a retired request is deleted and its address may be reused
  // by a request admitted before the snapshot is read)
  std::vector<uint64_t> flags_owner[2];
  int flags_pending[2] = {0, 0};
  int cap_flags = 0;
  WavePlan plan;
  bool table_dirty = true;
  // stats
  std::atomic<int64_t> waves{0}, completed{0}, particle_steps{0};
  std::atomic<int32_t> n_resident{0}, n_queued{0};
  std::atomic<int32_t> worker_error{0};
  // host-side fault injection for tests: the retirement of this ticket fails
  // after its result copies were queued (0 = off; SMC_SERVER_FAIL_TICKET)
  uint64_t fail_ticket = 0;
};

namespace {

// Flag buffers hold one entry per resident run; they are sized once for the
// resident-run cap so that a pending buffer is never reallocated under a copy.
smc_status alloc_flags(Server* S, int cap) {
  SMC_CUDA_TRY(cudaMalloc(&S->flags_dev, sizeof(RunFlags) * cap));
  for (int b = 0; b < 2; ++b) SMC_CUDA_TRY(cudaMallocHost(&S->flags_host[b], sizeof(RunFlags) * cap));
  S->cap_flags = cap;
  return SMC_OK;
}

// Rebuild the run table of the resident set and upload it (stream-ordered).
smc_status upload_table(Server* S) {
  std::vector<RunDev> runs;
  runs.reserve(S->resident.size());
  for (Request* q : S->resident) runs.push_back(q->dev);
  const size_t need = wave_meta_bytes(runs);
  // the previous upload must have been consumed before its staging is reused
  if (S->meta_ev) SMC_CUDA_TRY(cudaEventSynchronize(S->meta_ev));
  if (need > S->meta_bytes) {
    if (S->meta) SMC_CUDA_TRY(cudaFreeAsync(S->meta, S->stream));
    S->meta = nullptr;
    const size_t sz = std::max(need, 2 * S->meta_bytes);
    SMC_CUDA_TRY(cudaMallocAsync(&S->meta, sz, S->stream));
    S->meta_bytes = sz;
  }
  if (need > S->pinned_meta_bytes) {
    if (S->pinned_meta) cudaFreeHost(S->pinned_meta);
    S->pinned_meta = nullptr;
    const size_t sz = std::max(need, 2 * S->pinned_meta_bytes);
    SMC_CUDA_TRY(cudaMallocHost(&S->pinned_meta, sz));
    S->pinned_meta_bytes = sz;
  }
  // same layout as upload_wave, written into pinned staging
  std::vector<int2> maps[4];
  for (size_t r = 0; r < runs.size(); ++r) {
    const int b = bucket_for(runs[r].tile);
    for (int t = 0; t < runs[r].n_tiles; ++t) maps[b].push_back(make_int2((int)r, t));
  }
  std::memcpy(S->pinned_meta, runs.data(), sizeof(RunDev) * runs.size());
  size_t off = align_up(sizeof(RunDev) * runs.size(), 256);
  S->plan.runs = (const RunDev*)S->meta;
  for (int b = 0; b < 4; ++b) {
    S->plan.n_ctas[b] = (int)maps[b].size();
    S->plan.maps[b] = (const int2*)((char*)S->meta + off);
    if (!maps[b].empty()) std::memcpy(S->pinned_meta + off, maps[b].data(), sizeof(int2) * maps[b].size());
    off = align_up(off + sizeof(int2) * maps[b].size(), 256);
  }
  S->plan.kind = uniform_kind(runs);
  SMC_CUDA_TRY(cudaMemcpyAsync(S->meta, S->pinned_meta, off, cudaMemcpyHostToDevice, S->stream));
  SMC_CUDA_TRY(cudaEventRecord(S->meta_ev, S->stream));
  S->table_dirty = false;
  return SMC_OK;
}

void finish_ticket(Server* S, Request* q, int status) {
  std::lock_guard<std::mutex> lk(S->mu);
  S->cancel_req.erase(q->ticket);  // a cancel that came after the run finished
  S->state[q->ticket] = (status < 0 && status != SMC_EDEGENERATE && status != SMC_ESTEPLIMIT) ? T_FAILED : T_DONE;
  S->final_status[q->ticket] = status;
  S->latency[q->ticket] = now_s() - q->t_submit;
  S->cv_done.notify_all();
}

// A request taken out of the resident list whose retirement failed (its result
// copies, its completion event or its workspace release): wait until the copies
// already queued into its result buffers have ended, release its workspace and
// close its ticket as failed, so that a waiter never sees the ticket done while
// copies into its buffers are still in flight, and none is left to time out.
void fail_retiring(Server* S, Request* q, smc_status st) {
  cudaStreamSynchronize(S->stream);
  if (q->done_ev) cudaEventDestroy(q->done_ev);
  q->done_ev = nullptr;
  if (q->ws) cudaFreeAsync(q->ws, S->stream);
  S->in_use -= q->bytes;
  finish_ticket(S, q, st);
  S->completed += 1;
  delete q;
}

// Admit queued requests that fit.  Returns the number admitted.
int admit(Server* S, smc_status* err) {
  int n = 0;
  const int cap = S->cfg.max_resident_runs;
  for (;;) {
    Request* q = nullptr;
    {
      std::lock_guard<std::mutex> lk(S->mu);
      if (S->queue.empty() || (int)S->resident.size() >= cap) break;
      Request* head = S->queue.front();
      if (head->cancel) {
        S->queue.pop_front();
        S->n_queued = (int32_t)S->queue.size();
        S->state[head->ticket] = T_FAILED;
        S->final_status[head->ticket] = SMC_ECANCELLED;
        S->cv_done.notify_all();
        delete head;
        continue;
      }
      if (S->in_use + head->bytes > S->budget && !S->resident.empty()) break;
      S->queue.pop_front();
      S->n_queued = (int32_t)S->queue.size();
      q = head;
      S->state[q->ticket] = T_RESIDENT;
    }
    void* p = nullptr;
    cudaError_t e = cudaMallocAsync(&p, q->bytes, S->stream);
    if (e != cudaSuccess) {
      set_error(SMC_ENOMEM, "server workspace cudaMallocAsync(%zu): %s", q->bytes, cudaGetErrorString(e));
      finish_ticket(S, q, SMC_ENOMEM);
      delete q;
      continue;
    }
    q->ws = (char*)p;
    q->dev = make_rundev(q->model, &q->cfg, q->ly, q->ws);
    q->dev.start_wave = (unsigned)S->waves.load();  // its segment 0 runs in the next wave
    q->dev.redundant = combine_in_every_cta(q->ly.tile, q->ly.n_tiles, false);
    e = cudaMemsetAsync(q->dev.rs, 0, sizeof(RunState), S->stream);
    if (e != cudaSuccess) {  // the run never became resident: close its ticket
      *err = cuda_fail(e, "cudaMemsetAsync(run state)");
      cudaFreeAsync(q->ws, S->stream);
      finish_ticket(S, q, *err);
      delete q;
      return n;
    }
    S->in_use += q->bytes;
    S->resident.push_back(q);
    S->table_dirty = true;
    ++n;
  }
  S->n_resident = (int32_t)S->resident.size();
  return n;
}

// Retire the runs whose flags say done (flags of buffer b, taken after some wave).
smc_status retire(Server* S, int b) {
  const int n = S->flags_pending[b];
  const RunFlags* f = S->flags_host[b];
  const std::vector<uint64_t>& owners = S->flags_owner[b];
  {  // cancellations requested since the last look
    std::lock_guard<std::mutex> lk(S->mu);
    if (!S->cancel_req.empty())
      for (Request* r : S->resident)
        if (S->cancel_req.erase(r->ticket)) r->cancel = true;
  }
  std::unordered_map<uint64_t, Request*> live;
  live.reserve(S->resident.size() * 2 + 1);
  for (Request* r : S->resident) live.emplace(r->ticket, r);
  for (int i = 0; i < n; ++i) {
    const auto lv = live.find(owners[i]);
    if (lv == live.end()) continue;  // already retired
    Request* q = lv->second;
    if (!(f[i].done || q->cancel)) continue;
    live.erase(lv);
    S->resident.erase(std::find(S->resident.begin(), S->resident.end(), q));
    S->table_dirty = true;
    // a finished run's state no longer changes, so this snapshot is final
    RunState hrs;
    std::memset(&hrs, 0, sizeof(hrs));
    hrs.done = f[i].done;
    hrs.status = f[i].status;
    hrs.n_segments = f[i].n_segments;
    hrs.n_resamples = f[i].n_resamples;
    hrs.n_ess_near = f[i].n_ess_near;
    hrs.n_near = f[i].n_near;
    hrs.n_overflow = f[i].n_overflow;
    hrs.n_limit = f[i].n_limit;
    hrs.n_draws = f[i].n_draws;
    hrs.n_blocks = f[i].n_blocks;
    hrs.log_z_closed = f[i].log_z_closed;
    hrs.dbg_code = f[i].dbg_code;
    hrs.dbg_index = f[i].dbg_index;
    hrs.dbg_count = f[i].dbg_count;
    smc_status st = collect_run(q->model, &q->cfg, q->ly, q->ws, q->dev, hrs, q->result, S->stream);
    if (!st && q->ticket == S->fail_ticket)
      st = set_error(SMC_ECUDA, "injected failure retiring ticket %llu (SMC_SERVER_FAIL_TICKET)",
                     (unsigned long long)q->ticket);
    if (!st) {
      if (q->cancel) q->result->counters.status = SMC_ECANCELLED;
      cudaError_t e = cudaEventCreateWithFlags(&q->done_ev, cudaEventDisableTiming);
      if (e == cudaSuccess) e = cudaEventRecord(q->done_ev, S->stream);
      if (e == cudaSuccess) {
        e = cudaFreeAsync(q->ws, S->stream);  // stream-ordered after the copies
        if (e == cudaSuccess) q->ws = nullptr;
      }
      if (e != cudaSuccess) st = cuda_fail(e, "retiring a finished run");
    }
    if (st) {  // this request alone fails; the other runs go on
      fail_retiring(S, q, st);
      continue;
    }
    S->in_use -= q->bytes;
    S->completing.push_back(q);
    S->particle_steps += (int64_t)q->dev.N * hrs.n_segments;
  }
  S->flags_pending[b] = 0;
  S->n_resident = (int32_t)S->resident.size();
  return SMC_OK;
}

void reap(Server* S, bool block) {
  for (size_t i = 0; i < S->completing.size();) {
    Request* q = S->completing[i];
    cudaError_t e = block ? cudaEventSynchronize(q->done_ev) : cudaEventQuery(q->done_ev);
    if (e == cudaErrorNotReady) {
      ++i;
      continue;
    }
    cudaEventDestroy(q->done_ev);
    finish_ticket(S, q, e == cudaSuccess ? q->result->counters.status : SMC_ECUDA);
    S->completed += 1;
    delete q;
    S->completing[i] = S->completing.back();
    S->completing.pop_back();
  }
}

void worker_main(Server* S) {
  cudaSetDevice(S->device);
  int parity = 0;
  bool last_flags = false;
  smc_status err = SMC_OK;
  while (!err) {
    {
      NvtxRange nv("smc_server/admit");
      admit(S, &err);
    }
    if (err) break;
    if (S->resident.empty()) {
      if (last_flags) {
        cudaEventSynchronize(S->flags_ev[parity ^ 1]);
        S->flags_pending[parity ^ 1] = 0;
        last_flags = false;
      }
      reap(S, true);
      std::unique_lock<std::mutex> lk(S->mu);
      if (S->stop && S->queue.empty()) break;
      S->cv_work.wait_for(lk, std::chrono::milliseconds(2),
                          [&] { return S->stop || !S->queue.empty(); });
      continue;
    }
    if (S->table_dirty && (err = upload_table(S))) break;
    const int per_poll = std::max(1, S->cfg.poll_waves);
    NvtxRange nv_waves("smc_server/waves");
    for (int w = 0; w < per_poll && !err; ++w) {
      cudaError_t e = launch_wave(S->plan, S->cfg.precision, S->stream, (unsigned)S->waves.load());
      if (e != cudaSuccess) err = cuda_fail(e, "wave launch");
      S->waves += 1;
    }
    if (err) break;
    // flags of this wave into buffer `parity`
    const int n = (int)S->resident.size();
    gather_flags_kernel<<<(n + 127) / 128, 128, 0, S->stream>>>(S->plan.runs, n, S->flags_dev);
    cudaMemcpyAsync(S->flags_host[parity], S->flags_dev, sizeof(RunFlags) * n, cudaMemcpyDeviceToHost,
                    S->stream);
    cudaEventRecord(S->flags_ev[parity], S->stream);
    S->flags_owner[parity].clear();
    for (Request* q : S->resident) S->flags_owner[parity].push_back(q->ticket);
    S->flags_pending[parity] = n;
    // one wave behind: the flags of the previous wave
    if (last_flags) {
      if (cudaEventSynchronize(S->flags_ev[parity ^ 1]) != cudaSuccess) {
        err = set_error(SMC_ECUDA, "wave failed");
        break;
      }
      NvtxRange nv("smc_server/retire");
      if ((err = retire(S, parity ^ 1))) break;
    }
    last_flags = true;
    parity ^= 1;
    reap(S, false);
  }
  if (err) S->worker_error = err;
  // drain: fail whatever is left
  cudaStreamSynchronize(S->stream);
  reap(S, true);
  std::lock_guard<std::mutex> lk(S->mu);
  for (Request* q : S->resident) {
    if (q->ws) cudaFreeAsync(q->ws, S->stream);
    S->state[q->ticket] = T_FAILED;
    S->final_status[q->ticket] = err ? err : SMC_EINVAL;
    delete q;
  }
  S->resident.clear();
  for (Request* q : S->queue) {
    S->state[q->ticket] = T_FAILED;
    S->final_status[q->ticket] = err ? err : SMC_EINVAL;
    delete q;
  }
  S->queue.clear();
  S->cv_done.notify_all();
}

}  // namespace
}  // namespace smc

using namespace smc;

struct smc_server_s {
  Server s;
};

extern "C" smc_status smc_server_create(size_t device_mem_budget, const smc_server_cfg* cfg,
                                        smc_server_t* out) {
  if (!cfg || !out) return set_error(SMC_EINVAL, "NULL argument");
  if (cfg->precision != SMC_PREC_FP64 && cfg->precision != SMC_PREC_FP32)
    return set_error(SMC_EINVAL, "unknown precision");
  if (device_mem_budget < (1u << 20)) return set_error(SMC_EINVAL, "budget must be >= 1 MiB");
  smc_server_s* h = new (std::nothrow) smc_server_s();
  if (!h) return set_error(SMC_ENOMEM, "host allocation failed");
  Server* S = &h->s;
  S->cfg = *cfg;
  S->budget = device_mem_budget;
  cudaError_t e = cudaGetDevice(&S->device);
  if (e == cudaSuccess) e = cudaStreamCreateWithFlags(&S->stream, cudaStreamNonBlocking);
  if (e == cudaSuccess) e = cudaEventCreateWithFlags(&S->meta_ev, cudaEventDisableTiming);
  for (int b = 0; b < 2 && e == cudaSuccess; ++b)
    e = cudaEventCreateWithFlags(&S->flags_ev[b], cudaEventDisableTiming);
  if (e == cudaSuccess) {
    // keep freed workspaces in the stream-ordered pool between requests
    cudaMemPool_t pool;
    if (cudaDeviceGetDefaultMemPool(&pool, S->device) == cudaSuccess) {
      uint64_t thr = UINT64_MAX;
      cudaMemPoolSetAttribute(pool, cudaMemPoolAttrReleaseThreshold, &thr);
    }
  }
  if (e != cudaSuccess) {
    delete h;
    return cuda_fail(e, "server setup");
  }
  if (const char* inj = std::getenv("SMC_SERVER_FAIL_TICKET"))
    S->fail_ticket = std::strtoull(inj, nullptr, 10);
  if (S->cfg.max_resident_runs <= 0) S->cfg.max_resident_runs = 4096;
  if (S->cfg.poll_waves <= 0) S->cfg.poll_waves = 2;
  smc_status fs = alloc_flags(S, S->cfg.max_resident_runs);
  if (fs) {
    delete h;
    return fs;
  }
  S->worker = std::thread(worker_main, S);
  *out = h;
  return SMC_OK;
}

extern "C" smc_status smc_server_submit(smc_server_t h, smc_model_t m, const smc_run_cfg* c,
                                        smc_result* r, uint64_t* ticket) {
  if (!h || !ticket) return set_error(SMC_EINVAL, "NULL argument");
  smc_status st = check_cfg(m, c);
  if (st) return st;
  if ((st = check_result(r))) return st;
  Server* S = &h->s;
  if (c->precision != S->cfg.precision)
    return set_error(SMC_EINVAL, "request precision differs from the server's");
  if (c->resume_k != 0) return set_error(SMC_EINVAL, "resume is for smc_run only");
  if (S->worker_error) return set_error(S->worker_error, "server worker stopped after an error");
  Request* q = new (std::nothrow) Request();
  if (!q) return set_error(SMC_ENOMEM, "host allocation failed");
  q->model = m;
  q->cfg = *c;
  q->cfg.workspace = nullptr;
  q->result = r;
  q->ly = make_layout(m, &q->cfg);
  q->bytes = align_up(q->ly.total, 256);
  if (q->bytes > S->budget) {
    const size_t need = q->bytes;
    delete q;
    return set_error(SMC_ENOMEM, "request needs %zu bytes, more than the server budget", need);
  }
  q->t_submit = now_s();
  {
    std::lock_guard<std::mutex> lk(S->mu);
    if (S->stop) {
      delete q;
      return set_error(SMC_EBUSY, "server is shutting down");
    }
    q->ticket = S->next_ticket++;
    S->state[q->ticket] = T_QUEUED;
    S->queue.push_back(q);
    S->n_queued = (int32_t)S->queue.size();
  }
  S->cv_work.notify_one();
  *ticket = q->ticket;
  return SMC_OK;
}

extern "C" smc_status smc_server_poll(smc_server_t h, uint64_t ticket, int32_t* done) {
  if (!h || !done) return set_error(SMC_EINVAL, "NULL argument");
  Server* S = &h->s;
  std::lock_guard<std::mutex> lk(S->mu);
  auto it = S->state.find(ticket);
  if (it == S->state.end()) return set_error(SMC_EINVAL, "unknown ticket");
  *done = it->second >= T_DONE;
  if (*done) return S->final_status[ticket];
  return SMC_OK;
}

extern "C" smc_status smc_server_wait(smc_server_t h, uint64_t ticket, double timeout_s,
                                      double* latency_s) {
  if (!h) return set_error(SMC_EINVAL, "NULL server");
  Server* S = &h->s;
  std::unique_lock<std::mutex> lk(S->mu);
  auto it = S->state.find(ticket);
  if (it == S->state.end()) return set_error(SMC_EINVAL, "unknown ticket");
  const bool ok = S->cv_done.wait_for(lk, std::chrono::duration<double>(std::max(0.0, timeout_s)),
                                      [&] { return S->state[ticket] >= T_DONE; });
  if (!ok) return set_error(SMC_ETIMEOUT, "ticket %llu not finished within %.3f s",
                            (unsigned long long)ticket, timeout_s);
  if (latency_s) *latency_s = S->latency[ticket];
  const int st = S->final_status[ticket];
  return st;
}

extern "C" smc_status smc_server_cancel(smc_server_t h, uint64_t ticket) {
  if (!h) return set_error(SMC_EINVAL, "NULL server");
  Server* S = &h->s;
  std::lock_guard<std::mutex> lk(S->mu);
  auto it = S->state.find(ticket);
  if (it == S->state.end()) return set_error(SMC_EINVAL, "unknown ticket");
  if (it->second >= T_COMPLETING) return SMC_OK;
  if (it->second == T_QUEUED) {
    for (Request* q : S->queue)
      if (q->ticket == ticket) q->cancel = true;
  } else {
    S->cancel_req.insert(ticket);  // the worker marks the resident run
  }
  return SMC_OK;
}

extern "C" smc_status smc_server_stats(smc_server_t h, smc_server_stats_t* out) {
  if (!h || !out) return set_error(SMC_EINVAL, "NULL argument");
  Server* S = &h->s;
  out->waves = S->waves;
  out->completed = S->completed;
  out->particle_steps = S->particle_steps;
  out->resident = S->n_resident;
  out->queued = S->n_queued;
  out->worker_status = S->worker_error;
  out->pad_ = 0;
  return SMC_OK;
}

extern "C" void smc_server_destroy(smc_server_t h) {
  if (!h) return;
  Server* S = &h->s;
  {
    std::lock_guard<std::mutex> lk(S->mu);
    S->stop = true;
  }
  S->cv_work.notify_all();
  if (S->worker.joinable()) S->worker.join();
  if (S->meta) cudaFreeAsync(S->meta, S->stream);
  cudaStreamSynchronize(S->stream);
  if (S->pinned_meta) cudaFreeHost(S->pinned_meta);
  if (S->flags_dev) cudaFree(S->flags_dev);
  for (int b = 0; b < 2; ++b) {
    if (S->flags_host[b]) cudaFreeHost(S->flags_host[b]);
    if (S->flags_ev[b]) cudaEventDestroy(S->flags_ev[b]);
  }
  if (S->meta_ev) cudaEventDestroy(S->meta_ev);
  if (S->stream) cudaStreamDestroy(S->stream);
  delete h;
}
