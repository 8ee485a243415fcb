// smc_prims.cu -- the resampling primitives of Section 3.3 as standalone
// HBM-streaming kernels, the particle-duplication gather, the random-number
// parity hooks, and the library's error plumbing.
//
// smc_resample (parallel systematic resampling, three launches):
//   1. rs_tile_reduce: per tile of TPB*IT weights, M_t = max, its power-of-two
//      reference k_t = ceil(M_t / ln 2) and s_t = sum exp(x - k_t ln 2)
//   2. rs_combine (one CTA): k = max k_t, c_t = 2^(k_t - k) (exact), O_t =
//      exclusive prefix of c_t s_t (O_{T} = S), out3 = {k ln 2, S,
//      k ln 2 + (log S - log N)}, r = N / S; no exponential per tile
//   3. rs_ancestors: per tile, E_j = inclusive scan of exp(x_j - k_t ln 2),
//      q_j = (O_t + c_t E_j) r clamped to the tile's [O_t r, O_{t+1} r); element
//      j owns the offsets i with q_{j-1} <= i + u < q_j and writes a_i = j for
//      them (the last element owns everything above), so every i is written
//      exactly once and a_i = min{ j : q_j > i + u } up to rounding at tile seams.
#include <cuda_runtime.h>

#include <cmath>
#include <cstdarg>
#include <cstdio>
#include <cstring>
#include <mutex>

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

constexpr int RS_TPB = 256;
constexpr int RS_IT = 16;
constexpr int RS_TILE = RS_TPB * RS_IT;

__device__ __forceinline__ void load_tile(const double* __restrict__ x, int64_t N, int64_t base,
                                          double (&v)[RS_IT]) {
  const int64_t j0 = base + (int64_t)threadIdx.x * RS_IT;
  if (j0 + RS_IT <= N) {
    const double2* p = reinterpret_cast<const double2*>(x + j0);
#pragma unroll
    for (int q = 0; q < RS_IT / 2; ++q) {
      const double2 d = __ldcs(p + q);
      v[2 * q] = d.x;
      v[2 * q + 1] = d.y;
    }
  } else {
#pragma unroll
    for (int q = 0; q < RS_IT; ++q) v[q] = (j0 + q < N) ? x[j0 + q] : -INFINITY;
  }
}

__global__ void __launch_bounds__(RS_TPB) rs_tile_reduce(const double* __restrict__ x, int64_t N,
                                                         int32_t* __restrict__ tk,
                                                         double* __restrict__ ts) {
  __shared__ double sh[RS_TPB / 32 + 1];
  double v[RS_IT];
  load_tile(x, N, (int64_t)blockIdx.x * RS_TILE, v);
  double mx = -INFINITY;
#pragma unroll
  for (int q = 0; q < RS_IT; ++q) mx = fmax(mx, v[q]);
  const double Mt = block_max<RS_TPB>(mx, sh);
  const int kt = Mt == -INFINITY ? kDeadTile : tile_exponent(Mt);
  double s = 0.0;
  if (kt != kDeadTile) {
    const double R = (double)kt * kLn2;
#pragma unroll
    for (int q = 0; q < RS_IT; ++q) s = s + exp(v[q] - R);
  }
  const double tot = block_incl_scan<RS_TPB>(s, sh);
  if (threadIdx.x == RS_TPB - 1) {
    tk[blockIdx.x] = kt;
    ts[blockIdx.x] = tot;
  }
}

// Single CTA: combine nt tile results.  tO has nt + 1 entries (tO[nt] = S).
__global__ void __launch_bounds__(RS_TPB) rs_combine(const int32_t* __restrict__ tk,
                                                     const double* __restrict__ ts, int nt,
                                                     int64_t N, double* __restrict__ tc,
                                                     double* __restrict__ tO, double* out3,
                                                     double* r_out) {
  __shared__ double sh[RS_TPB / 32 + 2 + RS_TPB];
  int kloc = kDeadTile;
  for (int t = threadIdx.x; t < nt; t += RS_TPB) kloc = max(kloc, tk[t]);
  const int kmax = block_max_int<RS_TPB>(kloc, reinterpret_cast<int*>(sh));
  if (kmax == kDeadTile) {
    if (threadIdx.x == 0) {
      out3[0] = -INFINITY;
      out3[1] = 0.0;
      out3[2] = -INFINITY;
      *r_out = 0.0;
    }
    return;
  }
  double carry = 0.0;
  for (int base = 0; base < nt; base += RS_TPB) {
    const int t = base + threadIdx.x;
    double c = 0.0, v = 0.0;
    if (t < nt) {
      const int kt = tk[t];
      c = (kt == kDeadTile) ? 0.0 : pow2i(kt - kmax);
      v = ts[t] * c;  // exact: c is a power of two
    }
    const double incl = block_incl_scan<RS_TPB>(v, sh);
    __syncthreads();
    sh[RS_TPB / 32 + 1 + threadIdx.x] = incl;
    __syncthreads();
    const double excl = threadIdx.x ? sh[RS_TPB / 32 + threadIdx.x] : 0.0;
    if (t < nt) {
      tc[t] = c;
      tO[t] = carry + excl;
    }
    carry = carry + sh[RS_TPB / 32 + RS_TPB];
  }
  if (threadIdx.x == 0) {
    const double m = (double)kmax * kLn2;
    tO[nt] = carry;
    out3[0] = m;
    out3[1] = carry;
    out3[2] = m + (log(carry) - log((double)N));
    *r_out = (double)N / carry;
  }
}

// first offset index c in [0, N] with fl(c + u) >= bound (bound finite, >= 0)
__device__ __forceinline__ int64_t first_at_or_above(double bound, double u, int64_t N) {
  if (!(bound < (double)N + 1.0)) return N;
  double g = ceil(bound - u);
  int64_t c = g < 0.0 ? 0 : (int64_t)g;
  if (c > N) c = N;
  while (c > 0 && (double)(c - 1) + u >= bound) --c;
  while (c < N && (double)c + u < bound) ++c;
  return c;
}

__global__ void __launch_bounds__(RS_TPB) rs_ancestors(
    const double* __restrict__ x, int64_t N, double u, const int32_t* __restrict__ tk,
    const double* __restrict__ tc, const double* __restrict__ tO, const double* __restrict__ out3,
    const double* __restrict__ r_p, int32_t* __restrict__ anc, unsigned long long* n_near) {
  __shared__ double sh[RS_TPB / 32 + 1];
  __shared__ double sh_last[RS_TPB];
  const int t = blockIdx.x;
  const int64_t base = (int64_t)t * RS_TILE;
  const int64_t j0 = base + (int64_t)threadIdx.x * RS_IT;
  if (out3[0] == -INFINITY) {  // degenerate population: identity
    for (int q = 0; q < RS_IT; ++q)
      if (j0 + q < N) anc[j0 + q] = (int32_t)(j0 + q);
    return;
  }
  double v[RS_IT];
  load_tile(x, N, base, v);
  const int kt = tk[t];
  const double c = tc[t], O = tO[t], r = *r_p;
  const double R = kt == kDeadTile ? 0.0 : (double)kt * kLn2;
  const double lo_tile = O * r, hi_tile = tO[t + 1] * r;
  double loc = 0.0;
#pragma unroll
  for (int q = 0; q < RS_IT; ++q) {
    const double e = (kt == kDeadTile) ? 0.0 : exp(v[q] - R);
    loc = loc + e;
    v[q] = loc;  // thread-local inclusive prefix
  }
  const double incl = block_incl_scan<RS_TPB>(loc, sh);
  const double excl = incl - loc;  // only used to offset this thread's prefixes
  // The tile's offsets are split between threads at the running maximum of
  // each thread's last (clamped) boundary, so that consecutive threads hand
  // over exactly the same value even where rounding makes the per-thread
  // prefixes disagree in the last bit.
  double q_prev_thread_last;
  {
    const double Elast = excl + v[RS_IT - 1];
    const double ql = fmin((O + c * Elast) * r, hi_tile);
    const double pm = block_incl_max<RS_TPB>(fmax(ql, lo_tile), sh);
    sh_last[threadIdx.x] = pm;
    __syncthreads();
    q_prev_thread_last = threadIdx.x ? sh_last[threadIdx.x - 1] : lo_tile;
  }
  const double tol = kBoundaryEps * (double)N;
  double lo = q_prev_thread_last;
  unsigned long long near = 0;
#pragma unroll 1
  for (int q = 0; q < RS_IT; ++q) {
    const int64_t j = j0 + q;
    if (j >= N) break;
    const double qraw = (O + c * (excl + v[q])) * r;
    double hi = fmin(qraw, hi_tile);
    if (hi < lo) hi = lo;
    const int64_t i0 = first_at_or_above(lo, u, N);
    const int64_t i1 = (j == N - 1) ? N : first_at_or_above(hi, u, N);
    for (int64_t i = i0; i < i1; ++i) {
      anc[i] = (int32_t)j;
      const double y = (double)i + u;
      if (fabs(qraw - y) < tol || fabs(lo - y) < tol) ++near;
    }
    lo = hi;
  }
  near = __reduce_add_sync(0xffffffffu, (unsigned)near);
  if ((threadIdx.x & 31) == 0 && near) atomicAdd(n_near, near);
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
    default: v = (double)lognormal<R>(s, p1); break;
  }
  out[i] = v;
  if (blocks) blocks[i] = (int32_t)s.d;
}

__global__ void math_eval_kernel(int fn, const double* __restrict__ x, double* __restrict__ y,
                                 int64_t n, const MathTab* tab) {
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  const double v = x[i];
  const unsigned long long bits = (unsigned long long)__double_as_longlong(v);
  switch (fn) {
    case 0: y[i] = tang_log(v, tab); break;
    case 1: y[i] = tang_exp(v, tab); break;
    case 2: y[i] = log(v); break;
    case 3: y[i] = exp(v); break;
    case 4: y[i] = log_unif53(bits, tab); break;
    default: y[i] = tang_log(Unif<double>::from64(bits), tab); break;
  }
}

}  // namespace smc

using namespace smc;

extern "C" smc_status smc_math_eval(int32_t fn, const double* x, double* y, int64_t n, void* stream) {
  if (!x || !y || n < 0 || fn < 0 || fn > 5) return set_error(SMC_EINVAL, "bad argument");
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

extern "C" size_t smc_resample_workspace_bytes(int64_t N) {
  if (N < 1) return 0;
  const size_t nt = (size_t)((N + RS_TILE - 1) / RS_TILE);
  return align_up(8 * nt, 256) * 3 + align_up(8 * (nt + 1), 256) + 256;
}

extern "C" smc_status smc_resample(const double* logw, int64_t N, double u, int32_t* ancestors,
                                   double* out3, int64_t* n_near, void* workspace,
                                   size_t workspace_bytes, void* stream) {
  if (!logw || !ancestors || !out3 || !n_near || !workspace)
    return set_error(SMC_EINVAL, "NULL pointer");
  if (N < 1 || N > 0x7fffffffLL) return set_error(SMC_EINVAL, "N must be in 1..2^31-1");
  if (!(u > 0.0 && u < 1.0)) return set_error(SMC_EINVAL, "u must be in (0,1)");
  if (workspace_bytes < smc_resample_workspace_bytes(N))
    return set_error(SMC_EINVAL, "workspace too small");
  if ((reinterpret_cast<uintptr_t>(logw) & 15) != 0)
    return set_error(SMC_EINVAL, "logw must be 16-byte aligned");
  cudaStream_t cs = (cudaStream_t)stream;
  const int nt = (int)((N + RS_TILE - 1) / RS_TILE);
  char* w = (char*)workspace;
  int32_t* tM = (int32_t*)w;
  double* ts = (double*)(w + align_up(8 * (size_t)nt, 256));
  double* tc = (double*)(w + 2 * align_up(8 * (size_t)nt, 256));
  double* tO = (double*)(w + 3 * align_up(8 * (size_t)nt, 256));
  double* r = (double*)(w + 3 * align_up(8 * (size_t)nt, 256) + align_up(8 * (size_t)(nt + 1), 256));
  SMC_CUDA_TRY(cudaMemsetAsync(n_near, 0, sizeof(int64_t), cs));
  rs_tile_reduce<<<nt, RS_TPB, 0, cs>>>(logw, N, tM, ts);
  SMC_CUDA_TRY(cudaGetLastError());
  rs_combine<<<1, RS_TPB, 0, cs>>>(tM, ts, nt, N, tc, tO, out3, r);
  SMC_CUDA_TRY(cudaGetLastError());
  rs_ancestors<<<nt, RS_TPB, 0, cs>>>(logw, N, u, tM, tc, tO, out3, r, ancestors,
                                      reinterpret_cast<unsigned long long*>(n_near));
  SMC_CUDA_TRY(cudaGetLastError());
  return SMC_OK;
}

// ---------------------------------------------------------------------------
// smc_resample_static: smc_resample with its scratch in a fixed device array.
//
// Some callers cannot call cudaMalloc (code whose device memory is owned by
// another framework's pool, paths where an allocation's implicit device-wide
// synchronisation is not allowed, hosts that forbid allocation after start-up).
// For them the tile scratch of the three resampling kernels lives in this
// file-scope array, sized for populations of up to SMC_RESAMPLE_STATIC_MAX_N
// particles (4096 tiles): 3 x 4096 tile values + 4097 offsets + N/S, 131,136
// bytes that every GPU which loads the library keeps until the process exits.
// Every call shares the array and it keeps the last call's contents; nothing in
// it has to start at zero (each call writes every entry it later reads), but two
// calls that overlap on the GPU race on it.
constexpr int kStaticTiles = (int)((SMC_RESAMPLE_STATIC_MAX_N + RS_TILE - 1) / RS_TILE);
constexpr int kStaticDoubles = 3 * kStaticTiles + (kStaticTiles + 1) + 7;
static __device__ __align__(256) double g_resample_scratch[kStaticDoubles];

namespace {
std::mutex g_static_mu;
double* g_static_ptr[128] = {nullptr};  // device address of the array, per device

// Once per device, with that device current: resolve the array's device address.
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
  cudaStream_t cs = (cudaStream_t)stream;
  const int nt = (int)((N + RS_TILE - 1) / RS_TILE);
  int32_t* tM = reinterpret_cast<int32_t*>(base);
  double* ts = base + kStaticTiles;
  double* tc = base + 2 * kStaticTiles;
  double* tO = base + 3 * kStaticTiles;            // nt + 1 entries
  double* r = base + 4 * kStaticTiles + 1;
  SMC_CUDA_TRY(cudaMemsetAsync(n_near, 0, sizeof(int64_t), cs));
  rs_tile_reduce<<<nt, RS_TPB, 0, cs>>>(logw, N, tM, ts);
  SMC_CUDA_TRY(cudaGetLastError());
  rs_combine<<<1, RS_TPB, 0, cs>>>(tM, ts, nt, N, tc, tO, out3, r);
  SMC_CUDA_TRY(cudaGetLastError());
  rs_ancestors<<<nt, RS_TPB, 0, cs>>>(logw, N, u, tM, tc, tO, out3, r, ancestors,
                                      reinterpret_cast<unsigned long long*>(n_near));
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
  if (!out || n < 0 || dist < 0 || dist > 7) return set_error(SMC_EINVAL, "bad argument");
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
