// smc_probe.cu -- compute-peak probe: the throughput of the arithmetic the
// path's kernels use (FP64 and FP32 fused multiply-add, the special function
// unit's ex2, the 32-bit integer multiply-add, the 64-bit multiply-high),
// measured on the device at hand for the rooflines' denominators.
#include <cuda_runtime.h>

#include "smc_engine.h"
#include "smc_internal.h"

namespace smc {

// ---- compute peaks of the arithmetic the path uses, measured ----
// Eight independent dependency chains per thread, `iters` steps each, on a
// grid of 8 x 256-thread CTAs per SM: kind 0 = FP64 fused multiply-add,
// 1 = FP32 fused multiply-add, 2 = the FP32 base-2 exponential of the special
// function unit (ex2.approx), 3 = the 32-bit integer multiply-add, 4 = the
// 64-bit unsigned multiply-high (the integer chains multiply by a neighbouring
// chain's value, so that no step can be folded into the next).  Each thread writes its chains' sum to
// sink[thread] (so that nothing is optimised away).
template <int KIND>
__global__ void __launch_bounds__(256) peak_kernel(int64_t iters, double* __restrict__ sink) {
  const unsigned tid = blockIdx.x * blockDim.x + threadIdx.x;
  double out = 0.0;
  if (KIND == 0) {
    double a[8];
    const double m = 0.999999, c = 1e-7;
#pragma unroll
    for (int q = 0; q < 8; ++q) a[q] = 1.0 + 1e-3 * (double)((tid + q) & 15);
    for (int64_t i = 0; i < iters; ++i) {
#pragma unroll
      for (int q = 0; q < 8; ++q) a[q] = fma(a[q], m, c);
    }
#pragma unroll
    for (int q = 0; q < 8; ++q) out += a[q];
  } else if (KIND == 1) {
    float a[8];
    const float m = 0.9999f, c = 1e-5f;
#pragma unroll
    for (int q = 0; q < 8; ++q) a[q] = 1.0f + 1e-3f * (float)((tid + q) & 15);
    for (int64_t i = 0; i < iters; ++i) {
#pragma unroll
      for (int q = 0; q < 8; ++q) a[q] = fmaf(a[q], m, c);
    }
#pragma unroll
    for (int q = 0; q < 8; ++q) out += (double)a[q];
  } else if (KIND == 2) {
    float a[8];
#pragma unroll
    for (int q = 0; q < 8; ++q) a[q] = -1e-3f * (float)((tid + q) & 15);
    for (int64_t i = 0; i < iters; ++i) {
#pragma unroll
      for (int q = 0; q < 8; ++q) {
        float y;
        asm volatile("ex2.approx.ftz.f32 %0, %1;" : "=f"(y) : "f"(a[q]));
        a[q] = -y;  // stays in (-1, 0]: the chain neither overflows nor settles
      }
    }
#pragma unroll
    for (int q = 0; q < 8; ++q) out += (double)a[q];
  } else if (KIND == 3) {
    unsigned a[8];
#pragma unroll
    for (int q = 0; q < 8; ++q) a[q] = tid * 2654435761u + q;
    for (int64_t i = 0; i < iters; ++i) {  // products of two chains: nothing to fold
      unsigned b[8];
#pragma unroll
      for (int q = 0; q < 8; ++q) b[q] = a[q] * a[(q + 1) & 7] + 1013904223u;
#pragma unroll
      for (int q = 0; q < 8; ++q) a[q] = b[q];
    }
#pragma unroll
    for (int q = 0; q < 8; ++q) out += (double)a[q];
  } else {
    unsigned long long a[8];
#pragma unroll
    for (int q = 0; q < 8; ++q) a[q] = ((unsigned long long)tid << 32) | (0x9e3779b9u + q);
    for (int64_t i = 0; i < iters; ++i) {
      unsigned long long b[8];
#pragma unroll
      for (int q = 0; q < 8; ++q) b[q] = __umul64hi(a[q], a[(q + 1) & 7] | 1ull);
#pragma unroll
      for (int q = 0; q < 8; ++q) a[q] = b[q] | (1ull << 63);  // never collapses to 0
    }
#pragma unroll
    for (int q = 0; q < 8; ++q) out += (double)(a[q] & 0xffff);
  }
  sink[tid] = out;
}

}  // namespace smc

using namespace smc;

extern "C" int64_t smc_peak_probe_threads(void) {
  int dev = 0, sms = 0;
  if (cudaGetDevice(&dev) != cudaSuccess) return 0;
  if (cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess) return 0;
  return (int64_t)sms * 8 * 256;
}

extern "C" smc_status smc_peak_probe(int32_t kind, int64_t iters, double* sink, void* stream) {
  if (!sink || iters < 1 || kind < 0 || kind > 4) return set_error(SMC_EINVAL, "bad argument");
  const int64_t threads = smc_peak_probe_threads();
  if (threads < 256) return set_error(SMC_ECUDA, "no device");
  const unsigned grid = (unsigned)(threads / 256);
  cudaStream_t cs = (cudaStream_t)stream;
  switch (kind) {
    case 0: peak_kernel<0><<<grid, 256, 0, cs>>>(iters, sink); break;
    case 1: peak_kernel<1><<<grid, 256, 0, cs>>>(iters, sink); break;
    case 2: peak_kernel<2><<<grid, 256, 0, cs>>>(iters, sink); break;
    case 3: peak_kernel<3><<<grid, 256, 0, cs>>>(iters, sink); break;
    default: peak_kernel<4><<<grid, 256, 0, cs>>>(iters, sink); break;
  }
  SMC_CUDA_TRY(cudaGetLastError());
  return SMC_OK;
}

