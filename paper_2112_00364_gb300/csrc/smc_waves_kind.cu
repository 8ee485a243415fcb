// smc_waves_kind.cu -- the wave kernels of the linear-Gaussian and CRBD models
// alone.  A wave whose runs all run one of these models launches a kernel with
// only that model's block table compiled in (wave_kernel<R, TPB, KIND>, the
// per-tile code of smc_step.cuh), instead of the kernel that dispatches on each
// run's model: the same code path, so the same bits, with the code and
// registers of one model.  Kept in a translation unit of its own so that it
// compiles beside the dispatching kernels.
#include <cuda_runtime.h>

#include "smc_engine.h"
#include "smc_step.cuh"

namespace smc {

namespace {
template <int KIND>
cudaError_t launch_kind(const WavePlan& W, int precision, cudaStream_t st, unsigned wave) {
  for (int b = 0; b < 4; ++b) {
    if (!W.n_ctas[b]) continue;
    cudaError_t e = precision == SMC_PREC_FP32
                        ? launch_bucket<float, KIND>(b, W.runs, W.maps[b], W.n_ctas[b], st, wave)
                        : launch_bucket<double, KIND>(b, W.runs, W.maps[b], W.n_ctas[b], st, wave);
    if (e != cudaSuccess) return e;
  }
  return cudaSuccess;
}
}  // namespace

cudaError_t launch_wave_kind(const WavePlan& W, int precision, cudaStream_t st, unsigned wave) {
  return W.kind == SMC_MODEL_LG ? launch_kind<SMC_MODEL_LG>(W, precision, st, wave)
                                : launch_kind<SMC_MODEL_CRBD>(W, precision, st, wave);
}

}  // namespace smc
