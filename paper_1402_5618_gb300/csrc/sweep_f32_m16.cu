// FP32 instantiations of the fused line kernel (the mixed form) with
// 16-row thread chunks.
#include "sweeps.cuh"

namespace ppk {
cudaError_t launch_sweep_f32_m16(const LaunchCfg &c, const SweepArgs &a, long long nlines,
                                  cudaStream_t st) {
  return launch_dispatch<float, 16>(c, a, nlines, st);
}
}  // namespace ppk
