// FP32 instantiations of the fused line kernel (the mixed form) with
// 8-row thread chunks.
#include "sweeps.cuh"

namespace ppk {
cudaError_t launch_sweep_f32_m8(const LaunchCfg &c, const SweepArgs &a, long long nlines,
                                 cudaStream_t st) {
  return launch_dispatch<float, 8>(c, a, nlines, st);
}
}  // namespace ppk
