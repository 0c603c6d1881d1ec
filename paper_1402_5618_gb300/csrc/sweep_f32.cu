// FP32 instantiations of the fused line kernel (the mixed form: line
// arithmetic in FP32, state and stage combination in FP64).
#include "sweeps.cuh"

namespace ppk {
cudaError_t launch_sweep_f32(const LaunchCfg &c, const SweepArgs &a, long long nlines,
                             cudaStream_t st) {
  return launch_dispatch<float>(c, a, nlines, st);
}
}  // namespace ppk
