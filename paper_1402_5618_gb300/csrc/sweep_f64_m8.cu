// FP64 instantiations of the fused line kernel (the plain form) with
// 8-row thread chunks.
#include "sweeps.cuh"

namespace ppk {
cudaError_t launch_sweep_f64_m8(const LaunchCfg &c, const SweepArgs &a, long long nlines,
                                 cudaStream_t st) {
  return launch_dispatch<double, 8>(c, a, nlines, st);
}
}  // namespace ppk
