// FP64 instantiations of the fused line kernel (the plain form).
#include "sweeps.cuh"

namespace ppk {
cudaError_t launch_sweep_f64(const LaunchCfg &c, const SweepArgs &a, long long nlines,
                             cudaStream_t st) {
  return launch_dispatch<double>(c, a, nlines, st);
}
}  // namespace ppk
