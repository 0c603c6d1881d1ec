// FP64 instantiation of the characteristic-wise reconstruction (the plain form).
#include "char_recon_kernel.cuh"

namespace ppk {
cudaError_t launch_char_recon_f64(const CharArgs &a, int nv, bool periodic, int part, cudaStream_t st) {
  return chr::launch_char_recon_t<double>(a, nv, periodic, part, st);
}
}  // namespace ppk
