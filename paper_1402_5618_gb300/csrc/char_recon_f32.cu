// FP32 instantiation of the characteristic-wise reconstruction (the mixed
// form: FP32 line arithmetic on the hi parts of the state).
#include "char_recon_kernel.cuh"

namespace ppk {
cudaError_t launch_char_recon_f32(const CharArgs &a, int nv, bool periodic, int part, cudaStream_t st) {
  return chr::launch_char_recon_t<float>(a, nv, periodic, part, st);
}
}  // namespace ppk
