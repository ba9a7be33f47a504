// sweep_f32.cu - FP32 instantiations of the residual sweep (FP32 state and
// arithmetic on metrics that were built in FP64).
#include "sweep.cuh"

namespace fpk {
cudaError_t launch_sweep_f32(const SweepLaunch &L, int M, int scheme, int charwise, int fp,
                             cudaStream_t s) {
  return launch_sweep_t<float>(L, M, scheme, charwise, fp, s);
}
int prepare_sweep_f32(int M, int scheme) { return prepare_t<float>(M, scheme); }
}  // namespace fpk
