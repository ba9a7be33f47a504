// sweep_f32_bnd.cu - FP32 instantiations of the residual sweep with the slip-wall and
// C-grid cut boundary rules compiled in.
#include "sweep.cuh"

namespace fpk {
cudaError_t launch_sweep_f32_bnd(const SweepLaunch &L, int M, int scheme, int charwise, int fp,
                                 cudaStream_t s) {
  return launch_sweep_t<float, true>(L, M, scheme, charwise, fp, s);
}
int prepare_sweep_f32_bnd(int M, int scheme) { return prepare_t<float, true>(M, scheme); }
}  // namespace fpk
