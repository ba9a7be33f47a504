// sweep_f32.cu - FP32 instantiations of the residual sweep (FP32 state and
// arithmetic on metrics that were built in FP64), for directions without slip-wall
// or cut sides; sweep_f32_bnd.cu holds the variants with those boundary rules.
#include "sweep.cuh"

namespace fpk {
cudaError_t launch_sweep_f32(const SweepLaunch &L, int M, int scheme, int charwise, int fp,
                             cudaStream_t s) {
  return L.bnd ? launch_sweep_f32_bnd(L, M, scheme, charwise, fp, s)
               : launch_sweep_t<float, false>(L, M, scheme, charwise, fp, s);
}
int prepare_sweep_f32(int M, int scheme) {
  const int a = prepare_t<float, false>(M, scheme), b = prepare_sweep_f32_bnd(M, scheme);
  return a < b ? a : b;
}
}  // namespace fpk
