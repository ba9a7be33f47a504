// sweep_f64.cu - FP64 instantiations of the residual sweep (plain double precision),
// for directions without slip-wall or cut sides.
#include "sweep.cuh"

namespace fpk {
cudaError_t launch_sweep_f64(const SweepLaunch &L, int M, int scheme, int charwise, int fp,
                             cudaStream_t s) {
  return L.bnd ? launch_sweep_f64_bnd(L, M, scheme, charwise, fp, s)
               : launch_sweep_t<double, false>(L, M, scheme, charwise, fp, s);
}
int prepare_sweep_f64(int M, int scheme) {
  const int a = prepare_t<double, false>(M, scheme), b = prepare_sweep_f64_bnd(M, scheme);
  return a < b ? a : b;
}
}  // namespace fpk
