// sweep_f64.cu - FP64 instantiations of the residual sweep (plain double precision).
#include "sweep.cuh"

namespace fpk {
cudaError_t launch_sweep_f64(const SweepLaunch &L, int M, int scheme, int charwise, int fp,
                             cudaStream_t s) {
  return launch_sweep_t<double>(L, M, scheme, charwise, fp, s);
}
int prepare_sweep_f64(int M, int scheme) { return prepare_t<double>(M, scheme); }
}  // namespace fpk
