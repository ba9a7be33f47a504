// sweep_f64_bnd.cu - FP64 residual sweep with the slip-wall, cut, link and halo rules compiled in,
// switches read at run time.
#include "sweep.cuh"

namespace fpk {
FPK_SWEEP_UNIT(f64_bnd, double, true, 0)
}  // namespace fpk
