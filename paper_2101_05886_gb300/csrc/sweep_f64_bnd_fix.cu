// sweep_f64_bnd_fix.cu - FP64 residual sweep with the slip-wall, cut, link and halo rules compiled in,
// characteristic decomposition and FP form fixed on at compile time.
#include "sweep.cuh"

namespace fpk {
FPK_SWEEP_UNIT(f64_bnd_fix, double, true, 1)
}  // namespace fpk
