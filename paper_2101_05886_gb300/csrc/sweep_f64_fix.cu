// sweep_f64_fix.cu - FP64 residual sweep, plain sides, characteristic decomposition and FP form fixed
// on at compile time.
#include "sweep.cuh"

namespace fpk {
FPK_SWEEP_UNIT(f64_fix, double, false, 1)
}  // namespace fpk
