// sweep_f32_fix.cu - FP32 residual sweep, plain sides, characteristic decomposition and FP form fixed
// on at compile time.
#include "sweep.cuh"

namespace fpk {
FPK_SWEEP_UNIT(f32_fix, float, false, 1)
}  // namespace fpk
