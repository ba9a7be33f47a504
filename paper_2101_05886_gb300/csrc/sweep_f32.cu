// sweep_f32.cu - FP32 instantiations of the residual sweep (FP32 state and arithmetic on metrics that
// were built in FP64) for directions without slip-wall, cut, link or halo sides, with the
// characteristic and FP-form switches read at run time.
#include "sweep.cuh"

namespace fpk {
FPK_SWEEP_UNIT(f32, float, false, 0)
}  // namespace fpk
