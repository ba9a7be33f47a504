// sweep_f32_fix2.cu - FP32 residual sweep, plain sides, switches folded, alternative CTA shape
// (sweep_threads with fix = 2).
#include "sweep.cuh"

namespace fpk {
FPK_SWEEP_UNIT(f32_fix2, float, false, 2)
}  // namespace fpk
