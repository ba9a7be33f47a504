// sweep_f32_bnd_fix2.cu - FP32 residual sweep with the slip-wall, cut, link and halo rules
// compiled in, switches folded, alternative CTA shape (sweep_threads with fix = 2).
#include "sweep.cuh"

namespace fpk {
FPK_SWEEP_UNIT(f32_bnd_fix2, float, true, 2)
}  // namespace fpk
