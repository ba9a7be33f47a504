// sweep_f32_bnd.cu - FP32 residual sweep with the slip-wall, cut, link and halo rules compiled in,
// switches read at run time.
#include "sweep.cuh"

namespace fpk {
FPK_SWEEP_UNIT(f32_bnd, float, true, 0)
}  // namespace fpk
