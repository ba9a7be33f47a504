// sweep_f64.cu - FP64 instantiations of the residual sweep (plain double precision) for directions
// without slip-wall, cut, link or halo sides, switches read at run time.
#include "sweep.cuh"

namespace fpk {
FPK_SWEEP_UNIT(f64, double, false, 0)
}  // namespace fpk
