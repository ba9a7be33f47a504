// sweep2_f32.cu - instantiations of the two-lines-per-thread FP32 sweep (sweep2.cuh):
// WENO5-JS and linear upwind at metric orders 2, 4, 6, 8.
#include "sweep2.cuh"

namespace fpk {

cudaError_t launch_sweep2_f32(const SweepLaunch &L, int M, int scheme, int charwise, int fp, cudaStream_t s) {
#define FPK_CASE2(MM, SS) \
  if (M == MM && scheme == SS) return launch_one2<MM, SS>(L, charwise, fp, s);
  FPK_CASE2(2, 0) FPK_CASE2(4, 0) FPK_CASE2(6, 0) FPK_CASE2(8, 0)
  FPK_CASE2(2, 1) FPK_CASE2(4, 1) FPK_CASE2(6, 1) FPK_CASE2(8, 1)
#undef FPK_CASE2
  return cudaErrorInvalidValue;
}

int prepare_sweep2_f32(int M, int scheme) {
  int nb = 0;
#define FPK_OCC2(MM, SS)                                                                            \
  {                                                                                                 \
    cudaFuncSetAttribute(fp_sweep2<MM, SS>, cudaFuncAttributeMaxDynamicSharedMemorySize,            \
                         (int)kSweep2Smem);                                                         \
    if (M == MM && scheme == SS)                                                                    \
      cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, fp_sweep2<MM, SS>, kThreads, kSweep2Smem); \
  }
  FPK_OCC2(2, 0) FPK_OCC2(4, 0) FPK_OCC2(6, 0) FPK_OCC2(8, 0)
  FPK_OCC2(2, 1) FPK_OCC2(4, 1) FPK_OCC2(6, 1) FPK_OCC2(8, 1)
#undef FPK_OCC2
  return nb > 0 ? nb : 1;
}

}  // namespace fpk
