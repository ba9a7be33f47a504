// cfl.cu - time-step bound: max over points of sum_d (|u . grad d| + c |grad d|),
// grad d = J (d_x, d_y, d_z)/J, reduced to one value per launch.
#include <cuda_runtime.h>
#include <math.h>

#include "fp_internal.h"

namespace fpk {

namespace {

template <typename T>
__global__ void k_cfl(const BlockDev *blk, long long ncells, int ni, int nj, int dims,
                      unsigned long long *out) {
  __shared__ double red[256];
  const T *q = static_cast<const T *>(blk->q[0]);
  const T *met = static_cast<const T *>(blk->met);
  const long long qc = blk->qc, mc = blk->mc;
  const double g = blk->gamma;
  double best = 0.0;
  for (long long idx = blockIdx.x * (long long)blockDim.x + threadIdx.x; idx < ncells;
       idx += (long long)gridDim.x * blockDim.x) {
    const int i = (int)(idx % ni);
    const long long r = idx / ni;
    const int j = (int)(r % nj);
    const int k = (int)(r / nj);
    // lines of the xi direction run along i; their transverse strides are those of j and k
    const long long mo = blk->moff + i + j * blk->dir[0].mT1 + (dims == 3 ? k * blk->dir[0].mT2 : 0);
    const double rho = (double)q[idx];
    const double u = (double)q[qc + idx] / rho, v = (double)q[2 * qc + idx] / rho,
                 w = (double)q[3 * qc + idx] / rho;
    const double p = (g - 1.0) * ((double)q[4 * qc + idx] - 0.5 * rho * (u * u + v * v + w * w));
    const double c = sqrt(g * p / rho);
    const double Jc = 1.0 / (double)met[9 * mc + mo];
    double s = 0.0;
    for (int d = 0; d < dims; ++d) {
      const double gx = Jc * (double)met[(3 * d) * mc + mo];
      const double gy = Jc * (double)met[(3 * d + 1) * mc + mo];
      const double gz = Jc * (double)met[(3 * d + 2) * mc + mo];
      s += fabs(u * gx + v * gy + w * gz) + c * sqrt(gx * gx + gy * gy + gz * gz);
    }
    best = s > best ? s : best;
  }
  red[threadIdx.x] = best;
  __syncthreads();
  for (int h = blockDim.x / 2; h > 0; h >>= 1) {
    if (threadIdx.x < h) red[threadIdx.x] = fmax(red[threadIdx.x], red[threadIdx.x + h]);
    __syncthreads();
  }
  if (threadIdx.x == 0) atomicMax(out, (unsigned long long)__double_as_longlong(red[0]));
}

}  // namespace

cudaError_t launch_cfl(const BlockDev *blk, int is_f32, long long ncells, const int *n, int dims,
                       unsigned long long *out_bits, cudaStream_t s) {
  long long g = (ncells + 255) / 256;
  if (g > 152 * 16) g = 152 * 16;
  if (g < 1) g = 1;
  if (is_f32)
    k_cfl<float><<<(int)g, 256, 0, s>>>(blk, ncells, n[0], n[1], dims, out_bits);
  else
    k_cfl<double><<<(int)g, 256, 0, s>>>(blk, ncells, n[0], n[1], dims, out_bits);
  return cudaGetLastError();
}

}  // namespace fpk
