// cfl.cu - time-step bound: max over points of sum_d (|u . grad d| + c |grad d|),
// grad d = J (d_x, d_y, d_z)/J, reduced to one value per launch; the global Lax-Friedrichs
// speeds; and the packing of the cells a neighbouring process needs as its halo.
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
    const double Jc = 1.0 / (double)*FPK_IN(met + (9 * mc + mo), met, 10 * mc, blk->status);
    double s = 0.0;
    for (int d = 0; d < dims; ++d) {
      const double gx = Jc * (double)*FPK_IN(met + ((3 * d) * mc + mo), met, 10 * mc, blk->status);
      const double gy = Jc * (double)*FPK_IN(met + ((3 * d + 1) * mc + mo), met, 10 * mc, blk->status);
      const double gz = Jc * (double)*FPK_IN(met + ((3 * d + 2) * mc + mo), met, 10 * mc, blk->status);
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

template <typename T>
__global__ void k_lam_zero(const BlockDev *blocks, int nblocks) {
  const int b = blockIdx.x * blockDim.x + threadIdx.x;
  if (b < nblocks) {
    T *l = static_cast<T *>(blocks[b].lamg);
    for (int t = 0; t < 9; ++t) l[t] = T(0);
  }
}

__device__ __forceinline__ void atomic_max_nonneg(float *a, float v) {
  atomicMax(reinterpret_cast<unsigned int *>(a), __float_as_uint(v));
}
__device__ __forceinline__ void atomic_max_nonneg(double *a, double v) {
  atomicMax(reinterpret_cast<unsigned long long *>(a), (unsigned long long)__double_as_longlong(v));
}

// per item: max over its points of |U - c|grad d||, |U|, |U + c|grad d|| for every direction
template <typename T>
__global__ void k_lam_max(const BlockDev *blocks, const int2 *items, int nitems, int charwise, int stage) {
  __shared__ T red[9][256];
  for (int it = blockIdx.x; it < nitems; it += gridDim.x) {
    const int2 item = items[it];
    const BlockDev *B = blocks + item.x;
    const int dims = B->dims, ni = B->dir[0].nd, nj = B->dir[1].nd;
    const long long qc = B->qc, mc = B->mc;
    const T *q = static_cast<const T *>(B->q[stage]);
    const T *met = static_cast<const T *>(B->met);
    const T g = T(B->gamma);
    T best[9];
    for (int t = 0; t < 9; ++t) best[t] = T(0);
    const long long end = min((long long)item.y + kLamChunk, qc);
    for (long long idx = (long long)item.y + threadIdx.x; idx < end; idx += blockDim.x) {
      const int i = (int)(idx % ni);
      const long long r = idx / ni;
      const int j = (int)(r % nj);
      const int k = (int)(r / nj);
      const long long mo = B->moff + i + j * B->dir[0].mT1 + (dims == 3 ? k * B->dir[0].mT2 : 0);
      const T rho = q[idx], rinv = T(1) / rho;
      const T u = q[qc + idx] * rinv, v = q[2 * qc + idx] * rinv, w = q[3 * qc + idx] * rinv;
      const T p = (g - T(1)) * (q[4 * qc + idx] - T(0.5) * rho * (u * u + v * v + w * w));
      const T c = sqrt(g * p * rinv);
      const T Jc = T(1) / *FPK_IN(met + (9 * mc + mo), met, 10 * mc, B->status);
      for (int d = 0; d < dims; ++d) {
        const T gx = Jc * *FPK_IN(met + ((3 * d) * mc + mo), met, 10 * mc, B->status),
                gy = Jc * *FPK_IN(met + ((3 * d + 1) * mc + mo), met, 10 * mc, B->status),
                gz = Jc * *FPK_IN(met + ((3 * d + 2) * mc + mo), met, 10 * mc, B->status);
        const T U = u * gx + v * gy + w * gz, a = c * sqrt(gx * gx + gy * gy + gz * gz);
        T lm = fabs(U - a), l0 = fabs(U), lp = fabs(U + a);
        if (!charwise) { lm = fmax(lm, lp); l0 = lm; lp = lm; }
        best[3 * d] = fmax(best[3 * d], lm);
        best[3 * d + 1] = fmax(best[3 * d + 1], l0);
        best[3 * d + 2] = fmax(best[3 * d + 2], lp);
      }
    }
    for (int t = 0; t < 9; ++t) red[t][threadIdx.x] = best[t];
    __syncthreads();
    for (int h = blockDim.x / 2; h > 0; h >>= 1) {
      if (threadIdx.x < h)
        for (int t = 0; t < 9; ++t) red[t][threadIdx.x] = fmax(red[t][threadIdx.x], red[t][threadIdx.x + h]);
      __syncthreads();
    }
    if (threadIdx.x < 3 * dims) atomic_max_nonneg(static_cast<T *>(B->lamg) + threadIdx.x, red[threadIdx.x][0]);
    __syncthreads();
  }
}

// The G cells next to one side of a block, in the halo layout the receiving block reads:
// the state layout [5][nk][nj][ni] with the extent of direction `dir` replaced by G.  Low
// side: cells 0..G-1; high side: cells n-G..n-1 (index x - (n - G) in the buffer).
template <typename T>
__global__ void k_pack_halo(const T *__restrict__ q, T *__restrict__ out, int dir, int side, int G, int ni,
                            int nj, int nk, int *status) {
  int e[3] = {ni, nj, nk};
  const int nd = e[dir];
  e[dir] = G;
  const long long hc = (long long)e[0] * e[1] * e[2], qc = (long long)ni * nj * nk;
  for (long long idx = blockIdx.x * (long long)blockDim.x + threadIdx.x; idx < 5 * hc;
       idx += (long long)gridDim.x * blockDim.x) {
    const int v = (int)(idx / hc);
    long long r = idx - v * hc;
    int c[3];
    c[0] = (int)(r % e[0]);
    r /= e[0];
    c[1] = (int)(r % e[1]);
    c[2] = (int)(r / e[1]);
    c[dir] += side ? nd - G : 0;
    out[idx] = *FPK_IN(q + (v * qc + ((long long)c[2] * nj + c[1]) * ni + c[0]), q, 5 * qc, status);
  }
}

}  // namespace

cudaError_t launch_pack_halo(const void *q, int is_f32, int dir, int side, int G, const int *n, void *out,
                             int *status, cudaStream_t s) {
  int e[3] = {n[0], n[1], n[2]};
  e[dir] = G;
  const long long total = 5LL * e[0] * e[1] * e[2];
  const int threads = 256;
  const long long want = (total + threads - 1) / threads;
  const int grid = (int)(want < 4096 ? (want < 1 ? 1 : want) : 4096);
  if (is_f32)
    k_pack_halo<float><<<grid, threads, 0, s>>>(static_cast<const float *>(q), static_cast<float *>(out), dir, side, G,
                                                n[0], n[1], n[2], status);
  else
    k_pack_halo<double><<<grid, threads, 0, s>>>(static_cast<const double *>(q), static_cast<double *>(out), dir, side,
                                                 G, n[0], n[1], n[2], status);
  return cudaGetLastError();
}

cudaError_t launch_lambda(const BlockDev *blocks, int nblocks, const int2 *items, int nitems, int is_f32,
                          int charwise, int stage, cudaStream_t s) {
  const int zb = (nblocks + 127) / 128;
  int grid = nitems < 152 * 8 ? nitems : 152 * 8;
  if (grid < 1) grid = 1;
  if (is_f32) {
    k_lam_zero<float><<<zb, 128, 0, s>>>(blocks, nblocks);
    k_lam_max<float><<<grid, 256, 0, s>>>(blocks, items, nitems, charwise, stage);
  } else {
    k_lam_zero<double><<<zb, 128, 0, s>>>(blocks, nblocks);
    k_lam_max<double><<<grid, 256, 0, s>>>(blocks, items, nitems, charwise, stage);
  }
  return cudaGetLastError();
}

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
