// metrics.cu - FP64 construction of the symmetric conservative metrics (Eq. JBabc),
// the Jacobian (Eq. JB) and the face metrics (Eq. xidJ at order M) from node
// coordinates, on the GPU (arXiv 2101.05886, Secs. 2.1 and 3).
//
// Every derivative is the order-M central operator of Eq. (metric_discret),
// D f_p = I(f)_{p+1/2} - I(f)_{p-1/2}, applied in three passes over nested index
// boxes so that each point a sweep stencil can reach has metrics built by the
// same operator (the discrete surface conservation law then holds there):
//   B1 = [-(G+M), n+G+M)   first derivatives of the node coordinates
//   B2 = [-(G+M/2), n+G+M/2) metrics, from D of products of B1 values
//   B3 = [-G, n+G)          Jacobian, from D of x . metrics on B2
// The metric (d, a) uses the cyclic form of Eq. JBabc:
//   (d_a / J) = 1/2 [ D_f(b_e c - b c_e) + D_e(b c_f - b_f c) ]
// with (e, f) the directions and (b, c) the coordinates that follow d and a
// cyclically.  In 2-D the metrics are the four node derivatives and the
// Jacobian carries the factor 1/2.  The discrete SCMM is unchanged by a
// translation of the coordinates (the derivative operators commute), so each
// value is formed from coordinates and derivative stencils measured from the
// point itself: the sums then carry the rounding of the metric's own size and
// the discrete SCL residual stays at the metric round-off at any grid size.
// Finally k_{i+1/2} - k_{i-1/2} is formed per point and direction in FP64.
#include <cuda_runtime.h>

#include "fp_internal.h"

namespace fpk {

namespace {

struct Box {
  int lo[3], hi[3];
  long long s1, s2;   // strides of j and k (i stride is 1)
  __host__ __device__ long long size() const {
    return (long long)(hi[0] - lo[0]) * (hi[1] - lo[1]) * (hi[2] - lo[2]);
  }
  __host__ __device__ long long at(int i, int j, int k) const {
    return (long long)(i - lo[0]) + (long long)(j - lo[1]) * s1 + (long long)(k - lo[2]) * s2;
  }
};

Box make_box(int dims, const int n[3], int g) {
  Box b;
  for (int d = 0; d < 3; ++d) {
    bool on = d < dims;
    b.lo[d] = on ? -g : 0;
    b.hi[d] = on ? n[d] + g : 1;
  }
  b.s1 = b.hi[0] - b.lo[0];
  b.s2 = b.s1 * (b.hi[1] - b.lo[1]);
  return b;
}

struct Coef {
  double dc[9];   // derivative weights, t = -M/2 .. M/2 at dc[t + M/2]
  double w[8];    // midpoint weights, m = 0 .. M-1
  int M;
};

Coef make_coef(int M) {
  static const double W2[2] = {1, 1}, W4[4] = {-1, 7, 7, -1}, W6[6] = {1, -8, 37, 37, -8, 1},
                      W8[8] = {-3, 29, -139, 533, 533, -139, 29, -3};
  const double *W = M == 2 ? W2 : M == 4 ? W4 : M == 6 ? W6 : W8;
  const double den = M == 2 ? 2.0 : M == 4 ? 12.0 : M == 6 ? 60.0 : 840.0;
  Coef c;
  c.M = M;
  for (int m = 0; m < 8; ++m) c.w[m] = m < M ? W[m] / den : 0.0;
  const int h = M / 2;
  for (int t = -h; t <= h; ++t) {
    int jp = t + h - 1, jm = t + h;
    double wp = (jp >= 0 && jp < M) ? W[jp] : 0.0;
    double wm = (jm >= 0 && jm < M) ? W[jm] : 0.0;
    c.dc[t + h] = (wp - wm) / den;
  }
  for (int t = M + 1; t < 9; ++t) c.dc[t] = 0.0;
  return c;
}

__device__ __forceinline__ void unflat(long long idx, const Box &b, int p[3]) {
  long long nx = b.hi[0] - b.lo[0], ny = b.hi[1] - b.lo[1];
  p[0] = (int)(idx % nx) + b.lo[0];
  long long r = idx / nx;
  p[1] = (int)(r % ny) + b.lo[1];
  p[2] = (int)(r / ny) + b.lo[2];
}

// D along e of array A (on box Ab) at point p; the value at p is subtracted from
// the stencil first (the weights sum to zero), so the sum carries the rounding of
// the differences, not of the values.
__device__ __forceinline__ double dpt(const double *A, const Box &Ab, const Coef &C, int e, const int p[3]) {
  const int h = C.M / 2;
  const long long st = e == 0 ? 1 : (e == 1 ? Ab.s1 : Ab.s2);
  const long long o = Ab.at(p[0], p[1], p[2]);
  const double a0 = A[o];
  double s = 0.0;
  for (int t = -h; t <= h; ++t) s += C.dc[t + h] * (A[o + t * st] - a0);
  return s;
}

// pass 1: first derivatives d1[b*3+e] = D_e(x_b) on B1 (2-D: b,e < 2)
__global__ void k_first_derivs(const double *nodes, Box nb, Box b1, Coef C, int dims, double *d1) {
  long long n1 = b1.size();
  for (long long idx = blockIdx.x * (long long)blockDim.x + threadIdx.x; idx < n1;
       idx += (long long)gridDim.x * blockDim.x) {
    int p[3];
    unflat(idx, b1, p);
    for (int b = 0; b < dims; ++b)
      for (int e = 0; e < dims; ++e)
        d1[(b * 3 + e) * n1 + idx] = dpt(nodes + b * nb.size(), nb, C, e, p);
  }
}

// pass 2: metrics on B2 (9 arrays, layout [9][B2])
__global__ void k_metrics(const double *nodes, Box nb, const double *d1, Box b1, Box b2, Coef C,
                          int dims, double *m9) {
  long long n2 = b2.size(), n1 = b1.size(), nn = nb.size();
  const int h = C.M / 2;
  for (long long idx = blockIdx.x * (long long)blockDim.x + threadIdx.x; idx < n2;
       idx += (long long)gridDim.x * blockDim.x) {
    int p[3];
    unflat(idx, b2, p);
    if (dims == 2) {
      const long long o1 = b1.at(p[0], p[1], p[2]);
      m9[0 * n2 + idx] = d1[(1 * 3 + 1) * n1 + o1];    // xi_x/J  =  y_eta
      m9[1 * n2 + idx] = -d1[(0 * 3 + 1) * n1 + o1];   // xi_y/J  = -x_eta
      m9[2 * n2 + idx] = 0.0;
      m9[3 * n2 + idx] = -d1[(1 * 3 + 0) * n1 + o1];   // eta_x/J = -y_xi
      m9[4 * n2 + idx] = d1[(0 * 3 + 0) * n1 + o1];    // eta_y/J =  x_xi
      for (int t = 5; t < 9; ++t) m9[t * n2 + idx] = 0.0;
      continue;
    }
    for (int d = 0; d < 3; ++d) {
      const int e = (d + 1) % 3, f = (d + 2) % 3;
      const long long se = e == 0 ? 1 : (e == 1 ? b1.s1 : b1.s2);
      const long long sf = f == 0 ? 1 : (f == 1 ? b1.s1 : b1.s2);
      const long long sne = e == 0 ? 1 : (e == 1 ? nb.s1 : nb.s2);
      const long long snf = f == 0 ? 1 : (f == 1 ? nb.s1 : nb.s2);
      for (int a = 0; a < 3; ++a) {
        const int b = (a + 1) % 3, c = (a + 2) % 3;
        const double *xb = nodes + b * nn, *xc = nodes + c * nn;
        const double *be = d1 + (b * 3 + e) * n1, *ce = d1 + (c * 3 + e) * n1;
        const double *bf = d1 + (b * 3 + f) * n1, *cf = d1 + (c * 3 + f) * n1;
        const long long o1 = b1.at(p[0], p[1], p[2]);
        const long long on = nb.at(p[0], p[1], p[2]);
        // coordinates measured from the node at p (the SCMM is translation invariant)
        const double b0 = xb[on], c0 = xc[on];
        double sF = 0.0, sE = 0.0;
        for (int t = -h; t <= h; ++t) {
          // D_f of (b_e c - b c_e)
          long long r1 = o1 + t * sf, rn = on + t * snf;
          sF += C.dc[t + h] * (be[r1] * (xc[rn] - c0) - (xb[rn] - b0) * ce[r1]);
          // D_e of (b c_f - b_f c)
          r1 = o1 + t * se;
          rn = on + t * sne;
          sE += C.dc[t + h] * ((xb[rn] - b0) * cf[r1] - bf[r1] * (xc[rn] - c0));
        }
        m9[(3 * d + a) * n2 + idx] = 0.5 * (sF + sE);
      }
    }
  }
}

// pass 3: 1/J on B3 into met[9], and the 9 metrics cropped to B3 into met[0..8]
__global__ void k_jacobian(const double *nodes, Box nb, const double *m9, Box b2, Box b3, Coef C,
                           int dims, double *met) {
  long long n3 = b3.size(), n2 = b2.size(), nn = nb.size();
  const int h = C.M / 2;
  for (long long idx = blockIdx.x * (long long)blockDim.x + threadIdx.x; idx < n3;
       idx += (long long)gridDim.x * blockDim.x) {
    int p[3];
    unflat(idx, b3, p);
    const long long o2 = b2.at(p[0], p[1], p[2]);
    const long long on = nb.at(p[0], p[1], p[2]);
    double s = 0.0;
    for (int d = 0; d < dims; ++d) {
      const long long s2d = d == 0 ? 1 : (d == 1 ? b2.s1 : b2.s2);
      const long long snd = d == 0 ? 1 : (d == 1 ? nb.s1 : nb.s2);
      double acc = 0.0;
      for (int t = -h; t <= h; ++t) {
        double prod = 0.0;
        for (int a = 0; a < dims; ++a)
          prod += (nodes[a * nn + on + t * snd] - nodes[a * nn + on]) * m9[(3 * d + a) * n2 + o2 + t * s2d];
        acc += C.dc[t + h] * prod;
      }
      s += acc;
    }
    met[9 * n3 + idx] = s / (double)dims;
    for (int q = 0; q < 9; ++q) met[q * n3 + idx] = m9[q * n2 + o2];
  }
}

// face metrics of direction d: faces f+1/2, f = -1 .. n_d-1, interior transverse points
__global__ void k_face_metrics(const double *met, Box b3, Coef C, int d, int n0, int n1, int n2,
                               double *fm) {
  int nf[3] = {n0, n1, n2};
  nf[d] += 1;
  const long long nfaces = (long long)nf[0] * nf[1] * nf[2];
  const long long n3 = b3.size();
  const int M = C.M;
  const long long sd = d == 0 ? 1 : (d == 1 ? b3.s1 : b3.s2);
  for (long long idx = blockIdx.x * (long long)blockDim.x + threadIdx.x; idx < nfaces;
       idx += (long long)gridDim.x * blockDim.x) {
    int p[3];
    p[0] = (int)(idx % nf[0]);
    long long r = idx / nf[0];
    p[1] = (int)(r % nf[1]);
    p[2] = (int)(r / nf[1]);
    p[d] -= 1;                                   // face p_d + 1/2, p_d = -1 .. n_d - 1
    const long long o = b3.at(p[0], p[1], p[2]);
    for (int a = 0; a < 3; ++a) {
      double s = 0.0;
      for (int m = 0; m < M; ++m) s += C.w[m] * met[(3 * d + a) * n3 + o + (m - M / 2 + 1) * sd];
      fm[a * nfaces + idx] = s;
    }
  }
}

// metric difference across a cell along d: dk[a] = k_{i+1/2} - k_{i-1/2} (interior points,
// state layout [3][nk][nj][ni])
__global__ void k_face_diff(const double *fm, int d, int n0, int n1, int n2, double *dk) {
  const long long ncell = (long long)n0 * n1 * n2;
  int nf[3] = {n0, n1, n2};
  nf[d] += 1;
  const long long nfaces = (long long)nf[0] * nf[1] * nf[2];
  const long long sd = d == 0 ? 1 : (d == 1 ? nf[0] : (long long)nf[0] * nf[1]);
  for (long long idx = blockIdx.x * (long long)blockDim.x + threadIdx.x; idx < ncell;
       idx += (long long)gridDim.x * blockDim.x) {
    int p[3];
    p[0] = (int)(idx % n0);
    long long r = idx / n0;
    p[1] = (int)(r % n1);
    p[2] = (int)(r / n1);
    // face p_d + 1/2 sits at index p_d + 1 along d, face p_d - 1/2 at p_d
    const long long fo = (long long)p[0] + (long long)nf[0] * (p[1] + (long long)nf[1] * p[2]);
    for (int a = 0; a < 3; ++a) dk[a * ncell + idx] = fm[a * nfaces + fo + sd] - fm[a * nfaces + fo];
  }
}

__global__ void k_f64_to_f32(const double *src, float *dst, long long n) {
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n;
       i += (long long)gridDim.x * blockDim.x)
    dst[i] = (float)src[i];
}

int grid_for(long long n) {
  long long g = (n + 255) / 256;
  if (g > 152LL * 64) g = 152LL * 64;
  return g < 1 ? 1 : (int)g;
}

}  // namespace

cudaError_t build_metrics(const MetricJob &J, cudaStream_t s) {
  const int M = J.M, h = M / 2, G = J.G;
  Box nb = make_box(J.dims, J.n, J.Gn);
  Box b1 = make_box(J.dims, J.n, G + M);
  Box b2 = make_box(J.dims, J.n, G + h);
  Box b3 = make_box(J.dims, J.n, G);
  Coef C = make_coef(M);
  double *d1 = J.scratch;
  double *m9 = J.scratch + 9 * b1.size();
  k_first_derivs<<<grid_for(b1.size()), 256, 0, s>>>(J.nodes, nb, b1, C, J.dims, d1);
  k_metrics<<<grid_for(b2.size()), 256, 0, s>>>(J.nodes, nb, d1, b1, b2, C, J.dims, m9);
  k_jacobian<<<grid_for(b3.size()), 256, 0, s>>>(J.nodes, nb, m9, b2, b3, C, J.dims, J.met);
  for (int d = 0; d < J.dims; ++d) {
    long long nf = (long long)J.n[0] * J.n[1] * J.n[2] / J.n[d] * (J.n[d] + 1);
    k_face_metrics<<<grid_for(nf), 256, 0, s>>>(J.met, b3, C, d, J.n[0], J.n[1], J.n[2], J.fmet[d]);
    const long long nc = (long long)J.n[0] * J.n[1] * J.n[2];
    k_face_diff<<<grid_for(nc), 256, 0, s>>>(J.fmet[d], d, J.n[0], J.n[1], J.n[2], J.dk[d]);
  }
  return cudaGetLastError();
}

cudaError_t convert_f64_to_f32(const double *src, float *dst, long long n, cudaStream_t s) {
  k_f64_to_f32<<<grid_for(n), 256, 0, s>>>(src, dst, n);
  return cudaGetLastError();
}

}  // namespace fpk
