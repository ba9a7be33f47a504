// sweep.cuh - the directional residual sweep of the free-stream-preserving (FP)
// upwind finite-difference scheme (arXiv 2101.05886, Sec. 3.2), templated on the
// arithmetic type.
//
// One CTA owns a tile of TT lines along the swept direction and marches along
// them in chunks of S faces (S * TT = 256 threads, one face per thread).  Cells
// enter a shared-memory ring (2S slots per line) once and are reused by every
// face whose stencil covers them; per-cell primitives and spectral radii are
// formed once per cell.  Face fluxes go to a second ring, and each cell's
// residual contribution F'_{i+1/2} - F'_{i-1/2} (Eq. aderivative) is applied in
// the epilogue: written, accumulated, scaled into dQ/dt, or fused into the
// Runge-Kutta stage update.  Work items (block, line tile) are taken by a
// persistent grid, so one launch covers every block of a batch.
//
// Face flux in difference form (Eq. my_point1 with the split of Eq.
// flux_split_detail): with Q* = Q~_{i+1/2}/(1/J)_{i+1/2} (Eq. Q_star, order-M
// interpolation, Remark 3) written as Q* = Q_i + delta,
//   dF_m = (F(Q_m) - F(Q*)) . k_m,  dQ_m = (Q_m - Q*) (1/J)_m      m = i-2..i+3
// are formed directly from the state differences (never as a difference of two
// large fluxes), projected on the Roe left eigenvectors, split with local
// Lax-Friedrichs speeds and reconstructed by WENO5-JS or linear upwind into W.
// The reference face fluxes F~*_{i+-1/2} = F(Q*_{i+-1/2}) . k_{i+-1/2} enter the
// residual of point i through the exact identity
//   F~*_+ - F~*_- = [F(Q*_+) - F(Q*_-)] . k_+ + [F(Q*_-) - F(Qbar)] . (k_+ - k_-)
//                   + F(Qbar) . (k_+ - k_-),
// with Qbar the far-field state and k_+ - k_- formed in FP64 when the metrics
// are built.  Summed over the directions the last term is F(Qbar) times the
// discrete surface-conservation residual (Eq. SCL), zero to round-off for the
// symmetric conservative metrics, and is not formed.  Every remaining term is a
// product with a difference, so FP32 arithmetic keeps its relative accuracy on
// the residual, and a uniform free stream gives exactly zero in either precision.
#pragma once

#include <cuda_runtime.h>
#include <math.h>

#include "fp_internal.h"

namespace fpk {

template <typename T> struct Num;
template <> struct Num<double> {
  // reciprocal of a finite nonzero x: the PTX approximation (relative error about 2^-20)
  // refined by two Newton-Raphson steps y <- y + y (1 - x y), which square the error twice
  static __device__ __forceinline__ double rcp(double x) {
    double y;
    asm("rcp.approx.ftz.f64 %0, %1;" : "=d"(y) : "d"(x));
    y = fma(y, fma(-x, y, 1.0), y);
    return fma(y, fma(-x, y, 1.0), y);
  }
  static __device__ __forceinline__ double div(double a, double b) { return a / b; }
  static __device__ __forceinline__ double sqrt_(double x) { return sqrt(x); }
  static __device__ __forceinline__ double rsqrt_(double x) { return rsqrt(x); }
  static __device__ __forceinline__ double ld(const void *p, long long i) {
    return __ldg(static_cast<const double *>(p) + i);
  }
};
template <> struct Num<float> {
  // the PTX approximate reciprocal (one MUFU operation, max relative error 2^-23);
  // subnormal inputs are flushed, so 1/x of a value below 2^-126 is +-inf
  static __device__ __forceinline__ float rcp(float x) {
    float r;
    asm("rcp.approx.ftz.f32 %0, %1;" : "=f"(r) : "f"(x));
    return r;
  }
  static __device__ __forceinline__ float div(float a, float b) { return a * rcp(b); }
  static __device__ __forceinline__ float sqrt_(float x) {
    float r;
    asm("sqrt.approx.f32 %0, %1;" : "=f"(r) : "f"(x));
    return r;
  }
  static __device__ __forceinline__ float rsqrt_(float x) { return rsqrtf(x); }
  static __device__ __forceinline__ float ld(const void *p, long long i) {
    return __ldg(static_cast<const float *>(p) + i);
  }
};

// Pairs of values processed by one instruction: packed FP32x2 arithmetic (sm_100+
// FFMA2 / FADD2 / FMUL2) for float, two scalar operations for double.
struct dpair { double x, y; };
template <typename T> struct PairOf;
template <> struct PairOf<float> { using type = float2; };
template <> struct PairOf<double> { using type = dpair; };

__device__ __forceinline__ float2 pmk(float a, float b) { return make_float2(a, b); }
__device__ __forceinline__ dpair pmk(double a, double b) { return dpair{a, b}; }
__device__ __forceinline__ float2 pfma(float2 a, float2 b, float2 c) { return __ffma2_rn(a, b, c); }
__device__ __forceinline__ dpair pfma(dpair a, dpair b, dpair c) { return dpair{fma(a.x, b.x, c.x), fma(a.y, b.y, c.y)}; }
__device__ __forceinline__ float2 padd(float2 a, float2 b) { return __fadd2_rn(a, b); }
__device__ __forceinline__ dpair padd(dpair a, dpair b) { return dpair{a.x + b.x, a.y + b.y}; }
__device__ __forceinline__ float2 pmul(float2 a, float2 b) { return __fmul2_rn(a, b); }
__device__ __forceinline__ dpair pmul(dpair a, dpair b) { return dpair{a.x * b.x, a.y * b.y}; }
template <typename P> __device__ __forceinline__ P psub(P a, P b) { return pfma(b, pmk(decltype(a.x)(-1), decltype(a.x)(-1)), a); }
template <typename P> __device__ __forceinline__ P pc(decltype(P::x) v) { return pmk(v, v); }

// Fifth-order reconstruction of a pair of five-point stencils (the + side and the
// mirrored - side of one characteristic field) in first-difference form; returns
// the two reconstructed values.
template <typename T, int SCHEME>
__device__ __forceinline__ typename PairOf<T>::type recon5_pair(
    typename PairOf<T>::type v0, typename PairOf<T>::type v1, typename PairOf<T>::type v2,
    typename PairOf<T>::type v3, typename PairOf<T>::type v4) {
  using P = typename PairOf<T>::type;
  const P a = psub(v1, v0), b = psub(v2, v1), c = psub(v3, v2), d = psub(v4, v3);
  const P r0 = pfma(pc<P>(T(5)), b, pmul(pc<P>(T(-2)), a));      // 6 (q0 - v2)
  const P r1 = pfma(pc<P>(T(2)), c, b);                          // 6 (q1 - v2)
  const P r2 = pfma(pc<P>(T(4)), c, pmul(pc<P>(T(-1)), d));      // 6 (q2 - v2)
  if (SCHEME == 1) {
    const P s = pfma(pc<P>(T(0.3)), r2, pfma(pc<P>(T(0.6)), r1, pmul(pc<P>(T(0.1)), r0)));
    return pfma(pc<P>(T(1.0 / 6.0)), s, v2);
  }
  const P d0 = psub(b, a), e0 = pfma(pc<P>(T(3)), b, pmul(pc<P>(T(-1)), a));
  const P d1 = psub(c, b), e1 = padd(b, c);
  const P d2 = psub(d, c), e2 = pfma(pc<P>(T(-3)), c, d);
  const P c13 = pc<P>(T(13.0 / 12.0)), q4 = pc<P>(T(0.25)), eps = pc<P>(T(1.0e-6));
  const P b0 = pfma(c13, pmul(d0, d0), pfma(q4, pmul(e0, e0), eps));
  const P b1 = pfma(c13, pmul(d1, d1), pfma(q4, pmul(e1, e1), eps));
  const P b2 = pfma(c13, pmul(d2, d2), pfma(q4, pmul(e2, e2), eps));
  const P s0 = pmul(b0, b0), s1 = pmul(b1, b1), s2 = pmul(b2, b2);
  const P a0 = pmul(pc<P>(T(0.1)), pmk(Num<T>::rcp(s0.x), Num<T>::rcp(s0.y)));
  const P a1 = pmul(pc<P>(T(0.6)), pmk(Num<T>::rcp(s1.x), Num<T>::rcp(s1.y)));
  const P a2 = pmul(pc<P>(T(0.3)), pmk(Num<T>::rcp(s2.x), Num<T>::rcp(s2.y)));
  const P num = pfma(a2, r2, pfma(a1, r1, pmul(a0, r0)));
  const P den = pmul(pc<P>(T(6)), padd(padd(a0, a1), a2));
  return pfma(num, pmk(Num<T>::rcp(den.x), Num<T>::rcp(den.y)), v2);
}

// WENOCU6 (the sixth-order adaptive central-upwind WENO that Remark 2 names) for a pair
// of six-point stencils i-2..i+3, in the first differences a..e of the six values: the
// three upwind parabolic sub-stencils of WENO5 and the downwind {i+1, i+2, i+3}, linear
// weights (1, 9, 9, 1)/20 (the M6 central face value), the downwind stencil judged by the
// six-point indicator beta6 (integral definition; 120960 beta6 below), reference
// tau6 = |beta6 - (beta0 + 4 beta1 + beta2)/6|, alpha_k = d_k (20 + tau6/(beta_k + 1e-40))^2.
// The ratio is capped at 1e18 so that alpha stays finite in FP32; a cap that only binds
// where a sub-stencil is flat to 1e-18 of tau6.
template <typename T>
__device__ __forceinline__ T cu6_ratio(T tau, T beta) {
  if (!(tau > T(0))) return T(0);
  const T r = tau * Num<T>::rcp(beta + T(1.0e-40));   // +inf when the sum is below FP32 range
  return r < T(1.0e18) ? r : T(1.0e18);
}
template <typename T>
__device__ __forceinline__ typename PairOf<T>::type recon6cu_pair(const typename PairOf<T>::type v[6]) {
  using P = typename PairOf<T>::type;
  const P a = psub(v[1], v[0]), b = psub(v[2], v[1]), c = psub(v[3], v[2]);
  const P d = psub(v[4], v[3]), e = psub(v[5], v[4]);
  // 6 (q_k - v2)
  const P r0 = pfma(pc<P>(T(5)), b, pmul(pc<P>(T(-2)), a));
  const P r1 = pfma(pc<P>(T(2)), c, b);
  const P r2 = pfma(pc<P>(T(4)), c, pmul(pc<P>(T(-1)), d));
  const P r3 = pfma(pc<P>(T(2)), e, pfma(pc<P>(T(-5)), d, pmul(pc<P>(T(6)), c)));
  // WENO5 indicators of the three upwind sub-stencils
  const P d0 = psub(b, a), e0 = pfma(pc<P>(T(3)), b, pmul(pc<P>(T(-1)), a));
  const P d1 = psub(c, b), e1 = padd(b, c);
  const P d2 = psub(d, c), e2 = pfma(pc<P>(T(-3)), c, d);
  const P c13 = pc<P>(T(13.0 / 12.0)), q4 = pc<P>(T(0.25));
  const P b0 = pfma(c13, pmul(d0, d0), pmul(q4, pmul(e0, e0)));
  const P b1 = pfma(c13, pmul(d1, d1), pmul(q4, pmul(e1, e1)));
  const P b2 = pfma(c13, pmul(d2, d2), pmul(q4, pmul(e2, e2)));
  // 120960 beta6 as a quadratic form of the differences
  P f = pmul(a, pfma(pc<P>(T(271779)), a, pfma(pc<P>(T(-1837242)), b, pfma(pc<P>(T(2249110)), c,
             pfma(pc<P>(T(-1213142)), d, pmul(pc<P>(T(245620)), e))))));
  f = pfma(b, pfma(pc<P>(T(3544296)), b, pfma(pc<P>(T(-9252940)), c, pfma(pc<P>(T(5189840)), d,
             pmul(pc<P>(T(-1079386)), e)))), f);
  f = pfma(c, pfma(pc<P>(T(6713736)), c, pfma(pc<P>(T(-7947412)), d, pmul(pc<P>(T(1713274)), e))), f);
  f = pfma(d, pfma(pc<P>(T(2534504)), d, pmul(pc<P>(T(-1150710)), e)), f);
  f = pfma(e, pmul(pc<P>(T(139633)), e), f);
  const P b3 = pmul(f, pc<P>(T(1.0 / 120960.0)));
  const P tt = psub(b3, pmul(pc<P>(T(1.0 / 6.0)), pfma(pc<P>(T(4)), b1, padd(b0, b2))));
  const T tx = tt.x < T(0) ? -tt.x : tt.x, ty = tt.y < T(0) ? -tt.y : tt.y;
  const P w0 = padd(pc<P>(T(20)), pmk(cu6_ratio(tx, b0.x), cu6_ratio(ty, b0.y)));
  const P w1 = padd(pc<P>(T(20)), pmk(cu6_ratio(tx, b1.x), cu6_ratio(ty, b1.y)));
  const P w2 = padd(pc<P>(T(20)), pmk(cu6_ratio(tx, b2.x), cu6_ratio(ty, b2.y)));
  const P w3 = padd(pc<P>(T(20)), pmk(cu6_ratio(tx, b3.x), cu6_ratio(ty, b3.y)));
  const P a0 = pmul(pc<P>(T(0.05)), pmul(w0, w0)), a1 = pmul(pc<P>(T(0.45)), pmul(w1, w1));
  const P a2 = pmul(pc<P>(T(0.45)), pmul(w2, w2)), a3 = pmul(pc<P>(T(0.05)), pmul(w3, w3));
  const P num = pfma(a3, r3, pfma(a2, r2, pfma(a1, r1, pmul(a0, r0))));
  const P den = pmul(pc<P>(T(6)), padd(padd(a0, a1), padd(a2, a3)));
  return pfma(num, pmk(Num<T>::rcp(den.x), Num<T>::rcp(den.y)), v[2]);
}

// Seventh-order WENO-JS (four 4-point sub-stencils, optimal weights (1,12,18,4)/35,
// smoothness indicators of the integral definition) for a pair of seven-point stencils,
// written in the first differences d1..d6 of the seven values.
template <typename T>
__device__ __forceinline__ typename PairOf<T>::type recon7_pair(const typename PairOf<T>::type v[7]) {
  using P = typename PairOf<T>::type;
  const P d1 = psub(v[1], v[0]), d2 = psub(v[2], v[1]), d3 = psub(v[3], v[2]);
  const P d4 = psub(v[4], v[3]), d5 = psub(v[5], v[4]), d6 = psub(v[6], v[5]);
  // 12 (q_k - v3)
  const P r0 = pfma(pc<P>(T(13)), d3, pfma(pc<P>(T(-10)), d2, pmul(pc<P>(T(3)), d1)));
  const P r1 = pfma(pc<P>(T(3)), d4, pfma(pc<P>(T(4)), d3, pmul(pc<P>(T(-1)), d2)));
  const P r2 = pfma(pc<P>(T(-1)), d5, pfma(pc<P>(T(6)), d4, d3));
  const P r3 = pfma(pc<P>(T(9)), d4, pfma(pc<P>(T(-4)), d5, d6));
  // 240 beta_k as quadratic forms of the differences
  const P f0 = pfma(d1, pfma(pc<P>(T(547)), d1, pfma(pc<P>(T(-2788)), d2, pmul(pc<P>(T(1854)), d3))),
                    pfma(d2, pfma(pc<P>(T(3708)), d2, pmul(pc<P>(T(-5188)), d3)), pmul(pc<P>(T(2107)), pmul(d3, d3))));
  const P f1 = pfma(d2, pfma(pc<P>(T(267)), d2, pfma(pc<P>(T(-1108)), d3, pmul(pc<P>(T(494)), d4))),
                    pfma(d3, pfma(pc<P>(T(1468)), d3, pmul(pc<P>(T(-1428)), d4)), pmul(pc<P>(T(547)), pmul(d4, d4))));
  const P f2 = pfma(d3, pfma(pc<P>(T(547)), d3, pfma(pc<P>(T(-1428)), d4, pmul(pc<P>(T(494)), d5))),
                    pfma(d4, pfma(pc<P>(T(1468)), d4, pmul(pc<P>(T(-1108)), d5)), pmul(pc<P>(T(267)), pmul(d5, d5))));
  const P f3 = pfma(d4, pfma(pc<P>(T(2107)), d4, pfma(pc<P>(T(-5188)), d5, pmul(pc<P>(T(1854)), d6))),
                    pfma(d5, pfma(pc<P>(T(3708)), d5, pmul(pc<P>(T(-2788)), d6)), pmul(pc<P>(T(547)), pmul(d6, d6))));
  const P i240 = pc<P>(T(1.0 / 240.0)), eps = pc<P>(T(1.0e-6));
  const P b0 = pfma(f0, i240, eps), b1 = pfma(f1, i240, eps), b2 = pfma(f2, i240, eps), b3 = pfma(f3, i240, eps);
  const P s0 = pmul(b0, b0), s1 = pmul(b1, b1), s2 = pmul(b2, b2), s3 = pmul(b3, b3);
  const P a0 = pmul(pc<P>(T(1.0 / 35.0)), pmk(Num<T>::rcp(s0.x), Num<T>::rcp(s0.y)));
  const P a1 = pmul(pc<P>(T(12.0 / 35.0)), pmk(Num<T>::rcp(s1.x), Num<T>::rcp(s1.y)));
  const P a2 = pmul(pc<P>(T(18.0 / 35.0)), pmk(Num<T>::rcp(s2.x), Num<T>::rcp(s2.y)));
  const P a3 = pmul(pc<P>(T(4.0 / 35.0)), pmk(Num<T>::rcp(s3.x), Num<T>::rcp(s3.y)));
  const P num = pfma(a3, r3, pfma(a2, r2, pfma(a1, r1, pmul(a0, r0))));
  const P den = pmul(pc<P>(T(12)), padd(padd(a0, a1), padd(a2, a3)));
  return pfma(num, pmk(Num<T>::rcp(den.x), Num<T>::rcp(den.y)), v[3]);
}

// Slip-wall reflection of a ghost value (the mirror cell's state Q) about the boundary
// face metric fm (component stride fcs): m - 2 (m.k) k/|k|^2.
template <typename T>
__device__ __forceinline__ void wall_reflect(T Q[5], const T *fm, long long fcs) {
  const T n0 = fm[0], n1 = fm[fcs], n2 = fm[2 * fcs];
  const T s = T(2) * (Q[1] * n0 + Q[2] * n1 + Q[3] * n2) / (n0 * n0 + n1 * n1 + n2 * n2);
  Q[1] -= s * n0;
  Q[2] -= s * n1;
  Q[3] -= s * n2;
}

// Asynchronous global -> shared copies of single elements (sm_80+ cp.async).
template <typename T>
__device__ __forceinline__ void cp_async_el(T *smem, const T *gmem) {
  const unsigned sa = (unsigned)__cvta_generic_to_shared(smem);
  if (sizeof(T) == 4)
    asm volatile("cp.async.ca.shared.global [%0], [%1], 4;\n" ::"r"(sa), "l"(gmem));
  else
    asm volatile("cp.async.ca.shared.global [%0], [%1], 8;\n" ::"r"(sa), "l"(gmem));
}
__device__ __forceinline__ void cp_async16(void *smem, const void *gmem) {
  const unsigned sa = (unsigned)__cvta_generic_to_shared(smem);
  asm volatile("cp.async.ca.shared.global [%0], [%1], 16;\n" ::"r"(sa), "l"(gmem));
}
__device__ __forceinline__ void cp_async8(void *smem, const void *gmem) {
  const unsigned sa = (unsigned)__cvta_generic_to_shared(smem);
  asm volatile("cp.async.ca.shared.global [%0], [%1], 8;\n" ::"r"(sa), "l"(gmem));
}
__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;\n" ::); }
__device__ __forceinline__ void cp_async_wait_all() { asm volatile("cp.async.wait_group 0;\n" ::: "memory"); }

// Weights of the order-M midpoint formula (Sec. 3, Eq. metric_discret), stencil
// i-M/2+1 .. i+M/2 for the face i+1/2.
template <int M> struct MidW;
template <> struct MidW<2> { static __device__ __forceinline__ double w(int m) { return 0.5; } };
template <> struct MidW<4> {
  static __device__ __forceinline__ double w(int m) {
    return (m == 0 || m == 3) ? -1.0 / 12.0 : 7.0 / 12.0;
  }
};
template <> struct MidW<6> {
  static __device__ __forceinline__ double w(int m) {
    return (m == 0 || m == 5) ? 1.0 / 60.0 : (m == 1 || m == 4) ? -8.0 / 60.0 : 37.0 / 60.0;
  }
};
template <> struct MidW<8> {
  static __device__ __forceinline__ double w(int m) {
    return (m == 0 || m == 7) ? -3.0 / 840.0
         : (m == 1 || m == 6) ? 29.0 / 840.0
         : (m == 2 || m == 5) ? -139.0 / 840.0 : 533.0 / 840.0;
  }
};

// Fifth-order reconstruction at i+1/2 from v0..v4 = f_{i-2..i+2} (Sec. 2.2.2):
// WENO5-JS with eps = 1e-6 and power 2, or linear upwind (optimal weights).  Written
// in the first differences a..d of the five values: q_k - v2 and the smoothness
// indicators are short combinations of them, and the result is v2 + sum w_k (q_k - v2).
template <typename T, int SCHEME>
__device__ __forceinline__ T recon5(T v0, T v1, T v2, T v3, T v4) {
  const T a = v1 - v0, b = v2 - v1, c = v3 - v2, d = v4 - v3;
  // 6 (q_k - v2): (5b - 2a), (b + 2c), (4c - d)
  const T r0 = T(5) * b - T(2) * a;
  const T r1 = b + T(2) * c;
  const T r2 = T(4) * c - d;
  if (SCHEME == 1) {
    // optimal weights (1/10, 6/10, 3/10) over 6: (2,-13,47,27,-3)/60 relative to v2
    return v2 + (T(0.1) * r0 + T(0.6) * r1 + T(0.3) * r2) * T(1.0 / 6.0);
  }
  const T c13 = T(13.0 / 12.0), eps = T(1.0e-6);
  const T d0 = b - a, e0 = T(3) * b - a;
  const T d1 = c - b, e1 = b + c;
  const T d2 = d - c, e2 = d - T(3) * c;
  const T b0 = c13 * d0 * d0 + T(0.25) * e0 * e0 + eps;
  const T b1 = c13 * d1 * d1 + T(0.25) * e1 * e1 + eps;
  const T b2 = c13 * d2 * d2 + T(0.25) * e2 * e2 + eps;
  const T a0 = Num<T>::div(T(0.1), b0 * b0);
  const T a1 = Num<T>::div(T(0.6), b1 * b1);
  const T a2 = Num<T>::div(T(0.3), b2 * b2);
  return v2 + Num<T>::div(a0 * r0 + a1 * r1 + a2 * r2, T(6) * (a0 + a1 + a2));
}

// [F(B) - F(A)] . k from A's state (velocity uA, momentum mA, energy EA, pressure pA),
// the difference d = B - A, and B's 1/rho and velocity; every term is a product
// with a component of d, so the result carries the relative rounding of d.
template <typename T>
__device__ __forceinline__ void dflux(T g1, T rinvB, const T uB[3], const T uA[3], const T mA[3],
                                      T EA, T pA, const T d[5], const T k[3], T out[5]) {
  T du0 = (d[1] - uA[0] * d[0]) * rinvB;
  T du1 = (d[2] - uA[1] * d[0]) * rinvB;
  T du2 = (d[3] - uA[2] * d[0]) * rinvB;
  T dke = T(0.5) * (d[1] * uB[0] + d[2] * uB[1] + d[3] * uB[2] + mA[0] * du0 + mA[1] * du1 +
                    mA[2] * du2);
  T dp = g1 * (d[4] - dke);
  T UB = uB[0] * k[0] + uB[1] * k[1] + uB[2] * k[2];
  T dU = du0 * k[0] + du1 * k[1] + du2 * k[2];
  out[0] = d[1] * k[0] + d[2] * k[1] + d[3] * k[2];
  out[1] = d[1] * UB + mA[0] * dU + dp * k[0];
  out[2] = d[2] * UB + mA[1] * dU + dp * k[1];
  out[3] = d[3] * UB + mA[2] * dU + dp * k[2];
  out[4] = (d[4] + dp) * UB + (EA + pA) * dU;
}

// dflux for two stencil points at once (same A state, two B states), packed.
template <typename T>
__device__ __forceinline__ void dflux_pair(T g1, typename PairOf<T>::type rinvB,
                                           const typename PairOf<T>::type uB[3], const T uA[3],
                                           const T mA[3], T EA, T pA,
                                           const typename PairOf<T>::type d[5],
                                           const typename PairOf<T>::type k[3],
                                           typename PairOf<T>::type out[5]) {
  using P = typename PairOf<T>::type;
  const P du0 = pmul(pfma(pc<P>(-uA[0]), d[0], d[1]), rinvB);
  const P du1 = pmul(pfma(pc<P>(-uA[1]), d[0], d[2]), rinvB);
  const P du2 = pmul(pfma(pc<P>(-uA[2]), d[0], d[3]), rinvB);
  P dke = pmul(d[1], uB[0]);
  dke = pfma(d[2], uB[1], dke);
  dke = pfma(d[3], uB[2], dke);
  dke = pfma(pc<P>(mA[0]), du0, dke);
  dke = pfma(pc<P>(mA[1]), du1, dke);
  dke = pfma(pc<P>(mA[2]), du2, dke);
  const P dp = pmul(pc<P>(g1), pfma(pc<P>(T(-0.5)), dke, d[4]));
  const P UB = pfma(uB[2], k[2], pfma(uB[1], k[1], pmul(uB[0], k[0])));
  const P dU = pfma(du2, k[2], pfma(du1, k[1], pmul(du0, k[0])));
  out[0] = pfma(d[3], k[2], pfma(d[2], k[1], pmul(d[1], k[0])));
  out[1] = pfma(dp, k[0], pfma(pc<P>(mA[0]), dU, pmul(d[1], UB)));
  out[2] = pfma(dp, k[1], pfma(pc<P>(mA[1]), dU, pmul(d[2], UB)));
  out[3] = pfma(dp, k[2], pfma(pc<P>(mA[2]), dU, pmul(d[3], UB)));
  out[4] = pfma(pc<P>(EA + pA), dU, pmul(padd(d[4], dp), UB));
}

// FIX = 1 or 2: the characteristic decomposition and the FP form on, local Lax-Friedrichs speeds,
// all fixed at compile time (the configuration of the paper's workloads but the shock test), so
// their switches fold away; FIX = 0 reads them from the arguments and the block descriptor.
// FIX = 2 is the same sweep with the alternative CTA shape of sweep_threads (fp_internal.h).
template <typename T, int M, int SCHEME, bool BND, int FIX>
__global__ void __launch_bounds__(sweep_threads(sizeof(T) == 4, SCHEME, FIX), sweep_min_ctas(sizeof(T) == 4, SCHEME, FIX))
fp_sweep(const BlockDev *__restrict__ blocks, const int2 *__restrict__ items, int nitems, int dir,
         int mode, int stage, const double *__restrict__ dtp, int charwise_arg, int fpform_arg) {
  // this variant's CTA shape (fp_internal.h): threads, ring stride of a staged field, padding
  constexpr int kThreads = sweep_threads(sizeof(T) == 4, SCHEME, FIX);
  constexpr int kRing = sweep_ring(sizeof(T) == 4, SCHEME, FIX);
  constexpr bool kPad = sweep_padded(sizeof(T) == 4, SCHEME, FIX);
  const int charwise = FIX ? 1 : charwise_arg;
  const int fpform = FIX ? 1 : fpform_arg;
  // stencil points of a face: i-2..i+3 (5th order) or i-3..i+4 (WENO7), offset index Q0
  constexpr int NS = SCHEME == 2 ? 8 : 6;
  constexpr int Q0 = SCHEME == 2 ? 0 : 1;
  extern __shared__ __align__(16) unsigned char smraw[];
  T *const sm = reinterpret_cast<T *>(smraw);              // cell ring: kCellFields x kRing
  T *const fr = sm + kCellFields * kRing;                   // face ring: kFaceFields x kRing
  T *const nsb = fr + kFaceFields * kRing;                  // next chunk's cell and face metrics, per thread
  T *const epb = nsb + kNextFields * kThreads;              // epilogue operands, per thread
  const int tid = threadIdx.x;
  // Work-item descriptors in shared memory, double-buffered: during an item's first chunk
  // the next item's (block, first line) and its whole block descriptor are copied in with
  // cp.async, so an item starts without a chain of dependent global loads, and the chunk
  // loop reads buffer pointers from here rather than through an L1 that the streamed cells
  // keep evicting.
  static_assert(sizeof(BlockDev) % 16 == 0, "descriptor copied in 16-byte pieces");
  constexpr int kDescPieces = (int)(sizeof(BlockDev) / 16);
  __shared__ __align__(16) unsigned char s_desc[2][sizeof(BlockDev)];
  __shared__ __align__(16) int2 s_item[2];
  __shared__ T s_dt;
  __shared__ T s_lam[3];                // global Lax-Friedrichs speeds of this item's direction
  auto fetch_desc = [&](int buf, int blk) {
    for (int p = tid; p < kDescPieces; p += kThreads)
      cp_async16(s_desc[buf] + 16 * p, reinterpret_cast<const unsigned char *>(blocks + blk) + 16 * p);
  };
  if (blockIdx.x < nitems) {            // the first item's descriptor, loaded before the loop
    if (tid == 0) s_item[0] = items[blockIdx.x];
    __syncthreads();
    fetch_desc(0, s_item[0].x);
    cp_async_commit();
    cp_async_wait_all();
    __syncthreads();
  }

  int cur = 0;
  for (int it = blockIdx.x; it < nitems; it += gridDim.x, cur ^= 1) {
    const int2 item = s_item[cur];
    const BlockDev *B = reinterpret_cast<const BlockDev *>(s_desc[cur]);
    const DirDev *D = &B->dir[dir];
    const int nit = it + gridDim.x;
    // the next item's (block, first line): lands by this item's prologue barrier
    if (tid == 0 && nit < nitems) cp_async8(&s_item[cur ^ 1], items + nit);
    if (tid == 0) {                      // read after the prologue's barrier
      s_dt = mode == MODE_RK ? T(*dtp) : T(0);
      if (!FIX && B->global_lf)
        for (int c = 0; c < 3; ++c)
          s_lam[c] = *FPK_IN(static_cast<const T *>(B->lamg) + (3 * dir + c), static_cast<const T *>(B->lamg), 9, B->status);
    }
    const int S = D->S, TT = D->TT, W = 2 * S;
    // thread roles: along-line index tf and line index tl.  The xi pass puts
    // consecutive threads along the line (coalesced, i contiguous), the other passes
    // across lines.  Shared layout: slot-fast lines are 3S apart (conflict-free for
    // S < 32 as well) or, unpadded, 2S apart (the host then gives the xi pass S = 32),
    // line-fast slots are TT apart.
    const bool slotFast = (dir == 0);
    const int tf = slotFast ? (tid % S) : (tid / TT);
    const int tl = slotFast ? (tid / S) : (tid % TT);
    const int LS = slotFast ? (kPad ? 3 : 2) * S : 1;
    const int SS = slotFast ? 1 : TT;
    const int lbase = tl * LS;
    const int wm = W - 1;
    const int nd = D->nd;
    const long long L = (long long)item.y + tl;
    const bool lineOK = L < D->nlines;
    const int t1 = lineOK ? (int)(L % D->nt1) : 0;
    const int t2 = lineOK ? (int)(L / D->nt1) : 0;
    const long long qbase = t1 * D->qT1 + t2 * D->qT2, qsd = D->qsd;
    const long long mbase = B->moff + t1 * D->mT1 + t2 * D->mT2, msd = D->msd;
    const long long fbase = t1 * D->fT1 + t2 * D->fT2, fsd = D->fsd, fcs = D->fc;
    const long long qc = B->qc, mc = B->mc;
    const int G = B->G, bclo = D->bclo, bchi = D->bchi;
    const T *__restrict__ met = static_cast<const T *>(B->met) + mbase;
    const T *__restrict__ fmet = static_cast<const T *>(D->fmet) + fbase;
    const T *__restrict__ qin = static_cast<const T *>(B->q[stage]);
    const T g1 = T(B->gamma - 1.0), gam = T(B->gamma);
    const int glf = FIX ? 0 : B->global_lf;
    T qb[5];
#pragma unroll
    for (int v = 0; v < 5; ++v) qb[v] = T(B->qbar[v]);
    // far-field reference state primitives
    const T qbr = Num<T>::rcp(qb[0]);
    const T ub[3] = {qb[1] * qbr, qb[2] * qbr, qb[3] * qbr};
    const T pb = g1 * (qb[4] - T(0.5) * (qb[1] * ub[0] + qb[2] * ub[1] + qb[3] * ub[2]));
    const T mbq[3] = {qb[1], qb[2], qb[3]};

    auto off = [&](int x) -> int {
      const int o = lbase + (x & wm) * SS;
      FPK_CHK_ONLY(if (o < 0 || o >= kRing) { atomicOr(B->status, ST_BOUNDS); return 0; })
      return o;
    };
    FPK_CHK_ONLY(const T *const metb = static_cast<const T *>(B->met);
                 const T *const fmetb = static_cast<const T *>(D->fmet);)

    // boundary rule of a cell index x of this line: the source cell (its first component
    // at src, component stride cs), or the far-field state (far); `wall` asks for the
    // momentum to be reflected about the boundary face's normal.  Codes: 0 periodic, 1 far
    // field, 2 zero gradient, 3 slip wall (mirror cell), 4 C-grid cut (mirror cell on the line
    // with t1 reversed, wall outside the cut width), 5 another block of the batch (its cells
    // next to its opposite side, same transverse indices, same RK stage), 6 the caller's halo
    // buffer of that side (the cells another process holds, refreshed for every RK stage).
    auto bc_source = [&](int x, const T *&src, long long &cs, bool &far,
                         bool &wall FPK_CHK_ONLY(, const T *&sb, long long &sn)) {
      int xx = x;
      long long qsrc = qbase;
      cs = qc; far = false; wall = false;
      FPK_CHK_ONLY(sb = qin; sn = 5 * qc;)
      if (x < 0 || x >= nd) {
        const int bc = x < 0 ? bclo : bchi;
        if (bc == 0) { xx = x % nd; if (xx < 0) xx += nd; }
        else if (bc == 1) far = true;
        else if (bc == 2 || !BND) xx = x < 0 ? 0 : nd - 1;
        else if (bc == 6) {   // halo buffer: index x + G below the line, x - nd above it
          const long long hx = x < 0 ? (long long)(x + G) : (long long)(x - nd);
          src = static_cast<const T *>(D->halo[x < 0 ? 0 : 1]) + t1 * D->hT1 + t2 * D->hT2 + hx * D->hsd;
          cs = D->hc;
          FPK_CHK_ONLY(sb = static_cast<const T *>(D->halo[x < 0 ? 0 : 1]); sn = 5 * D->hc;)
          return;
        } else if (bc == 5) {   // rare path: the line's (t1, t2) are recovered from its offset
          const BlockDev *NB = blocks + B->nbr[dir][x < 0 ? 0 : 1];
          const DirDev *ND = &NB->dir[dir];
          const long long s2 = qbase / D->qT2, s1 = (qbase - s2 * D->qT2) / D->qT1;
          src = static_cast<const T *>(NB->q[stage]) + s1 * ND->qT1 + s2 * ND->qT2 +
                (long long)(x < 0 ? ND->nd + x : x - nd) * ND->qsd;
          cs = NB->qc;
          FPK_CHK_ONLY(sb = static_cast<const T *>(NB->q[stage]); sn = 5 * NB->qc;)
          return;
        } else {
          xx = x < 0 ? -1 - x : 2 * nd - 1 - x;
          const long long T1 = D->qT1;
          const int n1 = D->nt1, cw = B->cut;
          const int s1 = (int)((qbase / T1) % n1);
          if (bc == 4 && (s1 < cw || s1 >= n1 - cw)) qsrc = qbase + (long long)(n1 - 1 - 2 * s1) * T1;
          else wall = true;
        }
      }
      src = qin + qsrc + (long long)xx * qsd;
    };

    // global loads of one cell (Q, metric vector, 1/J) with the boundary rule applied
    auto fetch = [&](int x, T Q[5], T k[3], T &invJ) {
      if (x >= -G && x < nd + G) {
        const long long mo = (long long)x * msd;
#pragma unroll
        for (int a = 0; a < 3; ++a) k[a] = *FPK_IN(met + ((3LL * dir + a) * mc + mo), metb, 10 * mc, B->status);
        invJ = *FPK_IN(met + (9LL * mc + mo), metb, 10 * mc, B->status);
        const T *qp;
        long long cs;
        bool far, wall;
        FPK_CHK_ONLY(const T *sb; long long sn;)
        bc_source(x, qp, cs, far, wall FPK_CHK_ONLY(, sb, sn));
        if (far) {
#pragma unroll
          for (int v = 0; v < 5; ++v) Q[v] = qb[v];
        } else {
#pragma unroll
          for (int v = 0; v < 5; ++v) Q[v] = __ldg(FPK_IN(qp + v * cs, sb, sn, B->status));
          // slip wall: reflect about the boundary face of this line (face -1/2 or nd-1/2)
          if (BND && wall)
            wall_reflect<T>(Q, FPK_IN(fmet + (x < 0 ? 0LL : (long long)nd * fsd), fmetb, fcs, B->status), fcs);
        }
      } else {   // beyond every stencil that a face of this line uses
#pragma unroll
        for (int v = 0; v < 5; ++v) Q[v] = qb[v];
        k[0] = T(1); k[1] = T(0); k[2] = T(0);
        invJ = T(1);
      }
    };
    // primitives and spectral radius of a fetched cell into the ring
    auto stage_cell = [&](int x, const T Q[5], const T k[3], T invJ) {
      const T rinv = Num<T>::rcp(Q[0]);
      const T u0 = Q[1] * rinv, u1 = Q[2] * rinv, u2 = Q[3] * rinv;
      const T p = g1 * (Q[4] - T(0.5) * (Q[1] * u0 + Q[2] * u1 + Q[3] * u2));
      const T Jc = Num<T>::rcp(invJ);
      const T gx = Jc * k[0], gy = Jc * k[1], gz = Jc * k[2];
      const T c = Num<T>::sqrt_(gam * p * rinv);
      T *cp = sm + off(x);
#pragma unroll
      for (int v = 0; v < 5; ++v) cp[(CF_Q + v) * kRing] = Q[v];
      cp[(CF_K + 0) * kRing] = k[0];
      cp[(CF_K + 1) * kRing] = k[1];
      cp[(CF_K + 2) * kRing] = k[2];
      cp[CF_INVJ * kRing] = invJ;
      cp[CF_RINV * kRing] = rinv;
      cp[(CF_U + 0) * kRing] = u0;
      cp[(CF_U + 1) * kRing] = u1;
      cp[(CF_U + 2) * kRing] = u2;
      cp[CF_H * kRing] = (Q[4] + p) * rinv;
      cp[CF_SQR * kRing] = Num<T>::sqrt_(Q[0]);
      cp[CF_UC * kRing] = u0 * gx + u1 * gy + u2 * gz;
      cp[CF_AC * kRing] = c * Num<T>::sqrt_(gx * gx + gy * gy + gz * gz);
    };

    // asynchronous copy of one cell's loads into this thread's staging slots
    // asynchronous copy of the face metric of face ff into staging slot `slot` (0/1,
    // alternating between chunks)
    auto prefetch_face = [&](int ff, int slot) {
      T *dst = nsb + tid + (9 + 3 * slot) * kThreads;
#pragma unroll
      for (int c = 0; c < 3; ++c)
        cp_async_el(dst + c * kThreads, FPK_IN(fmet + c * fcs + (long long)(ff + 1) * fsd, fmetb, 3 * fcs, B->status));
    };
    auto prefetch_cell = [&](int x) {
      T *dst = nsb + tid;
      if (x >= -G && x < nd + G) {
        const long long mo = (long long)x * msd;
#pragma unroll
        for (int a = 0; a < 3; ++a)
          cp_async_el(dst + (5 + a) * kThreads, FPK_IN(met + (3LL * dir + a) * mc + mo, metb, 10 * mc, B->status));
        cp_async_el(dst + 8 * kThreads, FPK_IN(met + 9LL * mc + mo, metb, 10 * mc, B->status));
        const T *qp;
        long long cs;
        bool far, wall;
        FPK_CHK_ONLY(const T *sb; long long sn;)
        bc_source(x, qp, cs, far, wall FPK_CHK_ONLY(, sb, sn));
        if (far) {
#pragma unroll
          for (int v = 0; v < 5; ++v) dst[v * kThreads] = qb[v];
        } else {   // a wall ghost copies its mirror cell; the reflection is applied when staged
#pragma unroll
          for (int v = 0; v < 5; ++v) cp_async_el(dst + v * kThreads, FPK_IN(qp + v * cs, sb, sn, B->status));
        }
      } else {
#pragma unroll
        for (int v = 0; v < 5; ++v) dst[v * kThreads] = qb[v];
        dst[5 * kThreads] = T(1);
        dst[6 * kThreads] = T(0);
        dst[7 * kThreads] = T(0);
        dst[8 * kThreads] = T(1);
      }
    };
    // asynchronous copy of the epilogue operands of cell x (residual accumulator,
    // Q^n, metric differences, face metric of x+1/2) into this thread's slots
    auto prefetch_epilogue = [&](int x) {
      T *dst = epb + tid;
      const long long qo = qbase + (long long)x * qsd;
      if (mode != MODE_WRITE) {
        const T *ra = static_cast<const T *>(B->racc) + qo;
#pragma unroll
        for (int v = 0; v < 5; ++v)
          cp_async_el(dst + v * kThreads, FPK_IN(ra + v * qc, static_cast<const T *>(B->racc), 5 * qc, B->status));
      }
      if (mode == MODE_RK && stage != 0) {
        const T *qn = static_cast<const T *>(B->q[0]) + qo;
#pragma unroll
        for (int v = 0; v < 5; ++v)
          cp_async_el(dst + (5 + v) * kThreads, FPK_IN(qn + v * qc, static_cast<const T *>(B->q[0]), 5 * qc, B->status));
      }
      if (fpform) {
        const T *dkp = static_cast<const T *>(D->dk) + qo;
#pragma unroll
        for (int c = 0; c < 3; ++c)
          cp_async_el(dst + (10 + c) * kThreads, FPK_IN(dkp + c * qc, static_cast<const T *>(D->dk), 3 * qc, B->status));
      }
    };

    const int nch = (nd + 1 + S - 1) / S;
    // prologue: the first chunk's window [a0-4, a0+S+4), a0 = -1, and its faces' metrics
    if (lineOK) {
      if (tf - 1 < nd) prefetch_face(tf - 1, 0);
      cp_async_commit();
      // S >= 8, so the window's S + 8 cells are one per thread plus a second one for the
      // threads tf < 8: both loads are issued before either cell is staged
      const bool two = tf < 8;
      T Qa[5], ka[3], ija, Qb[5], kb[3], ijb;
      fetch(-5 + tf, Qa, ka, ija);
      if (two) fetch(-5 + tf + S, Qb, kb, ijb);
      stage_cell(-5 + tf, Qa, ka, ija);
      if (two) stage_cell(-5 + tf + S, Qb, kb, ijb);
    }
    cp_async_wait_all();
    __syncthreads();

    for (int ch = 0; ch < nch; ++ch) {
      const int a = ch * S - 1;                      // first face of the chunk
      // ---- start the loads this chunk's epilogue and the next chunk need
      const bool nextOK = lineOK && ch + 1 < nch;
      if (lineOK && a + tf >= 0 && a + tf < nd) prefetch_epilogue(a + tf);
      if (nextOK) prefetch_cell(a + S + 4 + tf);
      if (nextOK && a + S + tf < nd) prefetch_face(a + S + tf, (ch + 1) & 1);
      if (ch == 0 && nit < nitems) fetch_desc(cur ^ 1, s_item[cur ^ 1].x);   // next item's descriptor
      cp_async_commit();
      // ---- one face per thread: face ff + 1/2 between cells ff and ff+1
      const int ff = a + tf;
      if (lineOK && ff < nd) {
        const int i0 = ff;
        int o[8];
#pragma unroll
        for (int q = 0; q < 8; ++q) o[q] = off(i0 - 3 + q);
#define CELL(field, q) sm[(field) * kRing + o[(q)]]
        T Qi[5];
#pragma unroll
        for (int v = 0; v < 5; ++v) Qi[v] = CELL(CF_Q + v, 3);
        // face metric of this face, staged by the previous chunk (or the prologue)
        T kf[3];
#pragma unroll
        for (int c = 0; c < 3; ++c) kf[c] = nsb[(9 + 3 * (ch & 1) + c) * kThreads + tid];

        // reference face state Q* = Q_i + delta (Eqs. Q_star, QdJ_star, 1dJ at order M)
        using P = typename PairOf<T>::type;
        T dl[5] = {T(0), T(0), T(0), T(0), T(0)};
        // The cells q = kQlo .. kQlo + M - 1 of the weighted sum are taken in mirror pairs
        // (kQlo + m, kQlo + M - 1 - m), m < M/2, whose weights are equal, two cells per packed
        // instruction.  These are the stencil loops' pairs (q, 7 - q) of the same cells, so linear
        // upwind with the switches folded keeps the pairs' Q_q - Q_i and (1/J)_q for its stencil
        // differences instead of loading and subtracting them again.
        constexpr bool kKeep = SCHEME == 1 && FIX != 0;
        constexpr int kQlo = 3 - M / 2 + 1;
        P dqk[4][5], ijk[4];
        if (fpform) {
          P acc[5];
#pragma unroll
          for (int v = 0; v < 5; ++v) acc[v] = pc<P>(T(0));
          P wsum = pc<P>(T(0));
#pragma unroll
          for (int m = 0; m < M / 2; ++m) {
            const int q = kQlo + m, q2 = kQlo + M - 1 - m;
            const P ij = pmk(CELL(CF_INVJ, q), CELL(CF_INVJ, q2));
            const P w = pmul(pc<P>(T(MidW<M>::w(m))), ij);
            wsum = padd(wsum, w);
            if (kKeep) ijk[m] = ij;
#pragma unroll
            for (int v = 0; v < 5; ++v) {
              const P dq = psub(pmk(CELL(CF_Q + v, q), CELL(CF_Q + v, q2)), pc<P>(Qi[v]));
              if (kKeep) dqk[m][v] = dq;
              acc[v] = pfma(w, dq, acc[v]);
            }
          }
          const T wi = Num<T>::rcp(wsum.x + wsum.y);
#pragma unroll
          for (int v = 0; v < 5; ++v) dl[v] = (acc[v].x + acc[v].y) * wi;
        }
        T Qs[5];
#pragma unroll
        for (int v = 0; v < 5; ++v) Qs[v] = Qi[v] + dl[v];
        const T rinvs = Num<T>::rcp(Qs[0]);
        const T us[3] = {Qs[1] * rinvs, Qs[2] * rinvs, Qs[3] * rinvs};
        const T ps = g1 * (Qs[4] - T(0.5) * (Qs[1] * us[0] + Qs[2] * us[1] + Qs[3] * us[2]));
        const T ms[3] = {Qs[1], Qs[2], Qs[3]};

        // Lax-Friedrichs speeds: local (max over the stencil cells i-2..i+3) or global
        T lm = T(0), l0 = T(0), lp = T(0);
        if (glf) {
          lm = s_lam[0]; l0 = s_lam[1]; lp = s_lam[2];
        } else {
#pragma unroll
          for (int q = Q0; q < Q0 + NS; ++q) {
            const T U = CELL(CF_UC, q), ac = CELL(CF_AC, q);
            lm = fmax(lm, fabs(U - ac));
            l0 = fmax(l0, fabs(U));
            lp = fmax(lp, fabs(U + ac));
          }
        }
        T lam[5];
        if (charwise) {
          lam[0] = lm; lam[1] = l0; lam[2] = l0; lam[3] = l0; lam[4] = lp;
        } else {
          const T lmax = fmax(lm, lp);
          lam[0] = lam[1] = lam[2] = lam[3] = lam[4] = lmax;
        }

        // Roe average of cells i, i+1 and eigenvector basis in the face normal
        const T rl = CELL(CF_SQR, 3), rr = CELL(CF_SQR, 4);
        const T rs = Num<T>::rcp(rl + rr);
        T u[3];
#pragma unroll
        for (int c = 0; c < 3; ++c) u[c] = (rl * CELL(CF_U + c, 3) + rr * CELL(CF_U + c, 4)) * rs;
        const T H = (rl * CELL(CF_H, 3) + rr * CELL(CF_H, 4)) * rs;
        const T q2 = u[0] * u[0] + u[1] * u[1] + u[2] * u[2];
        const T c2 = g1 * (H - T(0.5) * q2);
        const T cs = Num<T>::sqrt_(c2);
        const T csi = Num<T>::rcp(cs);
        const T bb = g1 * csi * csi;
        const T knr = Num<T>::rsqrt_(kf[0] * kf[0] + kf[1] * kf[1] + kf[2] * kf[2]);
        const T n[3] = {kf[0] * knr, kf[1] * knr, kf[2] * knr};
        // first tangent, normalised: e_z x n where n is far from e_z, else n x e_x.  Chosen by
        // selects (faster for linear upwind, WENO7 and component-wise WENO5), except in the
        // folded WENO5 sweep, where the selects cost registers, and in WENOCU6: there a branch
        // measured faster.
        T t1[3], t2[3];
        const bool lowz = n[2] * n[2] <= T(0.5);
        if constexpr ((SCHEME == 0 && FIX != 0) || SCHEME == 3) {
          if (lowz) {
            const T s = Num<T>::rsqrt_(n[0] * n[0] + n[1] * n[1]);
            t1[0] = -n[1] * s; t1[1] = n[0] * s; t1[2] = T(0);
          } else {
            const T s = Num<T>::rsqrt_(n[1] * n[1] + n[2] * n[2]);
            t1[0] = T(0); t1[1] = n[2] * s; t1[2] = -n[1] * s;
          }
        } else {
          const T s = Num<T>::rsqrt_(lowz ? n[0] * n[0] + n[1] * n[1] : n[1] * n[1] + n[2] * n[2]);
          t1[0] = lowz ? -n[1] * s : T(0);
          t1[1] = (lowz ? n[0] : n[2]) * s;
          t1[2] = lowz ? T(0) : -n[1] * s;
        }
        t2[0] = n[1] * t1[2] - n[2] * t1[1];
        t2[1] = n[2] * t1[0] - n[0] * t1[2];
        t2[2] = n[0] * t1[1] - n[1] * t1[0];
        const T Un = u[0] * n[0] + u[1] * n[1] + u[2] * n[2];
        const T ut1 = u[0] * t1[0] + u[1] * t1[1] + u[2] * t1[2];
        const T ut2 = u[0] * t2[0] + u[1] * t2[1] + u[2] * t2[2];
        // half the left-eigenvector rows (the 1/2 of the Lax-Friedrichs split folded in)
        const T qbb = T(0.25) * bb, hq2 = T(0.5) * q2, qcs = T(0.25) * csi;
        const T h1[3] = {T(0.5) * t1[0], T(0.5) * t1[1], T(0.5) * t1[2]};
        const T h2[3] = {T(0.5) * t2[0], T(0.5) * t2[1], T(0.5) * t2[2]};
        const T hut1 = T(0.5) * ut1, hut2 = T(0.5) * ut2;

        // (1/2) l_s . d for the five characteristic fields
        auto project = [&](const T d[5], T c[5]) {
          if (!charwise) {
#pragma unroll
            for (int v = 0; v < 5; ++v) c[v] = T(0.5) * d[v];
            return;
          }
          const T X4 = qbb * (hq2 * d[0] - (u[0] * d[1] + u[1] * d[2] + u[2] * d[3]) + d[4]);
          const T Y4 = (Un * d[0] - (n[0] * d[1] + n[1] * d[2] + n[2] * d[3])) * qcs;
          c[0] = X4 + Y4;
          c[1] = T(0.5) * d[0] - T(2) * X4;
          c[2] = h1[0] * d[1] + h1[1] * d[2] + h1[2] * d[3] - hut1 * d[0];
          c[3] = h2[0] * d[1] + h2[1] * d[2] + h2[2] * d[3] - hut2 * d[0];
          c[4] = X4 - Y4;
        };

        // the same projection of two stencil points at once (the rows are the face's)
        auto project_pair = [&](const P d[5], P c[5]) {
          if (!charwise) {
#pragma unroll
            for (int v = 0; v < 5; ++v) c[v] = pmul(pc<P>(T(0.5)), d[v]);
            return;
          }
          const P ud = pfma(pc<P>(u[0]), d[1], pfma(pc<P>(u[1]), d[2], pmul(pc<P>(u[2]), d[3])));
          const P X4 = pmul(pc<P>(qbb), pfma(pc<P>(hq2), d[0], psub(d[4], ud)));
          const P nd = pfma(pc<P>(n[0]), d[1], pfma(pc<P>(n[1]), d[2], pmul(pc<P>(n[2]), d[3])));
          const P Y4 = pmul(pc<P>(qcs), psub(pmul(pc<P>(Un), d[0]), nd));
          c[0] = padd(X4, Y4);
          c[1] = pfma(pc<P>(T(-2)), X4, pmul(pc<P>(T(0.5)), d[0]));
          c[2] = pfma(pc<P>(h1[0]), d[1], pfma(pc<P>(h1[1]), d[2], pfma(pc<P>(h1[2]), d[3], pmul(pc<P>(-hut1), d[0]))));
          c[3] = pfma(pc<P>(h2[0]), d[1], pfma(pc<P>(h2[1]), d[2], pfma(pc<P>(h2[2]), d[3], pmul(pc<P>(-hut2), d[0]))));
          c[4] = psub(X4, Y4);
        };

        // h: the back-projected characteristic part of the face flux, cen: the part added
        // to it outside the projection (linear upwind only)
        T h[5], cen[5] = {T(0), T(0), T(0), T(0), T(0)};
        if constexpr (SCHEME == 1) {
          // Linear upwind (Eq. linear_upwind; Appendix Eq. new_form_linear_upwind) is linear in
          // the split values and the speeds are constant over the stencil, so the projection
          // commutes with the reconstruction:
          //   sum_s r_s [W+(f+_s) + W-(f-_s)] = C6(dF) + R Lambda L D(dQ~),
          // C6 = (1, -8, 37, 37, -8, 1)/60 (half the sum of the two upwind stencils) and
          // D = (1, -5, 10, -10, 5, -1)/60 (half their difference) over i-2..i+3.  One
          // projection per face instead of two per stencil point; dF and dQ~ = dQ (1/J)_m as
          // in the WENO branch (stencil point s paired with its mirror 5-s).
          constexpr T c6[3] = {T(1.0 / 60.0), T(-8.0 / 60.0), T(37.0 / 60.0)};
          constexpr T d5[3] = {T(1.0 / 60.0), T(-5.0 / 60.0), T(10.0 / 60.0)};
          P cenp[5], disp[5];
#pragma unroll
          for (int v = 0; v < 5; ++v) cenp[v] = disp[v] = pc<P>(T(0));
#pragma unroll
          for (int s = 0; s < 3; ++s) {
            const int q = s + 1, q2 = 6 - s;
            P dp[5], out[5];
            // the weighted sum's pair of these two cells, if it has one (every pair at M6 and M8)
            const int km = q - kQlo;
            const bool kept = kKeep && km >= 0;
            const int kmi = kept ? km : 0;
            if (fpform) {
              P kp2[3], uBp[3];
#pragma unroll
              for (int v = 0; v < 5; ++v)
                dp[v] = kept ? psub(dqk[kmi][v], pc<P>(dl[v]))
                             : psub(psub(pmk(CELL(CF_Q + v, q), CELL(CF_Q + v, q2)), pc<P>(Qi[v])), pc<P>(dl[v]));
#pragma unroll
              for (int c = 0; c < 3; ++c) {
                kp2[c] = pmk(CELL(CF_K + c, q), CELL(CF_K + c, q2));
                uBp[c] = pmk(CELL(CF_U + c, q), CELL(CF_U + c, q2));
              }
              dflux_pair<T>(g1, pmk(CELL(CF_RINV, q), CELL(CF_RINV, q2)), uBp, us, ms, Qs[4], ps, dp, kp2, out);
            } else {
              // plain scheme: F~_m and Q~_m themselves
              P uBp[3], kp2[3];
#pragma unroll
              for (int c = 0; c < 3; ++c) {
                kp2[c] = pmk(CELL(CF_K + c, q), CELL(CF_K + c, q2));
                uBp[c] = pmk(CELL(CF_U + c, q), CELL(CF_U + c, q2));
              }
#pragma unroll
              for (int v = 0; v < 5; ++v) dp[v] = pmk(CELL(CF_Q + v, q), CELL(CF_Q + v, q2));
              const P ke = pfma(dp[3], uBp[2], pfma(dp[2], uBp[1], pmul(dp[1], uBp[0])));
              const P pm = pmul(pc<P>(g1), pfma(pc<P>(T(-0.5)), ke, dp[4]));
              const P U = pfma(uBp[2], kp2[2], pfma(uBp[1], kp2[1], pmul(uBp[0], kp2[0])));
              out[0] = pmul(dp[0], U);
#pragma unroll
              for (int c = 0; c < 3; ++c) out[1 + c] = pfma(pm, kp2[c], pmul(dp[1 + c], U));
              out[4] = pmul(padd(dp[4], pm), U);
            }
            const P ijp = kept ? ijk[kmi] : pmk(CELL(CF_INVJ, q), CELL(CF_INVJ, q2));
            const P ds = pmk(d5[s], -d5[s]);
#pragma unroll
            for (int v = 0; v < 5; ++v) {
              cenp[v] = pfma(pc<P>(c6[s]), out[v], cenp[v]);
              disp[v] = pfma(ds, pmul(dp[v], ijp), disp[v]);
            }
          }
          T dis[5];
#pragma unroll
          for (int v = 0; v < 5; ++v) {
            cen[v] = cenp[v].x + cenp[v].y;
            dis[v] = disp[v].x + disp[v].y;
          }
          // lambda_s l_s . D (project() carries the 1/2 of the split: twice its rows)
          T c[5];
          project(dis, c);
#pragma unroll
          for (int v = 0; v < 5; ++v) h[v] = T(2) * lam[v] * c[v];
        } else {
          // split stencil values f+/- for the NS stencil points
          T fpl[NS][5], fmi[NS][5];
          // f+- = (1/2) l.(dF +- lambda d (1/J)_m) of one stencil point
          auto split_point = [&](int s, const T dF[5], const T d[5], T ijm) {
            T cF[5], cD[5];
            project(dF, cF);
            project(d, cD);
            const T mu0 = lam[0] * ijm, mu1 = lam[1] * ijm, mu4 = lam[4] * ijm;
            const T mu[5] = {mu0, mu1, mu1, mu1, mu4};
#pragma unroll
            for (int v = 0; v < 5; ++v) {
              fpl[s][v] = cF[v] + mu[v] * cD[v];
              fmi[s][v] = cF[v] - mu[v] * cD[v];
            }
          };
          if (fpform) {
            // reference-state differences of the stencil points two at a time (packed): points
            // s and its mirror NS-1-s, whose f+ and f- are the (+, -) lanes of the reconstruction
            // pair s; the mirror pair NS-1-s is formed lane by lane
            const P lpm[3] = {pmk(lam[0], -lam[0]), pmk(lam[1], -lam[1]), pmk(lam[4], -lam[4])};
#pragma unroll
            for (int s = 0; s < NS / 2; ++s) {
              const int mir = NS - 1 - s;
              const int q = s + Q0, q2 = mir + Q0;
              P dp[5], kp2[3], uBp[3], out[5];
#pragma unroll
              for (int v = 0; v < 5; ++v)
                dp[v] = psub(psub(pmk(CELL(CF_Q + v, q), CELL(CF_Q + v, q2)), pc<P>(Qi[v])), pc<P>(dl[v]));
#pragma unroll
              for (int c = 0; c < 3; ++c) {
                kp2[c] = pmk(CELL(CF_K + c, q), CELL(CF_K + c, q2));
                uBp[c] = pmk(CELL(CF_U + c, q), CELL(CF_U + c, q2));
              }
              dflux_pair<T>(g1, pmk(CELL(CF_RINV, q), CELL(CF_RINV, q2)), uBp, us, ms, Qs[4], ps, dp, kp2, out);
              P cF[5], cD[5];
              project_pair(out, cF);
              project_pair(dp, cD);
              // (lambda (1/J)_s, -lambda (1/J)_mirror) for the three speed classes
              const P ijp = pmk(CELL(CF_INVJ, q), CELL(CF_INVJ, q2));
              const P mp[3] = {pmul(lpm[0], ijp), pmul(lpm[1], ijp), pmul(lpm[2], ijp)};
#pragma unroll
              for (int v = 0; v < 5; ++v) {
                const P &mv = mp[v == 0 ? 0 : (v == 4 ? 2 : 1)];
                const P r = pfma(mv, cD[v], cF[v]);                 // (f+ of s, f- of the mirror)
                fpl[s][v] = r.x;
                fmi[mir][v] = r.y;
                fmi[s][v] = cF[v].x - mv.x * cD[v].x;
                fpl[mir][v] = cF[v].y - mv.y * cD[v].y;
              }
            }
          } else {
            // plain scheme: F~_m and Q~_m themselves
#pragma unroll
            for (int s = 0; s < NS; ++s) {
              const int q = s + Q0;
              T dF[5], d[5];
              const T km[3] = {CELL(CF_K, q), CELL(CF_K + 1, q), CELL(CF_K + 2, q)};
              const T uB[3] = {CELL(CF_U, q), CELL(CF_U + 1, q), CELL(CF_U + 2, q)};
#pragma unroll
              for (int v = 0; v < 5; ++v) d[v] = CELL(CF_Q + v, q);
              const T pm = g1 * (d[4] - T(0.5) * (d[1] * uB[0] + d[2] * uB[1] + d[3] * uB[2]));
              const T U = uB[0] * km[0] + uB[1] * km[1] + uB[2] * km[2];
              dF[0] = d[0] * U;
              dF[1] = d[1] * U + pm * km[0];
              dF[2] = d[2] * U + pm * km[1];
              dF[3] = d[3] * U + pm * km[2];
              dF[4] = (d[4] + pm) * U;
              split_point(s, dF, d, CELL(CF_INVJ, q));
            }
          }
#undef CELL
          // reconstruct each field from both sides (the - side mirrored) and back-project
#pragma unroll
          for (int v = 0; v < 5; ++v) {
            if constexpr (SCHEME == 2) {
              P w7[7];
#pragma unroll
              for (int t = 0; t < 7; ++t) w7[t] = pmk(fpl[t][v], fmi[7 - t][v]);   // i-3..i+3 / i+4..i-2
              const P r = recon7_pair<T>(w7);
              h[v] = r.x + r.y;
            } else if constexpr (SCHEME == 3) {
              P w6[6];
#pragma unroll
              for (int t = 0; t < 6; ++t) w6[t] = pmk(fpl[t][v], fmi[5 - t][v]);   // i-2..i+3 / i+3..i-2
              const P r = recon6cu_pair<T>(w6);
              h[v] = r.x + r.y;
            } else {
              const P r = recon5_pair<T, SCHEME>(pmk(fpl[0][v], fmi[5][v]), pmk(fpl[1][v], fmi[4][v]),
                                                 pmk(fpl[2][v], fmi[3][v]), pmk(fpl[3][v], fmi[2][v]),
                                                 pmk(fpl[4][v], fmi[1][v]));
              h[v] = r.x + r.y;
            }
          }
        }
        T F[5];
        if (charwise) {
          const T sa = h[0] + h[4], da = h[4] - h[0];
          F[0] = sa + h[1];
#pragma unroll
          for (int c = 0; c < 3; ++c) F[1 + c] = u[c] * (sa + h[1]) + cs * n[c] * da + t1[c] * h[2] + t2[c] * h[3];
          F[4] = H * sa + cs * Un * da + T(0.5) * q2 * h[1] + ut1 * h[2] + ut2 * h[3];
        } else {
#pragma unroll
          for (int v = 0; v < 5; ++v) F[v] = h[v];
        }
        T *fp = fr + off(ff);
#pragma unroll
        for (int v = 0; v < 5; ++v) {
          if constexpr (SCHEME == 1) F[v] += cen[v];
          fp[v * kRing] = F[v];
          fp[(5 + v) * kRing] = dl[v];
        }
      }
      cp_async_wait_all();
      __syncthreads();
      // ---- residual of cell x = a + tf from its two faces, then the epilogue
      const int x = a + tf;
      if (lineOK && x >= 0 && x < nd) {
        const long long qo = qbase + (long long)x * qsd;
        const int ox = off(x), oxm = off(x - 1);
        T R[5];
#pragma unroll
        for (int v = 0; v < 5; ++v) R[v] = fr[v * kRing + ox] - fr[v * kRing + oxm];
        if (fpform) {
          // reference states of the two faces: Q*_+ = Q_x + delta_+, Q*_- = Q_{x-1} + delta_-
          T Qp[5], Qm[5], dQ[5], dqm[5];
#pragma unroll
          for (int v = 0; v < 5; ++v) {
            const T qx = sm[(CF_Q + v) * kRing + ox], qx1 = sm[(CF_Q + v) * kRing + oxm];
            const T dp = fr[(5 + v) * kRing + ox], dm = fr[(5 + v) * kRing + oxm];
            Qp[v] = qx + dp;
            Qm[v] = qx1 + dm;
            dQ[v] = (qx - qx1) + (dp - dm);
            dqm[v] = (qx1 - qb[v]) + dm;
          }
          const T rA = Num<T>::rcp(Qm[0]);
          const T uA[3] = {Qm[1] * rA, Qm[2] * rA, Qm[3] * rA};
          const T pA = g1 * (Qm[4] - T(0.5) * (Qm[1] * uA[0] + Qm[2] * uA[1] + Qm[3] * uA[2]));
          const T mA[3] = {Qm[1], Qm[2], Qm[3]};
          const T rB = Num<T>::rcp(Qp[0]);
          const T uBp[3] = {Qp[1] * rB, Qp[2] * rB, Qp[3] * rB};
          // k_{x+1/2} is the metric of the face this thread computed in this chunk
          T kp[3], dk[3];
#pragma unroll
          for (int c = 0; c < 3; ++c) {
            dk[c] = epb[(10 + c) * kThreads + tid];
            kp[c] = nsb[(9 + 3 * (ch & 1) + c) * kThreads + tid];
          }
          T t1v[5], t2v[5];
          dflux<T>(g1, rB, uBp, uA, mA, Qm[4], pA, dQ, kp, t1v);          // [F(Q*_+) - F(Q*_-)] . k_+
          dflux<T>(g1, rA, uA, ub, mbq, qb[4], pb, dqm, dk, t2v);         // [F(Q*_-) - F(Qbar)] . (k_+ - k_-)
#pragma unroll
          for (int v = 0; v < 5; ++v) R[v] += t1v[v] + t2v[v];
        }
        T *racc = static_cast<T *>(B->racc) + qo;
        FPK_CHK_ONLY(T *const raccb = static_cast<T *>(B->racc);)
        const T *ra = epb + tid;                      // prefetched accumulator
        if (mode == MODE_WRITE) {
#pragma unroll
          for (int v = 0; v < 5; ++v) *FPK_IN(racc + v * qc, raccb, 5 * qc, B->status) = R[v];
        } else if (mode == MODE_ADD) {
#pragma unroll
          for (int v = 0; v < 5; ++v) *FPK_IN(racc + v * qc, raccb, 5 * qc, B->status) = ra[v * kThreads] + R[v];
        } else {
          const T Jc = Num<T>::rcp(sm[CF_INVJ * kRing + ox]);
          if (mode == MODE_RHS) {
            T *out = static_cast<T *>(B->dqdt) + qo;
#pragma unroll
            for (int v = 0; v < 5; ++v)
              *FPK_IN(out + v * qc, static_cast<T *>(B->dqdt), 5 * qc, B->status) = -Jc * (ra[v * kThreads] + R[v]);
          } else {
            // SSP-RK3 stage (Gottlieb & Shu) in increment form:
            // Q^(s+1) = Q^(s) + a_s (Q^n - Q^(s)) + b_s dt L(Q^(s))
            const T dt = s_dt;
            const T as = stage == 0 ? T(0) : (stage == 1 ? T(0.75) : T(1.0 / 3.0));
            const T bs = stage == 0 ? T(1) : (stage == 1 ? T(0.25) : T(2.0 / 3.0));
            T *qo_p = static_cast<T *>(B->q[(stage + 1) % 3]) + qo;
            bool bad = false;
#pragma unroll
            for (int v = 0; v < 5; ++v) {
              const T qk = sm[(CF_Q + v) * kRing + ox];
              const T Lv = -Jc * (ra[v * kThreads] + R[v]);
              T nv = qk + bs * dt * Lv;
              if (stage != 0) nv = qk + as * (ra[(5 + v) * kThreads] - qk) + bs * dt * Lv;
              *FPK_IN(qo_p + v * qc, static_cast<T *>(B->q[(stage + 1) % 3]), 5 * qc, B->status) = nv;
              bad |= !isfinite(nv);
            }
            if (bad) atomicOr(B->status, ST_NONFINITE);
          }
        }
      }
      __syncthreads();
      // ---- stage the next chunk's new cell from this thread's staging slots
      if (nextOK) {
        const int xs = a + S + 4 + tf;
        const T *src = nsb + tid;
        T Q[5] = {src[0], src[kThreads], src[2 * kThreads], src[3 * kThreads], src[4 * kThreads]};
        const T k[3] = {src[5 * kThreads], src[6 * kThreads], src[7 * kThreads]};
        if (BND && xs >= nd && xs < nd + G && bchi >= 3) {   // past the high end: slip-wall ghost?
          const T *qp;
          long long cs;
          bool far, wall;
          FPK_CHK_ONLY(const T *sb; long long sn;)
          bc_source(xs, qp, cs, far, wall FPK_CHK_ONLY(, sb, sn));
          if (wall) wall_reflect<T>(Q, FPK_IN(fmet + (long long)nd * fsd, fmetb, fcs, B->status), fcs);
        }
        stage_cell(xs, Q, k, src[8 * kThreads]);
      }
      __syncthreads();
    }
  }
}

// dynamic shared memory of a sweep variant: the cell and face rings, then the per-thread slots
template <typename T, int SCHEME, int FIX>
constexpr size_t sweep_smem() {
  return ((size_t)(kCellFields + kFaceFields) * sweep_ring(sizeof(T) == 4, SCHEME, FIX) +
          (size_t)(kNextFields + kEpiFields) * sweep_threads(sizeof(T) == 4, SCHEME, FIX)) * sizeof(T);
}

template <typename T, int M, int SCHEME, bool BND, int FIX>
cudaError_t launch_one(const SweepLaunch &L, int charwise, int fp, cudaStream_t s) {
  constexpr size_t smem = sweep_smem<T, SCHEME, FIX>();
  constexpr int nt = sweep_threads(sizeof(T) == 4, SCHEME, FIX);
  if (L.nitems <= 0) return cudaSuccess;
  fp_sweep<T, M, SCHEME, BND, FIX><<<L.grid, nt, smem, s>>>(L.blocks, L.items, L.nitems, L.dir, L.mode,
                                                            L.stage, L.dt, charwise, fp);
  return cudaGetLastError();
}

template <typename T, bool BND, int FIX>
cudaError_t launch_sweep_t(const SweepLaunch &L, int M, int scheme, int charwise, int fp,
                           cudaStream_t s) {
#define FPK_CASE(MM, SS) \
  if (M == MM && scheme == SS) return launch_one<T, MM, SS, BND, FIX>(L, charwise, fp, s);
  FPK_CASE(2, 0) FPK_CASE(4, 0) FPK_CASE(6, 0) FPK_CASE(8, 0)
  FPK_CASE(2, 1) FPK_CASE(4, 1) FPK_CASE(6, 1) FPK_CASE(8, 1)
  FPK_CASE(2, 2) FPK_CASE(4, 2) FPK_CASE(6, 2) FPK_CASE(8, 2)
  FPK_CASE(2, 3) FPK_CASE(4, 3) FPK_CASE(6, 3) FPK_CASE(8, 3)
#undef FPK_CASE
  return cudaErrorInvalidValue;
}

// Opt in to the dynamic shared memory of every variant and return the resident
// CTAs per SM of the requested one.  Called before any launch or graph capture.
template <typename T, bool BND, int FIX>
int prepare_t(int M, int scheme) {
  int nb = 0;
#define FPK_OCC(MM, SS)                                                                              \
  {                                                                                                  \
    constexpr size_t smem = sweep_smem<T, SS, FIX>();                                                \
    cudaFuncSetAttribute(fp_sweep<T, MM, SS, BND, FIX>, cudaFuncAttributeMaxDynamicSharedMemorySize,  \
                         (int)smem);                                                                 \
    if (M == MM && scheme == SS)                                                                     \
      cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, fp_sweep<T, MM, SS, BND, FIX>,              \
                                                    sweep_threads(sizeof(T) == 4, SS, FIX), smem);   \
  }
  FPK_OCC(2, 0) FPK_OCC(4, 0) FPK_OCC(6, 0) FPK_OCC(8, 0)
  FPK_OCC(2, 1) FPK_OCC(4, 1) FPK_OCC(6, 1) FPK_OCC(8, 1)
  FPK_OCC(2, 2) FPK_OCC(4, 2) FPK_OCC(6, 2) FPK_OCC(8, 2)
  FPK_OCC(2, 3) FPK_OCC(4, 3) FPK_OCC(6, 3) FPK_OCC(8, 3)
#undef FPK_OCC
  return nb > 0 ? nb : 1;
}

// One translation unit per (precision, boundary rules, fixed switches): the launcher and the
// preparation of its 16 (M, scheme) variants, named launch_sweep_<NAME> / prepare_sweep_<NAME>.
#define FPK_SWEEP_UNIT(NAME, T, BND, FIX)                                                           \
  cudaError_t launch_sweep_##NAME(const SweepLaunch &L, int M, int scheme, int charwise, int fp,    \
                                  cudaStream_t s) {                                                 \
    return launch_sweep_t<T, BND, FIX>(L, M, scheme, charwise, fp, s);                              \
  }                                                                                                 \
  int prepare_sweep_##NAME(int M, int scheme) { return prepare_t<T, BND, FIX>(M, scheme); }

}  // namespace fpk
