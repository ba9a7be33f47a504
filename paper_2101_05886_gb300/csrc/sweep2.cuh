// sweep2.cuh - the FP32 directional residual sweep with two grid lines per thread.
//
// The same face flux as fp_sweep (sweep.cuh: Sec. 3.2 free-stream-preserving WENO5-JS or
// linear upwind, the same algebra and operation order per line), but every thread carries
// the same face of two adjacent lines a and b, so every arithmetic step of the face, of the
// cell staging and of the epilogue is one packed FP32x2 instruction (FFMA2 / FADD2 / FMUL2)
// on (line a, line b), and the cell and face rings hold (a, b) float2 pairs read with one
// 64-bit shared load.  The WENO5 branch pairs lines instead of a stencil point with its
// mirror.  A CTA of 256 threads covers S faces of 2 TT lines; it needs about 220 KB of shared
// memory and up to 255 registers, so one CTA runs per SM: half the warps of fp_sweep, each
// doing twice the work per instruction.
//
// Lines are taken in pairs (2l, 2l + 1) of the item's lines; a missing second line (odd line
// count) repeats the first and is not stored.  Sides with slip-wall, cut, block-link or halo
// rules are left to fp_sweep.
#pragma once

#include "sweep.cuh"

namespace fpk {

using F2 = float2;

__device__ __forceinline__ F2 prcp2(F2 a) { return make_float2(Num<float>::rcp(a.x), Num<float>::rcp(a.y)); }
__device__ __forceinline__ F2 psqrt2(F2 a) { return make_float2(Num<float>::sqrt_(a.x), Num<float>::sqrt_(a.y)); }
__device__ __forceinline__ F2 prsqrt2(F2 a) { return make_float2(rsqrtf(a.x), rsqrtf(a.y)); }
__device__ __forceinline__ F2 pmaxabs2(F2 m, F2 a) { return make_float2(fmaxf(m.x, fabsf(a.x)), fmaxf(m.y, fabsf(a.y))); }
__device__ __forceinline__ F2 pneg2(F2 a) { return make_float2(-a.x, -a.y); }
__device__ __forceinline__ F2 pcf(float v) { return make_float2(v, v); }
// per-lane select: lane of a where c holds, else of b
__device__ __forceinline__ F2 psel2(bool cx, bool cy, F2 a, F2 b) { return make_float2(cx ? a.x : b.x, cy ? a.y : b.y); }

// [F(B) - F(A)] . k of sweep.cuh's dflux, for two lines; nuA = -(A's velocity)
__device__ __forceinline__ void dflux2(F2 g1, F2 rinvB, const F2 uB[3], const F2 nuA[3], const F2 mA[3], F2 EpA,
                                       const F2 d[5], const F2 k[3], F2 out[5]) {
  const F2 du0 = pmul(pfma(nuA[0], d[0], d[1]), rinvB);
  const F2 du1 = pmul(pfma(nuA[1], d[0], d[2]), rinvB);
  const F2 du2 = pmul(pfma(nuA[2], d[0], d[3]), rinvB);
  F2 dke = pmul(d[1], uB[0]);
  dke = pfma(d[2], uB[1], dke);
  dke = pfma(d[3], uB[2], dke);
  dke = pfma(mA[0], du0, dke);
  dke = pfma(mA[1], du1, dke);
  dke = pfma(mA[2], du2, dke);
  const F2 dp = pmul(g1, pfma(pcf(-0.5f), dke, d[4]));
  const F2 UB = pfma(uB[2], k[2], pfma(uB[1], k[1], pmul(uB[0], k[0])));
  const F2 dU = pfma(du2, k[2], pfma(du1, k[1], pmul(du0, k[0])));
  out[0] = pfma(d[3], k[2], pfma(d[2], k[1], pmul(d[1], k[0])));
  out[1] = pfma(dp, k[0], pfma(mA[0], dU, pmul(d[1], UB)));
  out[2] = pfma(dp, k[1], pfma(mA[1], dU, pmul(d[2], UB)));
  out[3] = pfma(dp, k[2], pfma(mA[2], dU, pmul(d[3], UB)));
  out[4] = pfma(EpA, dU, pmul(padd(d[4], dp), UB));
}

// Shared-memory layout: rings of float2 with the same slot indexing as fp_sweep (kRing
// entries per field), then per-thread staging slots of float2.
constexpr size_t kSweep2Smem =
    ((size_t)(kCellFields + kFaceFields) * kRing + (size_t)(kNextFields + kEpiFields) * kThreads) * sizeof(F2);

template <int M, int SCHEME>
__global__ void __launch_bounds__(kThreads, 1)
fp_sweep2(const BlockDev *__restrict__ blocks, const int2 *__restrict__ items, int nitems, int dir, int mode,
          int stage, const double *__restrict__ dtp, int charwise, int fpform) {
  static_assert(SCHEME == 0 || SCHEME == 1, "two-line sweep: WENO5-JS and linear upwind");
  constexpr int NS = 6;
  extern __shared__ __align__(16) unsigned char smraw2[];
  F2 *const sm = reinterpret_cast<F2 *>(smraw2);            // cell ring: kCellFields x kRing
  F2 *const fr = sm + kCellFields * kRing;                  // face ring: kFaceFields x kRing
  F2 *const nsb = fr + kFaceFields * kRing;                 // next chunk's cell, per thread: 9 x 256 (+ 6 face metric)
  F2 *const epb = nsb + kNextFields * kThreads;             // epilogue operands, per thread: 13 x 256
  float *const nsbf = reinterpret_cast<float *>(nsb);
  float *const epbf = reinterpret_cast<float *>(epb);
  const int tid = threadIdx.x;
  static_assert(sizeof(BlockDev) % 16 == 0, "descriptor copied in 16-byte pieces");
  constexpr int kDescPieces = (int)(sizeof(BlockDev) / 16);
  static_assert(kDescPieces <= kThreads, "one piece per thread");
  __shared__ __align__(16) unsigned char s_desc[2][sizeof(BlockDev)];
  __shared__ __align__(16) int2 s_item[2];
  __shared__ float s_dt;
  __shared__ float s_lam[3];
  auto fetch_desc = [&](int buf, int blk) {
    if (tid < kDescPieces)
      cp_async16(s_desc[buf] + 16 * tid, reinterpret_cast<const unsigned char *>(blocks + blk) + 16 * tid);
  };
  if (blockIdx.x < nitems) {
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
    if (tid == 0 && nit < nitems) cp_async8(&s_item[cur ^ 1], items + nit);
    if (tid == 0) {
      s_dt = mode == MODE_RK ? float(*dtp) : 0.f;
      if (B->global_lf)
        for (int c = 0; c < 3; ++c) s_lam[c] = static_cast<const float *>(B->lamg)[3 * dir + c];
    }
    const int S = D->S, TT = D->TT, W = 2 * S;
    const bool slotFast = (dir == 0);
    const int tf = slotFast ? (tid % S) : (tid / TT);
    const int tl = slotFast ? (tid / S) : (tid % TT);
    const int LS = slotFast ? 3 * S : 1;
    const int SS = slotFast ? 1 : TT;
    const int lbase = tl * LS;
    const int wm = W - 1;
    const int nd = D->nd;
    // the thread's two lines 2 tl and 2 tl + 1 of the item; a missing second line repeats the first
    const long long La = (long long)item.y + 2 * tl;
    const bool okA = La < D->nlines;
    const bool okB = La + 1 < D->nlines;
    const long long Lb = okB ? La + 1 : La;
    const int t1a = okA ? (int)(La % D->nt1) : 0, t2a = okA ? (int)(La / D->nt1) : 0;
    const int t1b = okA ? (int)(Lb % D->nt1) : 0, t2b = okA ? (int)(Lb / D->nt1) : 0;
    const long long qsd = D->qsd, msd = D->msd, fsd = D->fsd, fcs = D->fc;
    const long long qba = t1a * D->qT1 + t2a * D->qT2, qbb = t1b * D->qT1 + t2b * D->qT2;
    const long long mba = B->moff + t1a * D->mT1 + t2a * D->mT2, mbb = B->moff + t1b * D->mT1 + t2b * D->mT2;
    const long long fba = t1a * D->fT1 + t2a * D->fT2, fbb = t1b * D->fT1 + t2b * D->fT2;
    const long long qc = B->qc, mc = B->mc;
    const int G = B->G, bclo = D->bclo, bchi = D->bchi;
    const float *__restrict__ metb = static_cast<const float *>(B->met);
    const float *__restrict__ fmetb = static_cast<const float *>(D->fmet);
    const float *__restrict__ qin = static_cast<const float *>(B->q[stage]);
    const float g1s = float(B->gamma - 1.0), gams = float(B->gamma);
    const F2 g1 = pcf(g1s), gam = pcf(gams);
    const int glf = B->global_lf;
    float qbs[5];
#pragma unroll
    for (int v = 0; v < 5; ++v) qbs[v] = float(B->qbar[v]);
    F2 qb[5];
#pragma unroll
    for (int v = 0; v < 5; ++v) qb[v] = pcf(qbs[v]);
    const float qbr = Num<float>::rcp(qbs[0]);
    const float ubs[3] = {qbs[1] * qbr, qbs[2] * qbr, qbs[3] * qbr};
    const float pbs = g1s * (qbs[4] - 0.5f * (qbs[1] * ubs[0] + qbs[2] * ubs[1] + qbs[3] * ubs[2]));
    const F2 nub[3] = {pcf(-ubs[0]), pcf(-ubs[1]), pcf(-ubs[2])};
    const F2 mbq[3] = {qb[1], qb[2], qb[3]};
    const F2 Epb = pcf(qbs[4] + pbs);

    auto off = [&](int x) -> int { return lbase + (x & wm) * SS; };

    // source of cell x of the line whose state offset is qbase (periodic wrap, far field,
    // zero gradient): index along the line, or -1 for the far-field state
    auto src_index = [&](int x) -> int {
      if (x >= 0 && x < nd) return x;
      const int bc = x < 0 ? bclo : bchi;
      if (bc == 0) { int xx = x % nd; return xx < 0 ? xx + nd : xx; }
      if (bc == 1) return -1;
      return x < 0 ? 0 : nd - 1;
    };

    // staging slot (field f of this thread) as the float of line a (b = a + 1)
    auto nslot = [&](int f) -> float * { return nsbf + 2 * ((size_t)f * kThreads + tid); };
    auto eslot = [&](int f) -> float * { return epbf + 2 * ((size_t)f * kThreads + tid); };

    auto prefetch_face = [&](int ff, int slot) {
      float *dst = nslot(9 + 3 * slot);
      const long long fo = (long long)(ff + 1) * fsd;
#pragma unroll
      for (int c = 0; c < 3; ++c) {
        cp_async_el(dst + 2 * c * kThreads, fmetb + fba + c * fcs + fo);
        cp_async_el(dst + 2 * c * kThreads + 1, fmetb + fbb + c * fcs + fo);
      }
    };
    // next chunk's cell x of both lines into the staging slots (Q, k, 1/J)
    auto prefetch_cell = [&](int x) {
      float *dst = nslot(0);
      if (x >= -G && x < nd + G) {
        const long long mo = (long long)x * msd;
#pragma unroll
        for (int a = 0; a < 3; ++a) {
          cp_async_el(dst + 2 * (5 + a) * kThreads, metb + mba + (3LL * dir + a) * mc + mo);
          cp_async_el(dst + 2 * (5 + a) * kThreads + 1, metb + mbb + (3LL * dir + a) * mc + mo);
        }
        cp_async_el(dst + 2 * 8 * kThreads, metb + mba + 9LL * mc + mo);
        cp_async_el(dst + 2 * 8 * kThreads + 1, metb + mbb + 9LL * mc + mo);
        const int xs = src_index(x);
        if (xs < 0) {
#pragma unroll
          for (int v = 0; v < 5; ++v) { dst[2 * v * kThreads] = qbs[v]; dst[2 * v * kThreads + 1] = qbs[v]; }
        } else {
          const long long so = (long long)xs * qsd;
#pragma unroll
          for (int v = 0; v < 5; ++v) {
            cp_async_el(dst + 2 * v * kThreads, qin + qba + v * qc + so);
            cp_async_el(dst + 2 * v * kThreads + 1, qin + qbb + v * qc + so);
          }
        }
      } else {
#pragma unroll
        for (int v = 0; v < 5; ++v) { dst[2 * v * kThreads] = qbs[v]; dst[2 * v * kThreads + 1] = qbs[v]; }
        dst[2 * 5 * kThreads] = dst[2 * 5 * kThreads + 1] = 1.f;
        dst[2 * 6 * kThreads] = dst[2 * 6 * kThreads + 1] = 0.f;
        dst[2 * 7 * kThreads] = dst[2 * 7 * kThreads + 1] = 0.f;
        dst[2 * 8 * kThreads] = dst[2 * 8 * kThreads + 1] = 1.f;
      }
    };
    // epilogue operands of cell x (accumulator, Q^n, metric differences) of both lines
    auto prefetch_epilogue = [&](int x) {
      float *dst = eslot(0);
      const long long qa = qba + (long long)x * qsd, qbo = qbb + (long long)x * qsd;
      if (mode != MODE_WRITE) {
        const float *ra = static_cast<const float *>(B->racc);
#pragma unroll
        for (int v = 0; v < 5; ++v) {
          cp_async_el(dst + 2 * v * kThreads, ra + qa + v * qc);
          cp_async_el(dst + 2 * v * kThreads + 1, ra + qbo + v * qc);
        }
      }
      if (mode == MODE_RK && stage != 0) {
        const float *qn = static_cast<const float *>(B->q[0]);
#pragma unroll
        for (int v = 0; v < 5; ++v) {
          cp_async_el(dst + 2 * (5 + v) * kThreads, qn + qa + v * qc);
          cp_async_el(dst + 2 * (5 + v) * kThreads + 1, qn + qbo + v * qc);
        }
      }
      if (fpform) {
        const float *dkp = static_cast<const float *>(D->dk);
#pragma unroll
        for (int c = 0; c < 3; ++c) {
          cp_async_el(dst + 2 * (10 + c) * kThreads, dkp + qa + c * qc);
          cp_async_el(dst + 2 * (10 + c) * kThreads + 1, dkp + qbo + c * qc);
        }
      }
    };
    // direct loads of cell x of both lines (prologue)
    auto fetch = [&](int x, F2 Q[5], F2 k[3], F2 &invJ) {
      if (x >= -G && x < nd + G) {
        const long long mo = (long long)x * msd;
#pragma unroll
        for (int a = 0; a < 3; ++a)
          k[a] = make_float2(__ldg(metb + mba + (3LL * dir + a) * mc + mo), __ldg(metb + mbb + (3LL * dir + a) * mc + mo));
        invJ = make_float2(__ldg(metb + mba + 9LL * mc + mo), __ldg(metb + mbb + 9LL * mc + mo));
        const int xs = src_index(x);
        if (xs < 0) {
#pragma unroll
          for (int v = 0; v < 5; ++v) Q[v] = qb[v];
        } else {
          const long long so = (long long)xs * qsd;
#pragma unroll
          for (int v = 0; v < 5; ++v) Q[v] = make_float2(__ldg(qin + qba + v * qc + so), __ldg(qin + qbb + v * qc + so));
        }
      } else {
#pragma unroll
        for (int v = 0; v < 5; ++v) Q[v] = qb[v];
        k[0] = pcf(1.f); k[1] = pcf(0.f); k[2] = pcf(0.f);
        invJ = pcf(1.f);
      }
    };
    // primitives and spectral radius of a cell pair into the ring (fp_sweep's stage_cell)
    auto stage_cell = [&](int x, const F2 Q[5], const F2 k[3], F2 invJ) {
      const F2 rinv = prcp2(Q[0]);
      const F2 u0 = pmul(Q[1], rinv), u1 = pmul(Q[2], rinv), u2 = pmul(Q[3], rinv);
      const F2 p = pmul(g1, pfma(pcf(-0.5f), pfma(Q[3], u2, pfma(Q[2], u1, pmul(Q[1], u0))), Q[4]));
      const F2 Jc = prcp2(invJ);
      const F2 gx = pmul(Jc, k[0]), gy = pmul(Jc, k[1]), gz = pmul(Jc, k[2]);
      const F2 c = psqrt2(pmul(pmul(gam, p), rinv));
      F2 *cp = sm + off(x);
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
      cp[CF_H * kRing] = pmul(padd(Q[4], p), rinv);
      cp[CF_SQR * kRing] = psqrt2(Q[0]);
      cp[CF_UC * kRing] = pfma(u2, gz, pfma(u1, gy, pmul(u0, gx)));
      cp[CF_AC * kRing] = pmul(c, psqrt2(pfma(gz, gz, pfma(gy, gy, pmul(gx, gx)))));
    };

    const int nch = (nd + 1 + S - 1) / S;
    if (okA) {
      if (tf - 1 < nd) prefetch_face(tf - 1, 0);
      cp_async_commit();
      const bool two = tf < 8;
      F2 Qa[5], ka[3], ija, Qb[5], kb[3], ijb;
      fetch(-5 + tf, Qa, ka, ija);
      if (two) fetch(-5 + tf + S, Qb, kb, ijb);
      stage_cell(-5 + tf, Qa, ka, ija);
      if (two) stage_cell(-5 + tf + S, Qb, kb, ijb);
    }
    cp_async_wait_all();
    __syncthreads();

    for (int ch = 0; ch < nch; ++ch) {
      const int a = ch * S - 1;
      const bool nextOK = okA && ch + 1 < nch;
      if (okA && a + tf >= 0 && a + tf < nd) prefetch_epilogue(a + tf);
      if (nextOK) prefetch_cell(a + S + 4 + tf);
      if (nextOK && a + S + tf < nd) prefetch_face(a + S + tf, (ch + 1) & 1);
      if (ch == 0 && nit < nitems) fetch_desc(cur ^ 1, s_item[cur ^ 1].x);
      cp_async_commit();
      const int ff = a + tf;
      if (okA && ff < nd) {
        const int i0 = ff;
        int o[8];
#pragma unroll
        for (int q = 0; q < 8; ++q) o[q] = off(i0 - 3 + q);
#define CELL2(field, q) sm[(field) * kRing + o[(q)]]
        F2 Qi[5];
#pragma unroll
        for (int v = 0; v < 5; ++v) Qi[v] = CELL2(CF_Q + v, 3);
        F2 kf[3];
#pragma unroll
        for (int c = 0; c < 3; ++c) kf[c] = nsb[(9 + 3 * (ch & 1) + c) * kThreads + tid];

        // reference face state Q* = Q_i + delta (Eqs. Q_star, QdJ_star, 1dJ at order M)
        F2 dl[5] = {pcf(0.f), pcf(0.f), pcf(0.f), pcf(0.f), pcf(0.f)};
        if (fpform) {
          F2 acc[5] = {pcf(0.f), pcf(0.f), pcf(0.f), pcf(0.f), pcf(0.f)};
          F2 wsum = pcf(0.f);
#pragma unroll
          for (int m = 0; m < M; ++m) {
            const int q = 3 - M / 2 + 1 + m;
            const F2 w = pmul(pcf(float(MidW<M>::w(m))), CELL2(CF_INVJ, q));
            wsum = padd(wsum, w);
            if (q != 3) {       // the face's own cell contributes w (Q_i - Q_i) = 0
#pragma unroll
              for (int v = 0; v < 5; ++v) acc[v] = pfma(w, psub(CELL2(CF_Q + v, q), Qi[v]), acc[v]);
            }
          }
          const F2 wi = prcp2(wsum);
#pragma unroll
          for (int v = 0; v < 5; ++v) dl[v] = pmul(acc[v], wi);
        }
        F2 Qs[5];
#pragma unroll
        for (int v = 0; v < 5; ++v) Qs[v] = padd(Qi[v], dl[v]);
        const F2 rinvs = prcp2(Qs[0]);
        const F2 us[3] = {pmul(Qs[1], rinvs), pmul(Qs[2], rinvs), pmul(Qs[3], rinvs)};
        const F2 ps = pmul(g1, pfma(pcf(-0.5f), pfma(Qs[3], us[2], pfma(Qs[2], us[1], pmul(Qs[1], us[0]))), Qs[4]));
        const F2 nus[3] = {pneg2(us[0]), pneg2(us[1]), pneg2(us[2])};
        const F2 ms[3] = {Qs[1], Qs[2], Qs[3]};
        const F2 Eps = padd(Qs[4], ps);

        // Lax-Friedrichs speeds: local (max over the stencil cells i-2..i+3) or global
        F2 lm = pcf(0.f), l0 = pcf(0.f), lp = pcf(0.f);
        if (glf) {
          lm = pcf(s_lam[0]); l0 = pcf(s_lam[1]); lp = pcf(s_lam[2]);
        } else {
#pragma unroll
          for (int q = 1; q < 1 + NS; ++q) {
            const F2 U = CELL2(CF_UC, q), ac = CELL2(CF_AC, q);
            lm = pmaxabs2(lm, psub(U, ac));
            l0 = pmaxabs2(l0, U);
            lp = pmaxabs2(lp, padd(U, ac));
          }
        }
        F2 lam[5];
        if (charwise) {
          lam[0] = lm; lam[1] = l0; lam[2] = l0; lam[3] = l0; lam[4] = lp;
        } else {
          const F2 lmax = make_float2(fmaxf(lm.x, lp.x), fmaxf(lm.y, lp.y));
          lam[0] = lam[1] = lam[2] = lam[3] = lam[4] = lmax;
        }

        // Roe average of cells i, i+1 and eigenvector basis in the face normal
        const F2 rl = CELL2(CF_SQR, 3), rr = CELL2(CF_SQR, 4);
        const F2 rs = prcp2(padd(rl, rr));
        F2 u[3];
#pragma unroll
        for (int c = 0; c < 3; ++c) u[c] = pmul(pfma(rr, CELL2(CF_U + c, 4), pmul(rl, CELL2(CF_U + c, 3))), rs);
        const F2 H = pmul(pfma(rr, CELL2(CF_H, 4), pmul(rl, CELL2(CF_H, 3))), rs);
        const F2 q2 = pfma(u[2], u[2], pfma(u[1], u[1], pmul(u[0], u[0])));
        const F2 c2 = pmul(g1, pfma(pcf(-0.5f), q2, H));
        const F2 cs = psqrt2(c2);
        const F2 csi = prcp2(cs);
        const F2 bb = pmul(g1, pmul(csi, csi));
        const F2 knr = prsqrt2(pfma(kf[2], kf[2], pfma(kf[1], kf[1], pmul(kf[0], kf[0]))));
        const F2 n[3] = {pmul(kf[0], knr), pmul(kf[1], knr), pmul(kf[2], knr)};
        // t1 = normalise(e_z x n) if n_z^2 <= 1/2, else normalise(n x e_x), per line
        const F2 nz2 = pmul(n[2], n[2]);
        const bool sa = nz2.x <= 0.5f, sb = nz2.y <= 0.5f;
        const F2 sA = prsqrt2(pfma(n[1], n[1], pmul(n[0], n[0])));
        const F2 sB = prsqrt2(pfma(n[2], n[2], pmul(n[1], n[1])));
        F2 t1[3], t2[3];
        t1[0] = psel2(sa, sb, pmul(pneg2(n[1]), sA), pcf(0.f));
        t1[1] = psel2(sa, sb, pmul(n[0], sA), pmul(n[2], sB));
        t1[2] = psel2(sa, sb, pcf(0.f), pmul(pneg2(n[1]), sB));
        t2[0] = psub(pmul(n[1], t1[2]), pmul(n[2], t1[1]));
        t2[1] = psub(pmul(n[2], t1[0]), pmul(n[0], t1[2]));
        t2[2] = psub(pmul(n[0], t1[1]), pmul(n[1], t1[0]));
        const F2 Un = pfma(u[2], n[2], pfma(u[1], n[1], pmul(u[0], n[0])));
        const F2 ut1 = pfma(u[2], t1[2], pfma(u[1], t1[1], pmul(u[0], t1[0])));
        const F2 ut2 = pfma(u[2], t2[2], pfma(u[1], t2[1], pmul(u[0], t2[0])));
        const F2 qbbv = pmul(pcf(0.25f), bb), hq2 = pmul(pcf(0.5f), q2), qcs = pmul(pcf(0.25f), csi);
        const F2 h1[3] = {pmul(pcf(0.5f), t1[0]), pmul(pcf(0.5f), t1[1]), pmul(pcf(0.5f), t1[2])};
        const F2 h2[3] = {pmul(pcf(0.5f), t2[0]), pmul(pcf(0.5f), t2[1]), pmul(pcf(0.5f), t2[2])};
        const F2 nhut1 = pmul(pcf(-0.5f), ut1), nhut2 = pmul(pcf(-0.5f), ut2);

        // (1/2) l_s . d for the five characteristic fields of both lines
        auto project = [&](const F2 d[5], F2 c[5]) {
          if (!charwise) {
#pragma unroll
            for (int v = 0; v < 5; ++v) c[v] = pmul(pcf(0.5f), d[v]);
            return;
          }
          const F2 ud = pfma(u[0], d[1], pfma(u[1], d[2], pmul(u[2], d[3])));
          const F2 X4 = pmul(qbbv, pfma(hq2, d[0], psub(d[4], ud)));
          const F2 nd_ = pfma(n[0], d[1], pfma(n[1], d[2], pmul(n[2], d[3])));
          const F2 Y4 = pmul(qcs, psub(pmul(Un, d[0]), nd_));
          c[0] = padd(X4, Y4);
          c[1] = pfma(pcf(-2.f), X4, pmul(pcf(0.5f), d[0]));
          c[2] = pfma(h1[0], d[1], pfma(h1[1], d[2], pfma(h1[2], d[3], pmul(nhut1, d[0]))));
          c[3] = pfma(h2[0], d[1], pfma(h2[1], d[2], pfma(h2[2], d[3], pmul(nhut2, d[0]))));
          c[4] = psub(X4, Y4);
        };

        // stencil differences of point s (cells i-2..i+3): dF = (F(Q_s) - F(Q*)) . k_s and
        // dQ = Q_s - Q*, or F~_s and Q_s for the plain scheme
        auto stencil = [&](int s, F2 dp[5], F2 out[5]) {
          const int q = s + 1;
          F2 kq[3], uq[3];
#pragma unroll
          for (int c = 0; c < 3; ++c) {
            kq[c] = CELL2(CF_K + c, q);
            uq[c] = CELL2(CF_U + c, q);
          }
          if (fpform) {
#pragma unroll
            for (int v = 0; v < 5; ++v) dp[v] = psub(psub(CELL2(CF_Q + v, q), Qi[v]), dl[v]);
            dflux2(g1, CELL2(CF_RINV, q), uq, nus, ms, Eps, dp, kq, out);
          } else {
#pragma unroll
            for (int v = 0; v < 5; ++v) dp[v] = CELL2(CF_Q + v, q);
            const F2 ke = pfma(dp[3], uq[2], pfma(dp[2], uq[1], pmul(dp[1], uq[0])));
            const F2 pm = pmul(g1, pfma(pcf(-0.5f), ke, dp[4]));
            const F2 U = pfma(uq[2], kq[2], pfma(uq[1], kq[1], pmul(uq[0], kq[0])));
            out[0] = pmul(dp[0], U);
#pragma unroll
            for (int c = 0; c < 3; ++c) out[1 + c] = pfma(pm, kq[c], pmul(dp[1 + c], U));
            out[4] = pmul(padd(dp[4], pm), U);
          }
        };

        F2 h[5], cen[5];
        if constexpr (SCHEME == 1) {
          // linear upwind: C6(dF) + R Lambda L D(dQ~) (see fp_sweep)
          constexpr float c6[6] = {1.f / 60.f, -8.f / 60.f, 37.f / 60.f, 37.f / 60.f, -8.f / 60.f, 1.f / 60.f};
          constexpr float d5[6] = {1.f / 60.f, -5.f / 60.f, 10.f / 60.f, -10.f / 60.f, 5.f / 60.f, -1.f / 60.f};
          F2 dis[5];
#pragma unroll
          for (int v = 0; v < 5; ++v) cen[v] = dis[v] = pcf(0.f);
#pragma unroll
          for (int s = 0; s < NS; ++s) {
            F2 dp[5], out[5];
            stencil(s, dp, out);
            const F2 ij = CELL2(CF_INVJ, s + 1);
#pragma unroll
            for (int v = 0; v < 5; ++v) {
              cen[v] = pfma(pcf(c6[s]), out[v], cen[v]);
              dis[v] = pfma(pcf(d5[s]), pmul(dp[v], ij), dis[v]);
            }
          }
          F2 c[5];
          project(dis, c);
#pragma unroll
          for (int v = 0; v < 5; ++v) h[v] = pmul(pmul(pcf(2.f), lam[v]), c[v]);
        } else {
          // WENO5-JS: f+- = (1/2) l . (dF +- lambda dQ (1/J)_s) for the six stencil points,
          // reconstructed from both sides (the - side mirrored)
          F2 fpl[NS][5], fmi[NS][5];
#pragma unroll
          for (int s = 0; s < NS; ++s) {
            F2 dp[5], out[5], cF[5], cD[5];
            stencil(s, dp, out);
            project(out, cF);
            project(dp, cD);
            const F2 ij = CELL2(CF_INVJ, s + 1);
            const F2 mu0 = pmul(lam[0], ij), mu1 = pmul(lam[1], ij), mu4 = pmul(lam[4], ij);
#pragma unroll
            for (int v = 0; v < 5; ++v) {
              const F2 mv = v == 0 ? mu0 : (v == 4 ? mu4 : mu1);
              fpl[s][v] = pfma(mv, cD[v], cF[v]);
              fmi[s][v] = pfma(pneg2(mv), cD[v], cF[v]);
            }
          }
#pragma unroll
          for (int v = 0; v < 5; ++v) {
            const F2 rp = recon5_pair<float, 0>(fpl[0][v], fpl[1][v], fpl[2][v], fpl[3][v], fpl[4][v]);
            const F2 rm = recon5_pair<float, 0>(fmi[5][v], fmi[4][v], fmi[3][v], fmi[2][v], fmi[1][v]);
            h[v] = padd(rp, rm);
            cen[v] = pcf(0.f);
          }
        }
#undef CELL2
        F2 Fl[5];
        if (charwise) {
          const F2 sa2 = padd(h[0], h[4]), da = psub(h[4], h[0]);
          const F2 sah = padd(sa2, h[1]);
          Fl[0] = sah;
#pragma unroll
          for (int c = 0; c < 3; ++c)
            Fl[1 + c] = pfma(t2[c], h[3], pfma(t1[c], h[2], pfma(pmul(cs, n[c]), da, pmul(u[c], sah))));
          Fl[4] = pfma(ut2, h[3], pfma(ut1, h[2], pfma(pmul(pcf(0.5f), q2), h[1], pfma(pmul(cs, Un), da, pmul(H, sa2)))));
        } else {
#pragma unroll
          for (int v = 0; v < 5; ++v) Fl[v] = h[v];
        }
        F2 *fp = fr + off(ff);
#pragma unroll
        for (int v = 0; v < 5; ++v) {
          if constexpr (SCHEME == 1) Fl[v] = padd(Fl[v], cen[v]);
          fp[v * kRing] = Fl[v];
          fp[(5 + v) * kRing] = dl[v];
        }
      }
      cp_async_wait_all();
      __syncthreads();
      // ---- residual of cell x = a + tf from its two faces, then the epilogue
      const int x = a + tf;
      if (okA && x >= 0 && x < nd) {
        const int ox = off(x), oxm = off(x - 1);
        F2 R[5];
#pragma unroll
        for (int v = 0; v < 5; ++v) R[v] = psub(fr[v * kRing + ox], fr[v * kRing + oxm]);
        if (fpform) {
          F2 Qp[5], Qm[5], dQ[5], dqm[5];
#pragma unroll
          for (int v = 0; v < 5; ++v) {
            const F2 qx = sm[(CF_Q + v) * kRing + ox], qx1 = sm[(CF_Q + v) * kRing + oxm];
            const F2 dp = fr[(5 + v) * kRing + ox], dm = fr[(5 + v) * kRing + oxm];
            Qp[v] = padd(qx, dp);
            Qm[v] = padd(qx1, dm);
            dQ[v] = padd(psub(qx, qx1), psub(dp, dm));
            dqm[v] = padd(psub(qx1, qb[v]), dm);
          }
          const F2 rA = prcp2(Qm[0]);
          const F2 uA[3] = {pmul(Qm[1], rA), pmul(Qm[2], rA), pmul(Qm[3], rA)};
          const F2 pA = pmul(g1, pfma(pcf(-0.5f), pfma(Qm[3], uA[2], pfma(Qm[2], uA[1], pmul(Qm[1], uA[0]))), Qm[4]));
          const F2 nuA[3] = {pneg2(uA[0]), pneg2(uA[1]), pneg2(uA[2])};
          const F2 mA[3] = {Qm[1], Qm[2], Qm[3]};
          const F2 rB = prcp2(Qp[0]);
          const F2 uBp[3] = {pmul(Qp[1], rB), pmul(Qp[2], rB), pmul(Qp[3], rB)};
          F2 kp[3], dk[3];
#pragma unroll
          for (int c = 0; c < 3; ++c) {
            dk[c] = epb[(10 + c) * kThreads + tid];
            kp[c] = nsb[(9 + 3 * (ch & 1) + c) * kThreads + tid];
          }
          F2 t1v[5], t2v[5];
          dflux2(g1, rB, uBp, nuA, mA, padd(Qm[4], pA), dQ, kp, t1v);     // [F(Q*_+) - F(Q*_-)] . k_+
          dflux2(g1, rA, uA, nub, mbq, Epb, dqm, dk, t2v);                 // [F(Q*_-) - F(Qbar)] . (k_+ - k_-)
#pragma unroll
          for (int v = 0; v < 5; ++v) R[v] = padd(R[v], padd(t1v[v], t2v[v]));
        }
        const long long qa = qba + (long long)x * qsd, qbo = qbb + (long long)x * qsd;
        float *racc = static_cast<float *>(B->racc);
        const F2 *ra = epb + tid;
        auto store2 = [&](float *base, int v, F2 val) {
          base[qa + v * qc] = val.x;
          if (okB) base[qbo + v * qc] = val.y;
        };
        if (mode == MODE_WRITE) {
#pragma unroll
          for (int v = 0; v < 5; ++v) store2(racc, v, R[v]);
        } else if (mode == MODE_ADD) {
#pragma unroll
          for (int v = 0; v < 5; ++v) store2(racc, v, padd(ra[v * kThreads], R[v]));
        } else {
          const F2 nJc = pneg2(prcp2(sm[CF_INVJ * kRing + ox]));
          if (mode == MODE_RHS) {
            float *out = static_cast<float *>(B->dqdt);
#pragma unroll
            for (int v = 0; v < 5; ++v) store2(out, v, pmul(nJc, padd(ra[v * kThreads], R[v])));
          } else {
            // SSP-RK3 stage in increment form (as fp_sweep)
            const float dt = s_dt;
            const float as = stage == 0 ? 0.f : (stage == 1 ? 0.75f : 1.f / 3.f);
            const float bs = stage == 0 ? 1.f : (stage == 1 ? 0.25f : 2.f / 3.f);
            float *qo_p = static_cast<float *>(B->q[(stage + 1) % 3]);
            const F2 bdt = pcf(bs * dt);
            bool bad = false;
#pragma unroll
            for (int v = 0; v < 5; ++v) {
              const F2 qk = sm[(CF_Q + v) * kRing + ox];
              const F2 Lv = pmul(nJc, padd(ra[v * kThreads], R[v]));
              F2 nv = pfma(bdt, Lv, qk);
              if (stage != 0) nv = pfma(bdt, Lv, pfma(pcf(as), psub(ra[(5 + v) * kThreads], qk), qk));
              store2(qo_p, v, nv);
              bad |= !isfinite(nv.x) || (okB && !isfinite(nv.y));
            }
            if (bad) atomicOr(B->status, 1);
          }
        }
      }
      __syncthreads();
      // ---- stage the next chunk's new cell pair from this thread's staging slots
      if (nextOK) {
        const int xs = a + S + 4 + tf;
        const F2 *src = nsb + tid;
        const F2 Q[5] = {src[0], src[kThreads], src[2 * kThreads], src[3 * kThreads], src[4 * kThreads]};
        const F2 k[3] = {src[5 * kThreads], src[6 * kThreads], src[7 * kThreads]};
        stage_cell(xs, Q, k, src[8 * kThreads]);
      }
      __syncthreads();
    }
  }
}

template <int M, int SCHEME>
cudaError_t launch_one2(const SweepLaunch &L, int charwise, int fp, cudaStream_t s) {
  if (L.nitems <= 0) return cudaSuccess;
  fp_sweep2<M, SCHEME><<<L.grid, kThreads, kSweep2Smem, s>>>(L.blocks, L.items, L.nitems, L.dir, L.mode, L.stage,
                                                              L.dt, charwise, fp);
  return cudaGetLastError();
}

}  // namespace fpk
