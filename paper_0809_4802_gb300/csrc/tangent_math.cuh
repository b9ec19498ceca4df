// Consistent Newton tangent of one element and its Schur condensation (Section 4.2 Eq.
// NewtonUpdate2; Section 5 Eq. SchurUpdate), computed by one warp.
//
// The paper defers the element matrices to a companion paper; these blocks are the exact
// derivatives of the residuals of Section 4.1 with respect to the nodal velocities vhat_{b,k},
// nodal pressures phat_b and bubble coefficients beta_k (c_b = v.g_b, c_d = v.d, nut = 2 nu):
//   K_vv[(a,i),(b,k)] = int N_a (N_b L_ik + d_ik c_b) + nut d_ik g_a.g_b + tau d_ik N_a N_b
//   K_vp[(a,i),b] = -int g_ai N_b        K_pv[a,(b,k)] = -int N_a g_bk        K_pp = 0
//   K_vf[(a,i),k] = int N_a (b L_ik + d_ik c_d) + nut d_ik g_a.d
//   K_pf[a,k]     = -int N_a d_k
//   K_fv[i,(b,k)] = int b (N_b L_ik + d_ik c_b) + nut d_ik d.g_b + tau d_ik b N_b
//   K_fp[i,b]     = -int d_i N_b
//   K_ff[i,k]     = int b (b L_ik + d_ik c_d) + nut d_ik d.d
// The transient term acts on the coarse velocity only (Remark, Section 4.1), hence no tau in
// K_vf and K_ff.
//
// Work split inside the warp (lane L = 0..31):
//   phase 1: lane q evaluates geometry and fields at quadrature point q and stores per-point
//            coefficients in shared memory as 4-vectors (up to 32 points per pass);
//   phase 2: lane L accumulates the 4x4 coarse blocks of the node pairs (L>>3, L&7) and
//            (4 + (L>>3), L&7) as packed pairs (one packed FMA serves both blocks), row L of K_cf
//            and column L of K_fc;
//   phase 3: K_ff is reduced and inverted in FP64, and S_e = K_cc - K_cf K_ff^-1 K_fc is formed.
// T is the tangent arithmetic type (double in FP64 mode, float in mixed mode).
#pragma once

#include <cmath>
#include <cstring>

#include <vector_functions.h>
#include <vector_types.h>

#include "element_math.cuh"

namespace vms {

template <typename T>
struct alignas(4 * sizeof(T)) Vec4 {
  T x, y, z, w;
};

// Packed pairs: the lane's two node-pair blocks side by side.
template <typename T> struct PairOf;
template <> struct PairOf<float> { using type = float2; };
template <> struct PairOf<double> { using type = double2; };

VMS_HD float2 pk(float a, float b) { return make_float2(a, b); }
VMS_HD double2 pk(double a, double b) { return make_double2(a, b); }
VMS_HD float2 pfma(float2 a, float2 b, float2 c) {
#ifdef __CUDA_ARCH__
  return __ffma2_rn(a, b, c);
#else
  return make_float2(a.x * b.x + c.x, a.y * b.y + c.y);
#endif
}
VMS_HD double2 pfma(double2 a, double2 b, double2 c) {
  return make_double2(a.x * b.x + c.x, a.y * b.y + c.y);
}
VMS_HD float2 pmul(float2 a, float2 b) {
#ifdef __CUDA_ARCH__
  return __fmul2_rn(a, b);
#else
  return make_float2(a.x * b.x, a.y * b.y);
#endif
}
VMS_HD double2 pmul(double2 a, double2 b) { return make_double2(a.x * b.x, a.y * b.y); }
VMS_HD float2 padd(float2 a, float2 b) {
#ifdef __CUDA_ARCH__
  return __fadd2_rn(a, b);
#else
  return make_float2(a.x + b.x, a.y + b.y);
#endif
}
VMS_HD double2 padd(double2 a, double2 b) { return make_double2(a.x + b.x, a.y + b.y); }

// Per-quadrature-point coefficients (29 four-vectors).
template <typename T>
struct QpRec {
  Vec4<T> g[8];    // (dN_a/dx_j for j = 0..2, N_a)
  Vec4<T> gw[8];   // (omega dN_a/dx_j, omega (v.g_a) + tau omega N_a)
  Vec4<T> L[3];    // rows of L[i][j] = dv_i/dx_j (4th entry: omega)
  Vec4<T> Ycf[4];  // row c: K_cf coefficient of N_a for dof c
  Vec4<T> Yfc[4];  // row c: K_fc coefficient of N_b for dof c
  Vec4<T> Dv;      // nut omega d
  Vec4<T> Wv;      // omega b v + nut omega d
};

// Reference tables of one Gauss rule in type T.
template <typename T>
struct RefTab {
  const T* N;   // [nq][8]
  const T* dN;  // [nq][24] (a*3+al)
  const T* b;   // [nq]
  const T* db;  // [nq][3]
  const T* w;   // [nq]
};

// Shared memory of one warp (qp[] is sized at launch: min(nq, 32) records follow).
template <typename T>
struct WarpArea {
  T X[8][3];
  T V[8][3];
  T beta[3];
  int nd[8];
  T kffp[32][9];
  T Kcf[32][3];
  T Xs[3][32];     // X = K_ff^-1 K_fc rounded to T
  T Xl[3][32];     // X - Xs (its low part in T; zero in FP64)
  double Kff[9];
  double cof[9];
  double Kinv[9];
  T KffT[9];       // K_ff summed in T (before widening)
  T KinvT[9];
  unsigned int flag;
  QpRec<T> qp[1];
};

// Registers of one lane across the phases: K[i*4+k] holds entry (i,k) of the blocks (a0,b) in .x
// and (a1,b) in .y; index 3 is the pressure dof.
template <typename T>
struct LaneAcc {
  typename PairOf<T>::type K[16];
  T kcf[3], kfc[3], kff[9];
};

template <typename T>
VMS_HD void tan_zero(LaneAcc<T>& A) {
  VMS_UNROLL
  for (int i = 0; i < 16; ++i) A.K[i] = pk(T(0), T(0));
  VMS_UNROLL
  for (int i = 0; i < 3; ++i) { A.kcf[i] = T(0); A.kfc[i] = T(0); }
  VMS_UNROLL
  for (int i = 0; i < 9; ++i) A.kff[i] = T(0);
}

// Phase 1 for lane `lane`: quadrature point q = q0 + lane (if < nq).
template <typename T>
VMS_HD void tan_phase1(int lane, int q0, int nq, WarpArea<T>& W, const RefTab<T>& tab, T nut,
                       T tau, LaneAcc<T>& A) {
  const int q = q0 + lane;
  if (q >= nq) return;
  const T* dN = tab.dN + 24 * q;
  const T* N = tab.N + 8 * q;
  const T bq = tab.b[q];
  const T db[3] = {tab.db[3 * q], tab.db[3 * q + 1], tab.db[3 * q + 2]};
  T J[3][3];
  VMS_UNROLL
  for (int i = 0; i < 3; ++i)
    VMS_UNROLL
    for (int al = 0; al < 3; ++al) {
      T s = T(0);
      VMS_UNROLL
      for (int a = 0; a < 8; ++a) s += W.X[a][i] * dN[3 * a + al];
      J[i][al] = s;
    }
  T cof[3][3];
  T det = cofactor3(J, cof);
  if (!(det > T(0))) { W.flag = 1u; det = T(1); }
  const T rdet = T(1) / det;
  T Ji[3][3];  // Ji[al][j] = (J^-1)[al][j] = cof[j][al] / det
  VMS_UNROLL
  for (int al = 0; al < 3; ++al)
    VMS_UNROLL
    for (int j = 0; j < 3; ++j) Ji[al][j] = cof[j][al] * rdet;
  QpRec<T>& R = W.qp[lane];
  const T om = tab.w[q] * det;
  T g[8][3];
  VMS_UNROLL
  for (int a = 0; a < 8; ++a)
    VMS_UNROLL
    for (int j = 0; j < 3; ++j)
      g[a][j] = dN[3 * a] * Ji[0][j] + dN[3 * a + 1] * Ji[1][j] + dN[3 * a + 2] * Ji[2][j];
  T d[3];
  VMS_UNROLL
  for (int j = 0; j < 3; ++j) d[j] = db[0] * Ji[0][j] + db[1] * Ji[1][j] + db[2] * Ji[2][j];
  T v[3], L[3][3];
  VMS_UNROLL
  for (int i = 0; i < 3; ++i) {
    T s = T(0);
    VMS_UNROLL
    for (int a = 0; a < 8; ++a) s += N[a] * W.V[a][i];
    v[i] = s + bq * W.beta[i];
    VMS_UNROLL
    for (int j = 0; j < 3; ++j) {
      T t = W.beta[i] * d[j];
      VMS_UNROLL
      for (int a = 0; a < 8; ++a) t += W.V[a][i] * g[a][j];
      L[i][j] = t;
    }
  }
  VMS_UNROLL
  for (int a = 0; a < 8; ++a) {
    const T cb = v[0] * g[a][0] + v[1] * g[a][1] + v[2] * g[a][2];
    R.g[a] = Vec4<T>{g[a][0], g[a][1], g[a][2], N[a]};
    R.gw[a] = Vec4<T>{om * g[a][0], om * g[a][1], om * g[a][2], om * (cb + tau * N[a])};
  }
  VMS_UNROLL
  for (int i = 0; i < 3; ++i) R.L[i] = Vec4<T>{L[i][0], L[i][1], L[i][2], om};
  const T cd = v[0] * d[0] + v[1] * d[1] + v[2] * d[2];
  const T dd = d[0] * d[0] + d[1] * d[1] + d[2] * d[2];
  const T omb = om * bq;
  VMS_UNROLL
  for (int c = 0; c < 3; ++c) {
    R.Ycf[c] = Vec4<T>{omb * L[c][0] + (c == 0 ? om * cd : T(0)),
                       omb * L[c][1] + (c == 1 ? om * cd : T(0)),
                       omb * L[c][2] + (c == 2 ? om * cd : T(0)), T(0)};
    R.Yfc[c] = Vec4<T>{omb * (L[0][c] + (c == 0 ? tau : T(0))),
                       omb * (L[1][c] + (c == 1 ? tau : T(0))),
                       omb * (L[2][c] + (c == 2 ? tau : T(0))), T(0)};
  }
  R.Ycf[3] = Vec4<T>{-om * d[0], -om * d[1], -om * d[2], T(0)};
  R.Yfc[3] = R.Ycf[3];
  R.Dv = Vec4<T>{nut * om * d[0], nut * om * d[1], nut * om * d[2], T(0)};
  R.Wv = Vec4<T>{omb * v[0] + R.Dv.x, omb * v[1] + R.Dv.y, omb * v[2] + R.Dv.z, T(0)};
  VMS_UNROLL
  for (int i = 0; i < 3; ++i)
    VMS_UNROLL
    for (int k = 0; k < 3; ++k)
      A.kff[3 * i + k] += om * (bq * (bq * L[i][k] + (i == k ? cd : T(0))) + (i == k ? nut * dd : T(0)));
}

// Phase 2 for lane `lane`: accumulate over the nqc points stored by phase 1.
template <typename T>
VMS_HD void tan_phase2(int lane, int nqc, const WarpArea<T>& W, T nut, LaneAcc<T>& A) {
  using P = typename PairOf<T>::type;
  const int a0 = lane >> 3, a1 = a0 + 4, b = lane & 7;
  const int at = lane >> 2, ct = lane & 3;
  // Kronecker masks of the lane's dof ct (constant per lane, so no per-point selects)
  const T m0 = ct == 0 ? T(1) : T(0), m1 = ct == 1 ? T(1) : T(0), m2 = ct == 2 ? T(1) : T(0);
  for (int qq = 0; qq < nqc; ++qq) {
    const QpRec<T>& Q = W.qp[qq];
    const Vec4<T> gb = Q.g[b], gwb = Q.gw[b];
    const Vec4<T> g0 = Q.g[a0], g1 = Q.g[a1];
    const Vec4<T> w0 = Q.gw[a0], w1 = Q.gw[a1];
    const Vec4<T> L0 = Q.L[0], L1 = Q.L[1], L2 = Q.L[2];
    const T wNb = L0.w * gb.w;                 // omega N_b
    const P Na = pk(g0.w, g1.w);               // (N_a0, N_a1)
    const P m = pmul(Na, pk(wNb, wNb));        // omega N_a N_b
    // s = N_a (omega c_b + tau omega N_b) + nut g_a . (omega g_b)
    P dot = pmul(pk(g0.x, g1.x), pk(gwb.x, gwb.x));
    dot = pfma(pk(g0.y, g1.y), pk(gwb.y, gwb.y), dot);
    dot = pfma(pk(g0.z, g1.z), pk(gwb.z, gwb.z), dot);
    const P s = pfma(pk(nut, nut), dot, pmul(Na, pk(gwb.w, gwb.w)));
    const T Lr[9] = {L0.x, L0.y, L0.z, L1.x, L1.y, L1.z, L2.x, L2.y, L2.z};
    VMS_UNROLL
    for (int i = 0; i < 3; ++i) {
      VMS_UNROLL
      for (int k = 0; k < 3; ++k) A.K[4 * i + k] = pfma(m, pk(Lr[3 * i + k], Lr[3 * i + k]), A.K[4 * i + k]);
      A.K[5 * i] = padd(A.K[5 * i], s);
    }
    // K_vp: -omega g_ai N_b; K_pv: -N_a omega g_bk
    const T nNb = -gb.w;
    A.K[3] = pfma(pk(w0.x, w1.x), pk(nNb, nNb), A.K[3]);
    A.K[7] = pfma(pk(w0.y, w1.y), pk(nNb, nNb), A.K[7]);
    A.K[11] = pfma(pk(w0.z, w1.z), pk(nNb, nNb), A.K[11]);
    const P nNa = pk(-g0.w, -g1.w);
    A.K[12] = pfma(nNa, pk(gwb.x, gwb.x), A.K[12]);
    A.K[13] = pfma(nNa, pk(gwb.y, gwb.y), A.K[13]);
    A.K[14] = pfma(nNa, pk(gwb.z, gwb.z), A.K[14]);
    // row L of K_cf and column L of K_fc (node at, dof ct)
    const Vec4<T> gt = Q.g[at];
    const Vec4<T> yc = Q.Ycf[ct], yf = Q.Yfc[ct], dv = Q.Dv, wv = Q.Wv;
    const T gdv = gt.x * dv.x + gt.y * dv.y + gt.z * dv.z;
    const T gwv = gt.x * wv.x + gt.y * wv.y + gt.z * wv.z;
    if constexpr (sizeof(T) == 4) {
      // FP32: multiply by the 0/1 masks (cheaper than a select on the FMA pipe)
      A.kcf[0] += gt.w * yc.x + m0 * gdv;
      A.kcf[1] += gt.w * yc.y + m1 * gdv;
      A.kcf[2] += gt.w * yc.z + m2 * gdv;
      A.kfc[0] += gt.w * yf.x + m0 * gwv;
      A.kfc[1] += gt.w * yf.y + m1 * gwv;
      A.kfc[2] += gt.w * yf.z + m2 * gwv;
    } else {
      // FP64: selects run on the integer pipe, multiplies would take FP64 slots
      A.kcf[0] += gt.w * yc.x + (ct == 0 ? gdv : T(0));
      A.kcf[1] += gt.w * yc.y + (ct == 1 ? gdv : T(0));
      A.kcf[2] += gt.w * yc.z + (ct == 2 ? gdv : T(0));
      A.kfc[0] += gt.w * yf.x + (ct == 0 ? gwv : T(0));
      A.kfc[1] += gt.w * yf.y + (ct == 1 ? gwv : T(0));
      A.kfc[2] += gt.w * yf.z + (ct == 2 ? gwv : T(0));
    }
  }
}

// Phase 3a: publish the lane's K_ff partial sums.
template <typename T>
VMS_HD void tan_phase3a(int lane, WarpArea<T>& W, const LaneAcc<T>& A) {
  VMS_UNROLL
  for (int j = 0; j < 9; ++j) W.kffp[lane][j] = A.kff[j];
}

// Phase 3b: lanes 0..8 sum one K_ff entry each over the 32 partials (in T), then widen to FP64.
template <typename T>
VMS_HD void tan_phase3b(int lane, WarpArea<T>& W) {
  if (lane < 9) {
    T s = T(0);
    for (int l = 0; l < 32; ++l) s += W.kffp[l][lane];
    W.KffT[lane] = s;
    W.Kff[lane] = (double)s;
  }
}

// Phase 3c: lanes 0..8 each form one cofactor of K_ff (FP64).
template <typename T>
VMS_HD void tan_phase3c(int lane, WarpArea<T>& W) {
  if (lane < 9) {
    const int i = lane / 3, j = lane % 3;
    const int i1 = (i + 1) % 3, i2 = (i + 2) % 3, j1 = (j + 1) % 3, j2 = (j + 2) % 3;
    W.cof[lane] = W.Kff[3 * i1 + j1] * W.Kff[3 * i2 + j2] - W.Kff[3 * i1 + j2] * W.Kff[3 * i2 + j1];
  }
}

// Phase 3d: determinant and one reciprocal (every lane, FP64), then lanes 0..8 write one entry of
// K_ff^-1 = cof^T / det in FP64 and in T. A singular or non-finite K_ff raises flag bit 2.
template <typename T>
VMS_HD void tan_phase3d(int lane, WarpArea<T>& W) {
  const double det = W.Kff[0] * W.cof[0] + W.Kff[1] * W.cof[1] + W.Kff[2] * W.cof[2];
  // zero or not finite, tested on the bits (an FP64 compare takes a whole FP64 issue slot)
  uint64_t db;
  memcpy(&db, &det, sizeof db);
  const bool bad = (db << 1) == 0 || ((db >> 52) & 0x7ffu) == 0x7ffu;
  const double r = bad ? 0.0 : recip(det);
  if (lane < 9) {
    const double v = W.cof[3 * (lane % 3) + lane / 3] * r;
    W.Kinv[lane] = v;
    W.KinvT[lane] = T(v);
  }
  if (bad && lane == 0) W.flag |= 2u;
}

// Infinity-norm condition number of K_ff, in T, from the sums before widening and the inverse
// rounded to T. It only chooses between two correct condensation paths (in FP32 the choice may
// differ from an FP64 estimate only within rounding of the threshold), and in FP32 it takes no
// FP64 issue slot.
template <typename T>
VMS_HD T kff_cond_inf(const WarpArea<T>& W) {
  T nk = T(0), ni = T(0);
  VMS_UNROLL
  for (int i = 0; i < 3; ++i) {
    nk = fmax(nk, fabs(W.KffT[3 * i]) + fabs(W.KffT[3 * i + 1]) + fabs(W.KffT[3 * i + 2]));
    ni = fmax(ni, fabs(W.KinvT[3 * i]) + fabs(W.KinvT[3 * i + 1]) + fabs(W.KinvT[3 * i + 2]));
  }
  return nk * ni;
}

// Phase 3f: column L of X = K_ff^-1 K_fc and row L of K_cf, to shared memory. In FP32 with
// `accurate` (an ill-conditioned K_ff) X is formed in FP64 from the FP64 inverse and kept as a high
// and a low part in T; otherwise it is formed in T (Xl = 0).
template <typename T>
VMS_HD void tan_phase3f(int lane, WarpArea<T>& W, const LaneAcc<T>& A, bool accurate) {
  if (sizeof(T) == 8 || accurate) {
    const double f0 = (double)A.kfc[0], f1 = (double)A.kfc[1], f2 = (double)A.kfc[2];
    VMS_UNROLL
    for (int m = 0; m < 3; ++m) {
      const double x = W.Kinv[3 * m] * f0 + W.Kinv[3 * m + 1] * f1 + W.Kinv[3 * m + 2] * f2;
      const T xh = T(x);
      W.Xs[m][lane] = xh;
      W.Xl[m][lane] = T(x - (double)xh);
      W.Kcf[lane][m] = A.kcf[m];
    }
  } else {
    VMS_UNROLL
    for (int m = 0; m < 3; ++m) {
      W.Xs[m][lane] = W.KinvT[3 * m] * A.kfc[0] + W.KinvT[3 * m + 1] * A.kfc[1] +
                      W.KinvT[3 * m + 2] * A.kfc[2];
      W.Xl[m][lane] = T(0);
      W.Kcf[lane][m] = A.kcf[m];
    }
  }
}

#if defined(__CUDACC__)
// s + sum_m c_m (xh_m + xl_m) in FP32 with the rounding error of every product (exact by FMA) and
// of every addition (two-sum) carried in a compensation term (compensated dot product). The
// condensation subtracts K_cf X from K_cc, and on convection-dominated elements the terms are up to
// ~10^3 times larger than the result, so plain FP32 would lose three digits of S_e.
__device__ __forceinline__ float comp_dot3(float s, const float c[3], const float xh[3],
                                           const float xl[3]) {
  float comp = 0.f;
  VMS_UNROLL
  for (int m = 0; m < 3; ++m) {
    const float p = __fmul_rn(c[m], xh[m]);
    const float e = __fmaf_rn(c[m], xh[m], -p);
    const float t = __fadd_rn(s, p);
    const float bb = __fsub_rn(t, s);
    const float err = __fadd_rn(__fsub_rn(s, __fsub_rn(t, bb)), __fsub_rn(p, bb));
    comp = __fadd_rn(comp, __fadd_rn(err, e));
    comp = __fmaf_rn(c[m], xl[m], comp);
    s = t;
  }
  return __fadd_rn(s, comp);
}
#endif

// Phase 3e: S blocks of the lane's two node pairs, in place: K -= K_cf X (FP32 with `accurate`:
// compensated, with X = Xs + Xl; otherwise plain FMA with X = Xs, and Xs + Xl in FP64).
template <typename T>
VMS_HD void tan_phase3e(int lane, const WarpArea<T>& W, LaneAcc<T>& A, bool accurate) {
  const int a0 = lane >> 3, a1 = a0 + 4, b = lane & 7;
#if defined(__CUDA_ARCH__)
  if (sizeof(T) == 4 && accurate) {
    VMS_UNROLL
    for (int i = 0; i < 4; ++i) {
      const float ca[3] = {(float)-W.Kcf[4 * a0 + i][0], (float)-W.Kcf[4 * a0 + i][1],
                           (float)-W.Kcf[4 * a0 + i][2]};
      const float cb[3] = {(float)-W.Kcf[4 * a1 + i][0], (float)-W.Kcf[4 * a1 + i][1],
                           (float)-W.Kcf[4 * a1 + i][2]};
      VMS_UNROLL
      for (int k = 0; k < 4; ++k) {
        const float xh[3] = {(float)W.Xs[0][4 * b + k], (float)W.Xs[1][4 * b + k],
                             (float)W.Xs[2][4 * b + k]};
        const float xl[3] = {(float)W.Xl[0][4 * b + k], (float)W.Xl[1][4 * b + k],
                             (float)W.Xl[2][4 * b + k]};
        auto acc = A.K[4 * i + k];
        acc.x = comp_dot3((float)acc.x, ca, xh, xl);
        acc.y = comp_dot3((float)acc.y, cb, xh, xl);
        A.K[4 * i + k] = acc;
      }
    }
    return;
  }
#endif
  VMS_UNROLL
  for (int i = 0; i < 4; ++i) {
    const auto c0 = pk(-W.Kcf[4 * a0 + i][0], -W.Kcf[4 * a1 + i][0]);
    const auto c1 = pk(-W.Kcf[4 * a0 + i][1], -W.Kcf[4 * a1 + i][1]);
    const auto c2 = pk(-W.Kcf[4 * a0 + i][2], -W.Kcf[4 * a1 + i][2]);
    VMS_UNROLL
    for (int k = 0; k < 4; ++k) {
      const T x0 = sizeof(T) == 8 ? W.Xs[0][4 * b + k] + W.Xl[0][4 * b + k] : W.Xs[0][4 * b + k];
      const T x1 = sizeof(T) == 8 ? W.Xs[1][4 * b + k] + W.Xl[1][4 * b + k] : W.Xs[1][4 * b + k];
      const T x2 = sizeof(T) == 8 ? W.Xs[2][4 * b + k] + W.Xl[2][4 * b + k] : W.Xs[2][4 * b + k];
      auto acc = A.K[4 * i + k];
      acc = pfma(c0, pk(x0, x0), acc);
      acc = pfma(c1, pk(x1, x1), acc);
      acc = pfma(c2, pk(x2, x2), acc);
      A.K[4 * i + k] = acc;
    }
  }
}

}  // namespace vms
