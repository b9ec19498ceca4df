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
//            coefficients in shared memory (up to 32 points per pass);
//   phase 2: lane L accumulates the 4x4 coarse blocks of the node pairs (L>>3, L&7) and
//            (4 + (L>>3), L&7), row L of K_cf and column L of K_fc;
//   phase 3: K_ff is reduced, inverted in FP64, and S_e = K_cc - K_cf K_ff^-1 K_fc and
//            r_e = R_cp - K_cf K_ff^-1 R_f are formed (r_e in FP64).
// T is the tangent arithmetic type (double in FP64 mode, float in mixed mode).
#pragma once

#include "element_math.cuh"

namespace vms {

// Per-quadrature-point coefficients (73 entries: an odd stride keeps lane-indexed rows on
// distinct shared-memory banks).
template <typename T>
struct QpRec {
  T w;        // omega = w_q det J
  T g[24];    // g[a*3+j] = dN_a/dx_j
  T L[9];     // L[i*3+j] = dv_i/dx_j
  T cb[8];    // v . g_b
  T Ycf[12];  // [c*3+k]: K_cf row coefficient of N_a
  T Yfc[12];  // [c*3+i]: K_fc column coefficient of N_b
  T Dv[3];    // nut omega d
  T Wv[3];    // omega b v + nut omega d
  T pad;
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
  T Xs[3][32];
  double Kff[9];
  double cof[9];
  double Kinv[9];
  T KinvT[9];
  unsigned int flag;
  QpRec<T> qp[1];
};

// Registers of one lane across the phases.
template <typename T>
struct LaneAcc {
  T K0[16], K1[16];  // pair blocks [i*4+k], index 3 = pressure
  T kcf[3], kfc[3], kff[9];
};

template <typename T>
VMS_HD void tan_zero(LaneAcc<T>& A) {
  VMS_UNROLL
  for (int i = 0; i < 16; ++i) { A.K0[i] = T(0); A.K1[i] = T(0); }
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
  T g[8][3];
  VMS_UNROLL
  for (int a = 0; a < 8; ++a)
    VMS_UNROLL
    for (int j = 0; j < 3; ++j) {
      g[a][j] = dN[3 * a] * Ji[0][j] + dN[3 * a + 1] * Ji[1][j] + dN[3 * a + 2] * Ji[2][j];
      R.g[3 * a + j] = g[a][j];
    }
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
      R.L[3 * i + j] = t;
    }
  }
  VMS_UNROLL
  for (int a = 0; a < 8; ++a) R.cb[a] = v[0] * g[a][0] + v[1] * g[a][1] + v[2] * g[a][2];
  const T cd = v[0] * d[0] + v[1] * d[1] + v[2] * d[2];
  const T dd = d[0] * d[0] + d[1] * d[1] + d[2] * d[2];
  const T om = tab.w[q] * det;
  R.w = om;
  const T omb = om * bq;
  VMS_UNROLL
  for (int c = 0; c < 3; ++c)
    VMS_UNROLL
    for (int k = 0; k < 3; ++k) {
      R.Ycf[3 * c + k] = omb * L[c][k] + (c == k ? om * cd : T(0));
      R.Yfc[3 * c + k] = omb * (L[k][c] + (c == k ? tau : T(0)));
    }
  VMS_UNROLL
  for (int k = 0; k < 3; ++k) {
    R.Ycf[9 + k] = -om * d[k];
    R.Yfc[9 + k] = -om * d[k];
    R.Dv[k] = nut * om * d[k];
    R.Wv[k] = omb * v[k] + nut * om * d[k];
  }
  VMS_UNROLL
  for (int i = 0; i < 3; ++i)
    VMS_UNROLL
    for (int k = 0; k < 3; ++k)
      A.kff[3 * i + k] += om * (bq * (bq * L[i][k] + (i == k ? cd : T(0))) + (i == k ? nut * dd : T(0)));
}

// Phase 2 for lane `lane`: accumulate over the nqc points stored by phase 1.
template <typename T>
VMS_HD void tan_phase2(int lane, int q0, int nqc, const WarpArea<T>& W, const RefTab<T>& tab,
                       T nut, T tau, LaneAcc<T>& A) {
  const int a0 = lane >> 3, a1 = a0 + 4, b = lane & 7;
  const int at = lane >> 2, ct = lane & 3;
  for (int qq = 0; qq < nqc; ++qq) {
    const QpRec<T>& Q = W.qp[qq];
    const T* N = tab.N + 8 * (q0 + qq);
    const T w = Q.w;
    const T Nb = N[b], Na0 = N[a0], Na1 = N[a1], Nat = N[at];
    const T wNb = w * Nb;
    const T cbt = w * Q.cb[b] + tau * wNb;
    T wgb[3], nwgb[3], ga0[3], ga1[3], gat[3], L[9];
    VMS_UNROLL
    for (int j = 0; j < 3; ++j) {
      wgb[j] = w * Q.g[3 * b + j];
      nwgb[j] = nut * wgb[j];
      ga0[j] = Q.g[3 * a0 + j];
      ga1[j] = Q.g[3 * a1 + j];
      gat[j] = Q.g[3 * at + j];
    }
    VMS_UNROLL
    for (int j = 0; j < 9; ++j) L[j] = Q.L[j];
    const T m0 = Na0 * wNb, m1 = Na1 * wNb;
    const T s0 = Na0 * cbt + ga0[0] * nwgb[0] + ga0[1] * nwgb[1] + ga0[2] * nwgb[2];
    const T s1 = Na1 * cbt + ga1[0] * nwgb[0] + ga1[1] * nwgb[1] + ga1[2] * nwgb[2];
    VMS_UNROLL
    for (int i = 0; i < 3; ++i) {
      VMS_UNROLL
      for (int k = 0; k < 3; ++k) {
        A.K0[4 * i + k] += m0 * L[3 * i + k];
        A.K1[4 * i + k] += m1 * L[3 * i + k];
      }
      A.K0[5 * i] += s0;
      A.K1[5 * i] += s1;
      A.K0[4 * i + 3] -= ga0[i] * wNb;
      A.K1[4 * i + 3] -= ga1[i] * wNb;
      A.K0[12 + i] -= Na0 * wgb[i];
      A.K1[12 + i] -= Na1 * wgb[i];
    }
    const T gdv = gat[0] * Q.Dv[0] + gat[1] * Q.Dv[1] + gat[2] * Q.Dv[2];
    const T gwv = gat[0] * Q.Wv[0] + gat[1] * Q.Wv[1] + gat[2] * Q.Wv[2];
    VMS_UNROLL
    for (int k = 0; k < 3; ++k) {
      A.kcf[k] += Nat * Q.Ycf[3 * ct + k] + (k == ct ? gdv : T(0));
      A.kfc[k] += Nat * Q.Yfc[3 * ct + k] + (k == ct ? gwv : T(0));
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
  const bool bad = !(det != 0.0) || !(det - det == 0.0);
  const double r = bad ? 0.0 : 1.0 / det;
  if (lane < 9) {
    const double v = W.cof[3 * (lane % 3) + lane / 3] * r;
    W.Kinv[lane] = v;
    W.KinvT[lane] = T(v);
  }
  if (bad && lane == 0) W.flag |= 2u;
}

// Phase 3f: column L of X = K_ff^-1 K_fc and row L of K_cf to shared memory; row L of
// W = K_cf K_ff^-1 (used later for r_e = R_cp - W R_f) into Wl.
template <typename T>
VMS_HD void tan_phase3f(int lane, WarpArea<T>& W, const LaneAcc<T>& A, T Wl[3]) {
  VMS_UNROLL
  for (int m = 0; m < 3; ++m) {
    W.Xs[m][lane] = W.KinvT[3 * m] * A.kfc[0] + W.KinvT[3 * m + 1] * A.kfc[1] +
                    W.KinvT[3 * m + 2] * A.kfc[2];
    W.Kcf[lane][m] = A.kcf[m];
    Wl[m] = A.kcf[0] * W.KinvT[m] + A.kcf[1] * W.KinvT[3 + m] + A.kcf[2] * W.KinvT[6 + m];
  }
}

// Condensed residual entry (FP64): r_t = R_cp[t] - sum_m W[t][m] R_f[m]; y = K_ff^-1 R_f.
template <typename T>
VMS_HD double condensed_residual(double Rcp_t, const T Wt[3], const double Rf[3]) {
  return Rcp_t - ((double)Wt[0] * Rf[0] + (double)Wt[1] * Rf[1] + (double)Wt[2] * Rf[2]);
}

// Phase 3e: S blocks of the lane's two node pairs, in place in K0/K1.
template <typename T>
VMS_HD void tan_phase3e(int lane, const WarpArea<T>& W, LaneAcc<T>& A) {
  const int a0 = lane >> 3, a1 = a0 + 4, b = lane & 7;
  VMS_UNROLL
  for (int i = 0; i < 4; ++i) {
    const T c00 = W.Kcf[4 * a0 + i][0], c01 = W.Kcf[4 * a0 + i][1], c02 = W.Kcf[4 * a0 + i][2];
    const T c10 = W.Kcf[4 * a1 + i][0], c11 = W.Kcf[4 * a1 + i][1], c12 = W.Kcf[4 * a1 + i][2];
    VMS_UNROLL
    for (int k = 0; k < 4; ++k) {
      const T x0 = W.Xs[0][4 * b + k], x1 = W.Xs[1][4 * b + k], x2 = W.Xs[2][4 * b + k];
      A.K0[4 * i + k] -= c00 * x0 + c01 * x1 + c02 * x2;
      A.K1[4 * i + k] -= c10 * x0 + c11 * x1 + c12 * x2;
    }
  }
}

}  // namespace vms
