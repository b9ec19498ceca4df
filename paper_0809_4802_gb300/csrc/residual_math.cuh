// FP64 element residual of the two-level VMS weak form (Section 4.1: Eqs. SC_Coarse_Resid_Vec,
// SC_Coarse_Resid_Vec_2, SC_Fine_Resid_Vec and the backward-Euler Remark).
//
// Trilinear fields are evaluated in the monomial basis {1, xi, eta, zeta, xi eta, xi zeta,
// eta zeta, xi eta zeta}: nodal values map to coefficients by a butterfly (modal8), after which a
// value costs 7 FMA and a reference gradient 9 FMA. Test functions are accumulated in the same
// basis and mapped back to nodes once per element (nodal8).
//
// With omega = w_q det J, cof = det(J) J^-T and G[i][al] = dv_i/dxi_al:
//   omega conv_i = w_q sum_al G[i][al] (cof^T v)_al
//   P[i][al] = omega sum_j sigma_ij (J^-1)[al][j],  sigma = nut L - p I
//            = w_q ( (nut/det) sum_be G[i][be] (cof^T cof)[be][al] - p cof[i][al] )
//   Tp = -omega tr L = -w_q sum_{i,al} G[i][al] cof[i][al]
// so R_c[a][i] = sum_q N_a src_i + dN_a/dxi_al P[i][al], R_p[a] = sum_q N_a Tp,
// R_f[i] = sum_q b src_i + db/dxi_al P[i][al], src_i = omega (conv_i - f_i + tau dvbar_i).
// One reciprocal (1/det J) per quadrature point.
#pragma once

#include "element_math.cuh"

namespace vms {

// Coefficient slots: x-gradient coefficients (3 x 7), v (3 x 8), p (8), vbar - vbar_n (3 x 8).
constexpr int RC_X = 0, RC_V = 21, RC_P = 45, RC_DV = 53, RC_N = 77;

template <class Store>
VMS_HD void residual_load(Store& C, const double X[8][3], const double U[8][4],
                          const double Uprev[8][3], bool transient) {
  double f[8], c[8];
  VMS_UNROLL
  for (int i = 0; i < 3; ++i) {
    VMS_UNROLL
    for (int a = 0; a < 8; ++a) f[a] = X[a][i];
    modal8(f, c);
    VMS_UNROLL
    for (int m = 1; m < 8; ++m) C.set(RC_X + 7 * i + m - 1, 0.125 * c[m]);
  }
  VMS_UNROLL
  for (int i = 0; i < 3; ++i) {
    VMS_UNROLL
    for (int a = 0; a < 8; ++a) f[a] = U[a][i];
    modal8(f, c);
    VMS_UNROLL
    for (int m = 0; m < 8; ++m) C.set(RC_V + 8 * i + m, 0.125 * c[m]);
  }
  VMS_UNROLL
  for (int a = 0; a < 8; ++a) f[a] = U[a][3];
  modal8(f, c);
  VMS_UNROLL
  for (int m = 0; m < 8; ++m) C.set(RC_P + m, 0.125 * c[m]);
  if (transient) {
    VMS_UNROLL
    for (int i = 0; i < 3; ++i) {
      VMS_UNROLL
      for (int a = 0; a < 8; ++a) f[a] = U[a][i] - Uprev[a][i];
      modal8(f, c);
      VMS_UNROLL
      for (int m = 0; m < 8; ++m) C.set(RC_DV + 8 * i + m, 0.125 * c[m]);
    }
  }
}

// Quadrature loop. Rcp[32] (node-major 4a+c) and Rf[3] receive the element residual; returns
// false if det J <= 0 at some point (the offending point then uses det J = 1).
template <bool TRANSIENT, bool FORCE, class Store, class Table>
VMS_HD bool residual_qp_loop(const Store& C, const Table& tab, int nq, const double bet[3],
                             double nut, double tau, const double f[3], double Rcp[32],
                             double Rf[3]) {
  double rm[3][8], rp[8];
  VMS_UNROLL
  for (int m = 0; m < 8; ++m) { rm[0][m] = rm[1][m] = rm[2][m] = 0.0; rp[m] = 0.0; }
  Rf[0] = Rf[1] = Rf[2] = 0.0;
  bool ok = true;
  for (int q = 0; q < nq; ++q) {
    const double xi = tab.xi(q), eta = tab.eta(q), zeta = tab.zeta(q);
    const double xe = tab.xe(q), xz = tab.xz(q), ez = tab.ez(q), xez = tab.xez(q);
    const double bq = tab.b(q), db0 = tab.db(q, 0), db1 = tab.db(q, 1), db2 = tab.db(q, 2);
    const double wq = tab.w(q);

    double J[3][3];
    VMS_UNROLL
    for (int i = 0; i < 3; ++i) {
      const double c1 = C.get(RC_X + 7 * i + 0), c2 = C.get(RC_X + 7 * i + 1);
      const double c3 = C.get(RC_X + 7 * i + 2), c4 = C.get(RC_X + 7 * i + 3);
      const double c5 = C.get(RC_X + 7 * i + 4), c6 = C.get(RC_X + 7 * i + 5);
      const double c7 = C.get(RC_X + 7 * i + 6);
      J[i][0] = c1 + c4 * eta + c5 * zeta + c7 * ez;
      J[i][1] = c2 + c4 * xi + c6 * zeta + c7 * xz;
      J[i][2] = c3 + c5 * xi + c6 * eta + c7 * xe;
    }
    double cof[3][3];
    double det = cofactor3(J, cof);
    if (!(det > 0.0)) { ok = false; det = 1.0; }
    const double om = wq * det;

    const double bet0 = bet[0], bet1 = bet[1], bet2 = bet[2];
    const double betv[3] = {bet0, bet1, bet2};
    double v[3], G[3][3];
    VMS_UNROLL
    for (int i = 0; i < 3; ++i) {
      const double c0 = C.get(RC_V + 8 * i + 0), c1 = C.get(RC_V + 8 * i + 1);
      const double c2 = C.get(RC_V + 8 * i + 2), c3 = C.get(RC_V + 8 * i + 3);
      const double c4 = C.get(RC_V + 8 * i + 4), c5 = C.get(RC_V + 8 * i + 5);
      const double c6 = C.get(RC_V + 8 * i + 6), c7 = C.get(RC_V + 8 * i + 7);
      v[i] = c0 + c1 * xi + c2 * eta + c3 * zeta + c4 * xe + c5 * xz + c6 * ez + c7 * xez + bq * betv[i];
      G[i][0] = c1 + c4 * eta + c5 * zeta + c7 * ez + betv[i] * db0;
      G[i][1] = c2 + c4 * xi + c6 * zeta + c7 * xz + betv[i] * db1;
      G[i][2] = c3 + c5 * xi + c6 * eta + c7 * xe + betv[i] * db2;
    }
    const double p = C.get(RC_P + 0) + C.get(RC_P + 1) * xi + C.get(RC_P + 2) * eta +
                     C.get(RC_P + 3) * zeta + C.get(RC_P + 4) * xe + C.get(RC_P + 5) * xz +
                     C.get(RC_P + 6) * ez + C.get(RC_P + 7) * xez;

    double wv[3];
    VMS_UNROLL
    for (int al = 0; al < 3; ++al)
      wv[al] = wq * (cof[0][al] * v[0] + cof[1][al] * v[1] + cof[2][al] * v[2]);
    double src[3];
    VMS_UNROLL
    for (int i = 0; i < 3; ++i) src[i] = G[i][0] * wv[0] + G[i][1] * wv[1] + G[i][2] * wv[2];
    if (FORCE) {
      VMS_UNROLL
      for (int i = 0; i < 3; ++i) src[i] -= om * f[i];
    }
    if (TRANSIENT) {
      const double tom = tau * om;
      VMS_UNROLL
      for (int i = 0; i < 3; ++i) {
        const double dv = C.get(RC_DV + 8 * i + 0) + C.get(RC_DV + 8 * i + 1) * xi +
                          C.get(RC_DV + 8 * i + 2) * eta + C.get(RC_DV + 8 * i + 3) * zeta +
                          C.get(RC_DV + 8 * i + 4) * xe + C.get(RC_DV + 8 * i + 5) * xz +
                          C.get(RC_DV + 8 * i + 6) * ez + C.get(RC_DV + 8 * i + 7) * xez;
        src[i] += tom * dv;
      }
    }
    const double s = wq * nut / det;
    const double A00 = s * (cof[0][0] * cof[0][0] + cof[1][0] * cof[1][0] + cof[2][0] * cof[2][0]);
    const double A11 = s * (cof[0][1] * cof[0][1] + cof[1][1] * cof[1][1] + cof[2][1] * cof[2][1]);
    const double A22 = s * (cof[0][2] * cof[0][2] + cof[1][2] * cof[1][2] + cof[2][2] * cof[2][2]);
    const double A01 = s * (cof[0][0] * cof[0][1] + cof[1][0] * cof[1][1] + cof[2][0] * cof[2][1]);
    const double A02 = s * (cof[0][0] * cof[0][2] + cof[1][0] * cof[1][2] + cof[2][0] * cof[2][2]);
    const double A12 = s * (cof[0][1] * cof[0][2] + cof[1][1] * cof[1][2] + cof[2][1] * cof[2][2]);
    const double wp = wq * p;
    double P[3][3];
    double trw = 0.0;
    VMS_UNROLL
    for (int i = 0; i < 3; ++i) {
      P[i][0] = G[i][0] * A00 + G[i][1] * A01 + G[i][2] * A02 - wp * cof[i][0];
      P[i][1] = G[i][0] * A01 + G[i][1] * A11 + G[i][2] * A12 - wp * cof[i][1];
      P[i][2] = G[i][0] * A02 + G[i][1] * A12 + G[i][2] * A22 - wp * cof[i][2];
      trw += G[i][0] * cof[i][0] + G[i][1] * cof[i][1] + G[i][2] * cof[i][2];
    }
    const double Tp = -wq * trw;

    VMS_UNROLL
    for (int i = 0; i < 3; ++i) {
      Rf[i] += bq * src[i] + db0 * P[i][0] + db1 * P[i][1] + db2 * P[i][2];
      rm[i][0] += src[i];
      rm[i][1] += xi * src[i] + P[i][0];
      rm[i][2] += eta * src[i] + P[i][1];
      rm[i][3] += zeta * src[i] + P[i][2];
      rm[i][4] += xe * src[i] + eta * P[i][0] + xi * P[i][1];
      rm[i][5] += xz * src[i] + zeta * P[i][0] + xi * P[i][2];
      rm[i][6] += ez * src[i] + zeta * P[i][1] + eta * P[i][2];
      rm[i][7] += xez * src[i] + ez * P[i][0] + xz * P[i][1] + xe * P[i][2];
    }
    rp[0] += Tp;
    rp[1] += xi * Tp;
    rp[2] += eta * Tp;
    rp[3] += zeta * Tp;
    rp[4] += xe * Tp;
    rp[5] += xz * Tp;
    rp[6] += ez * Tp;
    rp[7] += xez * Tp;
  }
  double r[8];
  VMS_UNROLL
  for (int i = 0; i < 3; ++i) {
    nodal8(rm[i], r);
    VMS_UNROLL
    for (int a = 0; a < 8; ++a) Rcp[4 * a + i] = 0.125 * r[a];
  }
  nodal8(rp, r);
  VMS_UNROLL
  for (int a = 0; a < 8; ++a) Rcp[4 * a + 3] = 0.125 * r[a];
  return ok;
}

}  // namespace vms
