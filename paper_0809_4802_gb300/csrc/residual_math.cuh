// FP64 element residual of the two-level VMS weak form (Section 4.1: Eqs. SC_Coarse_Resid_Vec,
// SC_Coarse_Resid_Vec_2, SC_Fine_Resid_Vec and the backward-Euler Remark).
//
// Trilinear fields are evaluated in the monomial basis {1, xi, eta, zeta, xi eta, xi zeta,
// eta zeta, xi eta zeta}: nodal values map to coefficients by a butterfly (modal8), after which a
// value costs 7 FMA and a reference gradient 9 FMA. Test functions are accumulated in the same
// basis and mapped back to nodes once per element (nodal8).
//
// With omega = w_q det J, cof = det(J) J^-T, G[i][al] = dv_i/dxi_al and H = G cof^T (H[i][j] =
// det J dv_i/dx_j, the physical velocity gradient L times det J):
//   omega conv_i = w_q (H v)_i
//   P[i][al] = omega sum_j sigma_ij (J^-1)[al][j],  sigma = nut L - p I
//            = w_q sum_j ( (nut/det) H[i][j] - p delta_ij ) cof[j][al]
//   Tp = -omega tr L = -w_q tr H
// so R_c[a][i] = sum_q N_a src_i + dN_a/dxi_al P[i][al], R_p[a] = sum_q N_a Tp,
// R_f[i] = sum_q b src_i + db/dxi_al P[i][al], src_i = omega (conv_i - f_i + tau dvbar_i).
// One reciprocal (1/det J) per quadrature point.
#pragma once

#include "element_math.cuh"

namespace vms {

// Store slots: x-gradient coefficients (3 x 7), v (3 x 8), p (8), vbar - vbar_n (3 x 8), then the
// monomial sums of the momentum (3 x 8) and continuity (8) test functions.
constexpr int RC_X = 0, RC_V = 21, RC_P = 45, RC_DV = 53, RC_RM = 77, RC_RP = 101, RC_N = 109;

template <class Store>
VMS_HD void residual_load(const Store& C, const double X[8][3], const double U[8][4],
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
//
// The tensor Gauss rule is walked line by line (xi fastest; the table's point order). Along a
// line eta and zeta are fixed, so every trilinear field is a + xi b with a, b formed once per line:
// the three columns of J (J[.][0] constant along the line), the polynomial part of G (its first
// column is also the xi-slope b of v), v's a, p's a and b, and (transient) those of vbar - vbar_n. The test-function sums are factored the same way: a
// monomial xi^a eta^b zeta^c (or its derivative) is xi^a times a line constant, so each line keeps
// seven sums per component (src, xi src, P0, P1, xi P1, P2, xi P2) and two for the continuity term,
// and adds them into the eight monomial sums, which live in the store, once per line.
template <bool TRANSIENT, bool FORCE, int N1, class Store, class Table>
VMS_HD bool residual_qp_loop_n(const Store& C, const Table& tab, const double bet[3], double nut,
                               double tau, const double f[3], double Rcp[32], double Rf[3]) {
  constexpr int n1 = N1;
  VMS_UNROLL
  for (int m = 0; m < 32; ++m) C.set(RC_RM + m, 0.0);
  Rf[0] = Rf[1] = Rf[2] = 0.0;
  bool ok = true;
  for (int k = 0; k < n1; ++k) {
    // plane constants (zeta fixed): the parts of the line constants that do not depend on eta
    const double zeta = tab.zeta(k * n1 * n1);
    double aj0[3], j1a[3], j1b[3], g1a[3], g1b[3], ava[3], avb[3], ada[3], bda[3], adb[3], bdb[3];
    VMS_UNROLL
    for (int i = 0; i < 3; ++i) {
      aj0[i] = C.get(RC_X + 7 * i + 0) + C.get(RC_X + 7 * i + 4) * zeta;
      j1a[i] = C.get(RC_X + 7 * i + 1) + C.get(RC_X + 7 * i + 5) * zeta;
      j1b[i] = C.get(RC_X + 7 * i + 3) + C.get(RC_X + 7 * i + 6) * zeta;
      g1a[i] = C.get(RC_V + 8 * i + 2) + C.get(RC_V + 8 * i + 6) * zeta;
      g1b[i] = C.get(RC_V + 8 * i + 4) + C.get(RC_V + 8 * i + 7) * zeta;
      ava[i] = C.get(RC_V + 8 * i + 0) + C.get(RC_V + 8 * i + 3) * zeta;
      avb[i] = C.get(RC_V + 8 * i + 1) + C.get(RC_V + 8 * i + 5) * zeta;
      if (TRANSIENT) {
        ada[i] = C.get(RC_DV + 8 * i + 0) + C.get(RC_DV + 8 * i + 3) * zeta;
        bda[i] = C.get(RC_DV + 8 * i + 2) + C.get(RC_DV + 8 * i + 6) * zeta;
        adb[i] = C.get(RC_DV + 8 * i + 1) + C.get(RC_DV + 8 * i + 5) * zeta;
        bdb[i] = C.get(RC_DV + 8 * i + 4) + C.get(RC_DV + 8 * i + 7) * zeta;
      }
    }
    const double apa = C.get(RC_P + 0) + C.get(RC_P + 3) * zeta, bpa = C.get(RC_P + 2) + C.get(RC_P + 6) * zeta;
    const double apb = C.get(RC_P + 1) + C.get(RC_P + 5) * zeta, bpb = C.get(RC_P + 4) + C.get(RC_P + 7) * zeta;
    for (int j = 0; j < n1; ++j) {
      const int q0 = (k * n1 + j) * n1;
      const double eta = tab.eta(q0), ez = tab.ez(q0);
      // line constants: along the line J[i][1] = j1a + xi j1b, J[i][2] = j2a + xi j2b, and the
      // same for the reference velocity gradient (g1a, g1b, g2a, g2b); every trilinear field is
      // its plane part plus eta times its eta-slope
      double J0[3], vb[3], va[3], dva[3], dvb[3], j2a[3], j2b[3], g2a[3], g2b[3];
      VMS_UNROLL
      for (int i = 0; i < 3; ++i) {
        J0[i] = aj0[i] + j1b[i] * eta;
        j2a[i] = C.get(RC_X + 7 * i + 2) + C.get(RC_X + 7 * i + 5) * eta;
        j2b[i] = C.get(RC_X + 7 * i + 4) + C.get(RC_X + 7 * i + 6) * eta;
        g2a[i] = C.get(RC_V + 8 * i + 3) + C.get(RC_V + 8 * i + 6) * eta;
        g2b[i] = C.get(RC_V + 8 * i + 5) + C.get(RC_V + 8 * i + 7) * eta;
        vb[i] = avb[i] + g1b[i] * eta;
        va[i] = ava[i] + g1a[i] * eta;
        if (TRANSIENT) {
          dva[i] = ada[i] + bda[i] * eta;
          dvb[i] = adb[i] + bdb[i] * eta;
        }
      }
      const double pa = apa + bpa * eta, pb = apb + bpb * eta;
      // One point of the line: its source term src_i, the fluxes P_al,i paired with the
      // reference-gradient components of the test functions, and the continuity term Tp.
      struct Pt {
        double src[3], P0[3], P1[3], P2[3], Tp;
      };
      auto point = [&](int ii, Pt& o) {
        const int q = q0 + ii;
        const double xi = tab.xi(q);
        const double bq = tab.b(q), db0 = tab.db(q, 0), db1 = tab.db(q, 1), db2 = tab.db(q, 2);
        const double wq = tab.w(q);

        double J[3][3];
        VMS_UNROLL
        for (int i = 0; i < 3; ++i) {
          J[i][0] = J0[i];
          J[i][1] = j1a[i] + xi * j1b[i];
          J[i][2] = j2a[i] + xi * j2b[i];
        }
        double cof[3][3];
        double det = cofactor3(J, cof);
        if (!(det >= DET_MIN)) { ok = false; det = 1.0; }

        double v[3], G[3][3];
        VMS_UNROLL
        for (int i = 0; i < 3; ++i) {
          v[i] = va[i] + xi * vb[i] + bq * bet[i];
          G[i][0] = vb[i] + bet[i] * db0;
          G[i][1] = g1a[i] + xi * g1b[i] + bet[i] * db1;
          G[i][2] = g2a[i] + xi * g2b[i] + bet[i] * db2;
        }
        const double p = pa + xi * pb;

        // H = G cof^T: det J times the physical velocity gradient (H[i][j] = det dv_i/dx_j)
        double H[3][3];
        VMS_UNROLL
        for (int i = 0; i < 3; ++i)
          VMS_UNROLL
          for (int j = 0; j < 3; ++j)
            H[i][j] = G[i][0] * cof[j][0] + G[i][1] * cof[j][1] + G[i][2] * cof[j][2];
        // src_i = w_q (H v - det f + tau det (vbar - vbar_n))_i, Tp = -w_q tr H
        double y[3];
        VMS_UNROLL
        for (int i = 0; i < 3; ++i) y[i] = H[i][0] * v[0] + H[i][1] * v[1] + H[i][2] * v[2];
        if (FORCE) {
          VMS_UNROLL
          for (int i = 0; i < 3; ++i) y[i] -= det * f[i];
        }
        if (TRANSIENT) {
          const double td = tau * det;
          VMS_UNROLL
          for (int i = 0; i < 3; ++i) y[i] += td * (dva[i] + xi * dvb[i]);
        }
        VMS_UNROLL
        for (int i = 0; i < 3; ++i) o.src[i] = wq * y[i];
        o.Tp = -wq * (H[0][0] + H[1][1] + H[2][2]);
        // P = (s H - w_q p I) cof with s = w_q nut / det: w_q (nut L - p I) times det J^-T
        const double s = wq * nut * recip_normal(det);
        const double nwp = -wq * p;
        VMS_UNROLL
        for (int i = 0; i < 3; ++i)
          VMS_UNROLL
          for (int j = 0; j < 3; ++j) H[i][j] = i == j ? s * H[i][j] + nwp : s * H[i][j];
        VMS_UNROLL
        for (int i = 0; i < 3; ++i) {
          o.P0[i] = H[i][0] * cof[0][0] + H[i][1] * cof[1][0] + H[i][2] * cof[2][0];
          o.P1[i] = H[i][0] * cof[0][1] + H[i][1] * cof[1][1] + H[i][2] * cof[2][1];
          o.P2[i] = H[i][0] * cof[0][2] + H[i][1] * cof[1][2] + H[i][2] * cof[2][2];
        }
      };
      // line sums: src, xi src, P0, P1, xi P1, P2, xi P2 (per component), Tp, xi Tp. The points
      // are taken in symmetric pairs (-x, x): the Gauss points are symmetric about 0 (the middle
      // one of an odd rule is 0), b, db1, db2 are even in xi and db0 is odd, so with
      // u = y(x) + y(-x) and w = y(x) - y(-x) a pair adds u to a sum, x w to a xi-moment, and
      // b(x) u_src + db0(x) w_P0 + db1(x) u_P1 + db2(x) u_P2 to R_f.
      double s0[3], s1[3], b0[3], c0[3], c1[3], d0[3], d1[3], t0, t1;
      VMS_UNROLL
      for (int pp = 0; pp < n1 / 2; ++pp) {
        Pt lo, hi;
        point(pp, lo);
        point(n1 - 1 - pp, hi);
        const int qh = q0 + n1 - 1 - pp;
        const double x = tab.xi(qh), bh = tab.b(qh);
        const double e0 = tab.db(qh, 0), e1 = tab.db(qh, 1), e2 = tab.db(qh, 2);
        VMS_UNROLL
        for (int i = 0; i < 3; ++i) {
          const double us = hi.src[i] + lo.src[i], ws = hi.src[i] - lo.src[i];
          const double u0 = hi.P0[i] + lo.P0[i], w0 = hi.P0[i] - lo.P0[i];
          const double u1 = hi.P1[i] + lo.P1[i], w1 = hi.P1[i] - lo.P1[i];
          const double u2 = hi.P2[i] + lo.P2[i], w2 = hi.P2[i] - lo.P2[i];
          Rf[i] = Rf[i] + bh * us + e0 * w0 + e1 * u1 + e2 * u2;
          if (pp == 0) {
            s0[i] = us; s1[i] = x * ws; b0[i] = u0; c0[i] = u1; c1[i] = x * w1; d0[i] = u2;
            d1[i] = x * w2;
          } else {
            s0[i] += us; s1[i] += x * ws; b0[i] += u0; c0[i] += u1; c1[i] += x * w1; d0[i] += u2;
            d1[i] += x * w2;
          }
        }
        const double ut = hi.Tp + lo.Tp, wt = hi.Tp - lo.Tp;
        if (pp == 0) { t0 = ut; t1 = x * wt; }
        else { t0 += ut; t1 += x * wt; }
      }
      if (n1 & 1) {
        // the middle point, xi = 0: no xi-moment, db0 = 0
        Pt m;
        point(n1 / 2, m);
        const int qm = q0 + n1 / 2;
        const double bm = tab.b(qm), e1 = tab.db(qm, 1), e2 = tab.db(qm, 2);
        VMS_UNROLL
        for (int i = 0; i < 3; ++i) {
          Rf[i] = Rf[i] + bm * m.src[i] + e1 * m.P1[i] + e2 * m.P2[i];
          s0[i] += m.src[i]; b0[i] += m.P0[i]; c0[i] += m.P1[i]; d0[i] += m.P2[i];
        }
        t0 += m.Tp;
      }
      // the line's contributions to the monomial sums: xi^a eta^b zeta^c src_i and the
      // derivatives d/dxi (P0), d/deta (P1), d/dzeta (P2) of the same monomials
      VMS_UNROLL
      for (int i = 0; i < 3; ++i) {
        const double sb = s1[i] + b0[i];
        const int r = RC_RM + 8 * i;
        C.set(r + 0, C.get(r + 0) + s0[i]);
        C.set(r + 1, C.get(r + 1) + sb);
        C.set(r + 2, C.get(r + 2) + (eta * s0[i] + c0[i]));
        C.set(r + 3, C.get(r + 3) + (zeta * s0[i] + d0[i]));
        C.set(r + 4, C.get(r + 4) + (eta * sb + c1[i]));
        C.set(r + 5, C.get(r + 5) + (zeta * sb + d1[i]));
        C.set(r + 6, C.get(r + 6) + ez * s0[i] + zeta * c0[i] + eta * d0[i]);
        C.set(r + 7, C.get(r + 7) + ez * sb + zeta * c1[i] + eta * d1[i]);
      }
      C.set(RC_RP + 0, C.get(RC_RP + 0) + t0);
      C.set(RC_RP + 1, C.get(RC_RP + 1) + t1);
      C.set(RC_RP + 2, C.get(RC_RP + 2) + eta * t0);
      C.set(RC_RP + 3, C.get(RC_RP + 3) + zeta * t0);
      C.set(RC_RP + 4, C.get(RC_RP + 4) + eta * t1);
      C.set(RC_RP + 5, C.get(RC_RP + 5) + zeta * t1);
      C.set(RC_RP + 6, C.get(RC_RP + 6) + ez * t0);
      C.set(RC_RP + 7, C.get(RC_RP + 7) + ez * t1);
    }
  }
  double r[8], mm[8];
  VMS_UNROLL
  for (int i = 0; i < 3; ++i) {
    VMS_UNROLL
    for (int m = 0; m < 8; ++m) mm[m] = C.get(RC_RM + 8 * i + m);
    nodal8(mm, r);
    VMS_UNROLL
    for (int a = 0; a < 8; ++a) Rcp[4 * a + i] = 0.125 * r[a];
  }
  VMS_UNROLL
  for (int m = 0; m < 8; ++m) mm[m] = C.get(RC_RP + m);
  nodal8(mm, r);
  VMS_UNROLL
  for (int a = 0; a < 8; ++a) Rcp[4 * a + 3] = 0.125 * r[a];
  return ok;
}

// The quadrature loop for the Gauss rule of nq = 8, 27 or 64 points (the line loop unrolled).
template <bool TRANSIENT, bool FORCE, class Store, class Table>
VMS_HD bool residual_qp_loop(const Store& C, const Table& tab, int nq, const double bet[3],
                             double nut, double tau, const double f[3], double Rcp[32],
                             double Rf[3]) {
  if (nq == 27) return residual_qp_loop_n<TRANSIENT, FORCE, 3>(C, tab, bet, nut, tau, f, Rcp, Rf);
  if (nq == 8) return residual_qp_loop_n<TRANSIENT, FORCE, 2>(C, tab, bet, nut, tau, f, Rcp, Rf);
  return residual_qp_loop_n<TRANSIENT, FORCE, 4>(C, tab, bet, nut, tau, f, Rcp, Rf);
}

#if defined(__CUDACC__)
// One element's residual on one thread: gather the 8 nodes (and the previous step's velocities),
// map them to monomial coefficients in `C`, run the quadrature loop. Returns the element's error
// bits: 1 if det J <= 0 at some point, 4 if a residual entry is not finite (the values of
// FLAG_NEG_JACOBIAN and FLAG_NAN). P provides nut, visc_factor, nu_e, nq, tau and f.
template <bool TRANSIENT, bool FORCE, class Store, class Table, class P>
__device__ __forceinline__ unsigned residual_element(
    int64_t e, const Store& C, const Table& tab, const P& kp,
    const double4_32a* __restrict__ xyz, const double4_32a* __restrict__ u,
    const double4_32a* __restrict__ uprev, const int32_t* __restrict__ conn,
    const double* __restrict__ beta, int nd[8], double Rcp[32], double Rf[3]) {
  {
    const int4* cp = reinterpret_cast<const int4*>(conn + 8 * e);
    const int4 c0 = cp[0], c1 = cp[1];
    nd[0] = c0.x; nd[1] = c0.y; nd[2] = c0.z; nd[3] = c0.w;
    nd[4] = c1.x; nd[5] = c1.y; nd[6] = c1.z; nd[7] = c1.w;
  }
  {
    // one record type at a time, each mapped to its monomial coefficients before the next is
    // loaded (fewer values live at once than gathering all node data first)
    double f[8], c[8], U[8][3];
    {
      double X[8][3];
      VMS_UNROLL
      for (int a = 0; a < 8; ++a) {
        const double4_32a x = xyz[nd[a]];
        X[a][0] = x.x; X[a][1] = x.y; X[a][2] = x.z;
      }
      VMS_UNROLL
      for (int i = 0; i < 3; ++i) {
        VMS_UNROLL
        for (int a = 0; a < 8; ++a) f[a] = X[a][i];
        modal8(f, c);
        VMS_UNROLL
        for (int m = 1; m < 8; ++m) C.set(RC_X + 7 * i + m - 1, 0.125 * c[m]);
      }
    }
    {
      double pn[8];
      VMS_UNROLL
      for (int a = 0; a < 8; ++a) {
        const double4_32a w = u[nd[a]];
        U[a][0] = w.x; U[a][1] = w.y; U[a][2] = w.z; pn[a] = w.w;
      }
      modal8(pn, c);
      VMS_UNROLL
      for (int m = 0; m < 8; ++m) C.set(RC_P + m, 0.125 * c[m]);
    }
    VMS_UNROLL
    for (int i = 0; i < 3; ++i) {
      VMS_UNROLL
      for (int a = 0; a < 8; ++a) f[a] = U[a][i];
      modal8(f, c);
      VMS_UNROLL
      for (int m = 0; m < 8; ++m) C.set(RC_V + 8 * i + m, 0.125 * c[m]);
    }
    if (TRANSIENT) {
      VMS_UNROLL
      for (int a = 0; a < 8; ++a) {
        const double4_32a o = uprev[nd[a]];
        U[a][0] -= o.x; U[a][1] -= o.y; U[a][2] -= o.z;
      }
      VMS_UNROLL
      for (int i = 0; i < 3; ++i) {
        VMS_UNROLL
        for (int a = 0; a < 8; ++a) f[a] = U[a][i];
        modal8(f, c);
        VMS_UNROLL
        for (int m = 0; m < 8; ++m) C.set(RC_DV + 8 * i + m, 0.125 * c[m]);
      }
    }
  }
  const double bet[3] = {beta[3 * e + 0], beta[3 * e + 1], beta[3 * e + 2]};
  const double nut = kp.nu_e ? kp.visc_factor * __ldg(kp.nu_e + e) : kp.nut;
  const bool ok = residual_qp_loop<TRANSIENT, FORCE>(C, tab, kp.nq, bet, nut, kp.tau, kp.f, Rcp, Rf);
  bool finite = isfinite(Rf[0]) && isfinite(Rf[1]) && isfinite(Rf[2]);
  VMS_UNROLL
  for (int k = 0; k < 32; ++k) finite = finite && isfinite(Rcp[k]);
  return (ok ? 0u : 1u) | (finite ? 0u : 4u);
}

// Store the element residual in its 36-double record: R_cp (32, node-major), R_f (3), pad.
__device__ __forceinline__ void store_elem_residual(double* __restrict__ rec, const double Rcp[32],
                                                    const double Rf[3]) {
  double2* out = reinterpret_cast<double2*>(rec);
  VMS_UNROLL
  for (int k = 0; k < 16; ++k) out[k] = make_double2(Rcp[2 * k], Rcp[2 * k + 1]);
  out[16] = make_double2(Rf[0], Rf[1]);
  out[17] = make_double2(Rf[2], 0.0);
}
#endif

}  // namespace vms
