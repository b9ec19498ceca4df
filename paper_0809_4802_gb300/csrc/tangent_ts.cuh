// FP64 tangent blocks from sums of point fields against the reference basis (Section 4.2,
// Eq. NewtonUpdate2).
//
// Every entry of the coarse blocks and of the coarse-fine couplings is a sum over the quadrature
// points of a per-element field times a product of one-dimensional factors of the reference
// basis. With phi_0 = (1 - x)/2, phi_1 = (1 + x)/2 (so that N_a = prod_d phi_{a_d}(xi_d) for the
// corner bits a_d of node a), psi_s = phi_x phi_y for x + y = s, and dphi_x/dx = +-1/2:
//   N_a N_b                = prod_d psi_{a_d + b_d}                      (27 weights)
//   N_a dN_b/dxi_al        = +-1/2 phi_{a_al}(xi_al) prod_{d != al} psi   (18 per al)
//   dN_a/dxi_al dN_b/dxi_al = +-1/4 prod_{d != al} psi                    (9 per al)
//   dN_a/dxi_al dN_b/dxi_be = +-1/4 phi(xi_al) phi(xi_be) psi(xi_ga)      (12 per pair al < be)
//   N_a, dN_a/dxi_al       = prod phi, +-1/2 prod_{d != al} phi            (8, 4 per al)
// so only 164 distinct weights exist. Per element the warp forms 738 sums
//   T_j = sum_q W_j(xi_q) F[f_j][q]
// over 57 per-point fields F (omega L_ik + tau omega delta_ik; omega (J^-1 v)_al; omega J^-1[al][i];
// nut omega (J^-1 J^-T)_albe; the K_cf / K_fc coefficients Ycf, Yfc of tangent_math.cuh;
// nut omega (J^-1 d)_al and (J^-1 (omega b v + nut omega d))_al). The weights being products over
// the directions, each sum is taken one direction at a time on the tensor Gauss rule (ts_sums), and
// every block entry is then a signed combination of a few T_j: about 8 k FMA per element for 27
// points, where the node-pair loop takes ~51 k. Used for the 8- and 27-point rules in FP64 mode.
#pragma once

#include "tangent_math.cuh"
#include "ts_layout.h"

namespace vms {

// Per-warp storage: the 738 sums and the point fields (one array: the sums' plan addresses both).
struct TsArea {
  double T[TS_SUMS];
  double F[1];  // TS_FIELDS x ts_ld(nq), sized at launch
};
__host__ __device__ inline size_t ts_area_bytes(int nq) {
  return (offsetof(TsArea, F) + sizeof(double) * TS_FIELDS * ts_ld(nq) + 15) & ~size_t(15);
}

#if defined(__CUDACC__)
// Lane q = quadrature point (< nq): geometry, fields at q into F[.][q], and the lane's K_ff part.
// The coordinates and the coarse velocity are first mapped to their trilinear monomial coefficients
// (lanes 0..5, one field each, into C.T, which the sums overwrite later), so that a point's J, its
// reference velocity gradient and v take 3 and 7 FMA per entry instead of sums over the 8 nodes.
// B is the one-dimensional basis table (its row TS_ROW_X holds the Gauss points).
__device__ __forceinline__ void ts_phase1(int lane, int nq, WarpArea<double>& W, TsArea& C,
                                          const RefTab<double>& tab, const double* B, double nut,
                                          double tau, LaneAcc<double>& A) {
  double* M = C.T;  // [6][8]: x, y, z, v_x, v_y, v_z
  if (lane < 6) {
    double f[8], c[8];
#pragma unroll
    for (int a = 0; a < 8; ++a) f[a] = lane < 3 ? W.X[a][lane] : W.V[a][lane - 3];
    modal8(f, c);
#pragma unroll
    for (int m = 0; m < 8; ++m) M[8 * lane + m] = 0.125 * c[m];
  }
  __syncwarp();
  const int q = lane;
  if (q >= nq) return;
  const int ld = ts_ld(nq);
  double* F = C.F;
  const int n1 = nq == 8 ? 2 : 3;
  const double xi = B[4 * TS_ROW_X + q % n1], eta = B[4 * TS_ROW_X + (q / n1) % n1],
               zeta = B[4 * TS_ROW_X + q / (n1 * n1)];
  const double ez = eta * zeta, xz = xi * zeta, xe = xi * eta, xez = xe * zeta;
  const double bq = tab.b[q];
  const double db[3] = {tab.db[3 * q], tab.db[3 * q + 1], tab.db[3 * q + 2]};
  // monomials 1, xi, eta, zeta, xi eta, xi zeta, eta zeta, xi eta zeta
  double J[3][3], G[3][3], vc[3];
#pragma unroll
  for (int f = 0; f < 6; ++f) {
    const double* c = M + 8 * f;
    const double d0 = c[1] + c[4] * eta + c[5] * zeta + c[7] * ez;
    const double d1 = c[2] + c[4] * xi + c[6] * zeta + c[7] * xz;
    const double d2 = c[3] + c[5] * xi + c[6] * eta + c[7] * xe;
    if (f < 3) {
      J[f][0] = d0; J[f][1] = d1; J[f][2] = d2;
    } else {
      G[f - 3][0] = d0; G[f - 3][1] = d1; G[f - 3][2] = d2;  // reference gradient of the coarse velocity
      vc[f - 3] = c[0] + c[1] * xi + c[2] * eta + c[3] * zeta + c[4] * xe + c[5] * xz + c[6] * ez +
                  c[7] * xez;
    }
  }
  double cof[3][3];
  double det = cofactor3(J, cof);
  if (!(det >= DET_MIN)) { W.flag = 1u; det = 1.0; }
  const double rdet = recip_normal(det);
  double Ji[3][3];  // (J^-1)[al][j] = cof[j][al] / det
#pragma unroll
  for (int al = 0; al < 3; ++al)
#pragma unroll
    for (int j = 0; j < 3; ++j) Ji[al][j] = cof[j][al] * rdet;
  const double om = tab.w[q] * det;
  double d[3];
#pragma unroll
  for (int j = 0; j < 3; ++j) d[j] = db[0] * Ji[0][j] + db[1] * Ji[1][j] + db[2] * Ji[2][j];
  double v[3], L[3][3];
#pragma unroll
  for (int i = 0; i < 3; ++i) {
    v[i] = vc[i] + bq * W.beta[i];
#pragma unroll
    for (int k = 0; k < 3; ++k)
      L[i][k] = G[i][0] * Ji[0][k] + G[i][1] * Ji[1][k] + G[i][2] * Ji[2][k] + W.beta[i] * d[k];
  }
  const double cd = v[0] * d[0] + v[1] * d[1] + v[2] * d[2];
  const double dd = d[0] * d[0] + d[1] * d[1] + d[2] * d[2];
  const double omb = om * bq, nom = nut * om, tom = tau * om;
#pragma unroll
  for (int i = 0; i < 3; ++i)
#pragma unroll
    for (int k = 0; k < 3; ++k) F[(TF_L + 3 * i + k) * ld + q] = om * L[i][k] + (i == k ? tom : 0.0);
  const double Wv[3] = {omb * v[0] + nom * d[0], omb * v[1] + nom * d[1], omb * v[2] + nom * d[2]};
#pragma unroll
  for (int al = 0; al < 3; ++al) {
    F[(TF_ADV + al) * ld + q] = om * (Ji[al][0] * v[0] + Ji[al][1] * v[1] + Ji[al][2] * v[2]);
#pragma unroll
    for (int i = 0; i < 3; ++i) F[(TF_VP + 3 * al + i) * ld + q] = om * Ji[al][i];
    F[(TF_ZCF + al) * ld + q] = nom * (Ji[al][0] * d[0] + Ji[al][1] * d[1] + Ji[al][2] * d[2]);
    F[(TF_ZFC + al) * ld + q] = Ji[al][0] * Wv[0] + Ji[al][1] * Wv[1] + Ji[al][2] * Wv[2];
  }
  // nut omega (J^-1 J^-T): diagonal 00, 11, 22, then 01, 02, 12
  const int pa[6] = {0, 1, 2, 0, 0, 1}, pb[6] = {0, 1, 2, 1, 2, 2};
#pragma unroll
  for (int m = 0; m < 6; ++m)
    F[(TF_G + m) * ld + q] = nom * (Ji[pa[m]][0] * Ji[pb[m]][0] + Ji[pa[m]][1] * Ji[pb[m]][1] +
                                    Ji[pa[m]][2] * Ji[pb[m]][2]);
#pragma unroll
  for (int c = 0; c < 3; ++c)
#pragma unroll
    for (int k = 0; k < 3; ++k) {
      F[(TF_YCF + 3 * c + k) * ld + q] = omb * L[c][k] + (c == k ? om * cd : 0.0);
      F[(TF_YFC + 3 * c + k) * ld + q] = omb * (L[k][c] + (c == k ? tau : 0.0));
    }
#pragma unroll
  for (int k = 0; k < 3; ++k) {
    F[(TF_YCF + 9 + k) * ld + q] = -om * d[k];
    F[(TF_YFC + 9 + k) * ld + q] = -om * d[k];
  }
#pragma unroll
  for (int i = 0; i < 3; ++i)
#pragma unroll
    for (int k = 0; k < 3; ++k)
      A.kff[3 * i + k] += om * (bq * (bq * L[i][k] + (i == k ? cd : 0.0)) + (i == k ? nut * dd : 0.0));
}

// The 738 sums, by sum factorisation: a sum over the n1^3 points of a field times a product of
// one-dimensional factors prod_d B_d(xi_d) is taken one direction at a time (xi_0 first), each
// partial sum an n1-term dot product with one row of the one-dimensional basis table B (psi_0..2,
// phi_0..1, 1 at the n1 Gauss points; `basis`, 8 x 4 doubles). The host-built plan lists every
// partial sum of the six steps (three directions for the fields 0..26 of the coarse blocks, then
// three for the fields 27..56 of the couplings) as in | out << 12 | row << 24, in and out being
// offsets into the warp's TsArea taken as one array (the sums T, then the fields F); scratch of
// one step is placed where neither its own inputs, the fields still to come nor the sums already
// formed lie. plan[0..6] are the steps' first and last entries. About 8 k FMA per element for
// 27 points, where point sums take 20 k.
__device__ __forceinline__ void ts_sums(int lane, int nq, TsArea& C, const double* __restrict__ B,
                                        const uint32_t* __restrict__ plan) {
  double* A = C.T;
  for (int st = 0; st < TS_STEPS; ++st) {
    const int end = (int)__ldg(plan + st + 1);
    if (nq == 27) {
      for (int j = (int)__ldg(plan + st) + lane; j < end; j += 32) {
        const uint32_t en = __ldg(plan + j);
        const double* a = A + (en & 4095u);
        const double* b = B + 4 * (en >> 24);
        A[(en >> 12) & 4095u] = fma(b[2], a[2], fma(b[1], a[1], b[0] * a[0]));
      }
    } else {
      for (int j = (int)__ldg(plan + st) + lane; j < end; j += 32) {
        const uint32_t en = __ldg(plan + j);
        const double* a = A + (en & 4095u);
        const double* b = B + 4 * (en >> 24);
        A[(en >> 12) & 4095u] = fma(b[1], a[1], b[0] * a[0]);
      }
    }
    __syncwarp();
  }
}

__device__ __forceinline__ int ts_bit(int a, int d) {
  // corner bits of the local node order (-,-,-) (+,-,-) (+,+,-) (-,+,-) (-,-,+) (+,-,+) (+,+,+) (-,+,+)
  return d == 0 ? ((a + 1) >> 1) & 1 : (d == 1 ? (a >> 1) & 1 : (a >> 2) & 1);
}
__device__ __forceinline__ double ts_sgn(int bit) { return bit ? 1.0 : -1.0; }

// The lane's accumulators (blocks (a0, b), (a1, b) of K_cc; row lane of K_cf; column lane of K_fc)
// from the sums.
__device__ __forceinline__ void ts_gather(int lane, const TsArea& C, LaneAcc<double>& A) {
  const double* T = C.T;
  const int a0 = lane >> 3, b = lane & 7;
#pragma unroll
  for (int p = 0; p < 2; ++p) {
    const int a = a0 + 4 * p;
    int ab[3], bb[3], s[3];
#pragma unroll
    for (int dd = 0; dd < 3; ++dd) {
      ab[dd] = ts_bit(a, dd);
      bb[dd] = ts_bit(b, dd);
      s[dd] = ab[dd] + bb[dd];
    }
    const int tL = s[0] + 3 * s[1] + 9 * s[2];
    double diag = 0.0, vp[3] = {0.0, 0.0, 0.0}, pv[3] = {0.0, 0.0, 0.0};
#pragma unroll
    for (int al = 0; al < 3; ++al) {
      const int d1 = ts_d1(al), d2 = ts_d2(al);
      const int psi = s[d1] + 3 * s[d2];
      const int base = TJ_VP + 72 * al;
      diag += 0.5 * ts_sgn(bb[al]) * T[base + ab[al] + 2 * psi];                          // advection
      diag += (ab[al] == bb[al] ? 0.25 : -0.25) * T[TJ_DD + 9 * al + psi];                 // diffusion
#pragma unroll
      for (int i = 0; i < 3; ++i) {
        vp[i] -= 0.5 * ts_sgn(ab[al]) * T[base + 18 * (1 + i) + bb[al] + 2 * psi];        // K_vp
        pv[i] -= 0.5 * ts_sgn(bb[al]) * T[base + 18 * (1 + i) + ab[al] + 2 * psi];        // K_pv
      }
    }
    // off-diagonal diffusion: pairs (al, be) = (0,1), (0,2), (1,2), third direction ga
#pragma unroll
    for (int pp = 0; pp < 3; ++pp) {
      const int al = pp == 2 ? 1 : 0, be = pp == 0 ? 1 : 2, ga = 2 - pp;
      const double* Tp = T + TJ_OD + 12 * pp;
      diag += 0.25 * ts_sgn(ab[al]) * ts_sgn(bb[be]) * Tp[bb[al] + 2 * ab[be] + 4 * s[ga]];
      diag += 0.25 * ts_sgn(ab[be]) * ts_sgn(bb[al]) * Tp[ab[al] + 2 * bb[be] + 4 * s[ga]];
    }
    double k[16];
#pragma unroll
    for (int i = 0; i < 3; ++i) {
#pragma unroll
      for (int kk = 0; kk < 3; ++kk) k[4 * i + kk] = T[TJ_L + 27 * (3 * i + kk) + tL] + (i == kk ? diag : 0.0);
      k[4 * i + 3] = vp[i];
      k[12 + i] = pv[i];
    }
    k[15] = 0.0;
#pragma unroll
    for (int j = 0; j < 16; ++j) {
      if (p) A.K[j].y = k[j];
      else A.K[j].x = k[j];
    }
  }
  const int at = lane >> 2, ct = lane & 3;
  const int tb = ts_bit(at, 0) + 2 * ts_bit(at, 1) + 4 * ts_bit(at, 2);  // tensor order of node at
  double dcf = 0.0, dfc = 0.0;
#pragma unroll
  for (int al = 0; al < 3; ++al) {
    const int u = ts_bit(at, ts_d1(al)), w = ts_bit(at, ts_d2(al));
    const double sg = 0.5 * ts_sgn(ts_bit(at, al));
    dcf += sg * T[TJ_CFD + 4 * al + u + 2 * w];
    dfc += sg * T[TJ_FCD + 4 * al + u + 2 * w];
  }
#pragma unroll
  for (int kk = 0; kk < 3; ++kk) {
    A.kcf[kk] = T[TJ_CFN + 8 * (3 * ct + kk) + tb] + (ct == kk ? dcf : 0.0);
    A.kfc[kk] = T[TJ_FCN + 8 * (3 * ct + kk) + tb] + (ct == kk ? dfc : 0.0);
  }
}
#endif

}  // namespace vms
