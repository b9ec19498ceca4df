// Tetrahedral P1 + bubble element (the MINI-type element the paper cites): residual (Section 4.1),
// consistent tangent (Eq. NewtonUpdate2), static condensation of the three bubble unknowns (Eq.
// SchurUpdate) and scatter into the CSR system (Section 5), in one kernel.
//
// Reference tetrahedron (0,0,0), (1,0,0), (0,1,0), (0,0,1); N_a = lambda_a with lambda = (1 - xi -
// eta - zeta, xi, eta, zeta); bubble b = 256 lambda_0 lambda_1 lambda_2 lambda_3. The geometry is
// affine, so det J and the P1 gradients g_a are constant on the element; only the bubble gradient
// and the fields vary between quadrature points, as reference polynomials. Each integral is
// therefore a combination of reference moments of the quadrature rule (computed once per rule on
// the host) with element constants: the quadrature sums, regrouped.
//
// FP64 arithmetic in both precision modes (the values are stored in the mode's type); four lanes
// per element, no shared memory.
#include <cmath>
#include <vector>

#include "element_math.cuh"
#include "vms_internal.h"

namespace vms {

// ---------------------------------------------------------------------------------------------
// host: conical-product rule on the reference tetrahedron (Gauss-Jacobi points from the
// eigenvalues of the Jacobi matrix of the three-term recurrence, Golub-Welsch)
// ---------------------------------------------------------------------------------------------
namespace {

// Nodes and weights of the n-point Gauss rule for the weight (1 - x)^alpha on [-1, 1] (n <= 8).
void gauss_jacobi(int n, double alpha, double* x, double* w) {
  double A[8][8] = {};
  for (int k = 0; k < n; ++k) {
    const double s = 2.0 * k + alpha;
    A[k][k] = (k == 0) ? -alpha / (alpha + 2.0) : -(alpha * alpha) / (s * (s + 2.0));
    if (k + 1 < n) {
      const double kk = k + 1.0, t = 2.0 * kk + alpha;
      const double b2 = 4.0 * kk * (kk + alpha) * kk * (kk + alpha) / (t * t * (t + 1.0) * (t - 1.0));
      A[k][k + 1] = A[k + 1][k] = std::sqrt(b2);
    }
  }
  double Q[8][8] = {};
  for (int i = 0; i < n; ++i) Q[i][i] = 1.0;
  // cyclic Jacobi rotations until the matrix is diagonal
  for (int sweep = 0; sweep < 100; ++sweep) {
    double off = 0.0;
    for (int p = 0; p < n; ++p)
      for (int q = p + 1; q < n; ++q) off += A[p][q] * A[p][q];
    if (off < 1e-32) break;
    for (int p = 0; p < n; ++p)
      for (int q = p + 1; q < n; ++q) {
        if (std::fabs(A[p][q]) < 1e-300) continue;
        const double th = (A[q][q] - A[p][p]) / (2.0 * A[p][q]);
        const double t = (th >= 0 ? 1.0 : -1.0) / (std::fabs(th) + std::sqrt(th * th + 1.0));
        const double c = 1.0 / std::sqrt(t * t + 1.0), sn = t * c;
        for (int k = 0; k < n; ++k) {
          const double akp = A[k][p], akq = A[k][q];
          A[k][p] = c * akp - sn * akq;
          A[k][q] = sn * akp + c * akq;
        }
        for (int k = 0; k < n; ++k) {
          const double apk = A[p][k], aqk = A[q][k];
          A[p][k] = c * apk - sn * aqk;
          A[q][k] = sn * apk + c * aqk;
        }
        for (int k = 0; k < n; ++k) {
          const double qkp = Q[k][p], qkq = Q[k][q];
          Q[k][p] = c * qkp - sn * qkq;
          Q[k][q] = sn * qkp + c * qkq;
        }
      }
  }
  const double mu0 = std::pow(2.0, alpha + 1.0) / (alpha + 1.0);  // int (1-x)^alpha over [-1,1]
  for (int i = 0; i < n; ++i) {
    x[i] = A[i][i];
    w[i] = mu0 * Q[0][i] * Q[0][i];
  }
  for (int i = 1; i < n; ++i)  // ascending nodes
    for (int j = i; j > 0 && x[j] < x[j - 1]; --j) {
      std::swap(x[j], x[j - 1]);
      std::swap(w[j], w[j - 1]);
    }
}

}  // namespace

void tet_rule(int n, std::vector<double>& pts, std::vector<double>& wts) {
  double ux[8], uw[8], vx[8], vw[8], wx[8], ww[8];
  gauss_jacobi(n, 2.0, ux, uw);
  gauss_jacobi(n, 1.0, vx, vw);
  gauss_jacobi(n, 0.0, wx, ww);
  pts.clear();
  wts.clear();
  for (int i = 0; i < n; ++i)
    for (int j = 0; j < n; ++j)
      for (int k = 0; k < n; ++k) {
        const double u = 0.5 * (ux[i] + 1.0), v = 0.5 * (vx[j] + 1.0), w = 0.5 * (wx[k] + 1.0);
        pts.push_back(u);
        pts.push_back(v * (1.0 - u));
        pts.push_back(w * (1.0 - u) * (1.0 - v));
        wts.push_back(uw[i] / 8.0 * vw[j] / 4.0 * ww[k] / 2.0);
      }
}

// Reference moments of the rule with n points per direction (layout of TetMoments): the sums of
// w_q times products of lambda_a, b = 256 s lambda_0 lambda_1 lambda_2 lambda_3 (s the bubble
// scale) and db/dxi at the rule's points.
void tet_moments(int n, double bubble_scale, TetMoments& mom) {
  std::vector<double> pts, wts;
  tet_rule(n, pts, wts);
  double* M = mom.m;
  for (int i = 0; i < TM_COUNT; ++i) M[i] = 0.0;
  static const double dl[4][3] = {{-1, -1, -1}, {1, 0, 0}, {0, 1, 0}, {0, 0, 1}};
  for (size_t q = 0; q < wts.size(); ++q) {
    const double xi = pts[3 * q], eta = pts[3 * q + 1], zeta = pts[3 * q + 2];
    const double lam[4] = {1.0 - xi - eta - zeta, xi, eta, zeta};
    const double b = bubble_scale * 256.0 * lam[0] * lam[1] * lam[2] * lam[3];
    double db[3];
    for (int al = 0; al < 3; ++al) {
      double s = 0.0;
      for (int a = 0; a < 4; ++a) {
        double prod = 1.0;
        for (int c = 0; c < 4; ++c)
          if (c != a) prod *= lam[c];
        s += prod * dl[a][al];
      }
      db[al] = bubble_scale * 256.0 * s;
    }
    const double w = wts[q];
    M[TM_M0] += w;
    M[TM_MB] += w * b;
    M[TM_MBB] += w * b * b;
    for (int al = 0; al < 3; ++al) {
      M[TM_MD + al] += w * db[al];
      M[TM_MBBD + al] += w * b * b * db[al];
      for (int be = 0; be < 3; ++be) M[TM_MDD + 3 * al + be] += w * db[al] * db[be];
    }
    for (int a = 0; a < 4; ++a) {
      M[TM_M1 + a] += w * lam[a];
      M[TM_M1B + a] += w * lam[a] * b;
      for (int al = 0; al < 3; ++al) {
        M[TM_M1D + 3 * a + al] += w * lam[a] * db[al];
        M[TM_M1BD + 3 * a + al] += w * lam[a] * b * db[al];
      }
      for (int c = 0; c < 4; ++c) {
        M[TM_M2 + 4 * a + c] += w * lam[a] * lam[c];
        for (int al = 0; al < 3; ++al)
          M[TM_M2D + 12 * a + 3 * c + al] += w * lam[a] * lam[c] * db[al];
      }
    }
  }
}

// ---------------------------------------------------------------------------------------------
// device
//
// Four lanes per tetrahedron, eight tetrahedra per warp: lane a of a group owns node a (the rows
// 4a..4a+3 of R_cp, K_cc, K_cf and S_e) and the column block a of K_fc. With v = sum_c lambda_c V_c
// + b beta, L = G + beta (x) d (G the constant coarse gradient, d = grad b = J^-T db/dxi) and
// p = sum_c lambda_c P_c, each term of Section 4.1 and Eq. NewtonUpdate2 integrates to element
// constants times reference moments, e.g. int lambda_a lambda_b L_ik = det (G_ik M2[a][b] +
// beta_i sum_al M2d[a][b][al] Jinv[al][k]). Every value is formed in FP64; no lane loops over
// quadrature points.
// ---------------------------------------------------------------------------------------------
namespace {

constexpr int TET_WARPS = 2;     // warps per block
constexpr int TET_PER_WARP = 8;  // tetrahedra per warp

// What every lane of an element's group holds (a = the lane's node).
struct TetElem {
  int nd[4];
  int nda;           // node a
  bool ok;           // det J > 0
  double det;
  double Ji[3][3];   // J^-1: Ji[al][j] = d xi_al / d x_j
  double g[4][3];    // P1 gradients g_c = grad lambda_c
  double G[3][3];    // coarse velocity gradient G[i][j] = sum_c V_c[i] g_c[j]
  double beta[3];
  double Ua[3];      // int lambda_a v       (all integrals divided by det)
  double Ub[3];      // int b v
  double Aa;         // int lambda_a v.d
  double Ab;         // int b v.d
  double Bd;         // int lambda_a beta.d
  double Dint[3];    // int d
  double DD;         // int d.d
  double Pbar;       // int p
  double PdJ[3];     // int p d
  double dVa[3];     // int lambda_a (v - v_prev)
  double dVb[3];     // int b (v - v_prev)
  double ga[3];      // g_a
  // the moment rows of node a (selected without dynamic indexing)
  double m1a, m1ba, m2a[4], m1da[3], m1bda[3], m2da[12];
};

__device__ __forceinline__ double sel4(int a, double x0, double x1, double x2, double x3) {
  return a == 0 ? x0 : a == 1 ? x1 : a == 2 ? x2 : x3;
}

// Gather the element (every lane loads all four nodes; the group's lanes hit the same lines) and
// form the element constants and the integrals the residual and the tangent share.
__device__ __forceinline__ void tet_element(int a, int64_t e, const double4_32a* __restrict__ xyz,
                                            const double4_32a* __restrict__ u,
                                            const double4_32a* __restrict__ up,
                                            const int32_t* __restrict__ conn,
                                            const double* __restrict__ beta, bool transient,
                                            const double* __restrict__ M, TetElem& E) {
  double X[4][3], V[4][3], P[4];
#pragma unroll
  for (int c = 0; c < 4; ++c) {
    const int nd = conn[4 * e + c];
    E.nd[c] = nd;
    const double4_32a x = xyz[nd], w = u[nd];
    X[c][0] = x.x; X[c][1] = x.y; X[c][2] = x.z;
    V[c][0] = w.x; V[c][1] = w.y; V[c][2] = w.z; P[c] = w.w;
  }
#pragma unroll
  for (int i = 0; i < 3; ++i) E.beta[i] = beta[3 * e + i];
  E.nda = a == 0 ? E.nd[0] : a == 1 ? E.nd[1] : a == 2 ? E.nd[2] : E.nd[3];
  E.m1a = sel4(a, M[TM_M1], M[TM_M1 + 1], M[TM_M1 + 2], M[TM_M1 + 3]);
  E.m1ba = sel4(a, M[TM_M1B], M[TM_M1B + 1], M[TM_M1B + 2], M[TM_M1B + 3]);
#pragma unroll
  for (int c = 0; c < 4; ++c) E.m2a[c] = sel4(a, M[TM_M2 + c], M[TM_M2 + 4 + c], M[TM_M2 + 8 + c], M[TM_M2 + 12 + c]);
#pragma unroll
  for (int al = 0; al < 3; ++al) {
    E.m1da[al] = sel4(a, M[TM_M1D + al], M[TM_M1D + 3 + al], M[TM_M1D + 6 + al], M[TM_M1D + 9 + al]);
    E.m1bda[al] = sel4(a, M[TM_M1BD + al], M[TM_M1BD + 3 + al], M[TM_M1BD + 6 + al], M[TM_M1BD + 9 + al]);
  }
#pragma unroll
  for (int l = 0; l < 12; ++l)
    E.m2da[l] = sel4(a, M[TM_M2D + l], M[TM_M2D + 12 + l], M[TM_M2D + 24 + l], M[TM_M2D + 36 + l]);
  // J[i][al] = x_{al+1,i} - x_{0,i}; Jinv[al][j] = cof[j][al] / det
  double J[3][3], cof[3][3];
#pragma unroll
  for (int i = 0; i < 3; ++i)
#pragma unroll
    for (int al = 0; al < 3; ++al) J[i][al] = X[al + 1][i] - X[0][i];
  double det = cofactor3(J, cof);
  E.ok = det >= DET_MIN;
  if (!E.ok) det = 1.0;
  E.det = det;
  const double r = recip_normal(det);
#pragma unroll
  for (int al = 0; al < 3; ++al)
#pragma unroll
    for (int j = 0; j < 3; ++j) E.Ji[al][j] = cof[j][al] * r;
#pragma unroll
  for (int j = 0; j < 3; ++j) {
    E.g[1][j] = E.Ji[0][j];
    E.g[2][j] = E.Ji[1][j];
    E.g[3][j] = E.Ji[2][j];
    E.g[0][j] = -(E.Ji[0][j] + E.Ji[1][j] + E.Ji[2][j]);
    E.ga[j] = sel4(a, E.g[0][j], E.g[1][j], E.g[2][j], E.g[3][j]);
  }
  // The element constants below are the same on the group's four lanes. Each lane forms one part
  // of each (its own node's, or row / column a), in the same instruction stream as the others,
  // and the parts are exchanged by shuffles within the group: the FP64 pipe, which takes a whole
  // issue slot per warp instruction, then does each constant once per element instead of on all
  // four lanes.
  const int gb = threadIdx.x & 28;  // first lane of the group
  auto from = [gb](double v, int src) { return __shfl_sync(0xffffffffu, v, gb | src); };
  auto gsum = [](double v) {
    v += __shfl_xor_sync(0xffffffffu, v, 1);
    return v + __shfl_xor_sync(0xffffffffu, v, 2);
  };
  // w_c: component a of node c's velocity (a < 3) or its pressure (a = 3)
  double w[4];
#pragma unroll
  for (int c = 0; c < 4; ++c) w[c] = sel4(a, V[c][0], V[c][1], V[c][2], P[c]);
  // G[i][j] = sum_c V_c[i] g_c[j]: row a on lane a (lane 3 forms the pressure gradient, unused)
  {
    double Ga[3];
#pragma unroll
    for (int j = 0; j < 3; ++j)
      Ga[j] = w[0] * E.g[0][j] + w[1] * E.g[1][j] + w[2] * E.g[2][j] + w[3] * E.g[3][j];
#pragma unroll
    for (int i = 0; i < 3; ++i)
#pragma unroll
      for (int j = 0; j < 3; ++j) E.G[i][j] = from(Ga[j], i);
  }
  // Ub[j] = int b v_j: component a on lane a
  {
    const double ba = sel4(a, E.beta[0], E.beta[1], E.beta[2], 0.0);
    const double ub = M[TM_M1B] * w[0] + M[TM_M1B + 1] * w[1] + M[TM_M1B + 2] * w[2] +
                      M[TM_M1B + 3] * w[3] + M[TM_MBB] * ba;
#pragma unroll
    for (int j = 0; j < 3; ++j) E.Ub[j] = from(ub, j);
  }
  const double* M2a = E.m2a;
#pragma unroll
  for (int j = 0; j < 3; ++j)
    E.Ua[j] = M2a[0] * V[0][j] + M2a[1] * V[1][j] + M2a[2] * V[2][j] + M2a[3] * V[3][j] + E.m1ba * E.beta[j];
  // reference-frame components Vr_c = Jinv V_c (node c's on lane c) and br = Jinv beta
  double Vra[3], Vr[4][3], br[3];
  {
    double Va[3];
#pragma unroll
    for (int j = 0; j < 3; ++j) Va[j] = sel4(a, V[0][j], V[1][j], V[2][j], V[3][j]);
#pragma unroll
    for (int al = 0; al < 3; ++al) {
      Vra[al] = E.Ji[al][0] * Va[0] + E.Ji[al][1] * Va[1] + E.Ji[al][2] * Va[2];
      br[al] = E.Ji[al][0] * E.beta[0] + E.Ji[al][1] * E.beta[1] + E.Ji[al][2] * E.beta[2];
    }
#pragma unroll
    for (int c = 0; c < 4; ++c)
#pragma unroll
      for (int al = 0; al < 3; ++al) Vr[c][al] = from(Vra[al], c);
  }
  double Aa = 0.0, Bd = 0.0;
#pragma unroll
  for (int al = 0; al < 3; ++al) {
#pragma unroll
    for (int c = 0; c < 4; ++c) Aa += E.m2da[3 * c + al] * Vr[c][al];
    Aa += E.m1bda[al] * br[al];
    Bd += E.m1da[al] * br[al];
  }
  E.Aa = Aa;
  E.Bd = Bd;
  // Ab = int b v.d: node a's terms on lane a, summed over the group
  {
    double ab = 0.0;
#pragma unroll
    for (int al = 0; al < 3; ++al)
      ab += sel4(a, M[TM_M1BD + al], M[TM_M1BD + 3 + al], M[TM_M1BD + 6 + al], M[TM_M1BD + 9 + al]) * Vra[al];
    E.Ab = gsum(ab) + M[TM_MBBD] * br[0] + M[TM_MBBD + 1] * br[1] + M[TM_MBBD + 2] * br[2];
  }
  E.Pbar = M[TM_M1] * P[0] + M[TM_M1 + 1] * P[1] + M[TM_M1 + 2] * P[2] + M[TM_M1 + 3] * P[3];
  // column a of Jinv (lane 3: zero)
  double Jc[3];
#pragma unroll
  for (int al = 0; al < 3; ++al) Jc[al] = sel4(a, E.Ji[al][0], E.Ji[al][1], E.Ji[al][2], 0.0);
  // DD = int d.d = sum_{al,be} Mdd[al][be] (Jinv Jinv^T)[al][be]: row a of Jinv Jinv^T on lane a
  {
    double Jr[3];  // row a of Jinv (lane 3: zero)
#pragma unroll
    for (int j = 0; j < 3; ++j) Jr[j] = sel4(a, E.Ji[0][j], E.Ji[1][j], E.Ji[2][j], 0.0);
    double dd = 0.0;
#pragma unroll
    for (int be = 0; be < 3; ++be) {
      const double jj = Jr[0] * E.Ji[be][0] + Jr[1] * E.Ji[be][1] + Jr[2] * E.Ji[be][2];
      dd += sel4(a, M[TM_MDD + be], M[TM_MDD + 3 + be], M[TM_MDD + 6 + be], 0.0) * jj;
    }
    E.DD = gsum(dd);
  }
  // Pd[al] = int p d_al (reference): component a on lane a; then PdJ = Jinv^T Pd and
  // Dint = Jinv^T Md, component a on lane a
  {
    const double pda = sel4(a, M[TM_M1D], M[TM_M1D + 1], M[TM_M1D + 2], 0.0) * P[0] +
                       sel4(a, M[TM_M1D + 3], M[TM_M1D + 4], M[TM_M1D + 5], 0.0) * P[1] +
                       sel4(a, M[TM_M1D + 6], M[TM_M1D + 7], M[TM_M1D + 8], 0.0) * P[2] +
                       sel4(a, M[TM_M1D + 9], M[TM_M1D + 10], M[TM_M1D + 11], 0.0) * P[3];
    const double Pd[3] = {from(pda, 0), from(pda, 1), from(pda, 2)};
    const double pdj = Pd[0] * Jc[0] + Pd[1] * Jc[1] + Pd[2] * Jc[2];
    const double din = M[TM_MD] * Jc[0] + M[TM_MD + 1] * Jc[1] + M[TM_MD + 2] * Jc[2];
#pragma unroll
    for (int j = 0; j < 3; ++j) {
      E.PdJ[j] = from(pdj, j);
      E.Dint[j] = from(din, j);
    }
  }
  if (transient) {
    double dV[4][3];
#pragma unroll
    for (int c = 0; c < 4; ++c) {
      const double4_32a o = up[E.nd[c]];
      dV[c][0] = V[c][0] - o.x; dV[c][1] = V[c][1] - o.y; dV[c][2] = V[c][2] - o.z;
    }
#pragma unroll
    for (int i = 0; i < 3; ++i)
      E.dVa[i] = M2a[0] * dV[0][i] + M2a[1] * dV[1][i] + M2a[2] * dV[2][i] + M2a[3] * dV[3][i];
    // dVb[i] = int b (v - v_prev)_i: component a on lane a
    double dvb = 0.0;
#pragma unroll
    for (int c = 0; c < 4; ++c) dvb += M[TM_M1B + c] * sel4(a, dV[c][0], dV[c][1], dV[c][2], 0.0);
#pragma unroll
    for (int i = 0; i < 3; ++i) E.dVb[i] = from(dvb, i);
  } else {
#pragma unroll
    for (int i = 0; i < 3; ++i) E.dVa[i] = E.dVb[i] = 0.0;
  }
}

__device__ __forceinline__ double dot3(const double x[3], const double y[3]) {
  return x[0] * y[0] + x[1] * y[1] + x[2] * y[2];
}

// R_cp rows of node a (Eqs. SC_Coarse_Resid_Vec, SC_Coarse_Resid_Vec_2) and R_f (Eq.
// SC_Fine_Resid_Vec), every lane of the group holding the same R_f.
__device__ __forceinline__ void tet_residual(int a, const TetElem& E, const double* __restrict__ M,
                                             double nut, double tau, const double f[3],
                                             double Rcp[4], double Rf[3]) {
  const double gD = dot3(E.ga, E.Dint);
#pragma unroll
  for (int i = 0; i < 3; ++i) {
    const double s = dot3(E.G[i], E.Ua) + E.beta[i] * E.Aa - f[i] * E.m1a + tau * E.dVa[i] -
                     E.ga[i] * E.Pbar + nut * (M[TM_M0] * dot3(E.ga, E.G[i]) + E.beta[i] * gD);
    Rcp[i] = E.det * s;
    const double t = dot3(E.G[i], E.Ub) + E.beta[i] * E.Ab - f[i] * M[TM_MB] + tau * E.dVb[i] -
                     E.PdJ[i] + nut * (dot3(E.G[i], E.Dint) + E.beta[i] * E.DD);
    Rf[i] = E.det * t;
  }
  Rcp[3] = -E.det * (E.m1a * (E.G[0][0] + E.G[1][1] + E.G[2][2]) + E.Bd);
}

template <typename T>
__device__ __forceinline__ void tet_scatter_row(T* p, const double v[4], bool atomic);
template <>
__device__ __forceinline__ void tet_scatter_row<float>(float* p, const double v[4], bool atomic) {
  // one row of a 4x4 node block: four contiguous values, 16-byte aligned (offsets are multiples of 4)
  const float4 w = make_float4((float)v[0], (float)v[1], (float)v[2], (float)v[3]);
  if (atomic) {
    atomicAdd(reinterpret_cast<float4*>(p), w);
  } else {
    float4 o = *reinterpret_cast<float4*>(p);
    o.x += w.x; o.y += w.y; o.z += w.z; o.w += w.w;
    *reinterpret_cast<float4*>(p) = o;
  }
}
template <>
__device__ __forceinline__ void tet_scatter_row<double>(double* p, const double v[4], bool atomic) {
#pragma unroll
  for (int k = 0; k < 4; ++k) {
    if (v[k] == 0.0) continue;
    if (atomic) atomicAdd(p + k, v[k]); else p[k] += v[k];
  }
}

template <typename T, bool ELEM_OUT, bool ATOMIC>
__global__ void __launch_bounds__(TET_WARPS * 32) tet_assembly_kernel(
    const double4_32a* __restrict__ xyz, const double4_32a* __restrict__ u,
    const double4_32a* __restrict__ up, const int32_t* __restrict__ conn,
    const double* __restrict__ beta, const TetMoments mom, KParams kp,
    int64_t first, int64_t count, const int32_t* __restrict__ elem_list,
    const int32_t* __restrict__ blk, const int32_t* __restrict__ rowlen,
    const uint32_t* __restrict__ dir_mask, T* __restrict__ values, double* __restrict__ rhs,
    T* __restrict__ recX, double* __restrict__ recKinv,
    double* __restrict__ recY, double* __restrict__ oS, double* __restrict__ oR,
    double* __restrict__ oKcc, double* __restrict__ oKcf, double* __restrict__ oKfc,
    double* __restrict__ oKff, unsigned int* __restrict__ flags) {
  const double* M = mom.m;
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const int a = lane & 3, src0 = lane & ~3;
  const int64_t stride = (int64_t)gridDim.x * TET_WARPS * TET_PER_WARP;
  for (int64_t base = ((int64_t)blockIdx.x * TET_WARPS + warp) * TET_PER_WARP; base < count; base += stride) {
    // the loop is uniform over the warp (shuffles below); groups past the end redo element `base`
    // and store nothing
    const int64_t it0 = base + (lane >> 2);
    const bool valid = it0 < count;
    const int64_t it = valid ? it0 : base;
    const int64_t e = elem_list ? (int64_t)elem_list[first + it] : first + it;
    const double nut = kp.nu_e ? kp.visc_factor * kp.nu_e[e] : kp.nut;
    const double tau = kp.tau;
    TetElem E;
    tet_element(a, e, xyz, u, up, conn, beta, kp.transient != 0, M, E);
    double Rcp[4], Rf[3];
    tet_residual(a, E, M, nut, tau, kp.f, Rcp, Rf);
    const double det = E.det;

    // K_ff and its inverse (every lane)
    double Q[3], Kff[9];
#pragma unroll
    for (int k = 0; k < 3; ++k) Q[k] = M[TM_MBBD] * E.Ji[0][k] + M[TM_MBBD + 1] * E.Ji[1][k] + M[TM_MBBD + 2] * E.Ji[2][k];
#pragma unroll
    for (int i = 0; i < 3; ++i)
#pragma unroll
      for (int k = 0; k < 3; ++k)
        Kff[3 * i + k] = det * (M[TM_MBB] * E.G[i][k] + E.beta[i] * Q[k] + (i == k ? E.Ab + nut * E.DD : 0.0));
    double Kc[9];
#pragma unroll
    for (int l = 0; l < 9; ++l) {
      const int i = l / 3, j = l % 3;
      const int i1 = (i + 1) % 3, i2 = (i + 2) % 3, j1 = (j + 1) % 3, j2 = (j + 2) % 3;
      Kc[l] = Kff[3 * i1 + j1] * Kff[3 * i2 + j2] - Kff[3 * i1 + j2] * Kff[3 * i2 + j1];
    }
    const double kdet = Kff[0] * Kc[0] + Kff[1] * Kc[1] + Kff[2] * Kc[2];
    const bool bad = !(kdet != 0.0) || !isfinite(kdet);
    const double kr = bad ? 0.0 : 1.0 / kdet;
    double Kinv[9];
#pragma unroll
    for (int l = 0; l < 9; ++l) Kinv[l] = Kc[3 * (l % 3) + l / 3] * kr;

    // F_a = int lambda_a b d, H_a = int lambda_a d (divided by det)
    double F[3], H[3];
#pragma unroll
    for (int m = 0; m < 3; ++m) {
      F[m] = E.m1bda[0] * E.Ji[0][m] + E.m1bda[1] * E.Ji[1][m] + E.m1bda[2] * E.Ji[2][m];
      H[m] = E.m1da[0] * E.Ji[0][m] + E.m1da[1] * E.Ji[1][m] + E.m1da[2] * E.Ji[2][m];
    }
    const double gD = dot3(E.ga, E.Dint);
    const double m1b = E.m1ba;
    // K_fc column block a (3 x 4) and X_a = K_ff^-1 K_fc[:, block a]
    double Kfc[3][4], Xa[3][4];
    {
      const double gUb = dot3(E.ga, E.Ub);
#pragma unroll
      for (int m = 0; m < 3; ++m) {
#pragma unroll
        for (int k = 0; k < 3; ++k)
          Kfc[m][k] = det * (m1b * E.G[m][k] + E.beta[m] * F[k] + (m == k ? gUb + nut * gD + tau * m1b : 0.0));
        Kfc[m][3] = -det * H[m];
      }
#pragma unroll
      for (int m = 0; m < 3; ++m)
#pragma unroll
        for (int k = 0; k < 4; ++k)
          Xa[m][k] = Kinv[3 * m] * Kfc[0][k] + Kinv[3 * m + 1] * Kfc[1][k] + Kinv[3 * m + 2] * Kfc[2][k];
    }
    // K_cf rows of node a (4 x 3), W_a = K_cf K_ff^-1, condensed residual r = R_cp - W_a R_f
    double Kcf[4][3], rr[4];
#pragma unroll
    for (int i = 0; i < 3; ++i)
#pragma unroll
      for (int m = 0; m < 3; ++m)
        Kcf[i][m] = det * (m1b * E.G[i][m] + E.beta[i] * F[m] + (i == m ? E.Aa + nut * gD : 0.0));
#pragma unroll
    for (int m = 0; m < 3; ++m) Kcf[3][m] = -det * H[m];
    double Wa[4][3];
#pragma unroll
    for (int i = 0; i < 4; ++i) {
#pragma unroll
      for (int m = 0; m < 3; ++m) Wa[i][m] = Kcf[i][0] * Kinv[m] + Kcf[i][1] * Kinv[3 + m] + Kcf[i][2] * Kinv[6 + m];
      rr[i] = Rcp[i] - (Wa[i][0] * Rf[0] + Wa[i][1] * Rf[1] + Wa[i][2] * Rf[2]);
    }
    const uint32_t msk = dir_mask[e];
    if (valid) {
      if (!(isfinite(rr[0]) && isfinite(rr[1]) && isfinite(rr[2]) && isfinite(rr[3])))
        atomicOr(flags, FLAG_NAN);
      if (a == 0 && (!E.ok || bad)) atomicOr(flags, (E.ok ? 0u : FLAG_NEG_JACOBIAN) | (bad ? FLAG_SINGULAR_KFF : 0u));
#pragma unroll
      for (int m = 0; m < 3; ++m)
#pragma unroll
        for (int k = 0; k < 4; ++k) recX[96 * e + 32 * m + 4 * a + k] = T(Xa[m][k]);
      if (a < 3) {
        double kr3[3];
#pragma unroll
        for (int k = 0; k < 3; ++k) kr3[k] = a == 0 ? Kinv[k] : a == 1 ? Kinv[3 + k] : Kinv[6 + k];
        recY[3 * e + a] = kr3[0] * Rf[0] + kr3[1] * Rf[1] + kr3[2] * Rf[2];
#pragma unroll
        for (int k = 0; k < 3; ++k) recKinv[9 * e + 3 * a + k] = kr3[k];
      }
      if (ELEM_OUT) {
#pragma unroll
        for (int i = 0; i < 4; ++i) {
          if (oR) oR[16 * it + 4 * a + i] = rr[i];
#pragma unroll
          for (int m = 0; m < 3; ++m) {
            if (oKcf) oKcf[48 * it + 3 * (4 * a + i) + m] = Kcf[i][m];
          }
        }
#pragma unroll
        for (int m = 0; m < 3; ++m)
#pragma unroll
          for (int k = 0; k < 4; ++k)
            if (oKfc) oKfc[48 * it + 16 * m + 4 * a + k] = Kfc[m][k];
        if (oKff && a < 3)
#pragma unroll
          for (int k = 0; k < 3; ++k) oKff[9 * it + 3 * a + k] = a == 0 ? Kff[k] : a == 1 ? Kff[3 + k] : Kff[6 + k];
      } else {
#pragma unroll
        for (int i = 0; i < 4; ++i)
          if (!(msk >> (4 * a + i) & 1u)) {
            double* dst = rhs + 4 * (int64_t)E.nda + i;
            if (ATOMIC) atomicAdd(dst, rr[i]); else *dst += rr[i];
          }
      }
    }
    // S_e blocks (a, b) = K_cc(a, b) - K_cf(a rows) X_b, X_b from lane b of the group
    const int rl = valid && !ELEM_OUT ? rowlen[E.nda] : 0;
#pragma unroll
    for (int b = 0; b < 4; ++b) {
      double Xb[3][4];
#pragma unroll
      for (int m = 0; m < 3; ++m)
#pragma unroll
        for (int k = 0; k < 4; ++k) Xb[m][k] = __shfl_sync(0xffffffffu, Xa[m][k], src0 | b);
      const double m2 = E.m2a[b];
      double Eab[3];
#pragma unroll
      for (int k = 0; k < 3; ++k)
        Eab[k] = E.m2da[3 * b] * E.Ji[0][k] + E.m2da[3 * b + 1] * E.Ji[1][k] + E.m2da[3 * b + 2] * E.Ji[2][k];
      const double sd = dot3(E.g[b], E.Ua) + tau * m2 + nut * M[TM_M0] * dot3(E.ga, E.g[b]);
      double K[4][4];
#pragma unroll
      for (int i = 0; i < 3; ++i) {
#pragma unroll
        for (int k = 0; k < 3; ++k) K[i][k] = det * (E.G[i][k] * m2 + E.beta[i] * Eab[k] + (i == k ? sd : 0.0));
        K[i][3] = -det * E.ga[i] * M[TM_M1 + b];
      }
#pragma unroll
      for (int k = 0; k < 3; ++k) K[3][k] = -det * E.g[b][k] * E.m1a;
      K[3][3] = 0.0;
      if (!valid) continue;
#pragma unroll
      for (int i = 0; i < 4; ++i) {
        double v[4];
#pragma unroll
        for (int k = 0; k < 4; ++k) v[k] = K[i][k] - (Kcf[i][0] * Xb[0][k] + Kcf[i][1] * Xb[1][k] + Kcf[i][2] * Xb[2][k]);
        const int r = 4 * a + i;
        if (ELEM_OUT) {
#pragma unroll
          for (int k = 0; k < 4; ++k) {
            if (oS) oS[256 * it + 16 * r + 4 * b + k] = v[k];
            if (oKcc) oKcc[256 * it + 16 * r + 4 * b + k] = K[i][k];
          }
        } else if (!(msk >> r & 1u)) {
#pragma unroll
          for (int k = 0; k < 4; ++k)
            if (msk >> (4 * b + k) & 1u) v[k] = 0.0;
          tet_scatter_row<T>(values + blk[16 * e + 4 * a + b] + i * rl, v, ATOMIC);
        }
      }
    }
  }
}

// Residual only: mode 0 writes R_cp and R_f per element (elemR, stride 36), mode 1 adds R_cp into
// the assembled residual (constrained dofs skipped) and writes R_f after it.
__global__ void __launch_bounds__(TET_WARPS * 32) tet_residual_kernel(
    const double4_32a* __restrict__ xyz, const double4_32a* __restrict__ u,
    const double4_32a* __restrict__ up, const int32_t* __restrict__ conn,
    const double* __restrict__ beta, const TetMoments mom, KParams kp, int64_t first,
    int64_t count, double* __restrict__ elemR, double* __restrict__ resid,
    const uint32_t* __restrict__ dir_mask, int64_t n_nodes, int mode, unsigned int* __restrict__ flags) {
  const double* M = mom.m;
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const int a = lane & 3;
  const int64_t stride = (int64_t)gridDim.x * TET_WARPS * TET_PER_WARP;
  for (int64_t base = ((int64_t)blockIdx.x * TET_WARPS + warp) * TET_PER_WARP; base < count; base += stride) {
    // the loop is uniform over the warp (tet_element exchanges values by shuffles); groups past
    // the end redo element `base` and store nothing
    const int64_t it0 = base + (lane >> 2);
    const bool valid = it0 < count;
    const int64_t it = valid ? it0 : base;
    const int64_t e = first + it;
    const double nut = kp.nu_e ? kp.visc_factor * kp.nu_e[e] : kp.nut;
    TetElem E;
    tet_element(a, e, xyz, u, up, conn, beta, kp.transient != 0, M, E);
    double Rcp[4], Rf[3];
    tet_residual(a, E, M, nut, kp.tau, kp.f, Rcp, Rf);
    if (!valid) continue;
    if (!(isfinite(Rcp[0]) && isfinite(Rcp[1]) && isfinite(Rcp[2]) && isfinite(Rcp[3]) &&
          isfinite(Rf[0]) && isfinite(Rf[1]) && isfinite(Rf[2])))
      atomicOr(flags, FLAG_NAN);
    if (a == 0 && !E.ok) atomicOr(flags, FLAG_NEG_JACOBIAN);
    if (mode == 0) {
#pragma unroll
      for (int i = 0; i < 4; ++i) elemR[36 * e + 4 * a + i] = Rcp[i];
      if (a < 3) elemR[36 * e + 32 + a] = a == 0 ? Rf[0] : a == 1 ? Rf[1] : Rf[2];
    } else {
      const uint32_t msk = dir_mask[e];
#pragma unroll
      for (int i = 0; i < 4; ++i)
        if (!(msk >> (4 * a + i) & 1u)) atomicAdd(resid + 4 * (int64_t)E.nda + i, Rcp[i]);
      if (a < 3) resid[4 * n_nodes + 3 * e + a] = a == 0 ? Rf[0] : a == 1 ? Rf[1] : Rf[2];
    }
  }
}

unsigned tet_blocks(int64_t count) {
  const int64_t per = TET_WARPS * TET_PER_WARP;
  const int64_t b = (count + per - 1) / per, cap = (int64_t)sm_count() * 32;
  return (unsigned)(b < 1 ? 1 : (b > cap ? cap : b));
}

template <typename T, bool ELEM_OUT, bool ATOMIC>
void launch_ta(const Mesh& m, const State& s, const KParams& kp, const TetMoments& mom,
               const TangentOut& o, int64_t first, int64_t count, const int32_t* elem_list,
               unsigned int* flags, cudaStream_t st) {
  tet_assembly_kernel<T, ELEM_OUT, ATOMIC><<<tet_blocks(count), TET_WARPS * 32, 0, st>>>(
      m.xyz, s.u, s.u_prev, m.conn, s.beta, mom, kp, first, count, elem_list, m.blk, m.rowlen,
      m.dir_mask, reinterpret_cast<T*>(o.values), o.rhs, reinterpret_cast<T*>(o.recX),
      o.recKinv, o.recY, o.S,
      o.r, o.Kcc, o.Kcf, o.Kfc, o.Kff, flags);
}

}  // namespace

int launch_tet_assembly(bool fp32, const Mesh& m, const State& s, const KParams& kp,
                        const TetMoments& mom, const TangentOut& o, int64_t first, int64_t count,
                        const int32_t* elem_list, bool elem_outputs, bool atomic,
                        unsigned int* flags, cudaStream_t st) {
  if (count <= 0) return 0;
  if (elem_outputs && fp32) launch_ta<float, true, true>(m, s, kp, mom, o, first, count, elem_list, flags, st);
  else if (elem_outputs) launch_ta<double, true, true>(m, s, kp, mom, o, first, count, elem_list, flags, st);
  else if (fp32 && atomic) launch_ta<float, false, true>(m, s, kp, mom, o, first, count, elem_list, flags, st);
  else if (fp32) launch_ta<float, false, false>(m, s, kp, mom, o, first, count, elem_list, flags, st);
  else if (atomic) launch_ta<double, false, true>(m, s, kp, mom, o, first, count, elem_list, flags, st);
  else launch_ta<double, false, false>(m, s, kp, mom, o, first, count, elem_list, flags, st);
  return 1;
}

int launch_tet_residual(const Mesh& m, const State& s, const KParams& kp, const TetMoments& mom,
                        double* elemR, double* resid, int64_t first, int64_t count, int mode,
                        unsigned int* flags, cudaStream_t st) {
  if (count <= 0) return 0;
  tet_residual_kernel<<<tet_blocks(count), TET_WARPS * 32, 0, st>>>(
      m.xyz, s.u, s.u_prev, m.conn, s.beta, mom, kp, first, count, elemR, resid, m.dir_mask,
      m.n_nodes, mode, flags);
  return 1;
}

}  // namespace vms

extern "C" int vms_tet_rule(int n, double* pts, double* wts) {
  if (n < 1 || n > 8 || !pts || !wts) return VMS_ERR_INVALID_ARG;
  std::vector<double> p, w;
  vms::tet_rule(n, p, w);
  for (size_t i = 0; i < p.size(); ++i) pts[i] = p[i];
  for (size_t i = 0; i < w.size(); ++i) wts[i] = w[i];
  return VMS_OK;
}
