// Tetrahedral P1 + bubble element (the MINI-type element the paper cites): residual (Section 4.1),
// consistent tangent (Eq. NewtonUpdate2), static condensation of the three bubble unknowns (Eq.
// SchurUpdate) and scatter into the CSR system (Section 5), in one kernel.
//
// Reference tetrahedron (0,0,0), (1,0,0), (0,1,0), (0,0,1); N_a = lambda_a with lambda = (1 - xi -
// eta - zeta, xi, eta, zeta); bubble b = 256 lambda_0 lambda_1 lambda_2 lambda_3. The geometry is
// affine, so det J and the P1 gradients g_a are constant on the element; only the bubble gradient
// and the fields vary between quadrature points.
//
// One warp per element, FP64 arithmetic in both precision modes (the values are stored in the
// mode's type): lanes take quadrature points and write their point records to shared memory, then
// lanes take matrix entries and sum them over the points, then the warp condenses and scatters.
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

// Table row per point: lambda_0..3, b, db/dxi_0..2, weight.
void tet_table(int n, double bubble_scale, std::vector<double>& tab) {
  std::vector<double> pts, wts;
  tet_rule(n, pts, wts);
  const int nq = (int)wts.size();
  tab.assign((size_t)TET_ROW * nq, 0.0);
  static const double dl[4][3] = {{-1, -1, -1}, {1, 0, 0}, {0, 1, 0}, {0, 0, 1}};
  for (int q = 0; q < nq; ++q) {
    const double xi = pts[3 * q], eta = pts[3 * q + 1], zeta = pts[3 * q + 2];
    const double lam[4] = {1.0 - xi - eta - zeta, xi, eta, zeta};
    double* r = tab.data() + (size_t)TET_ROW * q;
    for (int a = 0; a < 4; ++a) r[a] = lam[a];
    r[4] = bubble_scale * 256.0 * lam[0] * lam[1] * lam[2] * lam[3];
    for (int al = 0; al < 3; ++al) {
      double s = 0.0;
      for (int a = 0; a < 4; ++a) {
        double prod = 1.0;
        for (int c = 0; c < 4; ++c)
          if (c != a) prod *= lam[c];
        s += prod * dl[a][al];
      }
      r[5 + al] = bubble_scale * 256.0 * s;
    }
    r[8] = wts[q];
  }
}

// ---------------------------------------------------------------------------------------------
// device
// ---------------------------------------------------------------------------------------------
namespace {

constexpr int TET_WARPS = 2;
constexpr int QREC = 36;  // doubles per point record

// point record layout
constexpr int Q_LAM = 0, Q_B = 4, Q_D = 5, Q_V = 8, Q_L = 11, Q_P = 20, Q_CONV = 21, Q_DV = 24,
              Q_OM = 27, Q_CD = 28, Q_DD = 29, Q_TRL = 30, Q_CB = 31;  // c_b = v . g_b (4)

struct TetWarp {
  double X[4][3];
  double V[4][3];
  double P[4];
  double Vp[4][3];
  double beta[3];
  int nd[4];
  double g[4][3];   // P1 gradients (constant)
  double vol;       // sum of the point weights times det J
  double Kcc[16][16];
  double Kcf[16][3];
  double Kfc[3][16];
  double Kff[9];
  double Rcp[16];
  double Rf[3];
  double cof[9];
  double Kinv[9];
  double Xs[3][16];
  unsigned int flag;
};

__host__ __device__ size_t tet_warp_bytes(int nq) {
  return ((sizeof(TetWarp) + 15) & ~size_t(15)) + sizeof(double) * QREC * nq;
}

template <typename T>
__device__ __forceinline__ void add_row(T* p, const double v[4], bool atomic) {
#pragma unroll
  for (int k = 0; k < 4; ++k) {
    if (v[k] == 0.0) continue;
    if (atomic) atomicAdd(p + k, T(v[k])); else p[k] += T(v[k]);
  }
}

// Phase A: gather, geometry (every lane, same values), point records (lanes = points).
__device__ bool tet_points(int lane, int64_t e, int nq, const double4_32a* __restrict__ xyz,
                           const double4_32a* __restrict__ u, const double4_32a* __restrict__ up,
                           const int32_t* __restrict__ conn, const double* __restrict__ beta,
                           const double* __restrict__ tab, double tau, bool transient,
                           TetWarp& W, double* __restrict__ rec) {
  if (lane < 4) {
    const int nd = conn[4 * e + lane];
    W.nd[lane] = nd;
    const double4_32a x = xyz[nd], w = u[nd];
    W.X[lane][0] = x.x; W.X[lane][1] = x.y; W.X[lane][2] = x.z;
    W.V[lane][0] = w.x; W.V[lane][1] = w.y; W.V[lane][2] = w.z; W.P[lane] = w.w;
    if (transient) {
      const double4_32a o = up[nd];
      W.Vp[lane][0] = o.x; W.Vp[lane][1] = o.y; W.Vp[lane][2] = o.z;
    } else {
      W.Vp[lane][0] = W.Vp[lane][1] = W.Vp[lane][2] = 0.0;
    }
  } else if (lane < 7) {
    W.beta[lane - 4] = beta[3 * e + lane - 4];
  } else if (lane == 7) {
    W.flag = 0u;
  }
  __syncwarp();
  // J[i][al] = x_{al+1,i} - x_{0,i}; cof; g_a[j] = sum_al dlambda_a[al] (J^-1)[al][j]
  double J[3][3], cof[3][3];
#pragma unroll
  for (int i = 0; i < 3; ++i)
#pragma unroll
    for (int al = 0; al < 3; ++al) J[i][al] = W.X[al + 1][i] - W.X[0][i];
  double det = cofactor3(J, cof);
  const bool ok = det > 0.0;
  if (!ok) det = 1.0;
  const double r = 1.0 / det;
  double g[4][3];
#pragma unroll
  for (int j = 0; j < 3; ++j) {
    // (J^-1)[al][j] = cof[j][al] / det; dlambda_0 = -(1,1,1), dlambda_{a} = e_{a-1}
    g[1][j] = cof[j][0] * r;
    g[2][j] = cof[j][1] * r;
    g[3][j] = cof[j][2] * r;
    g[0][j] = -(g[1][j] + g[2][j] + g[3][j]);
  }
  if (lane < 12) W.g[lane / 3][lane % 3] = g[lane / 3][lane % 3];
  for (int q = lane; q < nq; q += 32) {
    const double* t = tab + TET_ROW * q;
    double* R = rec + QREC * q;
    const double lam[4] = {t[0], t[1], t[2], t[3]};
    const double bq = t[4];
    double d[3];
#pragma unroll
    for (int j = 0; j < 3; ++j) d[j] = (t[5] * cof[j][0] + t[6] * cof[j][1] + t[7] * cof[j][2]) * r;
    double v[3], L[3][3], dv[3];
#pragma unroll
    for (int i = 0; i < 3; ++i) {
      double s = bq * W.beta[i], sp = 0.0;
#pragma unroll
      for (int a = 0; a < 4; ++a) {
        s += lam[a] * W.V[a][i];
        sp += lam[a] * (W.V[a][i] - W.Vp[a][i]);
      }
      v[i] = s;
      dv[i] = sp;
#pragma unroll
      for (int j = 0; j < 3; ++j) {
        double l = W.beta[i] * d[j];
#pragma unroll
        for (int a = 0; a < 4; ++a) l += W.V[a][i] * g[a][j];
        L[i][j] = l;
      }
    }
    double p = 0.0;
#pragma unroll
    for (int a = 0; a < 4; ++a) p += lam[a] * W.P[a];
#pragma unroll
    for (int a = 0; a < 4; ++a) R[Q_LAM + a] = lam[a];
    R[Q_B] = bq;
#pragma unroll
    for (int j = 0; j < 3; ++j) { R[Q_D + j] = d[j]; R[Q_V + j] = v[j]; R[Q_DV + j] = dv[j]; }
#pragma unroll
    for (int i = 0; i < 3; ++i) {
#pragma unroll
      for (int j = 0; j < 3; ++j) R[Q_L + 3 * i + j] = L[i][j];
      R[Q_CONV + i] = L[i][0] * v[0] + L[i][1] * v[1] + L[i][2] * v[2];
    }
    R[Q_P] = p;
    R[Q_OM] = t[8] * det;
    R[Q_CD] = v[0] * d[0] + v[1] * d[1] + v[2] * d[2];
    R[Q_DD] = d[0] * d[0] + d[1] * d[1] + d[2] * d[2];
    R[Q_TRL] = L[0][0] + L[1][1] + L[2][2];
#pragma unroll
    for (int b = 0; b < 4; ++b) R[Q_CB + b] = v[0] * g[b][0] + v[1] * g[b][1] + v[2] * g[b][2];
  }
  if (lane == 0 && !ok) W.flag |= 1u;
  __syncwarp();
  if (lane == 0) {
    double vol = 0.0;
    for (int q = 0; q < nq; ++q) vol += rec[QREC * q + Q_OM];
    W.vol = vol;
  }
  __syncwarp();
  return ok;
}

// Residual entries (lanes 0..15: R_cp, lanes 16..18: R_f) summed over the points.
__device__ void tet_residual_entries(int lane, int nq, const TetWarp& W, const double* rec,
                                     double nut, double tau, const double f[3], double& out) {
  out = 0.0;
  if (lane < 16) {
    const int a = lane >> 2, i = lane & 3;
    for (int q = 0; q < nq; ++q) {
      const double* R = rec + QREC * q;
      const double om = R[Q_OM], la = R[Q_LAM + a];
      if (i < 3) {
        double s = la * (R[Q_CONV + i] - f[i] + tau * R[Q_DV + i]) - W.g[a][i] * R[Q_P];
        s += nut * (W.g[a][0] * R[Q_L + 3 * i] + W.g[a][1] * R[Q_L + 3 * i + 1] + W.g[a][2] * R[Q_L + 3 * i + 2]);
        out += om * s;
      } else {
        out -= om * la * R[Q_TRL];
      }
    }
  } else if (lane < 19) {
    const int i = lane - 16;
    for (int q = 0; q < nq; ++q) {
      const double* R = rec + QREC * q;
      const double b = R[Q_B];
      double s = b * (R[Q_CONV + i] - f[i] + tau * R[Q_DV + i]) - R[Q_D + i] * R[Q_P];
      s += nut * (R[Q_D] * R[Q_L + 3 * i] + R[Q_D + 1] * R[Q_L + 3 * i + 1] + R[Q_D + 2] * R[Q_L + 3 * i + 2]);
      out += R[Q_OM] * s;
    }
  }
}

// Tangent blocks (lanes take entries; formulas of Eq. NewtonUpdate2 with the P1 basis).
__device__ void tet_tangent_entries(int lane, int nq, TetWarp& W, const double* rec, double nut,
                                    double tau) {
  for (int ent = lane; ent < 256; ent += 32) {
    const int r = ent >> 4, c = ent & 15;
    const int a = r >> 2, i = r & 3, b = c >> 2, k = c & 3;
    double s = 0.0;
    if (i < 3 && k < 3) {
      for (int q = 0; q < nq; ++q) {
        const double* R = rec + QREC * q;
        const double lab = R[Q_LAM + a] * R[Q_LAM + b];
        double t = lab * R[Q_L + 3 * i + k];
        if (i == k) t += R[Q_LAM + a] * R[Q_CB + b] + tau * lab;
        s += R[Q_OM] * t;
      }
      if (i == k) s += nut * W.vol * (W.g[a][0] * W.g[b][0] + W.g[a][1] * W.g[b][1] + W.g[a][2] * W.g[b][2]);
    } else if (i < 3 && k == 3) {
      for (int q = 0; q < nq; ++q) s += rec[QREC * q + Q_OM] * rec[QREC * q + Q_LAM + b];
      s *= -W.g[a][i];
    } else if (i == 3 && k < 3) {
      for (int q = 0; q < nq; ++q) s += rec[QREC * q + Q_OM] * rec[QREC * q + Q_LAM + a];
      s *= -W.g[b][k];
    }
    W.Kcc[r][c] = s;
  }
  for (int ent = lane; ent < 48; ent += 32) {
    const int r = ent / 3, m = ent % 3;   // K_cf[r][m]
    const int a = r >> 2, i = r & 3;
    double s = 0.0;
    for (int q = 0; q < nq; ++q) {
      const double* R = rec + QREC * q;
      const double om = R[Q_OM], la = R[Q_LAM + a];
      if (i < 3) {
        double t = la * R[Q_B] * R[Q_L + 3 * i + m];
        if (i == m) t += la * R[Q_CD] + nut * (W.g[a][0] * R[Q_D] + W.g[a][1] * R[Q_D + 1] + W.g[a][2] * R[Q_D + 2]);
        s += om * t;
      } else {
        s -= om * la * R[Q_D + m];
      }
    }
    W.Kcf[r][m] = s;
  }
  for (int ent = lane; ent < 48; ent += 32) {
    const int m = ent / 16, c = ent % 16;   // K_fc[m][c]
    const int b = c >> 2, k = c & 3;
    double s = 0.0;
    for (int q = 0; q < nq; ++q) {
      const double* R = rec + QREC * q;
      const double om = R[Q_OM], lb = R[Q_LAM + b], bq = R[Q_B];
      if (k < 3) {
        double t = bq * lb * R[Q_L + 3 * m + k];
        if (m == k)
          t += bq * R[Q_CB + b] + nut * (R[Q_D] * W.g[b][0] + R[Q_D + 1] * W.g[b][1] + R[Q_D + 2] * W.g[b][2]) +
               tau * bq * lb;
        s += om * t;
      } else {
        s -= om * R[Q_D + m] * lb;
      }
    }
    W.Kfc[m][c] = s;
  }
  if (lane < 9) {
    const int i = lane / 3, k = lane % 3;
    double s = 0.0;
    for (int q = 0; q < nq; ++q) {
      const double* R = rec + QREC * q;
      const double bq = R[Q_B];
      double t = bq * bq * R[Q_L + 3 * i + k];
      if (i == k) t += bq * R[Q_CD] + nut * R[Q_DD];
      s += R[Q_OM] * t;
    }
    W.Kff[lane] = s;
  }
}

template <typename T, bool ELEM_OUT, bool ATOMIC>
__global__ void __launch_bounds__(TET_WARPS * 32) tet_assembly_kernel(
    const double4_32a* __restrict__ xyz, const double4_32a* __restrict__ u,
    const double4_32a* __restrict__ up, const int32_t* __restrict__ conn,
    const double* __restrict__ beta, const double* __restrict__ tab, int nq, KParams kp,
    int64_t first, int64_t count, const int32_t* __restrict__ elem_list,
    const int32_t* __restrict__ blk, const int32_t* __restrict__ rowlen,
    const uint32_t* __restrict__ dir_mask, T* __restrict__ values, double* __restrict__ rhs,
    T* __restrict__ recX, double* __restrict__ recW, double* __restrict__ recKinv,
    double* __restrict__ recY, double* __restrict__ oS, double* __restrict__ oR,
    double* __restrict__ oKcc, double* __restrict__ oKcf, double* __restrict__ oKfc,
    double* __restrict__ oKff, unsigned int* __restrict__ flags) {
  extern __shared__ __align__(16) unsigned char smem[];
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  unsigned char* base = smem + warp * tet_warp_bytes(nq);
  TetWarp& W = *reinterpret_cast<TetWarp*>(base);
  double* rec = reinterpret_cast<double*>(base + ((sizeof(TetWarp) + 15) & ~size_t(15)));
  const int64_t total = (int64_t)gridDim.x * TET_WARPS;
  for (int64_t it = (int64_t)blockIdx.x * TET_WARPS + warp; it < count; it += total) {
    const int64_t e = elem_list ? (int64_t)elem_list[first + it] : first + it;
    const double nut = kp.nu_e ? kp.visc_factor * kp.nu_e[e] : kp.nut;
    tet_points(lane, e, nq, xyz, u, up, conn, beta, tab, kp.tau, kp.transient != 0, W, rec);
    double res;
    tet_residual_entries(lane, nq, W, rec, nut, kp.tau, kp.f, res);
    if (lane < 16) W.Rcp[lane] = res;
    else if (lane < 19) W.Rf[lane - 16] = res;
    tet_tangent_entries(lane, nq, W, rec, nut, kp.tau);
    __syncwarp();
    // K_ff^-1 (FP64, cofactors on lanes 0..8)
    if (lane < 9) {
      const int i = lane / 3, j = lane % 3;
      const int i1 = (i + 1) % 3, i2 = (i + 2) % 3, j1 = (j + 1) % 3, j2 = (j + 2) % 3;
      W.cof[lane] = W.Kff[3 * i1 + j1] * W.Kff[3 * i2 + j2] - W.Kff[3 * i1 + j2] * W.Kff[3 * i2 + j1];
    }
    __syncwarp();
    const double det = W.Kff[0] * W.cof[0] + W.Kff[1] * W.cof[1] + W.Kff[2] * W.cof[2];
    const bool bad = !(det != 0.0) || !isfinite(det);
    if (lane < 9) W.Kinv[lane] = bad ? 0.0 : W.cof[3 * (lane % 3) + lane / 3] / det;
    if (bad && lane == 0) W.flag |= 2u;
    __syncwarp();
    // X = K_ff^-1 K_fc (3 x 16), W_row = K_cf K_ff^-1 (16 x 3)
    for (int ent = lane; ent < 48; ent += 32) {
      const int m = ent / 16, c = ent % 16;
      W.Xs[m][c] = W.Kinv[3 * m] * W.Kfc[0][c] + W.Kinv[3 * m + 1] * W.Kfc[1][c] + W.Kinv[3 * m + 2] * W.Kfc[2][c];
    }
    __syncwarp();
    const uint32_t msk = dir_mask[e];
    // recovery data and the condensed residual r = R_cp - K_cf K_ff^-1 R_f
    double y[3];
#pragma unroll
    for (int m = 0; m < 3; ++m) y[m] = W.Kinv[3 * m] * W.Rf[0] + W.Kinv[3 * m + 1] * W.Rf[1] + W.Kinv[3 * m + 2] * W.Rf[2];
    for (int ent = lane; ent < 48; ent += 32) recX[96 * e + 32 * (ent / 16) + (ent % 16)] = T(W.Xs[ent / 16][ent % 16]);
    if (lane < 16) {
      double wr[3];
#pragma unroll
      for (int m = 0; m < 3; ++m)
        wr[m] = W.Kcf[lane][0] * W.Kinv[m] + W.Kcf[lane][1] * W.Kinv[3 + m] + W.Kcf[lane][2] * W.Kinv[6 + m];
#pragma unroll
      for (int m = 0; m < 3; ++m) recW[96 * e + 3 * lane + m] = wr[m];
      const double rr = W.Rcp[lane] - (wr[0] * W.Rf[0] + wr[1] * W.Rf[1] + wr[2] * W.Rf[2]);
      if (!isfinite(rr)) atomicOr(flags, FLAG_NAN);
      if (ELEM_OUT) {
        if (oR) oR[16 * it + lane] = rr;
      } else if (!(msk >> lane & 1u)) {
        double* dst = rhs + 4 * (int64_t)W.nd[lane >> 2] + (lane & 3);
        if (ATOMIC) atomicAdd(dst, rr); else *dst += rr;
      }
    }
    if (lane < 9) recKinv[9 * e + lane] = W.Kinv[lane];
    if (lane < 3) recY[3 * e + lane] = y[lane];
    // S = K_cc - K_cf X: lane -> block (a, b) = ((lane >> 1) >> 2, (lane >> 1) & 3), rows 2h, 2h+1
    const int blkid = lane >> 1, a = blkid >> 2, b = blkid & 3, h = lane & 1;
    for (int ii = 0; ii < 2; ++ii) {
      const int i = 2 * h + ii, r = 4 * a + i;
      double v[4];
#pragma unroll
      for (int k = 0; k < 4; ++k) {
        const int c = 4 * b + k;
        v[k] = W.Kcc[r][c] - (W.Kcf[r][0] * W.Xs[0][c] + W.Kcf[r][1] * W.Xs[1][c] + W.Kcf[r][2] * W.Xs[2][c]);
      }
      if (ELEM_OUT) {
        if (oS)
#pragma unroll
          for (int k = 0; k < 4; ++k) oS[256 * it + 16 * r + 4 * b + k] = v[k];
      } else if (!(msk >> r & 1u)) {
#pragma unroll
        for (int k = 0; k < 4; ++k)
          if (msk >> (4 * b + k) & 1u) v[k] = 0.0;
        const int32_t off = blk[16 * e + 4 * a + b] + i * rowlen[W.nd[a]];
        add_row(values + off, v, ATOMIC);
      }
    }
    if (ELEM_OUT) {
      if (oKcc)
        for (int ent = lane; ent < 256; ent += 32) oKcc[256 * it + ent] = W.Kcc[ent >> 4][ent & 15];
      if (oKcf)
        for (int ent = lane; ent < 48; ent += 32) oKcf[48 * it + ent] = W.Kcf[ent / 3][ent % 3];
      if (oKfc)
        for (int ent = lane; ent < 48; ent += 32) oKfc[48 * it + ent] = W.Kfc[ent / 16][ent % 16];
      if (oKff && lane < 9) oKff[9 * it + lane] = W.Kff[lane];
    }
    __syncwarp();
    if (lane == 0 && W.flag) atomicOr(flags, W.flag);
    __syncwarp();
  }
}

// Residual only: mode 0 writes R_cp and R_f per element (elemR, stride 36), mode 1 adds R_cp into
// the assembled residual (constrained dofs skipped) and writes R_f after it.
__global__ void __launch_bounds__(TET_WARPS * 32) tet_residual_kernel(
    const double4_32a* __restrict__ xyz, const double4_32a* __restrict__ u,
    const double4_32a* __restrict__ up, const int32_t* __restrict__ conn,
    const double* __restrict__ beta, const double* __restrict__ tab, int nq, KParams kp,
    int64_t first, int64_t count, double* __restrict__ elemR, double* __restrict__ resid,
    const uint32_t* __restrict__ dir_mask, int64_t n_nodes, int mode, unsigned int* __restrict__ flags) {
  extern __shared__ __align__(16) unsigned char smem[];
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  unsigned char* base = smem + warp * tet_warp_bytes(nq);
  TetWarp& W = *reinterpret_cast<TetWarp*>(base);
  double* rec = reinterpret_cast<double*>(base + ((sizeof(TetWarp) + 15) & ~size_t(15)));
  const int64_t total = (int64_t)gridDim.x * TET_WARPS;
  for (int64_t it = (int64_t)blockIdx.x * TET_WARPS + warp; it < count; it += total) {
    const int64_t e = first + it;
    const double nut = kp.nu_e ? kp.visc_factor * kp.nu_e[e] : kp.nut;
    tet_points(lane, e, nq, xyz, u, up, conn, beta, tab, kp.tau, kp.transient != 0, W, rec);
    double res;
    tet_residual_entries(lane, nq, W, rec, nut, kp.tau, kp.f, res);
    if (lane < 19 && !isfinite(res)) atomicOr(flags, FLAG_NAN);
    if (mode == 0) {
      if (lane < 16) elemR[36 * e + lane] = res;
      else if (lane < 19) elemR[36 * e + 32 + lane - 16] = res;
    } else {
      if (lane < 16) {
        if (!(dir_mask[e] >> lane & 1u)) atomicAdd(resid + 4 * (int64_t)W.nd[lane >> 2] + (lane & 3), res);
      } else if (lane < 19) {
        resid[4 * n_nodes + 3 * e + lane - 16] = res;
      }
    }
    __syncwarp();
    if (lane == 0 && W.flag) atomicOr(flags, W.flag);
    __syncwarp();
  }
}

unsigned tet_blocks(int64_t count) {
  int64_t b = (count + TET_WARPS - 1) / TET_WARPS;
  return (unsigned)(b < 1 ? 1 : (b > 152 * 64 ? 152 * 64 : b));
}

template <typename T, bool ELEM_OUT, bool ATOMIC>
void launch_ta(const Mesh& m, const State& s, const KParams& kp, const double* tab, int nq,
               const TangentOut& o, int64_t first, int64_t count, const int32_t* elem_list,
               unsigned int* flags, cudaStream_t st) {
  const size_t smem = TET_WARPS * tet_warp_bytes(nq);
  auto kern = tet_assembly_kernel<T, ELEM_OUT, ATOMIC>;
  cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  kern<<<tet_blocks(count), TET_WARPS * 32, smem, st>>>(
      m.xyz, s.u, s.u_prev, m.conn, s.beta, tab, nq, kp, first, count, elem_list, m.blk, m.rowlen,
      m.dir_mask, reinterpret_cast<T*>(o.values), o.rhs, reinterpret_cast<T*>(o.recX),
      reinterpret_cast<double*>(o.recW), o.recKinv, o.recY, o.S,
      o.r, o.Kcc, o.Kcf, o.Kfc, o.Kff, flags);
}

}  // namespace

int launch_tet_assembly(bool fp32, const Mesh& m, const State& s, const KParams& kp,
                        const double* tab, int nq, const TangentOut& o, int64_t first, int64_t count,
                        const int32_t* elem_list, bool elem_outputs, bool atomic,
                        unsigned int* flags, cudaStream_t st) {
  if (count <= 0) return 0;
  if (elem_outputs && fp32) launch_ta<float, true, true>(m, s, kp, tab, nq, o, first, count, elem_list, flags, st);
  else if (elem_outputs) launch_ta<double, true, true>(m, s, kp, tab, nq, o, first, count, elem_list, flags, st);
  else if (fp32 && atomic) launch_ta<float, false, true>(m, s, kp, tab, nq, o, first, count, elem_list, flags, st);
  else if (fp32) launch_ta<float, false, false>(m, s, kp, tab, nq, o, first, count, elem_list, flags, st);
  else if (atomic) launch_ta<double, false, true>(m, s, kp, tab, nq, o, first, count, elem_list, flags, st);
  else launch_ta<double, false, false>(m, s, kp, tab, nq, o, first, count, elem_list, flags, st);
  return 1;
}

int launch_tet_residual(const Mesh& m, const State& s, const KParams& kp, const double* tab, int nq,
                        double* elemR, double* resid, int64_t first, int64_t count, int mode,
                        unsigned int* flags, cudaStream_t st) {
  if (count <= 0) return 0;
  const size_t smem = TET_WARPS * tet_warp_bytes(nq);
  cudaFuncSetAttribute(tet_residual_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  tet_residual_kernel<<<tet_blocks(count), TET_WARPS * 32, smem, st>>>(
      m.xyz, s.u, s.u_prev, m.conn, s.beta, tab, nq, kp, first, count, elemR, resid, m.dir_mask,
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
