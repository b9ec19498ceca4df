// Element tangent, Schur condensation and scatter-add into the CSR system (Sections 4.2 and 5).
// One warp per element; the phases are in tangent_math.cuh.
//
// The tangent kernel does not read the residual: it stores, per element, X = K_ff^-1 K_fc,
// W = K_cf K_ff^-1 and K_ff^-1, and the FP64 finish kernel forms r_e = R_cp - W R_f and
// y = K_ff^-1 R_f once both the residual and the tangent kernels are done. The two element
// kernels are therefore independent and run concurrently (FP64 pipe and FP32 pipe).
#include <algorithm>

#include "residual_math.cuh"
#include "residual_table.cuh"
#include "tangent_math.cuh"
#include "tangent_tc.cuh"
#include "tangent_ts.cuh"
#include "vms_internal.h"

namespace vms {

// default warps per block: FP64 records are twice the size, so the FP64 kernel uses smaller
// blocks to keep several blocks (and enough warps for the FP64 pipe) resident per SM. The
// autotuner (vms_autotune) may choose another count from tan_warp_choices.
template <typename T> constexpr int tan_warps() { return sizeof(T) == 4 ? 4 : 2; }

// Shared memory of one warp: the fixed part and the records of at most QCH quadrature points
// (points are processed in chunks of QCH).
template <typename T, int QCH = 32>
__host__ __device__ inline size_t tan_warp_bytes(int nq) {
  int qc = nq < QCH ? nq : QCH;
  size_t b = offsetof(WarpArea<T>, qp) + (size_t)qc * sizeof(QpRec<T>);
  return (b + 15) & ~size_t(15);
}
template <typename T>
__host__ __device__ inline size_t tan_table_bytes(int nq) {
  return ((size_t)37 * nq * sizeof(T) + 15) & ~size_t(15);
}

// An FP32 K_ff is accurate to about 1e-7 of its largest entry (FP32 node data and quadrature
// sums), which is 1e-7 * cond(K_ff) relative to its weakest direction; the condensation divides by
// that direction, so elements whose K_ff is ill-conditioned (convection-dominated coarse elements)
// get their K_ff again in FP64 before they are condensed. cond_inf above this value triggers it,
// which bounds the K_ff part of the error of S_e near 1e-7 * 16.
constexpr double KFF_FP64_COND = 16.0;

#if defined(__CUDACC__)
// K_ff in FP64 (Eq. NewtonUpdate2, fine-fine block: int b (b L + I v.d) + nut I d.d) from the FP64
// node data of element e; lanes take quadrature points, the warp sums. Every lane returns K.
__device__ void kff_fp64(int lane, int nq, const int nd[8], const double4_32a* __restrict__ xyz,
                         const double4_32a* __restrict__ u, const double* __restrict__ beta,
                         int64_t e, const double* __restrict__ tab, double nut, double K[9]) {
  VMS_UNROLL
  for (int j = 0; j < 9; ++j) K[j] = 0.0;
  const double bt[3] = {beta[3 * e], beta[3 * e + 1], beta[3 * e + 2]};
  for (int q = lane; q < nq; q += 32) {
    const double* N = tab + 8 * q;
    const double* dN = tab + 8 * nq + 24 * q;
    const double bq = tab[32 * nq + q];
    const double* db = tab + 33 * nq + 3 * q;
    const double wq = tab[36 * nq + q];
    double J[3][3] = {}, G[3][3] = {}, v[3] = {};
    VMS_UNROLL
    for (int a = 0; a < 8; ++a) {
      const double4_32a x = xyz[nd[a]];
      const double4_32a w = u[nd[a]];
      const double xa[3] = {x.x, x.y, x.z}, va[3] = {w.x, w.y, w.z};
      VMS_UNROLL
      for (int i = 0; i < 3; ++i) {
        v[i] += __ldg(N + a) * va[i];
        VMS_UNROLL
        for (int al = 0; al < 3; ++al) {
          const double dn = __ldg(dN + 3 * a + al);
          J[i][al] += xa[i] * dn;
          G[i][al] += va[i] * dn;
        }
      }
    }
    double cof[3][3];
    double det = cofactor3(J, cof);
    if (!(det > 0.0)) det = 1.0;  // the FP32 pass has flagged the element already
    const double r = recip(det);
    double d[3];
    VMS_UNROLL
    for (int j = 0; j < 3; ++j) d[j] = (__ldg(db) * cof[j][0] + __ldg(db + 1) * cof[j][1] + __ldg(db + 2) * cof[j][2]) * r;
    VMS_UNROLL
    for (int i = 0; i < 3; ++i) {
      v[i] += bq * bt[i];
      VMS_UNROLL
      for (int al = 0; al < 3; ++al) G[i][al] += bt[i] * __ldg(db + al);
    }
    const double om = wq * det;
    const double cd = v[0] * d[0] + v[1] * d[1] + v[2] * d[2];
    const double dd = d[0] * d[0] + d[1] * d[1] + d[2] * d[2];
    VMS_UNROLL
    for (int i = 0; i < 3; ++i)
      VMS_UNROLL
      for (int k = 0; k < 3; ++k) {
        // L_ik = sum_al G[i][al] (J^-1)[al][k], (J^-1)[al][k] = cof[k][al] / det
        const double L = (G[i][0] * cof[k][0] + G[i][1] * cof[k][1] + G[i][2] * cof[k][2]) * r;
        K[3 * i + k] += om * (bq * (bq * L + (i == k ? cd : 0.0)) + (i == k ? nut * dd : 0.0));
      }
  }
  VMS_UNROLL
  for (int j = 0; j < 9; ++j)
    for (int o = 16; o > 0; o >>= 1) K[j] += __shfl_xor_sync(0xffffffffu, K[j], o);
}
#endif

// Add four contiguous values (one row of a 4x4 node block; 16-byte aligned in FP32 because
// every row offset and block offset is a multiple of 4). Constrained columns carry zeros.
__device__ __forceinline__ void scatter_row(float* p, const float v[4], bool atomic) {
  if (atomic) {
    atomicAdd(reinterpret_cast<float4*>(p), make_float4(v[0], v[1], v[2], v[3]));
  } else {
    float4 o = *reinterpret_cast<float4*>(p);
    o.x += v[0]; o.y += v[1]; o.z += v[2]; o.w += v[3];
    *reinterpret_cast<float4*>(p) = o;
  }
}
__device__ __forceinline__ void scatter_row(double* p, const double v[4], bool atomic) {
#pragma unroll
  for (int k = 0; k < 4; ++k) {
    if (v[k] == 0.0) continue;
    if (atomic) atomicAdd(p + k, v[k]); else p[k] += v[k];
  }
}

// Node records in the tangent's arithmetic type (FP64 mode reads the FP64 state directly).
template <typename T> struct NodeVec;
template <> struct NodeVec<double> { using type = double4_32a; };
template <> struct NodeVec<float> { using type = float4; };

// One element (a1-a8) for one warp: gather, quadrature-point coefficients, tangent blocks,
// condensation, recovery data and the scatter (or the element outputs). `it` is the element's
// position in the launch (element outputs), `e` its index in the mesh.
template <typename T, bool ELEM_OUT, bool ATOMIC, int QCH = 32, int ENG = 0>
__device__ __forceinline__ void tangent_element(
    int lane, int64_t it, int64_t e, WarpArea<T>& W, const RefTab<T>& tab, void* tcw,
    const void* __restrict__ ext0, const void* __restrict__ ext1,
    const typename NodeVec<T>::type* __restrict__ u, const int32_t* __restrict__ conn,
    const T* __restrict__ beta, int nq, T nut, T tau, const double* __restrict__ nu_e,
    double visc_factor, const double4_32a* __restrict__ xyz64, const float4* __restrict__ xhl,
    const double4_32a* __restrict__ u64,
    const double* __restrict__ beta64, const double* __restrict__ tab64,
    const int32_t* __restrict__ blk, const int32_t* __restrict__ rowlen,
    const uint32_t* __restrict__ dir_mask, T* __restrict__ values, T* __restrict__ recX,
    T* __restrict__ recKcf, double* __restrict__ recKinv, double* __restrict__ oS,
    double* __restrict__ oKcc, double* __restrict__ oKcf, double* __restrict__ oKfc,
    double* __restrict__ oKff, unsigned int* __restrict__ flags) {
  // gather (a1): 8 nodes and the bubble coefficients
  if (lane < 8) {
    const int nd = conn[8 * e + lane];
    W.nd[lane] = nd;
    const auto w = u[nd];
    if constexpr (sizeof(T) == 4) {
      // FP32 geometry from the coordinates relative to the element's first node: J is unchanged
      // (the basis gradients sum to zero), while FP32 copies of absolute coordinates far from the
      // origin would resolve the element's extent only to |x| * 6e-8 / h (2e-5 at x = 30 with
      // h = 1/13). With x = hi + lo (FP32 parts), (hi - hi_0) + (lo - lo_0) is the relative
      // coordinate to FP32 rounding: hi - hi_0 is exact where the two agree in sign and exponent
      // range (far from the origin) and rounds at the level of |x| ~ h near it; no FP64 arithmetic.
      const float4 h = xhl[2 * nd], l = xhl[2 * nd + 1];
      W.X[lane][0] = (h.x - __shfl_sync(0xffu, h.x, 0)) + (l.x - __shfl_sync(0xffu, l.x, 0));
      W.X[lane][1] = (h.y - __shfl_sync(0xffu, h.y, 0)) + (l.y - __shfl_sync(0xffu, l.y, 0));
      W.X[lane][2] = (h.z - __shfl_sync(0xffu, h.z, 0)) + (l.z - __shfl_sync(0xffu, l.z, 0));
    } else {
      const double4_32a x = xyz64[nd];
      W.X[lane][0] = x.x; W.X[lane][1] = x.y; W.X[lane][2] = x.z;
    }
    W.V[lane][0] = w.x; W.V[lane][1] = w.y; W.V[lane][2] = w.z;
  } else if (lane < 11) {
    W.beta[lane - 8] = beta[3 * e + lane - 8];
  } else if (lane == 11) {
    W.flag = 0u;
  }
  __syncwarp();
  const T nut_e = nu_e ? T(visc_factor * __ldg(nu_e + e)) : nut;
  LaneAcc<T> A;
  tan_zero(A);
  if constexpr (ENG == 0) {
    for (int q0 = 0; q0 < nq; q0 += QCH) {
      if (QCH == 32 || lane < QCH) tan_phase1(lane, q0, nq, W, tab, nut_e, tau, A);
      __syncwarp();
      tan_phase2(lane, nq - q0 < QCH ? nq - q0 : QCH, W, nut_e, A);
      __syncwarp();
    }
  } else if constexpr (ENG == TS_ENGINE) {
    // FP64 factorised sums (nq = 8 or 27, checked on the host): ext0 = one-dimensional basis
    // (shared), ext1 = plan of the partial sums (global)
    TsArea& C = *reinterpret_cast<TsArea*>(tcw);
    ts_phase1(lane, nq, W, C, tab, reinterpret_cast<const double*>(ext0), nut_e, tau, A);
    __syncwarp();
    ts_sums(lane, nq, C, reinterpret_cast<const double*>(ext0), reinterpret_cast<const uint32_t*>(ext1));
    __syncwarp();
    ts_gather(lane, C, A);
    __syncwarp();
  } else {
    // tensor-core contractions (FP32 only; nq <= 32, checked on the host); ext0 = B fragments
    TcArea<ENG>& C = *reinterpret_cast<TcArea<ENG>*>(tcw);
    tc_phase1<ENG>(lane, nq, W, C, tab, nut_e, tau, A);
    __syncwarp();
    tc_contract<ENG>(lane, C, reinterpret_cast<const uint32_t*>(ext0));
    __syncwarp();
    tc_gather<ENG>(lane, C, A);
    __syncwarp();
  }
  const int a0 = lane >> 3, a1 = a0 + 4, b = lane & 7;
  if (ELEM_OUT) {
    if (oKcc) {
      double* K = oKcc + 1024 * it;
#pragma unroll
      for (int i = 0; i < 4; ++i)
#pragma unroll
        for (int k = 0; k < 4; ++k) {
          K[(4 * a0 + i) * 32 + 4 * b + k] = (double)A.K[4 * i + k].x;
          K[(4 * a1 + i) * 32 + 4 * b + k] = (double)A.K[4 * i + k].y;
        }
    }
    if (oKcf)
      for (int k = 0; k < 3; ++k) oKcf[96 * it + 3 * lane + k] = (double)A.kcf[k];
    if (oKfc)
      for (int k = 0; k < 3; ++k) oKfc[96 * it + 32 * k + lane] = (double)A.kfc[k];
  }
  // condensation (a6)
  tan_phase3a(lane, W, A);
  __syncwarp();
  tan_phase3b(lane, W);
  __syncwarp();
  tan_phase3c(lane, W);
  __syncwarp();
  tan_phase3d(lane, W);
  __syncwarp();
  bool accurate = false;
  if constexpr (sizeof(T) == 4) {
    int ill = 0;
    if (lane == 0) ill = kff_cond_inf(W) > T(KFF_FP64_COND);
    accurate = __shfl_sync(0xffffffffu, ill, 0) != 0;  // warp-uniform
    if (accurate) {
      double K[9];
      const double nut64 = nu_e ? visc_factor * __ldg(nu_e + e) : (double)nut;
      kff_fp64(lane, nq, W.nd, xyz64, u64, beta64, e, tab64, nut64, K);
      __syncwarp();
      if (lane < 9) W.Kff[lane] = K[lane];
      __syncwarp();
      tan_phase3c(lane, W);
      __syncwarp();
      tan_phase3d(lane, W);
      __syncwarp();
    }
  }
  tan_phase3f(lane, W, A, accurate);
  __syncwarp();
  tan_phase3e(lane, W, A, accurate);
  // per-element data for the finish kernel (K_cf, K_ff^-1) and the fine-scale recovery (X)
#pragma unroll
  for (int m = 0; m < 3; ++m) {
    recX[96 * e + 32 * m + lane] = W.Xs[m][lane];
    recKcf[96 * e + 3 * lane + m] = A.kcf[m];
  }
  if (lane < 9) recKinv[9 * e + lane] = W.Kinv[lane];
  if (ELEM_OUT) {
    if (oS) {
      double* S = oS + 1024 * it;
#pragma unroll
      for (int i = 0; i < 4; ++i)
#pragma unroll
        for (int k = 0; k < 4; ++k) {
          S[(4 * a0 + i) * 32 + 4 * b + k] = (double)A.K[4 * i + k].x;
          S[(4 * a1 + i) * 32 + 4 * b + k] = (double)A.K[4 * i + k].y;
        }
    }
    if (oKff && lane < 9) oKff[9 * it + lane] = W.Kff[lane];
  } else {
    // scatter-add (a7), skipping constrained rows and columns (a8 is completed by the
    // diagonal kernel)
    const uint32_t msk = dir_mask[e];
    const int32_t* bk = blk + 64 * e;
#pragma unroll
    for (int p = 0; p < 2; ++p) {
      const int a = p ? a1 : a0;
      const int32_t off = bk[8 * a + b];
      const int32_t rl = rowlen[W.nd[a]];
#pragma unroll
      for (int i = 0; i < 4; ++i) {
        if (msk >> (4 * a + i) & 1u) continue;
        T v[4];
#pragma unroll
        for (int k = 0; k < 4; ++k)
          v[k] = (msk >> (4 * b + k) & 1u) ? T(0) : (p ? A.K[4 * i + k].y : A.K[4 * i + k].x);
        scatter_row(values + off + (int64_t)i * rl, v, ATOMIC);
      }
    }
  }
  __syncwarp();
  // flag bits 1 (det J <= 0) and 2 (singular K_ff) coincide with FLAG_NEG_JACOBIAN/SINGULAR_KFF
  if (lane == 0 && W.flag) atomicOr(flags, W.flag);
  __syncwarp();
}

// Shared memory of the tangent kernel: the reference table, the tensor-core right operands (ENG
// != 0), then per warp its WarpArea (point records only for the CUDA-core contractions) and its
// TcArea (tensor-core contractions).
template <typename T, int ENG>
__host__ __device__ inline size_t tan_bfrag_bytes() {
  if constexpr (ENG == 0) return 0;
  else if constexpr (ENG == TS_ENGINE) return sizeof(double) * 4 * TS_BASIS_ROWS;
  else return (size_t)tc_bsteps<ENG>() * 32 * tc_bwords<ENG>() * 4;
}
template <typename T, int ENG>
__host__ __device__ inline size_t tan_warp_total(int nq) {
  if constexpr (ENG == 0) return tan_warp_bytes<T>(nq);
  else if constexpr (ENG == TS_ENGINE) return tan_warp_bytes<T, 0>(nq) + ts_area_bytes(nq);
  else return tan_warp_bytes<T, 0>(nq) + ((sizeof(TcArea<ENG>) + 15) & ~size_t(15));
}

constexpr int TC_WARPS = 2;
constexpr int TS_WARPS = 4;  // FP64 weighted sums: ~24 KB of point fields and sums per warp

template <typename T, bool ELEM_OUT, bool ATOMIC, int WARPS, int ENG = 0>
__global__ void __launch_bounds__(WARPS * 32, ENG == 0 ? 1 : (ENG == TS_ENGINE ? 2 : 4)) tangent_kernel(
    const typename NodeVec<T>::type* __restrict__ u, const int32_t* __restrict__ conn, const T* __restrict__ beta, const T* __restrict__ gtab,
    int nq, T nut, T tau, const double* __restrict__ nu_e, double visc_factor,
    const double4_32a* __restrict__ xyz64, const float4* __restrict__ xhl,
    const double4_32a* __restrict__ u64,
    const double* __restrict__ beta64, const double* __restrict__ tab64, int64_t first,
    int64_t count, const int32_t* __restrict__ elem_list,
    const int32_t* __restrict__ blk, const int32_t* __restrict__ rowlen,
    const uint32_t* __restrict__ dir_mask, T* __restrict__ values, T* __restrict__ recX,
    T* __restrict__ recKcf, double* __restrict__ recKinv, double* __restrict__ oS,
    double* __restrict__ oKcc, double* __restrict__ oKcf, double* __restrict__ oKfc,
    double* __restrict__ oKff, unsigned int* __restrict__ flags, const double* __restrict__ tsbasis,
    const uint32_t* __restrict__ tsplan) {
  extern __shared__ __align__(16) unsigned char smem[];
  T* st = reinterpret_cast<T*>(smem);
  for (int i = threadIdx.x; i < 37 * nq; i += blockDim.x) st[i] = gtab[i];
  __syncthreads();
  const RefTab<T> tab{st, st + 8 * nq, st + 32 * nq, st + 33 * nq, st + 36 * nq};
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  uint32_t* bfrag = reinterpret_cast<uint32_t*>(smem + tan_table_bytes<T>(nq));
  unsigned char* wbase = smem + tan_table_bytes<T>(nq) + tan_bfrag_bytes<T, ENG>() +
                         (size_t)warp * tan_warp_total<T, ENG>(nq);
  WarpArea<T>& W = *reinterpret_cast<WarpArea<T>*>(wbase);
  void* tcw = nullptr;
  const void* ext0 = bfrag;
  const void* ext1 = nullptr;
  if constexpr (ENG == TS_ENGINE) {
    double* basis = reinterpret_cast<double*>(bfrag);
    for (int i = threadIdx.x; i < 4 * TS_BASIS_ROWS; i += blockDim.x) basis[i] = tsbasis[i];
    tcw = wbase + tan_warp_bytes<T, 0>(nq);
    ext0 = basis;
    ext1 = tsplan;
    __syncthreads();
  } else if constexpr (ENG != 0) {
    tc_build_b<ENG>(tab.N, tab.dN, nq, bfrag);
    tcw = wbase + tan_warp_bytes<T, 0>(nq);
    TcArea<ENG>& C = *reinterpret_cast<TcArea<ENG>*>(tcw);
    for (int i = lane; i < (TC_ROWS_D - 10) * tc_sd<ENG>(); i += 32) (&C.AD[10][0])[i] = 0.f;
    __syncthreads();
  }
  const int64_t total = (int64_t)gridDim.x * WARPS;
  for (int64_t it = (int64_t)blockIdx.x * WARPS + warp; it < count; it += total) {
    const int64_t e = elem_list ? (int64_t)elem_list[first + it] : first + it;
    tangent_element<T, ELEM_OUT, ATOMIC, 32, ENG>(lane, it, e, W, tab, tcw, ext0, ext1, u, conn, beta, nq, nut, tau, nu_e,
                                         visc_factor, xyz64, xhl, u64, beta64, tab64, blk, rowlen,
                                         dir_mask, values, recX, recKcf, recKinv, oS, oKcc, oKcf,
                                         oKfc, oKff, flags);
  }
}

// ---------------------------------------------------------------------------------------------
// Mixed precision, atomic scatter: the FP64 residual and the FP32 tangent in one persistent launch
// ---------------------------------------------------------------------------------------------
// The residual is bound by the FP64 pipe (a warp instruction occupies an SM partition's FP64 unit
// for many cycles, so one warp per partition keeps it busy) and the FP32 tangent by the latency of
// its warps. Launched as two kernels, the residual's blocks (226 registers per thread) take every
// SM and the tangent runs mostly after them. Here one CTA per SM holds both: warps 0-3 (one per
// partition) evaluate residuals, one element per thread, 32 elements per claim; warps 4-7 form
// tangents, one element per warp, FUSED_TCLAIM elements per claim. A residual warp whose queue is
// empty joins the tangent queue. The queues are two counters (zeroed before the launch); no warp
// ever waits for another.
// The tangent warps take quadrature points 16 at a time (two passes of 16 lanes for the 27-point
// rule), which halves their point records and lets the residual's store and eight warp areas fit
// in one SM's shared memory.
constexpr int FUSED_WARPS = 8, FUSED_RES_WARPS = 4, FUSED_TCLAIM = 4, FUSED_QCH = 16;
constexpr int FUSED_RES_THREADS = FUSED_RES_WARPS * 32;

__host__ __device__ inline size_t fused_res_bytes() {
  return sizeof(double) * RC_N * FUSED_RES_THREADS;
}
size_t fused_smem_bytes(int nq) {
  return fused_res_bytes() + tan_table_bytes<float>(nq) + FUSED_WARPS * tan_warp_bytes<float, FUSED_QCH>(nq);
}

template <bool TRANSIENT, bool FORCE>
__global__ void __launch_bounds__(FUSED_WARPS * 32, 1) fused_assembly_kernel(
    const double4_32a* __restrict__ xyz, const double4_32a* __restrict__ u64,
    const double4_32a* __restrict__ uprev, const int32_t* __restrict__ conn,
    const double* __restrict__ beta64, KParams kp, const QpRow* __restrict__ qp,
    double* __restrict__ elemR, const float4* __restrict__ u32, const float4* __restrict__ xhl32,
    const float* __restrict__ beta32,
    const float* __restrict__ gtab, float nut, float tau, const int32_t* __restrict__ blk,
    const int32_t* __restrict__ rowlen, const uint32_t* __restrict__ dir_mask,
    float* __restrict__ values, float* __restrict__ recX, float* __restrict__ recKcf,
    double* __restrict__ recKinv, int64_t n_elems, unsigned long long* __restrict__ queues,
    unsigned int* __restrict__ flags) {
  extern __shared__ __align__(16) unsigned char smem[];
  const int nq = kp.nq;
  float* st = reinterpret_cast<float*>(smem + fused_res_bytes());
  for (int i = threadIdx.x; i < 37 * nq; i += blockDim.x) st[i] = gtab[i];
  __syncthreads();
  const RefTab<float> tab{st, st + 8 * nq, st + 32 * nq, st + 33 * nq, st + 36 * nq};
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  if (warp < FUSED_RES_WARPS) {
    SmemStore<FUSED_RES_THREADS> C{reinterpret_cast<double (*)[FUSED_RES_THREADS]>(smem),
                                   (int)threadIdx.x};
    for (;;) {
      unsigned long long base = 0;
      if (lane == 0) base = atomicAdd(queues, 32ull);
      base = __shfl_sync(0xffffffffu, base, 0);
      if (base >= (unsigned long long)n_elems) break;
      const int64_t e = (int64_t)base + lane;
      if (e < n_elems) {
        int nd[8];
        double Rcp[32], Rf[3];
        const unsigned bad = residual_element<TRANSIENT, FORCE>(e, C, GlobalTable{qp}, kp, xyz, u64,
                                                                uprev, conn, beta64, nd, Rcp, Rf);
        if (bad) atomicOr(flags, bad);
        store_elem_residual(elemR + 36 * e, Rcp, Rf);
      }
    }
  }
  WarpArea<float>& W = *reinterpret_cast<WarpArea<float>*>(
      smem + fused_res_bytes() + tan_table_bytes<float>(nq) + warp * tan_warp_bytes<float, FUSED_QCH>(nq));
  for (;;) {
    unsigned long long base = 0;
    if (lane == 0) base = atomicAdd(queues + 1, (unsigned long long)FUSED_TCLAIM);
    base = __shfl_sync(0xffffffffu, base, 0);
    if (base >= (unsigned long long)n_elems) break;
    const int64_t end = (int64_t)base + FUSED_TCLAIM < n_elems ? (int64_t)base + FUSED_TCLAIM : n_elems;
    for (int64_t e = (int64_t)base; e < end; ++e)
      tangent_element<float, false, true, FUSED_QCH>(lane, e, e, W, tab, nullptr, nullptr, nullptr, u32, conn, beta32, nq, nut, tau,
                                          kp.nu_e, kp.visc_factor, xyz, xhl32, u64, beta64, kp.tab64, blk,
                                          rowlen, dir_mask, values, recX, recKcf, recKinv, nullptr,
                                          nullptr, nullptr, nullptr, nullptr, flags);
  }
}

int launch_fused_assembly(const Mesh& m, const State& s, const Fp32Copy& c32, const KParams& kp,
                          const QpRow* qp, const float* tab32, double* elemR, const TangentOut& o,
                          unsigned long long* queues, unsigned int* flags, cudaStream_t st) {
  if (m.n_elems <= 0) return 0;
  const size_t smem = fused_smem_bytes(kp.nq);
  auto launch = [&](auto kern) {
    cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    kern<<<(unsigned)sm_count(), FUSED_WARPS * 32, smem, st>>>(
        m.xyz, s.u, s.u_prev, m.conn, s.beta, kp, qp, elemR, c32.u, c32.xhl, c32.beta, tab32,
        (float)kp.nut, (float)kp.tau, m.blk, m.rowlen, m.dir_mask, reinterpret_cast<float*>(o.values),
        reinterpret_cast<float*>(o.recX), reinterpret_cast<float*>(o.recKcf), o.recKinv, m.n_elems,
        queues, flags);
  };
  if (kp.transient) {
    if (kp.has_force) launch(fused_assembly_kernel<true, true>);
    else launch(fused_assembly_kernel<true, false>);
  } else {
    if (kp.has_force) launch(fused_assembly_kernel<false, true>);
    else launch(fused_assembly_kernel<false, false>);
  }
  return 1;
}

// y = K_ff^-1 R_f (FP64, kept for the recovery) and r_e = R_cp - K_cf y (FP64 arithmetic on the
// stored K_cf, FP32 in mixed precision) scattered into the right-hand side. One thread per element.
template <typename T, bool ATOMIC>
__global__ void __launch_bounds__(128) finish_kernel(
    const int32_t* __restrict__ conn, const double* __restrict__ elemR, const T* __restrict__ recKcf,
    const double* __restrict__ recKinv, const uint32_t* __restrict__ dir_mask, int64_t first,
    int64_t count, const int32_t* __restrict__ elem_list, double* __restrict__ rhs,
    double* __restrict__ recY, double* __restrict__ oR) {
  const int64_t it = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (it >= count) return;
  const int64_t e = elem_list ? (int64_t)elem_list[first + it] : first + it;
  const double* R = elemR + 36 * e;
  const double Rf[3] = {R[32], R[33], R[34]};
  double y[3];
#pragma unroll
  for (int m = 0; m < 3; ++m) {
    const double* K = recKinv + 9 * e + 3 * m;
    y[m] = K[0] * Rf[0] + K[1] * Rf[1] + K[2] * Rf[2];
    recY[3 * e + m] = y[m];
  }
  const uint32_t msk = oR ? 0u : dir_mask[e];
  const T* kc = recKcf + 96 * e;
#pragma unroll 4
  for (int t = 0; t < 32; ++t) {
    const double r = R[t] - ((double)kc[3 * t] * y[0] + (double)kc[3 * t + 1] * y[1] +
                             (double)kc[3 * t + 2] * y[2]);
    if (oR) {
      oR[32 * it + t] = r;
    } else if (!(msk >> t & 1u)) {
      double* dst = rhs + 4 * (int64_t)conn[8 * e + (t >> 2)] + (t & 3);
      if (ATOMIC) atomicAdd(dst, r); else *dst += r;
    }
  }
}

// FP32 copies of the nodal state and bubble coefficients for the mixed-precision tangent, and the
// coordinates as FP32 high and low parts (x = hi + lo to about 2^-48 |x|) for its geometry.
__global__ void to_fp32_kernel(const double4_32a* __restrict__ u, const double* __restrict__ beta,
                               const double4_32a* __restrict__ xyz, float4* __restrict__ u32,
                               float* __restrict__ beta32, float4* __restrict__ xhl,
                               int64_t n_nodes, int64_t n_elems) {
  const int64_t stride = (int64_t)gridDim.x * blockDim.x;
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n_nodes; i += stride) {
    const double4_32a w = u[i];
    u32[i] = make_float4((float)w.x, (float)w.y, (float)w.z, (float)w.w);
    const double4_32a x = xyz[i];
    const float hx = (float)x.x, hy = (float)x.y, hz = (float)x.z;
    xhl[2 * i] = make_float4(hx, hy, hz, 0.f);
    xhl[2 * i + 1] = make_float4((float)(x.x - hx), (float)(x.y - hy), (float)(x.z - hz), 0.f);
  }
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < 3 * n_elems; i += stride)
    beta32[i] = (float)beta[i];
}

int launch_to_fp32(const Mesh& m, const State& s, const Fp32Copy& c, cudaStream_t st) {
  const int64_t n = m.n_nodes > 3 * m.n_elems ? m.n_nodes : 3 * m.n_elems;
  int64_t blocks = (n + 255) / 256;
  if (blocks > (int64_t)sm_count() * 8) blocks = (int64_t)sm_count() * 8;
  to_fp32_kernel<<<(unsigned)blocks, 256, 0, st>>>(s.u, s.beta, m.xyz, c.u, c.beta, c.xhl,
                                                   m.n_nodes, m.n_elems);
  return 1;
}

template <typename T, bool ELEM_OUT, bool ATOMIC, int WARPS, int ENG>
static void launch_w(const Mesh& m, const State& s, const Fp32Copy& c32, const KParams& kp,
                     const T* tab, const TangentOut& o, int64_t first, int64_t count,
                     const int32_t* elem_list, unsigned int* flags, cudaStream_t st) {
  const int nq = kp.nq;
  const size_t smem = tan_table_bytes<T>(nq) + tan_bfrag_bytes<T, ENG>() + WARPS * tan_warp_total<T, ENG>(nq);
  auto kern = tangent_kernel<T, ELEM_OUT, ATOMIC, WARPS, ENG>;
  cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  int64_t blocks = (count + WARPS - 1) / WARPS;
  if (blocks > (int64_t)sm_count() * 128) blocks = (int64_t)sm_count() * 128;
  using NV = typename NodeVec<T>::type;
  const NV* u;
  const T* beta;
  if constexpr (sizeof(T) == 4) {
    u = c32.u; beta = c32.beta;
  } else {
    u = s.u; beta = s.beta;
  }
  kern<<<(unsigned)blocks, WARPS * 32, smem, st>>>(
      u, m.conn, beta, tab, nq, T(kp.nut), T(kp.tau), kp.nu_e, kp.visc_factor, m.xyz, c32.xhl, s.u,
      s.beta, kp.tab64, first, count, elem_list, m.blk,
      m.rowlen, m.dir_mask, reinterpret_cast<T*>(o.values), reinterpret_cast<T*>(o.recX),
      reinterpret_cast<T*>(o.recKcf), o.recKinv, o.S, o.Kcc, o.Kcf, o.Kfc, o.Kff, flags, kp.ts_basis,
      kp.ts_plan);
}

// Warps per block: the default, or the tuned count when it is one of the compiled choices
// (FP32: 2, 4, 8; FP64: 1, 2, 4). Element outputs always use the default. The tensor-core
// engines (FP32 only) run TC_WARPS warps per block (their per-warp operand storage is ~28 KB).
template <typename T, bool ELEM_OUT, bool ATOMIC>
static void launch_t(const Mesh& m, const State& s, const Fp32Copy& c32, const KParams& kp,
                     const T* tab, const TangentOut& o, int64_t first, int64_t count,
                     const int32_t* elem_list, int engine, unsigned int* flags, cudaStream_t st) {
  if constexpr (sizeof(T) == 4) {
    if (engine == TC_BF16)
      return launch_w<T, ELEM_OUT, ATOMIC, TC_WARPS, TC_BF16>(m, s, c32, kp, tab, o, first, count, elem_list, flags, st);
    if (engine == TC_TF32X3)
      return launch_w<T, ELEM_OUT, ATOMIC, TC_WARPS, TC_TF32X3>(m, s, c32, kp, tab, o, first, count, elem_list, flags, st);
  }
  if constexpr (sizeof(T) == 8) {
    // FP64: weighted point sums for the 8- and 27-point rules (the tables exist), TS_WARPS per CTA
    if (kp.ts_plan && kp.nq <= 27)
      return launch_w<T, ELEM_OUT, ATOMIC, TS_WARPS, TS_ENGINE>(m, s, c32, kp, tab, o, first, count, elem_list, flags, st);
  }
  constexpr int D = tan_warps<T>();
  const int w = ELEM_OUT ? D : (kp.tangent_warps ? kp.tangent_warps : D);
  if constexpr (!ELEM_OUT) {
    if (w == D / 2) return launch_w<T, false, ATOMIC, D / 2, 0>(m, s, c32, kp, tab, o, first, count, elem_list, flags, st);
    if (w == 2 * D) return launch_w<T, false, ATOMIC, 2 * D, 0>(m, s, c32, kp, tab, o, first, count, elem_list, flags, st);
  }
  launch_w<T, ELEM_OUT, ATOMIC, D, 0>(m, s, c32, kp, tab, o, first, count, elem_list, flags, st);
}

int tangent_warp_choice(bool fp32, int k) {
  const int d = fp32 ? tan_warps<float>() : tan_warps<double>();
  return k == 0 ? d / 2 : (k == 1 ? d : 2 * d);
}

int launch_tangent(bool fp32, int engine, const Mesh& m, const State& s, const Fp32Copy& c32,
                   const KParams& kp, const void* tab, const TangentOut& out, int64_t first,
                   int64_t count, const int32_t* elem_list, bool elem_outputs, bool atomic,
                   unsigned int* flags, cudaStream_t st) {
  if (count <= 0) return 0;
  if (fp32) {
    const float* t = reinterpret_cast<const float*>(tab);
    if (elem_outputs) launch_t<float, true, true>(m, s, c32, kp, t, out, first, count, elem_list, engine, flags, st);
    else if (atomic) launch_t<float, false, true>(m, s, c32, kp, t, out, first, count, elem_list, engine, flags, st);
    else launch_t<float, false, false>(m, s, c32, kp, t, out, first, count, elem_list, engine, flags, st);
  } else {
    const double* t = reinterpret_cast<const double*>(tab);
    if (elem_outputs) launch_t<double, true, true>(m, s, c32, kp, t, out, first, count, elem_list, 0, flags, st);
    else if (atomic) launch_t<double, false, true>(m, s, c32, kp, t, out, first, count, elem_list, 0, flags, st);
    else launch_t<double, false, false>(m, s, c32, kp, t, out, first, count, elem_list, 0, flags, st);
  }
  return 1;
}

int launch_finish(bool fp32, const Mesh& m, const double* elemR, const TangentOut& o,
                  int64_t first, int64_t count, const int32_t* elem_list, bool atomic,
                  cudaStream_t st) {
  if (count <= 0) return 0;
  const unsigned blocks = (unsigned)((count + 127) / 128);
  auto go = [&](auto kern, auto* kcf) {
    kern<<<blocks, 128, 0, st>>>(m.conn, elemR, kcf, o.recKinv, m.dir_mask, first, count,
                                 elem_list, o.rhs, o.recY, o.r);
  };
  if (fp32) {
    const float* k = reinterpret_cast<const float*>(o.recKcf);
    if (atomic) go(finish_kernel<float, true>, k); else go(finish_kernel<float, false>, k);
  } else {
    const double* k = reinterpret_cast<const double*>(o.recKcf);
    if (atomic) go(finish_kernel<double, true>, k); else go(finish_kernel<double, false>, k);
  }
  return 1;
}

}  // namespace vms
