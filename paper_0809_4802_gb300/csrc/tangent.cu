// Element tangent, Schur condensation and scatter-add into the CSR system (Sections 4.2 and 5).
// One warp per element; the phases are in tangent_math.cuh.
#include "tangent_math.cuh"
#include "vms_internal.h"

namespace vms {

constexpr int TAN_WARPS = 4;

template <typename T>
__host__ __device__ inline size_t tan_warp_bytes(int nq) {
  int qc = nq < 32 ? nq : 32;
  size_t b = offsetof(WarpArea<T>, qp) + (size_t)qc * sizeof(QpRec<T>);
  return (b + 15) & ~size_t(15);
}
template <typename T>
__host__ __device__ inline size_t tan_table_bytes(int nq) {
  return ((size_t)37 * nq * sizeof(T) + 15) & ~size_t(15);
}

__device__ __forceinline__ void scatter_add(float* p, float v, bool atomic) {
  if (atomic) atomicAdd(p, v); else *p += v;
}
__device__ __forceinline__ void scatter_add(double* p, double v, bool atomic) {
  if (atomic) atomicAdd(p, v); else *p += v;
}

template <typename T, bool ELEM_OUT, bool ATOMIC>
__global__ void __launch_bounds__(TAN_WARPS * 32) tangent_kernel(
    const double4_32a* __restrict__ xyz, const double4_32a* __restrict__ u,
    const int32_t* __restrict__ conn, const double* __restrict__ beta,
    const double* __restrict__ elemR, const T* __restrict__ gtab, int nq, T nut, T tau,
    int64_t first, int64_t count, const int32_t* __restrict__ elem_list,
    const int32_t* __restrict__ blk, const int32_t* __restrict__ rowlen,
    const uint32_t* __restrict__ dir_mask, T* __restrict__ values, double* __restrict__ rhs,
    T* __restrict__ recX, double* __restrict__ recY, double* __restrict__ oS,
    double* __restrict__ oR, double* __restrict__ oKcc, double* __restrict__ oKcf,
    double* __restrict__ oKfc, double* __restrict__ oKff, unsigned int* __restrict__ flags) {
  extern __shared__ __align__(16) unsigned char smem[];
  T* st = reinterpret_cast<T*>(smem);
  for (int i = threadIdx.x; i < 37 * nq; i += blockDim.x) st[i] = gtab[i];
  __syncthreads();
  const RefTab<T> tab{st, st + 8 * nq, st + 32 * nq, st + 33 * nq, st + 36 * nq};
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  WarpArea<T>& W = *reinterpret_cast<WarpArea<T>*>(smem + tan_table_bytes<T>(nq) +
                                                   warp * tan_warp_bytes<T>(nq));
  const int64_t total = (int64_t)gridDim.x * TAN_WARPS;
  for (int64_t it = (int64_t)blockIdx.x * TAN_WARPS + warp; it < count; it += total) {
    const int64_t e = elem_list ? (int64_t)elem_list[first + it] : first + it;
    // gather (a1): 8 nodes and the bubble coefficients
    if (lane < 8) {
      const int nd = conn[8 * e + lane];
      W.nd[lane] = nd;
      const double4_32a x = xyz[nd];
      const double4_32a w = u[nd];
      W.X[lane][0] = T(x.x); W.X[lane][1] = T(x.y); W.X[lane][2] = T(x.z);
      W.V[lane][0] = T(w.x); W.V[lane][1] = T(w.y); W.V[lane][2] = T(w.z);
    } else if (lane < 11) {
      W.beta[lane - 8] = T(beta[3 * e + lane - 8]);
    } else if (lane == 11) {
      W.flag = 0u;
    }
    const double Rl = elemR[36 * e + lane];
    const double Rf[3] = {elemR[36 * e + 32], elemR[36 * e + 33], elemR[36 * e + 34]};
    __syncwarp();
    LaneAcc<T> A;
    tan_zero(A);
    for (int q0 = 0; q0 < nq; q0 += 32) {
      tan_phase1(lane, q0, nq, W, tab, nut, tau, A);
      __syncwarp();
      tan_phase2(lane, q0, nq - q0 < 32 ? nq - q0 : 32, W, tab, nut, tau, A);
      __syncwarp();
    }
    const int a0 = lane >> 3, a1 = a0 + 4, b = lane & 7;
    if (ELEM_OUT) {
      double* K = oKcc ? oKcc + 1024 * it : nullptr;
      if (K) {
#pragma unroll
        for (int i = 0; i < 4; ++i)
#pragma unroll
          for (int k = 0; k < 4; ++k) {
            K[(4 * a0 + i) * 32 + 4 * b + k] = (double)A.K0[4 * i + k];
            K[(4 * a1 + i) * 32 + 4 * b + k] = (double)A.K1[4 * i + k];
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
    tan_phase3c(lane, W, Rf);
    __syncwarp();
    tan_phase3d(lane, W, A, Rl);
    __syncwarp();
    tan_phase3e(lane, W, A);
    // data for the fine-scale recovery: K_ff^-1 K_fc and K_ff^-1 R_f
    if (recX) {
#pragma unroll
      for (int m = 0; m < 3; ++m) recX[96 * e + 32 * m + lane] = W.Xs[m][lane];
      if (lane < 3) recY[3 * e + lane] = W.y[lane];
    }
    if (ELEM_OUT) {
      if (oS) {
        double* S = oS + 1024 * it;
#pragma unroll
        for (int i = 0; i < 4; ++i)
#pragma unroll
          for (int k = 0; k < 4; ++k) {
            S[(4 * a0 + i) * 32 + 4 * b + k] = (double)A.K0[4 * i + k];
            S[(4 * a1 + i) * 32 + 4 * b + k] = (double)A.K1[4 * i + k];
          }
      }
      if (oR) oR[32 * it + lane] = A.r;
      if (oKff && lane < 9) oKff[9 * it + lane] = W.Kff[lane];
    } else {
      // scatter-add (a7), skipping constrained rows and columns (a8 is completed by the
      // diagonal kernel)
      const uint32_t msk = dir_mask[e];
      const int32_t* bk = blk + 64 * e;
#pragma unroll
      for (int p = 0; p < 2; ++p) {
        const int a = p ? a1 : a0;
        const T* Kp = p ? A.K1 : A.K0;
        const int32_t off = bk[8 * a + b];
        const int32_t rl = rowlen[W.nd[a]];
#pragma unroll
        for (int i = 0; i < 4; ++i) {
          if (msk >> (4 * a + i) & 1u) continue;
#pragma unroll
          for (int k = 0; k < 4; ++k) {
            if (msk >> (4 * b + k) & 1u) continue;
            scatter_add(values + off + (int64_t)i * rl + k, Kp[4 * i + k], ATOMIC);
          }
        }
      }
      if (!(msk >> lane & 1u)) scatter_add(rhs + 4 * (int64_t)W.nd[lane >> 2] + (lane & 3), A.r, ATOMIC);
    }
    __syncwarp();
    // flag bits 1 (det J <= 0) and 2 (singular K_ff) coincide with FLAG_NEG_JACOBIAN/SINGULAR_KFF
    if (lane == 0 && W.flag) atomicOr(flags, W.flag);
    __syncwarp();
  }
}

template <typename T, bool ELEM_OUT, bool ATOMIC>
static void launch_t(const Mesh& m, const State& s, const KParams& kp, const T* tab,
                     const double* elemR, const TangentOut& o, int64_t first, int64_t count,
                     const int32_t* elem_list, unsigned int* flags, cudaStream_t st) {
  const int nq = kp.nq;
  const size_t smem = tan_table_bytes<T>(nq) + TAN_WARPS * tan_warp_bytes<T>(nq);
  auto kern = tangent_kernel<T, ELEM_OUT, ATOMIC>;
  cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  int64_t blocks = (count + TAN_WARPS - 1) / TAN_WARPS;
  if (blocks > 152 * 64) blocks = 152 * 64;
  kern<<<(unsigned)blocks, TAN_WARPS * 32, smem, st>>>(
      m.xyz, s.u, m.conn, s.beta, elemR, tab, nq, T(kp.nut), T(kp.tau), first, count, elem_list,
      m.blk, m.rowlen, m.dir_mask, reinterpret_cast<T*>(o.values), o.rhs,
      reinterpret_cast<T*>(o.recX), o.recY, o.S, o.r, o.Kcc, o.Kcf, o.Kfc, o.Kff, flags);
}

int launch_tangent(bool fp32, const Mesh& m, const State& s, const KParams& kp,
                    const void* tab, const double* elemR, const TangentOut& out, int64_t first,
                    int64_t count, const int32_t* elem_list, bool elem_outputs, bool atomic,
                    unsigned int* flags, cudaStream_t st) {
  if (count <= 0) return 0;
  if (fp32) {
    const float* t = reinterpret_cast<const float*>(tab);
    if (elem_outputs) launch_t<float, true, true>(m, s, kp, t, elemR, out, first, count, elem_list, flags, st);
    else if (atomic) launch_t<float, false, true>(m, s, kp, t, elemR, out, first, count, elem_list, flags, st);
    else launch_t<float, false, false>(m, s, kp, t, elemR, out, first, count, elem_list, flags, st);
  } else {
    const double* t = reinterpret_cast<const double*>(tab);
    if (elem_outputs) launch_t<double, true, true>(m, s, kp, t, elemR, out, first, count, elem_list, flags, st);
    else if (atomic) launch_t<double, false, true>(m, s, kp, t, elemR, out, first, count, elem_list, flags, st);
    else launch_t<double, false, false>(m, s, kp, t, elemR, out, first, count, elem_list, flags, st);
  }
  return 1;
}

}  // namespace vms
