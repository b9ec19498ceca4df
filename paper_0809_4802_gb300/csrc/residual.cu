// FP64 element residual kernel (Section 4.1), one thread per element; arithmetic in
// residual_math.cuh.
#include "residual_math.cuh"
#include "residual_table.cuh"
#include "vms_internal.h"

namespace vms {

// Threads per block: 64 by default; the autotuner (vms_autotune) may choose 32.
constexpr int RES_THREADS = 64;
static_assert(FLAG_NEG_JACOBIAN == 1u && FLAG_NAN == 4u, "residual_element error bits");

template <bool TRANSIENT, bool FORCE, int THREADS>
__global__ void __launch_bounds__(THREADS) residual_kernel(
    const double4_32a* __restrict__ xyz, const double4_32a* __restrict__ u,
    const double4_32a* __restrict__ uprev, const int32_t* __restrict__ conn,
    const double* __restrict__ beta, KParams kp, const QpRow* __restrict__ qp, int64_t first,
    int64_t count,
    double* __restrict__ elemR, double* __restrict__ resid, const uint32_t* __restrict__ dir_mask,
    int64_t n_nodes, int mode, unsigned int* __restrict__ flags) {
  extern __shared__ __align__(16) unsigned char res_smem[];
  double (*sc)[THREADS] = reinterpret_cast<double (*)[THREADS]>(res_smem);
  const int tid = threadIdx.x;
  const int64_t t = (int64_t)blockIdx.x * THREADS + tid;
  if (t >= count) return;
  const int64_t e = first + t;

  int nd[8];
  SmemStore<THREADS> C{sc, tid};
  double Rcp[32], Rf[3];
  const unsigned bad = residual_element<TRANSIENT, FORCE>(e, C, GlobalTable{qp}, kp, xyz, u, uprev,
                                                          conn, beta, nd, Rcp, Rf);
  if (bad) atomicOr(flags, bad);  // bits 1 and 4: FLAG_NEG_JACOBIAN, FLAG_NAN
  if (mode == 0) {
    store_elem_residual(elemR + 36 * e, Rcp, Rf);
  } else {
    const uint32_t msk = dir_mask[e];
#pragma unroll
    for (int a = 0; a < 8; ++a)
#pragma unroll
      for (int c = 0; c < 4; ++c)
        if (!(msk >> (4 * a + c) & 1u)) atomicAdd(resid + 4 * (int64_t)nd[a] + c, Rcp[4 * a + c]);
    double* rf = resid + 4 * n_nodes + 3 * e;
    rf[0] = Rf[0]; rf[1] = Rf[1]; rf[2] = Rf[2];
  }
}

template <int THREADS>
static void launch_r(const Mesh& m, const State& s, const KParams& kp, const QpRow* qp,
                     double* elemR, double* resid, int64_t first, int64_t count, int mode,
                     unsigned int* flags, cudaStream_t st) {
  const dim3 grid((unsigned)((count + THREADS - 1) / THREADS));
  const size_t smem = sizeof(double) * RC_N * THREADS;  // the coefficient store: above 48 KB at 64
  auto launch = [&](auto kern) {
    cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    kern<<<grid, THREADS, smem, st>>>(m.xyz, s.u, s.u_prev, m.conn, s.beta, kp, qp, first, count,
                                      elemR, resid, m.dir_mask, m.n_nodes, mode, flags);
  };
  if (kp.transient) {
    if (kp.has_force) launch(residual_kernel<true, true, THREADS>);
    else launch(residual_kernel<true, false, THREADS>);
  } else {
    if (kp.has_force) launch(residual_kernel<false, true, THREADS>);
    else launch(residual_kernel<false, false, THREADS>);
  }
}

int launch_residual(const Mesh& m, const State& s, const KParams& kp, const QpRow* qp,
                     double* elemR, double* resid, int64_t first, int64_t count, int mode,
                     unsigned int* flags, cudaStream_t st) {
  if (count <= 0) return 0;
  if (kp.residual_threads == 32)
    launch_r<32>(m, s, kp, qp, elemR, resid, first, count, mode, flags, st);
  else
    launch_r<RES_THREADS>(m, s, kp, qp, elemR, resid, first, count, mode, flags, st);
  return 1;
}

}  // namespace vms
