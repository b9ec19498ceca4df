// FP64 element residual kernel (Section 4.1), one thread per element; arithmetic in
// residual_math.cuh.
#include "residual_math.cuh"
#include "vms_internal.h"

namespace vms {

// Threads per block: 64 by default; the autotuner (vms_autotune) may choose 32.
constexpr int RES_THREADS = 64;

// Monomial coefficients live in shared memory, one column per thread (conflict-free).
template <int THREADS>
struct SmemStore {
  double (*sc)[THREADS];
  int tid;
  __device__ __forceinline__ double get(int k) const { return sc[k][tid]; }
  __device__ __forceinline__ void set(int k, double v) { sc[k][tid] = v; }
};

// Per-point table in global memory; every thread of a warp reads the same row (broadcast).
struct GlobalTable {
  const QpRow* __restrict__ t;
  __device__ __forceinline__ double xi(int q) const { return __ldg(&t[q].xi); }
  __device__ __forceinline__ double eta(int q) const { return __ldg(&t[q].eta); }
  __device__ __forceinline__ double zeta(int q) const { return __ldg(&t[q].zeta); }
  __device__ __forceinline__ double xe(int q) const { return __ldg(&t[q].xe); }
  __device__ __forceinline__ double xz(int q) const { return __ldg(&t[q].xz); }
  __device__ __forceinline__ double ez(int q) const { return __ldg(&t[q].ez); }
  __device__ __forceinline__ double xez(int q) const { return __ldg(&t[q].xez); }
  __device__ __forceinline__ double b(int q) const { return __ldg(&t[q].b); }
  __device__ __forceinline__ double db(int q, int al) const {
    return al == 0 ? __ldg(&t[q].db0) : (al == 1 ? __ldg(&t[q].db1) : __ldg(&t[q].db2));
  }
  __device__ __forceinline__ double w(int q) const { return __ldg(&t[q].w); }
};

template <bool TRANSIENT, bool FORCE, int THREADS>
__global__ void __launch_bounds__(THREADS) residual_kernel(
    const double4_32a* __restrict__ xyz, const double4_32a* __restrict__ u,
    const double4_32a* __restrict__ uprev, const int32_t* __restrict__ conn,
    const double* __restrict__ beta, KParams kp, const QpRow* __restrict__ qp, int64_t first,
    int64_t count,
    double* __restrict__ elemR, double* __restrict__ resid, const uint32_t* __restrict__ dir_mask,
    int64_t n_nodes, int mode, unsigned int* __restrict__ flags) {
  __shared__ double sc[RC_N][THREADS];
  const int tid = threadIdx.x;
  const int64_t t = (int64_t)blockIdx.x * THREADS + tid;
  if (t >= count) return;
  const int64_t e = first + t;

  int nd[8];
  {
    const int4* cp = reinterpret_cast<const int4*>(conn + 8 * e);
    const int4 c0 = cp[0], c1 = cp[1];
    nd[0] = c0.x; nd[1] = c0.y; nd[2] = c0.z; nd[3] = c0.w;
    nd[4] = c1.x; nd[5] = c1.y; nd[6] = c1.z; nd[7] = c1.w;
  }
  SmemStore<THREADS> C{sc, tid};
  {
    double X[8][3], U[8][4], Up[8][3];
#pragma unroll
    for (int a = 0; a < 8; ++a) {
      const double4_32a x = xyz[nd[a]];
      const double4_32a w = u[nd[a]];
      X[a][0] = x.x; X[a][1] = x.y; X[a][2] = x.z;
      U[a][0] = w.x; U[a][1] = w.y; U[a][2] = w.z; U[a][3] = w.w;
      if (TRANSIENT) {
        const double4_32a o = uprev[nd[a]];
        Up[a][0] = o.x; Up[a][1] = o.y; Up[a][2] = o.z;
      }
    }
    residual_load(C, X, U, Up, TRANSIENT);
  }
  const double bet[3] = {beta[3 * e + 0], beta[3 * e + 1], beta[3 * e + 2]};
  double Rcp[32], Rf[3];
  const double nut = kp.nu_e ? kp.visc_factor * __ldg(kp.nu_e + e) : kp.nut;
  const bool ok = residual_qp_loop<TRANSIENT, FORCE>(C, GlobalTable{qp}, kp.nq, bet, nut, kp.tau,
                                                     kp.f, Rcp, Rf);
  if (!ok) atomicOr(flags, FLAG_NEG_JACOBIAN);
  bool finite = isfinite(Rf[0]) && isfinite(Rf[1]) && isfinite(Rf[2]);
#pragma unroll
  for (int k = 0; k < 32; ++k) finite = finite && isfinite(Rcp[k]);
  if (!finite) atomicOr(flags, FLAG_NAN);

  if (mode == 0) {
    double2* out = reinterpret_cast<double2*>(elemR + 36 * e);
#pragma unroll
    for (int k = 0; k < 16; ++k) out[k] = make_double2(Rcp[2 * k], Rcp[2 * k + 1]);
    out[16] = make_double2(Rf[0], Rf[1]);
    out[17] = make_double2(Rf[2], 0.0);
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
#define VMS_RES_ARGS m.xyz, s.u, s.u_prev, m.conn, s.beta, kp, qp, first, count, elemR, resid, \
                     m.dir_mask, m.n_nodes, mode, flags
  if (kp.transient) {
    if (kp.has_force) residual_kernel<true, true, THREADS><<<grid, THREADS, 0, st>>>(VMS_RES_ARGS);
    else residual_kernel<true, false, THREADS><<<grid, THREADS, 0, st>>>(VMS_RES_ARGS);
  } else {
    if (kp.has_force) residual_kernel<false, true, THREADS><<<grid, THREADS, 0, st>>>(VMS_RES_ARGS);
    else residual_kernel<false, false, THREADS><<<grid, THREADS, 0, st>>>(VMS_RES_ARGS);
  }
#undef VMS_RES_ARGS
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
