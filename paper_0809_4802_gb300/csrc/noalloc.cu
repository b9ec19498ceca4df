// Residual norm with caller-owned memory only (vms_residual_norm_noalloc in include/vms.h).
//
// This is a variant of the FP64 residual kernel for callers that cannot allocate device memory:
// processes whose device memory is handed entirely to their own pool (a framework's caching
// allocator or a fixed arena sized at start-up), and latency-critical loops that cannot afford
// the device-wide synchronisation that cudaMalloc and cudaFree imply. It needs no context: the
// caller passes the mesh, the state and the outputs as device pointers, and the scratch space
// (the assembled residual vector, the reduction partial sums, the quadrature table and the error
// flags) lives in one file-scope device array of fixed size. Every GPU that loads the library
// holds that array (VMS_NOALLOC_SCRATCH_BYTES) until the process exits.
#include <mutex>

#include "residual_math.cuh"
#include "vms_internal.h"

namespace vms {
namespace {

// scratch layout, in doubles: the assembled residual (at most VMS_NOALLOC_MAX_ENTRIES entries),
// the partial sums of its squares, the quadrature table (QpRow = 12 doubles per point), the
// error flags
constexpr int64_t NA_MAX = VMS_NOALLOC_MAX_ENTRIES;
constexpr int NA_BLOCKS = 512, NA_THREADS = 256;
constexpr int64_t NA_PART = NA_MAX;
constexpr int64_t NA_QP = NA_PART + NA_BLOCKS;
constexpr int64_t NA_FLAGS = NA_QP + (int64_t)MAX_QP * 12;
constexpr int64_t NA_TOTAL = NA_FLAGS + 4;
constexpr unsigned int NA_FLAG_INDEX = 8u;  // a node or dof index outside the mesh
static_assert(sizeof(QpRow) == 12 * sizeof(double), "QpRow layout");
static_assert(NA_TOTAL * 8 <= VMS_NOALLOC_SCRATCH_BYTES, "scratch size");

static __device__ __align__(256) double g_noalloc_scratch[VMS_NOALLOC_SCRATCH_BYTES / 8];

// Device address of the scratch array, looked up once per device (with that device current).
constexpr int NA_MAX_DEVICES = 64;
double* g_scratch_addr[NA_MAX_DEVICES] = {};
std::mutex g_scratch_mu;

cudaError_t scratch_address(int dev, double** out) {
  if (dev < 0 || dev >= NA_MAX_DEVICES) return cudaErrorInvalidDevice;
  std::lock_guard<std::mutex> lock(g_scratch_mu);
  if (!g_scratch_addr[dev]) {
    void* p = nullptr;
    const cudaError_t e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
    if (e != cudaSuccess) return e;
    g_scratch_addr[dev] = static_cast<double*>(p);
  }
  *out = g_scratch_addr[dev];
  return cudaSuccess;
}

__global__ void na_zero_kernel(double* __restrict__ p, int64_t n) {
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n;
       i += (int64_t)gridDim.x * blockDim.x)
    p[i] = 0.0;
}

struct NaStore {
  double (*sc)[64];
  int tid;
  __device__ __forceinline__ double get(int k) const { return sc[k][tid]; }
  __device__ __forceinline__ void set(int k, double v) const { sc[k][tid] = v; }
};

// The quadrature table is written by a kernel queued before the residual kernel, which only reads it.
struct NaTable {
  const QpRow* __restrict__ t;
  __device__ __forceinline__ double xi(int q) const { return __ldg(&t[q].xi); }
  __device__ __forceinline__ double eta(int q) const { return __ldg(&t[q].eta); }
  __device__ __forceinline__ double zeta(int q) const { return __ldg(&t[q].zeta); }
  __device__ __forceinline__ double ez(int q) const { return __ldg(&t[q].ez); }
  __device__ __forceinline__ double b(int q) const { return __ldg(&t[q].b); }
  __device__ __forceinline__ double db(int q, int al) const {
    return al == 0 ? __ldg(&t[q].db0) : (al == 1 ? __ldg(&t[q].db1) : __ldg(&t[q].db2));
  }
  __device__ __forceinline__ double w(int q) const { return __ldg(&t[q].w); }
};

// Same arithmetic as the residual kernel (residual_math.cuh); plain row-major inputs.
template <bool TRANSIENT, bool FORCE>
__global__ void __launch_bounds__(64) na_residual_kernel(
    const double* __restrict__ xyz, const double* __restrict__ u, const double* __restrict__ uprev,
    const int32_t* __restrict__ conn, const double* __restrict__ beta, KParams kp,
    int64_t n_nodes, int64_t n_elems, double* __restrict__ scratch) {
  extern __shared__ __align__(16) unsigned char na_smem[];
  double (*sc)[64] = reinterpret_cast<double (*)[64]>(na_smem);
  const int tid = threadIdx.x;
  const int64_t e = (int64_t)blockIdx.x * 64 + tid;
  if (e >= n_elems) return;
  unsigned int* flags = reinterpret_cast<unsigned int*>(scratch + NA_FLAGS);
  int nd[8];
  bool in_range = true;
#pragma unroll
  for (int a = 0; a < 8; ++a) {
    nd[a] = conn[8 * e + a];
    in_range = in_range && nd[a] >= 0 && nd[a] < n_nodes;
  }
  if (!in_range) {  // out-of-range node index: skip the element and report it
    atomicOr(flags, NA_FLAG_INDEX);
    return;
  }
  NaStore C{sc, tid};
  {
    // gather one field at a time into the monomial coefficients (same slots as residual_load)
    double f[8], c[8];
#pragma unroll
    for (int i = 0; i < 3; ++i) {
#pragma unroll
      for (int a = 0; a < 8; ++a) f[a] = xyz[3 * (int64_t)nd[a] + i];
      modal8(f, c);
#pragma unroll
      for (int m = 1; m < 8; ++m) C.set(RC_X + 7 * i + m - 1, 0.125 * c[m]);
    }
#pragma unroll
    for (int i = 0; i < 4; ++i) {
#pragma unroll
      for (int a = 0; a < 8; ++a) f[a] = u[4 * (int64_t)nd[a] + i];
      modal8(f, c);
      const int base = i < 3 ? RC_V + 8 * i : RC_P;
#pragma unroll
      for (int m = 0; m < 8; ++m) C.set(base + m, 0.125 * c[m]);
      if (TRANSIENT && i < 3) {
#pragma unroll
        for (int a = 0; a < 8; ++a) f[a] -= uprev[4 * (int64_t)nd[a] + i];
        modal8(f, c);
#pragma unroll
        for (int m = 0; m < 8; ++m) C.set(RC_DV + 8 * i + m, 0.125 * c[m]);
      }
    }
  }
  const double bet[3] = {beta ? beta[3 * e] : 0.0, beta ? beta[3 * e + 1] : 0.0,
                         beta ? beta[3 * e + 2] : 0.0};
  double Rcp[32], Rf[3];
  const bool ok = residual_qp_loop<TRANSIENT, FORCE>(
      C, NaTable{reinterpret_cast<const QpRow*>(scratch + NA_QP)}, kp.nq, bet, kp.nut, kp.tau,
      kp.f, Rcp, Rf);
  if (!ok) atomicOr(flags, FLAG_NEG_JACOBIAN);
  bool finite = isfinite(Rf[0]) && isfinite(Rf[1]) && isfinite(Rf[2]);
#pragma unroll
  for (int k = 0; k < 32; ++k) finite = finite && isfinite(Rcp[k]);
  if (!finite) atomicOr(flags, FLAG_NAN);
#pragma unroll
  for (int a = 0; a < 8; ++a)
#pragma unroll
    for (int c = 0; c < 4; ++c) atomicAdd(scratch + 4 * (int64_t)nd[a] + c, Rcp[4 * a + c]);
  double* rf = scratch + 4 * n_nodes + 3 * e;
  rf[0] = Rf[0]; rf[1] = Rf[1]; rf[2] = Rf[2];
}

__global__ void na_zero_dofs_kernel(const int64_t* __restrict__ dofs, int64_t n, int64_t n_coarse,
                                    double* __restrict__ scratch) {
  const int64_t k = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (k >= n) return;
  const int64_t d = dofs[k];
  if (d >= 0 && d < n_coarse) scratch[d] = 0.0;
  else atomicOr(reinterpret_cast<unsigned int*>(scratch + NA_FLAGS), NA_FLAG_INDEX);
}

__device__ __forceinline__ double na_block_sum(double v) {
  __shared__ double sh[NA_THREADS / 32];
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
  if (lane == 0) sh[w] = v;
  __syncthreads();
  v = threadIdx.x < NA_THREADS / 32 ? sh[threadIdx.x] : 0.0;
  if (w == 0)
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  return v;
}

__global__ void __launch_bounds__(NA_THREADS) na_sumsq_kernel(int64_t n, double* __restrict__ scratch) {
  double s = 0.0;
  for (int64_t i = (int64_t)blockIdx.x * NA_THREADS + threadIdx.x; i < n;
       i += (int64_t)NA_BLOCKS * NA_THREADS)
    s = fma(scratch[i], scratch[i], s);
  s = na_block_sum(s);
  if (threadIdx.x == 0) scratch[NA_PART + blockIdx.x] = s;
}

__global__ void __launch_bounds__(NA_THREADS) na_finish_kernel(const double* __restrict__ scratch,
                                                               double* __restrict__ norm,
                                                               int32_t* __restrict__ status) {
  double s = 0.0;
  for (int i = threadIdx.x; i < NA_BLOCKS; i += NA_THREADS) s += scratch[NA_PART + i];
  s = na_block_sum(s);
  if (threadIdx.x == 0) {
    *norm = sqrt(s);
    const unsigned int f = *reinterpret_cast<const unsigned int*>(scratch + NA_FLAGS);
    *status = (f & NA_FLAG_INDEX) ? VMS_ERR_INVALID_ARG
            : (f & FLAG_NEG_JACOBIAN) ? VMS_ERR_NEG_JACOBIAN
            : (f & FLAG_NAN) ? VMS_ERR_NAN : VMS_OK;
  }
}

// The quadrature table (the same rule as the context's tables), written on the device from the
// rule's order and the bubble scale passed by value: no host memory is read by the queued work.
__global__ void na_table_kernel(int n1, double bubble_scale, QpRow* __restrict__ rows) {
  double x[4], w[4];
  if (n1 == 2) {
    const double a = 1.0 / sqrt(3.0);
    x[0] = -a; x[1] = a; w[0] = w[1] = 1.0;
  } else if (n1 == 3) {
    const double a = sqrt(0.6);
    x[0] = -a; x[1] = 0.0; x[2] = a;
    w[0] = 5.0 / 9.0; w[1] = 8.0 / 9.0; w[2] = 5.0 / 9.0;
  } else {
    const double r = 2.0 / 7.0 * sqrt(6.0 / 5.0);
    const double a = sqrt(3.0 / 7.0 - r), b = sqrt(3.0 / 7.0 + r);
    x[0] = -b; x[1] = -a; x[2] = a; x[3] = b;
    w[0] = w[3] = (18.0 - sqrt(30.0)) / 36.0;
    w[1] = w[2] = (18.0 + sqrt(30.0)) / 36.0;
  }
  const int q = threadIdx.x;
  if (q >= n1 * n1 * n1) return;
  const int i = q % n1, j = (q / n1) % n1, k = q / (n1 * n1);
  QpRow& r = rows[q];
  const double p0 = x[i], p1 = x[j], p2 = x[k];
  r.xi = p0; r.eta = p1; r.zeta = p2;
  r.xe = p0 * p1; r.xz = p0 * p2; r.ez = p1 * p2; r.xez = p0 * p1 * p2;
  const double f0 = 1 - p0 * p0, f1 = 1 - p1 * p1, f2 = 1 - p2 * p2;
  r.b = bubble_scale * f0 * f1 * f2;
  r.db0 = bubble_scale * (-2 * p0) * f1 * f2;
  r.db1 = bubble_scale * (-2 * p1) * f0 * f2;
  r.db2 = bubble_scale * (-2 * p2) * f0 * f1;
  r.w = w[i] * w[j] * w[k];
}

}  // namespace
}  // namespace vms

using namespace vms;

extern "C" int vms_residual_norm_noalloc(int64_t n_nodes, const double* xyz, int64_t n_elems,
                                         const int32_t* conn, int64_t n_dir,
                                         const int64_t* dir_dof, const double* u,
                                         const double* beta, const double* u_prev,
                                         const vms_params* params, double* norm,
                                         int32_t* status, void* stream) {
  if (!xyz || !conn || !u || !params || !norm || !status || (n_dir > 0 && !dir_dof) ||
      n_nodes <= 0 || n_elems <= 0 || n_dir < 0)
    return VMS_ERR_INVALID_ARG;
  const vms_params& p = *params;
  if (!(p.nu > 0.0) || !(p.visc_factor > 0.0) || !(p.dt >= 0.0) || !(p.bubble_scale != 0.0) ||
      p.quad_order < 2 || p.quad_order > 4)
    return VMS_ERR_INVALID_ARG;
  if (n_nodes > NA_MAX / 4 || 4 * n_nodes + 3 * n_elems > NA_MAX) return VMS_ERR_TOO_LARGE;
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess) return VMS_ERR_CUDA;
  double* scratch = nullptr;
  if (scratch_address(dev, &scratch) != cudaSuccess) return VMS_ERR_CUDA;
  cudaStream_t st = reinterpret_cast<cudaStream_t>(stream);

  KParams kp{};
  kp.nut = p.visc_factor * p.nu;
  kp.tau = p.dt > 0 ? 1.0 / p.dt : 0.0;
  for (int i = 0; i < 3; ++i) kp.f[i] = p.f[i];
  kp.nq = p.quad_order * p.quad_order * p.quad_order;
  kp.transient = p.dt > 0 ? 1 : 0;
  kp.has_force = (p.f[0] != 0.0 || p.f[1] != 0.0 || p.f[2] != 0.0) ? 1 : 0;

  // the array keeps the previous call's contents: clear the residual, partials and flags
  const int64_t n = 4 * n_nodes + 3 * n_elems;
  na_zero_kernel<<<4 * sm_count(), 256, 0, st>>>(scratch, n);
  na_zero_kernel<<<1, 256, 0, st>>>(scratch + NA_PART, NA_BLOCKS);
  na_zero_kernel<<<1, 32, 0, st>>>(scratch + NA_FLAGS, 4);
  na_table_kernel<<<1, MAX_QP, 0, st>>>(p.quad_order, p.bubble_scale,
                                        reinterpret_cast<QpRow*>(scratch + NA_QP));
  const unsigned eb = (unsigned)((n_elems + 63) / 64);
  const double* up = u_prev ? u_prev : u;
  const size_t smem = sizeof(double) * RC_N * 64;  // the coefficient store (above 48 KB)
  auto launch = [&](auto kern) {
    cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    kern<<<eb, 64, smem, st>>>(xyz, u, up, conn, beta, kp, n_nodes, n_elems, scratch);
  };
  if (kp.transient) {
    if (kp.has_force) launch(na_residual_kernel<true, true>);
    else launch(na_residual_kernel<true, false>);
  } else {
    if (kp.has_force) launch(na_residual_kernel<false, true>);
    else launch(na_residual_kernel<false, false>);
  }
  if (n_dir > 0)
    na_zero_dofs_kernel<<<(unsigned)((n_dir + 255) / 256), 256, 0, st>>>(dir_dof, n_dir, 4 * n_nodes, scratch);
  na_sumsq_kernel<<<NA_BLOCKS, NA_THREADS, 0, st>>>(n, scratch);
  na_finish_kernel<<<1, NA_THREADS, 0, st>>>(scratch, norm, status);
  return cudaGetLastError() == cudaSuccess ? VMS_OK : VMS_ERR_CUDA;
}
