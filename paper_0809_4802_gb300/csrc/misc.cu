// Small kernels around the assembly: zero fill, Dirichlet rows/columns (Eq. SC_VelocityBC with
// zero Newton increments on constrained dofs), state imposition and a deterministic 2-norm.
#include "vms_internal.h"

namespace vms {

__global__ void fill_zero_kernel(uint4* __restrict__ p, size_t n16) {
  const size_t stride = (size_t)gridDim.x * blockDim.x;
  for (size_t i = (size_t)blockIdx.x * blockDim.x + threadIdx.x; i < n16; i += stride)
    p[i] = make_uint4(0u, 0u, 0u, 0u);
}
__global__ void fill_zero_tail(unsigned char* __restrict__ p, size_t n) {
  const size_t i = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i < n) p[i] = 0;
}

int launch_fill_zero(void* p, size_t bytes, cudaStream_t st) {
  if (bytes == 0) return 0;
  const size_t n16 = bytes / 16;
  int n = 0;
  if (n16) {
    ++n;
    size_t blocks = (n16 + 255) / 256;
    if (blocks > 152 * 16) blocks = 152 * 16;
    fill_zero_kernel<<<(unsigned)blocks, 256, 0, st>>>(reinterpret_cast<uint4*>(p), n16);
  }
  const size_t tail = bytes - 16 * n16;
  if (tail) {
    ++n;
    fill_zero_tail<<<1, 256, 0, st>>>(reinterpret_cast<unsigned char*>(p) + 16 * n16, tail);
  }
  return n;
}

// Constrained dofs: unit diagonal and zero right-hand side (rows and columns were skipped by the
// scatter, so they hold zeros).
template <typename T>
__global__ void dirichlet_diag_kernel(const int64_t* __restrict__ pos, const int64_t* __restrict__ dofs,
                                      int64_t n, T* __restrict__ values, double* __restrict__ rhs) {
  const int64_t k = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (k >= n) return;
  values[pos[k]] = T(1);
  rhs[dofs[k]] = 0.0;
}

int launch_dirichlet_diag(const Mesh& m, void* values, bool fp32, double* rhs, cudaStream_t st) {
  if (m.n_dir == 0) return 0;
  const unsigned blocks = (unsigned)((m.n_dir + 255) / 256);
  if (fp32)
    dirichlet_diag_kernel<float><<<blocks, 256, 0, st>>>(m.diag_pos, m.dir_dof, m.n_dir, reinterpret_cast<float*>(values), rhs);
  else
    dirichlet_diag_kernel<double><<<blocks, 256, 0, st>>>(m.diag_pos, m.dir_dof, m.n_dir, reinterpret_cast<double*>(values), rhs);
  return 1;
}

__global__ void zero_dofs_kernel(const int64_t* __restrict__ dofs, int64_t n, double* __restrict__ v) {
  const int64_t k = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (k < n) v[dofs[k]] = 0.0;
}
int launch_zero_dofs(const int64_t* dofs, int64_t n, double* v, cudaStream_t st) {
  if (n == 0) return 0;
  zero_dofs_kernel<<<(unsigned)((n + 255) / 256), 256, 0, st>>>(dofs, n, v);
  return 1;
}

__global__ void impose_kernel(const int64_t* __restrict__ dofs, const double* __restrict__ vals,
                              int64_t n, double* __restrict__ u) {
  const int64_t k = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (k < n) u[dofs[k]] = vals[k];
}
int launch_impose(const Mesh& m, double4_32a* u, cudaStream_t st) {
  if (m.n_dir == 0) return 0;
  impose_kernel<<<(unsigned)((m.n_dir + 255) / 256), 256, 0, st>>>(m.dir_dof, m.dir_val, m.n_dir,
                                                                   reinterpret_cast<double*>(u));
  return 1;
}

// Two-pass sum of squares with a fixed reduction tree (bitwise reproducible run to run).
constexpr int NORM_BLOCKS = 512, NORM_THREADS = 256;

__device__ __forceinline__ double block_sum(double v) {
  __shared__ double sh[NORM_THREADS / 32];
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
  if (lane == 0) sh[w] = v;
  __syncthreads();
  if (w == 0) {
    v = lane < NORM_THREADS / 32 ? sh[lane] : 0.0;
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  }
  return v;
}

__global__ void __launch_bounds__(NORM_THREADS) sumsq_pass1(const double* __restrict__ v, int64_t n,
                                                            double* __restrict__ partial) {
  double s = 0.0;
  for (int64_t i = (int64_t)blockIdx.x * NORM_THREADS + threadIdx.x; i < n;
       i += (int64_t)NORM_BLOCKS * NORM_THREADS)
    s = fma(v[i], v[i], s);
  s = block_sum(s);
  if (threadIdx.x == 0) partial[blockIdx.x] = s;
}
__global__ void __launch_bounds__(NORM_THREADS) sumsq_pass2(const double* __restrict__ partial,
                                                            double* __restrict__ out) {
  double s = 0.0;
  for (int i = threadIdx.x; i < NORM_BLOCKS; i += NORM_THREADS) s += partial[i];
  s = block_sum(s);
  if (threadIdx.x == 0) *out = s;
}

int launch_norm2(const double* v, int64_t n, double* partial, double* out, cudaStream_t st) {
  sumsq_pass1<<<NORM_BLOCKS, NORM_THREADS, 0, st>>>(v, n, partial);
  sumsq_pass2<<<1, NORM_THREADS, 0, st>>>(partial, out);
  return 2;
}

}  // namespace vms
