// Small kernels around the assembly: zero fill, Dirichlet rows/columns (Eq. SC_VelocityBC with
// zero Newton increments on constrained dofs), state imposition and a deterministic 2-norm.
#include "vms_internal.h"

namespace vms {

int sm_count() {
  constexpr int MAX_DEVICES = 64;
  static int counts[MAX_DEVICES] = {};  // 0: not looked up yet (every lookup writes the same value)
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= MAX_DEVICES) return 1;
  if (!counts[dev]) {
    int n = 0;
    if (cudaDeviceGetAttribute(&n, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess || n < 1) return 1;
    counts[dev] = n;
  }
  return counts[dev];
}

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
    if (blocks > (size_t)sm_count() * 16) blocks = (size_t)sm_count() * 16;
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

// ---- arithmetic throughput probe (vms_fma_throughput) ----------------------------------------
namespace vms {
constexpr int FMA_CHAINS = 8;     // independent accumulators per thread

template <typename T>
__device__ __forceinline__ T fma_step(T a, T x, T c) { return fma(a, x, c); }
template <>
__device__ __forceinline__ float fma_step<float>(float a, float x, float c) { return __fmaf_rn(a, x, c); }
template <>
__device__ __forceinline__ float2 fma_step<float2>(float2 a, float2 x, float2 c) { return __ffma2_rn(a, x, c); }

template <typename T> __device__ __forceinline__ T splat(float v);
template <> __device__ __forceinline__ double splat<double>(float v) { return (double)v; }
template <> __device__ __forceinline__ float splat<float>(float v) { return v; }
template <> __device__ __forceinline__ float2 splat<float2>(float v) { return make_float2(v, v); }
__device__ __forceinline__ bool is_one(double v) { return v == 1.0; }
__device__ __forceinline__ bool is_one(float v) { return v == 1.0f; }
__device__ __forceinline__ bool is_one(float2 v) { return v.x == 1.0f && v.y == 1.0f; }

// Each thread runs FMA_CHAINS independent chains x <- a x + c (a < 1: no overflow); the result is
// stored only if it is exactly one, which it never is, so the work cannot be removed.
template <typename T>
__global__ void __launch_bounds__(256) fma_probe_kernel(float a, float c, int steps, T* out) {
  T x[FMA_CHAINS];
  const T av = splat<T>(a), cv = splat<T>(c);
#pragma unroll
  for (int k = 0; k < FMA_CHAINS; ++k) x[k] = splat<T>(0.001f * (float)(threadIdx.x + k));
  for (int s = 0; s < steps; ++s)
#pragma unroll
    for (int k = 0; k < FMA_CHAINS; ++k) x[k] = fma_step<T>(av, x[k], cv);
  T t = x[0];
#pragma unroll
  for (int k = 1; k < FMA_CHAINS; ++k) t = fma_step<T>(av, t, x[k]);
  if (is_one(t)) out[threadIdx.x] = t;
}

template <typename T>
static int fma_probe(int lanes_per_value, int steps, double* tflops) {
  const int blocks = sm_count() * 8;
  T* out = nullptr;
  cudaEvent_t a = nullptr, b = nullptr;
  cudaStream_t st = nullptr;
  cudaError_t e = cudaMalloc(&out, 256 * sizeof(T));
  if (e == cudaSuccess) e = cudaStreamCreateWithFlags(&st, cudaStreamNonBlocking);
  if (e == cudaSuccess) e = cudaEventCreate(&a);
  if (e == cudaSuccess) e = cudaEventCreate(&b);
  float best = 0.f;
  for (int r = 0; r < 4 && e == cudaSuccess; ++r) {  // one warm-up, best of three
    cudaEventRecord(a, st);
    fma_probe_kernel<T><<<blocks, 256, 0, st>>>(0.999f, 1e-3f, steps, out);
    cudaEventRecord(b, st);
    e = cudaEventSynchronize(b);
    float ms = 0.f;
    if (e == cudaSuccess) e = cudaEventElapsedTime(&ms, a, b);
    if (e == cudaSuccess && r > 0 && ms > 0.f && (best == 0.f || ms < best)) best = ms;
  }
  if (e == cudaSuccess) e = cudaGetLastError();
  if (a) cudaEventDestroy(a);
  if (b) cudaEventDestroy(b);
  if (st) cudaStreamDestroy(st);
  if (out) cudaFree(out);
  if (e != cudaSuccess || best <= 0.f) return VMS_ERR_CUDA;
  const double fmas = (double)blocks * 256 * lanes_per_value * ((double)FMA_CHAINS * steps + FMA_CHAINS - 1);
  *tflops = 2.0 * fmas / (best * 1e-3) / 1e12;
  return VMS_OK;
}
}  // namespace vms

extern "C" int vms_fma_throughput(int device, int kind, double* tflops) {
  if (!tflops || kind < 0 || kind > 2) return VMS_ERR_INVALID_ARG;
  if (cudaSetDevice(device) != cudaSuccess) return VMS_ERR_CUDA;
  // about 15 ms per launch at the GB300's rates
  if (kind == 0) return vms::fma_probe<double>(1, 4096, tflops);
  if (kind == 1) return vms::fma_probe<float>(1, 131072, tflops);
  return vms::fma_probe<float2>(2, 65536, tflops);
}
