// Linear solve of the condensed system S du = -r (Eq. SchurUpdate), fine-scale recovery and the
// Newton-Schur driver (Sections 4.2 and 5; the paper used a Krylov solver with tolerance 1e-12 and
// at most 50 iterations, Section 6).
//
// Solver: restarted GMRES(m), right-preconditioned by block ILU(0) (precond.cu) or the inverses of
// the 4x4 diagonal node blocks, classical Gram-Schmidt with one re-orthogonalisation pass (CGS2).
// In mixed precision the Krylov vectors and the matrix are FP32 (dot products summed in FP32 within
// a warp and in FP64 across warps) and an outer FP64 iterative refinement recomputes r = b - S x
// in FP64 until the tolerance is met.
#include <algorithm>
#include <chrono>
#include <cmath>
#include <cstdio>
#include <type_traits>
#include <vector>

#include "solver.h"

namespace vms {

void free_solver(SolverWork& s) {
  void* bufs[] = {s.x, s.r, s.V, s.Z, s.Dinv, s.h, s.rfull, s.bf, s.xf, s.cx, s.pv, s.pz, s.Zf,
                  s.xb, s.rb, s.band};
  for (void* b : bufs)
    if (b) cudaFree(b);
  for (BandOrder& o : s.band_orders)
    if (o.perm) cudaFree(o.perm);
  const uint32_t lim = s.ilu.spin_limit;  // a setting of the context, kept across re-allocations
  free_ilu(s.ilu);
  s = SolverWork();
  s.ilu.spin_limit = lim;
}

// ---------------------------------------------------------------------------------------------
// kernels
// ---------------------------------------------------------------------------------------------
// y = S x on the rows of nodes [node0, node0 + n_nodes): one warp per node (its four scalar rows
// share one column pattern of 4x4 blocks), one lane per block, so a column index is read once per
// block instead of once per value. x and y are compact (x[c - 4 node0], y[4 (node - node0) + q]).
// FP32 accumulation when matrix and vectors are FP32 (the inner solve of the mixed mode), FP64
// otherwise.
template <typename T> struct Row4;
template <> struct Row4<float> {
  __device__ __forceinline__ static void ld(const float* p, float o[4]) {
    const float4 t = __ldg(reinterpret_cast<const float4*>(p));
    o[0] = t.x; o[1] = t.y; o[2] = t.z; o[3] = t.w;
  }
};
template <> struct Row4<double> {
  __device__ __forceinline__ static void ld(const double* p, double o[4]) {
    const double2 a = __ldg(reinterpret_cast<const double2*>(p));
    const double2 b = __ldg(reinterpret_cast<const double2*>(p) + 1);
    o[0] = a.x; o[1] = a.y; o[2] = b.x; o[3] = b.y;
  }
};

template <typename T, typename VT>
__global__ void __launch_bounds__(256) spmv_kernel(const int32_t* __restrict__ rowptr,
                                                   const int32_t* __restrict__ colidx,
                                                   const T* __restrict__ val,
                                                   const VT* __restrict__ x, VT* __restrict__ y,
                                                   int64_t node0, int64_t n_nodes) {
  using Acc = typename std::conditional<sizeof(T) == 4 && sizeof(VT) == 4, float, double>::type;
  const int64_t nd = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  const int lane = threadIdx.x & 31;
  if (nd >= n_nodes) return;  // uniform over the warp
  const int64_t g = node0 + nd;
  int32_t rp[4];
  for (int m = 0; m < 4; ++m) rp[m] = rowptr[4 * g + m];
  const int deg = (rp[1] - rp[0]) >> 2;
  Acc acc[4] = {Acc(0), Acc(0), Acc(0), Acc(0)};
  for (int kk = lane; kk < deg; kk += 32) {
    const int64_t c = (int64_t)colidx[rp[0] + 4 * kk] - 4 * node0;
    Acc xv[4];
    for (int m = 0; m < 4; ++m) xv[m] = (Acc)x[c + m];
    for (int r = 0; r < 4; ++r) {
      T v[4];
      Row4<T>::ld(val + rp[r] + 4 * kk, v);
      for (int m = 0; m < 4; ++m) acc[r] = fma((Acc)v[m], xv[m], acc[r]);
    }
  }
  // reduce-scatter of the four sums over the warp: lane L ends with component (L >> 3) & 3
  const bool h16 = lane & 16, h8 = lane & 8;
  const Acc s0 = h16 ? acc[0] : acc[2], s1 = h16 ? acc[1] : acc[3];
  const Acc b0 = (h16 ? acc[2] : acc[0]) + __shfl_xor_sync(0xffffffffu, s0, 16);
  const Acc b1 = (h16 ? acc[3] : acc[1]) + __shfl_xor_sync(0xffffffffu, s1, 16);
  Acc t = (h8 ? b1 : b0) + __shfl_xor_sync(0xffffffffu, h8 ? b0 : b1, 8);
  t += __shfl_xor_sync(0xffffffffu, t, 4);
  t += __shfl_xor_sync(0xffffffffu, t, 2);
  t += __shfl_xor_sync(0xffffffffu, t, 1);
  if ((lane & 7) == 0) y[4 * nd + (lane >> 3)] = VT(t);
}

template <typename T, typename VT>
static int spmv(const Mesh& m, const SysRange& R, const void* values, const VT* x, VT* y,
                cudaStream_t st) {
  const int64_t nodes = R.nodes();
  const unsigned blocks = (unsigned)((nodes * 32 + 255) / 256);
  spmv_kernel<T, VT><<<blocks, 256, 0, st>>>(m.rowptr, m.colidx, (const T*)values, x, y, R.n0,
                                             nodes);
  return 1;
}

int launch_spmv(const Mesh& m, const void* values, bool fp32, const double* x, double* y,
                cudaStream_t st) {
  const SysRange all{0, m.n_nodes, 0, m.n_elems};
  return fp32 ? spmv<float, double>(m, all, values, x, y, st)
              : spmv<double, double>(m, all, values, x, y, st);
}

// Inverse of each node's 4x4 diagonal block (Gauss-Jordan with partial pivoting, FP64); a block
// with a vanishing pivot is replaced by the identity.
template <typename T>
__global__ void block_diag_inv_kernel(const int32_t* __restrict__ rowptr,
                                      const int32_t* __restrict__ colidx,
                                      const T* __restrict__ val, int64_t n_nodes,
                                      double* __restrict__ Dinv) {
  const int64_t n = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (n >= n_nodes) return;
  const int32_t start = rowptr[4 * n];
  const int32_t nb = (rowptr[4 * n + 1] - start) / 4;
  int lo = 0, hi = nb;
  while (lo < hi) {
    const int mid = (lo + hi) >> 1;
    if (colidx[start + 4 * mid] < 4 * n) lo = mid + 1; else hi = mid;
  }
  double M[4][8];
  for (int i = 0; i < 4; ++i) {
    const int32_t off = rowptr[4 * n + i] + 4 * lo;
    for (int k = 0; k < 4; ++k) {
      M[i][k] = (double)val[off + k];
      M[i][4 + k] = (i == k) ? 1.0 : 0.0;
    }
  }
  double scale = 0.0;
  for (int i = 0; i < 4; ++i)
    for (int k = 0; k < 4; ++k) scale = fmax(scale, fabs(M[i][k]));
  bool ok = scale > 0.0;
  for (int c = 0; c < 4 && ok; ++c) {
    int p = c;
    for (int i = c + 1; i < 4; ++i)
      if (fabs(M[i][c]) > fabs(M[p][c])) p = i;
    if (!(fabs(M[p][c]) > 1e-14 * scale)) { ok = false; break; }
    if (p != c)
      for (int k = 0; k < 8; ++k) { const double t = M[c][k]; M[c][k] = M[p][k]; M[p][k] = t; }
    const double inv = 1.0 / M[c][c];
    for (int k = 0; k < 8; ++k) M[c][k] *= inv;
    for (int i = 0; i < 4; ++i) {
      if (i == c) continue;
      const double f = M[i][c];
      for (int k = 0; k < 8; ++k) M[i][k] -= f * M[c][k];
    }
  }
  for (int i = 0; i < 4; ++i)
    for (int k = 0; k < 4; ++k) Dinv[16 * n + 4 * i + k] = ok ? M[i][4 + k] : (i == k ? 1.0 : 0.0);
}

template <typename VT>
__global__ void block_apply_kernel(const double* __restrict__ Dinv, const VT* __restrict__ v,
                                   VT* __restrict__ z, int64_t n_nodes) {
  const int64_t n = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (n >= n_nodes) return;
  double x[4];
  for (int k = 0; k < 4; ++k) x[k] = (double)v[4 * n + k];
  for (int i = 0; i < 4; ++i) {
    const double* d = Dinv + 16 * n + 4 * i;
    z[4 * n + i] = VT(d[0] * x[0] + d[1] * x[1] + d[2] * x[2] + d[3] * x[3]);
  }
}

constexpr int DOT_THREADS = 256;
// device scratch layout (doubles): Gram-Schmidt coefficients of the two passes, a norm, the
// least-squares solution, then per-block partial sums
constexpr int MAX_RESTART = 480;
constexpr int H_PASS1 = 0, H_PASS2 = 512, H_NORM = 1024, H_Y = 1025, H_PART = 1536;

__device__ __forceinline__ double block_reduce(double v, double* sh) {
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
  __syncthreads();
  if (lane == 0) sh[w] = v;
  __syncthreads();
  v = threadIdx.x < DOT_THREADS / 32 ? sh[threadIdx.x] : 0.0;
  if (w == 0)
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  return v;
}

// Four consecutive entries of a vector as doubles (16-byte loads for FP32, two for FP64).
template <typename VT> struct Quad;
template <> struct Quad<float> {
  __device__ __forceinline__ static void ld(const float* p, double o[4]) {
    const float4 t = *reinterpret_cast<const float4*>(p);
    o[0] = t.x; o[1] = t.y; o[2] = t.z; o[3] = t.w;
  }
  __device__ __forceinline__ static void st(float* p, const double v[4]) {
    *reinterpret_cast<float4*>(p) = make_float4((float)v[0], (float)v[1], (float)v[2], (float)v[3]);
  }
};
template <> struct Quad<double> {
  __device__ __forceinline__ static void ld(const double* p, double o[4]) {
    const double2 a = reinterpret_cast<const double2*>(p)[0], b = reinterpret_cast<const double2*>(p)[1];
    o[0] = a.x; o[1] = a.y; o[2] = b.x; o[3] = b.y;
  }
  __device__ __forceinline__ static void st(double* p, const double v[4]) {
    reinterpret_cast<double2*>(p)[0] = make_double2(v[0], v[1]);
    reinterpret_cast<double2*>(p)[1] = make_double2(v[2], v[3]);
  }
};

constexpr int MD_K = 8;          // vectors per block of the multi-dot and per step of the combine
constexpr int MD_THREADS = 256;
constexpr int MD_MAX_BLOCKS = 256;
constexpr int H_SIZE = H_PART + (MAX_RESTART + 1) * MD_MAX_BLOCKS;

// partial[k * nb + bx] = this block's share of V_k . w for k in [MD_K by, MD_K by + MD_K) and
// k < m (FP64 accumulation). Rows are taken four at a time (quad) when every vector allows it.
template <typename VT>
__global__ void __launch_bounds__(MD_THREADS) mdot_kernel(const VT* __restrict__ V, int64_t ld, int m,
                                                          const VT* __restrict__ w, int64_t n,
                                                          bool quad, double* __restrict__ partial) {
  __shared__ double sh[MD_K][MD_THREADS / 32];
  const int k0 = blockIdx.y * MD_K;
  const int nb = gridDim.x;
  double acc[MD_K];
#pragma unroll
  for (int t = 0; t < MD_K; ++t) acc[t] = 0.0;
  const int lane = threadIdx.x & 31, wp = threadIdx.x >> 5;
  if (quad && sizeof(VT) == 4) {
    // FP32 vectors: each thread's products and the warp's sum (at most 128 products per warp in
    // the usual one quad per thread) are formed in FP32, the warps' and blocks' sums in FP64: the
    // FP64 pipe, 1/64 of FP32, would otherwise bound the kernel
    float accf[MD_K];
#pragma unroll
    for (int t = 0; t < MD_K; ++t) accf[t] = 0.f;
    const int64_t n4 = n >> 2;
    const float4* w4 = reinterpret_cast<const float4*>(w);
    for (int64_t i = (int64_t)blockIdx.x * MD_THREADS + threadIdx.x; i < n4; i += (int64_t)nb * MD_THREADS) {
      const float4 wv = w4[i];
      float4 vv[MD_K];
#pragma unroll
      for (int t = 0; t < MD_K; ++t)
        if (k0 + t < m) vv[t] = reinterpret_cast<const float4*>(V + (int64_t)(k0 + t) * ld)[i];
#pragma unroll
      for (int t = 0; t < MD_K; ++t)
        if (k0 + t < m)
          accf[t] = fmaf(vv[t].w, wv.w, fmaf(vv[t].z, wv.z, fmaf(vv[t].y, wv.y, fmaf(vv[t].x, wv.x, accf[t]))));
    }
#pragma unroll
    for (int t = 0; t < MD_K; ++t) {
      float v = accf[t];
      for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
      if (lane == 0) sh[t][wp] = (double)v;
    }
  } else {
    if (quad) {
      const int64_t n4 = n >> 2;
      for (int64_t i = (int64_t)blockIdx.x * MD_THREADS + threadIdx.x; i < n4; i += (int64_t)nb * MD_THREADS) {
        double wv[4], vv[MD_K][4];
        Quad<VT>::ld(w + 4 * i, wv);
#pragma unroll
        for (int t = 0; t < MD_K; ++t)
          if (k0 + t < m) Quad<VT>::ld(V + (int64_t)(k0 + t) * ld + 4 * i, vv[t]);
#pragma unroll
        for (int t = 0; t < MD_K; ++t)
          if (k0 + t < m)
            acc[t] = fma(vv[t][3], wv[3], fma(vv[t][2], wv[2], fma(vv[t][1], wv[1], fma(vv[t][0], wv[0], acc[t]))));
      }
    } else {
      for (int64_t i = (int64_t)blockIdx.x * MD_THREADS + threadIdx.x; i < n; i += (int64_t)nb * MD_THREADS) {
        const double wi = (double)w[i];
#pragma unroll
        for (int t = 0; t < MD_K; ++t)
          if (k0 + t < m) acc[t] = fma((double)V[(int64_t)(k0 + t) * ld + i], wi, acc[t]);
      }
    }
#pragma unroll
    for (int t = 0; t < MD_K; ++t) {
      double v = acc[t];
      for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
      if (lane == 0) sh[t][wp] = v;
    }
  }
  __syncthreads();
  if (threadIdx.x < MD_K && k0 + (int)threadIdx.x < m) {
    double v = 0.0;
    for (int q = 0; q < MD_THREADS / 32; ++q) v += sh[threadIdx.x][q];
    partial[(int64_t)(k0 + threadIdx.x) * nb + blockIdx.x] = v;
  }
}

// out[k] = sum_b partial[k * nb + b], one block per k
__global__ void __launch_bounds__(DOT_THREADS) reduce_partials_kernel(const double* __restrict__ partial,
                                                                      int nb, double* __restrict__ out) {
  __shared__ double sh[DOT_THREADS / 32];
  const int k = blockIdx.x;
  double s = 0.0;
  for (int b = threadIdx.x; b < nb; b += DOT_THREADS) s += partial[(int64_t)k * nb + b];
  s = block_reduce(s, sh);
  if (threadIdx.x == 0) out[k] = s;
}

// out = (base ? base : 0) + sign * sum_{k < m} c[k] V_k, rows four at a time when aligned, with
// MD_K vector loads in flight per thread
template <typename VT>
__global__ void __launch_bounds__(256) vcomb_kernel(const VT* __restrict__ V, int64_t ld,
                                                    const double* __restrict__ c, int m, double sign,
                                                    const VT* base, VT* out, int64_t n, bool quad) {
  __shared__ double cs[MAX_RESTART + 1];
  __shared__ float cs32[MAX_RESTART + 1];
  for (int k = threadIdx.x; k < m; k += blockDim.x) {
    cs[k] = sign * c[k];
    cs32[k] = (float)(sign * c[k]);
  }
  __syncthreads();
  if (quad && sizeof(VT) == 4) {
    // FP32 vectors are combined in FP32 (the inner solve's working precision)
    const int64_t n4 = n >> 2;
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n4;
         i += (int64_t)gridDim.x * blockDim.x) {
      float4 s = base ? reinterpret_cast<const float4*>(base)[i] : make_float4(0.f, 0.f, 0.f, 0.f);
      int k = 0;
      for (; k + MD_K <= m; k += MD_K) {
        float4 vv[MD_K];
#pragma unroll
        for (int t = 0; t < MD_K; ++t) vv[t] = reinterpret_cast<const float4*>(V + (int64_t)(k + t) * ld)[i];
#pragma unroll
        for (int t = 0; t < MD_K; ++t) {
          const float ct = cs32[k + t];
          s.x = fmaf(ct, vv[t].x, s.x); s.y = fmaf(ct, vv[t].y, s.y);
          s.z = fmaf(ct, vv[t].z, s.z); s.w = fmaf(ct, vv[t].w, s.w);
        }
      }
      for (; k < m; ++k) {
        const float4 vv = reinterpret_cast<const float4*>(V + (int64_t)k * ld)[i];
        const float ct = cs32[k];
        s.x = fmaf(ct, vv.x, s.x); s.y = fmaf(ct, vv.y, s.y);
        s.z = fmaf(ct, vv.z, s.z); s.w = fmaf(ct, vv.w, s.w);
      }
      reinterpret_cast<float4*>(out)[i] = s;
    }
  } else if (quad) {
    const int64_t n4 = n >> 2;
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n4;
         i += (int64_t)gridDim.x * blockDim.x) {
      double s[4] = {0.0, 0.0, 0.0, 0.0};
      if (base) Quad<VT>::ld(base + 4 * i, s);
      int k = 0;
      for (; k + MD_K <= m; k += MD_K) {
        double vv[MD_K][4];
#pragma unroll
        for (int t = 0; t < MD_K; ++t) Quad<VT>::ld(V + (int64_t)(k + t) * ld + 4 * i, vv[t]);
#pragma unroll
        for (int t = 0; t < MD_K; ++t)
#pragma unroll
          for (int e = 0; e < 4; ++e) s[e] = fma(cs[k + t], vv[t][e], s[e]);
      }
      for (; k < m; ++k) {
        double vv[4];
        Quad<VT>::ld(V + (int64_t)k * ld + 4 * i, vv);
#pragma unroll
        for (int e = 0; e < 4; ++e) s[e] = fma(cs[k], vv[e], s[e]);
      }
      Quad<VT>::st(out + 4 * i, s);
    }
  } else {
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n;
         i += (int64_t)gridDim.x * blockDim.x) {
      double s = base ? (double)base[i] : 0.0;
      for (int k = 0; k < m; ++k) s = fma(cs[k], (double)V[(int64_t)k * ld + i], s);
      out[i] = VT(s);
    }
  }
}

// y = x / sqrt(*nrm2) (device-side normalisation, no host round trip)
template <typename VT>
__global__ void scale_kernel(const VT* x, const double* __restrict__ nrm2, VT* y, int64_t n) {  // y may be x
  const double s = *nrm2 > 0.0 ? 1.0 / sqrt(*nrm2) : 0.0;
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n;
       i += (int64_t)gridDim.x * blockDim.x)
    y[i] = VT((double)x[i] * s);
}

// out = a * x + b * y (mixed vector types)
template <typename A, typename B, typename C>
__global__ void axpby_kernel(double a, const A* x, double b, const B* y, C* out, int64_t n) {
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n;
       i += (int64_t)gridDim.x * blockDim.x)
    out[i] = C(a * (double)x[i] + (y ? b * (double)y[i] : 0.0));
}

// Fine-scale recovery (Section 5): dbeta_e = -(K_ff^-1 R_f + K_ff^-1 K_fc du_e); beta += dbeta.
// Elements [e0, e1); du is compact over the nodes from n0 on.
template <typename T>
__global__ void recover_kernel(const int32_t* __restrict__ conn, int npe, const T* __restrict__ recX,
                               const double* __restrict__ recY, const double* __restrict__ du,
                               double* __restrict__ beta, int64_t e0, int64_t e1, int64_t n0) {
  const int64_t e = e0 + (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (e >= e1) return;
  double s[3] = {recY[3 * e], recY[3 * e + 1], recY[3 * e + 2]};
  for (int a = 0; a < npe; ++a) {
    const int64_t nd = conn[npe * e + a] - n0;
    for (int c = 0; c < 4; ++c) {
      const double d = du[4 * nd + c];
      for (int m = 0; m < 3; ++m) s[m] += (double)recX[96 * e + 32 * m + 4 * a + c] * d;
    }
  }
  for (int m = 0; m < 3; ++m) beta[3 * e + m] -= s[m];
}

// ---------------------------------------------------------------------------------------------
// host side
// ---------------------------------------------------------------------------------------------
static unsigned grid_for(int64_t n) {
  const int64_t b = (n + 255) / 256, cap = (int64_t)sm_count() * 8;
  return (unsigned)(b > cap ? cap : (b < 1 ? 1 : b));
}

// Rows can be taken four at a time when the length, the stride and every pointer allow 16-byte
// (FP32) or 32-byte (FP64) accesses.
static bool quad_ok(int64_t n, int64_t ld, size_t elem, std::initializer_list<const void*> ptrs) {
  if ((n & 3) || (ld & 3)) return false;
  for (const void* q : ptrs)
    if (q && ((uintptr_t)q % (4 * elem))) return false;
  return true;
}

// out[k] = V_k . w for k < m (m <= MAX_RESTART + 1), FP64 accumulation; `partial` holds
// m * MD_MAX_BLOCKS doubles. Returns the launches.
template <typename VT>
static int dots(const VT* V, int64_t ld, int m, const VT* w, int64_t n, double* partial,
                double* out, cudaStream_t st) {
  const bool quad = quad_ok(n, ld, sizeof(VT), {V, w});
  const int groups = (m + MD_K - 1) / MD_K;
  const int64_t units = quad ? n / 4 : n;
  int64_t nb = (4 * (int64_t)sm_count() + groups - 1) / groups;  // about four blocks per SM in all
  nb = std::min<int64_t>(nb, (units + MD_THREADS - 1) / MD_THREADS);
  nb = std::max<int64_t>(1, std::min<int64_t>(nb, MD_MAX_BLOCKS));
  mdot_kernel<VT><<<dim3((unsigned)nb, (unsigned)groups), MD_THREADS, 0, st>>>(V, ld, m, w, n, quad, partial);
  reduce_partials_kernel<<<m, DOT_THREADS, 0, st>>>(partial, (int)nb, out);
  return 2;
}

// out = (base ? base : 0) + sign * sum_{k < m} c[k] V_k (c on the device). Returns the launches.
template <typename VT>
static int vcomb(const VT* V, int64_t ld, const double* c, int m, double sign, const VT* base,
                 VT* out, int64_t n, cudaStream_t st) {
  const bool quad = quad_ok(n, ld, sizeof(VT), {V, base, out});
  vcomb_kernel<VT><<<grid_for(quad ? n / 4 : n), 256, 0, st>>>(V, ld, c, m, sign, base, out, n, quad);
  return 1;
}

struct Gmres {
  vms_ctx* ctx;
  const Mesh& m;
  SolverWork& w;
  cudaStream_t st;
  int64_t n;      // 4 R.nodes(): length of every (compact) vector
  SysRange R;
  void* Zflex = nullptr;  // flexible GMRES: restart preconditioned vectors kept (else null)
  int restart_cap = 0;    // > restart: a cycle that does not halve the residual doubles the
                          // restart length (up to this), the basis growing with it
  bool stall_exit = false;  // end the solve after a full cycle at the longest length whose rate,
                            // kept for the remaining iterations, would not reach rtol (a direct
                            // solve follows it)
  bool has_deadline = false;  // end the solve at this host time (the direct solve's estimated
  std::chrono::steady_clock::time_point deadline{};  // duration after the start, a direct solve
  bool timed_out = false;                             // following it)

  // z = M^-1 v with the preconditioner chosen for this solve
  template <typename T, typename VT>
  void precond(const VT* v, VT* z) {
    KScope k(ctx, VMS_K_PRECOND);
    if constexpr (std::is_same<T, float>::value && std::is_same<VT, double>::value) {
      if (w.use_ilu) {  // FP64 vectors: the FP64 factor the FP32 one was rounded from
        k.add(ilu_apply<double, double>(w.ilu, m, R.n0, R.n1, v, z, st));
        return;
      }
    }
    if (w.use_ilu) {
      k.add(ilu_apply<T, VT>(w.ilu, m, R.n0, R.n1, v, z, st));
    } else {
      block_apply_kernel<VT><<<grid_for(R.nodes()), 256, 0, st>>>(w.Dinv + 16 * R.n0, v, z, R.nodes());
      k.add(1);
    }
  }

  int sync_host(void* dst, const void* src, size_t bytes) {
    cudaError_t e = cudaMemcpyAsync(dst, src, bytes, cudaMemcpyDeviceToHost, st);
    if (e == cudaSuccess) e = cudaStreamSynchronize(st);
    return e == cudaSuccess ? VMS_OK : ctx_fail(ctx, VMS_ERR_CUDA, cudaGetErrorString(e));
  }

  // One restarted GMRES solve of A x = b from x = 0 in vector type VT; matrix values type T.
  // Returns VMS_OK with *iters and *relres; x receives the solution.
  // Grow the Krylov basis (and the kept preconditioned vectors) to `restart` vectors, keeping V_0.
  template <typename VT>
  int grow_basis(int restart) {
    double* nv = nullptr;
    cudaError_t e = cudaMalloc(&nv, sizeof(double) * (size_t)n * (restart + 1));
    if (e == cudaSuccess)
      e = cudaMemcpyAsync(nv, w.V, sizeof(VT) * (size_t)n, cudaMemcpyDeviceToDevice, st);
    if (e == cudaSuccess && Zflex) {
      double* nz = nullptr;
      e = cudaMalloc(&nz, sizeof(double) * (size_t)n * restart);
      if (e == cudaSuccess) {
        cudaFree(w.Zf);
        w.Zf = nz;
        w.zf_restart = restart;
        Zflex = nz;
      }
    }
    if (e != cudaSuccess) {
      if (nv) cudaFree(nv);
      return ctx_fail(ctx, e == cudaErrorMemoryAllocation ? VMS_ERR_OUT_OF_MEMORY : VMS_ERR_CUDA,
                      cudaGetErrorString(e));
    }
    cudaFree(w.V);  // waits for the work queued on it
    w.V = nv;
    w.restart = restart;
    return VMS_OK;
  }

  template <typename T, typename VT>
  int solve(const void* values, const VT* b, VT* x, double bnorm, double rtol, int maxit,
            int& restart, int* iters, double* relres) {
    VT* V = reinterpret_cast<VT*>(w.V);
    VT* z = reinterpret_cast<VT*>(w.Z);
    double* hd = w.h;
    std::vector<double> H((restart + 1) * restart, 0.0), cs(restart), sn(restart), g(restart + 1);
    std::vector<double> hh(restart + 2), hcol(H_NORM + 1);
    {
      KScope zs(ctx, VMS_K_FILL);
      zs.add(launch_fill_zero(x, sizeof(VT) * n, st));
    }
    int it = 0;
    double res = bnorm;
    // r0 = b (x = 0)
    {
      KScope k(ctx, VMS_K_KRYLOV);
      axpby_kernel<VT, VT, VT><<<grid_for(n), 256, 0, st>>>(1.0, b, 0.0, (const VT*)nullptr, V, n);
      k.add(1);
    }
    double cycle_res0 = res;
    while (it < maxit && res > rtol * bnorm && !timed_out) {
      // V_0 = r / |r|
      {
        KScope k(ctx, VMS_K_REDUCE);
        k.add(dots<VT>(V, n, 1, V, n, hd + H_PART, hd + H_NORM, st));
      }
      int rc = sync_host(&res, hd + H_NORM, sizeof(double));
      if (rc) return rc;
      res = std::sqrt(res);
      if (!(res > rtol * bnorm) || !(res == res)) break;
      {
        KScope k(ctx, VMS_K_KRYLOV);
        scale_kernel<VT><<<grid_for(n), 256, 0, st>>>(V, hd + H_NORM, V, n);
        k.add(1);
      }
      std::fill(g.begin(), g.end(), 0.0);
      g[0] = res;
      cycle_res0 = res;
      int j = 0;
      for (; j < restart && it < maxit; ++j, ++it) {
        VT* vj = V + (int64_t)j * n;
        VT* vn = V + (int64_t)(j + 1) * n;
        VT* zj = Zflex ? reinterpret_cast<VT*>(Zflex) + (int64_t)j * n : z;
        precond<T, VT>(vj, zj);
        { KScope k(ctx, VMS_K_SPMV); k.add(spmv<T, VT>(m, R, values, zj, vn, st)); }
        // CGS2 against V_0..V_j: first pass coefficients into hd[H_PASS1..], second into hd[H_PASS2..]
        const int kk = j + 1;
        double* partial = hd + H_PART;
        for (int pass = 0; pass < 2; ++pass) {
          {
            KScope k(ctx, VMS_K_REDUCE);
            k.add(dots<VT>(V, n, kk, vn, n, partial, hd + (pass ? H_PASS2 : H_PASS1), st));
          }
          KScope k(ctx, VMS_K_KRYLOV);
          k.add(vcomb<VT>(V, n, hd + (pass ? H_PASS2 : H_PASS1), kk, -1.0, vn, vn, n, st));
        }
        {
          KScope k(ctx, VMS_K_REDUCE);
          k.add(dots<VT>(vn, n, 1, vn, n, partial, hd + H_NORM, st));
        }
        {
          KScope k(ctx, VMS_K_KRYLOV);
          scale_kernel<VT><<<grid_for(n), 256, 0, st>>>(vn, hd + H_NORM, vn, n);
          k.add(1);
        }
        // bring the Hessenberg column (both passes and the norm) to the host in one copy
        if (int rc2 = sync_host(hcol.data(), hd, sizeof(double) * (H_NORM + 1))) return rc2;
        const double nrm2 = hcol[H_NORM];
        for (int i = 0; i < kk; ++i) hh[i] = hcol[H_PASS1 + i] + hcol[H_PASS2 + i];
        hh[kk] = std::sqrt(nrm2);
        // apply previous rotations, then a new one
        for (int i = 0; i < j; ++i) {
          const double t = cs[i] * hh[i] + sn[i] * hh[i + 1];
          hh[i + 1] = -sn[i] * hh[i] + cs[i] * hh[i + 1];
          hh[i] = t;
        }
        const double den = std::hypot(hh[j], hh[j + 1]);
        cs[j] = den > 0 ? hh[j] / den : 1.0;
        sn[j] = den > 0 ? hh[j + 1] / den : 0.0;
        hh[j] = den;
        hh[j + 1] = 0.0;
        g[j + 1] = -sn[j] * g[j];
        g[j] = cs[j] * g[j];
        for (int i = 0; i <= j; ++i) H[i * restart + j] = hh[i];
        res = std::fabs(g[j + 1]);
        if (!(res > rtol * bnorm) || nrm2 <= 0.0) { ++j; ++it; break; }
        if (has_deadline && std::chrono::steady_clock::now() > deadline) {
          timed_out = true;
          ++j;
          ++it;
          break;
        }
      }
      // y = H^-1 g (upper triangular j x j), x += M^-1 V y
      std::vector<double> y(j, 0.0);
      for (int i = j - 1; i >= 0; --i) {
        double s = g[i];
        for (int k2 = i + 1; k2 < j; ++k2) s -= H[i * restart + k2] * y[k2];
        y[i] = H[i * restart + i] != 0.0 ? s / H[i * restart + i] : 0.0;
      }
      cudaMemcpyAsync(hd + H_Y, y.data(), sizeof(double) * j, cudaMemcpyHostToDevice, st);
      if (Zflex) {  // x += Z y with the kept preconditioned vectors
        KScope k(ctx, VMS_K_KRYLOV);
        k.add(vcomb<VT>(reinterpret_cast<const VT*>(Zflex), n, hd + H_Y, j, 1.0, nullptr, V + n, n, st));
      } else {      // x += M^-1 V y
        {
          KScope k(ctx, VMS_K_KRYLOV);
          k.add(vcomb<VT>(V, n, hd + H_Y, j, 1.0, nullptr, z, n, st));
        }
        precond<T, VT>(z, V + n);
      }
      {
        KScope k(ctx, VMS_K_KRYLOV);
        axpby_kernel<VT, VT, VT><<<grid_for(n), 256, 0, st>>>(1.0, x, 1.0, V + n, x, n);
        k.add(1);
      }
      // restart: r = b - A x into V_0
      { KScope k(ctx, VMS_K_SPMV); k.add(spmv<T, VT>(m, R, values, x, z, st)); }
      {
        KScope k(ctx, VMS_K_KRYLOV);
        axpby_kernel<VT, VT, VT><<<grid_for(n), 256, 0, st>>>(1.0, b, -1.0, z, V, n);
        k.add(1);
      }
      cudaError_t e = cudaGetLastError();
      if (e != cudaSuccess) return ctx_fail(ctx, VMS_ERR_CUDA, cudaGetErrorString(e));
      // a full cycle that did not halve the residual: the cycle is too short to keep the slow
      // directions (coarse modes of large meshes); continue with a longer one
      if (j == restart && it < maxit && res > rtol * bnorm && res > 0.5 * cycle_res0 &&
          restart < restart_cap && !timed_out) {
        const int nr = std::min(2 * restart, restart_cap);
        if (int rc2 = grow_basis<VT>(nr)) return rc2;
        V = reinterpret_cast<VT*>(w.V);
        restart = nr;
        H.assign((size_t)(restart + 1) * restart, 0.0);
        cs.assign(restart, 0.0);
        sn.assign(restart, 0.0);
        g.assign(restart + 1, 0.0);
        hh.assign(restart + 2, 0.0);
      }
      // stagnation: the residual projected to maxit at this cycle's reduction factor q stays above
      // the target, res q^((maxit - it) / restart) > rtol |b|
      else if (stall_exit && j == restart && it < maxit && res > rtol * bnorm && cycle_res0 > 0.0 &&
               std::log(res / (rtol * bnorm)) >
                   -std::log(std::min(res / cycle_res0, 1.0)) * ((double)(maxit - it) / restart))
        break;
      // true residual norm for the next cycle's test is computed at the top of the loop
      if (!(res > rtol * bnorm)) {
        KScope k(ctx, VMS_K_REDUCE);
        k.add(dots<VT>(V, n, 1, V, n, hd + H_PART, hd + H_NORM, st));
        double r2 = 0.0;
        if (int rc2 = sync_host(&r2, hd + H_NORM, sizeof(double))) return rc2;
        res = std::sqrt(r2);
      }
    }
    *iters = it;
    *relres = bnorm > 0 ? res / bnorm : 0.0;
    return VMS_OK;
  }
};

static int ensure_solver(vms_ctx* ctx, int restart) {
  const Mesh& m = ctx_mesh(ctx);
  SolverWork& w = ctx_solver(ctx);
  const int64_t n = 4 * m.n_nodes;
  if (w.n == n && w.restart >= restart) return VMS_OK;
  free_solver(w);
  cudaError_t e = cudaSuccess;
  const size_t vb = sizeof(double);  // FP64 storage serves both vector types
  if (e == cudaSuccess) e = cudaMalloc(&w.x, vb * n);
  if (e == cudaSuccess) e = cudaMalloc(&w.r, vb * n);
  if (e == cudaSuccess) e = cudaMalloc(&w.V, vb * n * (restart + 1));
  if (e == cudaSuccess) e = cudaMalloc(&w.Z, vb * n);
  if (e == cudaSuccess) e = cudaMalloc(&w.Dinv, sizeof(double) * 16 * m.n_nodes);
  if (e == cudaSuccess) e = cudaMalloc(&w.h, sizeof(double) * H_SIZE);
  if (e == cudaSuccess) e = cudaMalloc(&w.rfull, sizeof(double) * n);
  if (e == cudaSuccess) e = cudaMalloc(&w.bf, sizeof(float) * n);
  if (e == cudaSuccess) e = cudaMalloc(&w.xf, sizeof(float) * n);
  if (e == cudaSuccess) e = cudaMalloc(&w.cx, sizeof(double) * n);
  if (e == cudaSuccess) e = cudaMalloc(&w.xb, sizeof(double) * n);
  if (e == cudaSuccess) e = cudaMalloc(&w.rb, sizeof(double) * n);
  if (e == cudaSuccess) e = cudaMalloc(&w.pv, sizeof(float) * n);
  if (e == cudaSuccess) e = cudaMalloc(&w.pz, sizeof(float) * n);
  if (e == cudaSuccess) e = cudaMalloc(&w.band, sizeof(int) * 4);
  if (e != cudaSuccess) {
    free_solver(w);
    return ctx_fail(ctx, e == cudaErrorMemoryAllocation ? VMS_ERR_OUT_OF_MEMORY : VMS_ERR_CUDA,
                    cudaGetErrorString(e));
  }
  w.n = n;
  w.restart = restart;
  return VMS_OK;
}

static int band_estimate(vms_ctx* ctx, const SysRange& R, int* kl_out, bool* fits);

// Solve S du = -rhs into w.x (FP64). Mixed: FP32 GMRES inside FP64 iterative refinement.
static int linear_solve(vms_ctx* ctx, const SysRange& R, double rtol, int maxit, int restart,
                        int restart_cap, int* iters_out, double* rel_out, bool block_jacobi = false) {
  const Mesh& m = ctx_mesh(ctx);
  Work& wk = ctx_work(ctx);
  SolverWork& w = ctx_solver(ctx);
  cudaStream_t st = ctx_stream(ctx);
  const int64_t n = 4 * R.nodes();
  const bool f32 = ctx_fp32(ctx);
  if (restart < 1 || restart > MAX_RESTART || maxit < 1 || !(rtol > 0.0))
    return ctx_fail(ctx, VMS_ERR_INVALID_ARG, "invalid solver parameters");
  if (int rc = ensure_solver(ctx, restart)) return rc;
  w.use_ilu = !block_jacobi && ctx_precond(ctx) != VMS_PRECOND_BLOCK_JACOBI;
  // the preconditioner covers the whole matrix (its blocks are independent) and is set up once
  // per assembly; the ILU(0) factor and the block-Jacobi inverses are kept apart, so that a
  // block-Jacobi solve does not discard the factor the other instances use
  if (w.use_ilu && (w.ilu_for != wk.assembly_id || !w.ilu.factored)) {
    KScope k(ctx, VMS_K_PRECOND);
    w.ilu_for = wk.assembly_id;
    int launched = 0;
    const int rc = ilu_factor(ctx, w.ilu, m, f32, wk.values, st, &launched);
    k.add(launched);
    if (rc) {
      w.ilu_for = 0;
      return rc;
    }
  } else if (!w.use_ilu && w.dinv_for != wk.assembly_id) {
    KScope k(ctx, VMS_K_PRECOND);
    w.dinv_for = wk.assembly_id;
    if (f32)
      block_diag_inv_kernel<float><<<grid_for(m.n_nodes), 256, 0, st>>>(m.rowptr, m.colidx, (const float*)wk.values, m.n_nodes, w.Dinv);
    else
      block_diag_inv_kernel<double><<<grid_for(m.n_nodes), 256, 0, st>>>(m.rowptr, m.colidx, (const double*)wk.values, m.n_nodes, w.Dinv);
    k.add(1);
  }
  // b = -rhs (FP64) in w.r
  {
    KScope k(ctx, VMS_K_KRYLOV);
    axpby_kernel<double, double, double><<<grid_for(n), 256, 0, st>>>(-1.0, wk.rhs + 4 * R.n0, 0.0, (const double*)nullptr, w.r, n);
    k.add(1);
  }
  double* hd = w.h;
  double bnorm2 = 0.0;
  {
    KScope k(ctx, VMS_K_REDUCE);
    dots<double>(w.r, n, 1, w.r, n, hd + H_PART, hd + H_NORM, st);
    k.add(2);
  }
  Gmres G{ctx, m, w, st, n, R};
  G.restart_cap = std::min(std::max(restart_cap, restart), MAX_RESTART);
  if (w.use_ilu && ctx_precond(ctx) == VMS_PRECOND_ILU0_FALLBACK) {
    // Where the direct solve will follow a failed ILU(0) solve, the Krylov attempt ends early: when
    // it stagnates, or once it has run as long as the direct solve is estimated to take (so the
    // two together take at most about twice the faster one). The estimate is per column of the
    // band a launch (about 10 us) plus the column's update at the rate measured on a GB300
    // (3.2 ns per thousand entries).
    int kl = 0;
    if (int rc = band_estimate(ctx, R, &kl, &G.stall_exit)) return rc;
    if (G.stall_exit) {
      const double est = (double)n * (1.0e-5 + 3.2e-12 * (double)kl * (2.0 * kl));
      G.has_deadline = true;
      G.deadline = std::chrono::steady_clock::now() +
                   std::chrono::duration_cast<std::chrono::steady_clock::duration>(std::chrono::duration<double>(est));
    }
  }
  if (int rc = G.sync_host(&bnorm2, hd + H_NORM, sizeof(double))) return rc;
  const double bnorm = std::sqrt(bnorm2);
  // a non-finite right-hand side is reported as such before any preconditioner sweep runs
  if (!std::isfinite(bnorm)) return ctx_fail(ctx, VMS_ERR_NAN, "non-finite right-hand side");
  if (bnorm == 0.0) {
    KScope k(ctx, VMS_K_FILL);
    k.add(launch_fill_zero(w.x, sizeof(double) * n, st));
    *iters_out = 0;
    *rel_out = 0.0;
    return VMS_OK;
  }
  if (!f32) {
    int it = 0;
    double rel = 0.0;
    if (int rc = G.solve<double, double>(wk.values, w.r, w.x, bnorm, rtol, maxit, restart, &it, &rel)) return rc;
    if (w.use_ilu)
      if (int rc = ilu_status(ctx, w.ilu, st)) return rc;
    *iters_out = it;
    *rel_out = rel;
    return rel <= rtol ? VMS_OK : ctx_fail(ctx, VMS_ERR_KRYLOV_MAXIT, "GMRES reached maxit");
  }
  // mixed: x = 0; repeat { r = b - S x (FP64); solve S c = r with FP32 GMRES; x += c }
  {
    KScope k(ctx, VMS_K_FILL);
    k.add(launch_fill_zero(w.x, sizeof(double) * n, st));
  }
  int total = 0;
  double rel = 1.0;
  double* rfull = w.rfull;
  float* bf = w.bf;
  float* xf = w.xf;
  int rc = VMS_OK;
  // The FP64 residual is recomputed after every correction, the last one included, so that the
  // reported relative residual always belongs to the returned x. A pass that does not halve the
  // residual ends the refinement: the FP32 inner solve cannot resolve directions whose singular
  // values lie below FP32 resolution (the near-null pressure modes of distorted meshes), and the
  // remaining correction is then solved with FP64 Krylov vectors (below).
  int last_it = -1;
  double prev_rel = HUGE_VAL;
  bool stalled = false;
  double r2 = 0.0;
  for (int outer = 0;; ++outer) {
    // FP64 residual of the refinement
    { KScope k(ctx, VMS_K_SPMV); k.add(spmv<float, double>(m, R, wk.values, w.x, rfull, st)); }
    {
      KScope k(ctx, VMS_K_KRYLOV);
      axpby_kernel<double, double, double><<<grid_for(n), 256, 0, st>>>(1.0, w.r, -1.0, rfull, rfull, n);
      k.add(1);
    }
    {
      KScope k(ctx, VMS_K_REDUCE);
      dots<double>(rfull, n, 1, rfull, n, hd + H_PART, hd + H_NORM, st);
      k.add(2);
    }
    if ((rc = G.sync_host(&r2, hd + H_NORM, sizeof(double)))) break;
    rel = std::sqrt(r2) / bnorm;
    if (!(rel <= prev_rel) && outer > 0) {
      // the last FP32 correction made things worse (or not finite): return to the iterate before it
      cudaMemcpyAsync(w.x, w.xb, sizeof(double) * n, cudaMemcpyDeviceToDevice, st);
      cudaMemcpyAsync(rfull, w.rb, sizeof(double) * n, cudaMemcpyDeviceToDevice, st);
      rel = prev_rel;
      r2 = (rel * bnorm) * (rel * bnorm);
      stalled = true;
      break;
    }
    if (rel <= rtol || outer == 20 || total >= maxit || last_it == 0 || G.timed_out) break;
    if (rel > 0.5 * prev_rel) { stalled = true; break; }
    prev_rel = rel;
    cudaMemcpyAsync(w.xb, w.x, sizeof(double) * n, cudaMemcpyDeviceToDevice, st);
    cudaMemcpyAsync(w.rb, rfull, sizeof(double) * n, cudaMemcpyDeviceToDevice, st);
    {
      KScope k(ctx, VMS_K_KRYLOV);
      axpby_kernel<double, double, float><<<grid_for(n), 256, 0, st>>>(1.0, rfull, 0.0, (const double*)nullptr, bf, n);
      k.add(1);
    }
    int it = 0;
    double irel = 0.0;
    const double inner = std::max(rtol / rel, 1e-3);
    if ((rc = G.solve<float, float>(wk.values, bf, xf, std::sqrt(r2), std::min(inner, 0.5),
                                    maxit - total, restart, &it, &irel)))
      break;
    total += it;
    {
      KScope k(ctx, VMS_K_KRYLOV);
      axpby_kernel<double, float, double><<<grid_for(n), 256, 0, st>>>(1.0, w.x, 1.0, xf, w.x, n);
      k.add(1);
    }
    last_it = it;
  }
  if (rc == VMS_OK && stalled && total < maxit && !G.timed_out) {
    // S c = b - S x with FP64 Krylov vectors, the FP32 matrix values and the FP64 preconditioner
    // (the ILU(0) factor the FP32 sweeps' copy is rounded from)
    int it = 0;
    double irel = 0.0;
    // the preconditioned vectors are kept (flexible form), so that the update x += Z y needs no
    // further preconditioner application
    if (!w.Zf || w.zf_restart < restart) {
      if (w.Zf) cudaFree(w.Zf);
      w.Zf = nullptr;
      const cudaError_t e = cudaMalloc(&w.Zf, sizeof(double) * (size_t)w.n * restart);
      if (e != cudaSuccess)
        return ctx_fail(ctx, e == cudaErrorMemoryAllocation ? VMS_ERR_OUT_OF_MEMORY : VMS_ERR_CUDA,
                        cudaGetErrorString(e));
      w.zf_restart = restart;
    }
    G.Zflex = w.Zf;
    rc = G.solve<float, double>(wk.values, rfull, w.cx, std::sqrt(r2), rtol / rel, maxit - total,
                                restart, &it, &irel);
    G.Zflex = nullptr;
    if (rc == VMS_OK) {
      total += it;
      {
        KScope k(ctx, VMS_K_KRYLOV);
        axpby_kernel<double, double, double><<<grid_for(n), 256, 0, st>>>(1.0, w.x, 1.0, w.cx, w.x, n);
        k.add(1);
      }
      { KScope k(ctx, VMS_K_SPMV); k.add(spmv<float, double>(m, R, wk.values, w.x, rfull, st)); }
      {
        KScope k(ctx, VMS_K_KRYLOV);
        axpby_kernel<double, double, double><<<grid_for(n), 256, 0, st>>>(1.0, w.r, -1.0, rfull, rfull, n);
        k.add(1);
      }
      {
        KScope k(ctx, VMS_K_REDUCE);
        dots<double>(rfull, n, 1, rfull, n, hd + H_PART, hd + H_NORM, st);
        k.add(2);
      }
      rc = G.sync_host(&r2, hd + H_NORM, sizeof(double));
      rel = std::sqrt(r2) / bnorm;
    }
  }
  if (rc) return rc;
  if (w.use_ilu)
    if (int rc2 = ilu_status(ctx, w.ilu, st)) return rc2;
  *iters_out = total;
  *rel_out = rel;
  return rel <= rtol ? VMS_OK : ctx_fail(ctx, VMS_ERR_KRYLOV_MAXIT, "refined GMRES reached maxit");
}

// ---------------------------------------------------------------------------------------------
// Direct solve of one instance by banded LU with partial pivoting (the fallback of
// VMS_PRECOND_ILU0_FALLBACK for systems whose ILU(0) factor is unstable). Band storage as in
// LAPACK's band routines: entry (i, j) of the N x N matrix at AB[(kv + i - j) + j * ldab] with
// kv = kl + ku and ldab = 2 kl + ku + 1 (the top kl rows take the fill of the row interchanges).
// The factorisation is Doolittle's elimination column by column (pivot search, interchange within
// the band, multipliers, rank-1 update of the band's trailing block); the solve applies the
// interchanges and multipliers forward and U backward. FP64 throughout.
// ---------------------------------------------------------------------------------------------

// the largest |column node - row node| of the block's rows: the bandwidth of its own node order
__global__ void band_width_kernel(const int32_t* __restrict__ rowptr, const int32_t* __restrict__ colidx,
                                  int64_t n0, int64_t nodes, int* __restrict__ bw) {
  const int64_t nd = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (nd >= nodes) return;
  const int64_t g = n0 + nd;
  int w = 0;
  for (int32_t t = rowptr[4 * g]; t < rowptr[4 * g + 1]; t += 4) {
    const int64_t d = (int64_t)(colidx[t] >> 2) - g;
    w = (int)std::max<int64_t>(w, d < 0 ? -d : d);
  }
  atomicMax(bw, w);
}

// the block's rows into the band in the band order perm (one warp per node row, one lane per 4x4
// block): entry (4 perm[a] + r, 4 perm[c] + m)
template <typename T>
__global__ void band_scatter_kernel(const int32_t* __restrict__ rowptr, const int32_t* __restrict__ colidx,
                                    const T* __restrict__ val, const int32_t* __restrict__ perm, int64_t n0,
                                    int64_t nodes, double* __restrict__ AB, int64_t ldab, int kl, int ku,
                                    int* __restrict__ err) {
  const int64_t nd = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  const int lane = threadIdx.x & 31;
  if (nd >= nodes) return;
  const int64_t g = n0 + nd, N = 4 * nodes, kv = kl + ku;
  const int64_t pr = perm[nd];
  int32_t rp[4];
  for (int m = 0; m < 4; ++m) rp[m] = rowptr[4 * g + m];
  const int deg = (rp[1] - rp[0]) >> 2;
  for (int kk = lane; kk < deg; kk += 32) {
    const int64_t hc = (int64_t)(colidx[rp[0] + 4 * kk] >> 2) - n0;
    if (hc < 0 || hc >= nodes) {
      atomicOr(err, 1);
      continue;
    }
    const int64_t pc = perm[hc];
    for (int r = 0; r < 4; ++r)
      for (int m = 0; m < 4; ++m) {
        const int64_t i = 4 * pr + r, j = 4 * pc + m;
        if (j < 0 || j >= N || i - j > kl || j - i > ku) {
          atomicOr(err, 1);
          continue;
        }
        AB[(kv + i - j) + j * ldab] = (double)val[rp[r] + 4 * kk + m];
      }
  }
}

// b[4 perm[a] + r] = s v[4 a + r] (to the band order) or v[4 a + r] = b[4 perm[a] + r] (back)
__global__ void band_permute_kernel(const double* __restrict__ v, const int32_t* __restrict__ perm,
                                    int64_t nodes, double s, double* __restrict__ b, int to_band) {
  const int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= 4 * nodes) return;
  const int64_t a = t >> 2, r = t & 3, q = 4 * (int64_t)perm[a] + r;
  if (to_band) b[q] = s * v[t];
  else b[t] = v[q];
}

constexpr int BAND_THREADS = 1024;  // the substitution kernel's block
constexpr int BAND_STEP_THREADS = 256;

// Pivot of column `col` (its final values): the largest |A(col + t, col)|, t = 0..km, the first on
// ties. ipiv[col] = col + t, jua[col] = the last column the interchanges up to col reach,
// state[1] = col + 1 for a zero (or not a number) pivot. All threads of the block call it.
__device__ void band_pivot_search(const double* __restrict__ AB, int64_t ldab, int N, int kl, int ku,
                                  int col, int ju_prev, int* __restrict__ ipiv, int* __restrict__ jua,
                                  int* __restrict__ state) {
  __shared__ double sv[BAND_STEP_THREADS];
  __shared__ int si[BAND_STEP_THREADS];
  const int tid = threadIdx.x;
  const int64_t kv = kl + ku;
  const int km = kl < N - 1 - col ? kl : N - 1 - col;
  const double* a = AB + (int64_t)col * ldab + kv;
  double best = -1.0;
  int bi = 0;
  for (int t = tid; t <= km; t += BAND_STEP_THREADS) {
    const double v = fabs(a[t]);
    if (v > best) { best = v; bi = t; }
  }
  sv[tid] = best;
  si[tid] = bi;
  __syncthreads();
  for (int h = BAND_STEP_THREADS / 2; h > 0; h >>= 1) {
    if (tid < h && (sv[tid + h] > sv[tid] || (sv[tid + h] == sv[tid] && si[tid + h] < si[tid]))) {
      sv[tid] = sv[tid + h];
      si[tid] = si[tid + h];
    }
    __syncthreads();
  }
  if (tid == 0) {
    const int jp = si[0];
    ipiv[col] = col + jp;
    const int reach = col + ku + jp < N - 1 ? col + ku + jp : N - 1;
    jua[col] = reach > ju_prev ? reach : ju_prev;
    if (!(sv[0] > 0.0)) atomicCAS(state + 1, 0, col + 1);
  }
}

__global__ void __launch_bounds__(BAND_STEP_THREADS) band_first_pivot_kernel(const double* __restrict__ AB, int64_t ldab,
                                                                             int N, int kl, int ku, int* __restrict__ ipiv,
                                                                             int* __restrict__ jua, int* __restrict__ state) {
  band_pivot_search(AB, ldab, N, kl, ku, 0, 0, ipiv, jua, state);
}

// Elimination step of column j, one launch per column. Column j is read as it stands (final, not
// yet interchanged or scaled): the multiplier of row j + r is l_r = A'(j + r, j) / A(j + jp, j),
// A' being column j with rows j and j + jp interchanged. Block b updates columns j + 1 + b,
// j + 1 + b + gridDim.x, ... up to jua[j]: row j takes the pivot row's value u = A(j + jp, c)
// and row j + r becomes A'(j + r, c) - l_r u. The block that owns column j + 1 (block 0) then
// searches its pivot for the next launch, and the last block stores column j - 1's multipliers
// and pivot (no block of this launch reads that column).
__global__ void __launch_bounds__(BAND_STEP_THREADS) band_step_kernel(double* __restrict__ AB, int64_t ldab, int N,
                                                                      int kl, int ku, int j, int* __restrict__ ipiv,
                                                                      int* __restrict__ jua, int* __restrict__ state) {
  __shared__ int s_stop;
  const int tid = threadIdx.x;
  if (tid == 0) s_stop = state[1];
  __syncthreads();
  if (s_stop != 0) return;  // an earlier column was singular (uniform within the block)
  const int64_t kv = kl + ku;
  const int km = kl < N - 1 - j ? kl : N - 1 - j;
  const int jp = ipiv[j] - j;
  const int ju = jua[j];
  const double* colj = AB + (int64_t)j * ldab + kv;  // colj[r] = A(j + r, j)
  const double rp = 1.0 / colj[jp], ajj = colj[0];
  for (int c = j + 1 + blockIdx.x; c <= ju; c += gridDim.x) {
    double* colc = AB + (int64_t)c * ldab + (kv + j - c);  // colc[r] = A(j + r, c)
    const double u = colc[jp], old = colc[0];
    __syncthreads();  // every thread holds u and old before the column is written
    for (int r = 1 + tid; r <= km; r += BAND_STEP_THREADS) {
      const double l = (r == jp ? ajj : colj[r]) * rp;
      const double v = r == jp ? old : colc[r];
      colc[r] = fma(-l, u, v);
    }
    if (jp != 0 && tid == 0) colc[0] = u;
    if (c == j + 1) {  // column j + 1 is final now: its pivot for the next launch
      __syncthreads();
      band_pivot_search(AB, ldab, N, kl, ku, j + 1, ju, ipiv, jua, state);
    }
  }
  if (j >= 1 && blockIdx.x == gridDim.x - 1) {
    const int jc = j - 1;
    double* cc = AB + (int64_t)jc * ldab + kv;
    const int jpc = ipiv[jc] - jc;
    const int kmc = kl < N - 1 - jc ? kl : N - 1 - jc;
    const double pc = cc[jpc], acc = cc[0];
    const double rpc = 1.0 / pc;
    __syncthreads();  // every thread holds pc and acc before the column is written
    for (int r = 1 + tid; r <= kmc; r += BAND_STEP_THREADS) cc[r] = (r == jpc ? acc : cc[r]) * rpc;
    if (tid == 0) cc[0] = pc;
  }
}

// x <- A^-1 x with the factor (one block; the steps are sequential)
__global__ void __launch_bounds__(BAND_THREADS) band_solve_kernel(const double* __restrict__ AB, int64_t ldab,
                                                                  int N, int kl, int ku,
                                                                  const int* __restrict__ ipiv,
                                                                  const int* __restrict__ state, double* __restrict__ x) {
  if (state[1] != 0) return;  // singular: the factor (and ipiv past the failing column) is incomplete
  const int tid = threadIdx.x;
  const int64_t kv = kl + ku;
  for (int j = 0; j < N - 1; ++j) {
    if (tid == 0) {
      const int l = ipiv[j];
      if (l != j) { const double t = x[l]; x[l] = x[j]; x[j] = t; }
    }
    __syncthreads();
    const int lm = kl < N - 1 - j ? kl : N - 1 - j;
    const double xj = x[j];
    for (int t = 1 + tid; t <= lm; t += BAND_THREADS) x[j + t] -= AB[kv + t + (int64_t)j * ldab] * xj;
    __syncthreads();
  }
  for (int j = N - 1; j >= 0; --j) {
    if (tid == 0) x[j] /= AB[kv + (int64_t)j * ldab];
    __syncthreads();
    const double xj = x[j];
    const int i0 = j - kl - ku > 0 ? j - kl - ku : 0;
    for (int i = i0 + tid; i < j; i += BAND_THREADS) x[i] -= AB[(kv + i - j) + (int64_t)j * ldab] * xj;
    __syncthreads();
  }
}

// the largest band the direct solve allocates (a sixth of a GB300's memory)
constexpr size_t BAND_MAX_BYTES = (size_t)48 << 30;

// Blocks above this many nodes are not ordered for the direct solve (their band would not fit).
constexpr int64_t BAND_ORDER_MAX_NODES = 262144;

// The block's band order (band_order_host, band_order.cpp) from the block's node pattern, computed
// on the host once per mesh.
static int band_order(vms_ctx* ctx, const SysRange& R, const BandOrder** out) {
  SolverWork& w = ctx_solver(ctx);
  for (const BandOrder& o : w.band_orders)
    if (o.n0 == R.n0 && o.n1 == R.n1) {
      *out = &o;
      return VMS_OK;
    }
  BandOrder o;
  o.n0 = R.n0;
  o.n1 = R.n1;
  const int64_t nodes = R.nodes();
  if (nodes > 0 && nodes <= BAND_ORDER_MAX_NODES) {
    const Mesh& m = ctx_mesh(ctx);
    std::vector<int32_t> rp(4 * nodes + 1);
    cudaError_t e = cudaMemcpy(rp.data(), m.rowptr + 4 * R.n0, sizeof(int32_t) * rp.size(), cudaMemcpyDeviceToHost);
    const int32_t c0 = rp[0];
    std::vector<int32_t> ci(e == cudaSuccess ? (size_t)(rp[4 * nodes] - c0) : 0);
    if (e == cudaSuccess && !ci.empty())
      e = cudaMemcpy(ci.data(), m.colidx + c0, sizeof(int32_t) * ci.size(), cudaMemcpyDeviceToHost);
    if (e != cudaSuccess) return ctx_fail(ctx, VMS_ERR_CUDA, cudaGetErrorString(e));
    // node adjacency (the first scalar row of each node carries the node's block columns)
    std::vector<int32_t> start(nodes + 1, 0), adj;
    adj.reserve((size_t)(rp[1] - rp[0]) / 4 * nodes);
    for (int64_t a = 0; a < nodes; ++a) {
      start[a] = (int32_t)adj.size();
      for (int32_t t = rp[4 * a] - c0; t < rp[4 * a + 1] - c0; t += 4) {
        const int64_t b = (int64_t)(ci[t] >> 2) - R.n0;
        if (b < 0 || b >= nodes) return ctx_fail(ctx, VMS_ERR_INVALID_ARG, "band order: a column outside the block");
        if (b != a) adj.push_back((int32_t)b);
      }
    }
    start[nodes] = (int32_t)adj.size();
    std::vector<int32_t> best(nodes);
    const int bw = band_order_host(nodes, start.data(), adj.data(), best.data());
    e = cudaMalloc(&o.perm, sizeof(int32_t) * nodes);
    if (e == cudaSuccess) e = cudaMemcpy(o.perm, best.data(), sizeof(int32_t) * nodes, cudaMemcpyHostToDevice);
    if (e != cudaSuccess) {
      cudaGetLastError();
      if (o.perm) cudaFree(o.perm);
      return ctx_fail(ctx, e == cudaErrorMemoryAllocation ? VMS_ERR_OUT_OF_MEMORY : VMS_ERR_CUDA, cudaGetErrorString(e));
    }
    o.bw = bw;
  }
  w.band_orders.push_back(o);
  *out = &w.band_orders.back();
  return VMS_OK;
}

// Half-width kl = ku of the block's band in its band order (4 times the order's bandwidth in nodes,
// plus 3) and whether the band storage fits BAND_MAX_BYTES.
static int band_shape(vms_ctx* ctx, const SysRange& R, int* kl_out, bool* fits) {
  const int64_t n = 4 * R.nodes();
  const BandOrder* o = nullptr;
  if (int rc = band_order(ctx, R, &o)) return rc;
  if (o->bw < 0) {
    *kl_out = 0;
    *fits = false;
    return VMS_OK;
  }
  *kl_out = 4 * o->bw + 3;
  const double ldab = 3.0 * *kl_out + 1.0;
  *fits = n <= INT32_MAX / 2 && sizeof(double) * ldab * (double)n <= (double)BAND_MAX_BYTES;
  return VMS_OK;
}

// kl and whether the band fits, for the deadline of a Krylov attempt that a direct solve would
// follow: from the block's band order where it has one, else from its own order (a device
// reduction; the band order, a host computation, is made only when a direct solve runs).
static int band_estimate(vms_ctx* ctx, const SysRange& R, int* kl_out, bool* fits) {
  SolverWork& w = ctx_solver(ctx);
  for (const BandOrder& o : w.band_orders)
    if (o.n0 == R.n0 && o.n1 == R.n1) return band_shape(ctx, R, kl_out, fits);
  const Mesh& m = ctx_mesh(ctx);
  cudaStream_t st = ctx_stream(ctx);
  const int64_t nodes = R.nodes(), n = 4 * nodes;
  if (nodes == 0) {
    *kl_out = 3;
    *fits = true;
    return VMS_OK;
  }
  int bw = 0;
  cudaMemsetAsync(w.band, 0, sizeof(int), st);
  {
    KScope k(ctx, VMS_K_PRECOND);
    band_width_kernel<<<(unsigned)((nodes + 255) / 256), 256, 0, st>>>(m.rowptr, m.colidx, R.n0, nodes, w.band);
    k.add(1);
  }
  cudaMemcpyAsync(&bw, w.band, sizeof(int), cudaMemcpyDeviceToHost, st);
  const cudaError_t e = cudaStreamSynchronize(st);
  if (e != cudaSuccess) return ctx_fail(ctx, VMS_ERR_CUDA, cudaGetErrorString(e));
  *kl_out = 4 * bw + 3;
  const double ldab = 3.0 * *kl_out + 1.0;
  *fits = n <= INT32_MAX / 2 && sizeof(double) * ldab * (double)n <= (double)BAND_MAX_BYTES;
  return VMS_OK;
}

// The instance's system S x = -rhs by banded LU into w.x; *rel_out = |b - S x| / |b| (the matrix
// the assembly left, FP32 or FP64 values). VMS_ERR_UNSUPPORTED if the band would exceed
// BAND_MAX_BYTES, VMS_ERR_ZERO_PIVOT for a singular band.
static int band_direct(vms_ctx* ctx, const SysRange& R, double* rel_out) {
  const Mesh& m = ctx_mesh(ctx);
  Work& wk = ctx_work(ctx);
  SolverWork& w = ctx_solver(ctx);
  cudaStream_t st = ctx_stream(ctx);
  const bool f32 = ctx_fp32(ctx);
  const int64_t nodes = R.nodes(), n = 4 * nodes;
  if (n == 0) {
    *rel_out = 0.0;
    return VMS_OK;
  }
  int kl = 0;
  bool fits = false;
  if (int rc = band_shape(ctx, R, &kl, &fits)) return rc;
  if (!fits) return ctx_fail(ctx, VMS_ERR_UNSUPPORTED, "band solve: band too large");
  const BandOrder* ord = nullptr;
  if (int rc = band_order(ctx, R, &ord)) return rc;
  const int32_t* perm = ord->perm;
  const int ku = kl;
  const int64_t ldab = 2 * (int64_t)kl + ku + 1;
  const size_t bytes = sizeof(double) * (size_t)ldab * (size_t)n;
  int* d_int = w.band;  // [1] the first singular column + 1, [3] scatter error
  int h[4] = {0, 0, 0, 0};
  cudaError_t e = cudaSuccess;
  double* AB = nullptr;
  int* ipiv = nullptr;
  e = cudaMalloc(&AB, bytes);
  if (e == cudaSuccess) e = cudaMalloc(&ipiv, sizeof(int) * 2 * n);
  int* jua = ipiv + n;  // per column: the last column the interchanges up to it reach
  if (e != cudaSuccess) {
    cudaGetLastError();  // an allocation failure is not sticky: clear it for the caller's checks
    cudaFree(AB);
    return ctx_fail(ctx, VMS_ERR_OUT_OF_MEMORY, cudaGetErrorString(e));
  }
  cudaMemsetAsync(AB, 0, bytes, st);
  cudaMemsetAsync(ipiv, 0, sizeof(int) * 2 * n, st);
  cudaMemsetAsync(d_int, 0, sizeof(int) * 4, st);
  {
    KScope kf(ctx, VMS_K_PRECOND);
    const unsigned wb = (unsigned)((nodes * 32 + 255) / 256);
    if (f32)
      band_scatter_kernel<float><<<wb, 256, 0, st>>>(m.rowptr, m.colidx, (const float*)wk.values, perm, R.n0, nodes, AB, ldab, kl, ku, d_int + 3);
    else
      band_scatter_kernel<double><<<wb, 256, 0, st>>>(m.rowptr, m.colidx, (const double*)wk.values, perm, R.n0, nodes, AB, ldab, kl, ku, d_int + 3);
    const unsigned gb = (unsigned)std::min<int64_t>((int64_t)kl + ku, 4 * (int64_t)sm_count());
    band_first_pivot_kernel<<<1, BAND_STEP_THREADS, 0, st>>>(AB, ldab, (int)n, kl, ku, ipiv, jua, d_int);
    for (int j = 0; j < (int)n; ++j)
      band_step_kernel<<<gb, BAND_STEP_THREADS, 0, st>>>(AB, ldab, (int)n, kl, ku, j, ipiv, jua, d_int);
    // b = -rhs into w.rb (block order) and into w.cx (band order), forward and backward
    // substitution in w.cx, the solution back into w.x in the block order
    axpby_kernel<double, double, double><<<grid_for(n), 256, 0, st>>>(-1.0, wk.rhs + 4 * R.n0, 0.0, (const double*)nullptr, w.rb, n);
    band_permute_kernel<<<grid_for(n), 256, 0, st>>>(w.rb, perm, nodes, 1.0, w.cx, 1);
    band_solve_kernel<<<1, BAND_THREADS, 0, st>>>(AB, ldab, (int)n, kl, ku, ipiv, d_int, w.cx);
    band_permute_kernel<<<grid_for(n), 256, 0, st>>>(w.cx, perm, nodes, 1.0, w.x, 0);
    kf.add(6 + (int)n);
  }
  cudaMemcpyAsync(h + 1, d_int + 1, sizeof(int) * 3, cudaMemcpyDeviceToHost, st);
  e = cudaStreamSynchronize(st);
  cudaFree(AB);
  cudaFree(ipiv);
  if (e == cudaSuccess) e = cudaGetLastError();
  if (e != cudaSuccess) return ctx_fail(ctx, VMS_ERR_CUDA, cudaGetErrorString(e));
  if (h[3] != 0) return ctx_fail(ctx, VMS_ERR_CUDA, "band solve: an entry outside the band");
  if (h[1] != 0) return ctx_fail(ctx, VMS_ERR_ZERO_PIVOT, "band solve: singular system");
  // relative residual |b - S x| / |b|
  double* y = w.rfull;
  KScope ks(ctx, VMS_K_SPMV);
  ks.add(f32 ? spmv<float, double>(m, R, wk.values, w.x, y, st) : spmv<double, double>(m, R, wk.values, w.x, y, st));
  axpby_kernel<double, double, double><<<grid_for(n), 256, 0, st>>>(1.0, w.rb, -1.0, y, y, n);
  ks.add(1);
  double* hd = w.h;
  double nb2 = 0.0, nr2 = 0.0;
  dots<double>(w.rb, n, 1, w.rb, n, hd + H_PART, hd + H_NORM, st);
  cudaMemcpyAsync(&nb2, hd + H_NORM, sizeof(double), cudaMemcpyDeviceToHost, st);
  e = cudaStreamSynchronize(st);
  dots<double>(y, n, 1, y, n, hd + H_PART, hd + H_NORM, st);
  ks.add(4);
  cudaMemcpyAsync(&nr2, hd + H_NORM, sizeof(double), cudaMemcpyDeviceToHost, st);
  if (e == cudaSuccess) e = cudaStreamSynchronize(st);
  if (e != cudaSuccess) return ctx_fail(ctx, VMS_ERR_CUDA, cudaGetErrorString(e));
  *rel_out = nb2 > 0.0 ? std::sqrt(nr2 / nb2) : 0.0;
  return VMS_OK;
}

static int recover_and_update(vms_ctx* ctx, const SysRange& R) {
  const Mesh& m = ctx_mesh(ctx);
  State& s = ctx_state(ctx);
  Work& wk = ctx_work(ctx);
  SolverWork& w = ctx_solver(ctx);
  cudaStream_t st = ctx_stream(ctx);
  KScope k(ctx, VMS_K_KRYLOV);
  const int64_t ne = R.e1 - R.e0;
  const unsigned eb = (unsigned)((ne + 127) / 128 > 0 ? (ne + 127) / 128 : 1);
  if (ctx_fp32(ctx))
    recover_kernel<float><<<eb, 128, 0, st>>>(m.conn, m.npe, (const float*)wk.recX, wk.recY, w.x, s.beta, R.e0, R.e1, R.n0);
  else
    recover_kernel<double><<<eb, 128, 0, st>>>(m.conn, m.npe, (const double*)wk.recX, wk.recY, w.x, s.beta, R.e0, R.e1, R.n0);
  const int64_t n = 4 * R.nodes();
  double* u = reinterpret_cast<double*>(s.u) + 4 * R.n0;
  axpby_kernel<double, double, double><<<grid_for(n), 256, 0, st>>>(1.0, u, 1.0, w.x, u, n);
  k.add(2);
  const cudaError_t e = cudaGetLastError();
  return e == cudaSuccess ? VMS_OK : ctx_fail(ctx, VMS_ERR_CUDA, cudaGetErrorString(e));
}

}  // namespace vms

using namespace vms;

extern "C" {

int vms_apply(vms_ctx* ctx, const double* x, double* y) {
  if (!ctx || !x || !y) return ctx_fail(ctx, VMS_ERR_INVALID_ARG, "null argument");
  if (!ctx_work(ctx).assembled) return ctx_fail(ctx, VMS_ERR_STATE, "nothing assembled");
  cudaSetDevice(ctx_device(ctx));
  {
    KScope k(ctx, VMS_K_SPMV);
    k.add(launch_spmv(ctx_mesh(ctx), ctx_work(ctx).values, ctx_fp32(ctx), x, y, ctx_stream(ctx)));
  }
  const cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return ctx_fail(ctx, VMS_ERR_CUDA, cudaGetErrorString(e));
  return VMS_OK;
}

}  // extern "C"

namespace vms {

// Krylov subspace of the Newton driver: the condensed systems of distorted meshes carry a few
// near-null pressure modes (singular values down to 1e-9 of the largest), which restarted GMRES
// resolves only when a cycle is long enough to keep them (GMRES(50) stagnates near 1e-5 on the
// late Newton systems of a jittered 32^3 cavity, GMRES(100) too, GMRES(120) converges). Larger
// meshes need longer cycles still (ILU(0)-preconditioned GMRES(150) stalls near 1e-2 on the first
// Newton system of the 39^3 tetrahedral cavity, GMRES(400) converges): the Newton driver starts at
// 150 and doubles the cycle whenever one does not halve the residual, up to MAX_RESTART.
constexpr int NEWTON_RESTART = 150;

static SysRange whole(vms_ctx* ctx) {
  const Mesh& m = ctx_mesh(ctx);
  return SysRange{0, m.n_nodes, 0, m.n_elems};
}

// Solve, then (if update) recover the bubble increments and update the state. A solve that stops
// at maxit is still applied when its relative residual is below accept_below (inexact Newton).
// instance < 0: the whole system (its state changes invalidate the assembly); instance >= 0: one
// diagonal block (its update leaves the other instances' blocks valid).
static int solve_impl(vms_ctx* ctx, const SysRange& R, int64_t instance, double rtol, int maxit,
                      int restart, int restart_cap, int update, double accept_below, int* iters,
                      double* rel) {
  if (!ctx) return VMS_ERR_INVALID_ARG;
  if (!ctx_work(ctx).assembled) return ctx_fail(ctx, VMS_ERR_STATE, "nothing assembled");
  if (ctx_stale(ctx, instance))
    return ctx_fail(ctx, VMS_ERR_STATE, "state updated since the last assembly");
  cudaSetDevice(ctx_device(ctx));
  int it = 0;
  double r = 0.0;
  int rc = linear_solve(ctx, R, rtol, maxit, restart, restart_cap, &it, &r);
  if ((rc == VMS_ERR_KRYLOV_MAXIT || rc == VMS_ERR_ZERO_PIVOT) &&
      ctx_precond(ctx) == VMS_PRECOND_ILU0_FALLBACK && !(rc == VMS_ERR_KRYLOV_MAXIT && r < accept_below)) {
    // ILU(0) loses all accuracy where its pivots do (growth factors of 1e7-1e16 were measured on
    // coarse high-Reynolds systems): solve directly by banded LU with partial pivoting where the
    // band fits, else repeat the solve from zero with the block-Jacobi preconditioner, whose 4x4
    // inverses are exact, and the longest cycle
    double r2 = 0.0;
    int rcb = band_direct(ctx, R, &r2);
    if (rcb == VMS_OK) {
      r = r2;
      char msg[96];
      std::snprintf(msg, sizeof msg, "banded direct solve above rtol (relative residual %.3e)", r2);
      rc = r2 <= rtol ? VMS_OK : ctx_fail(ctx, VMS_ERR_KRYLOV_MAXIT, msg);
    } else if (rcb == VMS_ERR_UNSUPPORTED || rcb == VMS_ERR_OUT_OF_MEMORY) {
      int it2 = 0;
      rc = linear_solve(ctx, R, rtol, maxit, MAX_RESTART, MAX_RESTART, &it2, &r2, true);
      it += it2;
      r = r2;
    } else {
      rc = rcb;
    }
  }
  ctx_solver_stats(ctx)[0] += 1;
  ctx_solver_stats(ctx)[1] += it;
  if (iters) *iters = it;
  if (rel) *rel = r;
  if (rc == VMS_ERR_KRYLOV_MAXIT && r < accept_below) rc = VMS_OK;
  if (rc != VMS_OK) return rc;
  if (update) {
    if (int rc2 = recover_and_update(ctx, R)) return rc2;
    if (instance < 0) ctx_work(ctx).assembled = false;  // the state changed
    else ctx_mark_stale(ctx, instance);
  }
  const cudaError_t e = cudaStreamSynchronize(ctx_stream(ctx));
  return e == cudaSuccess ? VMS_OK : ctx_fail(ctx, VMS_ERR_CUDA, cudaGetErrorString(e));
}

}  // namespace vms

extern "C" {

int vms_solve(vms_ctx* ctx, double rtol, int maxit, int restart, int update, int* iters,
              double* rel) {
  return solve_impl(ctx, whole(ctx), -1, rtol, maxit, restart, restart, update, 0.0, iters, rel);
}

int vms_set_wait_limit(vms_ctx* ctx, int64_t polls) {
  if (!ctx) return VMS_ERR_INVALID_ARG;
  if (polls < 0 || polls > ((int64_t)1 << 30)) return ctx_fail(ctx, VMS_ERR_INVALID_ARG, "wait limit out of range");
  ctx_solver(ctx).ilu.spin_limit = polls == 0 ? ILU_SPIN_DEFAULT : (uint32_t)polls;
  return VMS_OK;
}

int vms_solve_instance(vms_ctx* ctx, int64_t instance, double rtol, int maxit, int restart,
                       int update, int* iters, double* rel) {
  if (!ctx) return VMS_ERR_INVALID_ARG;
  SysRange R;
  if (!ctx_instance(ctx, instance, &R)) return ctx_fail(ctx, VMS_ERR_INVALID_ARG, "no such instance");
  return solve_impl(ctx, R, instance, rtol, maxit, restart, restart, update, 0.0, iters, rel);
}

int vms_newton_step(vms_ctx* ctx, double* res_norm) {
  if (!ctx) return VMS_ERR_INVALID_ARG;
  double r = 0.0;
  if (int rc = vms_residual(ctx, &r, nullptr)) return rc;
  if (res_norm) *res_norm = r;
  if (int rc = vms_assemble_newton_schur(ctx, nullptr)) return rc;
  int it = 0;
  double rel = 0.0;
  return solve_impl(ctx, whole(ctx), -1, 1e-10, 3000, NEWTON_RESTART, MAX_RESTART, 1, 0.1, &it, &rel);
}

int vms_newton_solve_to(vms_ctx* ctx, double target, int maxit, int* iters, double* hist) {
  if (!ctx || maxit < 0 || !(target > 0.0)) return ctx_fail(ctx, VMS_ERR_INVALID_ARG, "invalid arguments");
  double r0 = 0.0, r = 0.0;
  if (int rc = vms_residual(ctx, &r0, nullptr)) return rc;
  if (hist) hist[0] = r0;
  r = r0;
  int k = 0;
  double r_prev = 0.0, eta_prev = 0.0;
  const bool fp64 = !ctx_fp32(ctx);
  while (k < maxit && r > target) {
    if (int rc = vms_assemble_newton_schur(ctx, nullptr)) return rc;
    // inexact Newton, never tighter than the target needs (a linear residual of eta r <= target/2):
    // Eisenstat and Walker's choice 2 (gamma 0.5, exponent 2, eta_0 0.05, safeguarded by
    // gamma eta_prev^2 when that exceeds 0.1). In mixed precision only while ||R|| > 1e-3 ||R^0||,
    // then a forcing term proportional to the relative residual, capped at 1e-2: the looser late
    // solves of the former leave near-null pressure components that the FP32 inner solve cannot
    // resolve, and the last Newton system then does not converge within the iteration limit.
    double eta;
    if (fp64 || r > 1e-3 * r0) {
      if (k == 0) {
        eta = 0.05;
      } else {
        eta = 0.5 * (r / r_prev) * (r / r_prev);
        const double guard = 0.5 * eta_prev * eta_prev;
        if (guard > 0.1) eta = std::max(eta, guard);
      }
    } else {
      eta = std::min(1e-2, 0.1 * r / r0);
    }
    eta = std::min(0.5, std::max({eta, 0.5 * target / r, 1e-12}));
    r_prev = r;
    eta_prev = eta;
    int it = 0;
    double rel = 0.0;
    if (int rc = solve_impl(ctx, whole(ctx), -1, eta, 3000, NEWTON_RESTART, MAX_RESTART, 1, 0.1, &it, &rel)) return rc;
    ++k;
    if (int rc = vms_residual(ctx, &r, nullptr)) return rc;
    if (hist) hist[k] = r;
    if (!(r == r) || r > 1e6 * r0) {
      if (iters) *iters = k;
      return ctx_fail(ctx, VMS_ERR_NEWTON_DIVERGED, "Newton residual diverged");
    }
  }
  if (iters) *iters = k;
  if (r > target) return ctx_fail(ctx, VMS_ERR_NEWTON_DIVERGED, "Newton reached maxit");
  return VMS_OK;
}

int vms_newton_solve(vms_ctx* ctx, double rtol, int maxit, int* iters, double* hist) {
  if (!ctx || maxit < 0 || !(rtol > 0.0)) return ctx_fail(ctx, VMS_ERR_INVALID_ARG, "invalid arguments");
  double r0 = 0.0;
  if (int rc = vms_residual(ctx, &r0, nullptr)) return rc;
  if (r0 == 0.0) {
    if (iters) *iters = 0;
    if (hist) hist[0] = 0.0;
    return VMS_OK;
  }
  return vms_newton_solve_to(ctx, rtol * r0, maxit, iters, hist);
}

}  // extern "C"
