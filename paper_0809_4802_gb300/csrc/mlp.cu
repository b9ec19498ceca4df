// Learned warm start of the transient Newton iteration (Remark of Section 4.1, Section 4.2): a
// 3-layer MLP (12 -> 128 -> 128 -> 4, tanh) that predicts each node's increment over the next
// backward-Euler step. Weights are stored in BF16, biases, activations and accumulation in FP32.
// Forward, backward (mean squared error) and Adam run in these kernels; Newton then converges to
// the same tolerance from the predicted start, so the network only changes the starting point.
// The three 128-wide contractions of a 64-node tile (H1 W2 in the forward pass; H1^T D and D W2^T
// in the backward pass) run on the tensor cores (mma.sync m16n8k16, BF16 operands, FP32
// accumulation), the FP32 activations split into sums of BF16 terms (mma_bf16.cuh): three terms
// against the BF16 weights (exact products, FP32-level results), two times two terms (three
// products) for H1^T D. The 12-wide input layer, the 4-wide output layer and the small gradient
// blocks stay on the CUDA cores.
//
// Layout of the parameter vector (row-major): W1 [12][128], b1 [128], W2 [128][128], b2 [128],
// W3 [128][4], b3 [4].
#include <cuda_bf16.h>

#include <algorithm>
#include <cmath>
#include <vector>

#include "mma_bf16.cuh"
#include "solver.h"
#include "vms_internal.h"

struct vms_mlp {
  int device = 0;
  cudaStream_t stream = nullptr;
  float* master = nullptr;  // FP32 master copy of all parameters (Adam updates it)
  float* m = nullptr;       // Adam first moments
  float* v = nullptr;       // Adam second moments
  float* grad = nullptr;    // gradient of the last vms_mlp_grad call
  __nv_bfloat16* w = nullptr;  // W1, W2, W3 in BF16 (offsets below)
  float* bias = nullptr;       // b1, b2, b3 in FP32
  double* loss = nullptr;      // device loss accumulator
  float* scratch = nullptr;    // P_N floats (parameter read-back)
  double* colsum = nullptr;    // 16 column sums of squares (vms_mlp_column_rms)
  int t = 0;                   // Adam steps taken
  std::string err;
};

namespace {

using vms::bf16x2_split2;
using vms::bf16x2_split3;
using vms::mma_bf16;

constexpr int NI = VMS_MLP_IN, NW = VMS_MLP_WIDTH, NO = VMS_MLP_OUT;
constexpr int P_W1 = 0, P_B1 = P_W1 + NI * NW, P_W2 = P_B1 + NW, P_B2 = P_W2 + NW * NW,
              P_W3 = P_B2 + NW, P_B3 = P_W3 + NW * NO, P_N = P_B3 + NO;
static_assert(P_N == VMS_MLP_PARAMS, "parameter count");
// BF16 weight array: W1 | W2 | W3; FP32 bias array: b1 | b2 | b3
constexpr int WB_1 = 0, WB_2 = NI * NW, WB_3 = WB_2 + NW * NW, WB_N = WB_3 + NW * NO;
constexpr int BB_1 = 0, BB_2 = NW, BB_3 = 2 * NW, BB_N = 2 * NW + NO;

constexpr int TILE = 64;       // rows (nodes) per tile
constexpr int THREADS = 256;   // 8 warps
constexpr int HLD = NW + 4;    // padded FP32 activation row (conflict-free MMA fragment loads)
constexpr int WLD = NW + 8;    // padded BF16 weight row (68 words: conflict-free fragment loads)

struct Smem {
  float W1[NI][NW];
  __nv_bfloat16 W2t[NW][WLD];  // W2^T [j][k]: B operand of H1 W2 (K index contiguous)
  float W3[NW][NO];
  float b1[NW], b2[NW], b3[NO];
  float X[TILE][NI];
  float H1[TILE][HLD];
  float H2[TILE][HLD];
};
struct SmemGrad : Smem {
  __nv_bfloat16 W2[NW][WLD];   // W2 [k][j]: B operand of D W2^T
  float D[TILE][HLD];
  float dY[TILE][NO];
};

__device__ void load_weights(Smem& s, const __nv_bfloat16* __restrict__ w,
                             const float* __restrict__ bias, __nv_bfloat16 (*W2)[WLD] = nullptr) {
  for (int i = threadIdx.x; i < NI * NW; i += THREADS) s.W1[i / NW][i % NW] = __bfloat162float(w[WB_1 + i]);
  for (int i = threadIdx.x; i < NW * NW; i += THREADS) {
    const int k = i / NW, j = i % NW;
    s.W2t[j][k] = w[WB_2 + i];
    if (W2) W2[k][j] = w[WB_2 + i];
  }
  for (int i = threadIdx.x; i < NW * NO; i += THREADS) s.W3[i / NO][i % NO] = __bfloat162float(w[WB_3 + i]);
  for (int i = threadIdx.x; i < NW; i += THREADS) { s.b1[i] = bias[BB_1 + i]; s.b2[i] = bias[BB_2 + i]; }
  if (threadIdx.x < NO) s.b3[threadIdx.x] = bias[BB_3 + threadIdx.x];
}

// C[64 x 128] = A[64 x 128] B on the tensor cores, B given as Bk[n][k] (BF16, K contiguous), A
// FP32 split into three BF16 terms. Warp w owns rows 16 (w & 3) .. + 15 and columns
// 64 (w >> 2) .. + 63 (eight 8-wide tiles); acc[nt][*] is the standard m16n8 C fragment (rows g,
// g + 8 and columns 2t, 2t + 1 of tile nt, g = lane / 4, t = lane % 4), initialised by the caller.
__device__ __forceinline__ void mma_rows64(const float (*A)[HLD], const __nv_bfloat16 (*Bk)[WLD],
                                           float acc[8][4]) {
  const int w = threadIdx.x >> 5, lane = threadIdx.x & 31, g = lane >> 2, t = lane & 3;
  const int r0 = 16 * (w & 3) + g, c0 = 64 * (w >> 2);
#pragma unroll 2
  for (int k0 = 0; k0 < NW; k0 += 16) {
    uint32_t ah[4], am[4], al[4];
#pragma unroll
    for (int f = 0; f < 4; ++f) {
      const float2 x = *reinterpret_cast<const float2*>(&A[r0 + 8 * (f & 1)][k0 + 2 * t + 8 * (f >> 1)]);
      bf16x2_split3(x.x, x.y, ah[f], am[f], al[f]);
    }
#pragma unroll
    for (int nt = 0; nt < 8; ++nt) {
      const __nv_bfloat16* br = &Bk[c0 + 8 * nt + g][k0 + 2 * t];
      const uint32_t b0 = *reinterpret_cast<const uint32_t*>(br);
      const uint32_t b1 = *reinterpret_cast<const uint32_t*>(br + 8);
      mma_bf16(acc[nt], al, b0, b1);
      mma_bf16(acc[nt], am, b0, b1);
      mma_bf16(acc[nt], ah, b0, b1);
    }
  }
}

// H2 = tanh(H1 W2 + b2) on the tensor cores
__device__ __forceinline__ void dense2_tanh(Smem& s) {
  const int w = threadIdx.x >> 5, lane = threadIdx.x & 31, g = lane >> 2, t = lane & 3;
  const int r0 = 16 * (w & 3) + g, c0 = 64 * (w >> 2);
  float acc[8][4];
#pragma unroll
  for (int nt = 0; nt < 8; ++nt) {
    const int c = c0 + 8 * nt + 2 * t;
    acc[nt][0] = acc[nt][2] = s.b2[c];
    acc[nt][1] = acc[nt][3] = s.b2[c + 1];
  }
  mma_rows64(s.H1, s.W2t, acc);
#pragma unroll
  for (int nt = 0; nt < 8; ++nt) {
    const int c = c0 + 8 * nt + 2 * t;
    *reinterpret_cast<float2*>(&s.H2[r0][c]) = make_float2(tanhf(acc[nt][0]), tanhf(acc[nt][1]));
    *reinterpret_cast<float2*>(&s.H2[r0 + 8][c]) = make_float2(tanhf(acc[nt][2]), tanhf(acc[nt][3]));
  }
}

// rows [r0, r0 + TILE) of X (through `rows` if given) into shared memory, zero beyond n
__device__ void load_tile(Smem& s, const float* __restrict__ X, const int32_t* __restrict__ rows,
                          int64_t r0, int64_t n) {
  for (int i = threadIdx.x; i < TILE * NI; i += THREADS) {
    const int r = i / NI, c = i % NI;
    const int64_t g = r0 + r;
    float x = 0.f;
    if (g < n) x = X[(rows ? (int64_t)rows[g] : g) * NI + c];
    s.X[r][c] = x;
  }
}

// H = tanh(A W + b) for the tile on the CUDA cores (the 12-wide input layer): A [TILE][K] in
// shared memory, W [K][NW] (leading dimension LD); warp w owns rows 8w..8w+7, lane l columns
// l + 32 j
template <int K, int LD>
__device__ void dense_tanh(const float (*A)[K], const float* W, const float* b, float (*H)[HLD]) {
  const int w = threadIdx.x >> 5, l = threadIdx.x & 31;
  float acc[8][4];
#pragma unroll
  for (int r = 0; r < 8; ++r)
#pragma unroll
    for (int j = 0; j < 4; ++j) acc[r][j] = b[l + 32 * j];
#pragma unroll 4
  for (int k = 0; k < K; ++k) {
    float wv[4];
#pragma unroll
    for (int j = 0; j < 4; ++j) wv[j] = W[k * LD + l + 32 * j];
#pragma unroll
    for (int r = 0; r < 8; ++r) {
      const float a = A[8 * w + r][k];
#pragma unroll
      for (int j = 0; j < 4; ++j) acc[r][j] = fmaf(a, wv[j], acc[r][j]);
    }
  }
#pragma unroll
  for (int r = 0; r < 8; ++r)
#pragma unroll
    for (int j = 0; j < 4; ++j) H[8 * w + r][l + 32 * j] = tanhf(acc[r][j]);
}

// y[r][o] = b3[o] + sum_k H2[r][k] W3[k][o], thread = (r, o)
__device__ float dense_out(const Smem& s, int r, int o) {
  float y = s.b3[o];
#pragma unroll 8
  for (int k = 0; k < NW; ++k) y = fmaf(s.H2[r][k], s.W3[k][o], y);
  return y;
}

__global__ void __launch_bounds__(THREADS) mlp_forward_kernel(const __nv_bfloat16* __restrict__ w,
                                                              const float* __restrict__ bias,
                                                              const float* __restrict__ X,
                                                              int64_t n, float* __restrict__ Y) {
  extern __shared__ __align__(16) unsigned char raw[];
  Smem& s = *reinterpret_cast<Smem*>(raw);
  load_weights(s, w, bias);
  for (int64_t r0 = (int64_t)blockIdx.x * TILE; r0 < n; r0 += (int64_t)gridDim.x * TILE) {
    __syncthreads();
    load_tile(s, X, nullptr, r0, n);
    __syncthreads();
    dense_tanh<NI, NW>(s.X, &s.W1[0][0], s.b1, s.H1);
    __syncthreads();
    dense2_tanh(s);
    __syncthreads();
    const int r = threadIdx.x >> 2, o = threadIdx.x & 3;
    const float y = dense_out(s, r, o);
    if (r0 + r < n) Y[(r0 + r) * NO + o] = y;
  }
}

// Gradient of loss = sum over the n rows and 4 outputs of (y - t)^2 / (4 n), accumulated per CTA
// in registers and added to grad (FP32) once; the loss (FP64) likewise.
__global__ void __launch_bounds__(THREADS) mlp_grad_kernel(
    const __nv_bfloat16* __restrict__ w, const float* __restrict__ bias, const float* __restrict__ X,
    const float* __restrict__ T, const int32_t* __restrict__ rows, int64_t n, float scale,
    float* __restrict__ grad, double* __restrict__ loss) {
  extern __shared__ __align__(16) unsigned char raw[];
  SmemGrad& s = *reinterpret_cast<SmemGrad*>(raw);
  load_weights(s, w, bias, s.W2);
  const int tid = threadIdx.x, wp = tid >> 5, l = tid & 31, g = l >> 2, t = l & 3;
  // register partials: dW2 as MMA C fragments (warp wp: rows k = 16 wp + g (+ 8) of dW2, column
  // tiles 0..15), dW1 (6 entries), dW3 (2 entries), db1/db2 (threads < 128: column tid), db3
  // (threads < 4)
  float gW2[16][4], gW1[6], gW3[2], gb1 = 0.f, gb2 = 0.f, gb3 = 0.f;
#pragma unroll
  for (int nt = 0; nt < 16; ++nt)
#pragma unroll
    for (int q = 0; q < 4; ++q) gW2[nt][q] = 0.f;
#pragma unroll
  for (int i = 0; i < 6; ++i) gW1[i] = 0.f;
  gW3[0] = gW3[1] = 0.f;
  double lsum = 0.0;
  for (int64_t r0 = (int64_t)blockIdx.x * TILE; r0 < n; r0 += (int64_t)gridDim.x * TILE) {
    __syncthreads();
    load_tile(s, X, rows, r0, n);
    __syncthreads();
    dense_tanh<NI, NW>(s.X, &s.W1[0][0], s.b1, s.H1);
    __syncthreads();
    dense2_tanh(s);
    __syncthreads();
    {
      const int r = tid >> 2, o = tid & 3;
      const int64_t gr = r0 + r;
      float d = 0.f;
      if (gr < n) {
        const float y = dense_out(s, r, o);
        const float e = y - T[(rows ? (int64_t)rows[gr] : gr) * NO + o];
        lsum += (double)e * (double)e;
        d = 2.f * scale * e;
      }
      s.dY[r][o] = d;
    }
    __syncthreads();
    // dW3, db3
#pragma unroll
    for (int q = 0; q < 2; ++q) {
      const int e = tid + THREADS * q, k = e / NO, o = e % NO;
      float a = 0.f;
      for (int r = 0; r < TILE; ++r) a = fmaf(s.H2[r][k], s.dY[r][o], a);
      gW3[q] += a;
    }
    if (tid < NO)
      for (int r = 0; r < TILE; ++r) gb3 += s.dY[r][tid];
    // D = dH2 = (dY W3^T) * (1 - H2^2)
#pragma unroll
    for (int r = 0; r < 8; ++r)
#pragma unroll
      for (int j = 0; j < 4; ++j) {
        const int rr = 8 * wp + r, c = l + 32 * j;
        float a = 0.f;
#pragma unroll
        for (int o = 0; o < NO; ++o) a = fmaf(s.dY[rr][o], s.W3[c][o], a);
        const float h = s.H2[rr][c];
        s.D[rr][c] = a * (1.f - h * h);
      }
    __syncthreads();
    // dW2[k][j] += sum_r H1[r][k] D[r][j] on the tensor cores: A = H1^T (rows k = 16 wp ..), B = D,
    // both split into two BF16 terms, products hi hi + hi lo + lo hi
#pragma unroll 1
    for (int k0 = 0; k0 < TILE; k0 += 16) {
      uint32_t ah[4], al[4];
#pragma unroll
      for (int f = 0; f < 4; ++f) {
        const int m = 16 * wp + g + 8 * (f & 1), kr = k0 + 2 * t + 8 * (f >> 1);
        bf16x2_split2(s.H1[kr][m], s.H1[kr + 1][m], ah[f], al[f]);
      }
#pragma unroll
      for (int nt = 0; nt < 16; ++nt) {
        const int c = 8 * nt + g, kr = k0 + 2 * t;
        uint32_t bh0, bl0, bh1, bl1;
        bf16x2_split2(s.D[kr][c], s.D[kr + 1][c], bh0, bl0);
        bf16x2_split2(s.D[kr + 8][c], s.D[kr + 9][c], bh1, bl1);
        mma_bf16(gW2[nt], al, bh0, bh1);
        mma_bf16(gW2[nt], ah, bl0, bl1);
        mma_bf16(gW2[nt], ah, bh0, bh1);
      }
    }
    if (tid < NW)
      for (int r = 0; r < TILE; ++r) gb2 += s.D[r][tid];
    // dH1 = (D W2^T) * (1 - H1^2) on the tensor cores (B = W2 [k][j], K = j contiguous), written
    // over H2 (no longer needed)
    {
      const int rr = 16 * (wp & 3) + g, c0 = 64 * (wp >> 2);
      float acc[8][4];
#pragma unroll
      for (int nt = 0; nt < 8; ++nt)
#pragma unroll
        for (int q = 0; q < 4; ++q) acc[nt][q] = 0.f;
      mma_rows64(s.D, s.W2, acc);
#pragma unroll
      for (int nt = 0; nt < 8; ++nt) {
        const int c = c0 + 8 * nt + 2 * t;
#pragma unroll
        for (int hf = 0; hf < 2; ++hf) {
          const int r = rr + 8 * hf;
          const float h0 = s.H1[r][c], h1 = s.H1[r][c + 1];
          *reinterpret_cast<float2*>(&s.H2[r][c]) =
              make_float2(acc[nt][2 * hf] * (1.f - h0 * h0), acc[nt][2 * hf + 1] * (1.f - h1 * h1));
        }
      }
    }
    __syncthreads();
    // dW1[k][j] += sum_r X[r][k] dH1[r][j], db1
#pragma unroll
    for (int q = 0; q < 6; ++q) {
      const int e = tid + THREADS * q, k = e / NW, j = e % NW;
      float a = 0.f;
      for (int r = 0; r < TILE; ++r) a = fmaf(s.X[r][k], s.H2[r][j], a);
      gW1[q] += a;
    }
    if (tid < NW)
      for (int r = 0; r < TILE; ++r) gb1 += s.H2[r][tid];
  }
  // flush the partials
#pragma unroll
  for (int nt = 0; nt < 16; ++nt)
#pragma unroll
    for (int q = 0; q < 4; ++q) {
      const int k = 16 * wp + g + 8 * (q >> 1), j = 8 * nt + 2 * t + (q & 1);
      atomicAdd(grad + P_W2 + k * NW + j, gW2[nt][q]);
    }
#pragma unroll
  for (int q = 0; q < 6; ++q) atomicAdd(grad + P_W1 + tid + THREADS * q, gW1[q]);
#pragma unroll
  for (int q = 0; q < 2; ++q) atomicAdd(grad + P_W3 + tid + THREADS * q, gW3[q]);
  if (tid < NW) {
    atomicAdd(grad + P_B1 + tid, gb1);
    atomicAdd(grad + P_B2 + tid, gb2);
  }
  if (tid < NO) atomicAdd(grad + P_B3 + tid, gb3);
  for (int o = 16; o > 0; o >>= 1) lsum += __shfl_xor_sync(0xffffffffu, lsum, o);
  if (l == 0) atomicAdd(loss, lsum * (double)scale);
}

// Adam on every parameter; the BF16 weights and FP32 biases the kernels use are refreshed from
// the master copy. c1 = 1 / (1 - beta1^t), c2 = 1 / (1 - beta2^t).
__global__ void mlp_adam_kernel(float* __restrict__ master, float* __restrict__ m,
                                float* __restrict__ v, const float* __restrict__ grad,
                                __nv_bfloat16* __restrict__ w, float* __restrict__ bias, float lr,
                                float b1, float b2, float eps, float c1, float c2) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= P_N) return;
  const float g = grad[i];
  const float mi = b1 * m[i] + (1.f - b1) * g;
  const float vi = b2 * v[i] + (1.f - b2) * g * g;
  m[i] = mi;
  v[i] = vi;
  const float x = master[i] - lr * (mi * c1) / (sqrtf(vi * c2) + eps);
  master[i] = x;
  if (i < P_B1) w[WB_1 + i] = __float2bfloat16_rn(x);
  else if (i < P_W2) bias[BB_1 + i - P_B1] = x;
  else if (i < P_B2) w[WB_2 + i - P_W2] = __float2bfloat16_rn(x);
  else if (i < P_W3) bias[BB_2 + i - P_B2] = x;
  else if (i < P_B3) w[WB_3 + i - P_W3] = __float2bfloat16_rn(x);
  else bias[BB_3 + i - P_B3] = x;
}

__global__ void mlp_store_kernel(const float* __restrict__ master, __nv_bfloat16* __restrict__ w,
                                 float* __restrict__ bias) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= P_N) return;
  const float x = master[i];
  if (i < P_B1) w[WB_1 + i] = __float2bfloat16_rn(x);
  else if (i < P_W2) bias[BB_1 + i - P_B1] = x;
  else if (i < P_B2) w[WB_2 + i - P_W2] = __float2bfloat16_rn(x);
  else if (i < P_W3) bias[BB_2 + i - P_B2] = x;
  else if (i < P_B3) w[WB_3 + i - P_W3] = __float2bfloat16_rn(x);
  else bias[BB_3 + i - P_B3] = x;
}

__global__ void mlp_stored_kernel(const __nv_bfloat16* __restrict__ w, const float* __restrict__ bias,
                                  float* __restrict__ out) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= P_N) return;
  float x;
  if (i < P_B1) x = __bfloat162float(w[WB_1 + i]);
  else if (i < P_W2) x = bias[BB_1 + i - P_B1];
  else if (i < P_B2) x = __bfloat162float(w[WB_2 + i - P_W2]);
  else if (i < P_W3) x = bias[BB_2 + i - P_B2];
  else if (i < P_B3) x = __bfloat162float(w[WB_3 + i - P_W3]);
  else x = bias[BB_3 + i - P_B3];
  out[i] = x;
}

unsigned grid_rows(int64_t n) {
  const int64_t tiles = (n + TILE - 1) / TILE;
  const int64_t sms = vms::sm_count();
  return (unsigned)(tiles < 1 ? 1 : (tiles > sms ? sms : tiles));
}

int mfail(vms_mlp* p, int code, const char* msg) {
  if (p) p->err = msg;
  return code;
}

#define MCK(call)                                                             \
  do {                                                                        \
    cudaError_t e_ = (call);                                                  \
    if (e_ != cudaSuccess)                                                    \
      return mfail(mlp, e_ == cudaErrorMemoryAllocation ? VMS_ERR_OUT_OF_MEMORY \
                                                        : VMS_ERR_CUDA,        \
                   cudaGetErrorString(e_));                                   \
  } while (0)

// ---------------------------------------------------------------------------------------------
// node features and increments on a context's state
// ---------------------------------------------------------------------------------------------
struct Scales {
  float in[NI];
  float out[NO];
};

// X[n] = [u^n, u^{n-1}, mean of u^n over the 1-ring] / scale_in; the 1-ring is read from the CSR
// pattern (node row n lists its neighbours, the node itself included)
__global__ void node_features_kernel(const int32_t* __restrict__ rowptr,
                                     const int32_t* __restrict__ colidx,
                                     const double4_32a* __restrict__ u,
                                     const double4_32a* __restrict__ up, int64_t n_nodes,
                                     Scales sc, float* __restrict__ X) {
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n_nodes) return;
  const int32_t r0 = rowptr[4 * i];
  const int deg = (rowptr[4 * i + 1] - r0) >> 2;
  double s[4] = {0.0, 0.0, 0.0, 0.0};
  int cnt = 0;
  for (int k = 0; k < deg; ++k) {
    const int64_t j = colidx[r0 + 4 * k] >> 2;
    if (j == i) continue;
    const double4_32a w = u[j], wp = up[j];
    s[0] += w.x - wp.x; s[1] += w.y - wp.y; s[2] += w.z - wp.z; s[3] += w.w - wp.w;
    ++cnt;
  }
  const double inv = cnt ? 1.0 / cnt : 0.0;
  const double4_32a a = u[i], b = up[i];
  // the last step's increment is given directly: a network with BF16 weights cannot form it from
  // u^n and u^(n-1), which agree in their leading digits
  const double f[NI] = {a.x, a.y, a.z, a.w, a.x - b.x, a.y - b.y, a.z - b.z, a.w - b.w,
                        s[0] * inv, s[1] * inv, s[2] * inv, s[3] * inv};
#pragma unroll
  for (int c = 0; c < NI; ++c) X[i * NI + c] = (float)(f[c] / (double)sc.in[c]);
}

__global__ void node_increment_kernel(const double4_32a* __restrict__ u,
                                      const double4_32a* __restrict__ up, int64_t n_nodes,
                                      Scales sc, float* __restrict__ D) {
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n_nodes) return;
  const double4_32a a = u[i], b = up[i];
  D[4 * i + 0] = (float)((a.x - b.x) / sc.out[0]);
  D[4 * i + 1] = (float)((a.y - b.y) / sc.out[1]);
  D[4 * i + 2] = (float)((a.z - b.z) / sc.out[2]);
  D[4 * i + 3] = (float)((a.w - b.w) / sc.out[3]);
}

__global__ void apply_increment_kernel(double4_32a* __restrict__ u, int64_t n_nodes, Scales sc,
                                       const float* __restrict__ D) {
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n_nodes) return;
  double4_32a a = u[i];
  a.x += (double)sc.out[0] * D[4 * i + 0];
  a.y += (double)sc.out[1] * D[4 * i + 1];
  a.z += (double)sc.out[2] * D[4 * i + 2];
  a.w += (double)sc.out[3] * D[4 * i + 3];
  u[i] = a;
}

// per-column sums of squares (FP64): each thread accumulates the columns of a grid-stride set of
// rows, the block combines them in shared memory and adds them to sums once
constexpr int COLS_MAX = 16;
struct ColMul {
  float m[COLS_MAX];
};

__global__ void column_sumsq_kernel(const float* __restrict__ X, int64_t n, int cols,
                                    double* __restrict__ sums) {
  __shared__ double part[COLS_MAX];
  if (threadIdx.x < COLS_MAX) part[threadIdx.x] = 0.0;
  __syncthreads();
  double acc[COLS_MAX];
#pragma unroll
  for (int c = 0; c < COLS_MAX; ++c) acc[c] = 0.0;
  for (int64_t r = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; r < n; r += (int64_t)gridDim.x * blockDim.x)
#pragma unroll
    for (int c = 0; c < COLS_MAX; ++c)
      if (c < cols) {
        const double x = X[r * cols + c];
        acc[c] += x * x;
      }
  for (int c = 0; c < cols; ++c) {
    double v = acc[c];
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    if ((threadIdx.x & 31) == 0) atomicAdd(&part[c], v);
  }
  __syncthreads();
  if (threadIdx.x < cols) atomicAdd(sums + threadIdx.x, part[threadIdx.x]);
}

__global__ void scale_columns_kernel(const float* __restrict__ X, int64_t n, int cols, ColMul mul,
                                     float* __restrict__ out) {
  const int64_t total = n * cols;
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < total; i += (int64_t)gridDim.x * blockDim.x)
    out[i] = X[i] * mul.m[i % cols];
}

}  // namespace

extern "C" {

int vms_mlp_create(vms_mlp** out, int device) {
  if (!out) return VMS_ERR_INVALID_ARG;
  *out = nullptr;
  vms_mlp* mlp = new vms_mlp();
  mlp->device = device;
  auto cleanup = [&](int rc) { vms_mlp_destroy(mlp); return rc; };
  if (cudaSetDevice(device) != cudaSuccess) return cleanup(VMS_ERR_CUDA);
  cudaError_t e = cudaMalloc(&mlp->master, sizeof(float) * P_N);
  if (e == cudaSuccess) e = cudaMalloc(&mlp->m, sizeof(float) * P_N);
  if (e == cudaSuccess) e = cudaMalloc(&mlp->v, sizeof(float) * P_N);
  if (e == cudaSuccess) e = cudaMalloc(&mlp->grad, sizeof(float) * P_N);
  if (e == cudaSuccess) e = cudaMalloc(&mlp->w, sizeof(__nv_bfloat16) * WB_N);
  if (e == cudaSuccess) e = cudaMalloc(&mlp->bias, sizeof(float) * BB_N);
  if (e == cudaSuccess) e = cudaMalloc(&mlp->loss, sizeof(double));
  if (e == cudaSuccess) e = cudaMalloc(&mlp->scratch, sizeof(float) * P_N);
  if (e == cudaSuccess) e = cudaMalloc(&mlp->colsum, sizeof(double) * 16);
  for (void* p : {(void*)mlp->master, (void*)mlp->m, (void*)mlp->v, (void*)mlp->grad, (void*)mlp->bias})
    if (e == cudaSuccess) e = cudaMemset(p, 0, sizeof(float) * (p == (void*)mlp->bias ? BB_N : P_N));
  if (e == cudaSuccess) e = cudaMemset(mlp->w, 0, sizeof(__nv_bfloat16) * WB_N);
  if (e == cudaSuccess)
    e = cudaFuncSetAttribute(mlp_forward_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sizeof(Smem));
  if (e == cudaSuccess)
    e = cudaFuncSetAttribute(mlp_grad_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sizeof(SmemGrad));
  if (e != cudaSuccess) return cleanup(e == cudaErrorMemoryAllocation ? VMS_ERR_OUT_OF_MEMORY : VMS_ERR_CUDA);
  *out = mlp;
  return VMS_OK;
}

int vms_mlp_destroy(vms_mlp* mlp) {
  if (!mlp) return VMS_OK;
  cudaSetDevice(mlp->device);
  if (mlp->stream) cudaStreamSynchronize(mlp->stream);
  for (void* p : {(void*)mlp->master, (void*)mlp->m, (void*)mlp->v, (void*)mlp->grad, (void*)mlp->w,
                  (void*)mlp->bias, (void*)mlp->loss, (void*)mlp->scratch, (void*)mlp->colsum})
    if (p) cudaFree(p);
  delete mlp;
  return VMS_OK;
}

const char* vms_mlp_last_error(vms_mlp* mlp) { return mlp ? mlp->err.c_str() : "null handle"; }

int vms_mlp_set_stream(vms_mlp* mlp, void* stream) {
  if (!mlp) return VMS_ERR_INVALID_ARG;
  mlp->stream = reinterpret_cast<cudaStream_t>(stream);
  return VMS_OK;
}

int vms_mlp_set_params(vms_mlp* mlp, const float* params) {
  if (!mlp || !params) return mfail(mlp, VMS_ERR_INVALID_ARG, "null argument");
  MCK(cudaSetDevice(mlp->device));
  MCK(cudaMemcpyAsync(mlp->master, params, sizeof(float) * P_N, cudaMemcpyDefault, mlp->stream));
  MCK(cudaMemsetAsync(mlp->m, 0, sizeof(float) * P_N, mlp->stream));
  MCK(cudaMemsetAsync(mlp->v, 0, sizeof(float) * P_N, mlp->stream));
  mlp_store_kernel<<<(P_N + 255) / 256, 256, 0, mlp->stream>>>(mlp->master, mlp->w, mlp->bias);
  MCK(cudaGetLastError());
  MCK(cudaStreamSynchronize(mlp->stream));
  mlp->t = 0;
  return VMS_OK;
}

int vms_mlp_get_params(vms_mlp* mlp, float* params, int stored) {
  if (!mlp || !params) return mfail(mlp, VMS_ERR_INVALID_ARG, "null argument");
  MCK(cudaSetDevice(mlp->device));
  if (stored) {
    mlp_stored_kernel<<<(P_N + 255) / 256, 256, 0, mlp->stream>>>(mlp->w, mlp->bias, mlp->scratch);
    MCK(cudaGetLastError());
    MCK(cudaMemcpyAsync(params, mlp->scratch, sizeof(float) * P_N, cudaMemcpyDefault, mlp->stream));
  } else {
    MCK(cudaMemcpyAsync(params, mlp->master, sizeof(float) * P_N, cudaMemcpyDefault, mlp->stream));
  }
  MCK(cudaStreamSynchronize(mlp->stream));
  return VMS_OK;
}

int vms_mlp_forward(vms_mlp* mlp, int64_t n, const float* X, float* Y) {
  if (!mlp || n < 0 || (n > 0 && (!X || !Y))) return mfail(mlp, VMS_ERR_INVALID_ARG, "invalid arguments");
  if (n == 0) return VMS_OK;
  MCK(cudaSetDevice(mlp->device));
  mlp_forward_kernel<<<grid_rows(n), THREADS, sizeof(Smem), mlp->stream>>>(mlp->w, mlp->bias, X, n, Y);
  MCK(cudaGetLastError());
  return VMS_OK;
}

int vms_mlp_grad(vms_mlp* mlp, int64_t n, const int32_t* rows, const float* X, const float* T,
                 double* loss, float* grads) {
  if (!mlp || n <= 0 || !X || !T) return mfail(mlp, VMS_ERR_INVALID_ARG, "invalid arguments");
  MCK(cudaSetDevice(mlp->device));
  MCK(cudaMemsetAsync(mlp->grad, 0, sizeof(float) * P_N, mlp->stream));
  MCK(cudaMemsetAsync(mlp->loss, 0, sizeof(double), mlp->stream));
  const float scale = (float)(1.0 / (4.0 * (double)n));
  mlp_grad_kernel<<<grid_rows(n), THREADS, sizeof(SmemGrad), mlp->stream>>>(
      mlp->w, mlp->bias, X, T, rows, n, scale, mlp->grad, mlp->loss);
  MCK(cudaGetLastError());
  if (loss) MCK(cudaMemcpyAsync(loss, mlp->loss, sizeof(double), cudaMemcpyDeviceToHost, mlp->stream));
  if (grads) MCK(cudaMemcpyAsync(grads, mlp->grad, sizeof(float) * P_N, cudaMemcpyDefault, mlp->stream));
  if (loss || grads) MCK(cudaStreamSynchronize(mlp->stream));
  return VMS_OK;
}

int vms_mlp_adam(vms_mlp* mlp, float lr) {
  if (!mlp || !(lr > 0.f)) return mfail(mlp, VMS_ERR_INVALID_ARG, "invalid arguments");
  MCK(cudaSetDevice(mlp->device));
  mlp->t += 1;
  const double b1 = 0.9, b2 = 0.999;
  const float c1 = (float)(1.0 / (1.0 - std::pow(b1, mlp->t)));
  const float c2 = (float)(1.0 / (1.0 - std::pow(b2, mlp->t)));
  mlp_adam_kernel<<<(P_N + 255) / 256, 256, 0, mlp->stream>>>(mlp->master, mlp->m, mlp->v, mlp->grad,
                                                              mlp->w, mlp->bias, lr, (float)b1,
                                                              (float)b2, 1e-8f, c1, c2);
  MCK(cudaGetLastError());
  return VMS_OK;
}

int vms_mlp_column_rms(vms_mlp* mlp, int64_t n, int cols, const float* X, double* rms) {
  if (!mlp || n <= 0 || cols < 1 || cols > COLS_MAX || !X || !rms)
    return mfail(mlp, VMS_ERR_INVALID_ARG, "invalid arguments");
  MCK(cudaSetDevice(mlp->device));
  MCK(cudaMemsetAsync(mlp->colsum, 0, sizeof(double) * COLS_MAX, mlp->stream));
  const int64_t blocks = std::min<int64_t>((n + 255) / 256, 4 * (int64_t)vms::sm_count());
  column_sumsq_kernel<<<(unsigned)blocks, 256, 0, mlp->stream>>>(X, n, cols, mlp->colsum);
  MCK(cudaGetLastError());
  double h[COLS_MAX];
  MCK(cudaMemcpyAsync(h, mlp->colsum, sizeof(double) * cols, cudaMemcpyDeviceToHost, mlp->stream));
  MCK(cudaStreamSynchronize(mlp->stream));
  for (int c = 0; c < cols; ++c) rms[c] = std::sqrt(h[c] / (double)n);
  return VMS_OK;
}

int vms_mlp_scale_columns(vms_mlp* mlp, int64_t n, int cols, const float* X, const float* mul,
                          float* out) {
  if (!mlp || n < 0 || cols < 1 || cols > COLS_MAX || !mul || (n > 0 && (!X || !out)))
    return mfail(mlp, VMS_ERR_INVALID_ARG, "invalid arguments");
  if (n == 0) return VMS_OK;
  MCK(cudaSetDevice(mlp->device));
  ColMul m{};
  for (int c = 0; c < cols; ++c) m.m[c] = mul[c];
  const int64_t blocks = std::min<int64_t>((n * cols + 255) / 256, 4 * (int64_t)vms::sm_count());
  scale_columns_kernel<<<(unsigned)blocks, 256, 0, mlp->stream>>>(X, n, cols, m, out);
  MCK(cudaGetLastError());
  return VMS_OK;
}

}  // extern "C"

// ---------------------------------------------------------------------------------------------
// context-side calls of the transient driver
// ---------------------------------------------------------------------------------------------
using namespace vms;

extern "C" {

int vms_node_features(vms_ctx* ctx, const float* scale_in, float* X) {
  if (!ctx || !X) return ctx_fail(ctx, VMS_ERR_INVALID_ARG, "null argument");
  const Mesh& m = ctx_mesh(ctx);
  State& s = ctx_state(ctx);
  if (!s.valid) return ctx_fail(ctx, VMS_ERR_STATE, "no state uploaded");
  Scales sc;
  for (int c = 0; c < NI; ++c) sc.in[c] = scale_in ? scale_in[c] : 1.f;
  for (int c = 0; c < NO; ++c) sc.out[c] = 1.f;
  for (int c = 0; c < NI; ++c)
    if (!(sc.in[c] != 0.f)) return ctx_fail(ctx, VMS_ERR_INVALID_ARG, "zero feature scale");
  cudaSetDevice(ctx_device(ctx));
  const unsigned blocks = (unsigned)((m.n_nodes + 255) / 256);
  node_features_kernel<<<blocks, 256, 0, ctx_stream(ctx)>>>(m.rowptr, m.colidx, s.u, s.u_prev,
                                                              m.n_nodes, sc, X);
  const cudaError_t e = cudaGetLastError();
  return e == cudaSuccess ? VMS_OK : ctx_fail(ctx, VMS_ERR_CUDA, cudaGetErrorString(e));
}

int vms_node_increment(vms_ctx* ctx, const float* scale_out, float* D) {
  if (!ctx || !D) return ctx_fail(ctx, VMS_ERR_INVALID_ARG, "null argument");
  const Mesh& m = ctx_mesh(ctx);
  State& s = ctx_state(ctx);
  if (!s.valid) return ctx_fail(ctx, VMS_ERR_STATE, "no state uploaded");
  Scales sc;
  for (int c = 0; c < NO; ++c) sc.out[c] = scale_out ? scale_out[c] : 1.f;
  for (int c = 0; c < NO; ++c)
    if (!(sc.out[c] != 0.f)) return ctx_fail(ctx, VMS_ERR_INVALID_ARG, "zero output scale");
  cudaSetDevice(ctx_device(ctx));
  const unsigned blocks = (unsigned)((m.n_nodes + 255) / 256);
  node_increment_kernel<<<blocks, 256, 0, ctx_stream(ctx)>>>(s.u, s.u_prev, m.n_nodes, sc, D);
  const cudaError_t e = cudaGetLastError();
  return e == cudaSuccess ? VMS_OK : ctx_fail(ctx, VMS_ERR_CUDA, cudaGetErrorString(e));
}

int vms_apply_increment(vms_ctx* ctx, const float* scale_out, const float* D) {
  if (!ctx || !D) return ctx_fail(ctx, VMS_ERR_INVALID_ARG, "null argument");
  const Mesh& m = ctx_mesh(ctx);
  State& s = ctx_state(ctx);
  if (!s.valid) return ctx_fail(ctx, VMS_ERR_STATE, "no state uploaded");
  Scales sc;
  for (int c = 0; c < NO; ++c) sc.out[c] = scale_out ? scale_out[c] : 1.f;
  cudaSetDevice(ctx_device(ctx));
  const unsigned blocks = (unsigned)((m.n_nodes + 255) / 256);
  apply_increment_kernel<<<blocks, 256, 0, ctx_stream(ctx)>>>(s.u, m.n_nodes, sc, D);
  launch_impose(m, s.u, ctx_stream(ctx));
  ctx_work(ctx).assembled = false;
  const cudaError_t e = cudaGetLastError();
  return e == cudaSuccess ? VMS_OK : ctx_fail(ctx, VMS_ERR_CUDA, cudaGetErrorString(e));
}

int vms_shift_time(vms_ctx* ctx) {
  if (!ctx) return VMS_ERR_INVALID_ARG;
  const Mesh& m = ctx_mesh(ctx);
  State& s = ctx_state(ctx);
  if (!s.valid) return ctx_fail(ctx, VMS_ERR_STATE, "no state uploaded");
  cudaSetDevice(ctx_device(ctx));
  const cudaError_t e = cudaMemcpyAsync(s.u_prev, s.u, sizeof(double4_32a) * m.n_nodes,
                                        cudaMemcpyDeviceToDevice, ctx_stream(ctx));
  ctx_work(ctx).assembled = false;
  return e == cudaSuccess ? VMS_OK : ctx_fail(ctx, VMS_ERR_CUDA, cudaGetErrorString(e));
}

}  // extern "C"
