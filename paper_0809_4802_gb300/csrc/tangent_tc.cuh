// Tensor-core form of the element tangent's basis contractions (Section 4.2, Eq. NewtonUpdate2):
// every coarse block and the coarse-fine couplings are sums over quadrature points of a per-element
// coefficient times a reference basis function at the point (N_a, or dN_a/dxi_al), so for one
// element they form two small GEMMs with a constant right operand:
//
//   OutN[r][a] = sum_q   AN[r][q]      N_a(q)          (K = 32: the points, zero-padded)
//   OutD[r][a] = sum_q,al AD[r][3q+al] dN_a/dxi_al(q)  (K = 96)
//
// with the rows of the left operand, written by one lane per quadrature point:
//   AN  0..71   (b,i,k)  N_b omega L_ik               -> K_vv[(a,i),(b,k)] (the L term)
//   AN 72..79   b        omega (v.g_b + tau N_b)       -> K_vv diagonal (advection, mass)
//   AN 80..103  (b,i)    -omega g_bi                   -> K_pv[a,(b,i)] and K_vp[(b,i),a]
//   AN 104..115 (c,k)    Ycf[c][k]                     -> K_cf[(a,c),k] (N part)
//   AN 116..127 (c,k)    Yfc[c][k]                     -> K_fc[k,(a,c)] (N part)
//   AD 0..7     b        nut omega (J^-1 g_b)_al       -> K_vv diagonal (diffusion)
//   AD 8        .        nut omega (J^-1 d)_al         -> K_cf (the nut g_a.d part)
//   AD 9        .        (J^-1 (omega b v + nut omega d))_al -> K_fc (the g_b part)
// (Ycf, Yfc as in the CUDA-core form, tangent_math.cuh). The GEMMs run on mma.sync with either BF16
// operands (one product) or TF32 operands split into a high and a low part (three products, the
// corrections in their own accumulator), FP32 accumulation in both. K_ff and everything after the
// contractions (condensation, scatter) are unchanged.
#pragma once

#include <cuda_bf16.h>

#include "mma_bf16.cuh"
#include "tangent_math.cuh"

namespace vms {

constexpr int TC_BF16 = 1;   // engine: BF16 operands, one product
constexpr int TC_TF32X3 = 2; // engine: TF32 high/low operands, three products

constexpr int TC_ROWS_N = 128, TC_ROWS_D = 16;
constexpr int TC_KN = 32, TC_KD = 96;
// row strides (floats) of the left operands: conflict-free fragment loads (TF32: 4-byte loads at
// row g, column t: stride = 4 mod 32; BF16: 8-byte loads at row g, column 2t: stride = 8 mod 32)
template <int ENG> constexpr int tc_sn() { return ENG == TC_BF16 ? TC_KN + 8 : TC_KN + 4; }
template <int ENG> constexpr int tc_sd() { return ENG == TC_BF16 ? TC_KD + 8 : TC_KD + 4; }
// k-steps of one MMA: 16 (BF16) or 8 (TF32)
template <int ENG> constexpr int tc_kstep() { return ENG == TC_BF16 ? 16 : 8; }
// 32-bit words of one lane's B fragment: BF16 2, TF32 high + low 4
template <int ENG> constexpr int tc_bwords() { return ENG == TC_BF16 ? 2 : 4; }
template <int ENG> constexpr int tc_bsteps() { return TC_KN / tc_kstep<ENG>() + TC_KD / tc_kstep<ENG>(); }

// Per-warp operand and result storage of the tensor-core contractions.
// The results (Out, 144 x 8) overwrite the left operand AN: tile mt's results go to floats
// [128 mt, 128 mt + 128), which lie in AN tiles < mt (already consumed) or, for mt = 0, in tile 0
// itself after its loads; the D results (rows 128..143) are stored last, into AN tiles 1 and 2.
template <int ENG>
struct TcArea {
  float AN[TC_ROWS_N][tc_sn<ENG>()];
  float AD[TC_ROWS_D][tc_sd<ENG>()];
  __device__ float (*out())[8] { return reinterpret_cast<float (*)[8]>(&AN[0][0]); }
  __device__ const float (*out() const)[8] { return reinterpret_cast<const float (*)[8]>(&AN[0][0]); }
};
static_assert(TC_ROWS_N * (TC_KN + 4) >= 8 * (TC_ROWS_N + TC_ROWS_D), "results fit in AN");

#if defined(__CUDACC__)
__device__ __forceinline__ uint32_t tf32_rna(float x) {
  uint32_t r;
  asm("cvt.rna.tf32.f32 %0, %1;" : "=r"(r) : "f"(x));
  return r;
}
// x = hi + lo with hi, lo in TF32 (|x - hi - lo| <= 2^-22 |x|): the constant operands
__device__ __forceinline__ void tf32_split(float x, uint32_t& hi, uint32_t& lo) {
  hi = tf32_rna(x);
  lo = tf32_rna(x - __uint_as_float(hi));
}
// The per-element operands, with two instructions per value: hi = x with the 13 low mantissa bits
// cleared (a TF32 value), lo = x - hi (exact in FP32, |lo| < 2^-10 |x|), whose own low bits the
// TF32 multiply ignores: |x - hi - tf32(lo)| < 2^-20 |x|.
__device__ __forceinline__ void tf32_split_fast(float x, uint32_t& hi, uint32_t& lo) {
  hi = __float_as_uint(x) & 0xffffe000u;
  lo = __float_as_uint(x - __uint_as_float(hi));
}
__device__ __forceinline__ void mma_tf32(float d[4], const uint32_t a[4], uint32_t b0, uint32_t b1) {
  asm volatile(
      "mma.sync.aligned.m16n8k8.row.col.f32.tf32.tf32.f32 {%0,%1,%2,%3}, {%4,%5,%6,%7}, {%8,%9}, "
      "{%0,%1,%2,%3};"
      : "+f"(d[0]), "+f"(d[1]), "+f"(d[2]), "+f"(d[3])
      : "r"(a[0]), "r"(a[1]), "r"(a[2]), "r"(a[3]), "r"(b0), "r"(b1));
}

// The constant right operands in fragment order, from the FP32 reference table (N [nq][8],
// dN [nq][24]): for k-step s and lane (g = lane/4, t = lane%4) the lane's B fragment words, GEMM N
// first (rows = points), then GEMM D (rows = 3 point + al). Points >= nq are zero.
template <int ENG>
__device__ void tc_build_b(const float* __restrict__ N, const float* __restrict__ dN, int nq,
                           uint32_t* __restrict__ bf) {
  constexpr int KS = tc_kstep<ENG>(), SN = TC_KN / KS, ST = tc_bsteps<ENG>();
  auto B = [&](int s, int k, int n) -> float {
    if (s < SN) {
      const int q = s * KS + k;
      return q < nq ? N[8 * q + n] : 0.f;
    }
    const int kd = (s - SN) * KS + k, q = kd / 3, al = kd % 3;
    return q < nq ? dN[24 * q + 3 * n + al] : 0.f;
  };
  for (int i = threadIdx.x; i < ST * 32; i += blockDim.x) {
    const int s = i / 32, l = i % 32, g = l >> 2, t = l & 3;
    uint32_t* w = bf + (size_t)i * tc_bwords<ENG>();
    if constexpr (ENG == TC_BF16) {
      w[0] = bf16x2(B(s, 2 * t, g), B(s, 2 * t + 1, g));
      w[1] = bf16x2(B(s, 2 * t + 8, g), B(s, 2 * t + 9, g));
    } else {
      tf32_split(B(s, t, g), w[0], w[2]);
      tf32_split(B(s, t + 4, g), w[1], w[3]);
    }
  }
}

// Lane `lane` = quadrature point q (< nq <= 32): geometry and fields at q, its column of the left
// operands, and its K_ff contribution. Lanes q >= nq write zero columns (the K padding).
template <int ENG>
__device__ __forceinline__ void tc_phase1(int lane, int nq, WarpArea<float>& W,
                                          TcArea<ENG>& C, const RefTab<float>& tab, float nut,
                                          float tau, LaneAcc<float>& A) {
  const int q = lane;
  if (q >= nq) {
#pragma unroll 8
    for (int r = 0; r < TC_ROWS_N; ++r) C.AN[r][q] = 0.f;
#pragma unroll
    for (int r = 0; r < 10; ++r)
#pragma unroll
      for (int al = 0; al < 3; ++al) C.AD[r][3 * q + al] = 0.f;
    return;
  }
  const float* dN = tab.dN + 24 * q;
  const float* N = tab.N + 8 * q;
  const float bq = tab.b[q];
  const float db[3] = {tab.db[3 * q], tab.db[3 * q + 1], tab.db[3 * q + 2]};
  float J[3][3];
#pragma unroll
  for (int i = 0; i < 3; ++i)
#pragma unroll
    for (int al = 0; al < 3; ++al) {
      float s = 0.f;
#pragma unroll
      for (int a = 0; a < 8; ++a) s += W.X[a][i] * dN[3 * a + al];
      J[i][al] = s;
    }
  float cof[3][3];
  float det = cofactor3(J, cof);
  if (!(det > 0.f)) { W.flag = 1u; det = 1.f; }
  const float rdet = 1.f / det;
  float Ji[3][3];  // (J^-1)[al][j] = cof[j][al] / det
#pragma unroll
  for (int al = 0; al < 3; ++al)
#pragma unroll
    for (int j = 0; j < 3; ++j) Ji[al][j] = cof[j][al] * rdet;
  const float om = tab.w[q] * det;
  float g[8][3];
#pragma unroll
  for (int a = 0; a < 8; ++a)
#pragma unroll
    for (int j = 0; j < 3; ++j)
      g[a][j] = dN[3 * a] * Ji[0][j] + dN[3 * a + 1] * Ji[1][j] + dN[3 * a + 2] * Ji[2][j];
  float d[3];
#pragma unroll
  for (int j = 0; j < 3; ++j) d[j] = db[0] * Ji[0][j] + db[1] * Ji[1][j] + db[2] * Ji[2][j];
  float v[3], L[3][3];
#pragma unroll
  for (int i = 0; i < 3; ++i) {
    float s = 0.f;
#pragma unroll
    for (int a = 0; a < 8; ++a) s += N[a] * W.V[a][i];
    v[i] = s + bq * W.beta[i];
#pragma unroll
    for (int j = 0; j < 3; ++j) {
      float t = W.beta[i] * d[j];
#pragma unroll
      for (int a = 0; a < 8; ++a) t += W.V[a][i] * g[a][j];
      L[i][j] = t;
    }
  }
  const float cd = v[0] * d[0] + v[1] * d[1] + v[2] * d[2];
  const float dd = d[0] * d[0] + d[1] * d[1] + d[2] * d[2];
  const float omb = om * bq, nom = nut * om;
  // AN rows 0..103
#pragma unroll
  for (int b = 0; b < 8; ++b) {
    const float nb = om * N[b];
#pragma unroll
    for (int i = 0; i < 3; ++i)
#pragma unroll
      for (int k = 0; k < 3; ++k) C.AN[9 * b + 3 * i + k][q] = nb * L[i][k];
    const float cb = v[0] * g[b][0] + v[1] * g[b][1] + v[2] * g[b][2];
    C.AN[72 + b][q] = om * (cb + tau * N[b]);
#pragma unroll
    for (int i = 0; i < 3; ++i) C.AN[80 + 3 * b + i][q] = -om * g[b][i];
  }
  // AN rows 104..127: Ycf, Yfc (pressure rows: -omega d)
#pragma unroll
  for (int c = 0; c < 3; ++c)
#pragma unroll
    for (int k = 0; k < 3; ++k) {
      C.AN[104 + 3 * c + k][q] = omb * L[c][k] + (c == k ? om * cd : 0.f);
      C.AN[116 + 3 * c + k][q] = omb * (L[k][c] + (c == k ? tau : 0.f));
    }
#pragma unroll
  for (int k = 0; k < 3; ++k) {
    C.AN[113 + k][q] = -om * d[k];
    C.AN[125 + k][q] = -om * d[k];
  }
  // AD rows 0..9
  const float Wv[3] = {omb * v[0] + nom * d[0], omb * v[1] + nom * d[1], omb * v[2] + nom * d[2]};
#pragma unroll
  for (int al = 0; al < 3; ++al) {
#pragma unroll
    for (int b = 0; b < 8; ++b)
      C.AD[b][3 * q + al] = nom * (Ji[al][0] * g[b][0] + Ji[al][1] * g[b][1] + Ji[al][2] * g[b][2]);
    C.AD[8][3 * q + al] = nom * (Ji[al][0] * d[0] + Ji[al][1] * d[1] + Ji[al][2] * d[2]);
    C.AD[9][3 * q + al] = Ji[al][0] * Wv[0] + Ji[al][1] * Wv[1] + Ji[al][2] * Wv[2];
  }
#pragma unroll
  for (int i = 0; i < 3; ++i)
#pragma unroll
    for (int k = 0; k < 3; ++k)
      A.kff[3 * i + k] += om * (bq * (bq * L[i][k] + (i == k ? cd : 0.f)) + (i == k ? nut * dd : 0.f));
}

// One 16-row tile of a left operand (stride LD floats, rows r0..r0+15) times the constant right
// operand over `steps` k-steps starting at fragment step s0, into Out rows r0..r0+15.
template <int ENG, int LD>
__device__ __forceinline__ void tc_tile(int lane, const float* __restrict__ Arow, int steps,
                                        const uint32_t* __restrict__ bf, int s0,
                                        float (*Out)[8]) {
  const int g = lane >> 2, t = lane & 3;
  float acc[4] = {0.f, 0.f, 0.f, 0.f};
  float cor[4] = {0.f, 0.f, 0.f, 0.f};
  for (int s = 0; s < steps; ++s) {
    const uint32_t* w = bf + ((size_t)(s0 + s) * 32 + lane) * tc_bwords<ENG>();
    if constexpr (ENG == TC_BF16) {
      const float* p = Arow + s * 16 + 2 * t;
      const float2 x0 = *reinterpret_cast<const float2*>(p + g * LD);
      const float2 x1 = *reinterpret_cast<const float2*>(p + (g + 8) * LD);
      const float2 x2 = *reinterpret_cast<const float2*>(p + g * LD + 8);
      const float2 x3 = *reinterpret_cast<const float2*>(p + (g + 8) * LD + 8);
      const uint32_t a[4] = {bf16x2(x0.x, x0.y), bf16x2(x1.x, x1.y), bf16x2(x2.x, x2.y),
                             bf16x2(x3.x, x3.y)};
      const uint2 b = *reinterpret_cast<const uint2*>(w);
      mma_bf16(acc, a, b.x, b.y);
    } else {
      const float* p = Arow + s * 8 + t;
      uint32_t ah[4], al[4];
      tf32_split_fast(p[g * LD], ah[0], al[0]);
      tf32_split_fast(p[(g + 8) * LD], ah[1], al[1]);
      tf32_split_fast(p[g * LD + 4], ah[2], al[2]);
      tf32_split_fast(p[(g + 8) * LD + 4], ah[3], al[3]);
      const uint4 b = *reinterpret_cast<const uint4*>(w);  // high b0, b1, low b0, b1
      mma_tf32(acc, ah, b.x, b.y);
      mma_tf32(cor, ah, b.z, b.w);
      mma_tf32(cor, al, b.x, b.y);
    }
  }
  if constexpr (ENG != TC_BF16) {
#pragma unroll
    for (int j = 0; j < 4; ++j) acc[j] += cor[j];
  }
  __syncwarp();  // every lane's loads of this tile are done before the results overwrite it
  *reinterpret_cast<float2*>(&Out[g][2 * t]) = make_float2(acc[0], acc[1]);
  *reinterpret_cast<float2*>(&Out[g + 8][2 * t]) = make_float2(acc[2], acc[3]);
}

// Both contractions of one element (every lane of the warp), results in C.Out.
template <int ENG>
__device__ __forceinline__ void tc_contract(int lane, TcArea<ENG>& C, const uint32_t* __restrict__ bf) {
  constexpr int KS = tc_kstep<ENG>(), SN = TC_KN / KS, SD = TC_KD / KS;
  float (*Out)[8] = C.out();
#pragma unroll 1
  for (int mt = 0; mt < TC_ROWS_N / 16; ++mt)
    tc_tile<ENG, tc_sn<ENG>()>(lane, &C.AN[16 * mt][0], SN, bf, 0, &Out[16 * mt]);
  tc_tile<ENG, tc_sd<ENG>()>(lane, &C.AD[0][0], SD, bf, SN, &Out[TC_ROWS_N]);
}

// The lane's accumulators from the contraction results (the layout of LaneAcc: blocks (a0, b) and
// (a1, b) of K_cc with a0 = lane / 8, a1 = a0 + 4, b = lane % 8; row lane of K_cf; column lane of
// K_fc, lane = 4 node + dof).
template <int ENG>
__device__ __forceinline__ void tc_gather(int lane, const TcArea<ENG>& C, LaneAcc<float>& A) {
  const int a0 = lane >> 3, a1 = a0 + 4, b = lane & 7;
  const float (*O)[8] = C.out();
  const float* OD = &C.out()[TC_ROWS_N][0];
#pragma unroll
  for (int p = 0; p < 2; ++p) {
    const int a = p ? a1 : a0;
    const float diag = O[72 + b][a] + OD[8 * b + a];
    float k[16];
#pragma unroll
    for (int i = 0; i < 3; ++i) {
#pragma unroll
      for (int kk = 0; kk < 3; ++kk) k[4 * i + kk] = O[9 * b + 3 * i + kk][a] + (i == kk ? diag : 0.f);
      k[4 * i + 3] = O[80 + 3 * a + i][b];   // K_vp[(a,i),b]
      k[12 + i] = O[80 + 3 * b + i][a];      // K_pv[a,(b,i)]
    }
    k[15] = 0.f;
#pragma unroll
    for (int j = 0; j < 16; ++j) {
      if (p) A.K[j].y = k[j];
      else A.K[j].x = k[j];
    }
  }
  const int at = lane >> 2, ct = lane & 3;
#pragma unroll
  for (int kk = 0; kk < 3; ++kk) {
    A.kcf[kk] = O[104 + 3 * ct + kk][at] + (ct == kk ? OD[8 * 8 + at] : 0.f);
    A.kfc[kk] = O[116 + 3 * ct + kk][at] + (ct == kk ? OD[8 * 9 + at] : 0.f);
  }
}
#endif

}  // namespace vms
