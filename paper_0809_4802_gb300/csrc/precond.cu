// Block ILU(0) preconditioner of the condensed system (Section 6: Krylov solves with the solver
// library's default preconditioner, which on one process is an incomplete LU factorisation that
// keeps the sparsity pattern of the matrix).
//
// The matrix is viewed as 4x4 node blocks in natural node order. With no fill, the factorisation
// of block row i is, for each lower block k < i in increasing order,
//   L_ik = A_ik U_kk^-1,   A_ij -= L_ik U_kj   for every block j > k present in both rows,
// after which U_ii = A_ii and its inverse is kept for the backward sweep.
//
// GPU mapping of the factorisation: one warp owns one node row at a time and claims rows in order
// from a counter, so a row only ever waits for rows claimed earlier, by warps that are already
// running. A row publishes itself by writing its epoch into a flag with release semantics;
// dependants poll the flag with acquire loads (bounded: after Ilu::spin_limit polls the kernel
// records a timeout and returns), and read data published in the same launch through L2
// (ld.global.cg), never through L1. The triangular sweeps claim chunks of grid-line segments per
// CTA, one segment per warp (see ilu_sweep_kernel), so that most dependencies are resolved in
// registers and shared memory instead of L2.
#include <algorithm>
#include <vector>

#include "precond.h"
#include "solver.h"

namespace vms {

namespace {

constexpr int ILU_FWARPS = 4;    // warps per CTA of the factorisation
// warps per CTA of the sweeps (one segment each). Measured on the 33^3-node lattice (FP32 apply):
// 2 or 4 warps 0.244 ms, 8 warps 0.293 ms, 16 warps 0.269 ms, with one or several CTAs per SM
// alike; FP64 rows keep the FP64 pipe of their SM partition busy for ~1000 cycles, so FP64 sweeps
// spread over more SMs as well.
template <typename T> constexpr int sweep_warps() { return 4; }
constexpr unsigned FULL = 0xffffffffu;

__device__ __forceinline__ uint32_t ld_acquire(const uint32_t* p) {
  uint32_t v;
  asm volatile("ld.acquire.gpu.global.u32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
  return v;
}

__device__ __forceinline__ void st_release(uint32_t* p, uint32_t v) {
  asm volatile("st.release.gpu.global.u32 [%0], %1;" ::"l"(p), "r"(v) : "memory");
}

// Wait until *f == epoch. Gives up (returns false) when another warp has recorded an error or
// after `lim` polls (Ilu::spin_limit), recording a timeout.
__device__ __forceinline__ bool wait_ready(const uint32_t* f, uint32_t epoch, int* err, uint32_t lim) {
  if (ld_acquire(f) == epoch) return true;
  for (uint32_t it = 1; it <= lim; ++it) {
    __nanosleep(32);
    if (ld_acquire(f) == epoch) return true;
    if ((it & 1023u) == 0 && *(volatile int*)err != 0) return false;
  }
  atomicCAS(err, 0, ILU_ERR_TIMEOUT);
  return false;
}

// Claim the next row of this launch: 0 <= t < n_rows, or n_rows when none is left. A claim below
// the launch's base (the counter was disturbed by a launch that stopped early) records an error
// and also returns n_rows, so that no row index outside [0, n_rows) is ever formed.
__device__ __forceinline__ int64_t claim_row(unsigned long long* ticket, unsigned long long base,
                                             int64_t n_rows, int* err, int lane) {
  unsigned long long t = 0;
  if (lane == 0) t = atomicAdd(ticket, 1ull);
  t = __shfl_sync(FULL, t, 0);
  if (t < base) {
    if (lane == 0) atomicCAS(err, 0, ILU_ERR_TIMEOUT);
    return n_rows;
  }
  t -= base;
  return t < (unsigned long long)n_rows ? (int64_t)t : n_rows;
}

// ---------------------------------------------------------------------------------------------
// factorisation: one warp per node row; the row is eliminated in shared memory
// ---------------------------------------------------------------------------------------------
template <typename T>
__global__ void __launch_bounds__(ILU_FWARPS * 32)
    ilu_factor_kernel(const int32_t* __restrict__ rowptr, const int32_t* __restrict__ colidx,
                      const T* __restrict__ A, T* F, T* Dinv, const int32_t* __restrict__ dpos,
                      const int32_t* __restrict__ lptr, const int32_t* __restrict__ pptr,
                      const uint16_t* __restrict__ pairs, int64_t n_nodes, uint32_t* flags,
                      uint32_t epoch, unsigned long long* ticket, unsigned long long base, int* err,
                      uint32_t lim) {
  __shared__ T srow[ILU_FWARPS][ILU_MAX_DEG * 16];
  const int lane = threadIdx.x & 31;
  T* row = srow[threadIdx.x >> 5];
  for (;;) {
    const int64_t t = claim_row(ticket, base, n_nodes, err, lane);
    if (t >= n_nodes) return;
    const int64_t i = t;
    const int32_t r0 = rowptr[4 * i];
    const int deg = (rowptr[4 * i + 1] - r0) >> 2;
    // row i into shared memory, block-major: row[16 kk + 4 q + c] = A(4i+q, 4 adj_kk + c)
    for (int e = lane; e < deg * 16; e += 32)
      row[e] = A[rowptr[4 * i + ((e >> 2) & 3)] + 4 * (e >> 4) + (e & 3)];
    __syncwarp();
    const int dp = dpos[i];
    const int32_t l0 = lptr[i];
    const int q = (lane >> 2) & 3, c = lane & 3, half = lane >> 4;
    for (int kk = 0; kk < dp; ++kk) {
      const int64_t k = colidx[r0 + 4 * kk] >> 2;
      int ok = 1;
      if (lane == 0) ok = wait_ready(flags + k, epoch, err, lim);
      if (!__shfl_sync(FULL, ok, 0)) return;
      // L_ik = A_ik U_kk^-1 (lanes 0..15 hold entry (q, c))
      T l = T(0);
      if (lane < 16) {
        const T* d = Dinv + 16 * k + c;
        for (int m = 0; m < 4; ++m) l += row[16 * kk + 4 * q + m] * __ldcg(d + 4 * m);
      }
      __syncwarp();
      if (lane < 16) row[16 * kk + lane] = l;
      __syncwarp();
      // A_ij -= L_ik U_kj over the pairs of this lower block, two pairs per step (the products
      // are subtracted one by one, so that each is a fused multiply-add)
      int32_t rk[4];
      for (int m = 0; m < 4; ++m) rk[m] = rowptr[4 * k + m];
      const int32_t pe = pptr[l0 + kk + 1];
      for (int32_t p = pptr[l0 + kk] + half; p < pe; p += 2) {
        const uint32_t pr = pairs[p];
        const int jj = pr & 255, jk = pr >> 8;
        T s = row[16 * jj + 4 * q + c];
        for (int m = 0; m < 4; ++m) s -= row[16 * kk + 4 * q + m] * __ldcg(F + rk[m] + 4 * jk + c);
        row[16 * jj + 4 * q + c] = s;
      }
      __syncwarp();
    }
    // U_ii^-1 = adj(U_ii) / det on lanes 0..15 (lane 4r + c forms the cofactor of entry (r, c)):
    // a handful of FP64 instructions per lane instead of a serial elimination on one lane
    {
      const T* D = row + 16 * dp;
      const int r = (lane >> 2) & 3, c = lane & 3;
      double mnr[3][3];  // the minor: rows other than r, columns other than c
#pragma unroll
      for (int a2 = 0; a2 < 3; ++a2)
#pragma unroll
        for (int b2 = 0; b2 < 3; ++b2)
          mnr[a2][b2] = (double)D[4 * (a2 + (a2 >= r)) + b2 + (b2 >= c)];
      const double m3 = mnr[0][0] * (mnr[1][1] * mnr[2][2] - mnr[1][2] * mnr[2][1]) -
                        mnr[0][1] * (mnr[1][0] * mnr[2][2] - mnr[1][2] * mnr[2][0]) +
                        mnr[0][2] * (mnr[1][0] * mnr[2][1] - mnr[1][1] * mnr[2][0]);
      const double cf = ((r + c) & 1) ? -m3 : m3;
      const double dv = lane < 16 ? (double)D[lane] : 0.0;
      double dt = lane < 4 ? dv * cf : 0.0;  // det by the first row
      dt += __shfl_xor_sync(FULL, dt, 1);
      dt += __shfl_xor_sync(FULL, dt, 2);
      const double det = __shfl_sync(FULL, dt, 0);
      // singular unless |det| is a fair fraction of the product of the row norms (Hadamard's
      // bound; independent of the rows' scales), compared squared: det^2 > 1e-28 prod |row|^2
      double rn = dv * dv;
      rn += __shfl_xor_sync(FULL, rn, 1);
      rn += __shfl_xor_sync(FULL, rn, 2);
      const double hb2 = __shfl_sync(FULL, rn, 0) * __shfl_sync(FULL, rn, 4) *
                         __shfl_sync(FULL, rn, 8) * __shfl_sync(FULL, rn, 12);
      const bool good = isfinite(det) && hb2 > 0.0 && det * det > 1e-28 * hb2;
      if (!good && lane == 0) atomicCAS(err, 0, ILU_ERR_PIVOT);
      if (lane < 16) Dinv[16 * i + 4 * c + r] = good ? T(cf / det) : T(r == c ? 1.0 : 0.0);
    }
    for (int e = lane; e < deg * 16; e += 32)
      F[rowptr[4 * i + ((e >> 2) & 3)] + 4 * (e >> 4) + (e & 3)] = row[e];
    __threadfence();
    __syncwarp();
    if (lane == 0) st_release(flags + i, epoch);
  }
}

// ---------------------------------------------------------------------------------------------
// sweeps: y = L^-1 v (rows ascending), z = U^-1 y (rows descending)
// A warp solves the rows of one grid-line segment in order, one lane per neighbour block of the
// row (a node has at most 32 neighbours; FP64 rows with at most 16 blocks on the sweep's side take
// two lanes per block): every lane waits for its own neighbour at the same time.
// ---------------------------------------------------------------------------------------------

// FP32 sweeps publish every value in one 64-bit word together with the sweep's epoch (low half:
// the float's bits, high half: the epoch). Naturally aligned 64-bit accesses are single-copy
// atomic, so a reader that sees the current epoch in all four words of a node also holds their
// values: one L2 round trip detects readiness and delivers the data, with no flag and no fence.
__device__ __forceinline__ void st_packed(unsigned long long* p, float v, uint32_t ep) {
  const unsigned long long w = ((unsigned long long)ep << 32) | __float_as_uint(v);
  asm volatile("st.relaxed.gpu.global.u64 [%0], %1;" ::"l"(p), "l"(w) : "memory");
}

__device__ __forceinline__ void ld_relaxed2(const unsigned long long* p, unsigned long long& a,
                                            unsigned long long& b) {
  asm volatile("ld.relaxed.gpu.global.v2.u64 {%0, %1}, [%2];" : "=l"(a), "=l"(b) : "l"(p) : "memory");
}

// Wait until the four words of a node carry `ep`, then return their values.
__device__ __forceinline__ bool wait_packed(const unsigned long long* p, uint32_t ep, float out[4],
                                            int* err, uint32_t lim) {
  for (uint32_t it = 0; it <= lim; ++it) {
    unsigned long long a, b, c, d;
    ld_relaxed2(p, a, b);
    ld_relaxed2(p + 2, c, d);
    if ((uint32_t)(a >> 32) == ep && (uint32_t)(b >> 32) == ep && (uint32_t)(c >> 32) == ep &&
        (uint32_t)(d >> 32) == ep) {
      out[0] = __uint_as_float((uint32_t)a);
      out[1] = __uint_as_float((uint32_t)b);
      out[2] = __uint_as_float((uint32_t)c);
      out[3] = __uint_as_float((uint32_t)d);
      return true;
    }
    if (it >= 64) __nanosleep(32);
    if ((it & 1023u) == 1023u && *(volatile int*)err != 0) return false;
  }
  atomicCAS(err, 0, ILU_ERR_TIMEOUT);
  return false;
}

// FP64 sweeps write into buffers filled with an all-ones bit pattern before the sweep (a NaN that
// arithmetic never produces); a node is ready once none of its four words holds that pattern.
constexpr unsigned long long UNSET64 = ~0ull;

__device__ __forceinline__ bool wait_unset(const double* p, double out[4], int* err, uint32_t lim) {
  const unsigned long long* w = reinterpret_cast<const unsigned long long*>(p);
  for (uint32_t it = 0; it <= lim; ++it) {
    unsigned long long a, b, c, d;
    ld_relaxed2(w, a, b);
    ld_relaxed2(w + 2, c, d);
    if (a != UNSET64 && b != UNSET64 && c != UNSET64 && d != UNSET64) {
      out[0] = __longlong_as_double((long long)a);
      out[1] = __longlong_as_double((long long)b);
      out[2] = __longlong_as_double((long long)c);
      out[3] = __longlong_as_double((long long)d);
      return true;
    }
    if (it >= 64) __nanosleep(32);
    if ((it & 1023u) == 1023u && *(volatile int*)err != 0) return false;
  }
  atomicCAS(err, 0, ILU_ERR_TIMEOUT);
  return false;
}

__device__ __forceinline__ void st_relaxed_f64(double* p, double v) {
  asm volatile("st.relaxed.gpu.global.u64 [%0], %1;" ::"l"(p), "l"(__double_as_longlong(v)) : "memory");
}

// Sum of the four per-lane partials over the warp, reduce-scatter style (7 shuffles): on return
// lane L holds the full sum of component (L >> 3) & 3.
template <typename T>
__device__ __forceinline__ T warp_sum4_scatter(const T a[4], int lane) {
  const bool h16 = lane & 16, h8 = lane & 8;
  const T s0 = h16 ? a[0] : a[2], s1 = h16 ? a[1] : a[3];
  const T b0 = (h16 ? a[2] : a[0]) + __shfl_xor_sync(FULL, s0, 16);
  const T b1 = (h16 ? a[3] : a[1]) + __shfl_xor_sync(FULL, s1, 16);
  T c = (h8 ? b1 : b0) + __shfl_xor_sync(FULL, h8 ? b0 : b1, 8);
  c += __shfl_xor_sync(FULL, c, 4);
  c += __shfl_xor_sync(FULL, c, 2);
  c += __shfl_xor_sync(FULL, c, 1);
  return c;
}

// Shared-memory publication inside a chunk: the CTA fills the chunk's value slots with an all-ones
// bit pattern (a NaN that arithmetic never produces) when it takes the chunk, each writer lane then
// stores its value directly, and a reader polls until none of the node's four words holds the
// pattern. Every word is written once by one lane, so no flag and no fence is needed.
template <typename T> struct Bits;
template <> struct Bits<float> { using U = uint32_t; static constexpr U unset = 0xffffffffu; };
template <> struct Bits<double> { using U = unsigned long long; static constexpr U unset = ~0ull; };

template <typename T>
__device__ __forceinline__ bool wait_shared(const T* p, T out[4], int* err, uint32_t lim) {
  using U = typename Bits<T>::U;
  const volatile U* w = reinterpret_cast<const volatile U*>(p);
  for (uint32_t it = 0; it <= lim; ++it) {
    const U a = w[0], b = w[1], c = w[2], d = w[3];
    if (a != Bits<T>::unset && b != Bits<T>::unset && c != Bits<T>::unset && d != Bits<T>::unset) {
      const U u[4] = {a, b, c, d};
      for (int m = 0; m < 4; ++m) {
        if constexpr (sizeof(T) == 4) out[m] = __uint_as_float(u[m]);
        else out[m] = __longlong_as_double((long long)u[m]);
      }
      return true;
    }
    if (it >= 32) __nanosleep(8);
    if ((it & 1023u) == 1023u && *(volatile int*)err != 0) return false;
  }
  atomicCAS(err, 0, ILU_ERR_TIMEOUT);
  return false;
}

// Asynchronous global -> shared copies (per thread; completion tracked per thread by groups, so a
// thread only ever reads what it copied itself and no flag or barrier is involved).
__device__ __forceinline__ void cp_async16(void* dst, const void* src) {
  const unsigned d = (unsigned)__cvta_generic_to_shared(dst);
  asm volatile("cp.async.cg.shared.global [%0], [%1], 16;" ::"r"(d), "l"(src) : "memory");
}
__device__ __forceinline__ void cp_async4(void* dst, const void* src) {
  const unsigned d = (unsigned)__cvta_generic_to_shared(dst);
  asm volatile("cp.async.ca.shared.global [%0], [%1], 4;" ::"r"(d), "l"(src) : "memory");
}
__device__ __forceinline__ void cp_commit() { asm volatile("cp.async.commit_group;" ::: "memory"); }
template <int N>
__device__ __forceinline__ void cp_wait() { asm volatile("cp.async.wait_group %0;" ::"n"(N) : "memory"); }

// Rows of a segment in flight ahead of the row being solved, and the per-warp ring they land in:
// for each slot, every lane's 4x4 factor block, every lane's column index and the four rows of
// U_ii^-1 (backward sweep).
constexpr int ILU_PF = 4;
template <typename T>
struct SweepSlot {
  T f[32][16];
  int32_t col[32];
  T dinv[4][4];
};
template <typename T>
constexpr size_t sweep_ring_bytes(int warps) {
  return (size_t)warps * ILU_PF * sizeof(SweepSlot<T>);
}

// FP64 rows with at most 16 blocks on the sweep's side take two lanes per block (two block rows
// each): 8 DFMA instructions per row instead of 16 (the FP64 unit of an SM partition spends a
// full warp slot on every FP64 instruction, however many lanes are active).
template <typename T>
__device__ __forceinline__ bool split_rows_t(int side) { return sizeof(T) == 8 && side <= 16; }

// One row of the two-lanes-per-block mapping (lane 2 bl + h: rows 2h, 2h + 1 of block bl). The
// sums end on lanes 0, 16, 1, 17 for components 0..3. Returns false if a wait gave up.
template <typename T, bool LOWER>
__device__ __forceinline__ bool split_row(const SweepSlot<T>& sl, int r, int64_t i, int dp, int deg,
                                          int lane, const T (&o_rhs)[2][4], T* sx, int64_t a,
                                          int64_t b, void* pub, T* out, int64_t n0, uint32_t ep,
                                          int* err, uint32_t lim) {
  const int bl = lane >> 1, h = lane & 1;
  const int kk = LOWER ? bl : dp + 1 + bl;
  const bool mine = LOWER ? kk < dp : kk < deg;
  const int qw = 2 * h + ((lane >> 4) & 1);      // the component this lane's reduction ends with
  const bool wr = (lane & 14) == 0;              // lanes 0, 1, 16, 17
  T rhs = T(0);
  {
    const int src = r & 31;
    const bool hi = r >= 32;
    for (int m = 0; m < 4; ++m) {
      const T t = __shfl_sync(FULL, hi ? o_rhs[1][m] : o_rhs[0][m], src);
      if (m == qw) rhs = t;
    }
  }
  T acc0 = T(0), acc1 = T(0);
  bool ok = true;
  if (mine) {
    const int64_t k = sl.col[lane] >> 2;
    T xk[4];
    if (k >= a && k < b) {
      const int64_t sk = LOWER ? k - a : b - 1 - k;
      ok = wait_shared<T>(sx + 4 * sk, xk, err, lim);
    } else if constexpr (sizeof(T) == 4) {
      ok = wait_packed(reinterpret_cast<const unsigned long long*>(pub) + 4 * k, ep, xk, err, lim);
    } else {
      ok = wait_unset(reinterpret_cast<const double*>(pub) + 4 * k, xk, err, lim);
    }
    if (ok)
      for (int m = 0; m < 4; ++m) {
        acc0 += sl.f[lane][m] * xk[m];
        acc1 += sl.f[lane][4 + m] * xk[m];
      }
  }
  if (!__all_sync(FULL, ok)) return false;
  // sum over the 16 blocks (lane bits 1..4), rows 2h (lane bit 4 clear) or 2h + 1 (set)
  const bool b4 = lane & 16;
  T sm = (b4 ? acc1 : acc0) + __shfl_xor_sync(FULL, b4 ? acc0 : acc1, 16);
  sm += __shfl_xor_sync(FULL, sm, 8);
  sm += __shfl_xor_sync(FULL, sm, 4);
  sm += __shfl_xor_sync(FULL, sm, 2);
  const T w = wr ? rhs - sm : T(0);
  T res = w;
  if constexpr (!LOWER) {
    // components 0..3 sit on lanes 0, 16, 1, 17
    const T w0 = __shfl_sync(FULL, w, 0), w1 = __shfl_sync(FULL, w, 16);
    const T w2 = __shfl_sync(FULL, w, 1), w3 = __shfl_sync(FULL, w, 17);
    res = wr ? sl.dinv[qw][0] * w0 + sl.dinv[qw][1] * w1 + sl.dinv[qw][2] * w2 + sl.dinv[qw][3] * w3
             : T(0);
  }
  const int64_t si = LOWER ? i - a : b - 1 - i;
  if (wr) {
    *reinterpret_cast<volatile T*>(sx + 4 * si + qw) = res;
    if constexpr (sizeof(T) == 4)
      st_packed(reinterpret_cast<unsigned long long*>(pub) + 4 * i + qw, res, ep);
    else
      st_relaxed_f64(reinterpret_cast<double*>(pub) + 4 * i + qw, res);
    if (out) out[4 * (i - n0) + qw] = res;
  }
  return true;
}

// T: element type of the factor (float: packed publication, double: sentinel publication).
// Rows [n0, n0 + n_rows); `v` (forward sweep) and `out` are compact (index i - n0), the
// publication buffer `pub`, the FP64 backward-sweep input `v` and the FP32 one `vp` are indexed by
// node over the whole mesh.
//
// The rows are cut into segments (seg[s] .. seg[s+1]): maximal runs of consecutive nodes in which
// every node is coupled to the one before it (a grid line in a lattice numbering), at most
// ILU_SEG_MAX long. A CTA claims the next chunk of W segments in sweep order from the
// global counter and each of its warps takes one segment and does its rows in order, loading the
// next row while the current one waits. A row's dependency in the same chunk is read from shared
// memory once its value slots no longer hold the all-ones pattern (no L2 round trip; in the warp's
// own segment it is already there); a dependency in an earlier chunk is read from the L2
// publication. Chunks are claimed in order by running CTAs, so every wait is for work that is
// already in progress.
template <typename T, bool LOWER, int W = sweep_warps<T>()>
__global__ void __launch_bounds__(W * 32)
    ilu_sweep_kernel(const int32_t* __restrict__ rowptr, const int32_t* __restrict__ colidx,
                     const T* __restrict__ F, const T* __restrict__ Dinv,
                     const int32_t* __restrict__ dpos, const int32_t* __restrict__ seg, int64_t s0,
                     int64_t n_segs, const T* __restrict__ v,
                     const unsigned long long* __restrict__ vp, void* pub, T* __restrict__ out,
                     int64_t n0, int64_t n_rows, uint32_t ep, unsigned long long* ticket,
                     unsigned long long base, int* err, uint32_t lim) {
  constexpr int SLOTS = W * ILU_SEG_MAX;
  __shared__ __align__(16) T sx[SLOTS * 4];
  __shared__ int64_t s_chunk;
  extern __shared__ __align__(16) unsigned char sring[];
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  SweepSlot<T>* ring = reinterpret_cast<SweepSlot<T>*>(sring) + warp * ILU_PF;
  const int q = (lane >> 3) & 3;          // the component this lane's reduction ends with
  const bool writer = (lane & 7) == 0;    // lanes 0, 8, 16, 24 finish components 0..3
  const int64_t n1 = n0 + n_rows;
  const int64_t n_chunks = (n_segs + W - 1) / W;
  for (;;) {
    if (threadIdx.x == 0) {
      int64_t c = n_chunks;
      if (*(volatile int*)err == 0) {
        const unsigned long long t = atomicAdd(ticket, 1ull);
        if (t < base) atomicCAS(err, 0, ILU_ERR_TIMEOUT);  // the counter was disturbed
        else if (t - base < (unsigned long long)n_chunks) c = (int64_t)(t - base);
      }
      s_chunk = c;
    }
    for (int l = threadIdx.x; l < 4 * SLOTS; l += blockDim.x)
      reinterpret_cast<typename Bits<T>::U*>(sx)[l] = Bits<T>::unset;
    __syncthreads();
    const int64_t c = s_chunk;
    if (c >= n_chunks) return;
    // segments jlo .. jhi - 1 in sweep order; their nodes form the range [a, b)
    const int64_t jlo = c * W;
    const int64_t jhi = jlo + W < n_segs ? jlo + W : n_segs;
    int64_t a = LOWER ? seg[s0 + jlo] : seg[s0 + n_segs - jhi];
    int64_t b = LOWER ? seg[s0 + jhi] : seg[s0 + n_segs - jlo];
    a = a > n0 ? a : n0;
    b = b < n1 ? b : n1;
    const int64_t j = jlo + warp;
    if (j < jhi) {
      const int64_t s = LOWER ? s0 + j : s0 + n_segs - 1 - j;
      int64_t r_lo = seg[s], r_hi = seg[s + 1];
      r_lo = r_lo > n0 ? r_lo : n0;
      r_hi = r_hi < n1 ? r_hi : n1;
      const int len = (int)(r_hi - r_lo);
      // rows r of the segment in sweep order: node LOWER ? r_lo + r : r_hi - 1 - r. All rows'
      // offsets and right-hand sides are loaded at once (row r on lane r % 32, register set r / 32);
      // factor blocks, column indices and U_ii^-1 rows stream through the ring ILU_PF - 1 rows
      // ahead of the row being solved.
      int32_t o_rp[2][4], o_dp[2];
      T o_rhs[2][4];
      for (int h = 0; h < 2; ++h) {
        const int l = lane + 32 * h;
        o_dp[h] = 0;
        for (int m = 0; m < 4; ++m) { o_rp[h][m] = 0; o_rhs[h][m] = T(0); }
        if (l < len) {
          const int64_t il = LOWER ? r_lo + l : r_hi - 1 - l;
          for (int m = 0; m < 4; ++m) o_rp[h][m] = rowptr[4 * il + m];
          o_dp[h] = dpos[il];
          for (int m = 0; m < 4; ++m) {
            if constexpr (LOWER) {
              o_rhs[h][m] = v[4 * (il - n0) + m];
            } else if constexpr (sizeof(T) == 4) {
              o_rhs[h][m] = __uint_as_float((uint32_t)vp[4 * il + m]);
            } else {
              o_rhs[h][m] = v[4 * il + m];
            }
          }
        }
      }
      // offsets of row r (uniform r): broadcast from the lane that loaded them
      auto row_offsets = [&](int r, int32_t rp[4], int& dp) {
        const int src = r & 31;
        const bool hi = r >= 32;
        for (int m = 0; m < 4; ++m) rp[m] = __shfl_sync(FULL, hi ? o_rp[1][m] : o_rp[0][m], src);
        dp = __shfl_sync(FULL, hi ? o_dp[1] : o_dp[0], src);
      };
      auto split_rows = [&](int dp, int deg) { return split_rows_t<T>(LOWER ? dp : deg - dp - 1); };
      auto issue = [&](int r) {  // start the copies of row r (every lane commits one group)
        if (r < len) {
          int32_t rp[4], dp;
          row_offsets(r, rp, dp);
          const int deg = (rp[1] - rp[0]) >> 2;
          SweepSlot<T>& sl = ring[r % ILU_PF];
          constexpr int CH = (int)(4 * sizeof(T)) / 16;  // 16-byte pieces of a 4-value block row
          constexpr int EPC = 16 / (int)sizeof(T);        // values per piece
          if (split_rows(dp, deg)) {
            // two lanes per block: lane 2 bl + h copies rows 2h, 2h + 1 of block bl
            const int bl = lane >> 1, h = lane & 1;
            const int kk = LOWER ? bl : dp + 1 + bl;
            if (LOWER ? kk < dp : kk < deg) {
              const int32_t ra = h ? rp[2] : rp[0], rb = h ? rp[3] : rp[1];
              for (int c = 0; c < CH; ++c) {
                cp_async16(&sl.f[lane][c * EPC], F + ra + 4 * kk + c * EPC);
                cp_async16(&sl.f[lane][4 + c * EPC], F + rb + 4 * kk + c * EPC);
              }
              cp_async4(&sl.col[lane], colidx + rp[0] + 4 * kk);
            }
          } else {
            const int kk = LOWER ? lane : dp + 1 + lane;
            if (LOWER ? kk < dp : kk < deg) {
              for (int m = 0; m < 4; ++m)
                for (int c = 0; c < CH; ++c)
                  cp_async16(&sl.f[lane][4 * m + c * EPC], F + rp[m] + 4 * kk + c * EPC);
              cp_async4(&sl.col[lane], colidx + rp[0] + 4 * kk);
            }
          }
          if (!LOWER && writer) {
            const int64_t ir = r_hi - 1 - r;
            for (int c = 0; c < CH; ++c)
              cp_async16(&sl.dinv[q][c * EPC], Dinv + 16 * ir + 4 * q + c * EPC);
          }
        }
        cp_commit();
      };
      for (int r = 0; r < ILU_PF - 1; ++r) issue(r);
      for (int r = 0; r < len; ++r) {
        const int64_t i = LOWER ? r_lo + r : r_hi - 1 - r;
        issue(r + ILU_PF - 1);
        cp_wait<ILU_PF - 1>();  // this thread's copies of row r have landed
        __syncwarp();           // ... and every lane's (U_ii^-1 rows are read across lanes)
        const SweepSlot<T>& sl = ring[r % ILU_PF];
        int32_t rp[4], dp;
        row_offsets(r, rp, dp);
        const int deg = (rp[1] - rp[0]) >> 2;
        if (split_rows(dp, deg)) {
          if (!split_row<T, LOWER>(sl, r, i, dp, deg, lane, o_rhs, sx, a, b, pub, out, n0, ep, err, lim))
            break;  // an error was recorded; the CTA stops after this chunk
          continue;
        }
        const int kk = LOWER ? lane : dp + 1 + lane;
        const bool mine = LOWER ? kk < dp : kk < deg;
        T rhs = T(0);
        {
          const int src = r & 31;
          const bool hi = r >= 32;
          for (int m = 0; m < 4; ++m) {
            const T t = __shfl_sync(FULL, hi ? o_rhs[1][m] : o_rhs[0][m], src);
            if (m == q) rhs = t;
          }
        }
        T acc[4] = {T(0), T(0), T(0), T(0)};
        bool ok = true;
        if (mine) {
          const int64_t k = sl.col[lane] >> 2;
          T xk[4];
          if (k >= a && k < b) {  // a row of this chunk: shared memory
            const int64_t sk = LOWER ? k - a : b - 1 - k;
            ok = wait_shared<T>(sx + 4 * sk, xk, err, lim);
          } else if constexpr (sizeof(T) == 4) {
            ok = wait_packed(reinterpret_cast<const unsigned long long*>(pub) + 4 * k, ep, xk, err, lim);
          } else {
            ok = wait_unset(reinterpret_cast<const double*>(pub) + 4 * k, xk, err, lim);
          }
          if (ok)
            for (int rr = 0; rr < 4; ++rr)
              for (int m = 0; m < 4; ++m) acc[rr] += sl.f[lane][4 * rr + m] * xk[m];
        }
        if (!__all_sync(FULL, ok)) break;  // an error was recorded; the CTA stops after this chunk
        const T sum = warp_sum4_scatter(acc, lane);
        const T w = writer ? rhs - sum : T(0);
        T res = w;
        if constexpr (!LOWER) {
          T wq[4];
          for (int m = 0; m < 4; ++m) wq[m] = __shfl_sync(FULL, w, 8 * m);
          res = writer ? sl.dinv[q][0] * wq[0] + sl.dinv[q][1] * wq[1] + sl.dinv[q][2] * wq[2] +
                             sl.dinv[q][3] * wq[3]
                       : T(0);
        }
        const int64_t si = LOWER ? i - a : b - 1 - i;
        if (writer) {
          *reinterpret_cast<volatile T*>(sx + 4 * si + q) = res;
          if constexpr (sizeof(T) == 4)
            st_packed(reinterpret_cast<unsigned long long*>(pub) + 4 * i + q, res, ep);
          else
            st_relaxed_f64(reinterpret_cast<double*>(pub) + 4 * i + q, res);
          if (out) out[4 * (i - n0) + q] = res;
        }
      }
      cp_wait<0>();  // no copy of this segment may land in the ring after the warp has moved on
    }
    __syncthreads();
  }
}

unsigned resident_ctas(int64_t rows, int warps_per_cta, unsigned cap) {
  const int64_t b = (rows + warps_per_cta - 1) / warps_per_cta;
  return (unsigned)std::max<int64_t>(1, std::min<int64_t>(b, cap));
}

uint32_t next_epoch(Ilu& p, cudaStream_t st) {
  if (++p.epoch == 0) {  // wrapped: clear every flag so no stale epoch can match
    cudaMemsetAsync(p.flags, 0, sizeof(uint32_t) * p.n_nodes, st);
    cudaMemsetAsync(p.yp, 0, sizeof(unsigned long long) * 4 * p.n_nodes, st);
    cudaMemsetAsync(p.xp, 0, sizeof(unsigned long long) * 4 * p.n_nodes, st);
    p.epoch = 1;
  }
  return p.epoch;
}

// Host-side pattern of the factorisation from the CSR pattern: diagonal positions, lower blocks
// and, for every lower block (i, k), the pairs (j in row i, j in row k) with j > k.
int build_pattern(vms_ctx* ctx, Ilu& p, const Mesh& m) {
  const int64_t N = m.n_nodes;
  std::vector<int32_t> rowptr(4 * N + 1), colidx(m.nnz);
  cudaError_t e = cudaMemcpy(rowptr.data(), m.rowptr, sizeof(int32_t) * rowptr.size(), cudaMemcpyDeviceToHost);
  if (e == cudaSuccess) e = cudaMemcpy(colidx.data(), m.colidx, sizeof(int32_t) * colidx.size(), cudaMemcpyDeviceToHost);
  if (e != cudaSuccess) return ctx_fail(ctx, VMS_ERR_CUDA, cudaGetErrorString(e));
  std::vector<int32_t> start(N + 1), adj, dpos(N), lptr(N + 1, 0), pptr(1, 0);
  std::vector<uint16_t> pairs;
  adj.reserve((size_t)m.nnz / 16);
  for (int64_t i = 0; i < N; ++i) {
    const int32_t r0 = rowptr[4 * i];
    const int deg = (rowptr[4 * i + 1] - r0) / 4;
    if (deg > ILU_MAX_DEG)
      return ctx_fail(ctx, VMS_ERR_UNSUPPORTED, "ILU(0): a node has more than 32 neighbours");
    start[i] = (int32_t)adj.size();
    int d = -1;
    for (int kk = 0; kk < deg; ++kk) {
      const int32_t j = colidx[r0 + 4 * kk] / 4;
      if (j == i) d = kk;
      adj.push_back(j);
    }
    if (d < 0) return ctx_fail(ctx, VMS_ERR_INVALID_ARG, "ILU(0): a node belongs to no element");
    dpos[i] = d;
  }
  start[N] = (int32_t)adj.size();
  for (int64_t i = 0; i < N; ++i) {
    const int32_t* ai = adj.data() + start[i];
    const int degi = start[i + 1] - start[i];
    for (int kk = 0; kk < dpos[i]; ++kk) {
      const int32_t k = ai[kk];
      const int32_t* ak = adj.data() + start[k];
      const int degk = start[k + 1] - start[k];
      int jj = kk + 1;
      for (int jk = dpos[k] + 1; jk < degk; ++jk) {
        const int32_t j = ak[jk];
        while (jj < degi && ai[jj] < j) ++jj;
        if (jj < degi && ai[jj] == j) pairs.push_back((uint16_t)(jj | (jk << 8)));
      }
      pptr.push_back((int32_t)pairs.size());
    }
    lptr[i + 1] = lptr[i] + dpos[i];
  }
  if (pairs.size() >= (size_t)INT32_MAX)
    return ctx_fail(ctx, VMS_ERR_UNSUPPORTED, "ILU(0): too many update pairs");
  // sweep segments: node i continues the segment of i - 1 when the two are coupled (adjacency
  // lists are sorted, so i - 1 is the entry just before the diagonal)
  std::vector<int32_t> seg;
  seg.reserve((size_t)N / 8 + 2);
  int run = 0;
  for (int64_t i = 0; i < N; ++i) {
    const bool coupled = i > 0 && dpos[i] > 0 && adj[start[i] + dpos[i] - 1] == i - 1;
    if (coupled && run < ILU_SEG_MAX) {
      ++run;
    } else {
      seg.push_back((int32_t)i);
      run = 1;
    }
  }
  seg.push_back((int32_t)N);
  p.n_nodes = N;
  p.n_lower = lptr[N];
  p.n_pairs = (int64_t)pairs.size();
  p.n_segs = (int64_t)seg.size() - 1;
  e = cudaMalloc(&p.dpos, sizeof(int32_t) * N);
  if (e == cudaSuccess) e = cudaMalloc(&p.seg, sizeof(int32_t) * seg.size());
  if (e == cudaSuccess) e = cudaMemcpy(p.seg, seg.data(), sizeof(int32_t) * seg.size(), cudaMemcpyHostToDevice);
  p.seg_host = std::move(seg);
  if (e == cudaSuccess) e = cudaMalloc(&p.lptr, sizeof(int32_t) * (N + 1));
  if (e == cudaSuccess) e = cudaMalloc(&p.pptr, sizeof(int32_t) * pptr.size());
  if (e == cudaSuccess) e = cudaMalloc(&p.pairs, sizeof(uint16_t) * std::max<size_t>(1, pairs.size()));
  if (e == cudaSuccess) e = cudaMemcpy(p.dpos, dpos.data(), sizeof(int32_t) * N, cudaMemcpyHostToDevice);
  if (e == cudaSuccess) e = cudaMemcpy(p.lptr, lptr.data(), sizeof(int32_t) * (N + 1), cudaMemcpyHostToDevice);
  if (e == cudaSuccess) e = cudaMemcpy(p.pptr, pptr.data(), sizeof(int32_t) * pptr.size(), cudaMemcpyHostToDevice);
  if (e == cudaSuccess && !pairs.empty())
    e = cudaMemcpy(p.pairs, pairs.data(), sizeof(uint16_t) * pairs.size(), cudaMemcpyHostToDevice);
  if (e != cudaSuccess)
    return ctx_fail(ctx, e == cudaErrorMemoryAllocation ? VMS_ERR_OUT_OF_MEMORY : VMS_ERR_CUDA,
                    cudaGetErrorString(e));
  return VMS_OK;
}

int ensure_work(vms_ctx* ctx, Ilu& p, const Mesh& m, bool fp32) {
  cudaError_t e = cudaSuccess;
  if (!p.F) {
    e = cudaMalloc(&p.F, sizeof(double) * m.nnz);
    if (e == cudaSuccess) e = cudaMalloc(&p.Dinv, sizeof(double) * 16 * m.n_nodes);
    if (e == cudaSuccess) e = cudaMalloc(&p.y, sizeof(double) * 4 * m.n_nodes);
    if (e == cudaSuccess) e = cudaMalloc(&p.x64, sizeof(double) * 4 * m.n_nodes);
  }
  if (e == cudaSuccess && fp32 && !p.F32) {
    e = cudaMalloc(&p.F32, sizeof(float) * m.nnz);
    if (e == cudaSuccess) e = cudaMalloc(&p.Dinv32, sizeof(float) * 16 * m.n_nodes);
    if (e == cudaSuccess) e = cudaMalloc(&p.vals64, sizeof(double) * m.nnz);
  }
  if (e == cudaSuccess && !p.flags) {
    e = cudaMalloc(&p.flags, sizeof(uint32_t) * m.n_nodes);
    if (e == cudaSuccess) e = cudaMemset(p.flags, 0, sizeof(uint32_t) * m.n_nodes);
    if (e == cudaSuccess) e = cudaMalloc(&p.yp, sizeof(unsigned long long) * 4 * m.n_nodes);
    if (e == cudaSuccess) e = cudaMemset(p.yp, 0, sizeof(unsigned long long) * 4 * m.n_nodes);
    if (e == cudaSuccess) e = cudaMalloc(&p.xp, sizeof(unsigned long long) * 4 * m.n_nodes);
    if (e == cudaSuccess) e = cudaMemset(p.xp, 0, sizeof(unsigned long long) * 4 * m.n_nodes);
    if (e == cudaSuccess) e = cudaMalloc(&p.tickets, sizeof(unsigned long long));
    if (e == cudaSuccess) e = cudaMemset(p.tickets, 0, sizeof(unsigned long long));
    if (e == cudaSuccess) e = cudaMalloc(&p.err, sizeof(int));
    if (e == cudaSuccess) e = cudaMemset(p.err, 0, sizeof(int));
    p.epoch = 0;
    p.base = 0;
  }
  if (e != cudaSuccess)
    return ctx_fail(ctx, e == cudaErrorMemoryAllocation ? VMS_ERR_OUT_OF_MEMORY : VMS_ERR_CUDA,
                    cudaGetErrorString(e));
  return VMS_OK;
}

template <typename A, typename B>
__global__ void convert_kernel(const A* __restrict__ x, B* __restrict__ y, int64_t n) {
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n;
       i += (int64_t)gridDim.x * blockDim.x)
    y[i] = B(x[i]);
}

template <typename A, typename B>
int convert(const A* x, B* y, int64_t n, cudaStream_t st) {
  const int64_t b = (n + 255) / 256;
  const int64_t cap = (int64_t)sm_count() * 8;
  convert_kernel<A, B><<<(unsigned)(b > cap ? cap : (b < 1 ? 1 : b)), 256, 0, st>>>(x, y, n);
  return 1;
}

}  // namespace

void free_ilu(Ilu& p) {
  const uint32_t lim = p.spin_limit;  // a setting of the context, kept across meshes
  void* bufs[] = {p.dpos, p.lptr, p.pptr, p.pairs, p.F, p.Dinv, p.y, p.x64, p.F32, p.Dinv32,
                  p.vals64, p.flags, p.yp, p.xp, p.tickets, p.err, p.seg};
  for (void* b : bufs)
    if (b) cudaFree(b);
  p = Ilu();
  p.spin_limit = lim;
}

int ilu_factor(vms_ctx* ctx, Ilu& p, const Mesh& m, bool fp32, const void* values, cudaStream_t st,
               int* launches) {
  *launches = 0;
  if (p.dpos && p.n_nodes != m.n_nodes) free_ilu(p);
  if (!p.dpos)
    if (int rc = build_pattern(ctx, p, m)) return rc;
  if (int rc = ensure_work(ctx, p, m, fp32)) return rc;
  // The elimination always runs in FP64 (from the FP32 values in mixed precision): FP32
  // elimination of the condensed systems of distorted meshes, whose condition numbers reach
  // 1e9-1e10, gives factors too poor for GMRES to converge. Mixed precision then rounds the
  // finished factor to FP32 for the FP32 sweeps.
  const double* A = reinterpret_cast<const double*>(values);
  if (fp32) {
    *launches += convert<float, double>((const float*)values, p.vals64, m.nnz, st);
    A = p.vals64;
  }
  const unsigned ctas = resident_ctas(m.n_nodes, ILU_FWARPS, 8 * sm_count());
  const uint32_t ep = next_epoch(p, st);
  ilu_factor_kernel<double><<<ctas, ILU_FWARPS * 32, 0, st>>>(
      m.rowptr, m.colidx, A, p.F, p.Dinv, p.dpos, p.lptr, p.pptr, p.pairs, m.n_nodes, p.flags, ep,
      p.tickets, p.base, p.err, p.spin_limit);
  p.base += (unsigned long long)m.n_nodes + (unsigned long long)ctas * ILU_FWARPS;
  *launches += 1;
  if (fp32) {
    *launches += convert<double, float>(p.F, p.F32, m.nnz, st);
    *launches += convert<double, float>(p.Dinv, p.Dinv32, 16 * m.n_nodes, st);
  }
  p.factored = true;
  const cudaError_t e = cudaGetLastError();
  return e == cudaSuccess ? VMS_OK : ctx_fail(ctx, VMS_ERR_CUDA, cudaGetErrorString(e));
}

// Segments covering nodes [n0, n1): [s0, s0 + count). Rows outside [n0, n1) are clamped away in
// the kernel (a block solve has no couplings outside its rows, so n0 and n1 are segment starts).
static void segment_range(const Ilu& p, int64_t n0, int64_t n1, int64_t& s0, int64_t& count) {
  const std::vector<int32_t>& sg = p.seg_host;
  const int64_t a = (int64_t)(std::upper_bound(sg.begin(), sg.end() - 1, (int32_t)n0) - sg.begin()) - 1;
  const int64_t b = (int64_t)(std::lower_bound(sg.begin(), sg.end() - 1, (int32_t)n1) - sg.begin());
  s0 = a < 0 ? 0 : a;
  count = b - s0;
}

template <>
int ilu_apply<float, float>(Ilu& p, const Mesh& m, int64_t n0, int64_t n1, const float* v, float* z,
                            cudaStream_t st) {
  const int64_t rows = n1 - n0;
  int64_t s0 = 0, ns = 0;
  segment_range(p, n0, n1, s0, ns);
  constexpr int W = sweep_warps<float>();
  const int64_t chunks = (ns + W - 1) / W;
  const unsigned ctas = resident_ctas(chunks, 1, 4 * sm_count());  // at most four CTAs per SM
  const unsigned long long claims = (unsigned long long)chunks + ctas;  // + each CTA's last claim
  uint32_t ep = next_epoch(p, st);
  const size_t ring = sweep_ring_bytes<float>(W);
  // the ring needs more than the default 48 KB of dynamic shared memory (set for the current device)
  cudaFuncSetAttribute(ilu_sweep_kernel<float, true>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)ring);
  cudaFuncSetAttribute(ilu_sweep_kernel<float, false>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)ring);
  ilu_sweep_kernel<float, true><<<ctas, W * 32, ring, st>>>(
      m.rowptr, m.colidx, p.F32, nullptr, p.dpos, p.seg, s0, ns, v, nullptr, p.yp, nullptr, n0,
      rows, ep, p.tickets, p.base, p.err, p.spin_limit);
  p.base += claims;
  ep = next_epoch(p, st);
  ilu_sweep_kernel<float, false><<<ctas, W * 32, ring, st>>>(
      m.rowptr, m.colidx, p.F32, p.Dinv32, p.dpos, p.seg, s0, ns, nullptr, p.yp, p.xp, z, n0,
      rows, ep, p.tickets, p.base, p.err, p.spin_limit);
  p.base += claims;
  return 2;
}

template <>
int ilu_apply<double, double>(Ilu& p, const Mesh& m, int64_t n0, int64_t n1, const double* v,
                              double* z, cudaStream_t st) {
  const int64_t rows = n1 - n0;
  int64_t s0 = 0, ns = 0;
  segment_range(p, n0, n1, s0, ns);
  constexpr int W = sweep_warps<double>();
  const int64_t chunks = (ns + W - 1) / W;
  const unsigned ctas = resident_ctas(chunks, 1, 4 * sm_count());  // at most four CTAs per SM
  const unsigned long long claims = (unsigned long long)chunks + ctas;  // + each CTA's last claim
  double* y = p.y;
  double* x = p.x64;
  cudaMemsetAsync(y + 4 * n0, 0xff, sizeof(double) * 4 * rows, st);
  const size_t ring = sweep_ring_bytes<double>(W);
  // the ring needs more than the default 48 KB of dynamic shared memory (set for the current device)
  cudaFuncSetAttribute(ilu_sweep_kernel<double, true>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)ring);
  cudaFuncSetAttribute(ilu_sweep_kernel<double, false>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)ring);
  ilu_sweep_kernel<double, true><<<ctas, W * 32, ring, st>>>(
      m.rowptr, m.colidx, p.F, nullptr, p.dpos, p.seg, s0, ns, v, nullptr, y, nullptr, n0, rows, 0,
      p.tickets, p.base, p.err, p.spin_limit);
  p.base += claims;
  cudaMemsetAsync(x + 4 * n0, 0xff, sizeof(double) * 4 * rows, st);
  ilu_sweep_kernel<double, false><<<ctas, W * 32, ring, st>>>(
      m.rowptr, m.colidx, p.F, p.Dinv, p.dpos, p.seg, s0, ns, y, nullptr, x, z, n0, rows, 0,
      p.tickets, p.base, p.err, p.spin_limit);
  p.base += claims;
  return 4;
}

int ilu_status(vms_ctx* ctx, Ilu& p, cudaStream_t st) {
  if (!p.err) return VMS_OK;
  int h = 0;
  cudaError_t e = cudaMemcpyAsync(&h, p.err, sizeof(int), cudaMemcpyDeviceToHost, st);
  if (e == cudaSuccess) e = cudaStreamSynchronize(st);
  if (e != cudaSuccess) return ctx_fail(ctx, VMS_ERR_CUDA, cudaGetErrorString(e));
  if (h == 0) return VMS_OK;
  // a launch stopped early: its claims and flags are unknown, so start both afresh
  cudaMemsetAsync(p.err, 0, sizeof(int), st);
  cudaMemsetAsync(p.tickets, 0, sizeof(unsigned long long), st);
  cudaMemsetAsync(p.flags, 0, sizeof(uint32_t) * p.n_nodes, st);
  cudaMemsetAsync(p.yp, 0, sizeof(unsigned long long) * 4 * p.n_nodes, st);
  cudaMemsetAsync(p.xp, 0, sizeof(unsigned long long) * 4 * p.n_nodes, st);
  cudaStreamSynchronize(st);
  p.base = 0;
  p.epoch = 0;
  p.factored = false;
  return h == ILU_ERR_PIVOT
             ? ctx_fail(ctx, VMS_ERR_ZERO_PIVOT, "ILU(0): zero pivot in a diagonal block")
             : ctx_fail(ctx, VMS_ERR_TIMEOUT, "ILU(0): a row waited longer than its limit");
}

}  // namespace vms
