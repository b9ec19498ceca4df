// Preconditioners of the condensed system for the Krylov solve (Section 6: the linear systems were
// solved with a Krylov method whose default preconditioner, on one process, is an incomplete LU
// factorisation with no fill).
#pragma once

#include "vms_internal.h"

namespace vms {

constexpr int ILU_ERR_TIMEOUT = 1;
constexpr uint32_t ILU_SPIN_DEFAULT = 1u << 22;  // with a 32 ns sleep per poll: about 0.13 s
constexpr int ILU_ERR_PIVOT = 2;
constexpr int ILU_MAX_DEG = 32;
constexpr int ILU_SEG_MAX = 64;

// Block ILU(0) of the node-block matrix (4x4 blocks, natural node order), factored and applied on
// the device by warps that each own one node row and wait for the rows their row depends on.
struct Ilu {
  // pattern (built once per mesh, on first use)
  int32_t* dpos = nullptr;     // n_nodes: position of the diagonal block in the node row
  int32_t* lptr = nullptr;     // n_nodes + 1: first lower-block entry of each node row
  int32_t* pptr = nullptr;     // n_lower + 1: first update pair of each lower block
  uint16_t* pairs = nullptr;   // n_pairs: (jj | jk << 8) for A_ij -= L_ik U_kj
  int64_t n_nodes = 0, n_lower = 0, n_pairs = 0;
  // sweep segments: maximal runs of consecutive nodes each coupled to the one before (at most
  // ILU_SEG_MAX long); segment s is nodes seg[s] .. seg[s+1] - 1
  int32_t* seg = nullptr;           // device, n_segs + 1
  std::vector<int32_t> seg_host;    // host copy (segment ranges of node blocks)
  int64_t n_segs = 0;
  // factor (always eliminated in FP64) and sweep work
  double* F = nullptr;         // nnz: L (unit lower, strictly lower blocks) and U, CSR layout
  double* Dinv = nullptr;      // n_nodes * 16: inverses of the diagonal blocks of U
  float* F32 = nullptr;        // mixed precision: F rounded to FP32 (FP32 sweeps)
  float* Dinv32 = nullptr;     // mixed precision: Dinv rounded to FP32
  double* vals64 = nullptr;    // mixed precision: FP64 copy of the FP32 matrix values
  double* y = nullptr;         // 4 n_nodes: FP64 forward-sweep publication
  double* x64 = nullptr;       // 4 n_nodes: FP64 backward-sweep publication
  uint32_t* flags = nullptr;   // n_nodes: row-ready epochs (factorisation, FP64 sweeps)
  unsigned long long* yp = nullptr;  // 4 n_nodes: FP32 forward sweep, (epoch << 32 | value bits)
  unsigned long long* xp = nullptr;  // 4 n_nodes: FP32 backward sweep, same packing
  unsigned long long* tickets = nullptr;  // row-claim counters (never reset between launches)
  int* err = nullptr;          // device error word: 0, ILU_ERR_TIMEOUT or ILU_ERR_PIVOT
  uint32_t epoch = 0;
  unsigned long long base = 0; // claims made on `tickets` by earlier launches
  uint32_t spin_limit = ILU_SPIN_DEFAULT;  // polls of one device-side wait before it gives up
  bool factored = false;
};


void free_ilu(Ilu& p);

// Build the pattern if needed, allocate the work for element type T (float or double) and queue
// the factorisation of `values` on `st`. Returns a VMS status (host-side failures only); device-side
// failures (zero pivot, wait timeout) are reported by ilu_status().
int ilu_factor(vms_ctx* ctx, Ilu& p, const Mesh& m, bool fp32, const void* values, cudaStream_t st,
               int* launches);

// z = (LU)^-1 v. T is the element type of the factor, VT the vector type. Returns the launches.
// Rows of nodes [n0, n1) only (a block of the matrix with no couplings outside it); v and z are
// compact: entry 4 (i - n0) + c belongs to node i.
template <typename T, typename VT>
int ilu_apply(Ilu& p, const Mesh& m, int64_t n0, int64_t n1, const VT* v, VT* z, cudaStream_t st);
template <>
int ilu_apply<float, float>(Ilu& p, const Mesh& m, int64_t n0, int64_t n1, const float* v, float* z,
                            cudaStream_t st);
template <>
int ilu_apply<double, double>(Ilu& p, const Mesh& m, int64_t n0, int64_t n1, const double* v,
                              double* z, cudaStream_t st);

// Read the device error word (synchronises `st`); on error, resets the claim counters and flags.
int ilu_status(vms_ctx* ctx, Ilu& p, cudaStream_t st);

}  // namespace vms
