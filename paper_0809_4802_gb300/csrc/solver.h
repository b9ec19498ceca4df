// Krylov solve, fine-scale recovery and Newton driver of the condensed system (Sections 4.2, 5, 6).
#pragma once

#include <vector>

#include "precond.h"
#include "vms_internal.h"

namespace vms {

// A block of the condensed system: nodes [n0, n1) and elements [e0, e1), closed under the mesh
// connectivity (no element couples it to other nodes), so the rows of its nodes have no columns
// outside it. The whole mesh is one such block.
struct SysRange {
  int64_t n0 = 0, n1 = 0, e0 = 0, e1 = 0;
  int64_t nodes() const { return n1 - n0; }
};

// A bandwidth-reducing node order of one block of the system (reverse Cuthill-McKee), kept for the
// banded direct solve: perm[a] = position of node n0 + a in the band order (device), bw = the
// largest |position difference| of two coupled nodes (-1: the block is too large to be ordered).
struct BandOrder {
  int64_t n0 = 0, n1 = 0;
  int32_t* perm = nullptr;
  int bw = -1;
};

struct SolverWork {
  double* x = nullptr;       // n
  double* r = nullptr;       // n
  double* V = nullptr;       // (restart + 1) * n Krylov basis
  double* Z = nullptr;       // n preconditioned vector (FP32 views in mixed mode)
  double* Dinv = nullptr;    // n_nodes * 16: inverted 4x4 diagonal node blocks
  double* h = nullptr;       // device scalars for dots
  double* rfull = nullptr;   // n: FP64 refinement residual (mixed)
  float* bf = nullptr;       // n: FP32 right-hand side of the inner solve (mixed)
  float* xf = nullptr;       // n: FP32 inner correction (mixed)
  double* cx = nullptr;      // n: FP64 correction of the final stage of the mixed solve
  float* pv = nullptr;       // n: FP32 copy of a vector the FP32 factor is applied to
  float* pz = nullptr;       // n: its FP32 result
  double* Zf = nullptr;      // zf_restart * n: preconditioned vectors of the flexible final stage
  int zf_restart = 0;
  double* xb = nullptr;      // n: refinement iterate before the last FP32 correction
  double* rb = nullptr;      // n: its FP64 residual
  int* band = nullptr;       // 4 ints: the banded direct solve's state and error words
  std::vector<BandOrder> band_orders;  // per block solved directly so far
  Ilu ilu;                   // ILU(0) pattern, factor and sweep work
  bool use_ilu = false;      // preconditioner of the current solve: ILU(0) or block Jacobi
  uint64_t ilu_for = 0;      // assembly the ILU(0) factor was computed for (0: none)
  uint64_t dinv_for = 0;     // assembly the block-Jacobi inverses were computed for (0: none)
  int restart = 0;
  int64_t n = 0;
};

void free_solver(SolverWork& s);

// accessors defined in api.cu
const Mesh& ctx_mesh(vms_ctx* c);
State& ctx_state(vms_ctx* c);
Work& ctx_work(vms_ctx* c);
SolverWork& ctx_solver(vms_ctx* c);
cudaStream_t ctx_stream(vms_ctx* c);
int ctx_device(vms_ctx* c);
bool ctx_fp32(vms_ctx* c);
int ctx_precond(vms_ctx* c);
bool ctx_instance(vms_ctx* c, int64_t i, SysRange* out);
bool ctx_stale(vms_ctx* c, int64_t i);
void ctx_mark_stale(vms_ctx* c, int64_t i);
int64_t* ctx_solver_stats(vms_ctx* c);
double* ctx_dscalar(vms_ctx* c);
double* ctx_hscalar(vms_ctx* c);
int ctx_fail(vms_ctx* c, int code, const char* msg);
int ctx_flags_check(vms_ctx* c);

// Kernel accounting: counts the launches made inside the scope under `kind` and, when timing is
// enabled on the context, brackets them with CUDA events on the context's stream.
struct KScope {
  vms_ctx* c;
  int kind;
  int n = 0;
  cudaEvent_t a = nullptr;
  cudaStream_t s = nullptr;
  KScope(vms_ctx* c, int kind);
  KScope(vms_ctx* c, int kind, cudaStream_t stream);
  ~KScope();
  void add(int launches) { n += launches; }
};

}  // namespace vms
