// Internal declarations shared by the translation units of libvms_gb300.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include <string>
#include <vector>

#include "../../include/vms.h"
#include "band_order.h"

struct vms_ctx;

namespace vms {

// Error flags raised by kernels (bitwise OR into a device word, read back by the host).
enum : unsigned int {
  FLAG_NEG_JACOBIAN = 1u,
  FLAG_SINGULAR_KFF = 2u,
  FLAG_NAN = 4u,
};

// Reference-element tables for one Gauss rule (device memory owned by the context).
constexpr int MAX_QP = 64;  // quad_order <= 4

// Per-quadrature-point table row (FP64): coordinates and products for the modal (monomial)
// evaluation of trilinear fields, the bubble, its reference gradient and the weight.
struct QpRow {
  double xi, eta, zeta, xe, xz, ez, xez;  // xi, eta, zeta, xi*eta, xi*zeta, eta*zeta, xi*eta*zeta
  double b, db0, db1, db2;                 // bubble (times bubble_scale) and its reference gradient
  double w;                                // Gauss weight
};

// Scalar parameters passed by value to the element kernels.
struct KParams {
  double nut;    // visc_factor * nu
  double tau;    // 1/dt or 0
  double f[3];   // body force
  int nq;        // number of quadrature points
  int transient; // tau != 0
  int has_force; // f != 0
  const double* nu_e;  // per-element viscosity (device, n_elems) or null: nut = visc_factor * nu_e[e]
  double visc_factor;
  const double* tab64;   // FP64 reference table of the tangent kernel (37 nq), for FP64 K_ff
  int tangent_warps;     // warps per tangent block (0: default)
  int residual_threads;  // threads per residual block (0: default)
  const double* ts_basis = nullptr;  // FP64 tangent: one-dimensional basis (8 x 4), nq = 8 or 27
  const uint32_t* ts_plan = nullptr;  // FP64 tangent: plan of the factorised sums
};

// The once-per-mesh pattern (host side, built by pattern.cpp).
struct HostPattern {
  std::vector<int32_t> rowptr;    // 4*n_nodes + 1
  std::vector<int32_t> colidx;    // nnz
  std::vector<int32_t> blk;       // n_elems * npe^2: value offset of block (a,b), row 4*na, col 4*nb
  std::vector<int32_t> rowlen;    // n_nodes: entries per row of node n (4 * neighbours)
  std::vector<int32_t> colour;    // n_elems
  std::vector<int32_t> colour_order;  // elements sorted by colour
  std::vector<int32_t> colour_start;  // n_colours + 1
  std::vector<int64_t> diag_pos;  // per constrained dof: value index of its diagonal entry
  std::vector<uint32_t> dir_mask; // per element: bit 4a+c set if that coarse dof is constrained
  int n_colours = 0;
};

// One-dimensional basis rows (psi_0..2, phi_0..1, 1 at the n1 Gauss points x, 8 x 4 doubles) and
// the plan of the FP64 tangent's factorised sums for the n1^3-point rule (n1 = 2 or 3). False if
// the partial sums do not fit the per-warp area.
bool ts_tables(int n1, const double* x, std::vector<double>& basis, std::vector<uint32_t>& plan);

// Builds the CSR pattern, block map, colouring and Dirichlet masks. Returns "" or an error text.
std::string build_pattern(int64_t n_nodes, int64_t n_elems, const int32_t* conn, int64_t n_dir,
                          const int64_t* dir_dof, HostPattern& out, int npe);

// ---- device data and kernel launchers ----------------------------------------------------------

struct Mesh {
  int64_t n_nodes = 0, n_elems = 0, nnz = 0;
  int npe = 8;                   // nodes per element: 8 (hexahedron) or 4 (tetrahedron)
  double4_32a* xyz = nullptr;        // n_nodes (x, y, z, 0)
  int32_t* conn = nullptr;       // n_elems * npe
  int32_t* rowptr = nullptr;     // 4 n_nodes + 1
  int32_t* colidx = nullptr;     // nnz
  int32_t* blk = nullptr;        // n_elems * npe^2
  int32_t* rowlen = nullptr;     // n_nodes
  uint32_t* dir_mask = nullptr;  // n_elems
  int64_t n_dir = 0;
  int64_t* dir_dof = nullptr;    // n_dir
  double* dir_val = nullptr;     // n_dir
  int64_t* diag_pos = nullptr;   // n_dir
  int32_t* colour_order = nullptr;
  double* nu_e = nullptr;        // n_elems per-element viscosity, or null (vms_set_element_viscosity)
  std::vector<int32_t> colour_start;
  int n_colours = 0;
};

struct State {
  double4_32a* u = nullptr;       // n_nodes (v0, v1, v2, p)
  double4_32a* u_prev = nullptr;  // n_nodes
  double* beta = nullptr;     // n_elems * 3
  bool valid = false;
};

struct Fp32Copy {
  float4* u = nullptr;        // n_nodes (v, p) in FP32
  float* beta = nullptr;      // n_elems * 3
  float4* xhl = nullptr;      // n_nodes * 2: FP32 high and low parts of the coordinates (x = hi + lo)
};

struct Work {
  void* values = nullptr;     // nnz (double or float)
  double* rhs = nullptr;      // 4 n_nodes
  double* elemR = nullptr;    // n_elems * 36: R_cp (32), R_f (3), pad
  void* recX = nullptr;       // n_elems * 96 (T): K_ff^-1 K_fc
  void* recKcf = nullptr;     // n_elems * 96 (T): K_cf, row-major [32][3] (hexahedra)
  double* recKinv = nullptr;  // n_elems * 9: K_ff^-1 (FP64)
  double* recY = nullptr;     // n_elems * 3: K_ff^-1 R_f
  double* resid = nullptr;    // 4 n_nodes + 3 n_elems
  double* partial = nullptr;  // reduction partials
  unsigned int* flags = nullptr;
  unsigned long long* queues = nullptr;  // 2 work counters of the fused assembly kernel
  Fp32Copy f32;               // mixed precision only
  cudaStream_t aux = nullptr; // second stream for the tangent kernel
  cudaEvent_t fork = nullptr, join = nullptr;
  bool assembled = false;
  uint64_t assembly_id = 0;   // incremented by every assembly (preconditioner caching)
};

// Element residual (FP64, modal evaluation). mode 0: write elemR[36*e + ...] (R_cp 32, R_f 3);
// mode 1: accumulate the assembled residual into resid (4 n_nodes + 3 n_elems entries).
int launch_residual(const Mesh& m, const State& s, const KParams& kp, const QpRow* qp,
                     double* elemR, double* resid, int64_t first, int64_t count, int mode,
                     unsigned int* flags, cudaStream_t st);

// Element tangent + condensation + scatter (warp per element). T = double or float.
struct TangentOut {
  void* values = nullptr;      // CSR values (assembly)
  double* rhs = nullptr;       // condensed right-hand side (assembly, finish kernel)
  void* recX = nullptr;        // per element K_ff^-1 K_fc (T)
  void* recKcf = nullptr;      // per element K_cf (T), row-major [32][3] (finish kernel)
  double* recKinv = nullptr;   // per element K_ff^-1
  double* recY = nullptr;      // per element K_ff^-1 R_f (finish kernel)
  // element outputs (parity), FP64, may be null
  double *S = nullptr, *r = nullptr, *Kcc = nullptr, *Kcf = nullptr, *Kfc = nullptr,
         *Kff = nullptr;
};
// Tetrahedral element (tet.cu). On an affine tetrahedron every integrand of the residual and the
// tangent is a reference polynomial (products of lambda_a, b and db/dxi) times element constants,
// so the element needs only the reference moments below, summed once per quadrature rule with the
// rule's own points and weights (sum_q w_q f(xi_q)): the results equal the point-by-point sums up
// to the order of rounding.
enum : int {
  TM_M0 = 0,      // sum w
  TM_M1 = 1,      // [a]        lambda_a
  TM_M2 = 5,      // [a][c]     lambda_a lambda_c
  TM_M1B = 21,    // [a]        lambda_a b
  TM_MB = 25,     //            b
  TM_MBB = 26,    //            b^2
  TM_MD = 27,     // [al]       db_al
  TM_M1D = 30,    // [a][al]    lambda_a db_al
  TM_M2D = 42,    // [a][c][al] lambda_a lambda_c db_al
  TM_M1BD = 90,   // [a][al]    lambda_a b db_al
  TM_MBBD = 102,  // [al]       b^2 db_al
  TM_MDD = 105,   // [al][be]   db_al db_be
  TM_COUNT = 114,
};
struct TetMoments {
  double m[TM_COUNT];
};
void tet_moments(int n, double bubble_scale, TetMoments& mom);
// The whole assembly of a tetrahedral mesh (residual, tangent, condensation, scatter, r_e and the
// recovery data) in one kernel; FP64 arithmetic, values stored in FP32 when fp32.
int launch_tet_assembly(bool fp32, const Mesh& m, const State& s, const KParams& kp,
                        const TetMoments& mom, const TangentOut& o, int64_t first, int64_t count,
                        const int32_t* elem_list, bool elem_outputs, bool atomic,
                        unsigned int* flags, cudaStream_t st);
// Tetrahedral residual: mode 0 per element into elemR (stride 36), mode 1 assembled into resid.
int launch_tet_residual(const Mesh& m, const State& s, const KParams& kp, const TetMoments& mom,
                        double* elemR, double* resid, int64_t first, int64_t count, int mode,
                        unsigned int* flags, cudaStream_t st);

// The three warps-per-block counts the tangent kernel is compiled for (k = 0, 1, 2; 1 = default).
int tangent_warp_choice(bool fp32, int k);
// engine (FP32 only): 0 CUDA-core contractions, 1 BF16 tensor cores, 2 split-TF32 tensor cores.
int launch_tangent(bool fp32, int engine, const Mesh& m, const State& s, const Fp32Copy& c32,
                   const KParams& kp, const void* tab, const TangentOut& out, int64_t first,
                   int64_t count, const int32_t* elem_list, bool elem_outputs, bool atomic,
                   unsigned int* flags, cudaStream_t st);
// Mixed precision with the atomic scatter: the residual (into elemR) and the FP32 tangent (into
// out) in one persistent launch; `queues` holds two zeroed counters.
int launch_fused_assembly(const Mesh& m, const State& s, const Fp32Copy& c32, const KParams& kp,
                          const QpRow* qp, const float* tab32, double* elemR, const TangentOut& o,
                          unsigned long long* queues, unsigned int* flags, cudaStream_t st);
// y = K_ff^-1 R_f into recY and r_e = R_cp - K_cf y (FP64) into rhs (or into out.r).
int launch_finish(bool fp32, const Mesh& m, const double* elemR, const TangentOut& out,
                  int64_t first, int64_t count, const int32_t* elem_list, bool atomic,
                  cudaStream_t st);
// FP32 copies of the nodal state and of beta.
int launch_to_fp32(const Mesh& m, const State& s, const Fp32Copy& c, cudaStream_t st);

// Streaming multiprocessors of the current device (cudaDevAttrMultiProcessorCount, looked up once
// per device). Grid sizes are multiples of it.
int sm_count();

int launch_fill_zero(void* p, size_t bytes, cudaStream_t st);
int launch_dirichlet_diag(const Mesh& m, void* values, bool fp32, double* rhs, cudaStream_t st);
int launch_zero_dofs(const int64_t* dofs, int64_t n, double* v, cudaStream_t st);
int launch_impose(const Mesh& m, double4_32a* u, cudaStream_t st);
// sum of squares of v[0..n) -> *out (device double), two passes through `partial` (>= 512)
int launch_norm2(const double* v, int64_t n, double* partial, double* out, cudaStream_t st);
int launch_spmv(const Mesh& m, const void* values, bool fp32, const double* x, double* y,
                 cudaStream_t st);

}  // namespace vms
