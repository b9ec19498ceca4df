/*
 * vms.h - C-ABI of the GB300-native variational multiscale (VMS) Newton-Schur library.
 *
 * The library forms, on one GPU, the element-level consistent Newton tangent and residual of the
 * two-level VMS weak form of the incompressible Navier-Stokes equations (Turner, Nakshatrala &
 * Hjelmstad, Sections 3-4: Eqs. SC_CoarseScale_Momentum, SC_CoarseScale_Continuity,
 * SC_FineScale_Momentum, SC_Coarse_Resid_Vec, SC_Coarse_Resid_Vec_2, SC_Fine_Resid_Vec and the
 * backward-Euler Remark), statically condenses the per-element bubble unknowns into the Schur
 * complement S_e = K_cc - K_cf K_ff^-1 K_fc with r_e = R_cp - K_cf K_ff^-1 R_f (Section 5, Eq.
 * SchurUpdate), and scatter-adds S_e, r_e into a global non-symmetric CSR matrix whose sparsity
 * pattern is built once per mesh (the assembly operator A of Section 5).
 *
 * Element: 8-node trilinear hexahedron, equal-order velocity/pressure, one vector bubble
 * b = (1-xi^2)(1-eta^2)(1-zeta^2) per element (Eq. DefineBubbles3), Gauss rule of quad_order^3
 * points. Local node order: (-,-,-) (+,-,-) (+,+,-) (-,+,-) (-,-,+) (+,-,+) (+,+,+) (-,+,+).
 *
 * Degrees of freedom are node-major: global coarse dof 4*node + c, c = 0,1,2 velocity, c = 3
 * pressure. The three bubble unknowns of each element are internal (fine scale, Section 3.3).
 *
 * Conventions for every call:
 *  - Every function returns VMS_OK (0) or a negative VMS_ERR_* code and never aborts the process.
 *    vms_last_error() gives a one-line message for the last failure on that context.
 *  - Pointers marked "host or device" may point to host memory (pageable or pinned) or to device
 *    memory of the context's GPU; copies use unified addressing. The caller keeps ownership of
 *    every pointer it passes; the library copies what it needs before returning (except where a
 *    call says it writes into a caller buffer).
 *  - Pointers returned by the library (vms_csr_view) are device pointers it owns; they stay valid
 *    until the next call that changes the mesh or destroys the context.
 *  - All GPU work is ordered on the context's stream (vms_set_stream; default: the legacy default
 *    stream). Calls that return host values (norms, iteration counts) synchronise that stream.
 *  - A context is not thread-safe; use one context per host thread.
 */
#ifndef VMS_GB300_H
#define VMS_GB300_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

/* ---- status codes -------------------------------------------------------------------------- */
#define VMS_OK 0
#define VMS_ERR_INVALID_ARG -1      /* null pointer, size out of range, bad mode */
#define VMS_ERR_CUDA -2             /* a CUDA runtime call failed (message has the CUDA error) */
#define VMS_ERR_OUT_OF_MEMORY -3    /* device allocation failed */
#define VMS_ERR_NEG_JACOBIAN -4     /* det J <= 0 (or below the smallest normal FP64 value) at a
                                      quadrature point of some element */
#define VMS_ERR_SINGULAR_KFF -5     /* the 3x3 bubble block K_ff of some element is singular */
#define VMS_ERR_NAN -6              /* a non-finite value appeared in a residual or matrix */
#define VMS_ERR_KRYLOV_MAXIT -7     /* linear solve reached maxit without meeting its tolerance */
#define VMS_ERR_NEWTON_DIVERGED -8  /* Newton residual grew by 1e6 or maxit was reached */
#define VMS_ERR_STATE -9            /* call out of order (e.g. assemble before mesh/state upload) */
#define VMS_ERR_UNSUPPORTED -10     /* option not available in this build */
/* VMS_ERR_TOO_LARGE (-11) is defined with vms_residual_norm_noalloc below */
#define VMS_ERR_ZERO_PIVOT -12      /* a diagonal block of the ILU(0) factorisation is singular */
#define VMS_ERR_TIMEOUT -13         /* a device-side wait exceeded its limit (work abandoned) */

/* ---- precision modes (vms_create) ---------------------------------------------------------- */
#define VMS_PREC_FP64 0   /* all element arithmetic, matrix values and residuals in FP64 */
#define VMS_PREC_MIXED 1  /* tangent blocks and S_e in FP32; residual R, K_ff^-1, r_e in FP64 */
/* VMS_PREC_MIXED with the tangent's basis contractions (every coarse block and the coarse-fine
 * couplings: per element two small GEMMs against the reference basis at the quadrature points,
 * Eq. NewtonUpdate2) on the tensor cores (mma.sync), FP32 accumulation; K_ff, its FP64 inverse,
 * the condensation, the FP64 residual and r_e as in VMS_PREC_MIXED. Hexahedra, quad_order <= 3
 * (tetrahedral meshes assemble as in VMS_PREC_MIXED). */
#define VMS_PREC_MIXED_TC_BF16 2  /* BF16 operands, one product: blocks to ~1e-2 relative */
#define VMS_PREC_MIXED_TC_TF32 3  /* TF32 operands split into high and low parts, three products
                                     (the corrections accumulated apart): blocks to ~1e-6 */

/* ---- preconditioners of the Krylov solve (vms_set_preconditioner) ---------------------------- */
#define VMS_PRECOND_ILU0 0          /* block ILU(0), 4x4 node blocks, natural node order (default) */
#define VMS_PRECOND_BLOCK_JACOBI 1  /* inverses of the 4x4 diagonal node blocks */
#define VMS_PRECOND_ILU0_FALLBACK 2 /* ILU(0); a solve that does not converge (or meets a zero
                                       pivot) is repeated by a banded direct LU solve, or where
                                       the band would exceed 48 GiB by block Jacobi and
                                       GMRES(480) */

/* ---- scatter modes (vms_params.scatter_mode) ----------------------------------------------- */
#define VMS_SCATTER_ATOMIC 0  /* one launch, atomic adds into CSR values (order not fixed) */
#define VMS_SCATTER_COLOUR 1  /* one launch per element colour, plain read-modify-write (fixed order) */

typedef struct vms_ctx vms_ctx;

/* Physical and discretisation parameters (Section 2 Eq. SC_Equilibrium; Section 3.2). */
typedef struct {
  double nu;           /* kinematic viscosity nu > 0 */
  double visc_factor;  /* weak-form viscous coefficient nut = visc_factor * nu; 2 as printed in
                          Eq. SC_CoarseScale_Momentum ("2 nu grad w : grad v") */
  double dt;           /* backward-Euler time step (Remark in Section 4.1); 0 means steady */
  double f[3];         /* constant body force b */
  double bubble_scale; /* b = bubble_scale (1-xi^2)(1-eta^2)(1-zeta^2); S_e, r_e do not depend on it */
  int32_t quad_order;  /* Gauss points per direction: 2, 3 or 4 (default 3) */
  int32_t scatter_mode;/* VMS_SCATTER_* */
} vms_params;

/* View of the assembled, Dirichlet-applied condensed system S du = -r (Eq. SchurUpdate). */
typedef struct {
  int64_t n_rows;         /* 4 * n_nodes */
  int64_t nnz;            /* 16 * (number of node pairs sharing an element) */
  const int32_t* rowptr;  /* device, n_rows + 1 entries */
  const int32_t* colidx;  /* device, nnz entries; columns sorted by (node, component) per row */
  const void* values;     /* device, nnz entries; double (values_dtype 0) or float (1) */
  const double* rhs;      /* device, n_rows entries: the assembled condensed residual r (FP64) */
  int32_t values_dtype;   /* 0 = FP64, 1 = FP32 */
  int32_t n_colours;      /* element colours used by VMS_SCATTER_COLOUR */
} vms_csr_view;

/* Create a context on CUDA device `device` in precision mode `precision` (VMS_PREC_*).
 * *ctx receives the new context. Errors: VMS_ERR_INVALID_ARG, VMS_ERR_CUDA. The CSR values are
 * FP32 in every mode but VMS_PREC_FP64. */
int vms_create(vms_ctx** ctx, int device, int precision);

/* Release every device buffer of the context and the context itself. NULL is accepted. */
int vms_destroy(vms_ctx* ctx);

/* Order all later GPU work of the context on `stream` (a cudaStream_t, may be NULL = default). */
int vms_set_stream(vms_ctx* ctx, void* stream);

/* Upload a hexahedral mesh and its Dirichlet set, then build, once per mesh, the CSR pattern of
 * the condensed coarse system, the element-to-CSR block map and an element colouring
 * (Section 5, assembly operator A; the paper assembles after all element work, Section 6).
 *   xyz      host or device, n_nodes x 3 doubles (row-major)
 *   conn     host or device, n_elems x 8 int32 node indices in the local order above
 *   dir_dof  host or device, n_dir global coarse dofs (4*node+c) with prescribed values dir_val;
 *            their Newton increments are zero (Eq. SC_VelocityBC; a pressure pin is a c=3 entry)
 * Replaces any previous mesh and state. Errors: VMS_ERR_INVALID_ARG (sizes, node index out of
 * range, nnz >= 2^31), VMS_ERR_OUT_OF_MEMORY, VMS_ERR_CUDA. */
int vms_mesh_upload(vms_ctx* ctx, int64_t n_nodes, const double* xyz, int64_t n_elems,
                    const int32_t* conn, int64_t n_dir, const int64_t* dir_dof,
                    const double* dir_val);

/* vms_mesh_upload for a mesh of 4-node tetrahedra (P1 velocity and pressure plus one vector bubble
 * b = 256 lambda_0 lambda_1 lambda_2 lambda_3 per element: the MINI-type element the paper cites,
 * Section 3.3). conn: n_elems x 4 int32, positively oriented (reference vertices (0,0,0), (1,0,0),
 * (0,1,0), (0,0,1)). Element blocks have 16 coarse dofs (vms_element_matrices returns 16 x 16
 * S_e). Quadrature: the conical-product rule with params.quad_order points per direction (exact to
 * degree 2 quad_order - 1; vms_tet_rule). The tetrahedral kernels compute in FP64 in both
 * precision modes; VMS_PREC_MIXED stores the CSR values in FP32 for the mixed-precision solve.
 * Errors: as vms_mesh_upload. */
int vms_mesh_upload_tet(vms_ctx* ctx, int64_t n_nodes, const double* xyz, int64_t n_elems,
                        const int32_t* conn, int64_t n_dir, const int64_t* dir_dof,
                        const double* dir_val);

/* The tetrahedral quadrature rule (host only, no GPU needed): n^3 points (pts, 3 n^3 doubles,
 * reference coordinates) and weights (wts, n^3 doubles summing to 1/6), 1 <= n <= 8. */
int vms_tet_rule(int n, double* pts, double* wts);

/* Set nu, visc_factor, dt, body force, bubble scale, quadrature order and scatter mode.
 * Errors: VMS_ERR_INVALID_ARG (nu <= 0, quad_order not in {2,3,4}, dt < 0, bad mode),
 * VMS_ERR_UNSUPPORTED (quad_order 4 in a tensor-core mode). */
int vms_set_params(vms_ctx* ctx, const vms_params* params);

/* Upload the state: nodal (v, p) u [n_nodes x 4], bubble coefficients beta [n_elems x 3] (NULL =
 * zero), and the previous time step's nodal values u_prev [n_nodes x 4] (NULL = u; only read when
 * dt > 0). All host or device doubles. The Dirichlet values of vms_mesh_upload are imposed on u.
 * Errors: VMS_ERR_STATE (no mesh), VMS_ERR_INVALID_ARG. */
int vms_state_upload(vms_ctx* ctx, const double* u, const double* beta, const double* u_prev);

/* Copy the current state to caller buffers (host or device); either pointer may be NULL. */
int vms_state_download(vms_ctx* ctx, double* u, double* beta);

/* Previous time-step velocity and pressure (n_nodes x 4 doubles, host or device; the u_prev of
 * vms_state_upload, or u at the last vms_shift_time). Errors: VMS_ERR_STATE. */
int vms_state_download_prev(vms_ctx* ctx, double* u_prev);

/* One Newton-Schur tangent assembly: for every element, gather its nodes, evaluate geometry and
 * fields at every quadrature point, form R_c, R_p, R_f and the tangent blocks (Section 4),
 * condense the bubble unknowns (Section 5), scatter-add S_e and r_e into the CSR system, then
 * apply the Dirichlet rows and columns (identity rows/columns, zero right-hand side). Also keeps
 * K_ff^-1 K_fc and K_ff^-1 R_f of every element for the fine-scale recovery.
 * `out` (may be NULL) receives the device view of the assembled system.
 * Errors: VMS_ERR_STATE, VMS_ERR_NEG_JACOBIAN, VMS_ERR_SINGULAR_KFF, VMS_ERR_NAN, VMS_ERR_CUDA. */
int vms_assemble_newton_schur(vms_ctx* ctx, vms_csr_view* out);

/* Return the last assembled system without assembling again (VMS_ERR_STATE if none). */
int vms_get_csr(vms_ctx* ctx, vms_csr_view* out);

/* Copy the last assembled system to caller buffers (host or device; any may be NULL): rowptr
 * (4 n_nodes + 1 int32), colidx (nnz int32), values (nnz entries of the view's values_dtype: FP64
 * or FP32) and rhs (4 n_nodes doubles). Synchronises the context's stream. Errors: VMS_ERR_STATE
 * (nothing assembled), VMS_ERR_CUDA. */
int vms_csr_download(vms_ctx* ctx, int32_t* rowptr, int32_t* colidx, void* values, double* rhs);
/* Asynchronous form of vms_csr_download, for pipelines that overlap the transfer of one assembled
 * system with the assembly of the next. The copies to the caller's buffers run on a copy stream of
 * the library after the assembly; the call returns without waiting. While the copy of the values
 * is pending, the next vms_assemble_newton_schur writes a second values buffer of the same size
 * (allocated on first use; in graph mode, vms_set_graph, the values are instead first copied into
 * a device snapshot, as the captured assembly writes one buffer); the right-hand side is copied
 * through a device snapshot. vms_csr_download_wait blocks until the copies have landed. A new
 * vms_csr_download_async, a new mesh and vms_destroy first wait for a pending one. Device views
 * (vms_get_csr) point at the values of the last assembly. The host buffers should be page-locked
 * for the copy to run beside the next assembly; they must stay valid until the wait. Not part of
 * the paper's method: a transfer pipeline for serving.
 * Errors: VMS_ERR_STATE (nothing assembled), VMS_ERR_OUT_OF_MEMORY, VMS_ERR_CUDA. */
int vms_csr_download_async(vms_ctx* ctx, int32_t* rowptr, int32_t* colidx, void* values, double* rhs);
int vms_csr_download_wait(vms_ctx* ctx);

/* Residual-only evaluation in FP64 (Section 4.1 residual vectors, assembled): writes the 2-norm
 * of [R_c, R_p on free dofs; R_f of every element] to *norm (host). If R (host or device, may
 * be NULL) is given it receives the 4*n_nodes + 3*n_elems entries (constrained coarse entries 0).
 * Errors: VMS_ERR_STATE, VMS_ERR_NEG_JACOBIAN, VMS_ERR_NAN. */
int vms_residual(vms_ctx* ctx, double* norm, double* R);

/* Element-level outputs for elements [first, first+count), computed by the same kernels as the
 * assembly, written as FP64 to caller buffers (host or device; any may be NULL):
 *   S [count x 32 x 32], r [count x 32]              condensed matrix and residual (Section 5)
 *   Kcc [count x 32 x 32], Kcf [count x 32 x 3], Kfc [count x 3 x 32], Kff [count x 3 x 3],
 *   Rcp [count x 32], Rf [count x 3]                 tangent blocks and residuals (Section 4)
 * Row/column order is node-major (4a+c). Errors: VMS_ERR_INVALID_ARG (range), VMS_ERR_STATE. */
int vms_element_matrices(vms_ctx* ctx, int64_t first, int64_t count, double* S, double* r,
                         double* Kcc, double* Kcf, double* Kfc, double* Kff, double* Rcp,
                         double* Rf);

/* y = S x with the last assembled (Dirichlet-applied) CSR matrix; x, y device doubles of length
 * 4*n_nodes. Errors: VMS_ERR_STATE (nothing assembled), VMS_ERR_INVALID_ARG. */
int vms_apply(vms_ctx* ctx, const double* x, double* y);

/* ---- batches of independent problems (serving-style mixes) --------------------------------- */

/* Per-element kinematic viscosity nu_e (n_elems doubles, host or device; copied), replacing
 * params.nu element by element (weak-form coefficient visc_factor * nu_e): a batch of problems
 * with different Reynolds numbers assembled as one mesh in one launch. NULL restores params.nu.
 * Cleared by vms_mesh_upload. Errors: VMS_ERR_STATE (no mesh), VMS_ERR_INVALID_ARG (nu_e <= 0 or
 * not finite). */
int vms_set_element_viscosity(vms_ctx* ctx, const double* nu_e);

/* Declare the uploaded mesh a batch of `count` independent problems: instance i owns nodes
 * [node_offsets[i], node_offsets[i+1]) and elements [elem_offsets[i], elem_offsets[i+1]) (host
 * arrays of count + 1 entries, starting at 0 and ending at n_nodes and n_elems). Every element of
 * an instance must reference only nodes of that instance (checked), so each instance's rows form
 * a diagonal block of the condensed matrix. Cleared by vms_mesh_upload.
 * Errors: VMS_ERR_STATE (no mesh), VMS_ERR_INVALID_ARG. */
int vms_set_instances(vms_ctx* ctx, int64_t count, const int64_t* node_offsets,
                      const int64_t* elem_offsets);

/* vms_solve restricted to instance `instance` (vms_set_instances): GMRES on its diagonal block of
 * the last assembled system, then recovery of its bubble increments and, if update != 0, update of
 * its part of the state only (the other instances keep theirs and their assembled blocks stay
 * valid). The preconditioner is set up once per assembly for all instances. Same arguments,
 * results and errors as vms_solve, plus VMS_ERR_INVALID_ARG for an unknown instance and
 * VMS_ERR_STATE for an instance updated since the last assembly (vms_solve also returns
 * VMS_ERR_STATE while any instance is). */
int vms_solve_instance(vms_ctx* ctx, int64_t instance, double rtol, int maxit, int restart,
                       int update, int* iters, double* rel);

/* Kernel schedules of a mixed-precision assembly with the atomic scatter (vms_tuning.schedule). */
#define VMS_SCHEDULE_FUSED 0        /* one persistent launch: FP64 residual warps and FP32 tangent
                                       warps share every SM (default) */
#define VMS_SCHEDULE_TWO_STREAMS 1  /* residual and tangent kernels launched on two streams */

/* Launch shapes, kernel schedule and scatter order of the assembly kernels. */
typedef struct vms_tuning {
  int32_t tangent_warps;    /* warps (elements) per tangent block: FP32 2, 4 or 8, FP64 1, 2 or 4; 0 = default (4 / 2) */
  int32_t residual_threads; /* threads (elements) per residual block: 32 or 64; 0 = default (64) */
  int32_t scatter_mode;     /* VMS_SCATTER_*, or -1 for params.scatter_mode */
  int32_t schedule;         /* VMS_SCHEDULE_*: used in VMS_PREC_MIXED with the atomic scatter (the
                               fused kernel takes no block shape); the other cases run two kernels */
  double ms;                /* vms_autotune: median milliseconds of one assembly with these settings */
} vms_tuning;

/* Set or read the tuning of the context (defaults: {0, 0, -1, VMS_SCHEDULE_FUSED}). Results do not
 * depend on it except for the summation order of the atomic scatter. Errors: VMS_ERR_INVALID_ARG
 * (value not offered). */
int vms_set_tuning(vms_ctx* ctx, const vms_tuning* tuning);
int vms_get_tuning(vms_ctx* ctx, vms_tuning* tuning);

/* Autotuner: time `repeats` assemblies (CUDA events on the context's stream, after one warm-up)
 * of the current mesh and state for every offered tuning (in VMS_PREC_MIXED the fused schedule,
 * and every combination of tangent warps per block, residual threads per block and scatter mode
 * with two kernels), keep the fastest (median) as the context's tuning and return it in *best
 * (may be NULL). The assembled system is discarded (assemble again).
 * Errors: VMS_ERR_STATE (no state), those of vms_assemble_newton_schur. */
int vms_autotune(vms_ctx* ctx, int repeats, vms_tuning* best);

/* Record the kernels of one vms_assemble_newton_schur into a CUDA graph on first use and replay
 * the graph afterwards (enable != 0); recaptured after vms_mesh_upload, vms_set_params,
 * vms_set_element_viscosity or vms_set_tuning. Not used while kernel timing is enabled
 * (vms_profile_enable). Results are those of the same calls without the graph. */
int vms_set_graph(vms_ctx* ctx, int enable);

/* Choose the right preconditioner of vms_solve / vms_solve_instance / vms_newton_*:
 * VMS_PRECOND_ILU0 (default), VMS_PRECOND_BLOCK_JACOBI, or VMS_PRECOND_ILU0_FALLBACK (ILU(0), and
 * for a solve that does not converge, a direct solve of the instance by LU with partial pivoting
 * in band storage, FP64, on the device; the nodes are taken in the order of smallest bandwidth
 * among their own order and two reverse Cuthill-McKee orders, the band's half-width is 4 (that
 * order's largest distance of two coupled nodes) + 3, and where the band would need more than
 * 48 GiB a second solve from zero with
 * block Jacobi and the longest cycle instead. On coarse high-Reynolds systems the ILU(0) pivots
 * lose all size. Where the direct solve fits, the ILU(0) attempt also ends before maxit: after a
 * cycle whose rate would not reach rtol by maxit, or once it has run as long as the direct solve
 * is estimated to take, so which of the two solves a system depends on timing; either meets
 * rtol. *iters counts the Krylov iterations of both attempts, *relres is that of the last. The
 * direct solve's temporary band is allocated and freed within the call: VMS_ERR_OUT_OF_MEMORY
 * falls through to block Jacobi, VMS_ERR_ZERO_PIVOT reports a singular band). Section 6 solved every Newton system with a Krylov solver at its
 * library defaults; on one process that default preconditioner is an incomplete LU factorisation
 * without fill, which VMS_PRECOND_ILU0 computes on 4x4 node blocks (it is refactored at every
 * solve of a newly assembled system). ILU(0) needs at most 32 neighbours per node
 * (VMS_ERR_UNSUPPORTED otherwise). Errors: VMS_ERR_INVALID_ARG. */
int vms_set_preconditioner(vms_ctx* ctx, int kind);

/* Limit of every device-side wait of the ILU(0) factorisation and sweeps (a row waiting for a row
 * it depends on): after `polls` polls (about 32 ns apart) the kernel records a timeout and stops
 * its remaining work, and the solve returns VMS_ERR_TIMEOUT with the state unchanged; the context
 * stays usable. polls = 0 restores the default (2^22, about 0.13 s). A limit too small for the
 * rows' normal hand-over times makes every ILU(0) solve time out. Not part of the paper's method:
 * failure detection of the GPU solver. Errors: VMS_ERR_INVALID_ARG (polls < 0 or > 2^30). */
int vms_set_wait_limit(vms_ctx* ctx, int64_t polls);

/* Solve S du = -r with the last assembled system by restarted GMRES(restart), right-preconditioned
 * (vms_set_preconditioner; restart <= 480), FP32 inner iterations and FP64 iterative refinement in
 * VMS_PREC_MIXED (a refinement pass that does not halve the FP64 residual hands the remaining
 * correction to GMRES with FP64 vectors, the FP32 matrix and the FP64 preconditioner, keeping its
 * preconditioned vectors), FP64 throughout
 * in VMS_PREC_FP64, to relative residual rtol within maxit iterations in all (the paper
 * used a Krylov solver with tolerance 1e-12 and 50 iterations, Section 6). Then recovers the bubble
 * increments du' = K_ff^-1 (-R_f - K_fc du_e) per element (Section 5) and, if update != 0, adds
 * du and du' to the state. *iters (may be NULL) receives the Krylov iterations, *rel the final
 * relative residual. Errors: VMS_ERR_STATE, VMS_ERR_KRYLOV_MAXIT (state left unchanged),
 * VMS_ERR_ZERO_PIVOT, VMS_ERR_TIMEOUT (ILU(0) only; the state is left unchanged), VMS_ERR_NAN
 * (non-finite right-hand side). */
int vms_solve(vms_ctx* ctx, double rtol, int maxit, int restart, int update, int* iters,
              double* rel);

/* One Newton-Schur iteration (Sections 4.2 and 5): assemble, solve (GMRES(150) to 1e-10 relative,
 * the cycle doubled up to 480 whenever one does not halve the residual, at most 3000 iterations;
 * a solve that stops above 1e-10 but below 0.1 is still applied),
 * recover, update. *res_norm receives the FP64 residual norm before the update. */
int vms_newton_step(vms_ctx* ctx, double* res_norm);

/* Newton-Schur iteration until ||R|| <= rtol ||R^0|| or maxit iterations; hist (may be NULL,
 * maxit+1 doubles, host) receives the residual norms, *iters the iterations taken. Inexact
 * Newton: each linear solve (GMRES(150), the cycle doubled up to 480 whenever one does not halve
 * the residual, at most 3000 iterations) stops at the relative residual eta, capped at 0.5 and
 * at least rtol ||R^0|| / (2 ||R||): Eisenstat and Walker's choice 2 (eta_0 = 0.05,
 * eta_k = 0.5 (||R^k|| / ||R^{k-1}||)^2, or 0.5 eta_{k-1}^2 when that exceeds 0.1), in mixed mode
 * only while ||R|| > 1e-3 ||R^0|| and min(1e-2, 0.1 ||R|| / ||R^0||) after. A solve that stops
 * above eta but below 0.1 is still applied.
 * Errors: VMS_ERR_NEWTON_DIVERGED, VMS_ERR_KRYLOV_MAXIT and those of the steps. */
int vms_newton_solve(vms_ctx* ctx, double rtol, int maxit, int* iters, double* hist);

/* vms_newton_solve with an absolute target: iterate until ||R|| <= target (the same stopping
 * rule whatever the starting point, e.g. a predicted one; the forcing term uses the ratio to the
 * starting residual and is floored at target / (2 ||R||)). */
int vms_newton_solve_to(vms_ctx* ctx, double target, int maxit, int* iters, double* hist);

/* ---- learned warm start of the transient Newton iteration -------------------------------------
 * Remark of Section 4.1 (backward-Euler steps) and Section 4.2 (Newton): a network predicts, for
 * every node, the increment of (v, p) over the next time step from its state at the last two
 * steps and the mean of its 1-ring, and Newton starts from the predicted state instead of the
 * previous one. Newton still converges to the same tolerance, so the network only moves the
 * starting point (the previous-step start is the fallback). The paper has no counterpart; it is
 * an extension of the transient solver.
 *
 * Network: x (12) -> tanh(x W1 + b1) (128) -> tanh(. W2 + b2) (128) -> . W3 + b3 (4); weights
 * stored in BF16, biases, activations and accumulation in FP32. Parameter vector (FP32, row-major):
 * W1 [12][128], b1 [128], W2 [128][128], b2 [128], W3 [128][4], b3 [4]. */
#define VMS_MLP_IN 12
#define VMS_MLP_WIDTH 128
#define VMS_MLP_OUT 4
#define VMS_MLP_PARAMS 18692

typedef struct vms_mlp vms_mlp;

/* Create a network on `device` with all parameters zero. Errors: VMS_ERR_CUDA, OUT_OF_MEMORY. */
int vms_mlp_create(vms_mlp** mlp, int device);
int vms_mlp_destroy(vms_mlp* mlp);
const char* vms_mlp_last_error(vms_mlp* mlp);
/* Stream of every later call on this network (default: the legacy default stream). */
int vms_mlp_set_stream(vms_mlp* mlp, void* stream);
/* Set all VMS_MLP_PARAMS parameters (FP32, host or device; the weights are rounded to BF16 for
 * use) and reset the optimiser. */
int vms_mlp_set_params(vms_mlp* mlp, const float* params);
/* Read the parameters: stored != 0 gives the values the kernels use (BF16 weights as FP32),
 * stored == 0 the FP32 master copy the optimiser updates. */
int vms_mlp_get_params(vms_mlp* mlp, float* params, int stored);
/* Y (n x 4, device FP32) = network(X) for X (n x 12, device FP32), queued on the stream. */
int vms_mlp_forward(vms_mlp* mlp, int64_t n, const float* X, float* Y);
/* Gradient of the loss sum_r sum_c (y_rc - T_rc)^2 / (4 n) over n rows (rows: device int32
 * indices into X and T, or NULL for the first n rows); kept for vms_mlp_adam. *loss (host, may be
 * NULL) and grads (VMS_MLP_PARAMS, host or device, may be NULL) receive the loss and gradient
 * (synchronises the stream when either is given). */
int vms_mlp_grad(vms_mlp* mlp, int64_t n, const int32_t* rows, const float* X, const float* T,
                 double* loss, float* grads);
/* One Adam step (beta1 0.9, beta2 0.999, eps 1e-8, learning rate lr) with the kept gradient. */
int vms_mlp_adam(vms_mlp* mlp, float lr);
/* Training-data scaling (the inputs and targets are brought to unit RMS per column before
 * training): rms (host, cols doubles) = sqrt(mean over the n rows of X[r][c]^2) for X (device
 * FP32, n x cols, 1 <= cols <= 16), summed in FP64; synchronises the stream. Errors:
 * VMS_ERR_INVALID_ARG. */
int vms_mlp_column_rms(vms_mlp* mlp, int64_t n, int cols, const float* X, double* rms);
/* out[r][c] = X[r][c] * mul[c] for X, out device FP32 n x cols (out may be X), mul cols host floats
 * (1 <= cols <= 16), queued on the stream. Errors: VMS_ERR_INVALID_ARG. */
int vms_mlp_scale_columns(vms_mlp* mlp, int64_t n, int cols, const float* X, const float* mul,
                          float* out);

/* Features of every node from the context's state u (step n) and u_prev (step n-1), with
 * d = u - u_prev: X[i] = [u_i (4), d_i (4), mean of d over the nodes sharing an element with i (4)]
 * divided column-wise by scale_in (12 host floats, NULL = 1); X: n_nodes x 12 device FP32. */
int vms_node_features(vms_ctx* ctx, const float* scale_in, float* X);
/* D[i] = (u_i - u_prev_i) / scale_out (4 host floats, NULL = 1), n_nodes x 4 device FP32. */
int vms_node_increment(vms_ctx* ctx, const float* scale_out, float* D);
/* u_i += scale_out * D[i] (D device FP32, n_nodes x 4), then the Dirichlet values are imposed. */
int vms_apply_increment(vms_ctx* ctx, const float* scale_out, const float* D);
/* Start a new backward-Euler step: u_prev = u (on the device). */
int vms_shift_time(vms_ctx* ctx);

/* ---- kernel accounting (tracing) ----------------------------------------------------------- */
#define VMS_K_RESIDUAL 0  /* element residual kernel (FP64) */
#define VMS_K_TANGENT 1   /* element tangent + condensation + scatter kernel */
#define VMS_K_FILL 2      /* zero fills */
#define VMS_K_DIRICHLET 3 /* Dirichlet diagonal / state imposition */
#define VMS_K_REDUCE 4    /* norms and dot products */
#define VMS_K_SPMV 5      /* CSR matrix-vector products */
#define VMS_K_KRYLOV 6    /* other Krylov / recovery / update kernels */
#define VMS_K_PRECOND 7   /* preconditioner set-up and application (ILU(0) factor and sweeps) */
#define VMS_K_FUSED 8     /* fused residual + tangent kernel (VMS_SCHEDULE_FUSED) */
#define VMS_K_COUNT 9

/* Count every kernel launch of the context (always on) and, if `timing` != 0, bracket each launch
 * with CUDA events on the context's stream to accumulate its GPU time per kernel kind. */
int vms_profile_enable(vms_ctx* ctx, int timing);

/* Read the accumulated GPU milliseconds (ms, VMS_K_COUNT doubles, may be NULL; only filled while
 * timing is enabled) and launch counts (launches, VMS_K_COUNT int64, may be NULL) since the last
 * reset; synchronises the stream. If reset != 0 the counters are cleared after reading. */
int vms_profile_read(vms_ctx* ctx, int reset, double* ms, int64_t* launches);

/* Linear solves (vms_solve and those of the Newton drivers) and their Krylov iterations since the
 * last reset (either pointer may be NULL). Errors: VMS_ERR_INVALID_ARG. */
int vms_solver_stats(vms_ctx* ctx, int reset, int64_t* solves, int64_t* krylov_iterations);

/* ---- residual norm with caller-owned memory only ------------------------------------------
 * The paper has no counterpart to this call. It serves callers that cannot allocate device
 * memory: processes that hand all device memory to their own pool at start-up (a framework's
 * caching allocator, a fixed arena), and latency-critical loops that cannot afford the
 * device-wide synchronisation cudaMalloc and cudaFree imply. It computes the same FP64 norm as
 * vms_residual (R_c, R_p on free dofs and every element's R_f) without a context and without
 * allocating: its scratch space is one fixed device array of VMS_NOALLOC_SCRATCH_BYTES that every
 * GPU loading this library holds until the process exits.
 *   xyz [n_nodes x 3], conn [n_elems x 8] (int32), dir_dof [n_dir] (int64), u [n_nodes x 4],
 *   beta [n_elems x 3] (NULL = zero), u_prev [n_nodes x 4] (NULL = u; read only when dt > 0):
 *   device pointers on the current device, row-major, owned by the caller.
 *   params: host pointer (nu, visc_factor, dt, f, bubble_scale, quad_order; scatter_mode unused).
 *   norm (1 double) and status (1 int32): device pointers that receive the norm and VMS_OK,
 *   VMS_ERR_NEG_JACOBIAN, VMS_ERR_NAN or VMS_ERR_INVALID_ARG (a node or dof index outside the
 *   mesh; such entries are skipped).
 * The work is queued on `stream` (a cudaStream_t, NULL = legacy default stream) and the call
 * returns without waiting; *norm and *status are valid once the stream reaches that point.
 * Returns VMS_OK, VMS_ERR_INVALID_ARG (null pointer, bad parameters), VMS_ERR_TOO_LARGE
 * (4*n_nodes + 3*n_elems > VMS_NOALLOC_MAX_ENTRIES; nothing is queued) or VMS_ERR_CUDA.
 * The first call on a device looks up the scratch array's device address (cudaGetSymbolAddress)
 * with that device current and keeps it for the life of the process; make that first call before
 * any stream capture, and do not call it again on a device after a cudaDeviceReset of that device
 * (the kept address would be stale). Every call shares
 * the one array and clears what it needs at its start, so calls whose GPU work overlaps (other
 * streams, other host threads) race on it: order them on one stream or serialise them. */
#define VMS_ERR_TOO_LARGE -11
#define VMS_NOALLOC_MAX_ENTRIES 2097152
#define VMS_NOALLOC_SCRATCH_BYTES ((VMS_NOALLOC_MAX_ENTRIES + 4096) * 8)
int vms_residual_norm_noalloc(int64_t n_nodes, const double* xyz, int64_t n_elems,
                              const int32_t* conn, int64_t n_dir, const int64_t* dir_dof,
                              const double* u, const double* beta, const double* u_prev,
                              const vms_params* params, double* norm, int32_t* status,
                              void* stream);

/* Arithmetic throughput of the current GPU (no context needed): a kernel of independent fused
 * multiply-add chains, sized to a multiple of the SM count, timed with CUDA events on `device`.
 *   kind 0: FP64 FMA,  1: FP32 FMA,  2: packed FP32 FMA (two lanes per instruction)
 * *tflops receives the measured TFLOP/s (2 flops per FMA), the denominator of the element kernels'
 * rooflines. Not part of the paper's method. Errors: VMS_ERR_INVALID_ARG, VMS_ERR_CUDA. */
int vms_fma_throughput(int device, int kind, double* tflops);

/* Message of the last error on this context ("" if none); valid until the next call. */
const char* vms_last_error(vms_ctx* ctx);

/* Library version string. */
const char* vms_version(void);

#ifdef __cplusplus
}
#endif

#endif /* VMS_GB300_H */
