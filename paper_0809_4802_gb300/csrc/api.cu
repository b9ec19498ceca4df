// C-ABI of libvms_gb300 (declared in include/vms.h): context, mesh and state upload, the
// Newton-Schur assembly, residual evaluation and element-level outputs.
#include <algorithm>
#include <cmath>
#include <cstring>
#include <string>
#include <vector>

#include "vms_internal.h"
#include "solver.h"

using namespace vms;

struct vms_ctx {
  int device = 0;
  int precision = VMS_PREC_FP64;
  int precond = VMS_PRECOND_ILU0;
  cudaStream_t stream = nullptr;
  vms_params params{};
  int nq = 27;
  QpRow* d_qp = nullptr;     // nq rows (residual kernel)
  double* d_tab64 = nullptr; // 37 nq (tangent kernel, FP64)
  double* d_tsbasis = nullptr;   // FP64 tangent factorised sums: basis rows (quad_order 2, 3)
  uint32_t* d_tsplan = nullptr;  // and their plan
  float* d_tab32 = nullptr;  // 37 nq (tangent kernel, FP32)
  vms::TetMoments tet_mom{};  // reference moments of the tetrahedral rule (kernel parameter)
  Mesh mesh;
  State state;
  Work work;
  SolverWork solver;
  unsigned int* h_flags = nullptr;  // pinned
  double* h_scalar = nullptr;       // pinned, 8 entries
  double* d_scalar = nullptr;       // 8 entries
  std::string err;
  // kernel accounting
  bool timing = false;
  int64_t launches[VMS_K_COUNT] = {};
  int64_t solver_stats[2] = {};  // linear solves, Krylov iterations
  double ms[VMS_K_COUNT] = {};
  struct Ev { int kind; cudaEvent_t a, b; };
  std::vector<Ev> events;
  std::vector<cudaEvent_t> pool;
  // independent problems in one mesh (vms_set_instances): offsets, count + 1 entries each
  std::vector<int64_t> inst_nodes, inst_elems;
  std::vector<uint8_t> inst_stale;  // instance updated since the last assembly
  bool any_stale = false;
  vms_tuning tune{0, 0, -1, VMS_SCHEDULE_FUSED, 0.0};  // launch shapes, schedule, scatter (vms_set_tuning)
  // CUDA graph of one assembly (vms_set_graph)
  bool use_graph = false;
  bool graph_dirty = true;
  cudaStream_t cap_stream = nullptr;
  cudaGraphExec_t graph = nullptr;
  int64_t graph_launches[VMS_K_COUNT] = {};
  // vms_csr_download_async: the copy stream, the buffer a pending copy reads, the second values
  // buffer the next assembly writes meanwhile, and (graph mode) a device snapshot
  struct Stage {
    void* values = nullptr;      // snapshot of the values (graph mode: the captured buffer is fixed)
    double* rhs = nullptr;       // snapshot of the right-hand side
    size_t vbytes = 0, rbytes = 0;
    void* src = nullptr;         // values buffer the pending copy reads (no snapshot)
    void* alt = nullptr;         // the other values buffer (as large as work.values)
    cudaStream_t copy = nullptr;
    cudaEvent_t snap = nullptr, done = nullptr;
    bool pending = false;
  } stage;
};

namespace vms {

static cudaEvent_t take_event(vms_ctx* c) {
  if (!c->pool.empty()) {
    cudaEvent_t e = c->pool.back();
    c->pool.pop_back();
    return e;
  }
  cudaEvent_t e = nullptr;
  cudaEventCreate(&e);
  return e;
}

KScope::KScope(vms_ctx* ctx, int k) : KScope(ctx, k, ctx->stream) {}

KScope::KScope(vms_ctx* ctx, int k, cudaStream_t stream) : c(ctx), kind(k), s(stream) {
  if (c->timing) {
    a = take_event(c);
    cudaEventRecord(a, s);
  }
}

KScope::~KScope() {
  c->launches[kind] += n;
  if (a) {
    cudaEvent_t b = take_event(c);
    cudaEventRecord(b, s);
    c->events.push_back({kind, a, b});
  }
}

}  // namespace vms

namespace {

int fail(vms_ctx* c, int code, const std::string& msg) {
  if (c) c->err = msg;
  return code;
}

#define CK(call)                                                                           \
  do {                                                                                     \
    cudaError_t e_ = (call);                                                               \
    if (e_ != cudaSuccess)                                                                 \
      return fail(ctx, e_ == cudaErrorMemoryAllocation ? VMS_ERR_OUT_OF_MEMORY : VMS_ERR_CUDA, \
                  std::string(#call) + ": " + cudaGetErrorString(e_));                     \
  } while (0)

template <typename P>
void dfree(P*& p) {
  if (p) cudaFree((void*)p);
  p = nullptr;
}

// Waits for a pending vms_csr_download_async (its copy reads the mesh pattern and the snapshot).
int stage_wait(vms_ctx* c) {
  if (!c->stage.pending) return VMS_OK;
  c->stage.pending = false;
  const cudaError_t e = cudaEventSynchronize(c->stage.done);
  if (e != cudaSuccess) {
    c->err = cudaGetErrorString(e);
    return VMS_ERR_CUDA;
  }
  return VMS_OK;
}

void stage_free(vms_ctx* c) {
  stage_wait(c);
  auto& S = c->stage;
  dfree(S.values); dfree(S.rhs); dfree(S.alt);
  if (S.copy) cudaStreamDestroy(S.copy);
  if (S.snap) cudaEventDestroy(S.snap);
  if (S.done) cudaEventDestroy(S.done);
  S = vms_ctx::Stage();
}

void free_mesh(vms_ctx* c) {
  stage_free(c);
  Mesh& m = c->mesh;
  dfree(m.xyz); dfree(m.conn); dfree(m.rowptr); dfree(m.colidx); dfree(m.blk); dfree(m.rowlen);
  dfree(m.dir_mask); dfree(m.dir_dof); dfree(m.dir_val); dfree(m.diag_pos); dfree(m.colour_order);
  dfree(m.nu_e);
  m = Mesh();
  c->inst_nodes.clear();
  c->inst_elems.clear();
  c->inst_stale.clear();
  c->any_stale = false;
  c->graph_dirty = true;
  State& s = c->state;
  dfree(s.u); dfree(s.u_prev); dfree(s.beta);
  s = State();
  Work& w = c->work;
  dfree(w.values); dfree(w.rhs); dfree(w.elemR); dfree(w.recX); dfree(w.recKcf); dfree(w.recKinv);
  dfree(w.recY); dfree(w.resid); dfree(w.partial); dfree(w.flags); dfree(w.queues);
  dfree(w.f32.u); dfree(w.f32.beta); dfree(w.f32.xhl);
  cudaStream_t aux = w.aux;
  cudaEvent_t fork = w.fork, join = w.join;
  w = Work();
  w.aux = aux; w.fork = fork; w.join = join;
  free_solver(c->solver);
}

// FP32 tangent and CSR values (every mode but FP64)
bool fp32_mode(const vms_ctx* c) { return c->precision != VMS_PREC_FP64; }

// contractions of the FP32 tangent: 0 CUDA cores, TC_BF16 or TC_TF32X3 tensor cores
int engine(const vms_ctx* c) {
  return c->precision == VMS_PREC_MIXED_TC_BF16 ? 1 : (c->precision == VMS_PREC_MIXED_TC_TF32 ? 2 : 0);
}

KParams kparams(const vms_ctx* c) {
  KParams k{};
  k.nut = c->params.visc_factor * c->params.nu;
  k.tau = c->params.dt > 0 ? 1.0 / c->params.dt : 0.0;
  for (int i = 0; i < 3; ++i) k.f[i] = c->params.f[i];
  k.nq = c->nq;
  k.transient = c->params.dt > 0 ? 1 : 0;
  k.has_force = (k.f[0] != 0.0 || k.f[1] != 0.0 || k.f[2] != 0.0) ? 1 : 0;
  k.nu_e = c->mesh.nu_e;
  k.visc_factor = c->params.visc_factor;
  k.tab64 = c->d_tab64;
  k.tangent_warps = c->tune.tangent_warps;
  k.residual_threads = c->tune.residual_threads;
  k.ts_basis = c->d_tsbasis;
  k.ts_plan = c->d_tsplan;
  return k;
}

// Gauss-Legendre points (ascending) and weights on [-1, 1].
void gauss1d(int n, double* x, double* w) {
  if (n == 2) {
    const double a = 1.0 / std::sqrt(3.0);
    x[0] = -a; x[1] = a; w[0] = w[1] = 1.0;
  } else if (n == 3) {
    const double a = std::sqrt(0.6);
    x[0] = -a; x[1] = 0.0; x[2] = a;
    w[0] = 5.0 / 9.0; w[1] = 8.0 / 9.0; w[2] = 5.0 / 9.0;
  } else {
    const double r = 2.0 / 7.0 * std::sqrt(6.0 / 5.0);
    const double a = std::sqrt(3.0 / 7.0 - r), b = std::sqrt(3.0 / 7.0 + r);
    const double wa = (18.0 + std::sqrt(30.0)) / 36.0, wb = (18.0 - std::sqrt(30.0)) / 36.0;
    x[0] = -b; x[1] = -a; x[2] = a; x[3] = b;
    w[0] = wb; w[1] = wa; w[2] = wa; w[3] = wb;
  }
}

const int CORNER[8][3] = {{-1, -1, -1}, {1, -1, -1}, {1, 1, -1}, {-1, 1, -1},
                          {-1, -1, 1},  {1, -1, 1},  {1, 1, 1},  {-1, 1, 1}};

int upload_tables(vms_ctx* ctx) {
  const int n1 = ctx->params.quad_order;
  const int nq = n1 * n1 * n1;
  double x[4], w[4];
  gauss1d(n1, x, w);
  std::vector<QpRow> rows(nq);
  std::vector<double> t64(37 * nq);
  const double bs = ctx->params.bubble_scale;
  for (int k = 0; k < n1; ++k)
    for (int j = 0; j < n1; ++j)
      for (int i = 0; i < n1; ++i) {
        const int q = (k * n1 + j) * n1 + i;
        const double p[3] = {x[i], x[j], x[k]};
        QpRow& r = rows[q];
        r.xi = p[0]; r.eta = p[1]; r.zeta = p[2];
        r.xe = p[0] * p[1]; r.xz = p[0] * p[2]; r.ez = p[1] * p[2]; r.xez = p[0] * p[1] * p[2];
        const double f0 = 1 - p[0] * p[0], f1 = 1 - p[1] * p[1], f2 = 1 - p[2] * p[2];
        r.b = bs * f0 * f1 * f2;
        r.db0 = bs * (-2 * p[0]) * f1 * f2;
        r.db1 = bs * (-2 * p[1]) * f0 * f2;
        r.db2 = bs * (-2 * p[2]) * f0 * f1;
        r.w = w[i] * w[j] * w[k];
        for (int a = 0; a < 8; ++a) {
          double fac[3];
          for (int d = 0; d < 3; ++d) fac[d] = 1.0 + CORNER[a][d] * p[d];
          t64[8 * q + a] = fac[0] * fac[1] * fac[2] / 8.0;
          t64[8 * nq + 24 * q + 3 * a + 0] = CORNER[a][0] * fac[1] * fac[2] / 8.0;
          t64[8 * nq + 24 * q + 3 * a + 1] = CORNER[a][1] * fac[0] * fac[2] / 8.0;
          t64[8 * nq + 24 * q + 3 * a + 2] = CORNER[a][2] * fac[0] * fac[1] / 8.0;
        }
        t64[32 * nq + q] = r.b;
        t64[33 * nq + 3 * q + 0] = r.db0;
        t64[33 * nq + 3 * q + 1] = r.db1;
        t64[33 * nq + 3 * q + 2] = r.db2;
        t64[36 * nq + q] = r.w;
      }
  std::vector<float> t32(t64.begin(), t64.end());
  dfree(ctx->d_qp); dfree(ctx->d_tab64); dfree(ctx->d_tab32); dfree(ctx->d_tsbasis); dfree(ctx->d_tsplan);
  std::vector<double> tsb;
  std::vector<uint32_t> tsp;
  if ((n1 == 2 || n1 == 3) && ts_tables(n1, x, tsb, tsp)) {
    CK(cudaMalloc(&ctx->d_tsbasis, sizeof(double) * tsb.size()));
    CK(cudaMalloc(&ctx->d_tsplan, sizeof(uint32_t) * tsp.size()));
    CK(cudaMemcpy(ctx->d_tsbasis, tsb.data(), sizeof(double) * tsb.size(), cudaMemcpyHostToDevice));
    CK(cudaMemcpy(ctx->d_tsplan, tsp.data(), sizeof(uint32_t) * tsp.size(), cudaMemcpyHostToDevice));
  }
  CK(cudaMalloc(&ctx->d_qp, sizeof(QpRow) * nq));
  CK(cudaMalloc(&ctx->d_tab64, sizeof(double) * 37 * nq));
  CK(cudaMalloc(&ctx->d_tab32, sizeof(float) * 37 * nq));
  CK(cudaMemcpy(ctx->d_qp, rows.data(), sizeof(QpRow) * nq, cudaMemcpyHostToDevice));
  CK(cudaMemcpy(ctx->d_tab64, t64.data(), sizeof(double) * 37 * nq, cudaMemcpyHostToDevice));
  CK(cudaMemcpy(ctx->d_tab32, t32.data(), sizeof(float) * 37 * nq, cudaMemcpyHostToDevice));
  ctx->nq = nq;
  tet_moments(n1, bs, ctx->tet_mom);
  return VMS_OK;
}

int check_flags(vms_ctx* ctx) {
  CK(cudaMemcpyAsync(ctx->h_flags, ctx->work.flags, sizeof(unsigned int), cudaMemcpyDeviceToHost,
                     ctx->stream));
  CK(cudaStreamSynchronize(ctx->stream));
  const unsigned f = *ctx->h_flags;
  if (f & FLAG_NEG_JACOBIAN) return fail(ctx, VMS_ERR_NEG_JACOBIAN, "det J <= 0 at a quadrature point");
  if (f & FLAG_SINGULAR_KFF) return fail(ctx, VMS_ERR_SINGULAR_KFF, "singular bubble block K_ff");
  if (f & FLAG_NAN) return fail(ctx, VMS_ERR_NAN, "non-finite residual");
  return VMS_OK;
}

template <typename T>
int upload(vms_ctx* ctx, T*& dst, const void* src, size_t count) {
  CK(cudaMalloc(&dst, sizeof(T) * (count ? count : 1)));
  if (count && src) CK(cudaMemcpy(dst, src, sizeof(T) * count, cudaMemcpyDefault));
  return VMS_OK;
}

#define TRY(x)                \
  do {                        \
    int r_ = (x);             \
    if (r_ != VMS_OK) return r_; \
  } while (0)

}  // namespace

namespace vms {
int ctx_flags_check(vms_ctx* ctx) { return check_flags(ctx); }
}

extern "C" {

const char* vms_version(void) { return "vms-gb300 0.1 (sm_103a)"; }

const char* vms_last_error(vms_ctx* ctx) { return ctx ? ctx->err.c_str() : "null context"; }

int vms_create(vms_ctx** out, int device, int precision) {
  if (!out) return VMS_ERR_INVALID_ARG;
  *out = nullptr;
  if (precision < VMS_PREC_FP64 || precision > VMS_PREC_MIXED_TC_TF32) return VMS_ERR_INVALID_ARG;
  int ndev = 0;
  if (cudaGetDeviceCount(&ndev) != cudaSuccess || device < 0 || device >= ndev)
    return VMS_ERR_CUDA;
  if (cudaSetDevice(device) != cudaSuccess) return VMS_ERR_CUDA;
  vms_ctx* ctx = new vms_ctx();
  ctx->device = device;
  ctx->precision = precision;
  ctx->params.nu = 0.01;
  ctx->params.visc_factor = 2.0;
  ctx->params.dt = 0.0;
  ctx->params.bubble_scale = 1.0;
  ctx->params.quad_order = 3;
  ctx->params.scatter_mode = VMS_SCATTER_ATOMIC;
  if (cudaStreamCreateWithFlags(&ctx->work.aux, cudaStreamNonBlocking) != cudaSuccess ||
      cudaEventCreateWithFlags(&ctx->work.fork, cudaEventDisableTiming) != cudaSuccess ||
      cudaEventCreateWithFlags(&ctx->work.join, cudaEventDisableTiming) != cudaSuccess ||
      cudaMallocHost(&ctx->h_flags, sizeof(unsigned int)) != cudaSuccess ||
      cudaMallocHost(&ctx->h_scalar, 8 * sizeof(double)) != cudaSuccess ||
      cudaMalloc(&ctx->d_scalar, 8 * sizeof(double)) != cudaSuccess ||
      upload_tables(ctx) != VMS_OK) {
    vms_destroy(ctx);
    return VMS_ERR_CUDA;
  }
  *out = ctx;
  return VMS_OK;
}

int vms_destroy(vms_ctx* ctx) {
  if (!ctx) return VMS_OK;
  cudaSetDevice(ctx->device);
  if (ctx->stream) cudaStreamSynchronize(ctx->stream);
  free_mesh(ctx);
  for (auto& e : ctx->events) { cudaEventDestroy(e.a); cudaEventDestroy(e.b); }
  for (auto e : ctx->pool) cudaEventDestroy(e);
  dfree(ctx->d_qp); dfree(ctx->d_tab64); dfree(ctx->d_tab32); dfree(ctx->d_scalar);
  dfree(ctx->d_tsbasis); dfree(ctx->d_tsplan);
  if (ctx->graph) cudaGraphExecDestroy(ctx->graph);
  if (ctx->cap_stream) cudaStreamDestroy(ctx->cap_stream);
  if (ctx->work.aux) { cudaStreamSynchronize(ctx->work.aux); cudaStreamDestroy(ctx->work.aux); }
  if (ctx->work.fork) cudaEventDestroy(ctx->work.fork);
  if (ctx->work.join) cudaEventDestroy(ctx->work.join);
  if (ctx->h_flags) cudaFreeHost(ctx->h_flags);
  if (ctx->h_scalar) cudaFreeHost(ctx->h_scalar);
  delete ctx;
  return VMS_OK;
}

int vms_set_stream(vms_ctx* ctx, void* stream) {
  if (!ctx) return VMS_ERR_INVALID_ARG;
  ctx->stream = reinterpret_cast<cudaStream_t>(stream);
  return VMS_OK;
}

int vms_set_preconditioner(vms_ctx* ctx, int kind) {
  if (!ctx) return VMS_ERR_INVALID_ARG;
  if (kind != VMS_PRECOND_ILU0 && kind != VMS_PRECOND_BLOCK_JACOBI && kind != VMS_PRECOND_ILU0_FALLBACK)
    return fail(ctx, VMS_ERR_INVALID_ARG, "unknown preconditioner");
  ctx->precond = kind;
  return VMS_OK;
}

int vms_set_params(vms_ctx* ctx, const vms_params* p) {
  if (!ctx || !p) return fail(ctx, VMS_ERR_INVALID_ARG, "null argument");
  if (!(p->nu > 0.0) || !(p->visc_factor > 0.0) || !(p->dt >= 0.0) || !(p->bubble_scale != 0.0) ||
      p->quad_order < 2 || p->quad_order > 4 ||
      (p->scatter_mode != VMS_SCATTER_ATOMIC && p->scatter_mode != VMS_SCATTER_COLOUR))
    return fail(ctx, VMS_ERR_INVALID_ARG, "invalid parameters");
  if (engine(ctx) != 0 && p->quad_order > 3)
    return fail(ctx, VMS_ERR_UNSUPPORTED, "the tensor-core tangent takes at most 27 points (quad_order <= 3)");
  CK(cudaSetDevice(ctx->device));
  CK(cudaStreamSynchronize(ctx->stream));
  const bool retab = p->quad_order != ctx->params.quad_order || p->bubble_scale != ctx->params.bubble_scale;
  ctx->params = *p;
  if (retab) TRY(upload_tables(ctx));
  ctx->work.assembled = false;
  ctx->graph_dirty = true;
  return VMS_OK;
}

int vms_set_element_viscosity(vms_ctx* ctx, const double* nu) {
  if (!ctx) return VMS_ERR_INVALID_ARG;
  const Mesh& m0 = ctx->mesh;
  if (!m0.n_elems) return fail(ctx, VMS_ERR_STATE, "no mesh uploaded");
  CK(cudaSetDevice(ctx->device));
  CK(cudaStreamSynchronize(ctx->stream));
  Mesh& m = ctx->mesh;
  ctx->graph_dirty = true;
  ctx->work.assembled = false;
  if (!nu) {
    dfree(m.nu_e);
    return VMS_OK;
  }
  std::vector<double> h(m.n_elems);
  CK(cudaMemcpy(h.data(), nu, sizeof(double) * m.n_elems, cudaMemcpyDefault));
  for (double v : h)
    if (!(v > 0.0) || !std::isfinite(v)) return fail(ctx, VMS_ERR_INVALID_ARG, "viscosity must be positive and finite");
  if (!m.nu_e) TRY(upload(ctx, m.nu_e, h.data(), m.n_elems));
  else CK(cudaMemcpy(m.nu_e, h.data(), sizeof(double) * m.n_elems, cudaMemcpyHostToDevice));
  return VMS_OK;
}

int vms_set_instances(vms_ctx* ctx, int64_t count, const int64_t* node_offsets,
                      const int64_t* elem_offsets) {
  if (!ctx) return VMS_ERR_INVALID_ARG;
  const Mesh& m = ctx->mesh;
  if (!m.n_elems) return fail(ctx, VMS_ERR_STATE, "no mesh uploaded");
  if (count < 1 || !node_offsets || !elem_offsets) return fail(ctx, VMS_ERR_INVALID_ARG, "invalid instance arguments");
  std::vector<int64_t> nodes(node_offsets, node_offsets + count + 1), elems(elem_offsets, elem_offsets + count + 1);
  if (nodes[0] != 0 || elems[0] != 0 || nodes[count] != m.n_nodes || elems[count] != m.n_elems)
    return fail(ctx, VMS_ERR_INVALID_ARG, "instance offsets must run from 0 to n_nodes and n_elems");
  for (int64_t i = 0; i < count; ++i)
    if (nodes[i + 1] <= nodes[i] || elems[i + 1] <= elems[i])
      return fail(ctx, VMS_ERR_INVALID_ARG, "instance offsets must increase");
  CK(cudaSetDevice(ctx->device));
  std::vector<int32_t> conn(8 * m.n_elems);
  CK(cudaMemcpy(conn.data(), m.conn, sizeof(int32_t) * conn.size(), cudaMemcpyDeviceToHost));
  for (int64_t i = 0; i < count; ++i)
    for (int64_t e = elems[i]; e < elems[i + 1]; ++e)
      for (int a = 0; a < 8; ++a) {
        const int64_t nd = conn[8 * e + a];
        if (nd < nodes[i] || nd >= nodes[i + 1])
          return fail(ctx, VMS_ERR_INVALID_ARG, "an element of an instance touches a node of another");
      }
  ctx->inst_nodes = std::move(nodes);
  ctx->inst_elems = std::move(elems);
  ctx->inst_stale.assign(count, 0);
  ctx->any_stale = false;
  return VMS_OK;
}

int vms_set_tuning(vms_ctx* ctx, const vms_tuning* t) {
  if (!ctx || !t) return fail(ctx, VMS_ERR_INVALID_ARG, "null argument");
  const bool f32 = fp32_mode(ctx);
  bool warps_ok = t->tangent_warps == 0;
  for (int k = 0; k < 3; ++k) warps_ok = warps_ok || t->tangent_warps == tangent_warp_choice(f32, k);
  if (!warps_ok || (t->residual_threads != 0 && t->residual_threads != 32 && t->residual_threads != 64) ||
      t->scatter_mode < -1 || t->scatter_mode > VMS_SCATTER_COLOUR ||
      (t->schedule != VMS_SCHEDULE_FUSED && t->schedule != VMS_SCHEDULE_TWO_STREAMS))
    return fail(ctx, VMS_ERR_INVALID_ARG, "invalid tuning");
  ctx->tune = *t;
  ctx->graph_dirty = true;
  return VMS_OK;
}

int vms_get_tuning(vms_ctx* ctx, vms_tuning* t) {
  if (!ctx || !t) return fail(ctx, VMS_ERR_INVALID_ARG, "null argument");
  *t = ctx->tune;
  return VMS_OK;
}

int vms_autotune(vms_ctx* ctx, int repeats, vms_tuning* best) {
  if (!ctx || repeats < 1) return fail(ctx, VMS_ERR_INVALID_ARG, "invalid arguments");
  if (!ctx->state.valid) return fail(ctx, VMS_ERR_STATE, "mesh and state must be uploaded first");
  CK(cudaSetDevice(ctx->device));
  const bool f32 = fp32_mode(ctx);
  cudaEvent_t a = nullptr, b = nullptr;
  CK(cudaEventCreate(&a));
  CK(cudaEventCreate(&b));
  vms_tuning win{0, 0, -1, VMS_SCHEDULE_FUSED, HUGE_VAL};
  std::vector<vms_tuning> cands;
  if (f32 && engine(ctx) == 0) cands.push_back(vms_tuning{0, 0, VMS_SCATTER_ATOMIC, VMS_SCHEDULE_FUSED, 0.0});
  for (int wk = 0; wk < 3; ++wk)
    for (int rt : {32, 64})
      for (int sm = VMS_SCATTER_ATOMIC; sm <= VMS_SCATTER_COLOUR; ++sm)
        cands.push_back(vms_tuning{tangent_warp_choice(f32, wk), rt, sm, VMS_SCHEDULE_TWO_STREAMS, 0.0});
  int rc = VMS_OK;
  for (const vms_tuning& cand : cands) {
    ctx->tune = cand;
    ctx->graph_dirty = true;
    if ((rc = vms_assemble_newton_schur(ctx, nullptr))) break;  // warm-up (and graph capture)
    std::vector<float> t(repeats);
    for (int r = 0; r < repeats && rc == VMS_OK; ++r) {
      cudaEventRecord(a, ctx->stream);
      rc = vms_assemble_newton_schur(ctx, nullptr);
      cudaEventRecord(b, ctx->stream);
      cudaEventSynchronize(b);
      cudaEventElapsedTime(&t[r], a, b);
    }
    if (rc) break;
    std::sort(t.begin(), t.end());
    const double med = t[repeats / 2];
    if (med < win.ms) { win = cand; win.ms = med; }
  }
  cudaEventDestroy(a);
  cudaEventDestroy(b);
  ctx->tune = rc == VMS_OK ? win : vms_tuning{0, 0, -1, VMS_SCHEDULE_FUSED, 0.0};
  ctx->graph_dirty = true;
  ctx->work.assembled = false;
  if (rc) return rc;
  if (best) *best = win;
  return VMS_OK;
}

int vms_set_graph(vms_ctx* ctx, int enable) {
  if (!ctx) return VMS_ERR_INVALID_ARG;
  ctx->use_graph = enable != 0;
  ctx->graph_dirty = true;
  return VMS_OK;
}

static int mesh_upload_impl(vms_ctx* ctx, int npe, int64_t n_nodes, const double* xyz,
                            int64_t n_elems, const int32_t* conn, int64_t n_dir,
                            const int64_t* dir_dof, const double* dir_val);

int vms_mesh_upload(vms_ctx* ctx, int64_t n_nodes, const double* xyz, int64_t n_elems,
                    const int32_t* conn, int64_t n_dir, const int64_t* dir_dof,
                    const double* dir_val) {
  return mesh_upload_impl(ctx, 8, n_nodes, xyz, n_elems, conn, n_dir, dir_dof, dir_val);
}

int vms_mesh_upload_tet(vms_ctx* ctx, int64_t n_nodes, const double* xyz, int64_t n_elems,
                        const int32_t* conn, int64_t n_dir, const int64_t* dir_dof,
                        const double* dir_val) {
  return mesh_upload_impl(ctx, 4, n_nodes, xyz, n_elems, conn, n_dir, dir_dof, dir_val);
}

static int mesh_upload_impl(vms_ctx* ctx, int npe, int64_t n_nodes, const double* xyz,
                            int64_t n_elems, const int32_t* conn, int64_t n_dir,
                            const int64_t* dir_dof, const double* dir_val) {
  if (!ctx) return VMS_ERR_INVALID_ARG;
  if (n_nodes <= 0 || n_elems <= 0 || !xyz || !conn || n_dir < 0 || (n_dir > 0 && (!dir_dof || !dir_val)))
    return fail(ctx, VMS_ERR_INVALID_ARG, "invalid mesh arguments");
  if (n_nodes >= (int64_t)1 << 29 || n_elems >= (int64_t)1 << 28)
    return fail(ctx, VMS_ERR_INVALID_ARG, "mesh too large for int32 indexing");
  CK(cudaSetDevice(ctx->device));
  CK(cudaStreamSynchronize(ctx->stream));
  free_mesh(ctx);
  // bring inputs to the host (they may be device pointers)
  std::vector<double> hx(3 * n_nodes);
  std::vector<int32_t> hc((size_t)npe * n_elems);
  std::vector<int64_t> hd(n_dir);
  std::vector<double> hv(n_dir);
  CK(cudaMemcpy(hx.data(), xyz, sizeof(double) * 3 * n_nodes, cudaMemcpyDefault));
  CK(cudaMemcpy(hc.data(), conn, sizeof(int32_t) * npe * n_elems, cudaMemcpyDefault));
  if (n_dir) {
    CK(cudaMemcpy(hd.data(), dir_dof, sizeof(int64_t) * n_dir, cudaMemcpyDefault));
    CK(cudaMemcpy(hv.data(), dir_val, sizeof(double) * n_dir, cudaMemcpyDefault));
  }
  HostPattern pat;
  const std::string perr = build_pattern(n_nodes, n_elems, hc.data(), n_dir, hd.data(), pat, npe);
  if (!perr.empty()) return fail(ctx, VMS_ERR_INVALID_ARG, perr);

  Mesh& m = ctx->mesh;
  m.n_nodes = n_nodes;
  m.n_elems = n_elems;
  m.npe = npe;
  m.nnz = pat.rowptr.back();
  m.n_dir = n_dir;
  std::vector<double4_32a> x4(n_nodes);
  for (int64_t i = 0; i < n_nodes; ++i) x4[i] = make_double4_32a(hx[3 * i], hx[3 * i + 1], hx[3 * i + 2], 0.0);
  TRY(upload(ctx, m.xyz, x4.data(), n_nodes));
  TRY(upload(ctx, m.conn, hc.data(), (size_t)npe * n_elems));
  TRY(upload(ctx, m.rowptr, pat.rowptr.data(), pat.rowptr.size()));
  TRY(upload(ctx, m.colidx, pat.colidx.data(), pat.colidx.size()));
  TRY(upload(ctx, m.blk, pat.blk.data(), pat.blk.size()));
  TRY(upload(ctx, m.rowlen, pat.rowlen.data(), pat.rowlen.size()));
  TRY(upload(ctx, m.dir_mask, pat.dir_mask.data(), pat.dir_mask.size()));
  TRY(upload(ctx, m.dir_dof, hd.data(), n_dir));
  TRY(upload(ctx, m.dir_val, hv.data(), n_dir));
  TRY(upload(ctx, m.diag_pos, pat.diag_pos.data(), n_dir));
  TRY(upload(ctx, m.colour_order, pat.colour_order.data(), pat.colour_order.size()));
  m.colour_start = pat.colour_start;
  m.n_colours = pat.n_colours;

  State& s = ctx->state;
  CK(cudaMalloc(&s.u, sizeof(double4_32a) * n_nodes));
  CK(cudaMalloc(&s.u_prev, sizeof(double4_32a) * n_nodes));
  CK(cudaMalloc(&s.beta, sizeof(double) * 3 * n_elems));
  Work& w = ctx->work;
  CK(cudaMalloc(&w.values, (size_t)m.nnz * sizeof(double)));
  CK(cudaMalloc(&w.rhs, sizeof(double) * 4 * n_nodes));
  CK(cudaMalloc(&w.elemR, sizeof(double) * 36 * n_elems));
  CK(cudaMalloc(&w.recX, sizeof(double) * 96 * n_elems));
  CK(cudaMalloc(&w.recKcf, sizeof(double) * 96 * n_elems));
  CK(cudaMalloc(&w.recKinv, sizeof(double) * 9 * n_elems));
  CK(cudaMalloc(&w.recY, sizeof(double) * 3 * n_elems));
  CK(cudaMalloc(&w.f32.u, sizeof(float4) * n_nodes));
  CK(cudaMalloc(&w.f32.beta, sizeof(float) * 3 * n_elems));
  CK(cudaMalloc(&w.f32.xhl, sizeof(float4) * 2 * n_nodes));
  CK(cudaGetLastError());
  CK(cudaMalloc(&w.resid, sizeof(double) * (4 * n_nodes + 3 * n_elems)));
  CK(cudaMalloc(&w.partial, sizeof(double) * 1024));
  CK(cudaMalloc(&w.flags, sizeof(unsigned int)));
  CK(cudaMalloc(&w.queues, 2 * sizeof(unsigned long long)));
  return VMS_OK;
}

int vms_state_upload(vms_ctx* ctx, const double* u, const double* beta, const double* u_prev) {
  if (!ctx) return VMS_ERR_INVALID_ARG;
  if (!ctx->mesh.n_nodes) return fail(ctx, VMS_ERR_STATE, "no mesh uploaded");
  if (!u) return fail(ctx, VMS_ERR_INVALID_ARG, "u is null");
  CK(cudaSetDevice(ctx->device));
  const Mesh& m = ctx->mesh;
  State& s = ctx->state;
  CK(cudaMemcpyAsync(s.u, u, sizeof(double4_32a) * m.n_nodes, cudaMemcpyDefault, ctx->stream));
  { KScope k(ctx, VMS_K_DIRICHLET); k.add(launch_impose(m, s.u, ctx->stream)); }
  if (beta) {
    CK(cudaMemcpyAsync(s.beta, beta, sizeof(double) * 3 * m.n_elems, cudaMemcpyDefault, ctx->stream));
  } else {
    KScope k(ctx, VMS_K_FILL);
    k.add(launch_fill_zero(s.beta, sizeof(double) * 3 * m.n_elems, ctx->stream));
  }
  CK(cudaMemcpyAsync(s.u_prev, u_prev ? u_prev : u, sizeof(double4_32a) * m.n_nodes, cudaMemcpyDefault,
                     ctx->stream));
  CK(cudaGetLastError());
  s.valid = true;
  ctx->work.assembled = false;
  return VMS_OK;
}

int vms_state_download(vms_ctx* ctx, double* u, double* beta) {
  if (!ctx) return VMS_ERR_INVALID_ARG;
  if (!ctx->state.valid) return fail(ctx, VMS_ERR_STATE, "no state uploaded");
  CK(cudaSetDevice(ctx->device));
  if (u) CK(cudaMemcpyAsync(u, ctx->state.u, sizeof(double4_32a) * ctx->mesh.n_nodes, cudaMemcpyDefault, ctx->stream));
  if (beta) CK(cudaMemcpyAsync(beta, ctx->state.beta, sizeof(double) * 3 * ctx->mesh.n_elems, cudaMemcpyDefault, ctx->stream));
  CK(cudaStreamSynchronize(ctx->stream));
  return VMS_OK;
}

int vms_state_download_prev(vms_ctx* ctx, double* u_prev) {
  if (!ctx || !u_prev) return fail(ctx, VMS_ERR_INVALID_ARG, "null argument");
  if (!ctx->state.valid) return fail(ctx, VMS_ERR_STATE, "no state uploaded");
  CK(cudaSetDevice(ctx->device));
  CK(cudaMemcpyAsync(u_prev, ctx->state.u_prev, sizeof(double4_32a) * ctx->mesh.n_nodes, cudaMemcpyDefault, ctx->stream));
  CK(cudaStreamSynchronize(ctx->stream));
  return VMS_OK;
}

static void fill_view(vms_ctx* ctx, vms_csr_view* out) {
  out->n_rows = 4 * ctx->mesh.n_nodes;
  out->nnz = ctx->mesh.nnz;
  out->rowptr = ctx->mesh.rowptr;
  out->colidx = ctx->mesh.colidx;
  out->values = ctx->work.values;
  out->rhs = ctx->work.rhs;
  out->values_dtype = fp32_mode(ctx) ? 1 : 0;
  out->n_colours = ctx->mesh.n_colours;
}

// Queue one assembly on `st` (no host synchronisation): fills, FP32 copies, the residual and the
// tangent on two streams, the finish kernel and the Dirichlet rows.
static int enqueue_assembly(vms_ctx* ctx, cudaStream_t st) {
  const Mesh& m = ctx->mesh;
  Work& w = ctx->work;
  const bool f32 = fp32_mode(ctx);
  const KParams kp = kparams(ctx);
  {
    KScope k(ctx, VMS_K_FILL, st);
    k.add(launch_fill_zero(w.values, (size_t)m.nnz * (f32 ? sizeof(float) : sizeof(double)), st));
    k.add(launch_fill_zero(w.rhs, sizeof(double) * 4 * m.n_nodes, st));
    k.add(launch_fill_zero(w.flags, sizeof(unsigned int), st));
  }
  if (m.npe == 4) {  // tetrahedra: one kernel does residual, tangent, condensation and scatter
    TangentOut o;
    o.values = w.values; o.rhs = w.rhs; o.recX = w.recX; o.recKcf = w.recKcf; o.recKinv = w.recKinv;
    o.recY = w.recY;
    const int scatter = ctx->tune.scatter_mode >= 0 ? ctx->tune.scatter_mode : ctx->params.scatter_mode;
    {
      KScope k(ctx, VMS_K_TANGENT, st);
      if (scatter == VMS_SCATTER_COLOUR) {
        for (int c = 0; c < m.n_colours; ++c) {
          const int64_t b = m.colour_start[c], n = m.colour_start[c + 1] - b;
          k.add(launch_tet_assembly(f32, m, ctx->state, kp, ctx->tet_mom, o, b, n,
                                    m.colour_order, false, false, w.flags, st));
        }
      } else {
        k.add(launch_tet_assembly(f32, m, ctx->state, kp, ctx->tet_mom, o, 0,
                                  m.n_elems, nullptr, false, true, w.flags, st));
      }
    }
    { KScope k(ctx, VMS_K_DIRICHLET, st); k.add(launch_dirichlet_diag(m, w.values, f32, w.rhs, st)); }
    CK(cudaGetLastError());
    return VMS_OK;
  }
  if (f32) {
    KScope k(ctx, VMS_K_FILL, st);
    k.add(launch_to_fp32(m, ctx->state, w.f32, st));
  }
  TangentOut o;
  o.values = w.values; o.rhs = w.rhs; o.recX = w.recX; o.recKcf = w.recKcf; o.recKinv = w.recKinv;
  o.recY = w.recY;
  const void* tab = f32 ? (const void*)ctx->d_tab32 : (const void*)ctx->d_tab64;
  const int scatter = ctx->tune.scatter_mode >= 0 ? ctx->tune.scatter_mode : ctx->params.scatter_mode;
  const bool colour = scatter == VMS_SCATTER_COLOUR;
  if (f32 && engine(ctx) == 0 && !colour && ctx->tune.schedule == VMS_SCHEDULE_FUSED) {
    // residual and tangent in one persistent launch, then r_e and the Dirichlet rows
    {
      KScope k(ctx, VMS_K_FILL, st);
      k.add(launch_fill_zero(w.queues, 2 * sizeof(unsigned long long), st));
    }
    {
      KScope k(ctx, VMS_K_FUSED, st);
      k.add(launch_fused_assembly(m, ctx->state, w.f32, kp, ctx->d_qp, ctx->d_tab32, w.elemR, o,
                                  w.queues, w.flags, st));
    }
    {
      KScope k(ctx, VMS_K_DIRICHLET, st);
      k.add(launch_finish(f32, m, w.elemR, o, 0, m.n_elems, nullptr, true, st));
    }
    { KScope k(ctx, VMS_K_DIRICHLET, st); k.add(launch_dirichlet_diag(m, w.values, f32, w.rhs, st)); }
    CK(cudaGetLastError());
    return VMS_OK;
  }
  // the FP64 residual kernel (this stream) and the tangent kernel (auxiliary stream, FP32 or FP64
  // pipe) are independent and run concurrently; the finish kernel joins them
  CK(cudaEventRecord(w.fork, st));
  CK(cudaStreamWaitEvent(w.aux, w.fork, 0));
  {
    KScope k(ctx, VMS_K_RESIDUAL, st);
    k.add(launch_residual(m, ctx->state, kp, ctx->d_qp, w.elemR, nullptr, 0, m.n_elems, 0, w.flags, st));
  }
  {
    KScope k(ctx, VMS_K_TANGENT, w.aux);
    if (colour) {
      for (int c = 0; c < m.n_colours; ++c) {
        const int64_t b = m.colour_start[c], n = m.colour_start[c + 1] - b;
        k.add(launch_tangent(f32, engine(ctx), m, ctx->state, w.f32, kp, tab, o, b, n, m.colour_order, false,
                             false, w.flags, w.aux));
      }
    } else {
      k.add(launch_tangent(f32, engine(ctx), m, ctx->state, w.f32, kp, tab, o, 0, m.n_elems, nullptr, false,
                           true, w.flags, w.aux));
    }
  }
  CK(cudaEventRecord(w.join, w.aux));
  CK(cudaStreamWaitEvent(st, w.join, 0));
  {
    KScope k(ctx, VMS_K_DIRICHLET, st);
    if (colour) {
      for (int c = 0; c < m.n_colours; ++c) {
        const int64_t b = m.colour_start[c], n = m.colour_start[c + 1] - b;
        k.add(launch_finish(f32, m, w.elemR, o, b, n, m.colour_order, false, st));
      }
    } else {
      k.add(launch_finish(f32, m, w.elemR, o, 0, m.n_elems, nullptr, true, st));
    }
  }
  { KScope k(ctx, VMS_K_DIRICHLET, st); k.add(launch_dirichlet_diag(m, w.values, f32, w.rhs, st)); }
  CK(cudaGetLastError());
  return VMS_OK;
}

// Capture one assembly into a CUDA graph (on a private stream: the legacy default stream cannot
// be captured) and keep its launch counts per kernel kind for the accounting of every replay.
static int capture_assembly(vms_ctx* ctx) {
  if (ctx->graph) {
    cudaGraphExecDestroy(ctx->graph);
    ctx->graph = nullptr;
  }
  if (!ctx->cap_stream) CK(cudaStreamCreateWithFlags(&ctx->cap_stream, cudaStreamNonBlocking));
  int64_t before[VMS_K_COUNT];
  for (int k = 0; k < VMS_K_COUNT; ++k) before[k] = ctx->launches[k];
  CK(cudaStreamBeginCapture(ctx->cap_stream, cudaStreamCaptureModeRelaxed));
  const int rc = enqueue_assembly(ctx, ctx->cap_stream);
  cudaGraph_t g = nullptr;
  const cudaError_t e = cudaStreamEndCapture(ctx->cap_stream, &g);
  for (int k = 0; k < VMS_K_COUNT; ++k) {
    ctx->graph_launches[k] = ctx->launches[k] - before[k];
    ctx->launches[k] = before[k];
  }
  if (rc) {
    if (g) cudaGraphDestroy(g);
    return rc;
  }
  if (e != cudaSuccess) return fail(ctx, VMS_ERR_CUDA, cudaGetErrorString(e));
  const cudaError_t e2 = cudaGraphInstantiate(&ctx->graph, g, 0);
  cudaGraphDestroy(g);
  if (e2 != cudaSuccess) return fail(ctx, VMS_ERR_CUDA, cudaGetErrorString(e2));
  ctx->graph_dirty = false;
  return VMS_OK;
}

int vms_assemble_newton_schur(vms_ctx* ctx, vms_csr_view* out) {
  if (!ctx) return VMS_ERR_INVALID_ARG;
  if (!ctx->state.valid) return fail(ctx, VMS_ERR_STATE, "mesh and state must be uploaded first");
  CK(cudaSetDevice(ctx->device));
  Work& w = ctx->work;
  if (ctx->stage.pending && ctx->stage.src && ctx->stage.src == w.values && !ctx->use_graph) {
    // the last system's values are still being copied to the host (vms_csr_download_async):
    // assemble into the other buffer
    if (!ctx->stage.alt) CK(cudaMalloc(&ctx->stage.alt, (size_t)ctx->mesh.nnz * sizeof(double)));
    std::swap(w.values, ctx->stage.alt);
  }
  if (ctx->use_graph && !ctx->timing) {
    if (ctx->graph_dirty || !ctx->graph) TRY(capture_assembly(ctx));
    CK(cudaGraphLaunch(ctx->graph, ctx->stream));
    for (int k = 0; k < VMS_K_COUNT; ++k) ctx->launches[k] += ctx->graph_launches[k];
  } else {
    TRY(enqueue_assembly(ctx, ctx->stream));
  }
  TRY(check_flags(ctx));
  w.assembled = true;
  ++w.assembly_id;
  std::fill(ctx->inst_stale.begin(), ctx->inst_stale.end(), 0);
  ctx->any_stale = false;
  if (out) fill_view(ctx, out);
  return VMS_OK;
}

int vms_get_csr(vms_ctx* ctx, vms_csr_view* out) {
  if (!ctx || !out) return fail(ctx, VMS_ERR_INVALID_ARG, "null argument");
  if (!ctx->work.assembled) return fail(ctx, VMS_ERR_STATE, "nothing assembled");
  fill_view(ctx, out);
  return VMS_OK;
}

int vms_csr_download(vms_ctx* ctx, int32_t* rowptr, int32_t* colidx, void* values, double* rhs) {
  if (!ctx) return VMS_ERR_INVALID_ARG;
  if (!ctx->work.assembled) return fail(ctx, VMS_ERR_STATE, "nothing assembled");
  CK(cudaSetDevice(ctx->device));
  const Mesh& m = ctx->mesh;
  cudaStream_t st = ctx->stream;
  const size_t vbytes = (size_t)m.nnz * (fp32_mode(ctx) ? sizeof(float) : sizeof(double));
  if (rowptr) CK(cudaMemcpyAsync(rowptr, m.rowptr, sizeof(int32_t) * (4 * m.n_nodes + 1), cudaMemcpyDefault, st));
  if (colidx) CK(cudaMemcpyAsync(colidx, m.colidx, sizeof(int32_t) * m.nnz, cudaMemcpyDefault, st));
  if (values) CK(cudaMemcpyAsync(values, ctx->work.values, vbytes, cudaMemcpyDefault, st));
  if (rhs) CK(cudaMemcpyAsync(rhs, ctx->work.rhs, sizeof(double) * 4 * m.n_nodes, cudaMemcpyDefault, st));
  CK(cudaStreamSynchronize(st));
  return VMS_OK;
}

int vms_csr_download_async(vms_ctx* ctx, int32_t* rowptr, int32_t* colidx, void* values, double* rhs) {
  if (!ctx) return VMS_ERR_INVALID_ARG;
  if (!ctx->work.assembled) return fail(ctx, VMS_ERR_STATE, "nothing assembled");
  CK(cudaSetDevice(ctx->device));
  if (int rc = stage_wait(ctx)) return rc;
  const Mesh& m = ctx->mesh;
  auto& S = ctx->stage;
  cudaStream_t st = ctx->stream;
  const size_t vbytes = (size_t)m.nnz * (fp32_mode(ctx) ? sizeof(float) : sizeof(double));
  const size_t rbytes = sizeof(double) * 4 * m.n_nodes;
  if (!S.copy) {
    CK(cudaStreamCreateWithFlags(&S.copy, cudaStreamNonBlocking));
    CK(cudaEventCreateWithFlags(&S.snap, cudaEventDisableTiming));
    CK(cudaEventCreateWithFlags(&S.done, cudaEventDisableTiming));
  }
  if (ctx->use_graph && S.vbytes != vbytes) {
    dfree(S.values);
    S.vbytes = 0;
    CK(cudaMalloc(&S.values, vbytes));
    S.vbytes = vbytes;
  }
  if (S.rbytes != rbytes) {
    dfree(S.rhs);
    S.rbytes = 0;
    CK(cudaMalloc(&S.rhs, rbytes));
    S.rbytes = rbytes;
  }
  // The copy to the host runs on its own stream after an event recorded behind the assembly. The
  // values are read from the assembled buffer itself: the next assembly writes the other buffer
  // (vms_assemble_newton_schur swaps them while this copy is pending). A captured assembly graph
  // writes one fixed buffer, so in graph mode the values are first copied into the snapshot.
  const bool swap = !ctx->use_graph;
  if (values && !swap) CK(cudaMemcpyAsync(S.values, ctx->work.values, vbytes, cudaMemcpyDeviceToDevice, st));
  if (rhs) CK(cudaMemcpyAsync(S.rhs, ctx->work.rhs, rbytes, cudaMemcpyDeviceToDevice, st));
  CK(cudaEventRecord(S.snap, st));
  CK(cudaStreamWaitEvent(S.copy, S.snap, 0));
  S.src = values && swap ? ctx->work.values : nullptr;
  if (rowptr) CK(cudaMemcpyAsync(rowptr, m.rowptr, sizeof(int32_t) * (4 * m.n_nodes + 1), cudaMemcpyDefault, S.copy));
  if (colidx) CK(cudaMemcpyAsync(colidx, m.colidx, sizeof(int32_t) * m.nnz, cudaMemcpyDefault, S.copy));
  if (values) CK(cudaMemcpyAsync(values, swap ? ctx->work.values : S.values, vbytes, cudaMemcpyDefault, S.copy));
  if (rhs) CK(cudaMemcpyAsync(rhs, S.rhs, rbytes, cudaMemcpyDefault, S.copy));
  CK(cudaEventRecord(S.done, S.copy));
  S.pending = true;
  return VMS_OK;
}

int vms_csr_download_wait(vms_ctx* ctx) {
  if (!ctx) return VMS_ERR_INVALID_ARG;
  CK(cudaSetDevice(ctx->device));
  return stage_wait(ctx);
}

int vms_residual(vms_ctx* ctx, double* norm, double* R) {
  if (!ctx || !norm) return fail(ctx, VMS_ERR_INVALID_ARG, "null argument");
  if (!ctx->state.valid) return fail(ctx, VMS_ERR_STATE, "mesh and state must be uploaded first");
  CK(cudaSetDevice(ctx->device));
  const Mesh& m = ctx->mesh;
  Work& w = ctx->work;
  cudaStream_t st = ctx->stream;
  const int64_t n = 4 * m.n_nodes + 3 * m.n_elems;
  {
    KScope k(ctx, VMS_K_FILL);
    k.add(launch_fill_zero(w.resid, sizeof(double) * n, st));
    k.add(launch_fill_zero(w.flags, sizeof(unsigned int), st));
  }
  {
    KScope k(ctx, VMS_K_RESIDUAL);
    if (m.npe == 4)
      k.add(launch_tet_residual(m, ctx->state, kparams(ctx), ctx->tet_mom, nullptr,
                                w.resid, 0, m.n_elems, 1, w.flags, st));
    else
      k.add(launch_residual(m, ctx->state, kparams(ctx), ctx->d_qp, nullptr, w.resid, 0, m.n_elems, 1,
                            w.flags, st));
  }
  { KScope k(ctx, VMS_K_REDUCE); k.add(launch_norm2(w.resid, n, w.partial, ctx->d_scalar, st)); }
  CK(cudaGetLastError());
  CK(cudaMemcpyAsync(ctx->h_scalar, ctx->d_scalar, sizeof(double), cudaMemcpyDeviceToHost, st));
  if (R) CK(cudaMemcpyAsync(R, w.resid, sizeof(double) * n, cudaMemcpyDefault, st));
  TRY(check_flags(ctx));
  *norm = std::sqrt(ctx->h_scalar[0]);
  return VMS_OK;
}

// Element outputs of the tetrahedral kernel: blocks of 16 coarse dofs.
static int element_matrices_tet(vms_ctx* ctx, int64_t first, int64_t count, double* S, double* r,
                                double* Kcc, double* Kcf, double* Kfc, double* Kff, double* Rcp,
                                double* Rf) {
  const Mesh& m = ctx->mesh;
  Work& w = ctx->work;
  cudaStream_t st = ctx->stream;
  const KParams kp = kparams(ctx);
  const bool f32 = fp32_mode(ctx);
  {
    KScope k(ctx, VMS_K_RESIDUAL);
    k.add(launch_tet_residual(m, ctx->state, kp, ctx->tet_mom, w.elemR, nullptr,
                              first, count, 0, w.flags, st));
  }
  double* buf = nullptr;
  const size_t per = 256 + 16 + 256 + 48 + 48 + 9;
  CK(cudaMalloc(&buf, sizeof(double) * per * count));
  TangentOut o;
  o.S = buf; o.r = buf + 256 * count; o.Kcc = buf + 272 * count; o.Kcf = buf + 528 * count;
  o.Kfc = buf + 576 * count; o.Kff = buf + 624 * count;
  o.recX = w.recX; o.recKcf = w.recKcf; o.recKinv = w.recKinv; o.recY = w.recY;
  {
    KScope k(ctx, VMS_K_TANGENT);
    k.add(launch_tet_assembly(f32, m, ctx->state, kp, ctx->tet_mom, o, first, count,
                              nullptr, true, true, w.flags, st));
  }
  cudaError_t e = cudaGetLastError();
  struct Out { double* dst; double* src; size_t n; } outs[6] = {
      {S, o.S, 256}, {r, o.r, 16}, {Kcc, o.Kcc, 256}, {Kcf, o.Kcf, 48}, {Kfc, o.Kfc, 48}, {Kff, o.Kff, 9}};
  for (auto& x : outs)
    if (e == cudaSuccess && x.dst)
      e = cudaMemcpyAsync(x.dst, x.src, sizeof(double) * x.n * count, cudaMemcpyDefault, st);
  if (e == cudaSuccess && Rcp)
    e = cudaMemcpy2DAsync(Rcp, 16 * sizeof(double), w.elemR + 36 * first, 36 * sizeof(double),
                          16 * sizeof(double), count, cudaMemcpyDefault, st);
  if (e == cudaSuccess && Rf)
    e = cudaMemcpy2DAsync(Rf, 3 * sizeof(double), w.elemR + 36 * first + 32, 36 * sizeof(double),
                          3 * sizeof(double), count, cudaMemcpyDefault, st);
  if (e == cudaSuccess) e = cudaStreamSynchronize(st);
  cudaFree(buf);
  if (e != cudaSuccess) return fail(ctx, VMS_ERR_CUDA, cudaGetErrorString(e));
  return check_flags(ctx);
}

int vms_element_matrices(vms_ctx* ctx, int64_t first, int64_t count, double* S, double* r,
                         double* Kcc, double* Kcf, double* Kfc, double* Kff, double* Rcp,
                         double* Rf) {
  if (!ctx) return VMS_ERR_INVALID_ARG;
  if (!ctx->state.valid) return fail(ctx, VMS_ERR_STATE, "mesh and state must be uploaded first");
  const Mesh& m = ctx->mesh;
  if (first < 0 || count < 0 || first + count > m.n_elems)
    return fail(ctx, VMS_ERR_INVALID_ARG, "element range out of bounds");
  if (count == 0) return VMS_OK;
  CK(cudaSetDevice(ctx->device));
  Work& w = ctx->work;
  cudaStream_t st = ctx->stream;
  const KParams kp = kparams(ctx);
  const bool f32 = fp32_mode(ctx);
  { KScope k(ctx, VMS_K_FILL); k.add(launch_fill_zero(w.flags, sizeof(unsigned int), st)); }
  if (m.npe == 4) return element_matrices_tet(ctx, first, count, S, r, Kcc, Kcf, Kfc, Kff, Rcp, Rf);
  if (f32) {
    KScope k(ctx, VMS_K_FILL);
    k.add(launch_to_fp32(m, ctx->state, w.f32, st));
  }
  {
    KScope k(ctx, VMS_K_RESIDUAL);
    k.add(launch_residual(m, ctx->state, kp, ctx->d_qp, w.elemR, nullptr, first, count, 0, w.flags, st));
  }
  double* buf = nullptr;
  const size_t per = 1024 + 32 + 1024 + 96 + 96 + 9;
  CK(cudaMalloc(&buf, sizeof(double) * per * count));
  TangentOut o;
  o.S = buf; o.r = buf + 1024 * count; o.Kcc = buf + 1056 * count; o.Kcf = buf + 2080 * count;
  o.Kfc = buf + 2176 * count; o.Kff = buf + 2272 * count;
  o.recX = w.recX; o.recKcf = w.recKcf; o.recKinv = w.recKinv; o.recY = w.recY;
  {
    KScope k(ctx, VMS_K_TANGENT);
    k.add(launch_tangent(f32, engine(ctx), m, ctx->state, w.f32, kp,
                         f32 ? (const void*)ctx->d_tab32 : (const void*)ctx->d_tab64, o, first,
                         count, nullptr, true, true, w.flags, st));
  }
  {
    KScope k(ctx, VMS_K_DIRICHLET);
    k.add(launch_finish(f32, m, w.elemR, o, first, count, nullptr, true, st));
  }
  cudaError_t e = cudaGetLastError();
  struct Out { double* dst; double* src; size_t n; } outs[6] = {
      {S, o.S, 1024}, {r, o.r, 32}, {Kcc, o.Kcc, 1024}, {Kcf, o.Kcf, 96}, {Kfc, o.Kfc, 96}, {Kff, o.Kff, 9}};
  for (auto& x : outs)
    if (e == cudaSuccess && x.dst)
      e = cudaMemcpyAsync(x.dst, x.src, sizeof(double) * x.n * count, cudaMemcpyDefault, st);
  if (e == cudaSuccess && Rcp)
    e = cudaMemcpy2DAsync(Rcp, 32 * sizeof(double), w.elemR + 36 * first, 36 * sizeof(double),
                          32 * sizeof(double), count, cudaMemcpyDefault, st);
  if (e == cudaSuccess && Rf)
    e = cudaMemcpy2DAsync(Rf, 3 * sizeof(double), w.elemR + 36 * first + 32, 36 * sizeof(double),
                          3 * sizeof(double), count, cudaMemcpyDefault, st);
  if (e == cudaSuccess) e = cudaStreamSynchronize(st);
  cudaFree(buf);
  if (e != cudaSuccess) return fail(ctx, VMS_ERR_CUDA, cudaGetErrorString(e));
  return check_flags(ctx);
}

int vms_profile_enable(vms_ctx* ctx, int timing) {
  if (!ctx) return VMS_ERR_INVALID_ARG;
  ctx->timing = timing != 0;
  return VMS_OK;
}

int vms_profile_read(vms_ctx* ctx, int reset, double* ms, int64_t* launches) {
  if (!ctx) return VMS_ERR_INVALID_ARG;
  CK(cudaSetDevice(ctx->device));
  CK(cudaStreamSynchronize(ctx->stream));
  for (auto& e : ctx->events) {
    float t = 0.f;
    if (cudaEventElapsedTime(&t, e.a, e.b) == cudaSuccess) ctx->ms[e.kind] += t;
    ctx->pool.push_back(e.a);
    ctx->pool.push_back(e.b);
  }
  ctx->events.clear();
  for (int k = 0; k < VMS_K_COUNT; ++k) {
    if (ms) ms[k] = ctx->ms[k];
    if (launches) launches[k] = ctx->launches[k];
    if (reset) { ctx->ms[k] = 0.0; ctx->launches[k] = 0; }
  }
  return VMS_OK;
}

int vms_solver_stats(vms_ctx* ctx, int reset, int64_t* solves, int64_t* krylov_iterations) {
  if (!ctx) return VMS_ERR_INVALID_ARG;
  if (solves) *solves = ctx->solver_stats[0];
  if (krylov_iterations) *krylov_iterations = ctx->solver_stats[1];
  if (reset) ctx->solver_stats[0] = ctx->solver_stats[1] = 0;
  return VMS_OK;
}

}  // extern "C"

// Accessors used by the solver translation unit.
namespace vms {
const Mesh& ctx_mesh(vms_ctx* c) { return c->mesh; }
State& ctx_state(vms_ctx* c) { return c->state; }
Work& ctx_work(vms_ctx* c) { return c->work; }
SolverWork& ctx_solver(vms_ctx* c) { return c->solver; }
cudaStream_t ctx_stream(vms_ctx* c) { return c->stream; }
int ctx_device(vms_ctx* c) { return c->device; }
bool ctx_fp32(vms_ctx* c) { return fp32_mode(c); }
int ctx_precond(vms_ctx* c) { return c->precond; }
// The assembled block of instance i no longer matches its state (i < 0: the whole system).
bool ctx_stale(vms_ctx* c, int64_t i) { return i < 0 ? c->any_stale : c->inst_stale[i] != 0; }
void ctx_mark_stale(vms_ctx* c, int64_t i) {
  c->inst_stale[i] = 1;
  c->any_stale = true;
}
bool ctx_instance(vms_ctx* c, int64_t i, SysRange* out) {
  if (c->inst_nodes.empty() || i < 0 || i + 1 >= (int64_t)c->inst_nodes.size()) return false;
  *out = SysRange{c->inst_nodes[i], c->inst_nodes[i + 1], c->inst_elems[i], c->inst_elems[i + 1]};
  return true;
}
int64_t* ctx_solver_stats(vms_ctx* c) { return c->solver_stats; }
double* ctx_dscalar(vms_ctx* c) { return c->d_scalar; }
double* ctx_hscalar(vms_ctx* c) { return c->h_scalar; }
int ctx_fail(vms_ctx* c, int code, const char* msg) { return fail(c, code, msg); }
}  // namespace vms
