// C ABI of the library (include/mfcg.h): problem setup, operator, diagonal,
// right-hand side, the fused (Algorithm 5) and unfused (Algorithm 1) CG
// drivers, the FP64 defect correction around an FP32 fused CG, and the
// reordering helpers.
//
// Execution model: every call runs on a private non-blocking stream that is
// ordered after the caller's stream on entry and before it on exit (events),
// so CUDA graphs can be captured even when the caller uses the legacy stream.
// The CG iterations are captured once per problem as a graph of G iterations
// (an even number: odd and even iterations use swapped ping-pong buffers);
// the host replays it and reads the device-side convergence flag only once per
// graph, one graph behind, so there is no per-iteration host synchronisation.
#include <algorithm>
#include <array>
#include <chrono>
#include <cmath>
#include <cstdlib>
#include <cstring>
#include <new>
#include <vector>

#include "mfcg_internal.h"
#include "precision.cuh"
#include "tc_operator.cuh"

struct mfcg_problem;
int setup_impl(const mfcg_mesh* mesh, int degree, const mfcg_geometry* geom, const mfcg_options* opt,
               void* cuda_stream, mfcg_problem** out, const mfcg_problem* share);

namespace mfcg {
void build_coeffs(int p, const double h[3], double amplitude, int coef, OperatorCoeffs& c);
int vec_grid(int64_t n);
}  // namespace mfcg

using namespace mfcg;

struct mfcg_problem {
  int device = 0;
  cudaStream_t user = nullptr;
  cudaStream_t exec = nullptr;
  cudaEvent_t ev_in = nullptr, ev_out = nullptr;
  int degree = 0;
  mfcg_mesh mesh{};
  mfcg_geometry geom{};
  mfcg_options opt{};
  TileGeom g{};
  OperatorCoeffs c{};
  int geom_kind = GEOM_AFFINE;
  int ncomp = 1;           // components of the vector-valued operator
  int op_kind = OP_LAPLACE;
  int op_prec = PREC_F64;  // apply_operator and FP64-accurate residuals
  int cg_prec = PREC_F64;  // fused CG iterations
  // FP64 operator passes and fused iterations of Cartesian problems with the
  // contractions on the tensor cores (PREC_F64TC in place of PREC_F64)
  bool tc = false;
  uint2* tc_frag = nullptr;
  int tc_g2 = 0;
  int tc_r = 64;
  // fused CG vectors in the storage type of cg_prec (ping-pong r, p, v), x, M^{-1}
  void* r[2] = {nullptr, nullptr};
  void* p[2] = {nullptr, nullptr};
  void* v[2] = {nullptr, nullptr};
  void* xs = nullptr;
  void* dinv_s = nullptr;
  // FP64 vectors
  double* x = nullptr;      // unfused iterate / defect-correction iterate
  double* z = nullptr;      // unfused M^{-1} r
  double* ur = nullptr;     // unfused r
  double* up = nullptr;     // unfused p
  double* uv = nullptr;     // unfused v
  double* work = nullptr;   // A x0, residuals
  double* bdev = nullptr;   // host-array solves: b
  double* xdev = nullptr;   // host-array solves: x
  double* diag = nullptr;
  double* diag_inv = nullptr;
  void* shell = nullptr;
  double* partial = nullptr;
  double* geo = nullptr;    // FP64 per-point metric (deformed)
  void* geo_op = nullptr;   // metric in the operator precision
  void* geo_cg = nullptr;   // metric in the CG precision
  CGState* state = nullptr;
  CGState* h_state = nullptr;  // pinned, two slots
  int64_t tail_nodes = 0;
  int64_t fam[3] = {0, 0, 0};
  TailDiv tdiv{};
  int tail_ctas = 1;
  int ahead_op = 0;  // L2 prefetch distance (tiles) of the operator passes
  int stagger_lo = 0, stagger_hi = 0;  // start offset of the fused tensor-core iterations
  long long stagger_cycles = 0;
  int graph_iters = 16;
  cudaGraphExec_t graph_fused = nullptr;
  cudaGraphExec_t graph_unfused = nullptr;
  cudaGraphExec_t graph_semi = nullptr;
  cudaGraphExec_t graph_loop = nullptr;
  int64_t launches = 0;
  std::vector<void*> owned;  // every device allocation
  int64_t nv() const { return ncomp * g.n_dofs; }  // length of every vector of the ABI
};

// A batch: independent member problems whose fused iterations are captured
// as one graph with one branch per member.
struct mfcg_batch {
  int device = 0;
  cudaStream_t user = nullptr;
  cudaStream_t exec = nullptr;
  cudaEvent_t ev_in = nullptr, ev_out = nullptr, ev_fork = nullptr;
  std::vector<mfcg_problem*> members;
  std::vector<cudaEvent_t> ev_join;  // one per member
  int graph_iters = 16;
  cudaGraphExec_t graph = nullptr;
  CGState** d_states = nullptr;      // device array of the members' state pointers
  int* d_done = nullptr;             // device: done flag per member
  int* h_done = nullptr;             // pinned: two slots of count flags
};

namespace {

// the defect-correction precisions (FP64 outer residual around an inner fused CG)
bool inner_precision(int precision) {
  return precision == MFCG_PREC_FP32_INNER || precision == MFCG_PREC_DOUBLE_FLOAT_INNER;
}

// internal geometry kind of an mfcg_geometry_kind (MFCG_GEOM_USER data is stored like MFCG_GEOM_DEFORMED)
int geom_kind_of(int kind) {
  if (kind == MFCG_GEOM_AFFINE) return GEOM_AFFINE;
  if (kind == MFCG_GEOM_DEFORMED_TENSOR) return GEOM_TENSOR;
  if (kind == MFCG_GEOM_DEFORMED_QUADRATIC) return GEOM_QUAD;
  return GEOM_DEFORMED;
}

#define CK(call)                                   \
  do {                                             \
    cudaError_t e_ = (call);                       \
    if (e_ != cudaSuccess) return MFCG_CUDA_ERROR; \
  } while (0)

template <typename Ptr>
int alloc_bytes(mfcg_problem* P, Ptr* p, int64_t bytes) {
  void* q = nullptr;
  if (cudaMalloc(&q, (size_t)std::max<int64_t>(bytes, 16)) != cudaSuccess) {
    cudaGetLastError();
    *p = nullptr;
    return MFCG_OUT_OF_MEMORY;
  }
  P->owned.push_back(q);
  *p = static_cast<Ptr>(q);
  return MFCG_OK;
}

// default tile edge (cells) per degree: node bricks of about 17^3; the FP32
// inner solver of the defect correction at p = 4 runs faster on 21^3 bricks
// (three CTAs per SM still fit: 74 KB of shared memory, measured on Q4 64^3)
int default_tile(int p, int geom, int precision = MFCG_PREC_FP64) {
  static const int affine[9] = {0, 16, 8, 5, 4, 3, 3, 2, 2};
  static const int deformed[9] = {0, 8, 4, 4, 3, 2, 2, 2, 2};
  if (geom == GEOM_AFFINE && precision == MFCG_PREC_FP32_INNER && p == 4) return 5;
  return geom == GEOM_AFFINE ? affine[p] : deformed[p];
}

// arguments of a tile / tail launch in precision prec; the operator passes and
// fused iterations of FP64 run on the tensor-core operator when the problem has
// it (the set-up passes, MODE_RHS and MODE_DIAG, stay on PREC_F64)
TileArgs base_args(const mfcg_problem* P, int prec, const void* geo, int mode) {
  TileArgs a{};
  if (prec == PREC_F64 && P->tc && (mode == MODE_OPERATOR || mode == MODE_CG)) {
    prec = PREC_F64TC;
    a.tc_frag = P->tc_frag;
    a.tc_g2 = P->tc_g2;
    a.tc_r = P->tc_r;
  }
  a.g = P->g;
  a.shell = P->shell;
  a.partial = P->partial;
  a.geo = geo;
  a.state = P->state;
  a.tail_nodes = P->tail_nodes;
  for (int d = 0; d < 3; ++d) a.fam[d] = P->fam[d];
  a.tdiv = P->tdiv;
  a.geom = P->geom_kind;
  a.prec = prec;
  a.tail_ctas = P->tail_ctas;
  a.ncomp = P->ncomp;
  a.op_kind = P->op_kind;
  a.comp_stride = P->g.n_dofs;
  a.shell_comp_stride = P->g.n_tiles * P->g.face_stride;
  return a;
}

// operator-like pass (tile kernel + tail) with FP64 input/output; fp64_operator
// forces the FP64 operator (true residuals) whatever the operator precision
int run_pass(mfcg_problem* P, int mode, const double* src, double* dst, bool fp64_operator = false) {
  const int prec = mode == MODE_OPERATOR && !fp64_operator ? P->op_prec : PREC_F64;
  TileArgs a = base_args(P, prec, mode == MODE_OPERATOR && !fp64_operator ? P->geo_op : P->geo, mode);
  if (mode != MODE_OPERATOR) a.ncomp = 1;  // diagonal and right-hand side of the scalar operator
  a.prefetch_ahead = mode == MODE_OPERATOR && prec == P->op_prec ? P->ahead_op : 0;
  a.in0 = src;
  a.out0 = dst;
  CK(launch_tile(P->degree, mode, a, P->c, P->exec));
  CK(launch_tail(P->degree, mode, a, P->exec));
  P->launches += 2;
  return MFCG_OK;
}

// one fused CG iteration of the given parity (odd: buffers 0 -> 1)
int enqueue_fused_iteration(mfcg_problem* P, int odd, cudaEvent_t t0, cudaEvent_t t1) {
  const int o = odd ? 0 : 1, n = odd ? 1 : 0;
  TileArgs a = base_args(P, P->cg_prec, P->geo_cg, MODE_CG);  // no look-ahead prefetch (prefetch_ahead 0)
  a.stagger_lo = P->stagger_lo;
  a.stagger_hi = P->stagger_hi;
  a.stagger_cycles = P->stagger_cycles;
  a.in0 = P->r[o];
  a.in1 = P->v[o];
  a.in2 = P->p[o];
  a.diag_inv = P->dinv_s;
  a.out0 = P->r[n];
  a.out1 = P->v[n];
  a.out2 = P->p[n];
  a.x = P->xs;
  if (t0) CK(cudaEventRecord(t0, P->exec));
  CK(launch_tile(P->degree, MODE_CG, a, P->c, P->exec));
  if (t1) CK(cudaEventRecord(t1, P->exec));
  CK(launch_tail(P->degree, MODE_CG, a, P->exec));
  return MFCG_OK;
}

UnfusedArgs unfused_args(mfcg_problem* P) {
  UnfusedArgs u{};
  u.n = P->nv();
  u.diag_inv = P->diag_inv;
  u.x = P->x;
  u.r = P->ur;
  u.p = P->up;
  u.v = P->uv;
  u.z = P->z;
  u.partial = P->partial;
  u.state = P->state;
  return u;
}

int enqueue_unfused_iteration(mfcg_problem* P, cudaEvent_t t0, cudaEvent_t t1) {
  UnfusedArgs u = unfused_args(P);
  if (t0) CK(cudaEventRecord(t0, P->exec));
  // v = A p
  TileArgs a = base_args(P, P->op_prec, P->geo_op, MODE_OPERATOR);
  a.prefetch_ahead = P->ahead_op;
  a.stop_on_done = 1;
  a.in0 = u.p;
  a.out0 = u.v;
  CK(launch_tile(P->degree, MODE_OPERATOR, a, P->c, P->exec));
  if (t1) CK(cudaEventRecord(t1, P->exec));
  CK(launch_tail(P->degree, MODE_OPERATOR, a, P->exec));
  CK(launch_unfused_dot(0, u, P->exec));   // alpha = e / p.v
  CK(launch_unfused_axpy(0, u, P->exec));  // x += alpha p
  CK(launch_unfused_axpy(1, u, P->exec));  // r -= alpha v
  CK(launch_unfused_dot(1, u, P->exec));   // gamma = r.r, convergence
  CK(launch_unfused_axpy(2, u, P->exec));  // z = M^-1 r
  CK(launch_unfused_dot(2, u, P->exec));   // beta = r.z / e
  CK(launch_unfused_axpy(3, u, P->exec));  // p = z + beta p
  return MFCG_OK;
}

// Algorithm 1 with loop fusion in its vector regions: operator (tile + tail),
// p.v, one pass for x, r and r.r, one for z = M^-1 r and r.z, the p update
int enqueue_loop_fused_iteration(mfcg_problem* P, cudaEvent_t t0, cudaEvent_t t1) {
  UnfusedArgs u = unfused_args(P);
  if (t0) CK(cudaEventRecord(t0, P->exec));
  TileArgs a = base_args(P, P->op_prec, P->geo_op, MODE_OPERATOR);
  a.prefetch_ahead = P->ahead_op;
  a.stop_on_done = 1;
  a.in0 = u.p;
  a.out0 = u.v;
  CK(launch_tile(P->degree, MODE_OPERATOR, a, P->c, P->exec));
  if (t1) CK(cudaEventRecord(t1, P->exec));
  CK(launch_tail(P->degree, MODE_OPERATOR, a, P->exec));
  CK(launch_unfused_dot(0, u, P->exec));   // alpha = e / p.v
  CK(launch_loop_fused(0, u, P->exec));    // x += alpha p, r -= alpha v, gamma = r.r, convergence
  CK(launch_loop_fused(1, u, P->exec));    // z = M^-1 r, beta = r.z / e
  CK(launch_unfused_axpy(3, u, P->exec));  // p = z + beta p
  return MFCG_OK;
}

// semi-fused Algorithm 5: "pre" kernel, operator (tile + tail), "post" kernel
int enqueue_semi_iteration(mfcg_problem* P, cudaEvent_t t0, cudaEvent_t t1) {
  const int64_t n = P->nv();
  CK(launch_semi_pre(n, P->state, P->x, P->ur, P->up, P->uv, P->diag_inv, P->exec));
  TileArgs a = base_args(P, P->op_prec, P->geo_op, MODE_OPERATOR);
  a.prefetch_ahead = P->ahead_op;
  a.stop_on_done = 1;
  a.in0 = P->up;
  a.out0 = P->uv;
  if (t0) CK(cudaEventRecord(t0, P->exec));
  CK(launch_tile(P->degree, MODE_OPERATOR, a, P->c, P->exec));
  if (t1) CK(cudaEventRecord(t1, P->exec));
  CK(launch_tail(P->degree, MODE_OPERATOR, a, P->exec));
  CK(launch_semi_post(n, P->state, P->ur, P->up, P->uv, P->diag_inv, P->partial, P->exec));
  return MFCG_OK;
}

enum IterKind { ITER_FUSED = 0, ITER_UNFUSED = 1, ITER_SEMI = 2, ITER_LOOP_FUSED = 3 };
constexpr int kLaunchesPerIter[4] = {2, 9, 4, 6};

int enqueue_iteration(mfcg_problem* P, int kind, int odd, cudaEvent_t t0, cudaEvent_t t1) {
  if (kind == ITER_FUSED) return enqueue_fused_iteration(P, odd, t0, t1);
  if (kind == ITER_UNFUSED) return enqueue_unfused_iteration(P, t0, t1);
  if (kind == ITER_LOOP_FUSED) return enqueue_loop_fused_iteration(P, t0, t1);
  return enqueue_semi_iteration(P, t0, t1);
}

int capture_graph(mfcg_problem* P, int kind, cudaGraphExec_t* out) {
  cudaGraph_t graph;
  CK(cudaStreamBeginCapture(P->exec, cudaStreamCaptureModeThreadLocal));
  int st = MFCG_OK;
  for (int it = 0; it < P->graph_iters && st == MFCG_OK; ++it)
    st = enqueue_iteration(P, kind, (it & 1) == 0, nullptr, nullptr);
  cudaError_t e = cudaStreamEndCapture(P->exec, &graph);
  if (st != MFCG_OK || e != cudaSuccess) return MFCG_CUDA_ERROR;
  e = cudaGraphInstantiate(out, graph, 0);
  cudaGraphDestroy(graph);
  return e == cudaSuccess ? MFCG_OK : MFCG_CUDA_ERROR;
}

int enter(mfcg_problem* P) {
  CK(cudaSetDevice(P->device));
  CK(cudaEventRecord(P->ev_in, P->user));
  CK(cudaStreamWaitEvent(P->exec, P->ev_in, 0));
  return MFCG_OK;
}

int leave(mfcg_problem* P) {
  CK(cudaEventRecord(P->ev_out, P->exec));
  CK(cudaStreamWaitEvent(P->user, P->ev_out, 0));
  return MFCG_OK;
}

struct IterStats {
  double main_ms = 0.0;
  int main_launches = 0;
};

// Runs CG iterations until the device flag is set or maxit is reached: graphs
// of G iterations (no per-iteration host synchronisation), or direct launches
// with CUDA events around every operator-pass kernel when instrumenting.
int run_iterations(mfcg_problem* P, int kind, int maxit, IterStats& stats) {
  int st;
  const int per_iter = kLaunchesPerIter[kind];
  if (P->opt.instrument) {
    std::vector<cudaEvent_t> ev;
    int done_it = 0;
    while (done_it < maxit) {
      const int chunk = std::min(64, maxit - done_it);
      ev.resize(2 * chunk);
      for (auto& e : ev) CK(cudaEventCreate(&e));
      for (int i = 0; i < chunk; ++i) {
        const int k = done_it + i + 1;
        st = enqueue_iteration(P, kind, k & 1, ev[2 * i], ev[2 * i + 1]);
        if (st != MFCG_OK) return st;
      }
      P->launches += (int64_t)chunk * per_iter;
      CK(cudaMemcpyAsync(P->h_state, P->state, sizeof(CGState), cudaMemcpyDeviceToHost, P->exec));
      CK(cudaStreamSynchronize(P->exec));
      const int ran = std::min(chunk, std::max(0, P->h_state->iterations - done_it));
      for (int i = 0; i < ran; ++i) {
        float ms = 0.f;
        CK(cudaEventElapsedTime(&ms, ev[2 * i], ev[2 * i + 1]));
        stats.main_ms += ms;
        ++stats.main_launches;
      }
      for (auto& e : ev) cudaEventDestroy(e);
      done_it += chunk;
      if (P->h_state->done) break;
    }
    return MFCG_OK;
  }
  cudaGraphExec_t* const graphs[4] = {&P->graph_fused, &P->graph_unfused, &P->graph_semi, &P->graph_loop};
  cudaGraphExec_t* gexec = graphs[kind];
  if (!*gexec && (st = capture_graph(P, kind, gexec)) != MFCG_OK) return st;
  const int G = P->graph_iters;
  const int n_graphs = (maxit + G - 1) / G;
  cudaEvent_t evs[2];
  CK(cudaEventCreateWithFlags(&evs[0], cudaEventDisableTiming));
  CK(cudaEventCreateWithFlags(&evs[1], cudaEventDisableTiming));
  int launched = 0, checked = 0;
  bool finished = n_graphs == 0;
  while (!finished) {
    // keep one graph in flight ahead of the flag being read
    while (launched < n_graphs && launched < checked + 2) {
      CK(cudaGraphLaunch(*gexec, P->exec));
      CK(cudaMemcpyAsync(P->h_state + (launched & 1), P->state, sizeof(CGState), cudaMemcpyDeviceToHost, P->exec));
      CK(cudaEventRecord(evs[launched & 1], P->exec));
      P->launches += (int64_t)G * per_iter;
      ++launched;
    }
    if (checked >= launched) break;
    CK(cudaEventSynchronize(evs[checked & 1]));
    if (P->h_state[checked & 1].done) finished = true;
    ++checked;
    if (checked >= n_graphs) finished = true;
  }
  CK(cudaStreamSynchronize(P->exec));
  cudaEventDestroy(evs[0]);
  cudaEventDestroy(evs[1]);
  return MFCG_OK;
}

// Fused CG (Algorithm 5) in P->cg_prec on the system A x = b with the FP64
// initial residual r0 and the initial guess already in P->xs.
// start-up of the fused CG: scalars from (b, r0), r_0 in the CG precision, p and v zero
int fused_start(mfcg_problem* P, const double* b, const double* r0, double rtol, int maxit, int fixed) {
  const int64_t n = P->nv();
  const size_t es = prec_bytes(P->cg_prec);
  CK(launch_cg_init(P->state, b, r0, n, rtol, maxit, fixed, P->partial, P->opt.x_update_every_iteration, P->exec));
  CK(launch_to_prec(P->cg_prec, r0, P->r[0], n, P->exec));
  CK(cudaMemsetAsync(P->p[0], 0, n * es, P->exec));
  CK(cudaMemsetAsync(P->v[0], 0, n * es, P->exec));
  P->launches += 2;
  return MFCG_OK;
}

// parity-dependent finalisation of x (Algorithm 5)
int fused_finish(mfcg_problem* P) {
  CK(launch_finalize_fused(P->cg_prec, P->nv(), P->state, P->xs, P->p[0], P->p[1], P->r[0], P->r[1], P->dinv_s,
                           P->exec));
  P->launches += 1;
  return MFCG_OK;
}

int fused_core(mfcg_problem* P, const double* b, const double* r0, double rtol, int maxit, int fixed,
               IterStats& stats) {
  int st = fused_start(P, b, r0, rtol, maxit, fixed);
  if (st == MFCG_OK) st = run_iterations(P, ITER_FUSED, maxit, stats);
  if (st == MFCG_OK) st = fused_finish(P);
  return st;
}

// r0 = b - A x0 in FP64 (operator in the operator precision) and x0 in the CG precision
int fused_initial_residual(mfcg_problem* P, const double* b, const double* x_user) {
  const int64_t n = P->nv();
  int st = run_pass(P, MODE_OPERATOR, x_user, P->work);
  if (st != MFCG_OK) return st;
  CK(launch_residual(b, P->work, P->work, n, P->exec));
  CK(launch_to_prec(P->cg_prec, x_user, P->xs, n, P->exec));
  P->launches += 2;
  return MFCG_OK;
}

void fill_info(mfcg_problem* P, mfcg_solve_info* info, int status, int iterations, const IterStats& stats,
               int64_t launches0, int outer) {
  if (!info) return;
  const CGState& S = *P->h_state;
  info->iterations = iterations;
  info->converged = status == MFCG_OK && S.done == 1;
  info->status = status;
  info->main_kernel_launches = stats.main_launches;
  info->residual_sq_est = S.gamma_next;
  info->rhs_norm_sq = S.sums[7];
  info->main_kernel_ms = stats.main_ms;
  info->kernel_launches = P->launches - launches0;
  info->outer_cycles = outer;
  info->reserved2 = 0;
  info->true_residual_sq = -1.0;
}

int solve_direct(mfcg_problem* P, const double* b, double* x_user, double rtol, int maxit, mfcg_solve_info* info) {
  const int64_t n = P->nv();
  const int fused = P->opt.mode == MFCG_MODE_FUSED;
  const int64_t launches0 = P->launches;
  const int fixed = rtol == 0.0;
  IterStats stats;
  int st;
  // r0 = b - A x0 in FP64 (operator in the operator precision)
  if ((st = run_pass(P, MODE_OPERATOR, x_user, P->work)) != MFCG_OK) return st;
  CK(launch_residual(b, P->work, P->work, n, P->exec));
  P->launches += 1;
  if (fused) {
    CK(launch_to_prec(P->cg_prec, x_user, P->xs, n, P->exec));
    P->launches += 1;
    if ((st = fused_core(P, b, P->work, rtol, maxit, fixed, stats)) != MFCG_OK) return st;
    CK(launch_from_prec(P->cg_prec, P->xs, x_user, n, 0, P->exec));
    P->launches += 1;
  } else if (P->opt.mode == MFCG_MODE_SEMI_FUSED) {
    CK(cudaMemcpyAsync(P->x, x_user, n * sizeof(double), cudaMemcpyDeviceToDevice, P->exec));
    CK(cudaMemcpyAsync(P->ur, P->work, n * sizeof(double), cudaMemcpyDeviceToDevice, P->exec));
    CK(cudaMemsetAsync(P->up, 0, n * sizeof(double), P->exec));
    CK(cudaMemsetAsync(P->uv, 0, n * sizeof(double), P->exec));
    CK(launch_cg_init(P->state, b, P->ur, n, rtol, maxit, fixed, P->partial, P->opt.x_update_every_iteration,
                      P->exec));
    P->launches += 1;
    if ((st = run_iterations(P, ITER_SEMI, maxit, stats)) != MFCG_OK) return st;
    CK(launch_finalize_fused(PREC_F64, n, P->state, P->x, P->up, P->up, P->ur, P->ur, P->diag_inv, P->exec));
    CK(cudaMemcpyAsync(x_user, P->x, n * sizeof(double), cudaMemcpyDeviceToDevice, P->exec));
    P->launches += 1;
  } else {
    CK(cudaMemcpyAsync(P->x, x_user, n * sizeof(double), cudaMemcpyDeviceToDevice, P->exec));
    CK(cudaMemcpyAsync(P->ur, P->work, n * sizeof(double), cudaMemcpyDeviceToDevice, P->exec));
    CK(cudaMemsetAsync(P->uv, 0, n * sizeof(double), P->exec));
    CK(launch_cg_init(P->state, b, P->ur, n, rtol, maxit, fixed, P->partial, 0, P->exec));
    UnfusedArgs u = unfused_args(P);
    CK(launch_unfused_dot(3, u, P->exec));  // z0 = M^-1 r0, p0 = z0, e0 = r0.z0
    P->launches += 2;
    const int kind = P->opt.mode == MFCG_MODE_LOOP_FUSED ? ITER_LOOP_FUSED : ITER_UNFUSED;
    if ((st = run_iterations(P, kind, maxit, stats)) != MFCG_OK) return st;
    CK(cudaMemcpyAsync(x_user, P->x, n * sizeof(double), cudaMemcpyDeviceToDevice, P->exec));
  }
  CK(cudaMemcpyAsync(P->h_state, P->state, sizeof(CGState), cudaMemcpyDeviceToHost, P->exec));
  CK(cudaStreamSynchronize(P->exec));
  const CGState& S = *P->h_state;
  int status = MFCG_OK;
  if (S.done == 3) status = MFCG_BREAKDOWN;
  else if (S.done != 1 && !fixed) status = MFCG_NOT_CONVERGED;
  fill_info(P, info, status, S.iterations, stats, launches0, 0);
  return status;
}

// FP64 defect correction: x_{j+1} = x_j + d_j with A d_j = b - A x_j solved by
// the fused CG in the inner precision (FP32 or double-float) to a relative
// reduction inner_rtol; the true residual is formed with the FP64 operator and
// FP64 vectors.  Double-float inner solves without inner_rtol run to half the
// reduction the true residual still needs (at least 1e-12): the first cycle
// then usually reaches rtol, and a second one removes the rounding of the first.
int solve_defect_correction(mfcg_problem* P, const double* b, double* x_user, double rtol, int maxit,
                            mfcg_solve_info* info) {
  const int64_t n = P->nv();
  const int64_t launches0 = P->launches;
  const double inner = P->opt.inner_rtol > 0.0 ? P->opt.inner_rtol : 1e-3;
  const bool adaptive = P->opt.precision == MFCG_PREC_DOUBLE_FLOAT_INNER && !(P->opt.inner_rtol > 0.0);
  IterStats stats;
  int st;
  CK(cudaMemcpyAsync(P->x, x_user, n * sizeof(double), cudaMemcpyDeviceToDevice, P->exec));
  // ||b||^2 once (the reduction kernel of the CG start-up, applied to b alone)
  CK(launch_cg_init(P->state, b, b, n, 0.0, 1, 0, P->partial, 0, P->exec));
  CK(cudaMemcpyAsync(P->h_state, P->state, sizeof(CGState), cudaMemcpyDeviceToHost, P->exec));
  CK(cudaStreamSynchronize(P->exec));
  P->launches += 1;
  const double bb = P->h_state->sums[7];
  int total_it = 0, cycles = 0, status = MFCG_NOT_CONVERGED;
  double rr = 0.0;
  while (true) {
    // true residual r = b - A x; the start-up reduction of the inner CG on
    // (r, r) gives ||r||^2 and the inner tolerance inner_rtol^2 ||r||^2
    if ((st = run_pass(P, MODE_OPERATOR, P->x, P->work)) != MFCG_OK) return st;
    CK(launch_residual(b, P->work, P->work, n, P->exec));
    CK(launch_cg_init(P->state, P->work, P->work, n, inner, std::max(maxit - total_it, 1), 0, P->partial,
                      P->opt.x_update_every_iteration, P->exec));
    CK(cudaMemcpyAsync(P->h_state, P->state, sizeof(CGState), cudaMemcpyDeviceToHost, P->exec));
    CK(cudaStreamSynchronize(P->exec));
    P->launches += 2;
    rr = P->h_state->gamma_next;
    if (!std::isfinite(rr)) {
      status = MFCG_BREAKDOWN;
      break;
    }
    if (rr < rtol * rtol * bb || rr == 0.0) {
      status = MFCG_OK;
      break;
    }
    if (total_it >= maxit) break;
    if (adaptive) {
      // the inner tolerance for this cycle: the start-up again with it
      const double need = std::min(0.5, std::max(1e-12, 0.5 * rtol * std::sqrt(bb / rr)));
      CK(launch_cg_init(P->state, P->work, P->work, n, need, std::max(maxit - total_it, 1), 0, P->partial,
                        P->opt.x_update_every_iteration, P->exec));
      P->launches += 1;
    }
    // inner FP32 solve of A d = r from d = 0 (its scalars were set by cg_init above)
    const size_t es = prec_bytes(P->cg_prec);
    CK(launch_to_prec(P->cg_prec, P->work, P->r[0], n, P->exec));
    CK(cudaMemsetAsync(P->p[0], 0, n * es, P->exec));
    CK(cudaMemsetAsync(P->v[0], 0, n * es, P->exec));
    CK(cudaMemsetAsync(P->xs, 0, n * es, P->exec));
    P->launches += 1;
    if ((st = run_iterations(P, ITER_FUSED, maxit - total_it, stats)) != MFCG_OK) return st;
    CK(launch_finalize_fused(P->cg_prec, n, P->state, P->xs, P->p[0], P->p[1], P->r[0], P->r[1], P->dinv_s,
                             P->exec));
    CK(launch_from_prec(P->cg_prec, P->xs, P->x, n, 1, P->exec));  // x += d in FP64
    CK(cudaMemcpyAsync(P->h_state, P->state, sizeof(CGState), cudaMemcpyDeviceToHost, P->exec));
    CK(cudaStreamSynchronize(P->exec));
    P->launches += 2;
    total_it += P->h_state->iterations;
    ++cycles;
    if (P->h_state->done == 3) {
      status = MFCG_BREAKDOWN;
      break;
    }
  }
  CK(cudaMemcpyAsync(x_user, P->x, n * sizeof(double), cudaMemcpyDeviceToDevice, P->exec));
  CK(cudaStreamSynchronize(P->exec));
  fill_info(P, info, status, total_it, stats, launches0, cycles);
  if (info) {
    info->converged = status == MFCG_OK;
    info->residual_sq_est = rr;  // true residual of the last check
    info->rhs_norm_sq = bb;
  }
  return status;
}

// rtol == 0 with the FP32 inner form: one correction x += d with exactly maxit
// inner FP32 iterations on A d = b - A x (benchmark mode of the inner kernel).
int solve_fixed_inner(mfcg_problem* P, const double* b, double* x_user, int maxit, mfcg_solve_info* info) {
  const int64_t n = P->nv();
  const int64_t launches0 = P->launches;
  const size_t es = prec_bytes(P->cg_prec);
  IterStats stats;
  int st;
  if ((st = run_pass(P, MODE_OPERATOR, x_user, P->work)) != MFCG_OK) return st;
  CK(launch_residual(b, P->work, P->work, n, P->exec));
  CK(cudaMemsetAsync(P->xs, 0, n * es, P->exec));
  P->launches += 1;
  if ((st = fused_core(P, P->work, P->work, 0.0, maxit, 1, stats)) != MFCG_OK) return st;
  CK(launch_from_prec(P->cg_prec, P->xs, x_user, n, 1, P->exec));
  CK(cudaMemcpyAsync(P->h_state, P->state, sizeof(CGState), cudaMemcpyDeviceToHost, P->exec));
  CK(cudaStreamSynchronize(P->exec));
  P->launches += 1;
  const int status = P->h_state->done == 3 ? MFCG_BREAKDOWN : MFCG_OK;
  fill_info(P, info, status, P->h_state->iterations, stats, launches0, 1);
  return status;
}

int solve_impl(mfcg_problem* P, const double* b, double* x_user, double rtol, int maxit, mfcg_solve_info* info) {
  int st;
  if (inner_precision(P->opt.precision))
    st = rtol == 0.0 ? solve_fixed_inner(P, b, x_user, maxit, info) : solve_defect_correction(P, b, x_user, rtol, maxit, info);
  else
    st = solve_direct(P, b, x_user, rtol, maxit, info);
  if (!P->opt.true_residual || (st != MFCG_OK && st != MFCG_NOT_CONVERGED)) return st;
  // ||b - A x||^2 with the FP64 operator, one extra pass
  const int st2 = run_pass(P, MODE_OPERATOR, x_user, P->work, true);
  if (st2 != MFCG_OK) return st2;
  CK(launch_residual_norm(b, P->work, P->nv(), P->partial, &P->state->ticket, &P->state->sums[6], P->exec));
  double rr = 0.0;
  CK(cudaMemcpyAsync(&rr, &P->state->sums[6], sizeof(double), cudaMemcpyDeviceToHost, P->exec));
  CK(cudaStreamSynchronize(P->exec));
  P->launches += 1;
  if (info) {
    info->true_residual_sq = rr;
    info->kernel_launches += 3;
  }
  return st;
}

// ------------------------------------------------------------------ tile autotuning

// Candidate tiles around the default edge T of the degree: T^3, T^2 (T-1),
// T (T-1)^2, (T-1)^3 and (T+1)^3 -- smaller tiles trade halo work for more
// CTAs per SM, larger ones the reverse.
std::vector<std::array<int, 3>> tile_candidates(int degree, int geom_kind, int precision) {
  const int T = default_tile(degree, geom_kind, precision);
  const int lo = degree == 1 ? 2 : 1;
  std::vector<std::array<int, 3>> c;
  auto add = [&](int a, int b, int d) {
    if (a < lo || b < lo || d < lo || a > 16 || b > 16 || d > 16) return;
    const std::array<int, 3> t{a, b, d};
    if (std::find(c.begin(), c.end(), t) == c.end()) c.push_back(t);
  };
  add(T, T, T);
  add(T, T, T - 1);
  add(T, T - 1, T - 1);
  add(T - 1, T - 1, T - 1);
  add(T + 1, T + 1, T + 1);
  return c;
}

int setup_autotuned(const mfcg_mesh* mesh, int degree, const mfcg_geometry* geom, mfcg_options o,
                    void* cuda_stream, mfcg_problem** out) {
  const int kind = geom_kind_of(geom->kind);
  std::array<int, 3> best{0, 0, 0};
  double best_s = 1e300;
  for (const auto& t : tile_candidates(degree, kind, o.precision)) {
    mfcg_options oc = o;
    oc.instrument = 0;
    for (int d = 0; d < 3; ++d) oc.tile[d] = t[d];
    mfcg_problem* Q = nullptr;
    if (mfcg_setup(mesh, degree, geom, &oc, cuda_stream, &Q) != MFCG_OK) continue;  // e.g. too much shared memory
    double* b = nullptr;
    double* x = nullptr;
    const size_t bytes = (size_t)Q->nv() * sizeof(double);
    double secs = 1e300;
    if (cudaMalloc(&b, bytes) == cudaSuccess && cudaMalloc(&x, bytes) == cudaSuccess &&
        mfcg_rhs(Q, b) == MFCG_OK && cudaMemsetAsync(x, 0, bytes, Q->user) == cudaSuccess &&
        mfcg_cg_solve(Q, b, x, 0.0, 2 * Q->graph_iters, nullptr) == MFCG_OK) {
      for (int rep = 0; rep < 2; ++rep) {
        if (cudaStreamSynchronize(Q->user) != cudaSuccess) break;
        const auto t0 = std::chrono::steady_clock::now();
        if (mfcg_cg_solve(Q, b, x, 0.0, 2 * Q->graph_iters, nullptr) != MFCG_OK) break;
        if (cudaStreamSynchronize(Q->user) != cudaSuccess) break;
        secs = std::min(secs, std::chrono::duration<double>(std::chrono::steady_clock::now() - t0).count());
      }
    }
    cudaGetLastError();
    if (b) cudaFree(b);
    if (x) cudaFree(x);
    mfcg_destroy(Q);
    if (secs < best_s) {
      best_s = secs;
      best = t;
    }
  }
  if (best[0] == 0) return MFCG_INVALID_ARG;
  for (int d = 0; d < 3; ++d) o.tile[d] = best[d];
  return mfcg_setup(mesh, degree, geom, &o, cuda_stream, out);
}

// ------------------------------------------------------------------ batches

int batch_capture(mfcg_batch* B) {
  const int count = (int)B->members.size();
  cudaGraph_t graph;
  CK(cudaStreamBeginCapture(B->exec, cudaStreamCaptureModeThreadLocal));
  int st = MFCG_OK;
  if (cudaEventRecord(B->ev_fork, B->exec) != cudaSuccess) st = MFCG_CUDA_ERROR;
  for (int i = 0; i < count && st == MFCG_OK; ++i) {
    mfcg_problem* P = B->members[i];
    if (cudaStreamWaitEvent(P->exec, B->ev_fork, 0) != cudaSuccess) st = MFCG_CUDA_ERROR;
    for (int it = 0; it < B->graph_iters && st == MFCG_OK; ++it)
      st = enqueue_fused_iteration(P, (it & 1) == 0, nullptr, nullptr);
    if (st == MFCG_OK && (cudaEventRecord(B->ev_join[i], P->exec) != cudaSuccess ||
                          cudaStreamWaitEvent(B->exec, B->ev_join[i], 0) != cudaSuccess))
      st = MFCG_CUDA_ERROR;
  }
  if (st == MFCG_OK && launch_gather_done(B->d_states, count, B->d_done, B->exec) != cudaSuccess)
    st = MFCG_CUDA_ERROR;
  const cudaError_t e = cudaStreamEndCapture(B->exec, &graph);
  if (st != MFCG_OK || e != cudaSuccess) return MFCG_CUDA_ERROR;
  const cudaError_t e2 = cudaGraphInstantiate(&B->graph, graph, 0);
  cudaGraphDestroy(graph);
  return e2 == cudaSuccess ? MFCG_OK : MFCG_CUDA_ERROR;
}

// every member's stream waits for the batch stream
int batch_fork(mfcg_batch* B) {
  CK(cudaEventRecord(B->ev_fork, B->exec));
  for (mfcg_problem* P : B->members) CK(cudaStreamWaitEvent(P->exec, B->ev_fork, 0));
  return MFCG_OK;
}

// the batch stream waits for every member's stream
int batch_join(mfcg_batch* B) {
  for (size_t i = 0; i < B->members.size(); ++i) {
    CK(cudaEventRecord(B->ev_join[i], B->members[i]->exec));
    CK(cudaStreamWaitEvent(B->exec, B->ev_join[i], 0));
  }
  return MFCG_OK;
}

// graphs of G iterations of every member until all done flags are set or maxit
int batch_run_iterations(mfcg_batch* B, int maxit) {
  const int count = (int)B->members.size();
  int st;
  if (!B->graph && (st = batch_capture(B)) != MFCG_OK) return st;
  const int G = B->graph_iters;
  const int n_graphs = (maxit + G - 1) / G;
  cudaEvent_t evs[2];
  CK(cudaEventCreateWithFlags(&evs[0], cudaEventDisableTiming));
  CK(cudaEventCreateWithFlags(&evs[1], cudaEventDisableTiming));
  int launched = 0, checked = 0;
  bool finished = n_graphs == 0;
  while (!finished) {
    while (launched < n_graphs && launched < checked + 2) {
      CK(cudaGraphLaunch(B->graph, B->exec));
      CK(cudaMemcpyAsync(B->h_done + (launched & 1) * count, B->d_done, count * sizeof(int), cudaMemcpyDeviceToHost,
                         B->exec));
      CK(cudaEventRecord(evs[launched & 1], B->exec));
      for (mfcg_problem* P : B->members) P->launches += 2LL * G;
      ++launched;
    }
    if (checked >= launched) break;
    CK(cudaEventSynchronize(evs[checked & 1]));
    const int* f = B->h_done + (checked & 1) * count;
    bool all = true;
    for (int i = 0; i < count && all; ++i) all = f[i] != 0;
    if (all) finished = true;
    ++checked;
    if (checked >= n_graphs) finished = true;
  }
  CK(cudaStreamSynchronize(B->exec));
  cudaEventDestroy(evs[0]);
  cudaEventDestroy(evs[1]);
  return MFCG_OK;
}

int batch_solve(mfcg_batch* B, const double* const* b, double* const* x, double rtol, int maxit,
                mfcg_solve_info* infos) {
  const int count = (int)B->members.size();
  const int fixed = rtol == 0.0;
  std::vector<int64_t> launches0(count);
  for (int i = 0; i < count; ++i) launches0[i] = B->members[i]->launches;
  int st;
  // start-up of every member on its own stream
  if ((st = batch_fork(B)) != MFCG_OK) return st;
  for (int i = 0; i < count; ++i) {
    mfcg_problem* P = B->members[i];
    if ((st = fused_initial_residual(P, b[i], x[i])) != MFCG_OK) return st;
    if ((st = fused_start(P, b[i], P->work, rtol, maxit, fixed)) != MFCG_OK) return st;
  }
  if ((st = batch_join(B)) != MFCG_OK) return st;
  if ((st = batch_run_iterations(B, maxit)) != MFCG_OK) return st;
  // finalisation of every member on its own stream
  if ((st = batch_fork(B)) != MFCG_OK) return st;
  for (int i = 0; i < count; ++i) {
    mfcg_problem* P = B->members[i];
    if ((st = fused_finish(P)) != MFCG_OK) return st;
    CK(launch_from_prec(P->cg_prec, P->xs, x[i], P->nv(), 0, P->exec));
    CK(cudaMemcpyAsync(P->h_state, P->state, sizeof(CGState), cudaMemcpyDeviceToHost, P->exec));
    P->launches += 1;
  }
  if ((st = batch_join(B)) != MFCG_OK) return st;
  CK(cudaStreamSynchronize(B->exec));
  int status = MFCG_OK;
  for (int i = 0; i < count; ++i) {
    mfcg_problem* P = B->members[i];
    const CGState& S = *P->h_state;
    int si = MFCG_OK;
    if (S.done == 3) si = MFCG_BREAKDOWN;
    else if (S.done != 1 && !fixed) si = MFCG_NOT_CONVERGED;
    if (status == MFCG_OK) status = si;
    if (infos) fill_info(P, &infos[i], si, S.iterations, IterStats{}, launches0[i], 0);
  }
  return status;
}

}  // namespace

extern "C" {

int mfcg_setup_batch(int count, const mfcg_mesh* meshes, const int* degrees, const mfcg_geometry* geoms,
                     const mfcg_options* opt, void* cuda_stream, mfcg_batch** out) {
  if (!out) return MFCG_INVALID_ARG;
  *out = nullptr;
  if (count < 1 || count > 4096 || !meshes || !degrees || !geoms) return MFCG_INVALID_ARG;
  mfcg_options o{};
  if (opt) o = *opt;
  if (o.mode != MFCG_MODE_FUSED || (o.precision != MFCG_PREC_FP64 && o.precision != MFCG_PREC_DOUBLE_FLOAT) ||
      o.instrument)
    return MFCG_INVALID_ARG;
  mfcg_batch* B = new (std::nothrow) mfcg_batch();
  if (!B) return MFCG_OUT_OF_MEMORY;
  auto fail = [&](int code) {
    mfcg_destroy_batch(B);
    return code;
  };
  if (cudaGetDevice(&B->device) != cudaSuccess) return fail(MFCG_CUDA_ERROR);
  B->user = (cudaStream_t)cuda_stream;
  B->graph_iters = o.graph_iterations ? o.graph_iterations : 16;
  if (B->graph_iters < 0 || (B->graph_iters & 1)) return fail(MFCG_INVALID_ARG);
  B->members.reserve(count);
  for (int i = 0; i < count; ++i) {
    // a member identical to an earlier one shares its geometry and diagonal
    const mfcg_problem* share = nullptr;
    for (int j = 0; j < i && !share; ++j)
      if (degrees[j] == degrees[i] && meshes[j].nx == meshes[i].nx && meshes[j].ny == meshes[i].ny &&
          meshes[j].nz == meshes[i].nz && meshes[j].amplitude == meshes[i].amplitude &&
          geoms[j].kind == geoms[i].kind && geoms[j].coefficient == geoms[i].coefficient &&
          geoms[j].user_data == geoms[i].user_data)
        share = B->members[j];
    mfcg_problem* P = nullptr;
    const int st = setup_impl(&meshes[i], degrees[i], &geoms[i], &o, cuda_stream, &P, share);
    if (st != MFCG_OK) return fail(st);
    B->members.push_back(P);
  }
  if (cudaStreamCreateWithFlags(&B->exec, cudaStreamNonBlocking) != cudaSuccess) return fail(MFCG_CUDA_ERROR);
  if (cudaEventCreateWithFlags(&B->ev_in, cudaEventDisableTiming) != cudaSuccess) return fail(MFCG_CUDA_ERROR);
  if (cudaEventCreateWithFlags(&B->ev_out, cudaEventDisableTiming) != cudaSuccess) return fail(MFCG_CUDA_ERROR);
  if (cudaEventCreateWithFlags(&B->ev_fork, cudaEventDisableTiming) != cudaSuccess) return fail(MFCG_CUDA_ERROR);
  B->ev_join.assign(count, nullptr);
  for (auto& e : B->ev_join)
    if (cudaEventCreateWithFlags(&e, cudaEventDisableTiming) != cudaSuccess) return fail(MFCG_CUDA_ERROR);
  if (cudaMalloc(&B->d_states, count * sizeof(CGState*)) != cudaSuccess) return fail(MFCG_OUT_OF_MEMORY);
  if (cudaMalloc(&B->d_done, count * sizeof(int)) != cudaSuccess) return fail(MFCG_OUT_OF_MEMORY);
  if (cudaMallocHost(&B->h_done, 2 * count * sizeof(int)) != cudaSuccess) return fail(MFCG_OUT_OF_MEMORY);
  std::vector<CGState*> states(count);
  for (int i = 0; i < count; ++i) states[i] = B->members[i]->state;
  if (cudaMemcpy(B->d_states, states.data(), count * sizeof(CGState*), cudaMemcpyHostToDevice) != cudaSuccess)
    return fail(MFCG_CUDA_ERROR);
  *out = B;
  return MFCG_OK;
}

int mfcg_batch_member(mfcg_batch* B, int i, mfcg_problem** prob) {
  if (!B || !prob || i < 0 || i >= (int)B->members.size()) return MFCG_INVALID_ARG;
  *prob = B->members[i];
  return MFCG_OK;
}

int mfcg_cg_solve_batch(mfcg_batch* B, const double* const* b, double* const* x, double rtol, int maxit,
                        mfcg_solve_info* infos) {
  if (!B || !b || !x || maxit < 0 || !(rtol >= 0.0)) return MFCG_INVALID_ARG;
  for (size_t i = 0; i < B->members.size(); ++i)
    if (!b[i] || !x[i] || b[i] == x[i]) return MFCG_INVALID_ARG;
  CK(cudaSetDevice(B->device));
  CK(cudaEventRecord(B->ev_in, B->user));
  CK(cudaStreamWaitEvent(B->exec, B->ev_in, 0));
  const int st = batch_solve(B, b, x, rtol, maxit, infos);
  CK(cudaEventRecord(B->ev_out, B->exec));
  CK(cudaStreamWaitEvent(B->user, B->ev_out, 0));
  return st;
}

int mfcg_destroy_batch(mfcg_batch* B) {
  if (!B) return MFCG_OK;
  cudaSetDevice(B->device);
  if (B->exec) cudaStreamSynchronize(B->exec);
  if (B->graph) cudaGraphExecDestroy(B->graph);
  for (auto it = B->members.rbegin(); it != B->members.rend(); ++it) mfcg_destroy(*it);  // sharers first
  for (cudaEvent_t e : B->ev_join)
    if (e) cudaEventDestroy(e);
  if (B->ev_in) cudaEventDestroy(B->ev_in);
  if (B->ev_out) cudaEventDestroy(B->ev_out);
  if (B->ev_fork) cudaEventDestroy(B->ev_fork);
  if (B->d_states) cudaFree(B->d_states);
  if (B->d_done) cudaFree(B->d_done);
  if (B->h_done) cudaFreeHost(B->h_done);
  if (B->exec) cudaStreamDestroy(B->exec);
  delete B;
  return MFCG_OK;
}

const char* mfcg_status_string(int status) {
  switch (status) {
    case MFCG_OK: return "ok";
    case MFCG_INVALID_ARG: return "invalid argument";
    case MFCG_UNSUPPORTED_DEGREE: return "unsupported polynomial degree (1..8)";
    case MFCG_OUT_OF_MEMORY: return "device allocation failed";
    case MFCG_CUDA_ERROR: return "CUDA runtime error";
    case MFCG_NOT_CONVERGED: return "maximum number of iterations reached";
    case MFCG_BREAKDOWN: return "CG breakdown (non-positive or non-finite inner product)";
    case MFCG_DEVICE_TIMEOUT: return "bounded device wait expired";
    case MFCG_SCRATCH_TOO_SMALL: return "mesh too large for the fixed scratch array of mfcg_apply_operator_static";
    default: return "unknown status";
  }
}

int mfcg_destroy(mfcg_problem* P) {
  if (!P) return MFCG_OK;
  cudaSetDevice(P->device);
  if (P->exec) cudaStreamSynchronize(P->exec);
  if (P->graph_fused) cudaGraphExecDestroy(P->graph_fused);
  if (P->graph_unfused) cudaGraphExecDestroy(P->graph_unfused);
  if (P->graph_semi) cudaGraphExecDestroy(P->graph_semi);
  if (P->graph_loop) cudaGraphExecDestroy(P->graph_loop);
  for (void* q : P->owned) cudaFree(q);
  if (P->h_state) cudaFreeHost(P->h_state);
  if (P->ev_in) cudaEventDestroy(P->ev_in);
  if (P->ev_out) cudaEventDestroy(P->ev_out);
  if (P->exec) cudaStreamDestroy(P->exec);
  delete P;
  return MFCG_OK;
}

int mfcg_setup(const mfcg_mesh* mesh, int degree, const mfcg_geometry* geom, const mfcg_options* opt,
               void* cuda_stream, mfcg_problem** out) {
  return setup_impl(mesh, degree, geom, opt, cuda_stream, out, nullptr);
}

}  // extern "C"

// Set-up of one problem.  With `share` (a problem of the identical definition:
// mesh, degree, geometry and options) the stored geometry and the diagonal,
// its inverse and its converted copy are taken from `share` instead of being
// allocated and computed (batches of right-hand sides on one mesh).
int setup_impl(const mfcg_mesh* mesh, int degree, const mfcg_geometry* geom, const mfcg_options* opt,
               void* cuda_stream, mfcg_problem** out, const mfcg_problem* share) {
  if (!mesh || !geom || !out) return MFCG_INVALID_ARG;
  *out = nullptr;
  if (degree < 1 || degree > kMaxDegree) return MFCG_UNSUPPORTED_DEGREE;
  if (mesh->nx < 1 || mesh->ny < 1 || mesh->nz < 1) return MFCG_INVALID_ARG;
  if (!(std::fabs(mesh->amplitude) < 0.1)) return MFCG_INVALID_ARG;
  if (geom->kind != MFCG_GEOM_AFFINE && geom->kind != MFCG_GEOM_DEFORMED && geom->kind != MFCG_GEOM_DEFORMED_TENSOR &&
      geom->kind != MFCG_GEOM_USER && geom->kind != MFCG_GEOM_DEFORMED_QUADRATIC)
    return MFCG_INVALID_ARG;
  if (geom->kind == MFCG_GEOM_USER && !geom->user_data) return MFCG_INVALID_ARG;
  if (geom->coefficient != MFCG_COEF_CONSTANT && geom->coefficient != MFCG_COEF_SIN_X) return MFCG_INVALID_ARG;
  if (geom->kind == MFCG_GEOM_AFFINE && (mesh->amplitude != 0.0 || geom->coefficient != MFCG_COEF_CONSTANT))
    return MFCG_INVALID_ARG;
  mfcg_options o{};
  if (opt) o = *opt;
  if (o.mode != MFCG_MODE_FUSED && o.mode != MFCG_MODE_UNFUSED && o.mode != MFCG_MODE_SEMI_FUSED &&
      o.mode != MFCG_MODE_LOOP_FUSED)
    return MFCG_INVALID_ARG;
  if (o.preconditioner != MFCG_PRECOND_JACOBI && o.preconditioner != MFCG_PRECOND_NONE) return MFCG_INVALID_ARG;
  if (o.graph_iterations < 0 || (o.graph_iterations & 1)) return MFCG_INVALID_ARG;
  if (o.precision < MFCG_PREC_FP64 || o.precision > MFCG_PREC_DOUBLE_FLOAT_INNER) return MFCG_INVALID_ARG;
  if (inner_precision(o.precision) && o.mode != MFCG_MODE_FUSED) return MFCG_INVALID_ARG;
  if (!(o.inner_rtol >= 0.0 && o.inner_rtol < 1.0)) return MFCG_INVALID_ARG;
  if (o.x_update_every_iteration != 0 && o.x_update_every_iteration != 1) return MFCG_INVALID_ARG;
  if (o.true_residual != 0 && o.true_residual != 1) return MFCG_INVALID_ARG;
  if ((o.components != 0 && o.components != 1 && o.components != 3) || (o.components > 1 && o.mode != MFCG_MODE_FUSED))
    return MFCG_INVALID_ARG;
  if (o.components > 1 && geom->kind == MFCG_GEOM_DEFORMED_QUADRATIC) return MFCG_INVALID_ARG;
  if (o.operator_kind != MFCG_OP_LAPLACE && o.operator_kind != MFCG_OP_MASS) return MFCG_INVALID_ARG;
  if (o.operator_kind == MFCG_OP_MASS && geom->kind == MFCG_GEOM_DEFORMED_TENSOR) return MFCG_INVALID_ARG;
  if (o.fp64_contraction != MFCG_FP64_TENSOR_CORES && o.fp64_contraction != MFCG_FP64_PIPE) return MFCG_INVALID_ARG;
  if (o.tile[0] == -1 && o.tile[1] == -1 && o.tile[2] == -1) return setup_autotuned(mesh, degree, geom, o, cuda_stream, out);
  for (int d = 0; d < 3; ++d)
    if (o.tile[d] < 0 || o.tile[d] > 16) return MFCG_INVALID_ARG;
  const int64_t nn[3] = {(int64_t)degree * mesh->nx + 1, (int64_t)degree * mesh->ny + 1, (int64_t)degree * mesh->nz + 1};
  if (nn[0] > (1 << 20) || nn[1] > (1 << 20) || nn[2] > (1 << 20)) return MFCG_INVALID_ARG;

  mfcg_problem* P = new (std::nothrow) mfcg_problem();
  if (!P) return MFCG_OUT_OF_MEMORY;
  int st = MFCG_OK;
  auto fail = [&](int code) {
    mfcg_destroy(P);
    return code;
  };
  if (cudaGetDevice(&P->device) != cudaSuccess) return fail(MFCG_CUDA_ERROR);
  P->user = (cudaStream_t)cuda_stream;
  P->degree = degree;
  P->mesh = *mesh;
  P->geom = *geom;
  P->opt = o;
  P->ncomp = o.components ? o.components : 1;
  P->op_kind = o.operator_kind == MFCG_OP_MASS ? OP_MASS : OP_LAPLACE;
  P->geom_kind = geom_kind_of(geom->kind);
  P->geom.user_data = nullptr;  // read during set-up only
  // the defect correction forms its outer residual with the native FP64
  // operator: its true-residual floor is 2^5 lower than the double-float one
  P->op_prec = o.precision == MFCG_PREC_DOUBLE_FLOAT ? PREC_DD : PREC_F64;
  P->cg_prec = o.precision == MFCG_PREC_FP64 ? PREC_F64
               : (o.precision == MFCG_PREC_DOUBLE_FLOAT || o.precision == MFCG_PREC_DOUBLE_FLOAT_INNER ? PREC_DD
                                                                                                   : PREC_F32);
  P->graph_iters = o.graph_iterations ? o.graph_iterations : 16;
  if (cudaStreamCreateWithFlags(&P->exec, cudaStreamNonBlocking) != cudaSuccess) return fail(MFCG_CUDA_ERROR);
  if (cudaEventCreateWithFlags(&P->ev_in, cudaEventDisableTiming) != cudaSuccess) return fail(MFCG_CUDA_ERROR);
  if (cudaEventCreateWithFlags(&P->ev_out, cudaEventDisableTiming) != cudaSuccess) return fail(MFCG_CUDA_ERROR);

  TileGeom& g = P->g;
  const int N[3] = {mesh->nx, mesh->ny, mesh->nz};
  int T[3];
  for (int d = 0; d < 3; ++d) {
    T[d] = o.tile[d] ? o.tile[d] : default_tile(degree, P->geom_kind, o.precision);
    if (degree == 1 && T[d] < 2) T[d] = 2;
  }
  // FP64 on the tensor cores at degree 4: 4 x 4 x 3-cell tiles, whose bricks
  // and staging fit two CTAs per SM (4^3 fits one)
  if (degree == 4 && P->geom_kind == GEOM_AFFINE && o.precision == MFCG_PREC_FP64 &&
      o.fp64_contraction == MFCG_FP64_TENSOR_CORES && o.tile[2] == 0)
    T[2] = 3;
  init_tile_geom(degree, N, T, g, P->fam, &P->tdiv);
  int max_smem = 0;
  cudaDeviceGetAttribute(&max_smem, cudaDevAttrMaxSharedMemoryPerBlockOptin, P->device);
  const size_t static_smem = 8 * (kThreads / 32) * sizeof(double) + 2 * 512 * sizeof(int);
  // the tensor-core contractions where their staging fits next to the node
  // bricks (with the default tiles: degrees 1 to 7), else the FP64 sweeps
  P->tc = P->geom_kind == GEOM_AFFINE && o.fp64_contraction == MFCG_FP64_TENSOR_CORES && tc::tc_degree(degree) &&
          tile_smem_bytes(degree, P->geom_kind, PREC_F64TC, g) + static_smem <= (size_t)max_smem;
  const int precs[4] = {PREC_F64, P->op_prec, P->cg_prec, P->tc ? PREC_F64TC : PREC_F64};
  for (int pr : precs) {
    const size_t smem = tile_smem_bytes(degree, P->geom_kind, pr, g);
    if (smem + static_smem > (size_t)max_smem) return fail(MFCG_INVALID_ARG);
    if (prepare_tile(degree, P->geom_kind, pr, smem) != cudaSuccess) return fail(MFCG_CUDA_ERROR);
  }
  // prefetch distance of the operator passes: the CTAs resident in one wave
  // (the fused CG kernel has no look-ahead prefetch)
  int n_sm = 0;
  cudaDeviceGetAttribute(&n_sm, cudaDevAttrMultiProcessorCount, P->device);
  const int op_launch_prec = P->tc && P->op_prec == PREC_F64 ? PREC_F64TC : P->op_prec;
  P->ahead_op = n_sm * tile_occupancy(degree, MODE_OPERATOR, P->geom_kind, op_launch_prec, P->ncomp,
                                      tile_smem_bytes(degree, P->geom_kind, op_launch_prec, g, MODE_OPERATOR));
  // fused FP64 iterations on the tensor cores, two CTAs per SM: the first
  // wave's second CTA on each SM (blockIdx in [n_sm, 2 n_sm)) starts about
  // half a tile later (80,000 clocks for the 17 x 17 x 13-node brick of
  // degree 4, the best of 0-110,000 measured on Q4 128^3: +8 %), scaled by the
  // brick's node count for other tiles.  The delay costs about half a tile
  // once per launch, so it is applied only to launches of at least eight waves.
  if (P->tc && P->cg_prec == PREC_F64 && g.n_tiles >= 16LL * n_sm &&
      tile_occupancy(degree, MODE_CG, P->geom_kind, PREC_F64TC, P->ncomp,
                     tile_smem_bytes(degree, P->geom_kind, PREC_F64TC, g, MODE_CG)) == 2) {
    const double nodes = (double)(degree * g.T[0] + 1) * (degree * g.T[1] + 1) * (degree * g.T[2] + 1);
    P->stagger_lo = n_sm;
    P->stagger_hi = 2 * n_sm;
    P->stagger_cycles = (long long)(80000.0 * nodes / (17.0 * 17.0 * 13.0));
  }
  P->tail_nodes = P->fam[0] + P->fam[1] + P->fam[2];
  // about four shared-face nodes per tail thread (two iterations of two)
  P->tail_ctas = (int)std::min<int64_t>(std::max<int64_t>((P->tail_nodes + 4 * kThreads - 1) / (4 * kThreads), 1), 152 * 16);

  const double h[3] = {1.0 / N[0], 1.0 / N[1], 1.0 / N[2]};
  build_coeffs(degree, h, mesh->amplitude, geom->coefficient, P->c);
  if (P->tc) {
    // digit fragments of the cell matrix for the tensor-core operator
    std::vector<uint2> frag;
    if (build_tc_fragments(degree, P->c, P->op_kind, frag, P->tc_g2, P->tc_r) != 0) return fail(MFCG_INVALID_ARG);
    if ((st = alloc_bytes(P, &P->tc_frag, (int64_t)(frag.size() * sizeof(uint2)))) != MFCG_OK) return fail(st);
    if (cudaMemcpy(P->tc_frag, frag.data(), frag.size() * sizeof(uint2), cudaMemcpyHostToDevice) != cudaSuccess)
      return fail(MFCG_CUDA_ERROR);
  }

  const int64_t n = g.n_dofs;     // nodes (scalar set-up passes)
  const int64_t n8 = P->nv() * 8; // bytes of an FP64 vector of the ABI
  const int fused = o.mode == MFCG_MODE_FUSED;
  if (fused) {
    for (int i = 0; i < 2 && st == MFCG_OK; ++i) {
      if ((st = alloc_bytes(P, &P->r[i], n8)) != MFCG_OK) break;
      if ((st = alloc_bytes(P, &P->p[i], n8)) != MFCG_OK) break;
      st = alloc_bytes(P, &P->v[i], n8);
    }
    if (st == MFCG_OK) st = alloc_bytes(P, &P->xs, n8);
    if (st == MFCG_OK && !share) st = alloc_bytes(P, &P->dinv_s, n8);
    if (st == MFCG_OK && inner_precision(o.precision)) st = alloc_bytes(P, &P->x, n8);
  } else {
    if (st == MFCG_OK) st = alloc_bytes(P, &P->x, n8);
    if (st == MFCG_OK) st = alloc_bytes(P, &P->z, n8);
    if (st == MFCG_OK) st = alloc_bytes(P, &P->ur, n8);
    if (st == MFCG_OK) st = alloc_bytes(P, &P->up, n8);
    if (st == MFCG_OK) st = alloc_bytes(P, &P->uv, n8);
  }
  if (st == MFCG_OK) st = alloc_bytes(P, &P->work, n8);
  if (st == MFCG_OK && !share) st = alloc_bytes(P, &P->diag, n8);
  if (st == MFCG_OK && !share) st = alloc_bytes(P, &P->diag_inv, n8);
  if (st == MFCG_OK) st = alloc_bytes(P, &P->shell, P->ncomp * g.n_tiles * g.face_stride * 8);
  const int64_t nparts = std::max<int64_t>(g.n_tiles + P->tail_ctas, 152 * 8);
  if (st == MFCG_OK) st = alloc_bytes(P, &P->partial, nparts * 8 * 8);
  const int64_t ngeo = (int64_t)N[0] * N[1] * N[2] * geo_per_cell(P->geom_kind, degree);
  if (share) {
    P->geo = share->geo;
    P->geo_op = share->geo_op;
    P->geo_cg = share->geo_cg;
    P->diag = share->diag;
    P->diag_inv = share->diag_inv;
    P->dinv_s = share->dinv_s;
  }
  if (st == MFCG_OK && P->geom_kind != GEOM_AFFINE && !share) {
    st = alloc_bytes(P, &P->geo, ngeo * 8);
    if (st == MFCG_OK && P->op_prec != PREC_F64) st = alloc_bytes(P, &P->geo_op, ngeo * 8);
    if (st == MFCG_OK && P->cg_prec != PREC_F64 && P->cg_prec != P->op_prec)
      st = alloc_bytes(P, &P->geo_cg, ngeo * prec_bytes(P->cg_prec));
  }
  if (st != MFCG_OK) return fail(st);
  if (P->geom_kind != GEOM_AFFINE) {
    if (!P->geo_op) P->geo_op = P->geo;
    if (!P->geo_cg) P->geo_cg = P->cg_prec == PREC_F64 ? (void*)P->geo : P->geo_op;
  }
  if (alloc_bytes(P, &P->state, sizeof(CGState)) != MFCG_OK) return fail(MFCG_OUT_OF_MEMORY);
  if (cudaMallocHost(&P->h_state, 2 * sizeof(CGState)) != cudaSuccess) return fail(MFCG_OUT_OF_MEMORY);
  if (cudaMemsetAsync(P->state, 0, sizeof(CGState), P->exec) != cudaSuccess) return fail(MFCG_CUDA_ERROR);
  if (enter(P) != MFCG_OK) return fail(MFCG_CUDA_ERROR);
  if (share) {
    // geometry and diagonal come from the identical problem
    if (cudaStreamSynchronize(P->exec) != cudaSuccess) return fail(MFCG_CUDA_ERROR);
    if (leave(P) != MFCG_OK) return fail(MFCG_CUDA_ERROR);
    *out = P;
    return MFCG_OK;
  }
  if (P->geom_kind != GEOM_AFFINE) {
    if (geom->kind == MFCG_GEOM_USER) {
      if (cudaMemcpyAsync(P->geo, geom->user_data, ngeo * sizeof(double), cudaMemcpyHostToDevice, P->exec) !=
          cudaSuccess)
        return fail(MFCG_CUDA_ERROR);
    } else if (launch_geometry(g, P->c, P->geom_kind, P->geo, P->exec) != cudaSuccess) {
      return fail(MFCG_CUDA_ERROR);
    }
    if (P->geo_op != P->geo && launch_to_prec(P->op_prec, P->geo, P->geo_op, ngeo, P->exec) != cudaSuccess)
      return fail(MFCG_CUDA_ERROR);
    if (P->geo_cg != P->geo && P->geo_cg != P->geo_op &&
        launch_to_prec(P->cg_prec, P->geo, P->geo_cg, ngeo, P->exec) != cudaSuccess)
      return fail(MFCG_CUDA_ERROR);
  }
  // Jacobi preconditioner: exact diagonal and its inverse (FP64, converted for the fused CG)
  if ((st = run_pass(P, MODE_DIAG, nullptr, P->diag)) != MFCG_OK) return fail(st);
  // vector-valued operator: every component has the scalar diagonal (the
  // fused kernels read the first copy for all components)
  for (int comp = 1; comp < P->ncomp; ++comp)
    if (cudaMemcpyAsync(P->diag + comp * n, P->diag, n * sizeof(double), cudaMemcpyDeviceToDevice, P->exec) !=
        cudaSuccess)
      return fail(MFCG_CUDA_ERROR);
  const int64_t nvec = P->nv();
  if (o.preconditioner == MFCG_PRECOND_NONE) {
    if (launch_fill(P->diag_inv, 1.0, nvec, P->exec) != cudaSuccess) return fail(MFCG_CUDA_ERROR);
  } else if (launch_invert(P->diag, P->diag_inv, nvec, P->exec) != cudaSuccess) {
    return fail(MFCG_CUDA_ERROR);
  }
  if (fused && launch_to_prec(P->cg_prec, P->diag_inv, P->dinv_s, nvec, P->exec) != cudaSuccess)
    return fail(MFCG_CUDA_ERROR);
  if (cudaStreamSynchronize(P->exec) != cudaSuccess) return fail(MFCG_CUDA_ERROR);
  if (leave(P) != MFCG_OK) return fail(MFCG_CUDA_ERROR);
  *out = P;
  return MFCG_OK;
}

extern "C" {

int mfcg_n_dofs(const mfcg_problem* P, int64_t* n) {
  if (!P || !n) return MFCG_INVALID_ARG;
  *n = P->nv();
  return MFCG_OK;
}

int mfcg_apply_operator(mfcg_problem* P, const double* src, double* dst) {
  if (!P || !src || !dst || src == dst) return MFCG_INVALID_ARG;
  int st;
  if ((st = enter(P)) != MFCG_OK) return st;
  if ((st = run_pass(P, MODE_OPERATOR, src, dst)) != MFCG_OK) return st;
  return leave(P);
}

int mfcg_diagonal(mfcg_problem* P, double* diag) {
  if (!P || !diag) return MFCG_INVALID_ARG;
  int st;
  if ((st = enter(P)) != MFCG_OK) return st;
  CK(cudaMemcpyAsync(diag, P->diag, P->nv() * sizeof(double), cudaMemcpyDeviceToDevice, P->exec));
  return leave(P);
}

int mfcg_rhs(mfcg_problem* P, double* b) {
  if (!P || !b || P->geom.kind == MFCG_GEOM_USER) return MFCG_INVALID_ARG;
  int st;
  if ((st = enter(P)) != MFCG_OK) return st;
  if ((st = run_pass(P, MODE_RHS, nullptr, b)) != MFCG_OK) return st;
  // component c of a vector-valued problem: (c + 1) times the scalar b (u*_c = (c + 1) u*)
  for (int comp = 1; comp < P->ncomp; ++comp)
    CK(launch_scale(b, b + comp * P->g.n_dofs, (double)(comp + 1), P->g.n_dofs, P->exec));
  return leave(P);
}

int mfcg_cg_solve(mfcg_problem* P, const double* b, double* x, double rtol, int maxit, mfcg_solve_info* info) {
  if (!P || !b || !x || b == x || maxit < 0 || !(rtol >= 0.0)) return MFCG_INVALID_ARG;
  int st;
  if ((st = enter(P)) != MFCG_OK) return st;
  st = solve_impl(P, b, x, rtol, maxit, info);
  const int st2 = leave(P);
  return st != MFCG_OK ? st : st2;
}

int mfcg_cg_solve_host(mfcg_problem* P, const double* b_host, double* x_host, double rtol, int maxit,
                       mfcg_solve_info* info) {
  if (!P || !b_host || !x_host || maxit < 0 || !(rtol >= 0.0)) return MFCG_INVALID_ARG;
  const int64_t n = P->nv();
  int st;
  if ((st = enter(P)) != MFCG_OK) return st;
  if (!P->bdev && (st = alloc_bytes(P, &P->bdev, n * 8)) != MFCG_OK) return st;
  if (!P->xdev && (st = alloc_bytes(P, &P->xdev, n * 8)) != MFCG_OK) return st;
  CK(cudaMemcpyAsync(P->bdev, b_host, n * sizeof(double), cudaMemcpyHostToDevice, P->exec));
  CK(cudaMemcpyAsync(P->xdev, x_host, n * sizeof(double), cudaMemcpyHostToDevice, P->exec));
  st = solve_impl(P, P->bdev, P->xdev, rtol, maxit, info);
  if (st != MFCG_OK && st != MFCG_NOT_CONVERGED && st != MFCG_BREAKDOWN) return st;
  CK(cudaMemcpyAsync(x_host, P->xdev, n * sizeof(double), cudaMemcpyDeviceToHost, P->exec));
  CK(cudaStreamSynchronize(P->exec));
  const int st2 = leave(P);
  return st != MFCG_OK ? st : st2;
}

int mfcg_to_lexicographic(mfcg_problem* P, const double* in, double* out) {
  if (!P || !in || !out || in == out) return MFCG_INVALID_ARG;
  int st;
  if ((st = enter(P)) != MFCG_OK) return st;
  for (int comp = 0; comp < P->ncomp; ++comp)
    CK(launch_reorder(P->g, in + comp * P->g.n_dofs, out + comp * P->g.n_dofs, 1, P->exec));
  return leave(P);
}

int mfcg_from_lexicographic(mfcg_problem* P, const double* in, double* out) {
  if (!P || !in || !out || in == out) return MFCG_INVALID_ARG;
  int st;
  if ((st = enter(P)) != MFCG_OK) return st;
  for (int comp = 0; comp < P->ncomp; ++comp)
    CK(launch_reorder(P->g, in + comp * P->g.n_dofs, out + comp * P->g.n_dofs, 0, P->exec));
  return leave(P);
}

}  // extern "C"
