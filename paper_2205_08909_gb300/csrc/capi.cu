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
#include <cmath>
#include <cstdlib>
#include <cstring>
#include <new>
#include <vector>

#include "mfcg_internal.h"
#include "precision.cuh"

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
  int op_prec = PREC_F64;  // apply_operator and FP64-accurate residuals
  int cg_prec = PREC_F64;  // fused CG iterations
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
  int graph_iters = 16;
  cudaGraphExec_t graph_fused = nullptr;
  cudaGraphExec_t graph_unfused = nullptr;
  cudaGraphExec_t graph_semi = nullptr;
  int64_t launches = 0;
  std::vector<void*> owned;  // every device allocation
};

namespace {

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

// default tile edge (cells) per degree: node bricks of about 17^3
int default_tile(int p, int geom) {
  static const int affine[9] = {0, 16, 8, 5, 4, 3, 3, 2, 2};
  static const int deformed[9] = {0, 8, 4, 4, 3, 2, 2, 2, 2};
  return geom == GEOM_AFFINE ? affine[p] : deformed[p];
}

TileArgs base_args(const mfcg_problem* P, int prec, const void* geo) {
  TileArgs a{};
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
  return a;
}

// operator-like pass (tile kernel + tail) with FP64 input/output
int run_pass(mfcg_problem* P, int mode, const double* src, double* dst) {
  const int prec = mode == MODE_OPERATOR ? P->op_prec : PREC_F64;
  TileArgs a = base_args(P, prec, mode == MODE_OPERATOR ? P->geo_op : P->geo);
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
  TileArgs a = base_args(P, P->cg_prec, P->geo_cg);
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
  u.n = P->g.n_dofs;
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
  TileArgs a = base_args(P, P->op_prec, P->geo_op);
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

// semi-fused Algorithm 5: "pre" kernel, operator (tile + tail), "post" kernel
int enqueue_semi_iteration(mfcg_problem* P, cudaEvent_t t0, cudaEvent_t t1) {
  const int64_t n = P->g.n_dofs;
  CK(launch_semi_pre(n, P->state, P->x, P->ur, P->up, P->uv, P->diag_inv, P->exec));
  TileArgs a = base_args(P, P->op_prec, P->geo_op);
  a.in0 = P->up;
  a.out0 = P->uv;
  if (t0) CK(cudaEventRecord(t0, P->exec));
  CK(launch_tile(P->degree, MODE_OPERATOR, a, P->c, P->exec));
  if (t1) CK(cudaEventRecord(t1, P->exec));
  CK(launch_tail(P->degree, MODE_OPERATOR, a, P->exec));
  CK(launch_semi_post(n, P->state, P->ur, P->up, P->uv, P->diag_inv, P->partial, P->exec));
  return MFCG_OK;
}

enum IterKind { ITER_FUSED = 0, ITER_UNFUSED = 1, ITER_SEMI = 2 };
constexpr int kLaunchesPerIter[3] = {2, 9, 4};

int enqueue_iteration(mfcg_problem* P, int kind, int odd, cudaEvent_t t0, cudaEvent_t t1) {
  if (kind == ITER_FUSED) return enqueue_fused_iteration(P, odd, t0, t1);
  if (kind == ITER_UNFUSED) return enqueue_unfused_iteration(P, t0, t1);
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
  cudaGraphExec_t* gexec = kind == ITER_FUSED ? &P->graph_fused : (kind == ITER_UNFUSED ? &P->graph_unfused : &P->graph_semi);
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
int fused_core(mfcg_problem* P, const double* b, const double* r0, double rtol, int maxit, int fixed,
               IterStats& stats) {
  const int64_t n = P->g.n_dofs;
  const size_t es = prec_bytes(P->cg_prec);
  CK(launch_cg_init(P->state, b, r0, n, rtol, maxit, fixed, P->partial, 0, P->exec));
  CK(launch_to_prec(P->cg_prec, r0, P->r[0], n, P->exec));
  CK(cudaMemsetAsync(P->p[0], 0, n * es, P->exec));
  CK(cudaMemsetAsync(P->v[0], 0, n * es, P->exec));
  P->launches += 2;
  int st = run_iterations(P, ITER_FUSED, maxit, stats);
  if (st != MFCG_OK) return st;
  CK(launch_finalize_fused(P->cg_prec, n, P->state, P->xs, P->p[0], P->p[1], P->r[0], P->r[1], P->dinv_s, P->exec));
  P->launches += 1;
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
}

int solve_direct(mfcg_problem* P, const double* b, double* x_user, double rtol, int maxit, mfcg_solve_info* info) {
  const int64_t n = P->g.n_dofs;
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
    if ((st = fused_core(P, b, P->work, rtol, maxit, fixed, stats)) != MFCG_OK) return st;
    CK(launch_from_prec(P->cg_prec, P->xs, x_user, n, 0, P->exec));
    P->launches += 2;
  } else if (P->opt.mode == MFCG_MODE_SEMI_FUSED) {
    CK(cudaMemcpyAsync(P->x, x_user, n * sizeof(double), cudaMemcpyDeviceToDevice, P->exec));
    CK(cudaMemcpyAsync(P->ur, P->work, n * sizeof(double), cudaMemcpyDeviceToDevice, P->exec));
    CK(cudaMemsetAsync(P->up, 0, n * sizeof(double), P->exec));
    CK(cudaMemsetAsync(P->uv, 0, n * sizeof(double), P->exec));
    CK(launch_cg_init(P->state, b, P->ur, n, rtol, maxit, fixed, P->partial, 0, P->exec));
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
    if ((st = run_iterations(P, ITER_UNFUSED, maxit, stats)) != MFCG_OK) return st;
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
// the FP32 fused CG to a relative reduction inner_rtol; the true residual is
// formed with the FP64 operator and FP64 vectors.
int solve_defect_correction(mfcg_problem* P, const double* b, double* x_user, double rtol, int maxit,
                            mfcg_solve_info* info) {
  const int64_t n = P->g.n_dofs;
  const int64_t launches0 = P->launches;
  const double inner = P->opt.inner_rtol > 0.0 ? P->opt.inner_rtol : 1e-3;
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
    CK(launch_cg_init(P->state, P->work, P->work, n, inner, std::max(maxit - total_it, 1), 0, P->partial, 0,
                      P->exec));
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
  const int64_t n = P->g.n_dofs;
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
  if (P->opt.precision == MFCG_PREC_FP32_INNER) {
    if (rtol == 0.0) return solve_fixed_inner(P, b, x_user, maxit, info);
    return solve_defect_correction(P, b, x_user, rtol, maxit, info);
  }
  return solve_direct(P, b, x_user, rtol, maxit, info);
}

}  // namespace

extern "C" {

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
  if (!mesh || !geom || !out) return MFCG_INVALID_ARG;
  *out = nullptr;
  if (degree < 1 || degree > kMaxDegree) return MFCG_UNSUPPORTED_DEGREE;
  if (mesh->nx < 1 || mesh->ny < 1 || mesh->nz < 1) return MFCG_INVALID_ARG;
  if (!(std::fabs(mesh->amplitude) < 0.1)) return MFCG_INVALID_ARG;
  if (geom->kind != MFCG_GEOM_AFFINE && geom->kind != MFCG_GEOM_DEFORMED && geom->kind != MFCG_GEOM_DEFORMED_TENSOR)
    return MFCG_INVALID_ARG;
  if (geom->coefficient != MFCG_COEF_CONSTANT && geom->coefficient != MFCG_COEF_SIN_X) return MFCG_INVALID_ARG;
  if (geom->kind == MFCG_GEOM_AFFINE && (mesh->amplitude != 0.0 || geom->coefficient != MFCG_COEF_CONSTANT))
    return MFCG_INVALID_ARG;
  mfcg_options o{};
  if (opt) o = *opt;
  if (o.mode != MFCG_MODE_FUSED && o.mode != MFCG_MODE_UNFUSED && o.mode != MFCG_MODE_SEMI_FUSED)
    return MFCG_INVALID_ARG;
  if (o.preconditioner != MFCG_PRECOND_JACOBI && o.preconditioner != MFCG_PRECOND_NONE) return MFCG_INVALID_ARG;
  if (o.graph_iterations < 0 || (o.graph_iterations & 1)) return MFCG_INVALID_ARG;
  if (o.precision < MFCG_PREC_FP64 || o.precision > MFCG_PREC_FP32_INNER) return MFCG_INVALID_ARG;
  if (o.precision == MFCG_PREC_FP32_INNER && o.mode != MFCG_MODE_FUSED) return MFCG_INVALID_ARG;
  if (!(o.inner_rtol >= 0.0 && o.inner_rtol < 1.0)) return MFCG_INVALID_ARG;
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
  P->geom_kind = geom->kind == MFCG_GEOM_AFFINE ? GEOM_AFFINE
                  : (geom->kind == MFCG_GEOM_DEFORMED_TENSOR ? GEOM_TENSOR : GEOM_DEFORMED);
  // the defect correction forms its outer residual with the native FP64
  // operator: its true-residual floor is 2^5 lower than the double-float one
  P->op_prec = o.precision == MFCG_PREC_DOUBLE_FLOAT ? PREC_DD : PREC_F64;
  P->cg_prec = o.precision == MFCG_PREC_FP64 ? PREC_F64 : (o.precision == MFCG_PREC_DOUBLE_FLOAT ? PREC_DD : PREC_F32);
  P->graph_iters = o.graph_iterations ? o.graph_iterations : 16;
  if (cudaStreamCreateWithFlags(&P->exec, cudaStreamNonBlocking) != cudaSuccess) return fail(MFCG_CUDA_ERROR);
  if (cudaEventCreateWithFlags(&P->ev_in, cudaEventDisableTiming) != cudaSuccess) return fail(MFCG_CUDA_ERROR);
  if (cudaEventCreateWithFlags(&P->ev_out, cudaEventDisableTiming) != cudaSuccess) return fail(MFCG_CUDA_ERROR);

  TileGeom& g = P->g;
  const int N[3] = {mesh->nx, mesh->ny, mesh->nz};
  int T[3];
  for (int d = 0; d < 3; ++d) {
    T[d] = o.tile[d] ? o.tile[d] : default_tile(degree, P->geom_kind);
    if (degree == 1 && T[d] < 2) T[d] = 2;
  }
  init_tile_geom(degree, N, T, g, P->fam, &P->tdiv);
  int max_smem = 0;
  cudaDeviceGetAttribute(&max_smem, cudaDevAttrMaxSharedMemoryPerBlockOptin, P->device);
  const int precs[3] = {PREC_F64, P->op_prec, P->cg_prec};
  for (int pr : precs) {
    const size_t smem = tile_smem_bytes(degree, P->geom_kind, pr, g);
    const size_t static_smem = 8 * (kThreads / 32) * sizeof(double) + 2 * 512 * sizeof(int);
    if (smem + static_smem > (size_t)max_smem) return fail(MFCG_INVALID_ARG);
    if (prepare_tile(degree, P->geom_kind, pr, smem) != cudaSuccess) return fail(MFCG_CUDA_ERROR);
  }
  P->tail_nodes = P->fam[0] + P->fam[1] + P->fam[2];
  P->tail_ctas = (int)std::min<int64_t>(std::max<int64_t>((P->tail_nodes + 2 * kThreads - 1) / (2 * kThreads), 1), 152 * 32);

  const double h[3] = {1.0 / N[0], 1.0 / N[1], 1.0 / N[2]};
  build_coeffs(degree, h, mesh->amplitude, geom->coefficient, P->c);

  const int64_t n = g.n_dofs;
  const int64_t n8 = n * 8;
  const int fused = o.mode == MFCG_MODE_FUSED;
  if (fused) {
    for (int i = 0; i < 2 && st == MFCG_OK; ++i) {
      if ((st = alloc_bytes(P, &P->r[i], n8)) != MFCG_OK) break;
      if ((st = alloc_bytes(P, &P->p[i], n8)) != MFCG_OK) break;
      st = alloc_bytes(P, &P->v[i], n8);
    }
    if (st == MFCG_OK) st = alloc_bytes(P, &P->xs, n8);
    if (st == MFCG_OK) st = alloc_bytes(P, &P->dinv_s, n8);
    if (st == MFCG_OK && o.precision == MFCG_PREC_FP32_INNER) st = alloc_bytes(P, &P->x, n8);
  } else {
    if (st == MFCG_OK) st = alloc_bytes(P, &P->x, n8);
    if (st == MFCG_OK) st = alloc_bytes(P, &P->z, n8);
    if (st == MFCG_OK) st = alloc_bytes(P, &P->ur, n8);
    if (st == MFCG_OK) st = alloc_bytes(P, &P->up, n8);
    if (st == MFCG_OK) st = alloc_bytes(P, &P->uv, n8);
  }
  if (st == MFCG_OK) st = alloc_bytes(P, &P->work, n8);
  if (st == MFCG_OK) st = alloc_bytes(P, &P->diag, n8);
  if (st == MFCG_OK) st = alloc_bytes(P, &P->diag_inv, n8);
  if (st == MFCG_OK) st = alloc_bytes(P, &P->shell, g.n_tiles * g.face_stride * 8);
  const int64_t nparts = std::max<int64_t>(g.n_tiles + P->tail_ctas, 152 * 8);
  if (st == MFCG_OK) st = alloc_bytes(P, &P->partial, nparts * 8 * 8);
  const int64_t ngeo =
      (int64_t)N[0] * N[1] * N[2] * geo_values(P->geom_kind) * (degree + 1) * (degree + 1) * (degree + 1);
  if (st == MFCG_OK && P->geom_kind != GEOM_AFFINE) {
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
  if (P->geom_kind != GEOM_AFFINE) {
    if (launch_geometry(g, P->c, P->geom_kind, P->geo, P->exec) != cudaSuccess) return fail(MFCG_CUDA_ERROR);
    if (P->geo_op != P->geo && launch_to_prec(P->op_prec, P->geo, P->geo_op, ngeo, P->exec) != cudaSuccess)
      return fail(MFCG_CUDA_ERROR);
    if (P->geo_cg != P->geo && P->geo_cg != P->geo_op &&
        launch_to_prec(P->cg_prec, P->geo, P->geo_cg, ngeo, P->exec) != cudaSuccess)
      return fail(MFCG_CUDA_ERROR);
  }
  // Jacobi preconditioner: exact diagonal and its inverse (FP64, converted for the fused CG)
  if ((st = run_pass(P, MODE_DIAG, nullptr, P->diag)) != MFCG_OK) return fail(st);
  if (o.preconditioner == MFCG_PRECOND_NONE) {
    if (launch_fill(P->diag_inv, 1.0, n, P->exec) != cudaSuccess) return fail(MFCG_CUDA_ERROR);
  } else if (launch_invert(P->diag, P->diag_inv, n, P->exec) != cudaSuccess) {
    return fail(MFCG_CUDA_ERROR);
  }
  if (fused && launch_to_prec(P->cg_prec, P->diag_inv, P->dinv_s, n, P->exec) != cudaSuccess)
    return fail(MFCG_CUDA_ERROR);
  if (cudaStreamSynchronize(P->exec) != cudaSuccess) return fail(MFCG_CUDA_ERROR);
  if (leave(P) != MFCG_OK) return fail(MFCG_CUDA_ERROR);
  *out = P;
  return MFCG_OK;
}

int mfcg_n_dofs(const mfcg_problem* P, int64_t* n) {
  if (!P || !n) return MFCG_INVALID_ARG;
  *n = P->g.n_dofs;
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
  CK(cudaMemcpyAsync(diag, P->diag, P->g.n_dofs * sizeof(double), cudaMemcpyDeviceToDevice, P->exec));
  return leave(P);
}

int mfcg_rhs(mfcg_problem* P, double* b) {
  if (!P || !b) return MFCG_INVALID_ARG;
  int st;
  if ((st = enter(P)) != MFCG_OK) return st;
  if ((st = run_pass(P, MODE_RHS, nullptr, b)) != MFCG_OK) return st;
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
  const int64_t n = P->g.n_dofs;
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
  CK(launch_reorder(P->g, in, out, 1, P->exec));
  return leave(P);
}

int mfcg_from_lexicographic(mfcg_problem* P, const double* in, double* out) {
  if (!P || !in || !out || in == out) return MFCG_INVALID_ARG;
  int st;
  if ((st = enter(P)) != MFCG_OK) return st;
  CK(launch_reorder(P->g, in, out, 0, P->exec));
  return leave(P);
}

}  // extern "C"
