/*
 * mfcg.h -- C ABI of the fused matrix-free Jacobi-CG library for GB300 (sm_103a).
 *
 * The library solves A u = b for the continuous Q_p finite-element
 * discretisation of -div(a grad u) = f on the unit cube with homogeneous
 * Dirichlet data (Sec. 2, Eqs. 1-3), where the action of A is evaluated
 * matrix-free as a sum of cell contributions (Eq. 4) with the cell integrals
 * of Eq. 5 computed by sum factorisation on the tensor-product Gauss rule with
 * p+1 points per direction, and the solver is the preconditioned CG with
 * merged vector operations (Algorithm 5) whose vector updates and seven inner
 * products run inside the operator pass (Sec. 5).
 *
 * Conventions shared by every entry point
 * ---------------------------------------
 *  - Vectors are arrays of n doubles, n = (p*Nx+1)(p*Ny+1)(p*Nz+1), one per mesh
 *    node including the Dirichlet nodes, in the library's tile-blocked DoF
 *    ordering (the nodes each tile of cells owns are contiguous, its lower x
 *    face first; see mfcg_to_lexicographic for the conversion); with
 *    components = 3 the components follow one another.  Dirichlet nodes stay in the
 *    system as identity rows (Sec. 5.3): (A u)_i = u_i there.
 *  - Unless the name ends in _host, pointers are DEVICE pointers on the device
 *    that was current at mfcg_setup; the caller owns them and keeps them alive
 *    until the call's work has finished on the problem's stream.
 *  - All device work is enqueued on the stream given to mfcg_setup.  Calls that
 *    return results to the host (cg_solve, n_dofs) synchronise that stream.
 *  - Every function returns an mfcg_status code; no exception or abort crosses
 *    the ABI.  After MFCG_CUDA_ERROR the problem must be destroyed.
 */
#ifndef MFCG_H
#define MFCG_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef enum mfcg_status {
  MFCG_OK = 0,
  MFCG_INVALID_ARG = 1,          /* null pointer, bad size, bad enum value          */
  MFCG_UNSUPPORTED_DEGREE = 2,   /* degree outside 1..8                              */
  MFCG_OUT_OF_MEMORY = 3,        /* a device allocation failed                       */
  MFCG_CUDA_ERROR = 4,           /* a CUDA runtime call failed                        */
  MFCG_NOT_CONVERGED = 5,        /* maxit reached before the tolerance               */
  MFCG_BREAKDOWN = 6,            /* p^T A p <= 0, r^T M^-1 r <= 0 or a non-finite sum */
  MFCG_DEVICE_TIMEOUT = 7,       /* a bounded device-side wait gave up               */
  MFCG_SCRATCH_TOO_SMALL = 8     /* the mesh needs more scratch than the fixed array of
                                    mfcg_apply_operator_static holds                    */
} mfcg_status;

/* Mesh of Nx x Ny x Nz box cells on [0,1]^3.  amplitude A deforms the mesh by
 * x = X + A sin(2 pi X) sin(2 pi Y) sin(2 pi Z) on every component (A = 0 is
 * the Cartesian mesh); |A| < 0.1 keeps the map invertible. */
typedef struct mfcg_mesh {
  int32_t nx, ny, nz;
  double amplitude;
} mfcg_mesh;

typedef enum mfcg_geometry_kind {
  MFCG_GEOM_AFFINE = 0,     /* constant Jacobian per cell (Cartesian box cells), Sec. 2.2 "affine" variant */
  MFCG_GEOM_DEFORMED = 1,   /* per-quadrature-point inverse Jacobian and JxW stored in FP64, Sec. 2.2
                               "inverse Jacobian load" variant (10 values per point)                        */
  MFCG_GEOM_DEFORMED_TENSOR = 2, /* the same mesh with the symmetric tensor J^{-1} (w det J a) J^{-T}
                               stored per point, Sec. 2.2 "final tensor load" variant (6 values per point) */
  MFCG_GEOM_USER = 3,       /* per-point data supplied by the caller (mfcg_geometry.user_data), stored
                               like MFCG_GEOM_DEFORMED: any cell geometry and coefficient whose
                               mesh is logically the Nx x Ny x Nz box of cells                       */
  MFCG_GEOM_DEFORMED_QUADRATIC = 4 /* the deformed mesh represented per cell by the tri-quadratic
                               interpolant of its map through the reference points {0, 1/2, 1}^3:
                               27 x 3 coordinates stored per cell, the Jacobian, its inverse and
                               a(x) computed at every quadrature point, Sec. 2.2 "quadratic geometry
                               compute" variant (scalar operator: components = 1)                */
} mfcg_geometry_kind;

typedef enum mfcg_coefficient_kind {
  MFCG_COEF_CONSTANT = 0,   /* a(x) = 1                                  */
  MFCG_COEF_SIN_X = 1       /* a(x) = 1 + 0.5 sin(pi x), x physical     */
} mfcg_coefficient_kind;

typedef struct mfcg_geometry {
  int32_t kind;             /* mfcg_geometry_kind   */
  int32_t coefficient;      /* mfcg_coefficient_kind (MFCG_GEOM_USER: folded into user_data)       */
  const double* user_data;  /* MFCG_GEOM_USER: HOST array of Nx*Ny*Nz * 10 * (p+1)^3 doubles, read
                               during mfcg_setup only.  Cells in lexicographic order
                               (cx + Nx (cy + Ny cz)); per cell ten blocks of (p+1)^3 values at the
                               tensor Gauss points q = qa + (p+1)(qb + (p+1) qc) of the reference
                               cell [0,1]^3: the nine entries of J^{-1} row-major (J_ij = dx_i/dxhat_j),
                               then w_q det J_q a(x_q).  NULL for the other kinds.                  */
} mfcg_geometry;

typedef enum mfcg_mode {
  MFCG_MODE_FUSED = 0,      /* Algorithm 5 with pre/post inside the operator pass (Sec. 5)        */
  MFCG_MODE_UNFUSED = 1,    /* Algorithm 1 with a separate operator, axpy, Jacobi and dot kernel   */
  MFCG_MODE_SEMI_FUSED = 2, /* Algorithm 5 as separate "pre", operator and "post" kernels, the GPU
                               form of Sec. 6.4; FP64 vectors                                      */
  MFCG_MODE_LOOP_FUSED = 3  /* Algorithm 1 with loop fusion inside its vector regions (Sec. 3.1, as
                               compared in Sec. 5.4): operator, p.v, one pass for x, r and r.r, one
                               for z = M^-1 r and r.z, the p update; FP64 vectors, the same iterates
                               as MFCG_MODE_UNFUSED                                                  */
} mfcg_mode;

typedef enum mfcg_preconditioner {
  MFCG_PRECOND_JACOBI = 0,  /* M = diag(A) (Sec. 3, Algorithm 5)                                   */
  MFCG_PRECOND_NONE = 1     /* M = I: Algorithm 5 reduces to the merged CG of Algorithm 4 (Sec. 4.1) */
} mfcg_preconditioner;

/* The operator of the problem (the CEED bake-off family of Sec. 2). */
typedef enum mfcg_operator {
  MFCG_OP_LAPLACE = 0,      /* a(grad phi_i, grad phi_j) (Eq. 5): BP3, or BP4 with components = 3      */
  MFCG_OP_MASS = 1          /* (a phi_i, phi_j), same Gauss rule: BP1, or BP2 with components = 3;
                               affine meshes or MFCG_GEOM_DEFORMED (which stores JxW a)             */
} mfcg_operator;

/* Arithmetic of the operator and of the CG vectors.  The ABI is FP64 in every case. */
typedef enum mfcg_precision {
  MFCG_PREC_FP64 = 0,         /* native FP64 everywhere                                                 */
  MFCG_PREC_DOUBLE_FLOAT = 1, /* operator and fused CG vectors as unevaluated pairs of FP32 numbers
                                 (about 48 significant bits) on the FP32 pipes; operator results
                                 within 1e-13 (normwise) of FP64; scalars and reductions in FP64      */
  MFCG_PREC_FP32_INNER = 2,   /* FP64 defect correction: the true residual b - A x with the FP64
                                 operator, inner fused CG in FP32 (sums reduced in FP64) to
                                 inner_rtol per cycle, x updated in FP64; FUSED mode only             */
  MFCG_PREC_DOUBLE_FLOAT_INNER = 3 /* the same FP64 defect correction around the fused double-float
                                 CG: each inner solve runs to the reduction the true residual still
                                 needs (half of rtol ||b|| / ||b - A x||, at least 1e-12; inner_rtol
                                 overrides), so one or two cycles reach rtol on the true residual;
                                 FUSED mode only                                                      */
} mfcg_precision;

/* How FP64 operator contractions run on Cartesian (MFCG_GEOM_AFFINE) problems. */
typedef enum mfcg_fp64_contraction {
  MFCG_FP64_TENSOR_CORES = 0, /* default: the even-odd blocks of the cell matrix of Eq. 5 as dense products
                                 on the FP16 tensor cores, FP64 data and matrix split exactly into 8-bit
                                 digits of 64-bit fixed-point integers (one exponent per tile), the digit
                                 products summed exactly and recombined in 64-bit integers; results
                                 within a few units of 2^-53 of each tile's largest entry, as native FP64.
                                 Used at degrees 1-5 and 7 where its shared-memory staging fits (always
                                 with the default tiles); the FP64 sweeps serve degrees 6 and 8 and
                                 tiles too large for the staging                                        */
  MFCG_FP64_PIPE = 1          /* whole-brick sum-factorisation sweeps in native FP64 on the FP64 pipe      */
} mfcg_fp64_contraction;

typedef struct mfcg_options {
  int32_t mode;             /* mfcg_mode                                                            */
  int32_t graph_iterations; /* CG iterations per captured CUDA graph (even; 0 = 16)                   */
  int32_t instrument;       /* 1: launch without graphs and time every operator-pass kernel with
                               CUDA events (mfcg_solve_info.main_kernel_ms); 0: graphs, no timing      */
  int32_t tile[3];          /* cells per tile and direction; 0 = chosen from the degree; all three -1 =
                               autotune: mfcg_setup times short fixed-iteration solves with a few
                               candidate tiles around the default and keeps the fastest              */
  int32_t precision;        /* mfcg_precision                                                       */
  int32_t preconditioner;   /* mfcg_preconditioner                                                  */
  double inner_rtol;        /* MFCG_PREC_FP32_INNER: residual reduction of each inner solve (0 = 1e-3);
                               MFCG_PREC_DOUBLE_FLOAT_INNER: the same, 0 = what the true residual needs */
  int32_t components;       /* 0 or 1: scalar operator; 3: vector-valued operator (the BP2/BP4 form
                               of Sec. 2): every component is the scalar operator, one CG runs on the
                               coupled system, the Jacobi diagonal and the geometry are shared by the
                               components.  Vectors hold the components one after another (each in
                               the tile-blocked order); FUSED mode only                               */
  int32_t operator_kind;    /* mfcg_operator                                                        */
  int32_t x_update_every_iteration; /* 0: the delayed x update of Algorithm 5 (every other iteration,
                               two steps at once); 1: x_k = x_{k-1} + alpha_{k-1} p_{k-1} in every
                               iteration (FUSED and SEMI_FUSED; the same iterates in exact arithmetic) */
  int32_t true_residual;    /* 1: after a solve, form ||b - A x||^2 with the FP64 operator
                               (mfcg_solve_info.true_residual_sq)                                     */
  int32_t fp64_contraction; /* mfcg_fp64_contraction: the FP64 operator of Cartesian problems (the FP64
                               precision's operator and fused iterations, and the FP64 residuals of the
                               other precisions); ignored on deformed meshes                          */
} mfcg_options;

typedef struct mfcg_solve_info {
  int32_t iterations;         /* number of products A p performed                                  */
  int32_t converged;          /* 1 if ||r|| < rtol ||b|| was detected                               */
  int32_t status;             /* same value as the return code                                     */
  int32_t main_kernel_launches; /* operator-pass kernels timed (instrument = 1), else 0              */
  double residual_sq_est;     /* last ||r_{k+1}||^2: Eq. 8 expansion (fused) or explicit (unfused)   */
  double rhs_norm_sq;         /* ||b||^2                                                           */
  double main_kernel_ms;      /* summed CUDA-event time of the operator-pass kernels (instrument = 1) */
  int64_t kernel_launches;    /* kernels this call enqueued, graph replays included                */
  int32_t outer_cycles;       /* the *_INNER precisions: defect-correction cycles, else 0          */
  int32_t reserved2;
  double true_residual_sq;    /* mfcg_options.true_residual = 1: ||b - A x||^2 of the returned x with
                                 the FP64 operator (one extra operator pass); else -1               */
} mfcg_solve_info;

typedef struct mfcg_problem mfcg_problem;

/* mfcg_setup -- Sec. 2 (Eqs. 2-5) and Sec. 2.1: builds the 1D Gauss-Lobatto
 * basis of degree `degree`, the (degree+1)-point Gauss rule, the tile-blocked
 * DoF numbering (Sec. 5.3) and, for MFCG_GEOM_DEFORMED, the per-point metric
 * data; allocates every internal device buffer.
 *   mesh, geom    in: problem description (copied).
 *   opt           in: may be NULL for defaults.
 *   cuda_stream   in: cudaStream_t (NULL = legacy default stream) used by every call.
 *   out           out: new handle; release with mfcg_destroy.
 * With tile = {-1,-1,-1} the call sets up and times a few candidate tiles first
 * (short fixed-iteration solves) and keeps the fastest.
 * Errors: INVALID_ARG (cells < 1, |amplitude| >= 0.1, affine kind with A != 0 or
 * a != 1, bad enums, FP32_INNER or DOUBLE_FLOAT_INNER without FUSED, components
 * other than 0, 1, 3 or components 3 without FUSED or with
 * MFCG_GEOM_DEFORMED_QUADRATIC, MFCG_OP_MASS with MFCG_GEOM_DEFORMED_TENSOR,
 * MFCG_GEOM_USER without user_data), UNSUPPORTED_DEGREE, OUT_OF_MEMORY,
 * CUDA_ERROR. */
int mfcg_setup(const mfcg_mesh* mesh, int degree, const mfcg_geometry* geom, const mfcg_options* opt,
               void* cuda_stream, mfcg_problem** out);

/* mfcg_n_dofs -- number n of unknowns, all mesh nodes including Dirichlet ones
 * (Sec. 2: n counts the unique coefficients of the expansion), times the number
 * of components. */
int mfcg_n_dofs(const mfcg_problem* prob, int64_t* n);

/* mfcg_apply_operator -- dst = A src (Eq. 4 with the cell operator of Eq. 5),
 * Dirichlet rows identity.  src, dst: device, n doubles, must not overlap.
 * Asynchronous on the problem's stream. */
int mfcg_apply_operator(mfcg_problem* prob, const double* src, double* dst);

/* mfcg_diagonal -- diag(A) of the same operator (exact diagonal with the same
 * Gauss rule; 1 on Dirichlet nodes), the point-Jacobi preconditioner M of
 * Sec. 3.  diag: device, n doubles.  Asynchronous. */
int mfcg_diagonal(mfcg_problem* prob, double* diag);

/* mfcg_rhs -- right-hand side b_i = int f phi_i for the manufactured solution
 * u = sin(pi x) sin(pi y) sin(pi z) (f = -div(a grad u)), same Gauss rule,
 * 0 on Dirichlet nodes; for MFCG_OP_MASS the right-hand side of the same u
 * (f = a u).  Not defined for MFCG_GEOM_USER (INVALID_ARG).  b: device, n
 * doubles.  With components > 1, component c holds the right-hand side of
 * u_c = (c + 1) u.  Asynchronous. */
int mfcg_rhs(mfcg_problem* prob, double* b);

/* mfcg_cg_solve -- Jacobi-preconditioned CG from the initial guess in x
 * (Algorithm 5 in FUSED and SEMI_FUSED modes, Algorithm 1 in UNFUSED mode) until
 * ||r_k|| < rtol ||b|| (unpreconditioned residual, Sec. 3.1) or maxit products
 * A p.  rtol == 0 runs exactly maxit iterations and returns MFCG_OK.  With
 * MFCG_PREC_FP32_INNER or MFCG_PREC_DOUBLE_FLOAT_INNER the solve stops on the
 * true residual ||b - A x|| < rtol ||b|| and maxit counts all inner
 * iterations; rtol == 0 there applies one correction x += d with exactly maxit
 * inner iterations.
 *   b   in : device, n doubles, must be zero on Dirichlet nodes (INVALID_ARG is
 *            not checked on the device; a nonzero value there is solved as an
 *            identity row).
 *   x   in/out: device, n doubles; initial guess on entry (r_0 = b - A x_0 is
 *            always formed), solution on return.
 *   info out: may be NULL.
 * Synchronises the stream.  Returns OK, NOT_CONVERGED, BREAKDOWN or CUDA_ERROR. */
int mfcg_cg_solve(mfcg_problem* prob, const double* b, double* x, double rtol, int maxit,
                  mfcg_solve_info* info);

/* mfcg_cg_solve_host -- the same solve with HOST arrays (pinned memory gives
 * asynchronous copies): b is copied to a library-owned device buffer (allocated
 * on the first call, freed by mfcg_destroy), x is copied in and the solution
 * copied back before return (also after NOT_CONVERGED or BREAKDOWN).
 *   b_host in: n doubles; x_host in/out: n doubles; info out: may be NULL.
 * Errors: those of mfcg_cg_solve; INVALID_ARG for NULL arrays, maxit < 0 or
 * rtol < 0; OUT_OF_MEMORY when the device buffers cannot be allocated. */
int mfcg_cg_solve_host(mfcg_problem* prob, const double* b_host, double* x_host, double rtol, int maxit,
                       mfcg_solve_info* info);

/* mfcg_to_lexicographic / mfcg_from_lexicographic -- reorder a device vector
 * between the library's tile-blocked order and the lexicographic node order
 * g = i + (p Nx + 1)(j + (p Ny + 1) k).  in, out: device, n doubles, no overlap. */
int mfcg_to_lexicographic(mfcg_problem* prob, const double* in, double* out);
int mfcg_from_lexicographic(mfcg_problem* prob, const double* in, double* out);

/* mfcg_destroy -- frees every buffer the library owns; NULL is accepted. */
int mfcg_destroy(mfcg_problem* prob);

/* mfcg_apply_operator_static -- dst = A src like mfcg_apply_operator, for
 * callers that cannot allocate device memory: programs whose device memory is
 * handed to their own pool allocator at start-up, and loops that must not call
 * cudaMalloc/cudaFree because those calls can synchronise the whole device.
 * The paper has no counterpart; this is a service of the library.
 *   mesh    in: Cartesian mesh only (amplitude 0, coefficient 1), any Nx, Ny, Nz.
 *   degree  in: 1..8.
 *   src, dst: device, n doubles in the tile-blocked order that mfcg_setup uses
 *            with default options for the same mesh and degree (FP64); no overlap.
 *   cuda_stream: stream of the launch (NULL = legacy default stream).
 * The call allocates nothing: its only scratch, the partial sums of the nodes
 * shared between tiles, lives in one fixed 16 MiB array of device memory that
 * every GPU loading the library holds until the process exits.  Meshes whose
 * scratch exceeds it (for example Q4 beyond about 40^3 cells, Q2 beyond 84^3)
 * are rejected with MFCG_SCRATCH_TOO_SMALL before any GPU work.  The first call
 * on a device looks up the array's device address (cudaGetSymbolAddress) and
 * sets the kernel's shared-memory limit; make that first call before any
 * stream capture.  These per-device results are kept for the life of the
 * process: after cudaDeviceReset (or anything else that destroys and recreates
 * the device's primary context) the cached address is stale, so do not use
 * this entry point across a device reset.  The launches are those of
 * mfcg_apply_operator with mfcg_options.fp64_contraction = MFCG_FP64_PIPE (the
 * FP64 sweeps), including its L2 look-ahead prefetch; a tile whose shared
 * memory exceeds the device's limit is rejected with INVALID_ARG.  All calls
 * share the array: calls that overlap on the GPU
 * (concurrent streams, other host threads) race and give wrong results; every
 * value read from the array is written earlier in the same call, so nothing
 * needs clearing between calls.  Asynchronous on cuda_stream.  Errors:
 * INVALID_ARG, UNSUPPORTED_DEGREE, SCRATCH_TOO_SMALL, CUDA_ERROR. */
int mfcg_apply_operator_static(const mfcg_mesh* mesh, int degree, const double* src, double* dst, void* cuda_stream);

/* ---------------------------------------------------------------------------
 * Batches of independent problems.  Small problems cannot fill the GPU and are
 * bound by launch latency (Sec. 6: the GPU needs millions of unknowns for its
 * best throughput); a batch solves many independent problems of any degree and
 * mesh together: the fused iterations of all members are one CUDA graph with
 * one branch per member, so their kernels run concurrently and the host
 * synchronises once per graph for the whole batch.
 * --------------------------------------------------------------------------- */
typedef struct mfcg_batch mfcg_batch;

/* mfcg_setup_batch -- sets up `count` problems as mfcg_setup would, member i
 * with meshes[i], degrees[i] and geoms[i], all with the options *opt (mode
 * FUSED, precision FP64 or DOUBLE_FLOAT; NULL = defaults) on cuda_stream.
 *   count   in: 1..4096.
 *   meshes, degrees, geoms: host arrays of count entries, read during the call.
 *   out     out: new handle; release with mfcg_destroy_batch.
 * Members with the identical definition (mesh, degree and geometry; the
 * options are common) share the stored geometry and the Jacobi diagonal: a
 * block of right-hand sides on one mesh holds one copy of the operator data.
 * Errors: those of mfcg_setup for any member (nothing is left allocated),
 * INVALID_ARG for a mode or precision a batch does not support. */
int mfcg_setup_batch(int count, const mfcg_mesh* meshes, const int* degrees, const mfcg_geometry* geoms,
                     const mfcg_options* opt, void* cuda_stream, mfcg_batch** out);

/* mfcg_batch_member -- the problem handle of member i, owned by the batch (valid
 * until mfcg_destroy_batch; do not destroy it), for mfcg_n_dofs, mfcg_rhs,
 * mfcg_apply_operator and the reordering helpers. */
int mfcg_batch_member(mfcg_batch* batch, int i, mfcg_problem** prob);

/* mfcg_cg_solve_batch -- solves A_i x_i = b_i for every member i with the
 * fused Algorithm 5, each with its own convergence test ||r_k|| <= rtol ||b_i||
 * (rtol = 0: exactly maxit iterations each), like mfcg_cg_solve.
 *   b, x    in: host arrays of count DEVICE pointers (n_i doubles each, the
 *           member's tile-blocked order); x_i in: initial guess, out: solution.
 *   infos   out: host array of count records (may be NULL).
 * Returns OK when every member converged (or rtol = 0), else the first
 * non-OK member status (per-member status in infos[i].status). */
int mfcg_cg_solve_batch(mfcg_batch* batch, const double* const* b, double* const* x, double rtol, int maxit,
                        mfcg_solve_info* infos);

/* mfcg_destroy_batch -- destroys every member and the batch; NULL is accepted. */
int mfcg_destroy_batch(mfcg_batch* batch);

/* mfcg_status_string -- static description of a status code. */
const char* mfcg_status_string(int status);

#ifdef __cplusplus
}
#endif

#endif /* MFCG_H */
