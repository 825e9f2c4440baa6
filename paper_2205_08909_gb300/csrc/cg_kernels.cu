// Vector kernels of the library: the plain unfused Jacobi-CG of Algorithm 1
// (one kernel per vector operation, device-resident scalars), CG start-up and
// finalisation of Algorithm 5, reordering between the tile-blocked and the
// lexicographic numbering, and the per-point metric data of deformed meshes.
//
// Every reduction is two-stage and deterministic: per-CTA partial sums in a
// fixed order, then the last CTA to finish (elected with an atomic ticket, no
// waiting) adds the partials in CTA order and updates the scalars.
#include "mfcg_internal.h"
#include "precision.cuh"

namespace mfcg {

namespace {

constexpr int kVecThreads = 256;

__device__ __forceinline__ double warp_sum(double v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
  return v;
}

// fixed-order block sum of NV values; result valid in thread 0
template <int NV>
__device__ __forceinline__ void block_sum(double (&v)[NV]) {
  __shared__ double red[NV * (kVecThreads / 32)];
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
#pragma unroll
  for (int m = 0; m < NV; ++m) v[m] = warp_sum(v[m]);
  if (lane == 0)
#pragma unroll
    for (int m = 0; m < NV; ++m) red[warp * NV + m] = v[m];
  __syncthreads();
  if (threadIdx.x == 0) {
#pragma unroll
    for (int m = 0; m < NV; ++m) {
      double s = 0.0;
      for (int w = 0; w < kVecThreads / 32; ++w) s += red[w * NV + m];
      v[m] = s;
    }
  }
  __syncthreads();
}

// Stores this CTA's NV partial sums, elects the last CTA and, there, returns
// true with the fixed-order totals in tot (thread 0 only).
template <int NV>
__device__ bool grid_sum(double (&v)[NV], double* partial, unsigned int* ticket, double (&tot)[NV]) {
  __shared__ int last;
  block_sum<NV>(v);
  if (threadIdx.x == 0) {
#pragma unroll
    for (int m = 0; m < NV; ++m) partial[blockIdx.x * 8 + m] = v[m];
    __threadfence();
    last = atomicAdd(ticket, 1u) == gridDim.x - 1;
  }
  __syncthreads();
  if (!last) return false;
  __threadfence();
#pragma unroll
  for (int m = 0; m < NV; ++m) tot[m] = 0.0;
  for (int t = threadIdx.x; t < (int)gridDim.x; t += kVecThreads)
#pragma unroll
    for (int m = 0; m < NV; ++m) tot[m] += __ldcg(partial + t * 8 + m);
  block_sum<NV>(tot);
  if (threadIdx.x == 0) *ticket = 0u;
  return true;
}

// ||b - ax||^2 with a fixed-order grid reduction into *out
__global__ void residual_norm_kernel(const double* b, const double* ax, int64_t n, double* partial,
                                     unsigned int* ticket, double* out) {
  double v[1] = {0.0};
  for (int64_t i = blockIdx.x * (int64_t)kVecThreads + threadIdx.x; i < n; i += (int64_t)gridDim.x * kVecThreads) {
    const double r = b[i] - ax[i];
    v[0] = fma(r, r, v[0]);
  }
  double tot[1];
  if (!grid_sum<1>(v, partial, ticket, tot)) return;
  if (threadIdx.x == 0) *out = tot[0];
}

__global__ void fill_kernel(double* v, double value, int64_t n) {
  for (int64_t i = blockIdx.x * (int64_t)kVecThreads + threadIdx.x; i < n; i += (int64_t)gridDim.x * kVecThreads)
    v[i] = value;
}

__global__ void invert_kernel(const double* in, double* out, int64_t n) {
  for (int64_t i = blockIdx.x * (int64_t)kVecThreads + threadIdx.x; i < n; i += (int64_t)gridDim.x * kVecThreads)
    out[i] = 1.0 / in[i];
}

__global__ void reorder_kernel(const TileGeom g, const double* in, double* out, int to_lex) {
  const int64_t n = g.n_dofs;
  for (int64_t l = blockIdx.x * (int64_t)kVecThreads + threadIdx.x; l < n; l += (int64_t)gridDim.x * kVecThreads) {
    const int i = (int)(l % g.nn[0]);
    const int j = (int)((l / g.nn[0]) % g.nn[1]);
    const int k = (int)(l / ((int64_t)g.nn[0] * g.nn[1]));
    const int64_t t = node_index(g, i, j, k);
    if (to_lex)
      out[l] = in[t];
    else
      out[t] = in[l];
  }
}

// Per-point data of the deformed map x = X + A s(X) (1,1,1), X = h (c + xhat):
// J = (I + A 1 grad s^T) diag(h), so by Sherman-Morrison
// J^{-1}_{rc} = (delta_rc - A ds/dX_c / (1 + A sum grad s)) / h_r and
// det J = h_x h_y h_z (1 + A sum grad s).  GEOM_DEFORMED stores [cell][10][nq]:
// J^{-1} row-major, then w_q det J a(x_q); GEOM_TENSOR stores [cell][6][nq]:
// the upper triangle of C = (w_q det J a) J^{-1} J^{-T}.
// GEOM_QUAD stores [cell][3][27]: the map at the reference points (a, b, c) / 2.
__global__ void geometry_kernel(const TileGeom g, const OperatorCoeffs c, int geom, double* geo) {
  if (geom == GEOM_QUAD) {
    const int64_t total = (int64_t)g.N[0] * g.N[1] * g.N[2] * 27;
    const double twopi = 6.28318530717958647692;
    for (int64_t t = blockIdx.x * (int64_t)kVecThreads + threadIdx.x; t < total; t += (int64_t)gridDim.x * kVecThreads) {
      const int64_t cell = t / 27;
      const int m = (int)(t - cell * 27);
      const int cx = (int)(cell % g.N[0]), cy = (int)((cell / g.N[0]) % g.N[1]), cz = (int)(cell / ((int64_t)g.N[0] * g.N[1]));
      const double X = c.h[0] * (cx + 0.5 * (m % 3)), Y = c.h[1] * (cy + 0.5 * ((m / 3) % 3)),
                   Z = c.h[2] * (cz + 0.5 * (m / 9));
      const double s = c.amplitude * sin(twopi * X) * sin(twopi * Y) * sin(twopi * Z);
      double* out = geo + cell * 81 + m;
      out[0] = X + s;
      out[27] = Y + s;
      out[54] = Z + s;
    }
    return;
  }
  const int n1 = g.p + 1, nq = n1 * n1 * n1;
  const int nv = geo_values(geom);
  const int64_t total = (int64_t)g.N[0] * g.N[1] * g.N[2] * nq;
  const double twopi = 6.28318530717958647692, pi = 3.14159265358979323846;
  for (int64_t t = blockIdx.x * (int64_t)kVecThreads + threadIdx.x; t < total; t += (int64_t)gridDim.x * kVecThreads) {
    const int64_t cell = t / nq;
    const int q = (int)(t - cell * nq);
    const int qa = q % n1, qb = (q / n1) % n1, qc = q / (n1 * n1);
    const int cx = (int)(cell % g.N[0]), cy = (int)((cell / g.N[0]) % g.N[1]), cz = (int)(cell / ((int64_t)g.N[0] * g.N[1]));
    const double X = c.h[0] * (cx + c.g[qa]), Y = c.h[1] * (cy + c.g[qb]), Z = c.h[2] * (cz + c.g[qc]);
    const double sx = sin(twopi * X), sy = sin(twopi * Y), sz = sin(twopi * Z);
    const double gs[3] = {twopi * cos(twopi * X) * sy * sz, twopi * sx * cos(twopi * Y) * sz,
                          twopi * sx * sy * cos(twopi * Z)};
    const double A = c.amplitude;
    const double den = 1.0 + A * (gs[0] + gs[1] + gs[2]);
    double Ji[9];
    for (int r = 0; r < 3; ++r)
      for (int cc = 0; cc < 3; ++cc) Ji[3 * r + cc] = ((r == cc ? 1.0 : 0.0) - A * gs[cc] / den) / c.h[r];
    const double xphys = X + A * sx * sy * sz;
    const double coef = c.coef == MFCG_COEF_SIN_X ? 1.0 + 0.5 * sin(pi * xphys) : 1.0;
    const double jxw = c.w[qa] * c.w[qb] * c.w[qc] * c.h[0] * c.h[1] * c.h[2] * den * coef;
    double* out = geo + cell * nv * nq + q;
    if (geom == GEOM_TENSOR) {
      const int rr[6] = {0, 0, 0, 1, 1, 2}, ccn[6] = {0, 1, 2, 1, 2, 2};
      for (int m = 0; m < 6; ++m) {
        double s = 0.0;
        for (int l = 0; l < 3; ++l) s += Ji[3 * rr[m] + l] * Ji[3 * ccn[m] + l];
        out[m * nq] = jxw * s;
      }
    } else {
      for (int m = 0; m < 9; ++m) out[m * nq] = Ji[m];
      out[9 * nq] = jxw;
    }
  }
}

// r = b - Ax
__global__ void residual_kernel(const double* b, const double* ax, double* r, int64_t n) {
  for (int64_t i = blockIdx.x * (int64_t)kVecThreads + threadIdx.x; i < n; i += (int64_t)gridDim.x * kVecThreads)
    r[i] = b[i] - ax[i];
}

// CG start: eps^2 = rtol^2 ||b||^2; an exactly zero initial residual finishes at once.
__global__ void cg_init_kernel(CGState* st, const double* b, const double* r0, int64_t n, double rtol, int maxit,
                               int fixed, double* partial, int x_every_iter) {
  double v[2] = {0.0, 0.0};
  for (int64_t i = blockIdx.x * (int64_t)kVecThreads + threadIdx.x; i < n; i += (int64_t)gridDim.x * kVecThreads) {
    v[0] = fma(b[i], b[i], v[0]);
    v[1] = fma(r0[i], r0[i], v[1]);
  }
  double tot[2];
  if (!grid_sum<2>(v, partial, &st->ticket, tot)) return;
  if (threadIdx.x == 0) {
    st->alpha_prev = st->beta_prev = st->alpha_prev2 = st->beta_prev2 = 0.0;
    st->alpha_cur = 0.0;
    st->eps_sq = rtol * rtol * tot[0];
    st->gamma_next = tot[1];
    st->sums[7] = tot[0];
    st->k = 1;
    st->maxit = maxit;
    st->iterations = 0;
    st->fixed = fixed;
    st->x_every_iter = x_every_iter;
    st->done = (tot[1] == 0.0 || maxit <= 0) ? 1 : 0;
    if (!isfinite(tot[0]) || !isfinite(tot[1])) st->done = 3;
    prepare_iteration_scalars(st);
  }
}

// Finalisation of Algorithm 5 after the last iteration k: odd k: x += alpha_k p_k;
// even k: x += alpha_k p_k + alpha_{k-1}/beta_{k-1} (p_k - M^{-1} r_k).
template <int PREC>
__global__ void finalize_fused_kernel(int64_t n, const CGState* st, void* xv, const void* p0v, const void* p1v,
                                      const void* r0v, const void* r1v, const void* dinvv) {
  using T = typename Num<PREC>::T;
  const int k = st->iterations;
  if (k < 1 || st->done == 3) return;
  const T* p = static_cast<const T*>((k & 1) ? p1v : p0v);  // iteration k wrote buffer k & 1
  const T* r = static_cast<const T*>((k & 1) ? r1v : r0v);
  const T* dinv = static_cast<const T*>(dinvv);
  T* x = static_cast<T*>(xv);
  const bool current = (k & 1) || st->x_every_iter;  // x holds x_k: one plain step
  const T a = t_from_double<PREC>(st->alpha_cur);
  const T c = t_from_double<PREC>(current ? 0.0 : st->alpha_prev / st->beta_prev);
  for (int64_t i = blockIdx.x * (int64_t)kVecThreads + threadIdx.x; i < n; i += (int64_t)gridDim.x * kVecThreads) {
    const T pk = p[i];
    if (current)
      x[i] = t_axpy<PREC>(a, pk, x[i]);
    else
      x[i] = t_add<PREC>(x[i], t_axby<PREC>(a, pk, c, t_sub<PREC>(pk, t_mul<PREC>(dinv[i], r[i]))));
  }
}

// conversions between FP64 vectors and the storage type of a precision
template <int PREC>
__global__ void to_prec_kernel(const double* in, void* outv, int64_t n) {
  using T = typename Num<PREC>::T;
  T* out = static_cast<T*>(outv);
  for (int64_t i = blockIdx.x * (int64_t)kVecThreads + threadIdx.x; i < n; i += (int64_t)gridDim.x * kVecThreads)
    out[i] = t_from_double<PREC>(in[i]);
}

template <int PREC>
__global__ void from_prec_kernel(const void* inv, double* out, int64_t n, int accumulate) {
  using T = typename Num<PREC>::T;
  const T* in = static_cast<const T*>(inv);
  for (int64_t i = blockIdx.x * (int64_t)kVecThreads + threadIdx.x; i < n; i += (int64_t)gridDim.x * kVecThreads)
    out[i] = accumulate ? out[i] + t_to_double<PREC>(in[i]) : t_to_double<PREC>(in[i]);
}

// ---------------------------- unfused Algorithm 1 ----------------------------------
// Scalar step after the grid reduction s of one of the dot products of
// Algorithm 1 (thread 0 of the last CTA).  which: 0 s = p.v -> alpha = e / s;
// 1 s = r.r -> convergence test; 2 s = r.z -> beta = s / e, next iteration.
__device__ void unfused_scalars(CGState* st, int which, double s) {
  if (which == 0) {
    if (!(s > 0.0) || !isfinite(s)) {
      st->done = 3;
      st->iterations = st->k;
      return;
    }
    st->alpha_cur = st->e_cur / s;
    st->sums[1] = s;
  } else if (which == 1) {
    st->gamma_next = s;
    st->iterations = st->k;
    if (!isfinite(s)) st->done = 3;
    else if (!st->fixed && s < st->eps_sq) st->done = 1;
    else if (st->k >= st->maxit) st->done = 2;
  } else {
    if (!(st->e_cur > 0.0) || !isfinite(s)) {
      st->done = 3;
      return;
    }
    st->beta_prev = s / st->e_cur;
    st->e_cur = s;
    st->k += 1;
  }
}

// which: 0 a = p.v -> alpha = e/a; 1 gamma = r.r -> convergence; 2 e' = r.z -> beta;
//        3 start: z = M^-1 r, p = z, e = r.z
__global__ void unfused_dot_kernel(UnfusedArgs a, int which) {
  CGState* st = a.state;
  if (which != 3 && st->done) return;
  double v[1] = {0.0};
  for (int64_t i = blockIdx.x * (int64_t)kVecThreads + threadIdx.x; i < a.n; i += (int64_t)gridDim.x * kVecThreads) {
    if (which == 0) v[0] = fma(a.p[i], a.v[i], v[0]);
    else if (which == 1) v[0] = fma(a.r[i], a.r[i], v[0]);
    else if (which == 2) v[0] = fma(a.r[i], a.z[i], v[0]);
    else {
      const double z = a.diag_inv[i] * a.r[i];
      a.p[i] = z;
      v[0] = fma(a.r[i], z, v[0]);
    }
  }
  double tot[1];
  if (!grid_sum<1>(v, a.partial, &st->ticket, tot)) return;
  if (threadIdx.x != 0) return;
  if (which == 3) st->e_cur = tot[0];
  else unfused_scalars(st, which, tot[0]);
}

// Algorithm 1 with loop fusion inside its vector regions (Sec. 3.1; the
// "basic loop fusion" of the comparisons of Sec. 5.4 and Sec. 6): each pass
// ends in the reduction of its region.  which: 0 x += alpha p, r -= alpha v
// with gamma = r.r (convergence); 1 z = M^-1 r with e' = r.z (beta).  The
// products and the reduction order are those of the one-operation kernels, so
// both forms give bitwise the same iterates.
__global__ void loop_fused_kernel(UnfusedArgs a, int which) {
  CGState* st = a.state;
  if (st->done) return;
  const double alpha = st->alpha_cur;
  double v[1] = {0.0};
  for (int64_t i = blockIdx.x * (int64_t)kVecThreads + threadIdx.x; i < a.n; i += (int64_t)gridDim.x * kVecThreads) {
    if (which == 0) {
      a.x[i] = fma(alpha, a.p[i], a.x[i]);
      const double r = fma(-alpha, a.v[i], a.r[i]);
      a.r[i] = r;
      v[0] = fma(r, r, v[0]);
    } else {
      const double r = a.r[i];
      const double z = a.diag_inv[i] * r;
      a.z[i] = z;
      v[0] = fma(r, z, v[0]);
    }
  }
  double tot[1];
  if (!grid_sum<1>(v, a.partial, &st->ticket, tot)) return;
  if (threadIdx.x != 0) return;
  unfused_scalars(st, which + 1, tot[0]);
}

// which: 0 x += alpha p; 1 r -= alpha v; 2 z = M^-1 r; 3 p = z + beta p
__global__ void unfused_axpy_kernel(UnfusedArgs a, int which) {
  const CGState* st = a.state;
  if (st->done) return;
  const double alpha = st->alpha_cur, beta = st->beta_prev;
  for (int64_t i = blockIdx.x * (int64_t)kVecThreads + threadIdx.x; i < a.n; i += (int64_t)gridDim.x * kVecThreads) {
    if (which == 0) a.x[i] = fma(alpha, a.p[i], a.x[i]);
    else if (which == 1) a.r[i] = fma(-alpha, a.v[i], a.r[i]);
    else if (which == 2) a.z[i] = a.diag_inv[i] * a.r[i];
    else a.p[i] = fma(beta, a.p[i], a.z[i]);
  }
}

unsigned grid_for(int64_t n) {
  int64_t b = (n + kVecThreads - 1) / kVecThreads;
  const int64_t cap = 152 * 8;  // 8 resident CTAs per SM on the 152 SMs
  if (b > cap) b = cap;
  return (unsigned)(b < 1 ? 1 : b);
}

}  // namespace

int vec_grid(int64_t n) { return (int)grid_for(n); }

// done flags of a batch of CG states into one array (one read-back per batch)
__global__ void gather_done_kernel(const CGState* const* states, int count, int* done) {
  for (int i = blockIdx.x * kVecThreads + threadIdx.x; i < count; i += gridDim.x * kVecThreads)
    done[i] = states[i]->done;
}

cudaError_t launch_gather_done(const CGState* const* states, int count, int* done, cudaStream_t s) {
  gather_done_kernel<<<(count + kVecThreads - 1) / kVecThreads, kVecThreads, 0, s>>>(states, count, done);
  return cudaGetLastError();
}

__global__ void scale_kernel(const double* in, double* out, double factor, int64_t n) {
  for (int64_t i = blockIdx.x * (int64_t)kVecThreads + threadIdx.x; i < n; i += (int64_t)gridDim.x * kVecThreads)
    out[i] = factor * in[i];
}

cudaError_t launch_scale(const double* in, double* out, double factor, int64_t n, cudaStream_t s) {
  scale_kernel<<<grid_for(n), kVecThreads, 0, s>>>(in, out, factor, n);
  return cudaGetLastError();
}

cudaError_t launch_residual_norm(const double* b, const double* ax, int64_t n, double* partial, unsigned int* ticket,
                                 double* out, cudaStream_t s) {
  residual_norm_kernel<<<grid_for(n), kVecThreads, 0, s>>>(b, ax, n, partial, ticket, out);
  return cudaGetLastError();
}

cudaError_t launch_fill(double* v, double value, int64_t n, cudaStream_t s) {
  fill_kernel<<<grid_for(n), kVecThreads, 0, s>>>(v, value, n);
  return cudaGetLastError();
}

cudaError_t launch_invert(const double* in, double* out, int64_t n, cudaStream_t s) {
  invert_kernel<<<grid_for(n), kVecThreads, 0, s>>>(in, out, n);
  return cudaGetLastError();
}

cudaError_t launch_reorder(const TileGeom& g, const double* in, double* out, int to_lex, cudaStream_t s) {
  reorder_kernel<<<grid_for(g.n_dofs), kVecThreads, 0, s>>>(g, in, out, to_lex);
  return cudaGetLastError();
}

cudaError_t launch_geometry(const TileGeom& g, const OperatorCoeffs& c, int geom, double* geo, cudaStream_t s) {
  const int64_t total = (int64_t)g.N[0] * g.N[1] * g.N[2] * (geom == GEOM_QUAD ? 27 : (g.p + 1) * (g.p + 1) * (g.p + 1));
  geometry_kernel<<<grid_for(total), kVecThreads, 0, s>>>(g, c, geom, geo);
  return cudaGetLastError();
}

cudaError_t launch_residual(const double* b, const double* ax, double* r, int64_t n, cudaStream_t s) {
  residual_kernel<<<grid_for(n), kVecThreads, 0, s>>>(b, ax, r, n);
  return cudaGetLastError();
}

cudaError_t launch_cg_init(CGState* st, const double* b, const double* r0, int64_t n, double rtol, int maxit, int fixed,
                           double* partial, int x_every_iter, cudaStream_t s) {
  cg_init_kernel<<<grid_for(n), kVecThreads, 0, s>>>(st, b, r0, n, rtol, maxit, fixed, partial, x_every_iter);
  return cudaGetLastError();
}

cudaError_t launch_finalize_fused(int prec, int64_t n, CGState* st, void* x, const void* p0, const void* p1,
                                  const void* r0, const void* r1, const void* diag_inv, cudaStream_t s) {
  if (prec == PREC_F64)
    finalize_fused_kernel<PREC_F64><<<grid_for(n), kVecThreads, 0, s>>>(n, st, x, p0, p1, r0, r1, diag_inv);
  else if (prec == PREC_DD)
    finalize_fused_kernel<PREC_DD><<<grid_for(n), kVecThreads, 0, s>>>(n, st, x, p0, p1, r0, r1, diag_inv);
  else
    finalize_fused_kernel<PREC_F32><<<grid_for(n), kVecThreads, 0, s>>>(n, st, x, p0, p1, r0, r1, diag_inv);
  return cudaGetLastError();
}

cudaError_t launch_to_prec(int prec, const double* in, void* out, int64_t n, cudaStream_t s) {
  if (prec == PREC_F64)
    return cudaMemcpyAsync(out, in, n * sizeof(double), cudaMemcpyDeviceToDevice, s);
  if (prec == PREC_DD)
    to_prec_kernel<PREC_DD><<<grid_for(n), kVecThreads, 0, s>>>(in, out, n);
  else
    to_prec_kernel<PREC_F32><<<grid_for(n), kVecThreads, 0, s>>>(in, out, n);
  return cudaGetLastError();
}

cudaError_t launch_from_prec(int prec, const void* in, double* out, int64_t n, int accumulate, cudaStream_t s) {
  if (prec == PREC_F64 && !accumulate)
    return cudaMemcpyAsync(out, in, n * sizeof(double), cudaMemcpyDeviceToDevice, s);
  if (prec == PREC_F64)
    from_prec_kernel<PREC_F64><<<grid_for(n), kVecThreads, 0, s>>>(in, out, n, accumulate);
  else if (prec == PREC_DD)
    from_prec_kernel<PREC_DD><<<grid_for(n), kVecThreads, 0, s>>>(in, out, n, accumulate);
  else
    from_prec_kernel<PREC_F32><<<grid_for(n), kVecThreads, 0, s>>>(in, out, n, accumulate);
  return cudaGetLastError();
}

cudaError_t launch_unfused_dot(int which, const UnfusedArgs& a, cudaStream_t s) {
  unfused_dot_kernel<<<grid_for(a.n), kVecThreads, 0, s>>>(a, which);
  return cudaGetLastError();
}

cudaError_t launch_unfused_axpy(int which, const UnfusedArgs& a, cudaStream_t s) {
  unfused_axpy_kernel<<<grid_for(a.n), kVecThreads, 0, s>>>(a, which);
  return cudaGetLastError();
}

cudaError_t launch_loop_fused(int which, const UnfusedArgs& a, cudaStream_t s) {
  loop_fused_kernel<<<grid_for(a.n), kVecThreads, 0, s>>>(a, which);
  return cudaGetLastError();
}

}  // namespace mfcg
