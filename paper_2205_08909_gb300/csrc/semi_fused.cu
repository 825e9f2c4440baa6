// Semi-fused Algorithm 5: the GPU form of Sec. 6.4, with the "pre" vector
// updates, the operator and the "post" inner products as separate kernels on
// FP64 vectors.  It sits between the unfused Algorithm 1 (one kernel per
// vector operation) and the fused pass of tile_kernels.cuh, and reuses the
// scalar step of the fused tail (alpha_k, Eq. 8 estimate, beta_k by Eq. 7).
#include "tile_kernels.cuh"

namespace mfcg {

namespace {

constexpr int kVec = 256;

unsigned vec_grid_for(int64_t n) {
  int64_t b = (n + kVec - 1) / kVec;
  const int64_t cap = 152 * 8;
  if (b > cap) b = cap;
  return (unsigned)(b < 1 ? 1 : b);
}

// "pre": delayed x update on odd k > 1, r_k = r_{k-1} - alpha_{k-1} v_{k-1},
// p_k = M^{-1} r_k + beta_{k-1} p_{k-1}, in place
__global__ void semi_pre_kernel(int64_t n, const CGState* st, double* x, double* r, double* p, const double* v,
                                const double* dinv) {
  if (st->done) return;
  const int k = st->k;
  const bool xupd = k > 1 && ((k & 1) || st->x_every_iter);
  const double am = -st->alpha_prev, beta = st->beta_prev, xa = st->alpha_prev, xr = st->ratio;
  for (int64_t i = blockIdx.x * (int64_t)kVec + threadIdx.x; i < n; i += (int64_t)gridDim.x * kVec) {
    const double r_o = r[i], p_o = p[i], d = dinv[i];
    if (xupd) x[i] += fma(xa, p_o, xr * (p_o - d * r_o));
    const double rk = fma(am, v[i], r_o);
    r[i] = rk;
    p[i] = fma(beta, p_o, d * rk);
  }
}

// "post": the seven sums, a fixed-order grid reduction and the scalar step
__global__ void semi_post_kernel(int64_t n, CGState* st, const double* r, const double* p, const double* v,
                                 const double* dinv, double* partial) {
  __shared__ double red[8 * (kThreads / 32)];
  __shared__ int is_last;
  if (st->done) return;
  DotAcc<PREC_F64> sm[7];
  for (int64_t i = blockIdx.x * (int64_t)kVec + threadIdx.x; i < n; i += (int64_t)gridDim.x * kVec)
    post_sums<PREC_F64>(sm, r[i], p[i], v[i], dinv[i]);
  store_cta_sums<PREC_F64>(sm, red, partial, blockIdx.x);
  if (threadIdx.x == 0) {
    __threadfence();
    is_last = atomicAdd(&st->ticket, 1u) == gridDim.x - 1;
  }
  __syncthreads();
  if (!is_last) return;
  __threadfence();
  double s[7];
  reduce_partials<PREC_F64>(partial, gridDim.x, red, s);
  if (threadIdx.x == 0) {
    cg_scalar_step(st, s);
    st->ticket = 0u;
  }
}

}  // namespace

static_assert(kVec == kThreads, "the post kernel reuses the tile kernels' block reductions");

cudaError_t launch_semi_pre(int64_t n, const CGState* st, double* x, double* r, double* p, const double* v,
                            const double* dinv, cudaStream_t s) {
  semi_pre_kernel<<<vec_grid_for(n), kVec, 0, s>>>(n, st, x, r, p, v, dinv);
  return cudaGetLastError();
}

cudaError_t launch_semi_post(int64_t n, CGState* st, const double* r, const double* p, const double* v,
                             const double* dinv, double* partial, cudaStream_t s) {
  semi_post_kernel<<<vec_grid_for(n), kVec, 0, s>>>(n, st, r, p, v, dinv, partial);
  return cudaGetLastError();
}

}  // namespace mfcg
