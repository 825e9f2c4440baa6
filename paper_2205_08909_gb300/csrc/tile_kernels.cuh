// Tile kernels of the fused matrix-free CG: one CTA per tile of cells.
//
//   phase 1 ("pre", Algorithm 5):  r_k = r_{k-1} - alpha_{k-1} v_{k-1},
//            p_k = D^{-1} r_k + beta_{k-1} p_{k-1} on every node of the tile
//            (recomputed from the previous buffers for nodes shared with a
//            neighbour tile, stored by the owner only), the delayed x update
//            on odd k > 1, and p_k staged in shared memory;
//   phase 2 (Eq. 4 / Eq. 5): sum-factorised cell integrals of all cells of the
//            tile into a shared-memory node brick: on Cartesian tiles as three
//            even-odd sweeps along whole brick lines (the Kronecker sum of the
//            assembled 1D matrices), on deformed tiles cell batch by cell batch
//            with a fixed-order node gather, in the set-up passes one colour
//            (parity of the cell index) at a time -- no two threads ever add
//            into the same node;
//   phase 3 ("post"): nodes whose last contribution came from this tile are
//            final: v_k is stored and the seven sums of Algorithm 5 are
//            accumulated; nodes on faces shared with another tile store their
//            partial sum in the shell buffer.
// The tail kernel adds the shell partials of the shared-face nodes in a fixed
// order, finishes their post operation and, in its last CTA, reduces all
// per-CTA sums in a fixed order and computes alpha_k, the Eq. 8 residual
// estimate, the convergence flag and beta_k (Eq. 7) on the device.
//
// Every kernel is a template on the degree P, the mode, the geometry kind, the
// arithmetic precision (precision.cuh: FP64, double-float or FP32) and, for the
// tile kernel, the number of components (1 or 3).
#pragma once

#include <algorithm>

#include "mfcg_internal.h"
#include "precision.cuh"
#include "tc_operator.cuh"

namespace mfcg {

// largest number of cells of one colour in a tile (tile edges <= 16 cells)
constexpr int kMaxColorCells = 512;

// Per-cell scratch stride (elements) for ns arrays of (P+1)^3 values, padded
// so that stride = (P+1)^2 (mod 32): the pencils of consecutive threads then
// map to consecutive banks across cell boundaries in the first sweep.
__host__ __device__ constexpr int cell_stride(int P, int ns) {
  return ns * (P + 1) * (P + 1) * (P + 1) +
         ((((P + 1) * (P + 1) - ns * (P + 1) * (P + 1) * (P + 1)) % 32) + 32) % 32;
}

// Tri-quadratic geometry: the per-cell partial sums of the support points
// along y and z at every line (qb, qc) of Gauss points (quad_lines), 27 per
// line, kept after the four arrays of a cell's scratch (a multiple of 32
// elements, so the bank offset of the stride is unchanged)
__host__ __device__ constexpr int quad_line_elems(int P) { return (27 * (P + 1) * (P + 1) + 31) / 32 * 32; }

// per-cell scratch stride of the deformed cell operator
__host__ __device__ constexpr int deformed_stride(int P, int geom) {
  return cell_stride(P, 4) + (geom == GEOM_QUAD ? quad_line_elems(P) : 0);
}

// Cells of a tile that the deformed cell operator processes at once: as many
// as fit next to the two node bricks in kDeformedSmemBytes of shared memory
// (two CTAs per SM), balanced over the batches of a full tile.
constexpr int kDeformedSmemBytes = 110 * 1024;

__host__ __device__ inline int deformed_batch_cells(int P, int elem_bytes, const TileGeom& g, int geom) {
  const int ncell = g.T[0] * g.T[1] * g.T[2];
  const int64_t bricks = 2LL * (P * g.T[0] + 1) * (P * g.T[1] + 1) * (P * g.T[2] + 1) * elem_bytes;
  int64_t nb = (kDeformedSmemBytes - bricks) / ((int64_t)deformed_stride(P, geom) * elem_bytes);
  if (nb < 1) nb = 1;
  if (nb > ncell) nb = ncell;
  if (nb > kMaxColorCells) nb = kMaxColorCells;
  const int nbatch = (int)((ncell + nb - 1) / nb);
  return (ncell + nbatch - 1) / nbatch;
}

// ------------------------------------------------------------------------------------
// 1D contractions on a pencil of N1 = P+1 values held in registers
// ------------------------------------------------------------------------------------
// ------------------------------------------------------------------------------------
// Even-odd form of the centrosymmetric 1D matrices (M, K_d, the volume-scaled
// M): y = A x from the halves E (ceil(n/2)^2) and O (floor(n/2)^2) of the
// coefficient block, about half the multiply-adds of the plain product.
// ------------------------------------------------------------------------------------
// sum_j E_m[off + j] va_j (+ sum_j E_mb[offb + j] vb_j when TWO)
template <int PREC, int K, bool TWO>
__device__ __forceinline__ typename Num<PREC>::T eo_dot(const OperatorCoeffs& c, int ma, int offa,
                                                        const typename Num<PREC>::T (&va)[K], int mb, int offb,
                                                        const typename Num<PREC>::T (&vb)[K]) {
  if constexpr (PREC == PREC_DD) {
    dd_acc a;
    acc_set(a, dd{c.eoh[ma][offa], c.eol[ma][offa]}, va[0]);
#pragma unroll
    for (int j = 1; j < K; ++j) acc_madd(a, dd{c.eoh[ma][offa + j], c.eol[ma][offa + j]}, va[j]);
    if constexpr (TWO) {
#pragma unroll
      for (int j = 0; j < K; ++j) acc_madd(a, dd{c.eoh[mb][offb + j], c.eol[mb][offb + j]}, vb[j]);
    }
    return acc_get(a);
  } else if constexpr (PREC == PREC_F64) {
    double s = 0.0;
#pragma unroll
    for (int j = 0; j < K; ++j) s = fma(c.eo[ma][offa + j], va[j], s);
    if constexpr (TWO) {
#pragma unroll
      for (int j = 0; j < K; ++j) s = fma(c.eo[mb][offb + j], vb[j], s);
    }
    return s;
  } else {
    float s = 0.f;
#pragma unroll
    for (int j = 0; j < K; ++j) s = fmaf(c.eoh[ma][offa + j], va[j], s);
    if constexpr (TWO) {
#pragma unroll
      for (int j = 0; j < K; ++j) s = fmaf(c.eoh[mb][offb + j], vb[j], s);
    }
    return s;
  }
}

// ya = A_m1 x (WA) and yb = A_m2 x (+ A_m3 z when HZ) (WB), all in even-odd form
template <int PREC, int N1, bool WA, bool WB, bool HZ>
__device__ __forceinline__ void eo_apply(const OperatorCoeffs& c, int m1, int m2, int m3,
                                         const typename Num<PREC>::T (&x)[N1], const typename Num<PREC>::T (&z)[N1],
                                         typename Num<PREC>::T (&ya)[N1], typename Num<PREC>::T (&yb)[N1]) {
  using T = typename Num<PREC>::T;
  constexpr int H = N1 / 2, NE = N1 - H;
  T ex[NE], ox[H], ez[NE], oz[H];
#pragma unroll
  for (int j = 0; j < H; ++j) {
    ex[j] = t_add<PREC>(x[j], x[N1 - 1 - j]);
    ox[j] = t_sub<PREC>(x[j], x[N1 - 1 - j]);
    if constexpr (HZ) {
      ez[j] = t_add<PREC>(z[j], z[N1 - 1 - j]);
      oz[j] = t_sub<PREC>(z[j], z[N1 - 1 - j]);
    }
  }
  if constexpr (NE > H) {
    ex[H] = x[H];
    if constexpr (HZ) ez[H] = z[H];
  }
#pragma unroll
  for (int i = 0; i < H; ++i) {
    if constexpr (WA) {
      const T ye = eo_dot<PREC, NE, false>(c, m1, i * NE, ex, m1, 0, ex);
      const T yo = eo_dot<PREC, H, false>(c, m1, NE * NE + i * H, ox, m1, 0, ox);
      ya[i] = t_add<PREC>(ye, yo);
      ya[N1 - 1 - i] = t_sub<PREC>(ye, yo);
    }
    if constexpr (WB) {
      const T ye = eo_dot<PREC, NE, HZ>(c, m2, i * NE, ex, m3, i * NE, ez);
      const T yo = eo_dot<PREC, H, HZ>(c, m2, NE * NE + i * H, ox, m3, NE * NE + i * H, oz);
      yb[i] = t_add<PREC>(ye, yo);
      yb[N1 - 1 - i] = t_sub<PREC>(ye, yo);
    }
  }
  if constexpr (NE > H) {
    if constexpr (WA) ya[H] = eo_dot<PREC, NE, false>(c, m1, H * NE, ex, m1, 0, ex);
    if constexpr (WB) yb[H] = eo_dot<PREC, NE, HZ>(c, m2, H * NE, ex, m3, H * NE, ez);
  }
}

// y = A x for an anti-centrosymmetric A (the collocation derivative and its transpose)
template <int PREC, int N1>
__device__ __forceinline__ void eo_apply_anti(const OperatorCoeffs& c, int m, const typename Num<PREC>::T (&x)[N1],
                                              typename Num<PREC>::T (&y)[N1]) {
  using T = typename Num<PREC>::T;
  constexpr int H = N1 / 2, NE = N1 - H;
  T e[NE], o[H];
#pragma unroll
  for (int j = 0; j < H; ++j) {
    e[j] = t_add<PREC>(x[j], x[N1 - 1 - j]);
    o[j] = t_sub<PREC>(x[j], x[N1 - 1 - j]);
  }
  if constexpr (NE > H) e[H] = x[H];
#pragma unroll
  for (int i = 0; i < H; ++i) {
    const T yd = eo_dot<PREC, NE, false>(c, m, i * NE, e, m, 0, e);
    const T ys = eo_dot<PREC, H, false>(c, m, H * NE + i * H, o, m, 0, o);
    y[i] = t_add<PREC>(ys, yd);
    y[N1 - 1 - i] = t_sub<PREC>(ys, yd);
  }
  if constexpr (NE > H) y[H] = eo_dot<PREC, H, false>(c, m, H * NE + H * H, o, m, 0, o);
}

// y = A x (TRANS: A^T x) with the interpolation matrix (M = MAT_S) or the
// collocation derivative (M = MAT_DC), in even-odd form
template <int PREC, int N1, bool TRANS, int M>
__device__ __forceinline__ void mv(const OperatorCoeffs& c, const typename Num<PREC>::T (&x)[N1],
                                   typename Num<PREC>::T (&y)[N1]) {
  static_assert(M == MAT_S || M == MAT_DC, "interpolation or collocation derivative");
  if constexpr (M == MAT_S) {
    constexpr int ME = TRANS ? MAT_ST : MAT_S;
    eo_apply<PREC, N1, true, false, false>(c, ME, ME, ME, x, x, y, y);
  } else {
    eo_apply_anti<PREC, N1>(c, TRANS ? MAT_DCT : MAT_DC, x, y);
  }
}

// a0 b0 + a1 b1 + a2 b2
template <int PREC>
__device__ __forceinline__ typename Num<PREC>::T dot3(typename Num<PREC>::T a0, typename Num<PREC>::T b0,
                                                     typename Num<PREC>::T a1, typename Num<PREC>::T b1,
                                                     typename Num<PREC>::T a2, typename Num<PREC>::T b2) {
  if constexpr (PREC == PREC_DD) {
    dd_acc a;
    acc_set(a, a0, b0);
    acc_madd(a, a1, b1);
    acc_madd(a, a2, b2);
    return acc_get(a);
  } else {
    return fma(a0, b0, fma(a1, b1, a2 * b2));
  }
}

// position of element (a,b,c) of a cell array (x fastest)
template <int N1>
__device__ __forceinline__ int cidx(int a, int b, int c) {
  return a + N1 * (b + N1 * c);
}

// pencil along direction `dir` with transverse indices (e1, e2): element s of the pencil
template <int N1>
__device__ __forceinline__ int pencil_idx(int dir, int e1, int e2, int s) {
  return dir == 0 ? cidx<N1>(s, e1, e2) : (dir == 1 ? cidx<N1>(e1, s, e2) : cidx<N1>(e1, e2, s));
}

// first element and stride of the pencil along `dir` with transverse indices (e1, e2)
template <int N1>
__device__ __forceinline__ void pencil_base_step(int dir, int e1, int e2, int& base, int& step) {
  constexpr int N2 = N1 * N1;
  base = dir == 0 ? N1 * (e1 + N1 * e2) : (dir == 1 ? e1 + N2 * e2 : e1 + N1 * e2);
  step = dir == 0 ? 1 : (dir == 1 ? N1 : N2);
}

// In-place application of the 1D matrix M (or its transpose) along `dir` to
// the cell arrays arr + ci*stride, ci < nc.  Ends with a barrier.  Callers
// loop over dir without unrolling: one copy of the (long, fully unrolled)
// product serves the three directions, which keeps the deformed kernels
// within the instruction cache.
template <int PREC, int P, bool TRANS, int M>
__device__ __forceinline__ void sweep_inplace(typename Num<PREC>::T* arr, int stride, int nc, int dir,
                                              const OperatorCoeffs& c) {
  using T = typename Num<PREC>::T;
  constexpr int N1 = P + 1, N2 = N1 * N1;
  for (int t = threadIdx.x; t < nc * N2; t += kThreads) {
    const int ci = t / N2, e = t - ci * N2, e1 = e % N1, e2 = e / N1;
    int base, step;
    pencil_base_step<N1>(dir, e1, e2, base, step);
    T* a = arr + ci * stride + base;
    T x[N1], y[N1];
#pragma unroll
    for (int s = 0; s < N1; ++s) x[s] = a[s * step];
    mv<PREC, N1, TRANS, M>(c, x, y);
#pragma unroll
    for (int s = 0; s < N1; ++s) a[s * step] = y[s];
  }
  __syncthreads();
}

// out = A^(T) in (accum: out += ...) along `dir`, separate arrays.  Ends with a barrier.
template <int PREC, int P, bool TRANS, int M>
__device__ __forceinline__ void sweep_copy(const typename Num<PREC>::T* in, typename Num<PREC>::T* out, int stride,
                                           int nc, int dir, bool accum, const OperatorCoeffs& c) {
  using T = typename Num<PREC>::T;
  constexpr int N1 = P + 1, N2 = N1 * N1;
  for (int t = threadIdx.x; t < nc * N2; t += kThreads) {
    const int ci = t / N2, e = t - ci * N2, e1 = e % N1, e2 = e / N1;
    int base, step;
    pencil_base_step<N1>(dir, e1, e2, base, step);
    const T* a = in + ci * stride + base;
    T* o = out + ci * stride + base;
    T x[N1], y[N1];
#pragma unroll
    for (int s = 0; s < N1; ++s) x[s] = a[s * step];
    mv<PREC, N1, TRANS, M>(c, x, y);
#pragma unroll
    for (int s = 0; s < N1; ++s) o[s * step] = accum ? t_add<PREC>(o[s * step], y[s]) : y[s];
  }
  __syncthreads();
}

// FP64 sweep with the transpose of a raw 1D table (exact diagonal)
template <int P>
__device__ __forceinline__ void sweep_inplace_table_t(double* arr, int stride, int nc, int dir, const double* A) {
  constexpr int N1 = P + 1, N2 = N1 * N1;
  for (int t = threadIdx.x; t < nc * N2; t += kThreads) {
    const int ci = t / N2, e = t - ci * N2, e1 = e % N1, e2 = e / N1;
    double* a = arr + ci * stride;
    double x[N1];
#pragma unroll
    for (int s = 0; s < N1; ++s) x[s] = a[pencil_idx<N1>(dir, e1, e2, s)];
#pragma unroll
    for (int i = 0; i < N1; ++i) {
      double s = 0.0;
#pragma unroll
      for (int j = 0; j < N1; ++j) s = fma(A[j * N1 + i], x[j], s);
      a[pencil_idx<N1>(dir, e1, e2, i)] = s;
    }
  }
  __syncthreads();
}

// Cells of one colour (parity of the tile-local cell index) with their brick
// origin offsets and global cell indices tabulated in shared memory.
struct ColorCells {
  int n;              // number of cells
  const int* org;     // brick offset of the cell's (0,0,0) node
  const int* cell;    // global lexicographic cell index
  __device__ int count() const { return n; }
};

// ------------------------------------------------------------------------------------
// Cell operators.  U: p_k (Dirichlet-masked) on the node brick (bx x by x bz),
// V: accumulated result on the same brick, S: per-cell scratch.
// ------------------------------------------------------------------------------------

// Cartesian tile, whole-brick form.  On a box of identical cells the sum over
// the cells of the Kronecker sums K_x (x) M (x) M + M (x) K_y (x) M + M (x) M (x) K_z
// is the Kronecker sum of the 1D matrices assembled along the lines of the node
// brick.  Each sweep therefore runs along whole brick lines, one cell segment
// of P+1 nodes after the other, and carries the partial result of the node
// that a segment shares with the next one in registers: no per-cell scratch,
// no colouring, three barriers per tile.  KIND 0 (first sweep):
// A <- M A, B <- K A; KIND 1: A <- M A, B <- K A + M B; KIND 2: B <- K A + M B.
// The mass operator M (x) M (x) M uses KIND 3: A <- Mk A and KIND 4: B <- Mk A.
// In place is safe: a segment writes its first P nodes after reading them and
// its last (shared) node only when the next segment has read it.
//   nlines lines; line t starts at (t % n0) * s0 + (t / n0) * s1; st is the node
//   stride along the line, ncl the number of cell segments.
template <int PREC, int P, int KIND>
__device__ __forceinline__ void brick_line_sweep(const OperatorCoeffs& c, typename Num<PREC>::T* A,
                                                 typename Num<PREC>::T* B, int nlines, int n0, int s0, int s1,
                                                 int st, int ncl, int matK) {
  using T = typename Num<PREC>::T;
  constexpr int N1 = P + 1;
  for (int t = threadIdx.x; t < nlines; t += kThreads) {
    const int i1 = t / n0, i0 = t - i1 * n0;
    T* a0 = A + i0 * s0 + i1 * s1;
    T* b0 = B + i0 * s0 + i1 * s1;
    T ca = t_zero<PREC>(), cb = t_zero<PREC>();
#pragma unroll 1
    for (int seg = 0; seg < ncl; ++seg) {
      T* a = a0 + st * P * seg;
      T* b = b0 + st * P * seg;
      T x[N1], z[N1], ya[N1], yb[N1];
#pragma unroll
      for (int s = 0; s < N1; ++s) x[s] = a[s * st];
      if constexpr (KIND == 1 || KIND == 2) {
#pragma unroll
        for (int s = 0; s < N1; ++s) z[s] = b[s * st];
      }
      if constexpr (KIND == 0) {
        eo_apply<PREC, N1, true, true, false>(c, MAT_M, matK, MAT_M, x, z, ya, yb);
      } else if constexpr (KIND == 1) {
        eo_apply<PREC, N1, true, true, true>(c, MAT_M, matK, MAT_M, x, z, ya, yb);
      } else if constexpr (KIND == 2) {
        eo_apply<PREC, N1, false, true, true>(c, MAT_M, matK, MAT_M, x, z, ya, yb);
      } else if constexpr (KIND == 3) {
        eo_apply<PREC, N1, true, false, false>(c, matK, matK, matK, x, z, ya, yb);
      } else {
        eo_apply<PREC, N1, false, true, false>(c, matK, matK, matK, x, z, ya, yb);
      }
      constexpr bool WA = KIND == 0 || KIND == 1 || KIND == 3;  // writes A
      constexpr bool WB = KIND != 3;                             // writes B
      if (seg > 0) {
        if constexpr (WA) ya[0] = t_add<PREC>(ya[0], ca);
        if constexpr (WB) yb[0] = t_add<PREC>(yb[0], cb);
      }
#pragma unroll
      for (int s = 0; s < P; ++s) {
        if constexpr (WA) a[s * st] = ya[s];
        if constexpr (WB) b[s * st] = yb[s];
      }
      if constexpr (WA) ca = ya[P];
      if constexpr (WB) cb = yb[P];
    }
    if constexpr (KIND == 0 || KIND == 1 || KIND == 3) a0[st * P * ncl] = ca;
    if constexpr (KIND != 3) b0[st * P * ncl] = cb;
  }
}

// The operator on a Cartesian tile: z, y and x sweeps along the brick lines;
// U (p_k, Dirichlet-masked) is overwritten, the result is left in V.
template <int PREC, int P>
__device__ void brick_op_affine(const OperatorCoeffs& c, typename Num<PREC>::T* U, typename Num<PREC>::T* V, int bx,
                                int by, int bz, int ncx, int ncy, int ncz, int op_kind) {
  if (op_kind == OP_MASS) {
    // h_x h_y h_z M (x) M (x) M
    brick_line_sweep<PREC, P, 3>(c, U, V, bx * by, bx, 1, bx, bx * by, ncz, MAT_M);
    __syncthreads();
    brick_line_sweep<PREC, P, 3>(c, U, V, bx * bz, bx, 1, bx * by, bx, ncy, MAT_M);
    __syncthreads();
    brick_line_sweep<PREC, P, 4>(c, U, V, by * bz, by, bx, bx * by, 1, ncx, MAT_MV);
    __syncthreads();
    return;
  }
  brick_line_sweep<PREC, P, 0>(c, U, V, bx * by, bx, 1, bx, bx * by, ncz, MAT_K2);
  __syncthreads();
  brick_line_sweep<PREC, P, 1>(c, U, V, bx * bz, bx, 1, bx * by, bx, ncy, MAT_K1);
  __syncthreads();
  brick_line_sweep<PREC, P, 2>(c, U, V, by * bz, by, bx, bx * by, 1, ncx, MAT_K0);
  __syncthreads();
}

// ------------------------------------------------------------------------------------
// Tri-quadratic geometry (GEOM_QUAD, Sec. 2.2): per cell the 27 x 3 coordinates
// X[d][a + 3 (b + 3 c)] of the mapped points (a, b, c) / 2 of the reference
// cell; the map is x_d(xi) = sum_abc X[d][abc] L_a(xi_1) L_b(xi_2) L_c(xi_3)
// with the quadratic Lagrange polynomials L through 0, 1/2, 1.
// ------------------------------------------------------------------------------------
// the partial sums of a cell's support points over (b, c) on each line (qb, qc)
// of Gauss points, for every coordinate d and first index a:
//   G[(3 (3 d + a) + k) N2 + qb + N1 qc] = sum_bc X[d][abc] Lb Lc   (k = 0),
//   sum_bc X[d][abc] Lb' Lc (k = 1),  sum_bc X[d][abc] Lb Lc' (k = 2),
// with the polynomials at (g_qb, g_qc); one more sum over a gives a point's
// position (k = 0 with La) and Jacobian column 0 (k = 0 with La'), 1 (k = 1
// with La) and 2 (k = 2 with La).
template <int PREC, int P>
__device__ void quad_lines(const OperatorCoeffs& c, const typename Num<PREC>::T* __restrict__ geo,
                           typename Num<PREC>::T* S, int stride, const ColorCells& cc) {
  using T = typename Num<PREC>::T;
  constexpr int N1 = P + 1, N2 = N1 * N1;
  const int nc = cc.count();
  for (int t = threadIdx.x; t < nc * 9 * N2; t += kThreads) {
    const int ci = t / (9 * N2), r = t - ci * 9 * N2;
    const int da = r / N2, l = r - da * N2, qb = l % N1, qc = l / N1;
    const T* X = geo + (int64_t)cc.cell[ci] * 81 + (da / 3) * 27 + da % 3;
    T s0 = t_zero<PREC>(), s1 = t_zero<PREC>(), s2 = t_zero<PREC>();
#pragma unroll
    for (int b = 0; b < 3; ++b) {
      const T x0 = X[3 * b], x1 = X[3 * b + 9], x2 = X[3 * b + 18];
      const T e0 = dot3<PREC>(x0, t_from_double<PREC>(c.q2v[qc][0]), x1, t_from_double<PREC>(c.q2v[qc][1]), x2,
                              t_from_double<PREC>(c.q2v[qc][2]));
      const T e1 = dot3<PREC>(x0, t_from_double<PREC>(c.q2d[qc][0]), x1, t_from_double<PREC>(c.q2d[qc][1]), x2,
                              t_from_double<PREC>(c.q2d[qc][2]));
      s0 = t_axpy<PREC>(t_from_double<PREC>(c.q2v[qb][b]), e0, s0);
      s1 = t_axpy<PREC>(t_from_double<PREC>(c.q2d[qb][b]), e0, s1);
      s2 = t_axpy<PREC>(t_from_double<PREC>(c.q2v[qb][b]), e1, s2);
    }
    T* G = S + ci * stride + cell_stride(P, 4) + 3 * da * N2 + l;
    G[0] = s0;
    G[N2] = s1;
    G[2 * N2] = s2;
  }
}

// position x_0 (the coefficient's argument) and Jacobian J[d][e] = d x_d / d xi_e
// at Gauss point q of a cell from its line sums G
template <int PREC, int P>
__device__ __forceinline__ void quad_jacobian(const OperatorCoeffs& c, const typename Num<PREC>::T* G, int q,
                                              typename Num<PREC>::T (&J)[3][3], typename Num<PREC>::T& x0) {
  using T = typename Num<PREC>::T;
  constexpr int N1 = P + 1, N2 = N1 * N1;
  const int qa = q % N1, l = q / N1;
  const T v0 = t_from_double<PREC>(c.q2v[qa][0]), v1 = t_from_double<PREC>(c.q2v[qa][1]),
          v2 = t_from_double<PREC>(c.q2v[qa][2]);
  const T d0 = t_from_double<PREC>(c.q2d[qa][0]), d1 = t_from_double<PREC>(c.q2d[qa][1]),
          d2 = t_from_double<PREC>(c.q2d[qa][2]);
#pragma unroll
  for (int d = 0; d < 3; ++d) {
    const T* g = G + 9 * d * N2 + l;  // (3 (3 d + a) + k) N2
    const T a00 = g[0], a01 = g[N2], a02 = g[2 * N2];
    const T a10 = g[3 * N2], a11 = g[4 * N2], a12 = g[5 * N2];
    const T a20 = g[6 * N2], a21 = g[7 * N2], a22 = g[8 * N2];
    J[d][0] = dot3<PREC>(d0, a00, d1, a10, d2, a20);
    J[d][1] = dot3<PREC>(v0, a01, v1, a11, v2, a21);
    J[d][2] = dot3<PREC>(v0, a02, v1, a12, v2, a22);
    if (d == 0) x0 = dot3<PREC>(v0, a00, v1, a10, v2, a20);
  }
}

// tensor Gauss weight of point q
__device__ __forceinline__ double quad_weight(const OperatorCoeffs& c, int q, int n1) {
  return c.w[q % n1] * c.w[(q / n1) % n1] * c.w[q / (n1 * n1)];
}

// w a(x) / det J (Laplacian, divide) or w a(x) det J (mass): FP32 in the FP32
// kernels, FP64 otherwise (double-float rounds the FP64 result)
template <int PREC>
__device__ __forceinline__ typename Num<PREC>::T quad_factor(double w, int coef, typename Num<PREC>::T det,
                                                            typename Num<PREC>::T x0, bool divide) {
  if constexpr (PREC == PREC_F32) {
    const float a = coef == MFCG_COEF_SIN_X ? 1.0f + 0.5f * sinf(3.14159265358979f * x0) : 1.0f;
    return divide ? (float)w * a / det : (float)w * a * det;
  } else {
    const double xd = t_to_double<PREC>(x0), dd_ = t_to_double<PREC>(det);
    const double a = coef == MFCG_COEF_SIN_X ? 1.0 + 0.5 * sin(3.14159265358979323846 * xd) : 1.0;
    return t_from_double<PREC>(divide ? w * a / dd_ : w * a * dd_);
  }
}

// FP64 position and Jacobian of the tri-quadratic map at Gauss point
// (qa, qb, qc) directly from the cell's 81 coordinates (set-up passes)
__device__ inline void quad_point(const OperatorCoeffs& c, const double* __restrict__ X, int qa, int qb, int qc,
                                  double (&x)[3], double (&J)[3][3]) {
  for (int d = 0; d < 3; ++d) {
    x[d] = J[d][0] = J[d][1] = J[d][2] = 0.0;
    for (int cz = 0; cz < 3; ++cz)
      for (int b = 0; b < 3; ++b)
        for (int a = 0; a < 3; ++a) {
          const double v = __ldg(X + d * 27 + a + 3 * (b + 3 * cz));
          x[d] = fma(v, c.q2v[qa][a] * c.q2v[qb][b] * c.q2v[qc][cz], x[d]);
          J[d][0] = fma(v, c.q2d[qa][a] * c.q2v[qb][b] * c.q2v[qc][cz], J[d][0]);
          J[d][1] = fma(v, c.q2v[qa][a] * c.q2d[qb][b] * c.q2v[qc][cz], J[d][1]);
          J[d][2] = fma(v, c.q2v[qa][a] * c.q2v[qb][b] * c.q2d[qc][cz], J[d][2]);
        }
  }
}

// cofactor matrix and determinant of a 3 x 3 matrix (FP64)
__device__ inline double cofactors(const double (&J)[3][3], double (&C)[3][3]) {
  for (int i = 0; i < 3; ++i)
    for (int j = 0; j < 3; ++j) {
      const int i1 = (i + 1) % 3, i2 = (i + 2) % 3, j1 = (j + 1) % 3, j2 = (j + 2) % 3;
      C[i][j] = J[i1][j1] * J[i2][j2] - J[i1][j2] * J[i2][j1];
    }
  return J[0][0] * C[0][0] + J[0][1] * C[0][1] + J[0][2] * C[0][2];
}

// Deformed cells ("inverse Jacobian load", "final tensor load" and "quadratic
// geometry compute" variants of Sec. 2.2): values at the Gauss points by three
// sweeps with the interpolation matrix S, reference gradients by three sweeps
// with the Gauss collocation derivative Dc, the per-point metric
// J^{-1} (JxW a) J^{-T} (loaded, or computed from the cell's tri-quadratic
// map), and the transposed sweeps back.
// The results of the cells stay in their scratch (element (a,b,c) of cell ci
// at S[ci*stride + cidx(a,b,c)]); gather_cell_results sums them into V.
template <int PREC, int P, int GEOM>
__device__ void cell_op_deformed(const OperatorCoeffs& c, const typename Num<PREC>::T* U, typename Num<PREC>::T* S,
                                 int bx, int by, const ColorCells& cc, const typename Num<PREC>::T* __restrict__ geo,
                                 int op_kind) {
  using T = typename Num<PREC>::T;
  constexpr int N1 = P + 1, N2 = N1 * N1, N3 = N2 * N1;
  const int nc = cc.count();
  const int stride = deformed_stride(P, GEOM);
  // gather u into s0
  for (int t = threadIdx.x; t < nc * N3; t += kThreads) {
    const int ci = t / N3, e = t - ci * N3, a = e % N1, b = (e / N1) % N1, cz = e / N2;
    S[ci * stride + e] = U[cc.org[ci] + a + bx * (b + by * cz)];
  }
  if constexpr (GEOM == GEOM_QUAD) quad_lines<PREC, P>(c, geo, S, stride, cc);
  __syncthreads();
#pragma unroll 1
  for (int dir = 0; dir < 3; ++dir) sweep_inplace<PREC, P, false, MAT_S>(S, stride, nc, dir, c);
  if constexpr (GEOM == GEOM_DEFORMED || GEOM == GEOM_QUAD) {
    if (op_kind == OP_MASS) {
      // mass operator: values at the Gauss points times JxW a, transposed interpolation
      for (int t = threadIdx.x; t < nc * N3; t += kThreads) {
        const int ci = t / N3, q = t - ci * N3;
        T* s = S + ci * stride;
        T jxw;
        if constexpr (GEOM == GEOM_QUAD) {
          T J[3][3], x0;
          quad_jacobian<PREC, P>(c, s + cell_stride(P, 4), q, J, x0);
          const T det = dot3<PREC>(J[0][0], t_axby<PREC>(J[1][1], J[2][2], t_neg<PREC>(J[1][2]), J[2][1]), J[0][1],
                                   t_axby<PREC>(J[1][2], J[2][0], t_neg<PREC>(J[1][0]), J[2][2]), J[0][2],
                                   t_axby<PREC>(J[1][0], J[2][1], t_neg<PREC>(J[1][1]), J[2][0]));
          jxw = quad_factor<PREC>(quad_weight(c, q, N1), c.coef, det, x0, false);
        } else {
          jxw = geo[(int64_t)cc.cell[ci] * 10 * N3 + 9 * N3 + q];
        }
        s[q] = t_mul<PREC>(jxw, s[q]);
      }
      __syncthreads();
#pragma unroll 1
      for (int dir = 0; dir < 3; ++dir) sweep_inplace<PREC, P, true, MAT_S>(S, stride, nc, dir, c);
      return;
    }
  }
  // reference gradients at the Gauss points (single pass over all three directions)
  for (int t = threadIdx.x; t < nc * N2 * 3; t += kThreads) {
    const int dir = t / (nc * N2);
    const int tt = t - dir * nc * N2;
    const int ci = tt / N2, e = tt - ci * N2, e1 = e % N1, e2 = e / N1;
    int base, step;
    pencil_base_step<N1>(dir, e1, e2, base, step);
    const T* a = S + ci * stride + base;
    T* o = S + ci * stride + (1 + dir) * N3 + base;
    T x[N1], y[N1];
#pragma unroll
    for (int s = 0; s < N1; ++s) x[s] = a[s * step];
    mv<PREC, N1, false, MAT_DC>(c, x, y);
#pragma unroll
    for (int s = 0; s < N1; ++s) o[s * step] = y[s];
  }
  __syncthreads();
  // metric at each point: flux = J^{-1} (JxW a) J^{-T} grad_ref
  for (int t = threadIdx.x; t < nc * N3; t += kThreads) {
    const int ci = t / N3, q = t - ci * N3;
    T* s = S + ci * stride;
    const T g0 = s[N3 + q], g1 = s[2 * N3 + q], g2 = s[3 * N3 + q];
    if constexpr (GEOM == GEOM_QUAD) {
      // tri-quadratic geometry: J at the point, its cofactors C (J^{-1} =
      // C^T / det J), physical gradient C g / det J, and the reference flux
      // J^{-1} (w det J a) J^{-T} g = (w a / det J) C^T (C g)
      T J[3][3], x0;
      quad_jacobian<PREC, P>(c, s + cell_stride(P, 4), q, J, x0);
      T C[3][3];
#pragma unroll
      for (int i = 0; i < 3; ++i)
#pragma unroll
        for (int j = 0; j < 3; ++j) {
          const int i1 = (i + 1) % 3, i2 = (i + 2) % 3, j1 = (j + 1) % 3, j2 = (j + 2) % 3;
          C[i][j] = t_axby<PREC>(J[i1][j1], J[i2][j2], t_neg<PREC>(J[i1][j2]), J[i2][j1]);
        }
      const T det = dot3<PREC>(J[0][0], C[0][0], J[0][1], C[0][1], J[0][2], C[0][2]);
      const T f = quad_factor<PREC>(quad_weight(c, q, N1), c.coef, det, x0, true);
      const T y0 = t_mul<PREC>(f, dot3<PREC>(C[0][0], g0, C[0][1], g1, C[0][2], g2));
      const T y1 = t_mul<PREC>(f, dot3<PREC>(C[1][0], g0, C[1][1], g1, C[1][2], g2));
      const T y2 = t_mul<PREC>(f, dot3<PREC>(C[2][0], g0, C[2][1], g1, C[2][2], g2));
      s[N3 + q] = dot3<PREC>(C[0][0], y0, C[1][0], y1, C[2][0], y2);
      s[2 * N3 + q] = dot3<PREC>(C[0][1], y0, C[1][1], y1, C[2][1], y2);
      s[3 * N3 + q] = dot3<PREC>(C[0][2], y0, C[1][2], y1, C[2][2], y2);
    } else if constexpr (GEOM == GEOM_TENSOR) {
      // stored symmetric tensor C = J^{-1} (JxW a) J^{-T}: flux = C grad_ref
      const T* gq = geo + (int64_t)cc.cell[ci] * 6 * N3 + q;
      const T c00 = gq[0], c01 = gq[N3], c02 = gq[2 * N3], c11 = gq[3 * N3], c12 = gq[4 * N3], c22 = gq[5 * N3];
      s[N3 + q] = dot3<PREC>(c00, g0, c01, g1, c02, g2);
      s[2 * N3 + q] = dot3<PREC>(c01, g0, c11, g1, c12, g2);
      s[3 * N3 + q] = dot3<PREC>(c02, g0, c12, g1, c22, g2);
    } else {
      const T* gq = geo + (int64_t)cc.cell[ci] * 10 * N3 + q;
      T Ji[9];
#pragma unroll
      for (int m = 0; m < 9; ++m) Ji[m] = gq[m * N3];
      const T jxw = gq[9 * N3];
      // physical gradient (J^{-T} g)_m = sum_n Ji[n][m] g_n, scaled by JxW a
      const T f0 = t_mul<PREC>(jxw, dot3<PREC>(Ji[0], g0, Ji[3], g1, Ji[6], g2));
      const T f1 = t_mul<PREC>(jxw, dot3<PREC>(Ji[1], g0, Ji[4], g1, Ji[7], g2));
      const T f2 = t_mul<PREC>(jxw, dot3<PREC>(Ji[2], g0, Ji[5], g1, Ji[8], g2));
      s[N3 + q] = dot3<PREC>(Ji[0], f0, Ji[1], f1, Ji[2], f2);
      s[2 * N3 + q] = dot3<PREC>(Ji[3], f0, Ji[4], f1, Ji[5], f2);
      s[3 * N3 + q] = dot3<PREC>(Ji[6], f0, Ji[7], f1, Ji[8], f2);
    }
  }
  __syncthreads();
  // transposed derivative sweeps, summed into s0
#pragma unroll 1
  for (int dir = 0; dir < 3; ++dir) sweep_copy<PREC, P, true, MAT_DC>(S + (1 + dir) * N3, S, stride, nc, dir, dir > 0, c);
#pragma unroll 1
  for (int dir = 0; dir < 3; ++dir) sweep_inplace<PREC, P, true, MAT_S>(S, stride, nc, dir, c);
}

// Sum of the cell results of a batch of cells [c0, c0 + nb) (tile-local
// lexicographic cell order) into the node brick: every node of the slab of
// node planes the batch touches adds the results of the batch's cells that
// contain it, in a fixed (z, y, x) cell order -- deterministic without colours.
template <int PREC, int P>
__device__ void gather_cell_results(typename Num<PREC>::T* V, const typename Num<PREC>::T* S, int stride, int c0,
                                    int nb, int ncx, int ncy, int bx, int by, const FastDiv& fbx,
                                    const FastDiv& fby) {
  using T = typename Num<PREC>::T;
  constexpr int N1 = P + 1;
  const int nxy = ncx * ncy;
  const int cz_lo = c0 / nxy, cz_hi = (c0 + nb - 1) / nxy;
  const int k_lo = P * cz_lo;
  const int n = bx * by * (P * (cz_hi - cz_lo + 1) + 1);
  for (int t = threadIdx.x; t < n; t += kThreads) {
    const int r = (int)fdiv((uint32_t)t, fbx);
    const int li = t - r * bx;
    const int q = (int)fdiv((uint32_t)r, fby);
    const int lj = r - q * by, lk = k_lo + q;
    // cells containing the node along each direction: [lo, hi]
    const int xh = min(li / P, ncx - 1), xl = li > 0 ? (li - 1) / P : 0;
    const int yh = min(lj / P, ncy - 1), yl = lj > 0 ? (lj - 1) / P : 0;
    const int zh = min(lk / P, cz_hi), zl = max(lk > 0 ? (lk - 1) / P : 0, cz_lo);
    T acc = t_zero<PREC>();
    bool any = false;
    for (int cz = zl; cz <= zh; ++cz)
      for (int cy = yl; cy <= yh; ++cy)
        for (int cx = xl; cx <= xh; ++cx) {
          const int cid = cx + ncx * (cy + ncy * cz) - c0;
          if (cid < 0 || cid >= nb) continue;
          const T val = S[cid * stride + cidx<N1>(li - P * cx, lj - P * cy, lk - P * cz)];
          acc = any ? t_add<PREC>(acc, val) : val;
          any = true;
        }
    if (any) {
      T* v = V + li + bx * (lj + by * lk);
      *v = t_add<PREC>(*v, acc);
    }
  }
}

// Right-hand side b_e = sum_q w_q det J_q f(x_q) phi(xhat_q): forcing at the
// Gauss points, then three transposed interpolation sweeps (FP64).
__device__ inline double manufactured_forcing(double x, double y, double z, int coef, int op_kind) {
  const double pi = 3.14159265358979323846;
  const double u = sin(pi * x) * sin(pi * y) * sin(pi * z);
  if (op_kind == OP_MASS) return coef == MFCG_COEF_CONSTANT ? u : (1.0 + 0.5 * sin(pi * x)) * u;
  if (coef == MFCG_COEF_CONSTANT) return 3.0 * pi * pi * u;
  const double a = 1.0 + 0.5 * sin(pi * x);
  const double cx = cos(pi * x);
  return a * 3.0 * pi * pi * u - 0.5 * pi * pi * cx * cx * sin(pi * y) * sin(pi * z);
}

template <int P, int GEOM>
__device__ void cell_rhs(const OperatorCoeffs& c, double* V, double* S, int bx, int by, const ColorCells& cc,
                         const TileGeom& g, int stride, int op_kind, const double* __restrict__ geo) {
  constexpr int N1 = P + 1, N2 = N1 * N1, N3 = N2 * N1;
  const int nc = cc.count();
  const double twopi = 6.28318530717958647692;
  for (int t = threadIdx.x; t < nc * N3; t += kThreads) {
    const int ci = t / N3, q = t - ci * N3, qa = q % N1, qb = (q / N1) % N1, qc = q / N2;
    const int cell = cc.cell[ci];
    if constexpr (GEOM == GEOM_QUAD) {
      // position and det J of the cell's tri-quadratic map
      double x[3], J[3][3], C[3][3];
      quad_point(c, geo + (int64_t)cell * 81, qa, qb, qc, x, J);
      const double detJ = cofactors(J, C);
      S[ci * stride + q] = c.w[qa] * c.w[qb] * c.w[qc] * detJ * manufactured_forcing(x[0], x[1], x[2], c.coef, op_kind);
      continue;
    }
    const int gx = cell % g.N[0], gy = (cell / g.N[0]) % g.N[1], gz = cell / (g.N[0] * g.N[1]);
    const double X = c.h[0] * (gx + c.g[qa]);
    const double Y = c.h[1] * (gy + c.g[qb]);
    const double Z = c.h[2] * (gz + c.g[qc]);
    const double sx = sin(twopi * X), sy = sin(twopi * Y), sz = sin(twopi * Z);
    const double A = c.amplitude;
    const double s = sx * sy * sz;
    const double dsum = twopi * (cos(twopi * X) * sy * sz + sx * cos(twopi * Y) * sz + sx * sy * cos(twopi * Z));
    const double detJ = c.h[0] * c.h[1] * c.h[2] * (1.0 + A * dsum);
    const double f = manufactured_forcing(X + A * s, Y + A * s, Z + A * s, c.coef, op_kind);
    S[ci * stride + q] = c.w[qa] * c.w[qb] * c.w[qc] * detJ * f;
  }
  __syncthreads();
#pragma unroll 1
  for (int dir = 0; dir < 3; ++dir) sweep_inplace<PREC_F64, P, true, MAT_S>(S, stride, nc, dir, c);
  for (int t = threadIdx.x; t < nc * N3; t += kThreads) {
    const int ci = t / N3, e = t - ci * N3, a = e % N1, b = (e / N1) % N1, cz = e / N2;
    V[cc.org[ci] + a + bx * (b + by * cz)] += S[ci * stride + e];
  }
  __syncthreads();
}

// Exact diagonal of the cell matrix of Eq. 5 with the same Gauss rule (FP64):
// diag_e(i) = sum_q sum_{d,d'} G_d(q,i) C_q^{dd'} G_{d'}(q,i), C_q = JxW a J^{-1} J^{-T},
// where G_d(q,i) is a product of 1D tables; each (d,d') term is a 3D
// contraction of C^{dd'} with the element-wise products SS, DS or DD of the 1D
// tables along each direction, i.e. three transposed sweeps.
template <int P, int GEOM>
__device__ void cell_diag(const OperatorCoeffs& c, double* V, double* S, int bx, int by, const ColorCells& cc,
                          const double* __restrict__ geo, int stride, int op_kind) {
  constexpr int N1 = P + 1, N2 = N1 * N1, N3 = N2 * N1;
  const int nc = cc.count();
  for (int t = threadIdx.x; t < nc * N3; t += kThreads) {
    const int ci = t / N3, e = t - ci * N3;
    S[ci * stride + N3 + e] = 0.0;
  }
  const int combos[6][2] = {{0, 0}, {1, 1}, {2, 2}, {0, 1}, {0, 2}, {1, 2}};
  const bool mass = op_kind == OP_MASS;
  const int ncombo = mass ? 1 : (GEOM == GEOM_AFFINE ? 3 : 6);
  for (int cb = 0; cb < ncombo; ++cb) {
    const int d0 = combos[cb][0], d1 = combos[cb][1];
    const double factor = d0 == d1 ? 1.0 : 2.0;
    for (int t = threadIdx.x; t < nc * N3; t += kThreads) {
      const int ci = t / N3, q = t - ci * N3;
      double C;
      if (GEOM == GEOM_QUAD) {
        // tri-quadratic map: JxW a (mass) or JxW a (J^{-1} J^{-T})_{d0 d1}
        // = (w a / det J) sum_m C[m][d0] C[m][d1] with the cofactors C
        const int qa = q % N1, qb = (q / N1) % N1, qc = q / N2;
        double x[3], J[3][3], Cf[3][3];
        quad_point(c, geo + (int64_t)cc.cell[ci] * 81, qa, qb, qc, x, J);
        const double det = cofactors(J, Cf);
        const double wa = c.w[qa] * c.w[qb] * c.w[qc] *
                          (c.coef == MFCG_COEF_SIN_X ? 1.0 + 0.5 * sin(3.14159265358979323846 * x[0]) : 1.0);
        if (mass) {
          C = wa * det;
        } else {
          double s = 0.0;
          for (int m = 0; m < 3; ++m) s = fma(Cf[m][d0], Cf[m][d1], s);
          C = wa / det * s;
        }
      } else if (mass) {
        // mass matrix: diag_e(i) = sum_q JxW_q a_q S(q,i)^2
        if (GEOM == GEOM_AFFINE) {
          const int qa = q % N1, qb = (q / N1) % N1, qc = q / N2;
          C = c.w[qa] * c.w[qb] * c.w[qc] * c.h[0] * c.h[1] * c.h[2];
        } else if (GEOM == GEOM_DEFORMED) {
          C = __ldg(geo + (int64_t)cc.cell[ci] * 10 * N3 + 9 * N3 + q);
        } else {
          C = 0.0;  // the final tensor stores no JxW: set-up rejects the mass operator there
        }
      } else if (GEOM == GEOM_AFFINE) {
        const int qa = q % N1, qb = (q / N1) % N1, qc = q / N2;
        C = c.w[qa] * c.w[qb] * c.w[qc] * c.h[0] * c.h[1] * c.h[2] / (c.h[d0] * c.h[d0]);
      } else if (GEOM == GEOM_TENSOR) {
        const int m = d0 == d1 ? (d0 == 0 ? 0 : (d0 == 1 ? 3 : 5)) : (d0 + d1 == 1 ? 1 : (d0 + d1 == 2 ? 2 : 4));
        C = __ldg(geo + (int64_t)cc.cell[ci] * 6 * N3 + m * N3 + q);
      } else {
        const double* gq = geo + (int64_t)cc.cell[ci] * 10 * N3 + q;
        double s = 0.0;
#pragma unroll
        for (int m = 0; m < 3; ++m) s = fma(__ldg(gq + (3 * d0 + m) * N3), __ldg(gq + (3 * d1 + m) * N3), s);
        C = __ldg(gq + 9 * N3) * s;
      }
      S[ci * stride + q] = factor * C;
    }
    __syncthreads();
#pragma unroll 1
    for (int dim = 0; dim < 3; ++dim) {
      const int nd = mass ? 0 : (dim == d0) + (dim == d1);
      sweep_inplace_table_t<P>(S, stride, nc, dim, c.T2[nd]);
    }
    for (int t = threadIdx.x; t < nc * N3; t += kThreads) {
      const int ci = t / N3, e = t - ci * N3;
      S[ci * stride + N3 + e] += S[ci * stride + e];
    }
    __syncthreads();
  }
  for (int t = threadIdx.x; t < nc * N3; t += kThreads) {
    const int ci = t / N3, e = t - ci * N3, a = e % N1, b = (e / N1) % N1, cz = e / N2;
    V[cc.org[ci] + a + bx * (b + by * cz)] += S[ci * stride + N3 + e];
  }
  __syncthreads();
}

// ------------------------------------------------------------------------------------
// Reductions of the seven sums, in a fixed order.  FP64 precision: FP64
// throughout.  Double-float and FP32 precisions: the per-thread partial sums,
// the warp and CTA stages and the grid stage are double-float pairs (FP32
// pipes); only the final seven values are converted to FP64, because on GB300
// a handful of FP64 operations per thread serialises on the FP64 pipe.
// Per-CTA rows of `partial` hold 8 doubles (FP64) or 7 float pairs.
// ------------------------------------------------------------------------------------
template <int NV>
__device__ __forceinline__ void block_reduce(double (&v)[NV], double* red) {
#pragma unroll
  for (int m = 0; m < NV; ++m) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v[m] += __shfl_down_sync(0xffffffffu, v[m], o);
  }
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  if (lane == 0) {
#pragma unroll
    for (int m = 0; m < NV; ++m) red[warp * NV + m] = v[m];
  }
  __syncthreads();
  if (threadIdx.x == 0) {
#pragma unroll
    for (int m = 0; m < NV; ++m) {
      double s = 0.0;
      for (int w = 0; w < kThreads / 32; ++w) s += red[w * NV + m];
      v[m] = s;
    }
  }
  __syncthreads();
}

__device__ __forceinline__ dd dd_shfl_down(dd a, int o) {
  return dd{__shfl_down_sync(0xffffffffu, a.hi, o), __shfl_down_sync(0xffffffffu, a.lo, o)};
}

// block sum of 7 double-float values; result valid in thread 0; red >= 56 dd
__device__ __forceinline__ void block_reduce_dd(dd (&v)[7], dd* red) {
#pragma unroll
  for (int m = 0; m < 7; ++m) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v[m] = dd_add(v[m], dd_shfl_down(v[m], o));
  }
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  if (lane == 0) {
#pragma unroll
    for (int m = 0; m < 7; ++m) red[warp * 7 + m] = v[m];
  }
  __syncthreads();
  if (threadIdx.x == 0) {
#pragma unroll
    for (int m = 0; m < 7; ++m) {
      dd s = red[m];
      for (int w = 1; w < kThreads / 32; ++w) s = dd_add(s, red[w * 7 + m]);
      v[m] = s;
    }
  }
  __syncthreads();
}

template <int PREC>
__device__ __forceinline__ dd dot_to_dd(const DotAcc<PREC>& a) {
  if constexpr (PREC == PREC_DD)
    return acc_get(a.a);
  else
    return dd{(float)a.v, 0.f};
}

// stores this CTA's seven sums into row `row` of the partial buffer
template <int PREC>
__device__ __forceinline__ void store_cta_sums(DotAcc<PREC> (&sm)[7], double* red, double* partial, int64_t row) {
  if constexpr (is_f64(PREC)) {
    double s[7];
#pragma unroll
    for (int m = 0; m < 7; ++m) s[m] = sm[m].get();
    block_reduce<7>(s, red);
    if (threadIdx.x == 0) {
#pragma unroll
      for (int m = 0; m < 7; ++m) partial[row * 8 + m] = s[m];
    }
  } else {
    dd s[7];
#pragma unroll
    for (int m = 0; m < 7; ++m) s[m] = dot_to_dd<PREC>(sm[m]);
    block_reduce_dd(s, reinterpret_cast<dd*>(red));
    if (threadIdx.x == 0) {
      dd* out = reinterpret_cast<dd*>(partial + row * 8);
#pragma unroll
      for (int m = 0; m < 7; ++m) out[m] = s[m];
    }
  }
}

// fixed-order sum of rows [0, nrows) of the partial buffer; valid in thread 0
template <int PREC>
__device__ __forceinline__ void reduce_partials(const double* partial, int64_t nrows, double* red, double (&out)[7]) {
  if constexpr (is_f64(PREC)) {
#pragma unroll
    for (int m = 0; m < 7; ++m) out[m] = 0.0;
    for (int64_t t = threadIdx.x; t < nrows; t += kThreads) {
#pragma unroll
      for (int m = 0; m < 7; ++m) out[m] += __ldcg(partial + t * 8 + m);
    }
    block_reduce<7>(out, red);
  } else {
    dd s[7];
#pragma unroll
    for (int m = 0; m < 7; ++m) s[m] = dd{0.f, 0.f};
    for (int64_t t = threadIdx.x; t < nrows; t += kThreads) {
      const float2* row = reinterpret_cast<const float2*>(partial + t * 8);
#pragma unroll
      for (int m = 0; m < 7; ++m) {
        const float2 v = __ldcg(row + m);
        s[m] = dd_add(s[m], dd{v.x, v.y});
      }
    }
    block_reduce_dd(s, reinterpret_cast<dd*>(red));
#pragma unroll
    for (int m = 0; m < 7; ++m) out[m] = dd_to_double(s[m]);
  }
}

// accumulate the seven sums of Algorithm 5 for one finalised node
template <int PREC>
__device__ __forceinline__ void post_sums(DotAcc<PREC> (&sm)[7], typename Num<PREC>::T r, typename Num<PREC>::T p,
                                          typename Num<PREC>::T v, typename Num<PREC>::T dinv) {
  using T = typename Num<PREC>::T;
  const T z = t_mul<PREC>(dinv, r);   // M^{-1} r
  const T zv = t_mul<PREC>(dinv, v);  // M^{-1} v
  sm[0].madd(r, r);                    // gamma = r.r
  sm[1].madd(p, v);                    // a = p.v
  sm[2].madd(r, v);                    // b = r.v
  sm[3].madd(v, v);                    // c = v.v
  sm[4].madd(r, z);                    // d = r.M^-1 r
  sm[5].madd(r, zv);                   // e = r.M^-1 v
  sm[6].madd(v, zv);                   // f = v.M^-1 v
}

// ------------------------------------------------------------------------------------
// The tile kernel
// ------------------------------------------------------------------------------------

// 16-byte loads and stores of VN = 16 / sizeof(T) consecutive values
template <typename T>
__device__ __forceinline__ void ld16(const T* p, T (&v)[16 / sizeof(T)]) {
  const float4 raw = *reinterpret_cast<const float4*>(p);
  memcpy(&v[0], &raw, 16);
}
template <typename T>
__device__ __forceinline__ void st16(T* p, const T (&v)[16 / sizeof(T)]) {
  float4 raw;
  memcpy(&raw, &v[0], 16);
  *reinterpret_cast<float4*>(p) = raw;
}

// position in the tile-blocked vector of brick node (li, lj, lk) of tile
// (tx, ty, tz) whose own block starts at `base` with extents (ox, oy, oz);
// nodes past the owned extent belong to the next tile along that direction
__device__ __forceinline__ int64_t brick_global_index(const TileGeom& g, int tx, int ty, int tz, int li, int lj,
                                                      int lk, int ox, int oy, int oz, int64_t base) {
  if (li < ox && lj < oy && lk < oz) return base + owned_offset(li, lj, lk, ox, oy, oz);
  const int ntx = li < ox ? tx : tx + 1, nty = lj < oy ? ty : ty + 1, ntz = lk < oz ? tz : tz + 1;
  const int nli = li < ox ? li : li - ox, nlj = lj < oy ? lj : lj - oy, nlk = lk < oz ? lk : lk - oz;
  const int nox = owned_count(g, 0, ntx), noy = owned_count(g, 1, nty), noz = owned_count(g, 2, ntz);
  return tile_base(g, ntx, nty, ntz) + owned_offset(nli, nlj, nlk, nox, noy, noz);
}

// FP32 tiles run three CTAs per SM (their shared memory allows it): keep their
// registers within 85 per thread.  The others pass 0, which leaves the register
// target to the compiler as a bound without the argument does; a minimum of
// one CTA per SM instead lets it use up to 255 registers, which halved the
// resident CTAs of many degree/mode combinations (degree 5 double-float: 150
// instead of 128 registers, 44% slower).  The tensor-core FP64 tiles are
// bounded to two CTAs per SM (their shared memory allows two): unbounded they
// take 160 registers (one CTA), and a run-time indexed table had put them at
// 128 with a 400-byte stack whose spills to L2 and DRAM doubled the kernel's
// DRAM writes.
template <int P, int MODE, int GEOM, int PREC, int NC>
__global__ void __launch_bounds__(kThreads, PREC == PREC_F32 ? 3 : (PREC == PREC_F64TC ? 2 : 0))
    tile_kernel(const TileArgs a_all, const OperatorCoeffs c) {
  using T = typename Num<PREC>::T;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  __shared__ double red[8 * (kThreads / 32)];
  // cell tables of the colour / batch loops (unused by the tensor-core operator)
  __shared__ int s_org[PREC == PREC_F64TC ? 1 : kMaxColorCells];
  __shared__ int s_cell[PREC == PREC_F64TC ? 1 : kMaxColorCells];
  const TileGeom& g = a_all.g;

  // an operator pass inside CG iterations that have already stopped
  if constexpr (MODE == MODE_OPERATOR)
    if (a_all.stop_on_done && a_all.state->done) return;
  T alpha_m = t_zero<PREC>(), beta_t = t_zero<PREC>(), xa = t_zero<PREC>(), xr = t_zero<PREC>();
  bool xupd = false;
  if constexpr (MODE == MODE_CG) {
    const CGState* st = a_all.state;
    if (st->done) return;
    // The CTAs that start beside another one on the same SM begin a fixed
    // number of clocks later, so that the two CTAs of an SM run different
    // phases (the FP64 vector work of "pre"/"post" against the integer and
    // tensor-core work of the operator) instead of the same phase in step.
    if constexpr (PREC == PREC_F64TC) {
      if (blockIdx.x >= a_all.stagger_lo && blockIdx.x < a_all.stagger_hi) {
        const long long t0 = clock64();
        while (clock64() - t0 < a_all.stagger_cycles) __nanosleep(256);
      }
    }
    const int k = st->k;
    xupd = (k > 1) && ((k & 1) || st->x_every_iter);
    if constexpr (is_f64(PREC)) {
      alpha_m = -st->alpha_prev;
      beta_t = st->beta_prev;
      xa = st->alpha_prev;
      xr = st->ratio;
    } else if constexpr (PREC == PREC_DD) {
      alpha_m = dd{st->sc[0], st->sc[1]};
      beta_t = dd{st->sc[2], st->sc[3]};
      xa = dd{st->sc[4], st->sc[5]};
      xr = dd{st->sc[6], st->sc[7]};
    } else {
      alpha_m = st->sc[0];
      beta_t = st->sc[2];
      xa = st->sc[4];
      xr = st->sc[6];
    }
  }

  const int64_t tile = blockIdx.x;
  const int tx = (int)(tile % g.nt[0]);
  const int ty = (int)((tile / g.nt[0]) % g.nt[1]);
  const int tz = (int)(tile / ((int64_t)g.nt[0] * g.nt[1]));
  const int cx0 = tx * g.T[0], cy0 = ty * g.T[1], cz0 = tz * g.T[2];
  const int ncx = min(g.T[0], g.N[0] - cx0), ncy = min(g.T[1], g.N[1] - cy0), ncz = min(g.T[2], g.N[2] - cz0);
  const int bx = P * ncx + 1, by = P * ncy + 1, bz = P * ncz + 1;
  const int Bmax = (P * g.T[0] + 1) * (P * g.T[1] + 1) * (P * g.T[2] + 1);
  const int gi0 = P * cx0, gj0 = P * cy0, gk0 = P * cz0;
  const bool lastx = tx == g.nt[0] - 1, lasty = ty == g.nt[1] - 1, lastz = tz == g.nt[2] - 1;
  const int ox = owned_count(g, 0, tx), oy = owned_count(g, 1, ty), oz = owned_count(g, 2, tz);
  const int64_t base = tile_base(g, tx, ty, tz);

  T* U = reinterpret_cast<T*>(smem_raw);
  T* V = U + Bmax;
  T* S = U + 2 * Bmax;

  // Node loops.  A tile's brick = its owned block (contiguous in the
  // tile-blocked vector: index base + o) plus the "+" faces owned by the next
  // tiles.  Dirichlet tests only in tiles that touch the domain boundary.
  const bool bnd_tile = tx == 0 || ty == 0 || tz == 0 || lastx || lasty || lastz;
  const int n_own = ox * oy * oz;
  const FastDiv fox = make_fastdiv((uint32_t)ox);
  const FastDiv fby = make_fastdiv((uint32_t)by);
  const int nfx = lastx ? 0 : by * bz, nfy = lasty ? 0 : ox * bz, nfz = lastz ? 0 : ox * oy;
  const int n_face = nfx + nfy + nfz;
  // (li, lj, lk) of owned node o (x face first, see owned_offset) and the step to the next one
  const OwnedShape osh = owned_shape(ox, oy, oz);
  auto own_coords = [&](int o, int& li, int& lj, int& lk) { owned_coords(osh, o, li, lj, lk); };
  auto own_next = [&](int& li, int& lj, int& lk) { owned_next(osh, li, lj, lk); };
  // (li, lj, lk) of "+" face node f
  auto face_coords = [&](int f, int& li, int& lj, int& lk) {
    if (f < nfx) {
      li = ox;
      lk = (int)fdiv((uint32_t)f, fby);
      lj = f - lk * by;
    } else if (f < nfx + nfy) {
      f -= nfx;
      lj = oy;
      lk = (int)fdiv((uint32_t)f, fox);
      li = f - lk * ox;
    } else {
      f -= nfx + nfy;
      lk = oz;
      lj = (int)fdiv((uint32_t)f, fox);
      li = f - lj * ox;
    }
  };

  // Deformed cells: start streaming the tile's stored geometry into L2 while
  // phase 1 runs (every prefetched line lies inside the cell's block).
  if constexpr (GEOM != GEOM_AFFINE && (MODE == MODE_CG || MODE == MODE_OPERATOR)) {
    const int cell_bytes = geo_per_cell(GEOM, P) * (int)sizeof(T);
    const int lines = (cell_bytes + 127) / 128;
    const int ncell = ncx * ncy * ncz;
    const char* geo = static_cast<const char*>(a_all.geo);
    for (int t = threadIdx.x; t < ncell * lines; t += kThreads) {
      const int ci = t / lines, l = t - ci * lines;
      const int cx = ci % ncx, cy = (ci / ncx) % ncy, cz = ci / (ncx * ncy);
      const int64_t cell = (cx0 + cx) + (int64_t)g.N[0] * ((cy0 + cy) + (int64_t)g.N[1] * (cz0 + cz));
      const size_t ptr = __cvta_generic_to_global(geo + cell * cell_bytes + (int64_t)l * 128);
      asm volatile("prefetch.global.L2 [%0];" ::"l"(ptr));
    }
  }

  // Vector-valued operator: the components one after another through phases
  // 1-3, with the per-CTA sums accumulated over all of them; the geometry and
  // the Jacobi diagonal are shared by the components.
  DotAcc<PREC> sm[7];
  // NC (1 or 3) is a template parameter: a run-time trip count moves the
  // FP64 kernel's per-thread arrays to local memory
#pragma unroll 1
  for (int comp = 0; comp < NC; ++comp) {
  const TileArgs& a = a_all;
  // this component's vectors (the diagonal, geometry and scalars are shared)
  const int64_t co = comp * a_all.comp_stride;
  constexpr int64_t ve = MODE == MODE_CG ? (int64_t)sizeof(T) : (int64_t)sizeof(double);
  auto shifted = [&](const void* ptr) -> void* {
    return ptr ? const_cast<char*>(static_cast<const char*>(ptr)) + co * ve : nullptr;
  };
  const void* const c_in0 = shifted(a_all.in0);
  const void* const c_in1 = shifted(a_all.in1);
  const void* const c_in2 = shifted(a_all.in2);
  void* const c_out0 = shifted(a_all.out0);
  void* const c_out1 = shifted(a_all.out1);
  void* const c_out2 = shifted(a_all.out2);
  void* const c_x = shifted(a_all.x);
  void* const c_shell = static_cast<char*>(a_all.shell) + comp * a_all.shell_comp_stride * (int64_t)sizeof(T);
  if (comp > 0) __syncthreads();  // the previous component is finished with U and V

  // ---------------- phase 1: pre ----------------
  // CG mode: the owned block is processed in 16-byte chunks of VN nodes (it is
  // contiguous and, when base and n_own are multiples of VN, aligned), CH
  // chunks per thread in flight; the remaining owned nodes and the "+" face
  // nodes take the scalar path with NB nodes per thread in flight.
  constexpr int NB = PREC == PREC_F32 ? 4 : 2;
  constexpr int VN = 16 / sizeof(T);
  // 16-byte chunks in flight per thread in the owned-block loops (four
  // measured slower for double-float and spill for FP64)
  constexpr int CH = 2;
  // the whole-brick affine operator overwrites V completely; the cell-wise ones accumulate into it
  constexpr bool kZeroV = !(GEOM == GEOM_AFFINE && (MODE == MODE_CG || MODE == MODE_OPERATOR));
  // 16-byte accesses need the tile's block aligned in every vector: the
  // component's vectors start co elements in, the shared diagonal does not
  const bool vec_ok = MODE == MODE_CG && (base % VN) == 0 && (co % VN) == 0 && (n_own % VN) == 0;
  const int n_chunks = vec_ok ? n_own / VN : 0;
  const int scalar_begin = vec_ok ? n_own : 0;
  if constexpr (MODE == MODE_CG) {
    const T* r_old = static_cast<const T*>(c_in0) + base;
    const T* v_old = static_cast<const T*>(c_in1) + base;
    const T* p_old = static_cast<const T*>(c_in2) + base;
    const T* dinv_o = static_cast<const T*>(a.diag_inv) + base;
    T* r_new = static_cast<T*>(c_out0) + base;
    T* p_new = static_cast<T*>(c_out2) + base;
    T* x_o = static_cast<T*>(c_x) + base;
    for (int c0 = threadIdx.x; c0 < n_chunks; c0 += CH * kThreads) {
      T r4[CH][VN], v4[CH][VN], p4[CH][VN], d4[CH][VN];
#pragma unroll
      for (int h = 0; h < CH; ++h) {
        const int c = min(c0 + h * kThreads, n_chunks - 1);
        ld16(r_old + c * VN, r4[h]);
        ld16(v_old + c * VN, v4[h]);
        ld16(p_old + c * VN, p4[h]);
        ld16(dinv_o + c * VN, d4[h]);
      }
#pragma unroll
      for (int h = 0; h < CH; ++h) {
        const int c = c0 + h * kThreads;
        if (c >= n_chunks) continue;
        T rk[VN], pk[VN];
        int li, lj, lk;
        own_coords(c * VN, li, lj, lk);
#pragma unroll
        for (int e = 0; e < VN; ++e) {
          if (e > 0) own_next(li, lj, lk);
          rk[e] = t_axpy<PREC>(alpha_m, v4[h][e], r4[h][e]);        // r_{k-1} - alpha_{k-1} v_{k-1}
          pk[e] = t_axby<PREC>(d4[h][e], rk[e], beta_t, p4[h][e]);  // M^{-1} r_k + beta_{k-1} p_{k-1}
          const int sidx = li + bx * (lj + by * lk);
          const bool dir = bnd_tile && is_dirichlet(g, gi0 + li, gj0 + lj, gk0 + lk);
          U[sidx] = dir ? t_zero<PREC>() : pk[e];
          if constexpr (kZeroV) V[sidx] = t_zero<PREC>();
        }
        st16(r_new + c * VN, rk);
        st16(p_new + c * VN, pk);
        if (xupd) {
          T xv[VN];
          ld16(x_o + c * VN, xv);
#pragma unroll
          for (int e = 0; e < VN; ++e) {
            const T dp = t_sub<PREC>(p4[h][e], t_mul<PREC>(d4[h][e], r4[h][e]));  // p_{k-1} - M^{-1} r_{k-1}
            xv[e] = t_add<PREC>(xv[e], t_axby<PREC>(xa, p4[h][e], xr, dp));
          }
          st16(x_o + c * VN, xv);
        }
      }
    }
  }
  for (int n0 = scalar_begin + threadIdx.x; n0 < n_own + n_face; n0 += NB * kThreads) {
    int64_t gi[NB];
    int sidx[NB];
    bool ok[NB], own[NB], dir[NB];
#pragma unroll
    for (int b = 0; b < NB; ++b) {
      const int n = n0 + b * kThreads;
      ok[b] = n < n_own + n_face;
      own[b] = n < n_own;
      int li, lj, lk;
      if (own[b]) {
        own_coords(n, li, lj, lk);
        gi[b] = base + n;
      } else {
        face_coords(ok[b] ? n - n_own : 0, li, lj, lk);
        gi[b] = ok[b] ? brick_global_index(g, tx, ty, tz, li, lj, lk, ox, oy, oz, base) : base;
      }
      sidx[b] = li + bx * (lj + by * lk);
      dir[b] = bnd_tile && is_dirichlet(g, gi0 + li, gj0 + lj, gk0 + lk);
    }
    if constexpr (MODE == MODE_OPERATOR) {
      double src[NB];
#pragma unroll
      for (int b = 0; b < NB; ++b) src[b] = static_cast<const double*>(c_in0)[gi[b]];
#pragma unroll
      for (int b = 0; b < NB; ++b)
        if (ok[b]) U[sidx[b]] = dir[b] ? t_zero<PREC>() : t_from_double<PREC>(src[b]);
    } else if constexpr (MODE == MODE_CG) {
      T r_o[NB], v_o[NB], p_o[NB], dinv[NB];
#pragma unroll
      for (int b = 0; b < NB; ++b) {
        r_o[b] = static_cast<const T*>(c_in0)[gi[b]];
        v_o[b] = static_cast<const T*>(c_in1)[gi[b]];
        p_o[b] = static_cast<const T*>(c_in2)[gi[b]];
        dinv[b] = static_cast<const T*>(a.diag_inv)[gi[b]];
      }
#pragma unroll
      for (int b = 0; b < NB; ++b) {
        if (!ok[b]) continue;
        const T rk = t_axpy<PREC>(alpha_m, v_o[b], r_o[b]);          // r_{k-1} - alpha_{k-1} v_{k-1}
        const T pk = t_axby<PREC>(dinv[b], rk, beta_t, p_o[b]);      // M^{-1} r_k + beta_{k-1} p_{k-1}
        U[sidx[b]] = dir[b] ? t_zero<PREC>() : pk;
        if (own[b]) {
          static_cast<T*>(c_out0)[gi[b]] = rk;
          static_cast<T*>(c_out2)[gi[b]] = pk;
          if (xupd) {
            T* x = static_cast<T*>(c_x);
            const T dp = t_sub<PREC>(p_o[b], t_mul<PREC>(dinv[b], r_o[b]));  // p_{k-1} - M^{-1} r_{k-1}
            x[gi[b]] = t_add<PREC>(x[gi[b]], t_axby<PREC>(xa, p_o[b], xr, dp));
          }
        }
      }
    }
#pragma unroll
    for (int b = 0; b < NB; ++b)
      if (kZeroV && ok[b]) V[sidx[b]] = t_zero<PREC>();
  }

  // Operator passes: L2 prefetch for the tile one wave of resident CTAs ahead
  // -- its owned input block (contiguous) and, on deformed meshes, its
  // geometry -- so that its gather reads from L2 (every prefetched line lies
  // inside the prefetched block).  The fused CG kernel, which reads four
  // vectors per node, measured 3-5% slower with it and does without.
  if constexpr (MODE == MODE_OPERATOR) {
    const int64_t ahead = tile + a_all.prefetch_ahead;
    if (a_all.prefetch_ahead > 0 && ahead < g.n_tiles) {
      const int px = (int)(ahead % g.nt[0]), py = (int)((ahead / g.nt[0]) % g.nt[1]);
      const int pz = (int)(ahead / ((int64_t)g.nt[0] * g.nt[1]));
      const int64_t pbase = tile_base(g, px, py, pz);
      const int64_t pown = (int64_t)owned_count(g, 0, px) * owned_count(g, 1, py) * owned_count(g, 2, pz);
      auto prefetch_block = [&](const void* vec, int64_t first, int64_t bytes) {
        const char* p0 = static_cast<const char*>(vec) + first;
        for (int64_t l = threadIdx.x; l * 128 < bytes; l += kThreads)
          asm volatile("prefetch.global.L2 [%0];" ::"l"(__cvta_generic_to_global(p0 + l * 128)));
      };
      constexpr int64_t ve = MODE == MODE_CG ? (int64_t)sizeof(T) : (int64_t)sizeof(double);
      prefetch_block(c_in0, pbase * ve, pown * ve);
      if constexpr (MODE == MODE_CG) {
        prefetch_block(c_in1, pbase * ve, pown * ve);
        prefetch_block(c_in2, pbase * ve, pown * ve);
        if (comp == 0) prefetch_block(a.diag_inv, pbase * ve, pown * ve);
        if (xupd) prefetch_block(c_x, pbase * ve, pown * ve);
      }
      if constexpr (GEOM != GEOM_AFFINE) {
        if (comp == 0) {
          const int64_t cell_bytes = (int64_t)geo_per_cell(GEOM, P) * (int64_t)sizeof(T);
          const int pcx = min(g.T[0], g.N[0] - px * g.T[0]), pcy = min(g.T[1], g.N[1] - py * g.T[1]);
          const int pcz = min(g.T[2], g.N[2] - pz * g.T[2]);
          // cells of one row of the tile are consecutive in the geometry array
          for (int r = 0; r < pcy * pcz; ++r) {
            const int cy = r % pcy, cz = r / pcy;
            const int64_t cell0 = (int64_t)px * g.T[0] + g.N[0] * ((int64_t)py * g.T[1] + cy + (int64_t)g.N[1] * ((int64_t)pz * g.T[2] + cz));
            prefetch_block(a.geo, cell0 * cell_bytes, pcx * cell_bytes);
          }
        }
      }
    }
  }

  // ---------------- phase 2: cell integrals ----------------
  if constexpr (PREC == PREC_F64TC && GEOM == GEOM_AFFINE && (MODE == MODE_CG || MODE == MODE_OPERATOR)) {
    __syncthreads();  // phase 1 finished with U
    tc::brick_op_affine_tc<P>(U, V, reinterpret_cast<long long*>(U + 2 * Bmax), bx, by, bz, ncx, ncy, ncz,
                              min(4, g.T[0]), min(4, g.T[1]), a.tc_frag, a.tc_g2, a.tc_r,
                              reinterpret_cast<int*>(red));
  } else if constexpr (GEOM == GEOM_AFFINE && (MODE == MODE_CG || MODE == MODE_OPERATOR)) {
    __syncthreads();  // phase 1 finished with U
    brick_op_affine<PREC, P>(c, U, V, bx, by, bz, ncx, ncy, ncz, a.op_kind);
  } else if constexpr (GEOM != GEOM_AFFINE && (MODE == MODE_CG || MODE == MODE_OPERATOR)) {
    // deformed cells: batches of consecutive cells, all cells of a batch at
    // once with their results in the scratch, then a fixed-order node gather
    const int ncell = ncx * ncy * ncz;
    const int nbmax = deformed_batch_cells(P, (int)sizeof(T), g, GEOM);
    const int stride = deformed_stride(P, GEOM);
    const FastDiv fbx = make_fastdiv((uint32_t)bx);
    for (int c0 = 0; c0 < ncell; c0 += nbmax) {
      const int nb = min(nbmax, ncell - c0);
      __syncthreads();  // previous batch gathered (and phase 1 finished with U, V)
      for (int ci = threadIdx.x; ci < nb; ci += kThreads) {
        const int cid = c0 + ci;
        const int cx = cid % ncx, cy = (cid / ncx) % ncy, cz = cid / (ncx * ncy);
        s_org[ci] = P * cx + bx * (P * cy + by * P * cz);
        s_cell[ci] = (cx0 + cx) + g.N[0] * ((cy0 + cy) + g.N[1] * (cz0 + cz));
      }
      __syncthreads();
      const ColorCells cc{nb, s_org, s_cell};
      cell_op_deformed<PREC, P, GEOM>(c, U, S, bx, by, cc, static_cast<const T*>(a.geo), a.op_kind);
      gather_cell_results<PREC, P>(V, S, stride, c0, nb, ncx, ncy, bx, by, fbx, fby);
    }
    __syncthreads();
  } else
  for (int color = 0; color < 8; ++color) {
    const int px = color & 1, py = (color >> 1) & 1, pz = color >> 2;
    const int mx = (ncx - px + 1) / 2, my = (ncy - py + 1) / 2, mz = (ncz - pz + 1) / 2;
    const int nc = mx * my * mz;
    if (nc == 0) continue;
    __syncthreads();  // previous colour finished with the tables (and phase 1 with U, V)
    for (int ci = threadIdx.x; ci < nc; ci += kThreads) {
      const int cx = px + 2 * (ci % mx), cy = py + 2 * ((ci / mx) % my), cz = pz + 2 * (ci / (mx * my));
      s_org[ci] = P * cx + bx * (P * cy + by * P * cz);
      s_cell[ci] = (cx0 + cx) + g.N[0] * ((cy0 + cy) + g.N[1] * (cz0 + cz));
    }
    __syncthreads();
    const ColorCells cc{nc, s_org, s_cell};
    if constexpr (MODE == MODE_RHS) {
      cell_rhs<P, GEOM>(c, V, S, bx, by, cc, g, cell_stride(P, GEOM == GEOM_AFFINE ? 2 : 4), a.op_kind,
                        static_cast<const double*>(a.geo));
    } else if constexpr (MODE == MODE_DIAG) {
      cell_diag<P, GEOM>(c, V, S, bx, by, cc, static_cast<const double*>(a.geo),
                         cell_stride(P, GEOM == GEOM_AFFINE ? 2 : 4), a.op_kind);
    }
  }

  // ---------------- phase 3: post ----------------
  // Owned nodes on the "-" faces of a tile with a lower neighbour, and all
  // non-Dirichlet "+" face nodes, are shared: their partial sums go to the
  // shell; the other owned nodes are final.  In the chunked path the value
  // stored for a shared owned node is a placeholder that the tail kernel
  // overwrites with the complete sum.
  T* shell = static_cast<T*>(c_shell);
  if constexpr (MODE == MODE_CG) {
    const T* r_k = static_cast<const T*>(c_out0) + base;
    const T* p_k = static_cast<const T*>(c_out2) + base;
    const T* dinv_o = static_cast<const T*>(a.diag_inv) + base;
    T* v_new = static_cast<T*>(c_out1) + base;
    for (int c0 = threadIdx.x; c0 < n_chunks; c0 += CH * kThreads) {
      T r4[CH][VN], p4[CH][VN], d4[CH][VN];
#pragma unroll
      for (int h = 0; h < CH; ++h) {
        const int c = min(c0 + h * kThreads, n_chunks - 1);
        ld16(r_k + c * VN, r4[h]);
        ld16(p_k + c * VN, p4[h]);
        ld16(dinv_o + c * VN, d4[h]);
      }
#pragma unroll
      for (int h = 0; h < CH; ++h) {
        const int c = c0 + h * kThreads;
        if (c >= n_chunks) continue;
        T vv[VN];
        int li, lj, lk;
        own_coords(c * VN, li, lj, lk);
#pragma unroll
        for (int e = 0; e < VN; ++e) {
          if (e > 0) own_next(li, lj, lk);
          const int sidx = li + bx * (lj + by * lk);
          const bool dir = bnd_tile && is_dirichlet(g, gi0 + li, gj0 + lj, gk0 + lk);
          const bool shared = !dir && ((li == 0 && tx > 0) || (lj == 0 && ty > 0) || (lk == 0 && tz > 0));
          const T vs = V[sidx];
          if (shared) {
            shell[tile * g.face_stride + shell_slot(g, li, lj, lk, bx, by, bz)] = vs;
            vv[e] = vs;
          } else {
            // p_k as stored in phase 1 (the U brick may have been overwritten by the operator)
            const T pk = p4[h][e];
            vv[e] = dir ? pk : vs;
            post_sums<PREC>(sm, r4[h][e], pk, vv[e], d4[h][e]);
          }
        }
        st16(v_new + c * VN, vv);
      }
    }
  }
  for (int n0 = scalar_begin + threadIdx.x; n0 < n_own + n_face; n0 += NB * kThreads) {
    int64_t gi[NB];
    int sidx[NB];
    bool fin[NB], dir[NB];
#pragma unroll
    for (int b = 0; b < NB; ++b) {
      const int n = n0 + b * kThreads;
      fin[b] = false;
      gi[b] = base;
      sidx[b] = 0;
      dir[b] = false;
      if (n >= n_own + n_face) continue;
      int li, lj, lk;
      const bool own = n < n_own;
      if (own)
        own_coords(n, li, lj, lk);
      else
        face_coords(n - n_own, li, lj, lk);
      sidx[b] = li + bx * (lj + by * lk);
      dir[b] = bnd_tile && is_dirichlet(g, gi0 + li, gj0 + lj, gk0 + lk);
      const bool shared = !dir[b] && (!own || (li == 0 && tx > 0) || (lj == 0 && ty > 0) || (lk == 0 && tz > 0));
      if (shared) {
        shell[tile * g.face_stride + shell_slot(g, li, lj, lk, bx, by, bz)] = V[sidx[b]];
      } else if (own) {
        fin[b] = true;
        gi[b] = base + n;
      }
    }
    if constexpr (MODE == MODE_CG) {
      T rk[NB], dv[NB], pd[NB];
#pragma unroll
      for (int b = 0; b < NB; ++b) {
        rk[b] = static_cast<const T*>(c_out0)[gi[b]];
        dv[b] = static_cast<const T*>(a.diag_inv)[gi[b]];
        pd[b] = static_cast<const T*>(c_out2)[gi[b]];
      }
#pragma unroll
      for (int b = 0; b < NB; ++b) {
        if (!fin[b]) continue;
        const T pk = pd[b];
        const T v = dir[b] ? pk : V[sidx[b]];
        static_cast<T*>(c_out1)[gi[b]] = v;
        post_sums<PREC>(sm, rk[b], pk, v, dv[b]);
      }
    } else {
#pragma unroll
      for (int b = 0; b < NB; ++b) {
        if (!fin[b]) continue;
        double* out = static_cast<double*>(c_out0);
        if constexpr (MODE == MODE_OPERATOR)
          out[gi[b]] = dir[b] ? static_cast<const double*>(c_in0)[gi[b]] : t_to_double<PREC>(V[sidx[b]]);
        else if constexpr (MODE == MODE_RHS)
          out[gi[b]] = dir[b] ? 0.0 : t_to_double<PREC>(V[sidx[b]]);
        else
          out[gi[b]] = dir[b] ? 1.0 : t_to_double<PREC>(V[sidx[b]]);
      }
    }
  }
  }  // components

  if constexpr (MODE == MODE_CG) store_cta_sums<PREC>(sm, red, a_all.partial, tile);
}

// ------------------------------------------------------------------------------------
// Tail: shared-face nodes and the scalar step of Algorithm 5
// ------------------------------------------------------------------------------------
__device__ inline void cg_scalar_step(CGState* st, const double (&s)[7]) {
  const double gam = s[0], av = s[1], bv = s[2], cv = s[3], dv = s[4], ev = s[5], fv = s[6];
  const int k = st->k;
  for (int m = 0; m < 7; ++m) st->sums[m] = s[m];
  st->iterations = k;
  bool finite = true;
  for (int m = 0; m < 7; ++m) finite = finite && isfinite(s[m]);
  if (!finite || !(av > 0.0) || !(dv > 0.0)) {
    st->done = 3;
    return;
  }
  const double alpha = dv / av;                                   // alpha_k = d_k / a_k
  double gn = fma(alpha * alpha, cv, fma(-2.0 * alpha, bv, gam)); // Eq. 8: ||r_{k+1}||^2
  if (gn < 0.0) gn = 0.0;
  st->alpha_cur = alpha;
  st->gamma_next = gn;
  if (!st->fixed && gn < st->eps_sq) {
    st->done = 1;
    return;
  }
  if (k >= st->maxit) {
    st->done = 2;
    return;
  }
  const double beta = fma(alpha * alpha, fv, fma(-2.0 * alpha, ev, dv)) / dv;  // Eq. 7
  if (!st->x_every_iter && (k + 1) % 2 == 1 && !(st->beta_prev != 0.0)) {
    // the delayed update of the next (odd) iteration divides by beta_{k-1}
    st->done = 3;
    return;
  }
  st->alpha_prev2 = st->alpha_prev;
  st->beta_prev2 = st->beta_prev;
  st->alpha_prev = alpha;
  st->beta_prev = beta;
  st->k = k + 1;
  prepare_iteration_scalars(st);
}

// three CTAs per SM (at most 85 registers) keep more of the tail's loads in flight
template <int P, int MODE, int PREC>
__global__ void __launch_bounds__(kThreads, 3) tail_kernel(const TileArgs a) {
  using T = typename Num<PREC>::T;
  __shared__ double red[8 * (kThreads / 32)];
  __shared__ int is_last;
  const TileGeom& g = a.g;
  if ((MODE == MODE_CG || a.stop_on_done) && a.state->done) return;
  DotAcc<PREC> sm[7];
  for (int comp = 0; comp < a.ncomp; ++comp) {
  const int64_t co = comp * a.comp_stride;
  const T* shell = static_cast<const T*>(a.shell) + comp * a.shell_comp_stride;
  const T* r_k = nullptr;
  const T* p_k = nullptr;
  T* v_k = nullptr;
  double* dst = nullptr;
  if constexpr (MODE == MODE_CG) {
    r_k = static_cast<const T*>(a.out0) + co;
    p_k = static_cast<const T*>(a.out2) + co;
    v_k = static_cast<T*>(a.out1) + co;
  } else {
    dst = static_cast<double*>(a.out0) + co;
  }
  // Two nodes per thread and iteration, each summing its (up to eight) shell
  // partials through a fixed 2x2x2 loop of predicated loads, so that all loads
  // of both nodes -- with r_k, p_k and D^-1 in CG mode -- are in flight
  // together; the sum order is the fixed (z, y, x) order of the contributing
  // tiles.
  const int64_t gstride = (int64_t)gridDim.x * kThreads;
  for (int64_t t0 = (int64_t)blockIdx.x * kThreads + threadIdx.x; t0 < a.tail_nodes; t0 += 2 * gstride) {
    T v[2];
    int64_t gi[2];
    bool ok[2];
    T rk[2], pk[2], dv[2];  // CG: r_k, p_k and D^-1 of the node, loaded with its shell partials
#pragma unroll
    for (int h = 0; h < 2; ++h) {
      const int64_t t = t0 + h * gstride;
      ok[h] = t < a.tail_nodes;
      v[h] = t_zero<PREC>();
      gi[h] = 0;
      if (!ok[h]) continue;
      int i, j, k;
      decode_tail_node(g, a.fam, a.tdiv, t, i, j, k);
      gi[h] = node_index(g, i, j, k);
      if constexpr (MODE == MODE_CG) {
        rk[h] = r_k[gi[h]];
        pk[h] = p_k[gi[h]];
        dv[h] = static_cast<const T*>(a.diag_inv)[gi[h]];
      }
      int txs[2], lis[2], tys[2], ljs[2], tzs[2], lks[2];
      const int nx = contributors(g, 0, i, txs, lis);
      const int ny = contributors(g, 1, j, tys, ljs);
      const int nz = contributors(g, 2, k, tzs, lks);
      T part[8];
#pragma unroll
      for (int m = 0; m < 8; ++m) {
        const int cx = m & 1, cy = (m >> 1) & 1, cz = m >> 2;
        const bool use = cx < nx && cy < ny && cz < nz;
        const int ux = use ? cx : 0, uy = use ? cy : 0, uz = use ? cz : 0;
        const int64_t tl = txs[ux] + (int64_t)g.nt[0] * (tys[uy] + (int64_t)g.nt[1] * tzs[uz]);
        const int bx = brick_extent(g, 0, txs[ux]), by = brick_extent(g, 1, tys[uy]), bz = brick_extent(g, 2, tzs[uz]);
        part[m] = use ? shell[tl * g.face_stride + shell_slot(g, lis[ux], ljs[uy], lks[uz], bx, by, bz)]
                      : t_zero<PREC>();
      }
      // the same (z, y, x) order as the contributing tiles
#pragma unroll
      for (int m = 0; m < 8; ++m) {
        const int cx = m & 1, cy = (m >> 1) & 1, cz = m >> 2;
        if (cx < nx && cy < ny && cz < nz) v[h] = m == 0 ? part[m] : t_add<PREC>(v[h], part[m]);
      }
    }
    if constexpr (MODE == MODE_CG) {
#pragma unroll
      for (int h = 0; h < 2; ++h) {
        if (!ok[h]) continue;
        v_k[gi[h]] = v[h];
        post_sums<PREC>(sm, rk[h], pk[h], v[h], dv[h]);
      }
    } else {
#pragma unroll
      for (int h = 0; h < 2; ++h)
        if (ok[h]) dst[gi[h]] = t_to_double<PREC>(v[h]);
    }
  }
  }  // components
  if constexpr (MODE == MODE_CG) {
    store_cta_sums<PREC>(sm, red, a.partial, a.g.n_tiles + blockIdx.x);
    if (threadIdx.x == 0) {
      __threadfence();
      const unsigned prev = atomicAdd(&a.state->ticket, 1u);
      is_last = (prev == gridDim.x - 1);
    }
    __syncthreads();
    if (!is_last) return;
    __threadfence();
    // last CTA: fixed-order reduction of all per-CTA sums, then the scalar step
    double s[7];
    reduce_partials<PREC>(a.partial, a.g.n_tiles + gridDim.x, red, s);
    if (threadIdx.x == 0) {
      cg_scalar_step(a.state, s);
      a.state->ticket = 0u;
    }
  }
}

// ------------------------------------------------------------------------------------
// launch helpers
// ------------------------------------------------------------------------------------
// elements of dynamic shared memory for a mode (-1: the largest over the
// modes): node bricks U and V, and the cell scratch -- none for the
// whole-brick affine operator, one colour of cells for the set-up passes, one
// batch of cells for the deformed operator
inline size_t tile_smem_elems(int P, int geom, int elem_bytes, const TileGeom& g, int mode = -1, int prec = -1) {
  const size_t Bmax = (size_t)(P * g.T[0] + 1) * (P * g.T[1] + 1) * (P * g.T[2] + 1);
  // tensor-core operator: the two bricks and the row-tile staging
  if (prec == PREC_F64TC && geom == GEOM_AFFINE && (mode == MODE_CG || mode == MODE_OPERATOR || mode == -1))
    return 2 * Bmax + tc_staging_elems(P, std::min(4, g.T[0]), std::min(4, g.T[1]));
  const size_t colour = (size_t)((g.T[0] + 1) / 2) * ((g.T[1] + 1) / 2) * ((g.T[2] + 1) / 2);
  const bool iter = mode == MODE_CG || mode == MODE_OPERATOR;
  const bool setup = mode == MODE_RHS || mode == MODE_DIAG;
  // set-up passes: one colour of cells; deformed operator passes: one batch
  const size_t colour_elems = colour * (size_t)cell_stride(P, geom == GEOM_AFFINE ? 2 : 4);
  const size_t batch_elems =
      geom == GEOM_AFFINE ? 0 : (size_t)deformed_batch_cells(P, elem_bytes, g, geom) * deformed_stride(P, geom);
  const size_t cells = iter ? batch_elems : (setup ? colour_elems : std::max(colour_elems, batch_elems));
  return 2 * Bmax + cells;
}

template <int P>
using TileFn = void (*)(const TileArgs, const OperatorCoeffs);

// supported (mode, precision, component count) triples; nullptr otherwise
template <int P, int GEOM, int NC>
TileFn<P> tile_fn_gn(int mode, int prec) {
  switch (mode) {
    case MODE_CG:
      if constexpr (GEOM == GEOM_AFFINE && tc::tc_degree(P))
        if (prec == PREC_F64TC) return tile_kernel<P, MODE_CG, GEOM, PREC_F64TC, NC>;
      return prec == PREC_F64 ? tile_kernel<P, MODE_CG, GEOM, PREC_F64, NC>
                              : (prec == PREC_DD ? tile_kernel<P, MODE_CG, GEOM, PREC_DD, NC>
                                                 : (prec == PREC_F32 ? tile_kernel<P, MODE_CG, GEOM, PREC_F32, NC>
                                                                     : nullptr));
    case MODE_OPERATOR:
      if constexpr (GEOM == GEOM_AFFINE && tc::tc_degree(P))
        if (prec == PREC_F64TC) return tile_kernel<P, MODE_OPERATOR, GEOM, PREC_F64TC, NC>;
      return prec == PREC_F64 ? tile_kernel<P, MODE_OPERATOR, GEOM, PREC_F64, NC>
                              : (prec == PREC_DD ? tile_kernel<P, MODE_OPERATOR, GEOM, PREC_DD, NC> : nullptr);
    case MODE_RHS:
      if constexpr (NC == 1) return prec == PREC_F64 ? tile_kernel<P, MODE_RHS, GEOM, PREC_F64, 1> : nullptr;
      return nullptr;
    case MODE_DIAG:
      if constexpr (NC == 1) return prec == PREC_F64 ? tile_kernel<P, MODE_DIAG, GEOM, PREC_F64, 1> : nullptr;
      return nullptr;
    default: return nullptr;
  }
}

template <int P, int GEOM>
TileFn<P> tile_fn_g(int mode, int prec, int ncomp) {
  // the tri-quadratic geometry has the scalar operator only
  if constexpr (GEOM == GEOM_QUAD)
    return ncomp == 1 ? tile_fn_gn<P, GEOM, 1>(mode, prec) : nullptr;
  else
    return ncomp == 3 ? tile_fn_gn<P, GEOM, 3>(mode, prec) : tile_fn_gn<P, GEOM, 1>(mode, prec);
}

template <int P>
TileFn<P> tile_fn(int mode, int geom, int prec, int ncomp) {
  if (geom == GEOM_AFFINE) return tile_fn_g<P, GEOM_AFFINE>(mode, prec, ncomp);
  if (geom == GEOM_TENSOR) return tile_fn_g<P, GEOM_TENSOR>(mode, prec, ncomp);
  if (geom == GEOM_QUAD) return tile_fn_g<P, GEOM_QUAD>(mode, prec, ncomp);
  return tile_fn_g<P, GEOM_DEFORMED>(mode, prec, ncomp);
}

// once per problem (outside any stream capture): allow the dynamic shared memory
template <int P>
cudaError_t prepare_tile_p(int geom, int prec, size_t smem) {
  for (int k = 0; k < 8; ++k) {
    TileFn<P> fn = tile_fn<P>(k & 3, geom, prec, k < 4 ? 1 : 3);
    if (!fn) continue;
    cudaError_t e = cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    // FP32 and whole-brick affine kernels can fit three CTAs per SM by
    // registers: give them the shared memory for it
    if (prec == PREC_F32 || geom == GEOM_AFFINE) {
      e = cudaFuncSetAttribute(fn, cudaFuncAttributePreferredSharedMemoryCarveout,
                               (int)cudaSharedmemCarveoutMaxShared);
      if (e != cudaSuccess) return e;
    }
  }
  return cudaSuccess;
}

template <int P>
int tile_occupancy_p(int mode, int geom, int prec, int ncomp, size_t smem) {
  TileFn<P> fn = tile_fn<P>(mode, geom, prec, ncomp);
  int blocks = 0;
  if (!fn || cudaOccupancyMaxActiveBlocksPerMultiprocessor(&blocks, fn, kThreads, smem) != cudaSuccess) {
    cudaGetLastError();
    return 0;
  }
  return blocks;
}

template <int P>
cudaError_t launch_tile_p(int mode, const TileArgs& a, const OperatorCoeffs& c, cudaStream_t s) {
  TileFn<P> fn = tile_fn<P>(mode, a.geom, a.prec, a.ncomp);
  if (!fn) return cudaErrorInvalidValue;
  const size_t smem = tile_smem_elems(P, a.geom, prec_bytes(a.prec), a.g, mode, a.prec) * prec_bytes(a.prec);
  fn<<<(unsigned)a.g.n_tiles, kThreads, smem, s>>>(a, c);
  return cudaGetLastError();
}

template <int P>
cudaError_t launch_tail_p(int mode, const TileArgs& a, cudaStream_t s) {
  const unsigned grid = (unsigned)(a.tail_ctas > 0 ? a.tail_ctas : 1);
  // the tensor-core operator's shell partials and sums are FP64 like PREC_F64's
  if (mode == MODE_CG) {
    if (is_f64(a.prec)) tail_kernel<P, MODE_CG, PREC_F64><<<grid, kThreads, 0, s>>>(a);
    else if (a.prec == PREC_DD) tail_kernel<P, MODE_CG, PREC_DD><<<grid, kThreads, 0, s>>>(a);
    else tail_kernel<P, MODE_CG, PREC_F32><<<grid, kThreads, 0, s>>>(a);
  } else {
    if (a.prec == PREC_DD) tail_kernel<P, MODE_OPERATOR, PREC_DD><<<grid, kThreads, 0, s>>>(a);
    else if (is_f64(a.prec)) tail_kernel<P, MODE_OPERATOR, PREC_F64><<<grid, kThreads, 0, s>>>(a);
    else return cudaErrorInvalidValue;
  }
  return cudaGetLastError();
}

}  // namespace mfcg
