// Internal declarations of the mfcg library: tile geometry, DoF numbering,
// kernel argument blocks and launch entry points.  Nothing here is part of the
// C ABI (include/mfcg.h).
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include <vector>

#include "../../include/mfcg.h"

namespace mfcg {

constexpr int kMaxDegree = 8;
constexpr int kThreads = 256;  // threads per CTA of every tile kernel

// ------------------------------------------------------------------------------------
// Tile geometry and the tile-blocked numbering of unknowns (Sec. 5.3).
//
// Cells are grouped into tiles of T[0] x T[1] x T[2] cells (ragged at the high
// end).  Every mesh node is owned by exactly one tile: along each direction
// the node index i (0..p*N) belongs to tile min(i / (p*T), nt-1), so a tile
// owns the nodes [p*T*t, p*T*(t+1)) and the last tile also owns the final
// node plane.  The unknowns of a tile are numbered contiguously (tiles in
// lexicographic order, x fastest; inside a tile lexicographic), which is the
// GPU form of "unknowns touched by a single cell batch are numbered together".
// ------------------------------------------------------------------------------------
// Division by a runtime constant d >= 1 with a multiply-high and a shift
// (round-up method): for n < 2^31, n / d == (umulhi(n, m) + n) >> s.
struct FastDiv {
  uint32_t d, m, s;
};

__host__ __device__ inline FastDiv make_fastdiv(uint32_t d) {
  FastDiv f;
  f.d = d;
  uint32_t l = 0;
  while ((1ull << l) < d) ++l;  // ceil(log2 d)
  f.s = l;
  f.m = (uint32_t)((((1ull << l) - d) << 32) / d + 1);
  return f;
}

__host__ __device__ inline uint32_t fdiv(uint32_t n, const FastDiv& f) {
#ifdef __CUDA_ARCH__
  return (__umulhi(n, f.m) + n) >> f.s;
#else
  return (uint32_t)((((uint64_t)n * f.m) >> 32) + n) >> f.s;
#endif
}

struct TileGeom {
  int p;
  int N[3];         // cells per direction
  int T[3];         // cells per tile per direction
  int nt[3];        // tiles per direction
  int nn[3];        // nodes per direction, p*N+1
  int own_last[3];  // nodes owned by the last tile per direction
  int face_stride;  // values per tile in the shell (face partial) buffer
  int64_t n_tiles;
  int64_t n_dofs;
  FastDiv div_pT[3];  // division by p*T[d]
};

__host__ __device__ inline int owned_count(const TileGeom& g, int d, int t) {
  return t == g.nt[d] - 1 ? g.own_last[d] : g.p * g.T[d];
}

__host__ __device__ inline int tile_of(const TileGeom& g, int d, int i) {
  const int t = (int)fdiv((uint32_t)i, g.div_pT[d]);
  return t < g.nt[d] - 1 ? t : g.nt[d] - 1;
}

// first index of the owned block of tile (tx, ty, tz)
__host__ __device__ inline int64_t tile_base(const TileGeom& g, int tx, int ty, int tz) {
  const int oy = owned_count(g, 1, ty), oz = owned_count(g, 2, tz);
  return (int64_t)g.nn[0] * g.nn[1] * (g.p * g.T[2]) * tz + (int64_t)g.nn[0] * (g.p * g.T[1]) * ty * oz +
         (int64_t)(g.p * g.T[0]) * tx * oy * oz;
}

// Position of owned node (li, lj, lk) inside its tile's block of ox*oy*oz
// values, "x face first": the li = 0 plane (lj fastest) comes first, then the
// nodes with li >= 1 in lexicographic order (rows of ox - 1; ox >= 2 always).
// The li = 0 plane holds the nodes shared with the lower x neighbour, so the
// tail kernel reads and writes them contiguously.
__host__ __device__ inline int64_t owned_offset(int li, int lj, int lk, int ox, int oy, int oz) {
  if (li == 0) return lj + (int64_t)oy * lk;
  return (int64_t)oy * oz + (li - 1) + (int64_t)(ox - 1) * (lj + (int64_t)oy * lk);
}

// Decoding of owned positions in the same order: coordinates of position o,
// and the step to the next position.
struct OwnedShape {
  int ox, oy, oz;
  FastDiv foy, fox1;
};

__host__ __device__ inline OwnedShape owned_shape(int ox, int oy, int oz) {
  return {ox, oy, oz, make_fastdiv((uint32_t)oy), make_fastdiv((uint32_t)(ox - 1))};
}

__host__ __device__ inline void owned_coords(const OwnedShape& s, int o, int& li, int& lj, int& lk) {
  const int n_xface = s.oy * s.oz;
  if (o < n_xface) {
    li = 0;
    lk = (int)fdiv((uint32_t)o, s.foy);
    lj = o - lk * s.oy;
    return;
  }
  const int r = o - n_xface;
  const int row = (int)fdiv((uint32_t)r, s.fox1);
  li = 1 + r - row * (s.ox - 1);
  lk = (int)fdiv((uint32_t)row, s.foy);
  lj = row - lk * s.oy;
}

__host__ __device__ inline void owned_next(const OwnedShape& s, int& li, int& lj, int& lk) {
  if (li == 0) {
    if (++lj == s.oy) {
      lj = 0;
      if (++lk == s.oz) {
        lk = 0;
        li = 1;
      }
    }
  } else if (++li == s.ox) {
    li = 1;
    if (++lj == s.oy) {
      lj = 0;
      ++lk;
    }
  }
}

// position of node (i,j,k) in the tile-blocked vector
__host__ __device__ inline int64_t node_index(const TileGeom& g, int i, int j, int k) {
  const int tx = tile_of(g, 0, i), ty = tile_of(g, 1, j), tz = tile_of(g, 2, k);
  const int ox = owned_count(g, 0, tx), oy = owned_count(g, 1, ty), oz = owned_count(g, 2, tz);
  const int pTx = g.p * g.T[0], pTy = g.p * g.T[1], pTz = g.p * g.T[2];
  const int li = i - pTx * tx, lj = j - pTy * ty, lk = k - pTz * tz;
  const int64_t base = (int64_t)g.nn[0] * g.nn[1] * pTz * tz + (int64_t)g.nn[0] * pTy * ty * oz +
                       (int64_t)pTx * tx * oy * oz;
  return base + owned_offset(li, lj, lk, ox, oy, oz);
}

__host__ __device__ inline bool is_dirichlet(const TileGeom& g, int i, int j, int k) {
  return i == 0 || j == 0 || k == 0 || i == g.nn[0] - 1 || j == g.nn[1] - 1 || k == g.nn[2] - 1;
}

// Shell buffer: every tile stores the partial operator result of its boundary
// nodes that are shared with a neighbouring tile, face by face (x-, x+, y-, y+,
// z-, z+); a node on several faces of the tile is stored on the first of them
// in that order.  Slot of tile-local node (li,lj,lk) with brick extents
// bx,by,bz (= p*cells+1 of this tile) and maximal extents Bx,By,Bz.
__host__ __device__ inline int shell_slot(const TileGeom& g, int li, int lj, int lk, int bx, int by, int bz) {
  const int Bx = g.p * g.T[0] + 1, By = g.p * g.T[1] + 1, Bz = g.p * g.T[2] + 1;
  const int FX = By * Bz, FY = Bx * Bz, FZ = Bx * By;
  if (li == 0) return lj + By * lk;
  if (li == bx - 1) return FX + lj + By * lk;
  if (lj == 0) return 2 * FX + li + Bx * lk;
  if (lj == by - 1) return 2 * FX + FY + li + Bx * lk;
  if (lk == 0) return 2 * FX + 2 * FY + li + Bx * lj;
  return 2 * FX + 2 * FY + FZ + li + Bx * lj;
}

// ------------------------------------------------------------------------------------
// Enumeration of the shared-face nodes finalised by the tail kernel: interior
// (non-Dirichlet) nodes lying on at least one tile boundary plane, split into
// three families (on an x plane; on a y plane but no x plane; on a z plane
// only), each a product set that is decoded arithmetically.
// ------------------------------------------------------------------------------------
// Divisors of the tail enumeration (fixed per problem).
struct TailDiv {
  FastDiv yz;    // (nn_y - 2)(nn_z - 2): x-plane family
  FastDiv y;     // nn_y - 2
  FastDiv xz;    // nxr (nn_z - 2): y-plane family
  FastDiv xr;    // nxr = interior x indices off the x planes
  FastDiv xy;    // nxr * nyr: z-plane family
  FastDiv pTm1[2];  // p*T - 1 along x and y (rank -> index off the planes)
};

// rank r of an interior node index that is not a tile boundary plane -> index
__host__ __device__ inline int skip_planes(int r, const FastDiv& pTm1) { return r + 1 + (int)fdiv((uint32_t)r, pTm1); }

__host__ __device__ inline void decode_tail_node(const TileGeom& g, const int64_t (&fam)[3], const TailDiv& td,
                                                 int64_t t64, int& i, int& j, int& k) {
  const int pTx = g.p * g.T[0], pTy = g.p * g.T[1], pTz = g.p * g.T[2];
  uint32_t t = (uint32_t)t64;
  if (t64 < fam[0]) {  // i on an x plane, j, k interior
    const uint32_t b = fdiv(t, td.yz);
    const uint32_t rem = t - b * td.yz.d;
    const uint32_t q = fdiv(rem, td.y);
    i = pTx * (int)(b + 1);
    j = 1 + (int)(rem - q * td.y.d);
    k = 1 + (int)q;
    return;
  }
  t = (uint32_t)(t64 - fam[0]);
  if (t64 < fam[0] + fam[1]) {  // j on a y plane
    const uint32_t b = fdiv(t, td.xz);
    const uint32_t rem = t - b * td.xz.d;
    const uint32_t q = fdiv(rem, td.xr);
    j = pTy * (int)(b + 1);
    i = skip_planes((int)(rem - q * td.xr.d), td.pTm1[0]);
    k = 1 + (int)q;
    return;
  }
  t = (uint32_t)(t64 - fam[0] - fam[1]);
  const uint32_t b = fdiv(t, td.xy);
  const uint32_t rem = t - b * td.xy.d;
  const uint32_t q = fdiv(rem, td.xr);
  k = pTz * (int)(b + 1);
  i = skip_planes((int)(rem - q * td.xr.d), td.pTm1[0]);
  j = skip_planes((int)q, td.pTm1[1]);
}

// tiles containing node index i along direction d: up to two (tile, local index) pairs
__host__ __device__ inline int contributors(const TileGeom& g, int d, int i, int (&t)[2], int (&l)[2]) {
  const int pT = g.p * g.T[d];
  const int q = (int)fdiv((uint32_t)i, g.div_pT[d]);
  if (i == q * pT && i > 0 && i < g.nn[d] - 1) {
    t[0] = q - 1;
    l[0] = pT;
    t[1] = q;
    l[1] = 0;
    return 2;
  }
  t[0] = q < g.nt[d] - 1 ? q : g.nt[d] - 1;
  l[0] = i - pT * t[0];
  return 1;
}

__host__ __device__ inline int brick_extent(const TileGeom& g, int d, int t) {
  const int cells = g.N[d] - t * g.T[d];
  return g.p * (g.T[d] < cells ? g.T[d] : cells) + 1;
}

// Tile geometry for degree p, cells N and tile edges T (each clamped to N),
// and the sizes of the three tail-node families.
inline void init_tile_geom(int p, const int N[3], const int T[3], TileGeom& g, int64_t (&fam)[3], TailDiv* td = nullptr) {
  g.p = p;
  for (int d = 0; d < 3; ++d) {
    g.N[d] = N[d];
    g.T[d] = T[d] < N[d] ? T[d] : N[d];
    g.nt[d] = (N[d] + g.T[d] - 1) / g.T[d];
    g.nn[d] = p * N[d] + 1;
    g.own_last[d] = g.nn[d] - p * g.T[d] * (g.nt[d] - 1);
  }
  for (int d = 0; d < 3; ++d) g.div_pT[d] = make_fastdiv((uint32_t)(p * g.T[d]));
  const int Bx = p * g.T[0] + 1, By = p * g.T[1] + 1, Bz = p * g.T[2] + 1;
  g.face_stride = 2 * (By * Bz + Bx * Bz + Bx * By);
  g.n_tiles = (int64_t)g.nt[0] * g.nt[1] * g.nt[2];
  g.n_dofs = (int64_t)g.nn[0] * g.nn[1] * g.nn[2];
  const int64_t nbx = g.nt[0] - 1, nby = g.nt[1] - 1, nbz = g.nt[2] - 1;
  const int64_t nix = g.nn[0] - 2, niy = g.nn[1] - 2, niz = g.nn[2] - 2;
  fam[0] = fam[1] = fam[2] = 0;
  if (nix > 0 && niy > 0 && niz > 0) {
    fam[0] = nbx * niy * niz;
    fam[1] = nby * (nix - nbx) * niz;
    fam[2] = nbz * (nix - nbx) * (niy - nby);
  }
  if (td) {
    auto nz1 = [](int64_t v) { return (uint32_t)(v > 0 ? v : 1); };
    td->yz = make_fastdiv(nz1(niy * niz));
    td->y = make_fastdiv(nz1(niy));
    td->xz = make_fastdiv(nz1((nix - nbx) * niz));
    td->xr = make_fastdiv(nz1(nix - nbx));
    td->xy = make_fastdiv(nz1((nix - nbx) * (niy - nby)));
    td->pTm1[0] = make_fastdiv(nz1(p * g.T[0] - 1));
    td->pTm1[1] = make_fastdiv(nz1(p * g.T[1] - 1));
  }
}

// ------------------------------------------------------------------------------------
// Device-resident CG scalars (Algorithm 5 / Algorithm 1); no host round trip
// per iteration.
// ------------------------------------------------------------------------------------
struct CGState {
  double alpha_prev, beta_prev;    // alpha_{k-1}, beta_{k-1}
  double alpha_prev2, beta_prev2;  // alpha_{k-2}, beta_{k-2}
  double alpha_cur;                // alpha_k of the last finished iteration
  double gamma_next;               // ||r_{k+1}||^2 (Eq. 8 expansion or explicit)
  double eps_sq;                   // (rtol ||b||)^2
  double e_cur;                    // r^T z of Algorithm 1 (unfused path)
  double sums[8];                  // last reduced sums
  int k;                           // iteration to run next (1-based)
  int done;                        // 0 running, 1 converged, 2 maxit, 3 breakdown
  int maxit;
  int iterations;                  // finished iterations
  unsigned int ticket;             // last-CTA election counter
  int x_every_iter;                // 1: x += alpha_{k-1} p_{k-1} every iteration instead of the delayed update
  int fixed;                       // 1: ignore the tolerance, run maxit iterations
  int pad;
  // scalars of the next iteration, prepared once by the scalar step so that the
  // tile kernels need no FP64 arithmetic: ratio = alpha_{k-2}/beta_{k-2} (0 unless
  // k is odd and > 1), and float pairs (hi, lo) of -alpha_{k-1}, beta_{k-1},
  // alpha_{k-1}, ratio
  double ratio;
  float sc[8];
};

// fills ratio and sc[] from alpha_prev, beta_prev, alpha_prev2, beta_prev2, k
__host__ __device__ inline void prepare_iteration_scalars(CGState* st) {
  const int k = st->k;
  st->ratio = (!st->x_every_iter && k > 1 && (k & 1)) ? st->alpha_prev2 / st->beta_prev2 : 0.0;
  const double v[4] = {-st->alpha_prev, st->beta_prev, st->alpha_prev, st->ratio};
  for (int m = 0; m < 4; ++m) {
    const float hi = (float)v[m];
    st->sc[2 * m] = hi;
    st->sc[2 * m + 1] = (float)(v[m] - (double)hi);
  }
}

enum TileMode { MODE_OPERATOR = 0, MODE_CG = 1, MODE_RHS = 2, MODE_DIAG = 3 };

// GEOM_QUAD: the tri-quadratic geometry of Sec. 2.2, 27 x 3 point
// coordinates per cell with the metric computed at each quadrature point
enum GeomKind { GEOM_AFFINE = 0, GEOM_DEFORMED = 1, GEOM_TENSOR = 2, GEOM_QUAD = 3 };

// values stored per quadrature point by the geometry kinds with per-point data
__host__ __device__ constexpr int geo_values(int geom) { return geom == GEOM_TENSOR ? 6 : 10; }

// values stored per cell: the per-point data of (p+1)^3 points, or the 81
// support-point coordinates of the tri-quadratic geometry ([3][27], point
// a + 3 (b + 3 c) at the reference coordinates (a, b, c) / 2)
__host__ __device__ constexpr int geo_per_cell(int geom, int p) {
  return geom == GEOM_QUAD ? 81 : geo_values(geom) * (p + 1) * (p + 1) * (p + 1);
}

enum MatId { MAT_M = 0, MAT_K0 = 1, MAT_K1 = 2, MAT_K2 = 3, MAT_S = 4, MAT_DC = 5, MAT_MV = 6, MAT_ST = 7, MAT_DCT = 8, NMAT = 9 };

// operator of the problem: Laplacian (Eq. 5) or mass matrix
enum OpKind { OP_LAPLACE = 0, OP_MASS = 1 };
constexpr int kMat = (kMaxDegree + 1) * (kMaxDegree + 1);

struct OperatorCoeffs {
  // 1D matrices, row-major (P+1)x(P+1): MAT_M the reference mass matrix,
  // MAT_K0..2 the reference stiffness scaled per direction for box cells
  // (h_y h_z / h_x, ...), MAT_S the interpolation from the Gauss-Lobatto
  // nodes to the Gauss points, MAT_DC the Gauss collocation derivative,
  // MAT_MV the mass matrix scaled by the cell volume h_x h_y h_z, MAT_ST and
  // MAT_DCT the transposes of MAT_S and MAT_DC.
  double mat[NMAT][kMat];
  // products of 1D tables used by the exact diagonal: SS = S.*S, DS = D.*S,
  // DD = D.*D with D[q][a] = L_a'(g_q)
  double T2[3][kMat];
  // the same matrices as float pairs (hi + lo) for the double-float and FP32 paths
  // Even-odd form, with e_j = x_j + x_{n-1-j}, o_j = x_j - x_{n-1-j} (j < h =
  // n/2) and e_h = x_h for odd n.  Centrosymmetric matrices (A[n-1-i][n-1-j]
  // = A[i][j]: M, K_d, S, S^T, the scaled M): ye = E e (ceil(n/2) rows,
  // stride ceil(n/2)) and yo = O o (h rows, stride h, stored after E) give
  // y_i = ye_i + yo_i, y_{n-1-i} = ye_i - yo_i (i < h), y_h = ye_h.
  // Anti-centrosymmetric matrices (A[n-1-i][n-1-j] = -A[i][j]: the collocation
  // derivative and its transpose): yd = E' e (h rows, stride ceil(n/2)) and
  // ys = O' o (ceil(n/2) rows, stride h, stored after E') give
  // y_i = ys_i + yd_i, y_{n-1-i} = ys_i - yd_i (i < h), y_h = ys_h.
  double eo[NMAT][kMat];
  float eoh[NMAT][kMat];
  float eol[NMAT][kMat];
  double w[kMaxDegree + 1];  // Gauss weights on [0,1]
  double g[kMaxDegree + 1];  // Gauss points on [0,1]
  // quadratic Lagrange polynomials through 0, 1/2, 1 (the tri-quadratic
  // geometry) and their derivatives at the Gauss points: [q][a]
  double q2v[kMaxDegree + 1][3];
  double q2d[kMaxDegree + 1][3];
  double h[3];               // cell sizes
  double amplitude;
  int coef;
};

struct TileArgs {
  TileGeom g;
  // operator / right-hand side / diagonal modes: in0 = src (FP64), out0 = dst (FP64)
  // CG mode (vectors in the storage type of the precision): in0 = r_old,
  // in1 = v_old, in2 = p_old, diag_inv; out0 = r_new, out1 = v_new, out2 = p_new, x
  const void* in0;
  const void* in1;
  const void* in2;
  const void* diag_inv;
  void* out0;
  void* out1;
  void* out2;
  void* x;
  void* shell;           // partial sums of shared-face nodes, arithmetic type of the precision
  double* partial;       // [n_tiles][8] (main) and [tail CTAs][8] (tail)
  const void* geo;       // deformed: [cell][10][nq] = J^{-1} row-major, JxW*a; tensor: [cell][6][nq]
                         // = C00 C01 C02 C11 C12 C22 of J^{-1} (JxW a) J^{-T} (precision's type)
  CGState* state;
  int stop_on_done;      // operator passes inside CG iterations: return at once when state->done is
                         // set (the remaining iterations of a CUDA graph after convergence)
  int64_t tail_nodes;    // number of shared-face nodes handled by the tail kernel
  int64_t fam[3];        // tail enumeration: nodes in the x / y / z boundary-plane families
  TailDiv tdiv;          // divisors of the tail enumeration
  int geom;              // GeomKind
  int prec;              // Prec (precision.cuh)
  int ncomp;             // components of the vector-valued operator (1: scalar); the vectors hold
                         // them one after another, comp_stride nodes apart; diag_inv is shared
  int64_t comp_stride;   // nodes per component (= g.n_dofs)
  int64_t shell_comp_stride;  // shell elements per component (= g.n_tiles * g.face_stride)
  int op_kind;           // OpKind
  int tail_ctas;
  int stagger_lo, stagger_hi;  // fused tensor-core iterations: CTAs blockIdx in [lo, hi) -- those that
  long long stagger_cycles;    // start beside another CTA on the same SM -- begin stagger_cycles later
  int prefetch_ahead;    // operator passes: during its cell phase, a CTA prefetches into L2 the
                         // owned input block (and geometry) of tile blockIdx + prefetch_ahead
                         // (the CTAs resident in one wave); 0 = off
  const uint2* tc_frag;  // PREC_F64TC: digit fragments of the even-odd cell-matrix blocks (tc_tables.cu)
  int tc_g2;             // PREC_F64TC: the blocks are Bint 2^-tc_g2
  int tc_r;              // PREC_F64TC: right shift of the recombined digit products (56..72)
};

// tensor-core cell operator (tc_tables.cu): B-fragment table, fixed-point
// exponent g2 and result shift r of the degree-p Cartesian cell matrix (0 on
// success), and the shared-memory elements of its staging areas for row tiles
// of up to mx x my cells
int build_tc_fragments(int p, const OperatorCoeffs& c, int op_kind, std::vector<uint2>& frag, int& g2, int& r);
size_t tc_staging_elems(int p, int mx, int my);

// launchers (one set per degree, see tile_kernels.cuh)
cudaError_t launch_tile(int degree, int mode, const TileArgs& a, const OperatorCoeffs& c, cudaStream_t s);
cudaError_t launch_tail(int degree, int mode, const TileArgs& a, cudaStream_t s);
// dynamic shared memory of a tile kernel launch of `mode` (-1: the largest over the modes)
size_t tile_smem_bytes(int degree, int geom, int prec, const TileGeom& g, int mode = -1);
cudaError_t prepare_tile(int degree, int geom, int prec, size_t smem);
// resident CTAs per SM of the fused CG tile kernel (0 on error)
int tile_occupancy(int degree, int mode, int geom, int prec, int ncomp, size_t smem);

// BLAS-1 / reduction / utility kernels (cg_kernels.cu)
cudaError_t launch_fill(double* v, double value, int64_t n, cudaStream_t s);
cudaError_t launch_invert(const double* in, double* out, int64_t n, cudaStream_t s);
cudaError_t launch_reorder(const TileGeom& g, const double* in, double* out, int to_lex, cudaStream_t s);
cudaError_t launch_geometry(const TileGeom& g, const OperatorCoeffs& c, int geom, double* geo, cudaStream_t s);

// CG drivers (cg_kernels.cu)
struct UnfusedArgs {
  int64_t n;
  const double* diag_inv;
  double* x;
  double* r;
  double* p;
  double* v;
  double* z;
  double* partial;
  int n_ctas;
  CGState* state;
};
cudaError_t launch_unfused_dot(int which, const UnfusedArgs& a, cudaStream_t s);
cudaError_t launch_unfused_axpy(int which, const UnfusedArgs& a, cudaStream_t s);
cudaError_t launch_loop_fused(int which, const UnfusedArgs& a, cudaStream_t s);
cudaError_t launch_cg_init(CGState* st, const double* b, const double* r0, int64_t n, double rtol, int maxit,
                           int fixed, double* partial, int x_every_iter, cudaStream_t s);
cudaError_t launch_residual(const double* b, const double* ax, double* r, int64_t n, cudaStream_t s);
cudaError_t launch_residual_norm(const double* b, const double* ax, int64_t n, double* partial, unsigned int* ticket,
                                 double* out, cudaStream_t s);
cudaError_t launch_scale(const double* in, double* out, double factor, int64_t n, cudaStream_t s);
cudaError_t launch_gather_done(const CGState* const* states, int count, int* done, cudaStream_t s);
cudaError_t launch_finalize_fused(int prec, int64_t n, CGState* st, void* x, const void* p0, const void* p1,
                                  const void* r0, const void* r1, const void* diag_inv, cudaStream_t s);
cudaError_t launch_to_prec(int prec, const double* in, void* out, int64_t n, cudaStream_t s);
cudaError_t launch_semi_pre(int64_t n, const CGState* st, double* x, double* r, double* p, const double* v,
                            const double* dinv, cudaStream_t s);
cudaError_t launch_semi_post(int64_t n, CGState* st, const double* r, const double* p, const double* v,
                             const double* dinv, double* partial, cudaStream_t s);
cudaError_t launch_from_prec(int prec, const void* in, double* out, int64_t n, int accumulate, cudaStream_t s);

}  // namespace mfcg
