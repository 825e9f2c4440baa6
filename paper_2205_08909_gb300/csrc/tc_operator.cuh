// Cartesian cell operator of Eq. 5 on the FP16 tensor cores with FP64 accuracy.
//
// On a tile of identical box cells every cell applies the same matrix
//   A_e = (h_y h_z/h_x) K (x) M (x) M + (h_x h_z/h_y) M (x) K (x) M + (h_x h_y/h_z) M (x) M (x) K
// (x fastest; M, K the 1D Gauss-Lobatto mass and stiffness matrices with the
// (p+1)-point Gauss rule).  The 1D matrices are centrosymmetric, so the even-odd
// transform of a cell's (p+1)^3 values along x, y and z (e_j = u_j + u_{n-1-j},
// o_j = u_j - u_{n-1-j}, the middle value kept) makes A_e block diagonal with
// eight blocks B_(sx,sy,sz), one per parity triple, each the same Kronecker sum
// of the 1D even/odd blocks.  Per block and row tile of 16 cells, Y = X B^T is
// a small dense product: the GEMM of this operator.
//
// Exactness.  The tile's values become 64-bit fixed-point integers with one
// exponent per tile (|X| <= 2^57; the transform adds at most 2^3), the block
// matrices 64-bit fixed-point integers with one exponent per problem
// (|B| < 2^62).  Both split into eight balanced 8-bit digits in [-128, 127],
// X = sum_k 2^(8k) d_k (the bytes of X + 0x8080...80, each minus 128) and
// B = sum_l 2^(8l) c_l.  Every digit is an integer that FP16 holds exactly,
// every digit product is exact in the tensor core, and the FP32 accumulator
// sums them exactly while every partial sum is an integer below 2^22; digit
// pairs of equal weight s = k + l share an accumulator within that bound
// (Plan).  Pairs with s < kSmin are dropped (their weight is below 2^-57 of the
// result's range).  The accumulators are converted to integers, recombined as
// sum_s 2^(8s - R) D_s in 64-bit arithmetic (R per problem, so that the final
// node values use the whole 62-bit range), transformed back, summed over
// the cells of each node (integer additions: order-independent, so reruns are
// bitwise identical) and converted to FP64 once per node.  Against the
// product of the FP64 input and the same block matrices in extended precision
// the result differs by a few units of 2^-53 of the tile's largest entry up to
// degree 4 (up to about 30 units at degree 8); the scheme is restated and
// checked in exact arithmetic by the host tests.
//
// This is an Ozaki-type error-free splitting (Ozaki, Ogita, Oishi, Rump,
// "Error-free transformations of matrix multiplication by using fast routines
// of matrix multiplication and its applications", Numer. Algorithms 2012),
// here with fixed-point digits and integer recombination.
#pragma once

#include <cuda_fp16.h>

#include "mfcg_internal.h"

namespace mfcg {
namespace tc {

constexpr int kDigits = 8;           // 8-bit digits per 64-bit operand
constexpr int kSmin = 6;             // digit pairs (k, l) with k + l >= kSmin are kept
constexpr int kXBits = 57;           // |X| <= 2^57 in the tile's fixed point
constexpr int kRBase = 64;           // result = (sum over the digit pairs) / 2^R, R = 64 + delta, |delta| <= 8
constexpr int kKChunk = 32;          // contraction indices per accumulator pass (two k16 steps)
constexpr int kAccLimit = 1 << 22;   // exact-integer range of an accumulator (float -> int via 1.5 2^23)
constexpr int kMCells = 16;          // cells per MMA row tile (m16)

// Degrees with tensor-core kernels.  At degrees 6 and 8 the staging does not
// fit the 227 KB of shared memory next to the default node bricks (19^3 and
// 17^3 nodes), so those degrees keep the FP64 sweeps and their tensor-core
// kernels are not instantiated (they also take the compiler many minutes).
__host__ __device__ constexpr bool tc_degree(int P) { return P <= 5 || P == 7; }

template <int P>
struct Shape {
  static constexpr int N1 = P + 1;
  static constexpr int NO = N1 / 2;   // odd part
  static constexpr int NE = N1 - NO;  // even part (includes the middle value for odd N1)
  static constexpr int N3 = N1 * N1 * N1;
  __host__ __device__ static constexpr int ext(int s) { return s ? NO : NE; }
  // block b = sx + 2 sy + 4 sz
  __host__ __device__ static constexpr int bsize(int b) { return ext(b & 1) * ext((b >> 1) & 1) * ext(b >> 2); }
  __host__ __device__ static constexpr int kpad(int b) { return (bsize(b) + 15) / 16 * 16; }
  __host__ __device__ static constexpr int npad(int b) { return (bsize(b) + 7) / 8 * 8; }
  __host__ __device__ static constexpr int ksteps(int b) { return kpad(b) / 16; }
  __host__ __device__ static constexpr int ntiles(int b) { return npad(b) / 8; }
  // staging rows hold the blocks one after another, each rounded up to an even
  // count (16-byte pairs); columns a fragment reads beyond a block are zero
  // by predication, the rounding slot is zero in memory
  __host__ __device__ static constexpr int bev(int b) { return (bsize(b) + 1) / 2 * 2; }
  __host__ __device__ static constexpr int boff(int b) {
    int o = 0;
    for (int i = 0; i < b; ++i) o += bev(i);
    return o;
  }
  // per-cell stride (64-bit elements) of both staging areas, = 8 (mod 16) so
  // that the 16-byte accesses of the eight row groups of a fragment hit
  // disjoint banks
  static constexpr int XS = (boff(8) + 15) / 16 * 16 + 8;
  // B-fragment layout: [b][ks][nt][l][lane] of uint2
  __host__ __device__ static constexpr int frag_off(int b) {
    int o = 0;
    for (int i = 0; i < b; ++i) o += ksteps(i) * ntiles(i) * kDigits * 32;
    return o;
  }
  static constexpr int kFrag = frag_off(8);
  static constexpr int kItems = ntiles(0) + ntiles(1) + ntiles(2) + ntiles(3) + ntiles(4) + ntiles(5) + ntiles(6) +
                                ntiles(7);
  static constexpr int kPlanK = bsize(0) < kKChunk ? bsize(0) : kKChunk;  // block 0 (all even) is the largest
};

// Accumulator plan: the digit pairs of each weight s grouped greedily (k
// ascending) so that the worst-case sum over kmax contraction indices stays
// below kAccLimit for every input.
struct Plan {
  int nacc;
  int acc[kDigits][kDigits];       // accumulator of digit pair (k, l); -1: dropped
  int s[kDigits * kDigits];        // weight exponent of accumulator a
};

__host__ __device__ constexpr int data_digit_max(int k) { return k < kDigits - 1 ? 128 : 17; }     // |X| <= 2^60
__host__ __device__ constexpr int matrix_digit_max(int l) { return l < kDigits - 1 ? 128 : 65; }   // |B| < 2^62

__host__ __device__ constexpr Plan make_plan(int kmax) {
  Plan pl{};
  pl.nacc = 0;
  for (int k = 0; k < kDigits; ++k)
    for (int l = 0; l < kDigits; ++l) pl.acc[k][l] = -1;
  for (int s = kSmin; s <= 2 * kDigits - 2; ++s) {
    long long bound = 0;
    int cur = -1;
    for (int k = 0; k < kDigits; ++k) {
      const int l = s - k;
      if (l < 0 || l >= kDigits) continue;
      const long long b = (long long)kmax * data_digit_max(k) * matrix_digit_max(l);
      if (cur >= 0 && bound + b >= kAccLimit) cur = -1;
      if (cur < 0) {
        cur = pl.nacc++;
        pl.s[cur] = s;
        bound = 0;
      }
      pl.acc[k][l] = cur;
      bound += b;
    }
  }
  return pl;
}

// Work item `it` of one 16-cell row tile: a (block, n-tile) pair, items with
// more k steps first (dealt round-robin to the warps).  Evaluated with
// compile-time loop bounds, so a run-time `it` needs no table in local memory.
template <int P>
__host__ __device__ __forceinline__ void item_of(int it, int& b, int& nt) {
  using S = Shape<P>;
  int n = 0;
  b = 0;
  nt = 0;
#pragma unroll
  for (int k = 8; k >= 1; --k) {
#pragma unroll
    for (int bb = 0; bb < 8; ++bb) {
      if (S::ksteps(bb) == k) {
        if (it >= n && it < n + S::ntiles(bb)) {
          b = bb;
          nt = it - n;
        }
        n += S::ntiles(bb);
      }
    }
  }
}

// ------------------------------------------------------------------------------------
// integer helpers
// ------------------------------------------------------------------------------------
// biased exponent field of a double (2047: not finite)
__device__ __forceinline__ int exp_field(double u) {
  return (int)((unsigned long long)__double_as_longlong(u) >> 52) & 0x7FF;
}

// round(u 2^(kXBits - E)) (half away from zero) for |u| < 2^E, exact integer arithmetic
__device__ __forceinline__ long long to_fixed(double u, int E) {
  const unsigned long long bits = (unsigned long long)__double_as_longlong(u);
  const int be = (int)(bits >> 52) & 0x7FF;
  if (be == 0) return 0;  // zero (subnormals are far below any tile's range)
  const long long m = (long long)((bits & 0xFFFFFFFFFFFFFull) | 0x10000000000000ull);
  // u = m 2^(be - 1075), X = m 2^(be - 1075 + kXBits - E); be - 1022 <= E
  const int sh = be - 1075 + kXBits - E;
  long long x;
  if (sh >= 0)
    x = m << sh;
  else if (sh > -63)
    x = (m + (1ll << (-sh - 1))) >> (-sh);
  else
    x = 0;
  return (bits >> 63) ? -x : x;
}

// V 2^e2 rounded to the nearest double (ties to even), integer arithmetic only
__device__ __forceinline__ double fixed_to_double(long long V, int e2) {
  if (V == 0) return 0.0;
  const unsigned long long sgn = V < 0 ? 0x8000000000000000ull : 0ull;
  unsigned long long a = V < 0 ? (unsigned long long)(-V) : (unsigned long long)V;
  const int nb = 64 - __clzll((long long)a);
  int ex = e2 + nb - 1;  // exponent of the leading bit
  if (nb > 53) {
    const int sh = nb - 53;
    const unsigned long long rem = a & ((1ull << sh) - 1), half = 1ull << (sh - 1);
    a >>= sh;
    if (rem > half || (rem == half && (a & 1))) {
      ++a;
      if (a >> 53) {
        a >>= 1;
        ++ex;
      }
    }
  } else {
    a <<= (53 - nb);
  }
  if (ex < -1022 || ex > 1023) return (double)(V < 0 ? -1.0 : 1.0) * ldexp((double)(a), ex - 52);
  return __longlong_as_double((long long)(sgn | ((unsigned long long)(ex + 1023) << 52) | (a & 0xFFFFFFFFFFFFFull)));
}

// FP16 pair of digit K of two biased values (X + 0x8080...80): w0, w1 are the
// 32-bit words that hold byte K of each (the low words for K < 4); the byte
// goes into the mantissa of 1024 and 1024 + 128 is subtracted in FP16: exact
template <int K>
__device__ __forceinline__ uint32_t digit_pair(uint32_t w0, uint32_t w1) {
  constexpr uint32_t sel = (uint32_t)(K & 3) | ((uint32_t)(4 + (K & 3)) << 8);
  uint32_t r = (__byte_perm(w0, w1, sel) & 0x00FF00FFu) | 0x64006400u;
  const __half2 bias = __halves2half2(__ushort_as_half((unsigned short)0x6480), __ushort_as_half((unsigned short)0x6480));
  __half2 h = __hsub2(*reinterpret_cast<__half2*>(&r), bias);
  return *reinterpret_cast<uint32_t*>(&h);
}

// D += A B (m16n8k16, FP16 inputs, FP32 accumulation)
__device__ __forceinline__ void mma16816(float (&d)[4], const uint32_t (&a)[4], uint32_t b0, uint32_t b1) {
  asm("mma.sync.aligned.m16n8k16.row.col.f32.f16.f16.f32 {%0,%1,%2,%3}, {%4,%5,%6,%7}, {%8,%9}, "
      "{%0,%1,%2,%3};"
      : "+f"(d[0]), "+f"(d[1]), "+f"(d[2]), "+f"(d[3])
      : "r"(a[0]), "r"(a[1]), "r"(a[2]), "r"(a[3]), "r"(b0), "r"(b1));
}

// exact integer of an accumulator holding an integer below 2^22 in magnitude
__device__ __forceinline__ int acc_to_int(float f) { return __float_as_int(__fadd_rn(f, 12582912.0f)) - 0x4B400000; }

// ------------------------------------------------------------------------------------
// the operator on a brick
// ------------------------------------------------------------------------------------
// The cells are processed in row tiles of up to 4 x 4 x 1 cells (cell (cxl,
// cyl) of the row tile is MMA row cxl + 4 cyl).  The even-odd transforms run
// as three line passes over the row tile's slab of nodes -- along x on the
// brick, along y, along z -- each thread taking one cell segment of one line:
// contiguous loads, exact integer additions, and on the way back the nodes
// two segments share are summed in registers, so every brick node is written
// by one thread (no atomics).
//
// Shared memory (64-bit elements) beyond the two bricks: Xs [16][XS] the
// transformed inputs, region A [max(16 XS, T1)] holding the block outputs Ys
// and the x-pass lines T1, region B [T2] the y-pass lines.
template <int P>
__host__ __device__ constexpr int t1_elems(int mx, int my) {
  return (P + 1) * (P * my + 1) * (mx * (P + 1));
}
template <int P>
__host__ __device__ constexpr int t2_elems(int mx, int my) {
  return (P + 1) * (my * (P + 1)) * (mx * (P + 1));
}
// mx, my: largest row-tile extents (min(4, tile cells) along x and y)
template <int P>
__host__ __device__ constexpr int staging_elems(int mx, int my) {
  const int ys = kMCells * Shape<P>::XS;
  const int t1 = t1_elems<P>(mx, my);
  return kMCells * Shape<P>::XS + (ys > t1 ? ys : t1) + (t2_elems<P>(mx, my) + 1) / 2 * 2;
}

// even-odd outputs of a pencil (out < NE: e_out, else o_(out - NE)) and back
template <int P>
__device__ __forceinline__ void eo_forward(const long long (&u)[P + 1], long long (&o)[P + 1]) {
  constexpr int N1 = P + 1, NO = N1 / 2, NE = N1 - NO;
#pragma unroll
  for (int i = 0; i < NO; ++i) {
    o[i] = u[i] + u[N1 - 1 - i];
    o[NE + i] = u[i] - u[N1 - 1 - i];
  }
  if constexpr (NE > NO) o[NO] = u[NO];
}
template <int P>
__device__ __forceinline__ void eo_backward(const long long (&o)[P + 1], long long (&u)[P + 1]) {
  constexpr int N1 = P + 1, NO = N1 / 2, NE = N1 - NO;
#pragma unroll
  for (int i = 0; i < NO; ++i) {
    u[i] = o[i] + o[NE + i];
    u[N1 - 1 - i] = o[i] - o[NE + i];
  }
  if constexpr (NE > NO) u[NO] = o[NO];
}

// Forward transform of one row tile of mx x my cells (CMX, CMY: the same as
// compile-time constants, 0 = run time): x pass on the brick (origin u0) into
// T1[z][y][cxl N1 + out], y pass into T2[z][cyl N1 + out][xt], z pass into the
// Xs rows (cxl + 4 cyl) at the block positions; rows of absent cells zero.
template <int P, int CMX, int CMY>
__device__ __forceinline__ void forward_passes(const long long* __restrict__ u0, int bx, int by, int mx_rt, int my_rt,
                                               long long* __restrict__ T1, long long* __restrict__ T2,
                                               long long* __restrict__ Xs) {
  using S = Shape<P>;
  constexpr int N1 = S::N1, NE = S::NE, XS = S::XS;
  const int mx = CMX ? CMX : mx_rt, my = CMY ? CMY : my_rt;
  const int ny1 = P * my + 1, xw = mx * N1, yw = my * N1;
  for (int task = threadIdx.x; task < N1 * ny1 * mx; task += kThreads) {
    const int cxl = task % mx, rest = task / mx, y = rest % ny1, z = rest / ny1;
    const long long* src = u0 + P * cxl + bx * (y + by * z);
    long long u[N1], o[N1];
#pragma unroll
    for (int a = 0; a < N1; ++a) u[a] = src[a];
    eo_forward<P>(u, o);
    long long* dst = T1 + (z * ny1 + y) * xw + cxl * N1;
#pragma unroll
    for (int a = 0; a < N1; ++a) dst[a] = o[a];
  }
  __syncthreads();
  for (int task = threadIdx.x; task < N1 * my * xw; task += kThreads) {
    const int xt = task % xw, rest = task / xw, cyl = rest % my, z = rest / my;
    const long long* src = T1 + (z * ny1 + P * cyl) * xw + xt;
    long long u[N1], o[N1];
#pragma unroll
    for (int b = 0; b < N1; ++b) u[b] = src[b * xw];
    eo_forward<P>(u, o);
    long long* dst = T2 + (z * yw + cyl * N1) * xw + xt;
#pragma unroll
    for (int b = 0; b < N1; ++b) dst[b * xw] = o[b];
  }
  __syncthreads();
  for (int task = threadIdx.x; task < 16 * N1 * N1; task += kThreads) {
    const int xt = task % (4 * N1), yt = task / (4 * N1);
    const int cxl = xt / N1, cyl = yt / N1, ox = xt - cxl * N1, oy = yt - cyl * N1;
    const int sx = ox >= NE, sy = oy >= NE;
    const int i = ox - sx * NE, j = oy - sy * NE;
    const bool exist = cxl < mx && cyl < my;
    long long u[N1], o[N1];
#pragma unroll
    for (int c = 0; c < N1; ++c) u[c] = exist ? T2[(c * yw + yt) * xw + xt] : 0;
    eo_forward<P>(u, o);
    long long* row = Xs + (cxl + 4 * cyl) * XS;
    const int ex = S::ext(sx), ey = S::ext(sy);
    const int b0 = sx + 2 * sy;
#pragma unroll
    for (int c = 0; c < N1; ++c) {
      const int sz = c >= NE, k = c - sz * NE;
      row[S::boff(b0 + 4 * sz) + i + ex * (j + ey * k)] = o[c];
    }
  }
}

// Backward transform of one row tile: Ys rows -> T2 (z back) -> T1 (y back,
// nodes shared by two cell segments summed in registers) -> added to the
// brick accumulator at origin v0 (x back, each node of the slab by one thread).
template <int P, int CMX, int CMY>
__device__ __forceinline__ void backward_passes(long long* __restrict__ v0, int bx, int by, int mx_rt, int my_rt,
                                                const long long* Ys, long long* T1, long long* __restrict__ T2) {
  using S = Shape<P>;
  constexpr int N1 = S::N1, NE = S::NE, XS = S::XS;
  const int mx = CMX ? CMX : mx_rt, my = CMY ? CMY : my_rt;
  const int ny1 = P * my + 1, xw = mx * N1, yw = my * N1;
  for (int task = threadIdx.x; task < yw * xw; task += kThreads) {
    const int xt = task % xw, yt = task / xw;
    const int cxl = xt / N1, cyl = yt / N1, ox = xt - cxl * N1, oy = yt - cyl * N1;
    const int sx = ox >= NE, sy = oy >= NE;
    const int i = ox - sx * NE, j = oy - sy * NE;
    const int ex = S::ext(sx), ey = S::ext(sy);
    const int b0 = sx + 2 * sy;
    const long long* row = Ys + (cxl + 4 * cyl) * XS;
    long long o[N1], u[N1];
#pragma unroll
    for (int c = 0; c < N1; ++c) {
      const int sz = c >= NE, k = c - sz * NE;
      o[c] = row[S::boff(b0 + 4 * sz) + i + ex * (j + ey * k)];
    }
    eo_backward<P>(o, u);
#pragma unroll
    for (int c = 0; c < N1; ++c) T2[(c * yw + yt) * xw + xt] = u[c];
  }
  __syncthreads();
  for (int task = threadIdx.x; task < N1 * xw; task += kThreads) {
    const int xt = task % xw, z = task / xw;
    long long carry = 0;
    for (int cyl = 0; cyl < my; ++cyl) {
      const long long* src = T2 + (z * yw + cyl * N1) * xw + xt;
      long long o[N1], u[N1];
#pragma unroll
      for (int b = 0; b < N1; ++b) o[b] = src[b * xw];
      eo_backward<P>(o, u);
      long long* dst = T1 + (z * ny1 + P * cyl) * xw + xt;
      dst[0] = u[0] + carry;
#pragma unroll
      for (int b = 1; b < P; ++b) dst[b * xw] = u[b];
      carry = u[P];
    }
    T1[(z * ny1 + P * my) * xw + xt] = carry;
  }
  __syncthreads();
  for (int task = threadIdx.x; task < N1 * ny1; task += kThreads) {
    const int y = task % ny1, z = task / ny1;
    const long long* src = T1 + (z * ny1 + y) * xw;
    long long* dst = v0 + bx * (y + by * z);
    long long carry = 0;
    for (int cxl = 0; cxl < mx; ++cxl) {
      long long o[N1], u[N1];
#pragma unroll
      for (int a = 0; a < N1; ++a) o[a] = src[cxl * N1 + a];
      eo_backward<P>(o, u);
      dst[P * cxl] += u[0] + carry;
#pragma unroll
      for (int a = 1; a < P; ++a) dst[P * cxl + a] += u[a];
      carry = u[P];
    }
    dst[P * mx] += carry;
  }
}

// U: p on the brick (bx x by x bz nodes, Dirichlet nodes zero), FP64 in; on
// return V holds the operator result on the brick in FP64 (U is overwritten).
//   stage: the staging area (staging_elems<P>(mxm, mym) elements), sized for
//   row tiles of up to mxm x mym cells,
//   frag: B-fragment table of the problem, g2: exponent of its fixed point
//   (B = Bint 2^-g2), R: the result shift (56..72), s_misc: one int of shared
//   scratch.
template <int P>
__device__ void brick_op_affine_tc(double* U, double* V, long long* stage, int bx, int by, int bz, int ncx, int ncy,
                                   int ncz, int mxm, int mym, const uint2* __restrict__ frag, int g2, int R,
                                   int* s_misc) {
  using S = Shape<P>;
  constexpr int XS = S::XS;
  constexpr Plan pl = make_plan(S::kPlanK);
  constexpr int NACC = pl.nacc;
  const int nbrick = bx * by * bz;
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  long long* UX = reinterpret_cast<long long*>(U);
  long long* VX = reinterpret_cast<long long*>(V);
  long long* Xs = stage;
  long long* Ys = stage + kMCells * XS;  // region A
  long long* T1 = Ys;                    // region A
  const int ys_elems = kMCells * XS, t1e = t1_elems<P>(mxm, mym);
  long long* T2 = Ys + (ys_elems > t1e ? ys_elems : t1e);  // region B

  // tile exponent E (max |u| < 2^E) and a non-finite flag
  if (threadIdx.x == 0) s_misc[0] = 0;
  for (int i = threadIdx.x; i < kMCells * XS; i += kThreads) Xs[i] = 0;  // rounding slots stay zero
  __syncthreads();
  {
    int emax = 0;
    for (int i = threadIdx.x; i < nbrick; i += kThreads) emax = max(emax, exp_field(U[i]));
    emax = __reduce_max_sync(0xffffffffu, emax);
    if (lane == 0) atomicMax(&s_misc[0], emax);
  }
  __syncthreads();
  const int be_max = s_misc[0];
  const bool finite = be_max < 0x7FF;
  const int E = be_max - 1022;  // |u| < 2^E
  for (int i = threadIdx.x; i < nbrick; i += kThreads) {
    UX[i] = finite ? to_fixed(U[i], E) : 0;
    VX[i] = 0;
  }

  const int g = lane >> 2, t = lane & 3;
  constexpr unsigned long long kBias = 0x8080808080808080ull;

  // row tiles: boxes of up to 4 x 4 cells in one cell layer
  const int nrx = (ncx + 3) / 4, nry = (ncy + 3) / 4;
  const int nrt = nrx * nry * ncz;
  for (int rt = 0; rt < nrt; ++rt) {
    const int rtx = rt % nrx, rty = (rt / nrx) % nry, cz = rt / (nrx * nry);
    const int cx0 = 4 * rtx, cy0 = 4 * rty;
    const int mx = min(4, ncx - cx0), my = min(4, ncy - cy0);
    const int base = P * cx0 + bx * (P * cy0 + by * P * cz);
    __syncthreads();  // U converted (first) / previous row tile finished with T1, T2 (x back read T1)
    if (mx == 4 && my == 4)
      forward_passes<P, 4, 4>(UX + base, bx, by, 4, 4, T1, T2, Xs);
    else
      forward_passes<P, 0, 0>(UX + base, bx, by, mx, my, T1, T2, Xs);
    __syncthreads();
    // products: items (block, n-tile) dealt round-robin to the warps
    for (int it = warp; it < S::kItems; it += kThreads / 32) {
      int b, nt;
      item_of<P>(it, b, nt);
      const int ksb = S::ksteps(b), bev = S::bev(b), bo = S::boff(b);
      long long out[4] = {0, 0, 0, 0};
      for (int kc = 0; kc < ksb; kc += 2) {
        float acc[NACC][4];
#pragma unroll
        for (int a = 0; a < NACC; ++a) acc[a][0] = acc[a][1] = acc[a][2] = acc[a][3] = 0.f;
        const int kend = min(kc + 2, ksb);
        // matrix digits of the first k step; each step loads the next one's
        // before its products, so the L2 latency overlaps the digit work
        const uint2* fbase = frag + S::frag_off(b) + nt * kDigits * 32 + lane;
        const int fstep = S::ntiles(b) * kDigits * 32;
        uint2 Bn[kDigits];
#pragma unroll
        for (int l = 0; l < kDigits; ++l) Bn[l] = __ldg(fbase + kc * fstep + l * 32);
        for (int ks = kc; ks < kend; ++ks) {
          uint2 B[kDigits];
#pragma unroll
          for (int l = 0; l < kDigits; ++l) B[l] = Bn[l];
          if (ks + 1 < kend) {
#pragma unroll
            for (int l = 0; l < kDigits; ++l) Bn[l] = __ldg(fbase + (ks + 1) * fstep + l * 32);
          }
          // data of this lane's fragment: rows g, g + 8; columns c0, c0+1 and c0+8, c0+9
          const int c0 = 16 * ks + 2 * t;
          const long long* x0 = Xs + g * XS + bo + c0;
          const long long* x1 = x0 + 8 * XS;
          const longlong2 z2 = make_longlong2(0, 0);
          const longlong2 v00 = c0 < bev ? *reinterpret_cast<const longlong2*>(x0) : z2;
          const longlong2 v01 = c0 + 8 < bev ? *reinterpret_cast<const longlong2*>(x0 + 8) : z2;
          const longlong2 v10 = c0 < bev ? *reinterpret_cast<const longlong2*>(x1) : z2;
          const longlong2 v11 = c0 + 8 < bev ? *reinterpret_cast<const longlong2*>(x1 + 8) : z2;
          // balanced digits: bytes of X + 0x8080...80
          auto biased = [](long long x) { return (unsigned long long)x + kBias; };
          const unsigned long long u00a = biased(v00.x), u00b = biased(v00.y), u01a = biased(v01.x),
                                   u01b = biased(v01.y), u10a = biased(v10.x), u10b = biased(v10.y),
                                   u11a = biased(v11.x), u11b = biased(v11.y);
          uint32_t A[kDigits][4];
#pragma unroll
          for (int k = 0; k < kDigits; ++k) {
            const int sh = k < 4 ? 0 : 32;
            auto w = [&](unsigned long long u) { return (uint32_t)(u >> sh); };
            switch (k) {
#define MFCG_TC_DIGIT(K)                       \
  case K:                                      \
    A[K][0] = digit_pair<K>(w(u00a), w(u00b)); \
    A[K][1] = digit_pair<K>(w(u10a), w(u10b)); \
    A[K][2] = digit_pair<K>(w(u01a), w(u01b)); \
    A[K][3] = digit_pair<K>(w(u11a), w(u11b)); \
    break;
              MFCG_TC_DIGIT(0)
              MFCG_TC_DIGIT(1)
              MFCG_TC_DIGIT(2)
              MFCG_TC_DIGIT(3)
              MFCG_TC_DIGIT(4)
              MFCG_TC_DIGIT(5)
              MFCG_TC_DIGIT(6)
              MFCG_TC_DIGIT(7)
#undef MFCG_TC_DIGIT
            }
          }
          // digit pairs round-robin over the accumulators: consecutive products
          // go to different accumulators
#pragma unroll
          for (int rnd = 0; rnd < kDigits; ++rnd) {
#pragma unroll
            for (int a = 0; a < NACC; ++a) {
              // the rnd-th pair of accumulator a (pairs ordered by k)
              int cnt = 0, kk = -1;
#pragma unroll
              for (int k = 0; k < kDigits; ++k)
#pragma unroll
                for (int l = 0; l < kDigits; ++l)
                  if (pl.acc[k][l] == a) {
                    if (cnt == rnd) kk = k * kDigits + l;
                    ++cnt;
                  }
              if (kk >= 0) mma16816(acc[a], A[kk / kDigits], B[kk % kDigits].x, B[kk % kDigits].y);
            }
          }
        }
        // recombination: out += sum_a 2^(8 s_a - R) D_a; with 56 <= R <= 72
        // weights s >= 9 shift left and s <= 7 right.  With one accumulator
        // per weight (the plan for balanced digits), two adjacent weights are
        // first combined in 32 bits, D_s + 2^8 D_(s+1) (|D| < 2^22).
        auto add_shifted = [&](long long& o, long long v, int s) {
          const int sh = 8 * s - R;
          if (s >= 9)
            o += v << sh;
          else if (s <= 7)
            o += v >> -sh;
          else
            o += sh >= 0 ? (v << sh) : (v >> -sh);
        };
        constexpr bool kOnePerWeight = NACC == 2 * kDigits - 1 - kSmin;
        if constexpr (kOnePerWeight) {
#pragma unroll
          for (int i = 0; i < 4; ++i) {
#pragma unroll
            for (int a = 0; a < NACC; a += 2) {
              int v = acc_to_int(acc[a][i]);
              if (a + 1 < NACC) v += acc_to_int(acc[a + 1][i]) << 8;
              add_shifted(out[i], (long long)v, pl.s[a]);
            }
          }
        } else {
#pragma unroll
          for (int a = 0; a < NACC; ++a)
#pragma unroll
            for (int i = 0; i < 4; ++i) add_shifted(out[i], (long long)acc_to_int(acc[a][i]), pl.s[a]);
        }
      }
      // C fragment: (row g, cols n0, n0+1) and (row g + 8, same columns)
      const int n0 = 8 * nt + 2 * t;
      if (n0 < bev) {
        long long* y0 = Ys + g * XS + bo + n0;
        *reinterpret_cast<longlong2*>(y0) = make_longlong2(out[0], out[1]);
        *reinterpret_cast<longlong2*>(y0 + 8 * XS) = make_longlong2(out[2], out[3]);
      }
    }
    __syncthreads();
    if (mx == 4 && my == 4)
      backward_passes<P, 4, 4>(VX + base, bx, by, 4, 4, Ys, T1, T2);
    else
      backward_passes<P, 0, 0>(VX + base, bx, by, mx, my, Ys, T1, T2);
  }
  __syncthreads();
  // back to FP64: v = V 2^(E + R - kXBits - g2)
  const int e2 = E + R - kXBits - g2;
  const double qnan = __longlong_as_double(0x7FF8000000000000ll);
  for (int i = threadIdx.x; i < nbrick; i += kThreads) V[i] = finite ? fixed_to_double(VX[i], e2) : qnan;
  __syncthreads();
}

}  // namespace tc
}  // namespace mfcg
