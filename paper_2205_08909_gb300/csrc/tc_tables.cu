// Host tables of the tensor-core cell operator (tc_operator.cuh): the eight
// even-odd blocks of the Cartesian cell matrix of Eq. 5 as 64-bit fixed-point
// integers, split into balanced 8-bit digits and packed in the per-lane order
// of the B operand of mma.m16n8k16 (col-major 16 x 8 FP16: lane (g, t) holds
// rows 2t, 2t+1 and 2t+8, 2t+9 of column g).
#include <cmath>
#include <cstdint>
#include <vector>

#include "tc_operator.cuh"

namespace mfcg {
namespace {

using LD = long double;

// even (ne x ne) and odd (no x no) blocks of a centrosymmetric n x n matrix:
// y_i = (E e)_i + (O o)_i, y_{n-1-i} = (E e)_i - (O o)_i, y_h = (E e)_h for
// e_j = x_j + x_{n-1-j} (j < n/2), e_h = x_h (odd n), o_j = x_j - x_{n-1-j}
void reduce_1d(int n, const double* A, std::vector<LD>& E, std::vector<LD>& O) {
  const int h = n / 2, ne = n - h;
  E.assign((size_t)ne * ne, 0.0L);
  O.assign((size_t)h * h, 0.0L);
  for (int i = 0; i < ne; ++i) {
    for (int j = 0; j < h; ++j) E[i * ne + j] = ((LD)A[i * n + j] + (LD)A[i * n + n - 1 - j]) / 2;
    if (ne > h) E[i * ne + h] = A[i * n + h];
  }
  for (int i = 0; i < h; ++i)
    for (int j = 0; j < h; ++j) O[i * h + j] = ((LD)A[i * n + j] - (LD)A[i * n + n - 1 - j]) / 2;
}

// FP16 bits of an integer |c| <= 2^11 (exact)
uint16_t half_of_int(long long c) {
  if (c == 0) return 0;
  const uint16_t sgn = c < 0 ? 0x8000 : 0;
  unsigned a = (unsigned)(c < 0 ? -c : c);
  int e = 0;
  while ((a >> (e + 1)) != 0) ++e;  // a in [2^e, 2^(e+1))
  const unsigned mant = (a << (10 - e)) & 0x3FF;
  return (uint16_t)(sgn | ((e + 15) << 10) | mant);
}

template <int P>
int build(const OperatorCoeffs& c, int op_kind, std::vector<uint2>& frag, int& g2, int& rshift) {
  using S = tc::Shape<P>;
  constexpr int n = P + 1;
  // 1D factors per direction: the cell matrix is sum_t kron(Z_t, kron(Y_t, X_t))
  // (x fastest) with Laplace terms (K0, M, M), (M, K1, M), (M, M, K2) and the
  // mass term (MV, M, M)
  const int nterm = op_kind == OP_MASS ? 1 : 3;
  int fac[3][3];  // [term][direction] -> matrix id
  if (op_kind == OP_MASS) {
    fac[0][0] = MAT_MV;
    fac[0][1] = MAT_M;
    fac[0][2] = MAT_M;
  } else {
    for (int t = 0; t < 3; ++t)
      for (int d = 0; d < 3; ++d) fac[t][d] = d == t ? MAT_K0 + d : MAT_M;
  }
  std::vector<LD> red[NMAT][2];
  for (int t = 0; t < nterm; ++t)
    for (int d = 0; d < 3; ++d) {
      const int m = fac[t][d];
      if (red[m][0].empty()) reduce_1d(n, c.mat[m], red[m][0], red[m][1]);
    }
  // block matrices B_b[(i,j,k)][(i',j',k')] (row = output, column = input),
  // formed in long double (in FP64 the Kronecker sums lose up to ten units of
  // 2^-53 at high degree)
  std::vector<LD> B[8];
  LD bmax = 0;
  for (int b = 0; b < 8; ++b) {
    const int s[3] = {b & 1, (b >> 1) & 1, b >> 2};
    const int e[3] = {S::ext(s[0]), S::ext(s[1]), S::ext(s[2])};
    const int bs = S::bsize(b);
    B[b].assign((size_t)bs * bs, 0.0L);
    for (int r = 0; r < bs; ++r) {
      const int ri[3] = {r % e[0], (r / e[0]) % e[1], r / (e[0] * e[1])};
      for (int q = 0; q < bs; ++q) {
        const int qi[3] = {q % e[0], (q / e[0]) % e[1], q / (e[0] * e[1])};
        LD v = 0;
        for (int t = 0; t < nterm; ++t) {
          LD prod = 1;
          for (int d = 0; d < 3; ++d) prod *= red[fac[t][d]][s[d]][ri[d] * e[d] + qi[d]];
          v += prod;
        }
        B[b][(size_t)r * bs + q] = v;
        if (fabsl(v) > bmax) bmax = fabsl(v);
      }
    }
  }
  // largest absolute row sum of the nodal cell matrix, times 8 cells per node
  LD row = 0;
  for (int r = 0; r < S::N3; ++r) {
    const int ri[3] = {r % n, (r / n) % n, r / (n * n)};
    LD sum = 0;
    for (int q = 0; q < S::N3; ++q) {
      const int qi[3] = {q % n, (q / n) % n, q / (n * n)};
      LD v = 0;
      for (int t = 0; t < nterm; ++t) {
        LD prod = 1;
        for (int d = 0; d < 3; ++d) prod *= (LD)c.mat[fac[t][d]][ri[d] * n + qi[d]];
        v += prod;
      }
      sum += fabsl(v);
    }
    if (sum > row) row = sum;
  }
  row *= 8;
  if (!(bmax > 0) || !(row > 0)) return -1;
  int F = 0;
  frexpl(bmax, &F);  // bmax < 2^F
  // fixed point of the matrix, B = Bint 2^-g2 with |Bint| < 2^62, and result
  // shift R: every final node value |V| = |sum Bint X| 2^-R <= row 2^(57 + g2 - R)
  // stays below 2^62 for |X| <= 2^57.  R = 64 + delta, |delta| <= 8, is chosen
  // so that the matrix keeps its 62 bits and V uses the whole range.
  const int lr = (int)ceill(log2l(row));
  int delta = lr - F - 6;
  delta = delta < -8 ? -8 : (delta > 8 ? 8 : delta);
  const int g_digits = 62 - F;
  const int g_range = 68 + delta - lr;
  g2 = g_digits < g_range ? g_digits : g_range;
  rshift = tc::kRBase + delta;
  // balanced digits of every entry, packed per fragment
  frag.assign(S::kFrag, make_uint2(0u, 0u));
  for (int b = 0; b < 8; ++b) {
    const int bs = S::bsize(b);
    std::vector<signed char> dig((size_t)bs * bs * tc::kDigits);
    for (size_t i = 0; i < (size_t)bs * bs; ++i) {
      long long v = llroundl(ldexpl(B[b][i], g2));
      for (int l = 0; l < tc::kDigits; ++l) {
        long long r = v & 255;
        if (r >= 128) r -= 256;
        dig[i * tc::kDigits + l] = (signed char)r;
        v = (v - r) >> 8;
      }
      if (v != 0) return -1;
    }
    auto digit = [&](int row_out, int col_in, int l) -> long long {
      if (row_out >= bs || col_in >= bs) return 0;
      return dig[((size_t)row_out * bs + col_in) * tc::kDigits + l];
    };
    for (int ks = 0; ks < S::ksteps(b); ++ks)
      for (int nt = 0; nt < S::ntiles(b); ++nt)
        for (int l = 0; l < tc::kDigits; ++l)
          for (int lane = 0; lane < 32; ++lane) {
            const int gq = lane >> 2, tq = lane & 3;
            const int nr = nt * 8 + gq, k0 = ks * 16 + 2 * tq;
            uint2 f;
            f.x = (uint32_t)half_of_int(digit(nr, k0, l)) | ((uint32_t)half_of_int(digit(nr, k0 + 1, l)) << 16);
            f.y = (uint32_t)half_of_int(digit(nr, k0 + 8, l)) | ((uint32_t)half_of_int(digit(nr, k0 + 9, l)) << 16);
            frag[S::frag_off(b) + ((ks * S::ntiles(b) + nt) * tc::kDigits + l) * 32 + lane] = f;
          }
  }
  return 0;
}

}  // namespace

// B-fragment table of the degree-p tensor-core operator, the exponent g2 of
// its fixed point and the result shift r; 0 on success
int build_tc_fragments(int p, const OperatorCoeffs& c, int op_kind, std::vector<uint2>& frag, int& g2, int& r) {
  switch (p) {
    case 1: return build<1>(c, op_kind, frag, g2, r);
    case 2: return build<2>(c, op_kind, frag, g2, r);
    case 3: return build<3>(c, op_kind, frag, g2, r);
    case 4: return build<4>(c, op_kind, frag, g2, r);
    case 5: return build<5>(c, op_kind, frag, g2, r);
    case 6: return build<6>(c, op_kind, frag, g2, r);
    case 7: return build<7>(c, op_kind, frag, g2, r);
    case 8: return build<8>(c, op_kind, frag, g2, r);
    default: return -1;
  }
}

// shared-memory elements (64-bit) of the staging areas of the degree-p
// operator for row tiles of up to mx x my cells
size_t tc_staging_elems(int p, int mx, int my) {
  switch (p) {
    case 1: return tc::staging_elems<1>(mx, my);
    case 2: return tc::staging_elems<2>(mx, my);
    case 3: return tc::staging_elems<3>(mx, my);
    case 4: return tc::staging_elems<4>(mx, my);
    case 5: return tc::staging_elems<5>(mx, my);
    case 6: return tc::staging_elems<6>(mx, my);
    case 7: return tc::staging_elems<7>(mx, my);
    case 8: return tc::staging_elems<8>(mx, my);
    default: return 0;
  }
}

}  // namespace mfcg
