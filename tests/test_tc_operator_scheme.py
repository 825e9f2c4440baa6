"""CPU emulation of the tensor-core form of the Cartesian cell operator.

The FP64 operator of Cartesian tiles runs its contractions on the FP16 tensor
cores by an exact split into 8-bit digits (an Ozaki-type error-free
splitting): the p_k values of a tile become 64-bit fixed-point integers with
one exponent per tile, each cell's values pass an even-odd transform along
x, y and z (exact integer additions), which makes the cell matrix of Eq. 5
block diagonal with eight blocks, and every block product Y = B X is the sum
over digit pairs (k, l) of 2^(8(k+l)) B_l X_k with balanced 8-bit digits X_k
of the data and B_l of the block matrix.  Each digit product is an exact
FP16 x FP16 product and the FP32 accumulator of the tensor core sums them
exactly as long as every partial sum stays below 2^22 (then it is an integer
of at most 22 bits); digit pairs of equal weight share an accumulator within
that bound.  The accumulators are recombined into 64-bit integers, transformed
back, summed over the cells of each node and converted to FP64.

This file restates that scheme in exact integer arithmetic (numpy int64 with
wrap-around and Python integers) and checks it against the oracle's operator,
and checks the bounds that make every step exact: the planned accumulator
groups stay below 2^22 for ANY input, and the final 64-bit values cannot
overflow.  The constants and conventions are the kernel's (tc_operator.cuh,
tc_tables.cu).
"""
from fractions import Fraction

import numpy as np
import pytest

from oracle import fem

DIGITS = 8        # digits per operand (64 bits)
S_MIN = 6         # digit pairs (k, l), LSB-first, with k + l >= S_MIN are kept
R_BASE = 64       # result = (sum over the digit pairs) / 2^R, R = R_BASE + delta, delta in [-8, 8]
X_BITS = 57       # cell inputs: |X| <= 2^57 in the tile's fixed point
T_BITS = 60       # after the three butterfly levels |T| <= 2^60
B_BITS = 62       # block matrix entries: |B| < 2^62 in the matrix fixed point
ACC_LIMIT = 1 << 22  # FP32 accumulators hold exact integers below 2^22 (float -> int by 1.5 * 2^23)
K_CHUNK = 32      # at most this many contraction indices per accumulator pass


# ----------------------------------------------------------------- even-odd blocks

def reduced_1d(A):
    """Even and odd blocks of a centrosymmetric matrix (A[n-1-i][n-1-j] = A[i][j]):
    with e_j = x_j + x_{n-1-j} (j < h), e_h = x_h (odd n) and
    o_j = x_j - x_{n-1-j}, y = A x is y_i = (E e)_i + (O o)_i and
    y_{n-1-i} = (E e)_i - (O o)_i, y_h = (E e)_h."""
    n = A.shape[0]
    h = n // 2
    ne = n - h
    E = np.zeros((ne, ne), dtype=A.dtype)
    O = np.zeros((h, h), dtype=A.dtype)
    for i in range(ne):
        for j in range(h):
            E[i, j] = (A[i, j] + A[i, n - 1 - j]) / 2
        if ne > h:
            E[i, h] = A[i, h]
    for i in range(h):
        for j in range(h):
            O[i, j] = (A[i, j] - A[i, n - 1 - j]) / 2
    return E, O


def block_matrices(p, h, dtype=np.float64):
    """The eight blocks (sx, sy, sz) of the Cartesian Laplace cell matrix
    (hy hz / hx) K (x) M (x) M + ... in the even-odd basis, x fastest, formed in
    `dtype` from the FP64 1D matrices (the library forms them in long double:
    at high degree the FP64 Kronecker sums lose up to ten units of 2^-53)."""
    K, M = (x.astype(dtype) for x in fem.element_matrices_1d(p))
    h = [dtype(v) for v in h]
    sc = (h[1] * h[2] / h[0], h[0] * h[2] / h[1], h[0] * h[1] / h[2])
    red_m = reduced_1d(M)
    red_k = [reduced_1d(s * K) for s in sc]
    blocks = {}
    for sz in range(2):
        for sy in range(2):
            for sx in range(2):
                kx, ky, kz = red_k[0][sx], red_k[1][sy], red_k[2][sz]
                mx, my, mz = red_m[sx], red_m[sy], red_m[sz]
                B = np.kron(mz, np.kron(my, kx)) + np.kron(mz, np.kron(ky, mx)) + np.kron(kz, np.kron(my, mx))
                blocks[(sx, sy, sz)] = B
    return blocks


def forward_butterfly(u, n):
    """Even-odd transform of one cell's n^3 values (x fastest) along x, y, z;
    returns {(sx, sy, sz): flattened block values} (exact for integers)."""
    h = n // 2
    ne = n - h
    cube = np.asarray(u).reshape(n, n, n)  # [z][y][x]

    def split(a, axis):
        a = np.moveaxis(a, axis, 0)
        lo, hi = a[:h], a[n - h:][::-1]
        e = lo + hi
        if ne > h:
            e = np.concatenate([e, a[h:h + 1]], axis=0)
        o = lo - hi
        return np.moveaxis(e, 0, axis), np.moveaxis(o, 0, axis)

    out = {}
    ex, ox = split(cube, 2)
    for sx, ax in enumerate((ex, ox)):
        ey, oy = split(ax, 1)
        for sy, ay in enumerate((ey, oy)):
            ez, oz = split(ay, 0)
            for sz, az in enumerate((ez, oz)):
                out[(sx, sy, sz)] = az.reshape(-1)
    return out


def backward_butterfly(blocks, n):
    """Inverse of the output side: y_i = ye_i + yo_i, y_{n-1-i} = ye_i - yo_i,
    y_h = ye_h, along z, y, x; returns the n^3 values (x fastest)."""
    h = n // 2
    ne = n - h
    sizes = (ne, h)

    def join(e, o, axis):
        e = np.moveaxis(e, axis, 0)
        o = np.moveaxis(o, axis, 0)
        out = np.empty((n,) + e.shape[1:], dtype=e.dtype)
        out[:h] = e[:h] + o
        out[n - h:] = (e[:h] - o)[::-1]
        if ne > h:
            out[h] = e[h]
        return np.moveaxis(out, 0, axis)

    def blk(sx, sy, sz):
        return blocks[(sx, sy, sz)].reshape(sizes[sz], sizes[sy], sizes[sx])

    xs = []
    for sx in range(2):
        ys = []
        for sy in range(2):
            ys.append(join(blk(sx, sy, 0), blk(sx, sy, 1), 0))
        xs.append(join(ys[0], ys[1], 1))
    return join(xs[0], xs[1], 2).reshape(-1)


# ----------------------------------------------------------------- digits and plan

BIAS = 0x8080808080808080  # 128 in every byte


def data_digits(T):
    """Balanced digits d_k in [-128, 127], LSB first, of int64 values |T| <= 2^60:
    the bytes of T + 0x8080...80 (mod 2^64), each minus 128."""
    T = np.asarray(T, dtype=np.int64)
    U = T.astype(np.uint64) + np.uint64(BIAS)
    return [((U >> np.uint64(8 * k)) & np.uint64(0xFF)).astype(np.int64) - 128 for k in range(DIGITS)]


def balanced_digits(v: int):
    """Digits c_l in [-128, 127] with v = sum c_l 256^l (LSB first)."""
    out = []
    for _ in range(DIGITS):
        c = ((v + 128) % 256) - 128
        out.append(c)
        v = (v - c) // 256
    assert v == 0
    return out


def digit_bounds():
    """Largest magnitude of data digit k and matrix digit l (both balanced)."""
    dmax = [128] * (DIGITS - 1) + [(1 << (T_BITS - 56)) + 1]
    cmax = [128] * (DIGITS - 1) + [(1 << (B_BITS - 56)) + 1]
    return dmax, cmax


def accumulator_plan(kmax: int):
    """Digit pairs of each weight s = k + l >= S_MIN grouped greedily (k
    ascending) into accumulators whose worst-case sum over kmax contraction
    indices stays below ACC_LIMIT.  Returns [(s, [(k, l), ...]), ...]."""
    dmax, cmax = digit_bounds()
    plan = []
    for s in range(S_MIN, 2 * DIGITS - 1):
        group, bound = [], 0
        for k in range(DIGITS):
            l = s - k
            if not 0 <= l < DIGITS:
                continue
            b = kmax * dmax[k] * cmax[l]
            if group and bound + b >= ACC_LIMIT:
                plan.append((s, group))
                group, bound = [], 0
            group.append((k, l))
            bound += b
        if group:
            plan.append((s, group))
    return plan


def matrix_exponent(p, h):
    """Exponent g2 of the matrix fixed point B = Bint 2^-g2 and the shift R of
    the result: |Bint| < 2^62 and every final node value
    |V| <= row 2^(X_BITS + g2 - R) < 2^62 (row: the largest absolute row sum of
    the cell matrix times 8 cells per node); R = 64 + delta with delta in
    [-8, 8] chosen so that the matrix keeps all 62 bits and the result uses
    the whole 62-bit range where possible."""
    K, M = fem.element_matrices_1d(p)
    sc = (h[1] * h[2] / h[0], h[0] * h[2] / h[1], h[0] * h[1] / h[2])
    Ae = sc[0] * np.kron(M, np.kron(M, K)) + sc[1] * np.kron(M, np.kron(K, M)) + sc[2] * np.kron(K, np.kron(M, M))
    row = np.abs(Ae).sum(axis=1).max() * 8
    bmax = max(np.abs(B).max() for B in block_matrices(p, h).values())
    F = int(np.frexp(bmax)[1])  # bmax < 2^F
    lr = int(np.ceil(np.log2(row)))
    delta = min(max(lr - F - 6, -8), 8)
    g2 = min(B_BITS - F, 68 + delta - lr)
    return g2, R_BASE + delta


# ----------------------------------------------------------------- the scheme

def to_fixed(u, E):
    """X = round(u 2^(X_BITS - E)) (half away from zero), exact."""
    out = np.zeros(len(u), dtype=np.int64)
    for i, v in enumerate(u):
        f = Fraction(float(v)) * Fraction(2) ** (X_BITS - E)
        a = abs(f)
        q = int(a + Fraction(1, 2))
        out[i] = q if f >= 0 else -q
    return out


def tc_brick_operator(p, cells, u_lex):
    """The kernel's arithmetic on one brick holding the whole mesh (Dirichlet
    nodes zeroed on input, as in the tile kernels): returns the FP64 result
    on every node and the largest accumulator partial-sum bound seen."""
    n = p + 1
    nn = [p * c + 1 for c in cells]
    h = [1.0 / c for c in cells]
    u = np.array(u_lex, dtype=float).reshape(nn[2], nn[1], nn[0])
    u[0], u[-1], u[:, 0], u[:, -1], u[:, :, 0], u[:, :, -1] = 0, 0, 0, 0, 0, 0
    umax = np.abs(u).max()
    E = int(np.frexp(umax)[1]) if umax > 0 else 0
    X = to_fixed(u.reshape(-1), E).reshape(u.shape)
    g2, R = matrix_exponent(p, h)
    blocks = block_matrices(p, h, np.longdouble)
    bdig = {}
    for key, B in blocks.items():
        dig = [np.zeros(B.shape, dtype=np.int64) for _ in range(DIGITS)]
        for i, row in enumerate(B):
            for j, b in enumerate(row):
                f = Fraction(*np.longdouble(b).as_integer_ratio()) * Fraction(2) ** g2
                v = int(abs(f) + Fraction(1, 2)) * (1 if f >= 0 else -1)
                assert abs(v) < 2 ** B_BITS
                for l, c in enumerate(balanced_digits(v)):
                    dig[l][i, j] = c
        bdig[key] = dig
    V = np.zeros(u.shape, dtype=np.int64)
    worst = 0
    for cz in range(cells[2]):
        for cy in range(cells[1]):
            for cx in range(cells[0]):
                sl = np.s_[p * cz:p * cz + n, p * cy:p * cy + n, p * cx:p * cx + n]
                T = forward_butterfly(X[sl].reshape(-1), n)
                Y = {}
                for key, tb in T.items():
                    kb = len(tb)
                    dd = data_digits(tb)
                    acc_out = np.zeros(blocks[key].shape[0], dtype=np.int64)
                    for k0 in range(0, kb, K_CHUNK):
                        ks = slice(k0, min(kb, k0 + K_CHUNK))
                        plan = accumulator_plan(min(kb, K_CHUNK))
                        accs = []
                        for s, group in plan:
                            D = np.zeros(blocks[key].shape[0], dtype=np.int64)
                            bound = np.zeros(blocks[key].shape[0], dtype=np.int64)
                            for (k, l) in group:
                                D += bdig[key][l][:, ks] @ dd[k][ks]
                                bound += np.abs(bdig[key][l][:, ks]) @ np.abs(dd[k][ks])
                            worst = max(worst, int(bound.max()))
                            accs.append((s, D))
                        # one accumulator per weight: adjacent weights combine in
                        # 32 bits first, D_s + 2^8 D_(s+1); weights s >= 9 shift
                        # left, s <= 7 right (|delta| <= 8)
                        assert [a[0] for a in accs] == list(range(S_MIN, 2 * DIGITS - 1))
                        for i in range(0, len(accs), 2):
                            s, D = accs[i]
                            if i + 1 < len(accs):
                                D = D + (accs[i + 1][1] << 8)
                            assert np.abs(D).max() < 2 ** 31
                            acc_out += (D << (8 * s - R)) if 8 * s >= R else (D >> (R - 8 * s))
                    Y[key] = acc_out
                V[sl] += backward_butterfly(Y, n).reshape(n, n, n)
    assert np.abs(V).max() < 2 ** 62
    scale = 2.0 ** (E + R - X_BITS - g2)
    return V.astype(np.float64).reshape(-1) * scale, worst


# ----------------------------------------------------------------- tests


@pytest.mark.parametrize("p", range(1, 9))
def test_even_odd_blocks_reassemble_the_cell_matrix(p):
    n = p + 1
    h = (0.5, 0.25, 1.0 / 3.0)
    K, M = fem.element_matrices_1d(p)
    sc = (h[1] * h[2] / h[0], h[0] * h[2] / h[1], h[0] * h[1] / h[2])
    Ae = sc[0] * np.kron(M, np.kron(M, K)) + sc[1] * np.kron(M, np.kron(K, M)) + sc[2] * np.kron(K, np.kron(M, M))
    blocks = block_matrices(p, h)
    rng = np.random.default_rng(p)
    u = rng.standard_normal(n ** 3)
    T = forward_butterfly(u, n)
    Y = {key: blocks[key] @ T[key] for key in blocks}
    np.testing.assert_allclose(backward_butterfly(Y, n), Ae @ u, atol=1e-13 * np.abs(Ae @ u).max())


@pytest.mark.parametrize("p", range(1, 9))
def test_accumulator_groups_stay_exact_for_any_input(p):
    # worst case over all inputs: every digit at its bound, every index of the
    # largest block (n_even^3, at most K_CHUNK per pass) contributing
    ne = (p + 2) // 2
    kmax = min(ne ** 3, K_CHUNK)
    dmax, cmax = digit_bounds()
    plan = accumulator_plan(kmax)
    pairs = [pr for _, g in plan for pr in g]
    assert sorted(pairs) == sorted((k, l) for k in range(DIGITS) for l in range(DIGITS) if k + l >= S_MIN)
    for _, group in plan:
        assert sum(kmax * dmax[k] * cmax[l] for k, l in group) < ACC_LIMIT
    # with balanced digits every weight fits one accumulator
    assert len(plan) == 2 * DIGITS - 1 - S_MIN


def _oracle_rows(p, cells, u):
    prob = fem.Problem(p, cells)
    A = fem.assemble(prob)
    interior = ~fem.boundary_mask(prob)
    return (A @ u)[interior], interior


def _extended_blocks(p, cells, u):
    """The same even-odd block operator applied in extended precision (long
    double, no digits): what the digit scheme computes up to its truncations.
    (It differs from the nodal product of the FP64 1D matrices by their
    centrosymmetry defect, up to about 1e-14 relative at degree 7 and 8, which
    the FP64 sweeps share: the even-odd form takes the lower rows of each 1D
    matrix from its upper rows.)"""
    n = p + 1
    nn = [p * c + 1 for c in cells]
    B = block_matrices(p, [1.0 / c for c in cells], np.longdouble)
    uu = np.array(u, dtype=np.longdouble).reshape(nn[2], nn[1], nn[0])
    uu[0], uu[-1], uu[:, 0], uu[:, -1], uu[:, :, 0], uu[:, :, -1] = 0, 0, 0, 0, 0, 0
    V = np.zeros(uu.shape, dtype=np.longdouble)
    for cz in range(cells[2]):
        for cy in range(cells[1]):
            for cx in range(cells[0]):
                sl = np.s_[p * cz:p * cz + n, p * cy:p * cy + n, p * cx:p * cx + n]
                T = forward_butterfly(uu[sl].reshape(-1), n)
                V[sl] += backward_butterfly({k: B[k] @ T[k] for k in B}, n).reshape(n, n, n)
    return V.reshape(-1)


@pytest.mark.parametrize("p,cells", [(1, (3, 2, 2)), (2, (2, 3, 2)), (3, (2, 2, 2)), (4, (2, 2, 3)),
                                     (5, (2, 1, 2)), (6, (1, 2, 2)), (7, (2, 1, 1)), (8, (1, 1, 2))])
def test_integer_scheme_matches_the_oracle_operator(p, cells):
    prob = fem.Problem(p, cells)
    rng = np.random.default_rng(40 + p)
    u = rng.standard_normal(prob.n_dofs) * np.exp(rng.uniform(-3, 3, prob.n_dofs))
    got, worst = tc_brick_operator(p, cells, u)
    assert worst < ACC_LIMIT
    ref, interior = _oracle_rows(p, cells, u)
    # the oracle's operator (FP64 CSR) within the operator tolerance of the GPU tests
    assert np.abs(got[interior] - ref).max() <= 1e-13 * np.abs(ref).max()
    # the digit scheme itself: a few units of 2^-53 of the largest entry up to
    # degree 4; the dropped digit pairs sum over larger contractions at higher
    # degree (up to 30 units at degree 8, where the FP64 CSR product of the
    # oracle is itself 13 units away from the extended-precision one)
    ext = _extended_blocks(p, cells, u)[interior]
    err = float(np.abs(got[interior] - ext).max() / np.abs(ext).max())
    assert err < (4 if p <= 4 else 32) * 2.0 ** -53, err


def test_final_values_fit_64_bits_for_the_worst_input():
    # the input that maximises the centre node's row of A (shared by 8 cells):
    # the signs of that row at the tile's largest magnitude
    for p in (2, 4, 6):
        cells = (2, 2, 2)
        prob = fem.Problem(p, cells)
        A = fem.assemble(prob, dirichlet=False).toarray()
        nn = prob.nodes_per_dim
        i = p + nn[0] * (p + nn[1] * p)
        u = np.sign(A[i])
        got, worst = tc_brick_operator(p, cells, u)
        g2, R = matrix_exponent(p, [1.0 / c for c in cells])
        E = 1  # max |u| = 1 < 2^1
        assert abs(got[i]) / 2.0 ** (E + R - X_BITS - g2) < 2.0 ** 62
        interior = ~fem.boundary_mask(prob)
        um = np.where(interior, u, 0.0)
        assert abs(got[i] - A[i] @ um) <= 1e-14 * abs(got[i])
