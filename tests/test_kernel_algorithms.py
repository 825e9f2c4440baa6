"""CPU checks of the algorithmic identities the tile kernels rely on.

Each test restates a kernel's index and arithmetic scheme in numpy and checks
it against the plain definition it replaces:
  * whole-brick line sweeps with the shared-node partial carried from one cell
    segment to the next equal the cell-by-cell Kronecker-sum operator;
  * the even-odd halves of centrosymmetric and anti-centrosymmetric 1D
    matrices reproduce the plain matrix-vector product;
  * the batched cell schedule of deformed tiles with its node gather adds every
    (cell, local node) contribution exactly once and stays inside the brick;
  * the tri-quadratic metric -- per-line partial sums of the 27 support points,
    one more sum per point, cyclic cofactors and the flux (w a / det J) C^T (C g)
    -- equals J^{-1} (w det J a) J^{-T} g with J from the plain tensor-product
    interpolation.
"""
import itertools

import numpy as np
import pytest


def _cell_stride(P, ns):
    return ns * (P + 1) ** 3 + ((((P + 1) ** 2 - ns * (P + 1) ** 3) % 32) + 32) % 32


@pytest.mark.parametrize("P,nc", [(1, (4, 4, 4)), (2, (3, 1, 2)), (4, (4, 4, 4)), (5, (1, 1, 1)), (4, (2, 3, 1))])
def test_brick_line_sweeps_equal_cellwise_kronecker_sum(P, nc):
    rng = np.random.default_rng(P)
    ncx, ncy, ncz = nc
    N1 = P + 1
    M = rng.standard_normal((N1, N1))
    K = [rng.standard_normal((N1, N1)) for _ in range(3)]
    bx, by, bz = P * ncx + 1, P * ncy + 1, P * ncz + 1
    u = rng.standard_normal((bz, by, bx))
    ref = np.zeros_like(u)
    for cz, cy, cx in itertools.product(range(ncz), range(ncy), range(ncx)):
        ue = u[P * cz:P * cz + N1, P * cy:P * cy + N1, P * cx:P * cx + N1]
        z1, z2 = np.einsum("ka,ajb->kjb", M, ue), np.einsum("ka,ajb->kjb", K[2], ue)
        y1 = np.einsum("ja,kab->kjb", M, z1)
        y2 = np.einsum("ja,kab->kjb", K[1], z1) + np.einsum("ja,kab->kjb", M, z2)
        out = np.einsum("ia,kja->kji", K[0], y1) + np.einsum("ia,kja->kji", M, y2)
        ref[P * cz:P * cz + N1, P * cy:P * cy + N1, P * cx:P * cx + N1] += out
    A, B = u.reshape(-1).copy(), np.zeros(u.size)

    def sweep(kind, nlines, n0, s0, s1, st, ncl, Km):
        for t in range(nlines):
            i1, i0 = divmod(t, n0)
            b0 = i0 * s0 + i1 * s1
            ca = cb = 0.0
            for seg in range(ncl):
                idx = [b0 + st * (P * seg + s) for s in range(N1)]
                x = A[idx].copy()
                if kind == 0:
                    ya, yb = M @ x, Km @ x
                else:
                    z = B[idx].copy()
                    ya, yb = M @ x, Km @ x + M @ z
                if seg > 0:
                    ya[0] += ca
                    yb[0] += cb
                for s in range(P):
                    if kind != 2:
                        A[idx[s]] = ya[s]
                    B[idx[s]] = yb[s]
                ca, cb = ya[P], yb[P]
            if kind != 2:
                A[b0 + st * P * ncl] = ca
            B[b0 + st * P * ncl] = cb

    sweep(0, bx * by, bx, 1, bx, bx * by, ncz, K[2])
    sweep(1, bx * bz, bx, 1, bx * by, bx, ncy, K[1])
    sweep(2, by * bz, by, bx, bx * by, 1, ncx, K[0])
    np.testing.assert_allclose(B.reshape(bz, by, bx), ref, atol=1e-13 * np.abs(ref).max())


def _even_odd(x, n1):
    h, ne = n1 // 2, n1 - n1 // 2
    e = np.array([x[j] + x[n1 - 1 - j] for j in range(h)] + ([x[h]] if ne > h else []))
    o = np.array([x[j] - x[n1 - 1 - j] for j in range(h)])
    return e, o


@pytest.mark.parametrize("n1", range(2, 10))
def test_even_odd_products(n1):
    rng = np.random.default_rng(n1)
    h, ne = n1 // 2, n1 - n1 // 2
    x = rng.standard_normal(n1)
    e, o = _even_odd(x, n1)
    # centrosymmetric: y_i = E_i e + O_i o, y_{n-1-i} = E_i e - O_i o, y_h = E_h e
    A = rng.standard_normal((n1, n1))
    A = A + A[::-1, ::-1]
    E = np.array([[(0.5 * (A[i, j] + A[i, n1 - 1 - j]) if i < h else A[i, j]) if j < h else A[i, j]
                   for j in range(ne)] for i in range(ne)])
    O = np.array([[0.5 * (A[i, j] - A[i, n1 - 1 - j]) for j in range(h)] for i in range(h)])
    y = np.zeros(n1)
    for i in range(h):
        y[i], y[n1 - 1 - i] = E[i] @ e + O[i] @ o, E[i] @ e - O[i] @ o
    if ne > h:
        y[h] = E[h] @ e
    np.testing.assert_allclose(y, A @ x, atol=1e-13)
    # anti-centrosymmetric: y_i = O'_i o + E'_i e, y_{n-1-i} = O'_i o - E'_i e, y_h = O'_h o
    D = rng.standard_normal((n1, n1))
    D = D - D[::-1, ::-1]
    Ep = np.array([[0.5 * (D[i, j] + D[i, n1 - 1 - j]) if j < h else D[i, j] for j in range(ne)] for i in range(h)])
    Op = np.array([[0.5 * (D[i, j] - D[i, n1 - 1 - j]) if i < h else D[i, j] for j in range(h)] for i in range(ne)])
    y = np.zeros(n1)
    for i in range(h):
        y[i], y[n1 - 1 - i] = Op[i] @ o + Ep[i] @ e, Op[i] @ o - Ep[i] @ e
    if ne > h:
        y[h] = Op[h] @ o
    np.testing.assert_allclose(y, D @ x, atol=1e-13)


def _batch_cells(P, es, T, budget=110 * 1024):
    ncell = T[0] * T[1] * T[2]
    bricks = 2 * (P * T[0] + 1) * (P * T[1] + 1) * (P * T[2] + 1) * es
    nb = max(1, min((budget - bricks) // (_cell_stride(P, 4) * es), ncell, 512))
    nbatch = -(-ncell // nb)
    return -(-ncell // nbatch)


@pytest.mark.parametrize("P", range(1, 9))
def test_deformed_batch_gather_covers_every_contribution_once(P):
    for es in (4, 8):
        for T in [(2, 2, 2), (3, 3, 3), (4, 3, 2), (1, 2, 1)]:
            nbmax = _batch_cells(P, es, T)
            Bmax = (P * T[0] + 1) * (P * T[1] + 1) * (P * T[2] + 1)
            for nc in itertools.product(*[range(1, t + 1) for t in T]):
                ncx, ncy, ncz = nc
                bx, by = P * ncx + 1, P * ncy + 1
                count = {}
                ncell = ncx * ncy * ncz
                for c0 in range(0, ncell, nbmax):
                    nb = min(nbmax, ncell - c0)
                    nxy = ncx * ncy
                    cz_lo, cz_hi = c0 // nxy, (c0 + nb - 1) // nxy
                    for t in range(bx * by * (P * (cz_hi - cz_lo + 1) + 1)):
                        r, li = divmod(t, bx)
                        q, lj = divmod(r, by)
                        lk = P * cz_lo + q
                        xs = range((li - 1) // P if li > 0 else 0, min(li // P, ncx - 1) + 1)
                        ys = range((lj - 1) // P if lj > 0 else 0, min(lj // P, ncy - 1) + 1)
                        zs = range(max((lk - 1) // P if lk > 0 else 0, cz_lo), min(lk // P, cz_hi) + 1)
                        for cz, cy, cx in itertools.product(zs, ys, xs):
                            cid = cx + ncx * (cy + ncy * cz) - c0
                            if not 0 <= cid < nb:
                                continue
                            a, b, c = li - P * cx, lj - P * cy, lk - P * cz
                            assert 0 <= min(a, b, c) and max(a, b, c) <= P
                            assert li + bx * (lj + by * lk) < Bmax
                            key = (cx, cy, cz, a, b, c)
                            count[key] = count.get(key, 0) + 1
                assert len(count) == ncell * (P + 1) ** 3 and set(count.values()) == {1}


def _quadratic_tables(g):
    """Values and derivatives of the quadratic Lagrange polynomials through
    0, 1/2, 1 at the points g: [q][a]."""
    v = np.stack([2 * (g - 0.5) * (g - 1), -4 * g * (g - 1), 2 * g * (g - 0.5)], axis=1)
    d = np.stack([4 * g - 3, -8 * g + 4, 4 * g - 1], axis=1)
    return v, d


@pytest.mark.parametrize("P", [1, 3, 6])
def test_quadratic_metric_scheme(P):
    rng = np.random.default_rng(40 + P)
    N1 = P + 1
    x, w = np.polynomial.legendre.leggauss(N1)
    g, w = 0.5 * (x + 1), 0.5 * w
    v, dv = _quadratic_tables(g)
    s3 = np.array([0.0, 0.5, 1.0])
    # support points X[d][a + 3 (b + 3 c)]: a scaled cube, perturbed
    ref_pts = np.stack(np.meshgrid(s3, s3, s3, indexing="ij"), axis=-1)  # [a][b][c][d]
    pts = 0.3 * ref_pts + 0.01 * rng.standard_normal(ref_pts.shape)
    X = np.array([[pts[m % 3, (m // 3) % 3, m // 9, d] for m in range(27)] for d in range(3)])
    coef = lambda x0: 1.0 + 0.5 * np.sin(np.pi * x0)
    # kernel scheme: line sums G[d][a][k][qb][qc]
    G = np.zeros((3, 3, 3, N1, N1))
    for d, a, qb, qc in itertools.product(range(3), range(3), range(N1), range(N1)):
        s0 = s1 = s2 = 0.0
        for b in range(3):
            col = [X[d][a + 3 * b + 9 * c] for c in range(3)]
            e0 = sum(col[c] * v[qc, c] for c in range(3))
            e1 = sum(col[c] * dv[qc, c] for c in range(3))
            s0 += v[qb, b] * e0
            s1 += dv[qb, b] * e0
            s2 += v[qb, b] * e1
        G[d, a, :, qb, qc] = (s0, s1, s2)
    for qa, qb, qc in itertools.product(range(N1), repeat=3):
        J = np.zeros((3, 3))
        for d in range(3):
            J[d, 0] = sum(dv[qa, a] * G[d, a, 0, qb, qc] for a in range(3))
            J[d, 1] = sum(v[qa, a] * G[d, a, 1, qb, qc] for a in range(3))
            J[d, 2] = sum(v[qa, a] * G[d, a, 2, qb, qc] for a in range(3))
        x0 = sum(v[qa, a] * G[0, a, 0, qb, qc] for a in range(3))
        C = np.zeros((3, 3))
        for i, j in itertools.product(range(3), repeat=2):
            i1, i2, j1, j2 = (i + 1) % 3, (i + 2) % 3, (j + 1) % 3, (j + 2) % 3
            C[i, j] = J[i1, j1] * J[i2, j2] - J[i1, j2] * J[i2, j1]
        det = J[0] @ C[0]
        wq = w[qa] * w[qb] * w[qc]
        grad = rng.standard_normal(3)
        flux = (wq * coef(x0) / det) * (C.T @ (C @ grad))
        # plain definition: J from the tensor-product interpolation of the map
        phi = np.einsum("a,b,c->abc", v[qa], v[qb], v[qc])
        Jd = np.stack([np.einsum("abcd,a,b,c->d", pts, dv[qa], v[qb], v[qc]),
                       np.einsum("abcd,a,b,c->d", pts, v[qa], dv[qb], v[qc]),
                       np.einsum("abcd,a,b,c->d", pts, v[qa], v[qb], dv[qc])], axis=1)
        xd = np.einsum("abcd,abc->d", pts, phi)
        np.testing.assert_allclose(J, Jd, atol=1e-14)
        assert abs(x0 - xd[0]) < 1e-14
        Ji = np.linalg.inv(Jd)
        ref = Ji @ ((wq * np.linalg.det(Jd) * coef(xd[0])) * (Ji.T @ grad))
        np.testing.assert_allclose(flux, ref, rtol=1e-12, atol=1e-14 * np.abs(ref).max())
