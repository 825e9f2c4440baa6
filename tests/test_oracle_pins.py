"""Pins of the CPU oracle against facts fixed by mathematics, not by the oracle.

Each test would fail for a plausible mistake in the oracle: a wrong node set,
a dropped quadrature weight, a transposed basis table, a missing Jacobian
factor, a wrong sign in the forcing, a wrong index in Algorithm 5.
"""
import math
import os
from fractions import Fraction

import numpy as np
import pytest
import scipy.sparse as sp
import scipy.sparse.linalg as spla

from oracle import cg, fastdiag, fem

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


def _read_golden(name):
    rows = []
    with open(os.path.join(GOLDEN, name)) as fh:
        for line in fh:
            line = line.strip()
            if line and not line.startswith("#"):
                rows.append(line.split())
    return rows


# ---------------------------------------------------------------- 1D rules


def test_gauss_lobatto_nodes_closed_forms():
    for row in _read_golden("gauss_lobatto_nodes.txt"):
        p = int(row[0])
        xi = np.array([eval(t, {"sqrt": math.sqrt}) for t in row[1:]])
        np.testing.assert_allclose(fem.gauss_lobatto_nodes(p), 0.5 * (xi + 1.0), atol=2e-15)


def test_gauss_rule_exactness_degree():
    # n-point Gauss is exact up to degree 2n-1 and not for degree 2n
    for n in range(1, 10):
        x, w = fem.gauss_rule(n)
        for k in range(2 * n):
            assert abs(w @ x ** k - 1.0 / (k + 1)) < 1e-14
        assert abs(w @ x ** (2 * n) - 1.0 / (2 * n + 1)) > 1e-12
    x, w = fem.gauss_rule(3)
    np.testing.assert_allclose(x, [0.5 - math.sqrt(15) / 10, 0.5, 0.5 + math.sqrt(15) / 10], atol=1e-15)
    np.testing.assert_allclose(w, [5 / 18, 8 / 18, 5 / 18], atol=1e-15)


def test_lagrange_tables_reproduce_polynomials():
    rng = np.random.default_rng(1)
    for p in range(1, 9):
        nodes = fem.gauss_lobatto_nodes(p)
        x = rng.random(7)
        V = fem.lagrange_values(nodes, x)
        D = fem.lagrange_derivatives(nodes, x)
        np.testing.assert_allclose(fem.lagrange_values(nodes, nodes), np.eye(p + 1), atol=1e-13)
        for m in range(p + 1):
            np.testing.assert_allclose(V @ nodes ** m, x ** m, atol=1e-12)
            deriv = m * x ** (m - 1) if m > 0 else np.zeros_like(x)
            np.testing.assert_allclose(D @ nodes ** m, deriv, atol=1e-10)


def test_1d_matrices_exact_q1_q2():
    for row in _read_golden("q1_q2_1d_matrices.txt"):
        name, p = row[0], int(row[1])
        exact = np.array([float(Fraction(t)) for t in row[2:]]).reshape(p + 1, p + 1)
        K, M = fem.element_matrices_1d(p)
        np.testing.assert_allclose(K if name == "K" else M, exact, atol=1e-14)


def test_1d_matrices_match_symbolic_integration():
    sympy = pytest.importorskip("sympy")
    X = sympy.Symbol("x")
    for p in (3, 4, 5):
        xi = sorted(sympy.Poly(sympy.diff(sympy.legendre(p, X), X), X).nroots(n=40))
        nodes = [sympy.Integer(0)] + [(t + 1) / 2 for t in xi] + [sympy.Integer(1)]
        L = []
        for j in range(p + 1):
            e = sympy.Integer(1)
            for k in range(p + 1):
                if k != j:
                    e *= (X - nodes[k]) / (nodes[j] - nodes[k])
            L.append(sympy.expand(e))
        K_ex = np.array([[float(sympy.integrate(sympy.diff(L[i], X) * sympy.diff(L[j], X), (X, 0, 1)))
                          for j in range(p + 1)] for i in range(p + 1)])
        M_ex = np.array([[float(sympy.integrate(L[i] * L[j], (X, 0, 1))) for j in range(p + 1)]
                         for i in range(p + 1)])
        K, M = fem.element_matrices_1d(p)
        np.testing.assert_allclose(K, K_ex, atol=1e-12 * np.abs(K_ex).max())
        np.testing.assert_allclose(M, M_ex, atol=1e-13)


# ---------------------------------------------------------------- operator


def _kronecker_operator(p, cells, K1, M1):
    """Independent construction A = sum of Kronecker products of 1D assembled
    matrices (x fastest), Dirichlet identity rows."""
    mats = []
    for d in range(3):
        n = p * cells[d] + 1
        h = 1.0 / cells[d]
        Kg = np.zeros((n, n))
        Mg = np.zeros((n, n))
        for c in range(cells[d]):
            s = slice(p * c, p * c + p + 1)
            Kg[s, s] += K1 / h
            Mg[s, s] += M1 * h
        mats.append((sp.csr_matrix(Kg), sp.csr_matrix(Mg)))
    (Kx, Mx), (Ky, My), (Kz, Mz) = mats
    A = sp.kron(Kz, sp.kron(My, Mx)) + sp.kron(Mz, sp.kron(Ky, Mx)) + sp.kron(Mz, sp.kron(My, Kx))
    prob = fem.Problem(p, cells)
    bnd = fem.boundary_mask(prob)
    keep = sp.diags((~bnd).astype(float))
    return (keep @ A @ keep + sp.diags(bnd.astype(float))).tocsr()


def test_assembled_equals_kronecker_q2_exact_1d():
    rows = {(r[0], int(r[1])): np.array([float(Fraction(t)) for t in r[2:]]) for r in _read_golden("q1_q2_1d_matrices.txt")}
    K1, M1 = rows[("K", 2)].reshape(3, 3), rows[("M", 2)].reshape(3, 3)
    cells = (3, 2, 4)
    A = fem.assemble(fem.Problem(2, cells))
    B = _kronecker_operator(2, cells, K1, M1)
    assert abs(A - B).max() < 1e-13 * abs(B).max()


def test_assembled_equals_kronecker_higher_degree():
    for p, cells in ((4, (2, 3, 2)), (6, (2, 2, 1))):
        K1, M1 = fem.element_matrices_1d(p)
        A = fem.assemble(fem.Problem(p, cells))
        B = _kronecker_operator(p, cells, K1, M1)
        assert abs(A - B).max() < 1e-13 * abs(B).max()


def test_q1_27_point_stencil():
    vals = {r[0]: float(Fraction(r[1])) for r in _read_golden("q1_stencil.txt")}
    N = 4
    prob = fem.Problem(1, (N, N, N))
    A = fem.assemble(prob)
    h = 1.0 / N
    nx = N + 1
    c = 2 + nx * (2 + nx * 2)
    row = A.getrow(c).toarray().ravel()
    for dz in (-1, 0, 1):
        for dy in (-1, 0, 1):
            for dx in (-1, 0, 1):
                nnz = abs(dx) + abs(dy) + abs(dz)
                cls = ["centre", "face", "edge", "corner"][nnz]
                assert abs(row[c + dx + nx * (dy + nx * dz)] - vals[cls] * h) < 1e-14


@pytest.mark.parametrize("amp,coef,gdeg", [(0.0, fem.COEF_CONSTANT, 0), (0.05, fem.COEF_SIN_X, 0),
                                           (0.08, fem.COEF_CONSTANT, 0), (0.08, fem.COEF_SIN_X, 2)])
def test_symmetric_positive_definite(amp, coef, gdeg):
    prob = fem.Problem(3, (2, 3, 2), amp, coef, geometry_degree=gdeg)
    A = fem.assemble(prob).toarray()
    assert np.abs(A - A.T).max() < 1e-14 * np.abs(A).max()
    np.linalg.cholesky(A)
    assert np.linalg.eigvalsh(A).min() > 0


@pytest.mark.parametrize("amp,coef,gdeg", [(0.0, fem.COEF_CONSTANT, 0), (0.05, fem.COEF_SIN_X, 0),
                                           (0.08, fem.COEF_SIN_X, 0), (0.08, fem.COEF_SIN_X, 2)])
def test_neumann_constant_null_space(amp, coef, gdeg):
    prob = fem.Problem(4, (2, 2, 3), amp, coef, geometry_degree=gdeg)
    A = fem.assemble(prob, dirichlet=False)
    r = A @ np.ones(prob.n_dofs)
    assert np.abs(r).max() < 1e-14 * abs(A).max() * 10


def test_deformed_jacobian_matches_finite_differences():
    prob = fem.Problem(3, (2, 2, 2), 0.07)
    x, J, detJ, _ = fem.quadrature_geometry(prob, np.array([0, 5]))
    # perturb the reference coordinate of one point through a shifted rule is not
    # available, so difference the physical map directly: x(X) = X + A s(X)(1,1,1)
    h = 0.5
    g, _ = fem.gauss_rule(4)
    for e, (cx, cy, cz) in enumerate([(0, 0, 0), (1, 0, 1)]):
        for q in (0, 17, 40):
            qa, qb, qc = q % 4, (q // 4) % 4, q // 16
            xh = np.array([g[qa], g[qb], g[qc]])
            c = np.array([cx, cy, cz])

            def phys(xhat):
                X = h * (c + xhat)
                s = np.sin(2 * np.pi * X[0]) * np.sin(2 * np.pi * X[1]) * np.sin(2 * np.pi * X[2])
                return X + 0.07 * s

            eps = 1e-6
            Jfd = np.stack([(phys(xh + eps * np.eye(3)[d]) - phys(xh - eps * np.eye(3)[d])) / (2 * eps)
                            for d in range(3)], axis=1)
            np.testing.assert_allclose(J[e, q], Jfd, atol=1e-8)
            np.testing.assert_allclose(x[e, q], phys(xh), atol=1e-15)
            assert detJ[e, q] > 0


# ---------------------------------------------------------------- tri-quadratic geometry


def test_quadratic_geometry_is_exact_for_triquadratic_maps():
    # a map of degree <= 2 in each reference coordinate is its own interpolant:
    # its values and derivatives at the Gauss points come out exactly
    rng = np.random.default_rng(17)
    C = rng.standard_normal((3, 3, 3, 3))  # C[d, i, j, k]: coefficient of u^i v^j w^k in component d

    def f(u, v, w):
        return np.array([sum(C[d, i, j, k] * u ** i * v ** j * w ** k
                             for i in range(3) for j in range(3) for k in range(3)) for d in range(3)])

    def df(u, v, w, e):
        out = np.zeros(3)
        for d in range(3):
            for i in range(3):
                for j in range(3):
                    for k in range(3):
                        ex = [i, j, k]
                        if ex[e] == 0:
                            continue
                        fac = ex[e]
                        ex[e] -= 1
                        out[d] += C[d, i, j, k] * fac * u ** ex[0] * v ** ex[1] * w ** ex[2]
        return out

    s3 = fem.QUADRATIC_SUPPORT
    pts = np.array([[[f(s3[a], s3[b], s3[c]) for c in range(3)] for b in range(3)] for a in range(3)])[None]
    g, _ = fem.gauss_rule(4)
    x, J = fem.quadratic_geometry(pts, g)
    for q in (0, 7, 21, 42, 63):
        qa, qb, qc = q % 4, (q // 4) % 4, q // 16
        u, v, w = g[qa], g[qb], g[qc]
        np.testing.assert_allclose(x[0, q], f(u, v, w), atol=1e-13)
        for e in range(3):
            np.testing.assert_allclose(J[0, q, :, e], df(u, v, w, e), atol=1e-12)


@pytest.mark.parametrize("p", [1, 3, 5])
def test_quadratic_geometry_of_cartesian_cells_is_exact(p):
    # the interpolant of an affine map is the map: same element matrices
    pe = fem.Problem(p, (3, 2, 4))
    pq = fem.Problem(p, (3, 2, 4), geometry_degree=2)
    ids = np.array([0, 5, 23])
    Ae, Aq = fem.element_matrices(pe, ids), fem.element_matrices(pq, ids)
    np.testing.assert_allclose(Aq, Ae, atol=1e-13 * np.abs(Ae).max())


def test_quadratic_geometry_interpolates_the_deformed_map():
    # through the 27 support points of every cell, and within O(h^3) of the
    # map (positions and d x / d xhat, which carries a factor h) between them
    prob = fem.Problem(2, (3, 4, 3), 0.07, geometry_degree=2)
    ids = np.array([0, 11, 35])
    x, _ = fem.quadratic_geometry(fem.quadratic_support_points(prob, ids), fem.QUADRATIC_SUPPORT)
    exact = fem.Problem(2, (3, 4, 3), 0.07)
    h = np.array([1 / 3, 1 / 4, 1 / 3])
    cx, cy, cz = fem.cell_index_arrays(exact, ids)
    s3 = fem.QUADRATIC_SUPPORT
    for t in range(len(ids)):
        for q in range(27):
            a, b, c = q % 3, (q // 3) % 3, q // 9
            X = h * (np.array([cx[t], cy[t], cz[t]]) + np.array([s3[a], s3[b], s3[c]]))
            sb = np.prod(np.sin(2 * np.pi * X))
            np.testing.assert_allclose(x[t, q], X + 0.07 * sb, atol=1e-15)
    errs = []
    for N in (8, 16):
        x0, J0, _, _ = fem.quadrature_geometry(fem.Problem(2, (N, N, N), 0.05))
        x2, J2, _, _ = fem.quadrature_geometry(fem.Problem(2, (N, N, N), 0.05, geometry_degree=2))
        errs.append((np.abs(x0 - x2).max(), np.abs(J0 - J2).max()))
    for m in range(2):
        assert abs(math.log2(errs[0][m] / errs[1][m]) - 3) < 0.15, errs


def test_l2_convergence_rate_quadratic_geometry():
    # the tri-quadratic cells tile the unit cube exactly (the map fixes the
    # boundary), so the discrete solution keeps the rate p + 1
    for p, Ns, tol in ((2, (2, 4, 8), 0.1), (3, (4, 8), 0.4)):
        errs = []
        for N in Ns:
            prob = fem.Problem(p, (N, N, N), 0.05, fem.COEF_SIN_X, geometry_degree=2)
            u = spla.spsolve(fem.assemble(prob).tocsc(), fem.rhs(prob))
            errs.append(fem.l2_error(prob, u))
        rate = math.log(errs[-2] / errs[-1]) / math.log(Ns[-1] / Ns[-2])
        assert abs(rate - (p + 1)) <= tol, (p, errs, rate)


def test_forcing_matches_finite_difference_operator():
    rng = np.random.default_rng(3)
    for coef in (fem.COEF_CONSTANT, fem.COEF_SIN_X):
        prob = fem.Problem(2, (2, 2, 2), 0.0, coef)
        pts = 0.1 + 0.8 * rng.random((5, 3))
        eps = 1e-4

        def a(x):
            return fem.coefficient(prob, x)

        for x in pts:
            div = 0.0
            for d in range(3):
                e = eps * np.eye(3)[d]
                fp = a(x + e / 2) * (fem.manufactured_solution(x + e) - fem.manufactured_solution(x)) / eps
                fm = a(x - e / 2) * (fem.manufactured_solution(x) - fem.manufactured_solution(x - e)) / eps
                div += (fp - fm) / eps
            assert abs(-div - fem.manufactured_forcing(prob, x)) < 1e-5 * 30


@pytest.mark.parametrize("p,amp,coef", [(2, 0.0, fem.COEF_CONSTANT), (3, 0.0, fem.COEF_SIN_X),
                                        (2, 0.05, fem.COEF_SIN_X), (2, 0.08, fem.COEF_CONSTANT)])
def test_l2_convergence_rate(p, amp, coef):
    # the sine deformation has unit wavelength, so its Jacobian varies on a
    # scale of 1/(2 pi); rates on deformed meshes are read between N = 4 and 8
    errs = []
    Ns = (2, 4, 8) if p == 2 else (2, 4, 6)
    for N in Ns:
        prob = fem.Problem(p, (N, N, N), amp, coef)
        A = fem.assemble(prob)
        u = spla.spsolve(A.tocsc(), fem.rhs(prob))
        errs.append(fem.l2_error(prob, u))
    rate = math.log(errs[-2] / errs[-1]) / math.log(Ns[-1] / Ns[-2])
    assert rate > p + 1 - 0.35, (errs, rate)


@pytest.mark.parametrize("p", [4, 5, 6])
def test_l2_convergence_rate_high_degree_cartesian(p):
    # the exact discrete solution by fast diagonalisation (independent of the
    # assembled matrix) converges at the rate p + 1 in L2, within +-0.1
    errs = []
    Ns = (2, 4, 8)
    for N in Ns:
        prob = fem.Problem(p, (N, N, N))
        u = fastdiag.solve(prob, fem.rhs(prob))
        errs.append(fem.l2_error(prob, u))
    rate = math.log(errs[-2] / errs[-1]) / math.log(Ns[-1] / Ns[-2])
    assert abs(rate - (p + 1)) <= 0.1, (errs, rate)


def test_l2_convergence_rate_degree4_deformed():
    # deformed mesh with the variable coefficient at degree 4: rate 5 within
    # +-0.1 between N = 4 and 6 (higher degrees on this unit-wavelength
    # deformation are still pre-asymptotic below N = 8)
    errs = []
    Ns = (2, 4, 6)
    for N in Ns:
        prob = fem.Problem(4, (N, N, N), 0.05, fem.COEF_SIN_X)
        A = fem.assemble(prob)
        u = spla.spsolve(A.tocsc(), fem.rhs(prob))
        errs.append(fem.l2_error(prob, u))
    rate = math.log(errs[-2] / errs[-1]) / math.log(Ns[-1] / Ns[-2])
    assert abs(rate - 5) <= 0.1, (errs, rate)


def test_apply_rows_matches_assembled_matrix():
    rng = np.random.default_rng(5)
    for prob in (fem.Problem(2, (3, 2, 3)), fem.Problem(3, (2, 2, 2), 0.05, fem.COEF_SIN_X)):
        A = fem.assemble(prob)
        u = rng.standard_normal(prob.n_dofs)
        rows = rng.choice(prob.n_dofs, 40, replace=False)
        np.testing.assert_allclose(fem.apply_rows(prob, u, rows), (A @ u)[rows], atol=1e-13 * np.abs(A @ u).max())
        np.testing.assert_allclose(fem.diagonal_rows(prob, rows), A.diagonal()[rows], atol=1e-14)


# ---------------------------------------------------------------- solvers


def _exact_q2_system(cells):
    rows = {(r[0], int(r[1])): [Fraction(t) for t in r[2:]] for r in _read_golden("q1_q2_1d_matrices.txt")}
    K1 = np.array(rows[("K", 2)], dtype=object).reshape(3, 3)
    M1 = np.array(rows[("M", 2)], dtype=object).reshape(3, 3)
    mats = []
    for d in range(3):
        n = 2 * cells[d] + 1
        h = Fraction(1, cells[d])
        Kg = np.zeros((n, n), dtype=object)
        Mg = np.zeros((n, n), dtype=object)
        Kg[:] = Fraction(0)
        Mg[:] = Fraction(0)
        for c in range(cells[d]):
            for i in range(3):
                for j in range(3):
                    Kg[2 * c + i, 2 * c + j] += K1[i, j] / h
                    Mg[2 * c + i, 2 * c + j] += M1[i, j] * h
        mats.append((Kg[1:-1, 1:-1], Mg[1:-1, 1:-1]))
    (Kx, Mx), (Ky, My), (Kz, Mz) = mats
    A = np.kron(Kz, np.kron(My, Mx)) + np.kron(Mz, np.kron(Ky, Mx)) + np.kron(Mz, np.kron(My, Kx))
    return A


def test_algorithm5_equals_algorithm1_exact_rationals():
    A = _exact_q2_system((2, 2, 2))  # 27 interior unknowns
    n = A.shape[0]
    b = np.array([Fraction((7 * i) % 5 - 2) for i in range(n)], dtype=object)
    inv_diag = np.array([1 / A[i, i] for i in range(n)], dtype=object)

    def apply_A(x):
        return A.dot(x)

    rtol = Fraction(1, 10 ** 8)
    r1 = cg.pcg_algorithm1(apply_A, b, inv_diag, rtol, 100)
    r5 = cg.pcg_algorithm5(apply_A, b, inv_diag, rtol, 100)
    assert r1.iterations == r5.iterations
    assert r1.alphas == r5.alphas
    assert r1.betas == r5.betas
    assert r1.residual_sq_history == r5.residual_sq_history
    assert list(r1.x) == list(r5.x)
    # CG terminates in at most n steps in exact arithmetic with the exact solution
    assert r1.iterations <= n


def test_algorithm5_odd_and_even_finalisation_exact():
    A = _exact_q2_system((2, 2, 2))
    n = A.shape[0]
    b = np.array([Fraction((3 * i) % 7 - 3) for i in range(n)], dtype=object)
    inv_diag = np.array([1 / A[i, i] for i in range(n)], dtype=object)
    for maxit in (1, 2, 3, 4, 5, 6):
        r1 = cg.pcg_algorithm1(lambda x: A.dot(x), b, inv_diag, Fraction(0), maxit)
        r5 = cg.pcg_algorithm5(lambda x: A.dot(x), b, inv_diag, Fraction(0), maxit)
        assert r1.iterations == r5.iterations == maxit
        assert list(r1.x) == list(r5.x)


def test_cg_fp64_converges_to_direct_solution():
    prob = fem.Problem(2, (8, 8, 8))
    A = fem.assemble(prob)
    b = fem.rhs(prob)
    inv_diag = 1.0 / A.diagonal()
    x_direct = spla.spsolve(A.tocsc(), b)
    r1 = cg.pcg_algorithm1(lambda x: A @ x, b, inv_diag, 1e-10, 1000)
    r5 = cg.pcg_algorithm5(lambda x: A @ x, b, inv_diag, 1e-10, 1000)
    assert r1.converged and r5.converged
    assert abs(r1.iterations - r5.iterations) <= 1
    assert np.linalg.norm(b - A @ r1.x) < 1e-10 * np.linalg.norm(b)
    assert np.abs(r1.x - x_direct).max() < 1e-8 * np.abs(x_direct).max()
    assert np.abs(r5.x - r1.x).max() < 1e-9 * np.abs(r1.x).max()


def test_fast_diagonalisation_matches_direct_solve():
    rng = np.random.default_rng(11)
    for p, cells in ((2, (3, 4, 2)), (4, (2, 2, 3))):
        prob = fem.Problem(p, cells)
        A = fem.assemble(prob)
        b = rng.standard_normal(prob.n_dofs)
        x = fastdiag.solve(prob, b)
        np.testing.assert_allclose(A @ x, b, atol=1e-11 * np.abs(b).max())


def test_kronecker_apply_matches_assembled_matrix():
    rng = np.random.default_rng(13)
    for p, cells in ((1, (3, 4, 2)), (2, (3, 2, 4)), (4, (2, 3, 2)), (7, (1, 2, 2))):
        prob = fem.Problem(p, cells)
        A = fem.assemble(prob)
        u = rng.standard_normal(prob.n_dofs)
        ref = A @ u
        np.testing.assert_allclose(fastdiag.apply(prob, u), ref, atol=1e-13 * np.abs(ref).max())



def test_algorithm5_with_identity_is_algorithm4_exact_rationals():
    # M = I: Algorithm 5 becomes the merged CG of Algorithm 4 and must reproduce
    # plain CG (Algorithm 1 with M = I) exactly
    A = _exact_q2_system((2, 2, 2))
    n = A.shape[0]
    b = np.array([Fraction((5 * i) % 9 - 4) for i in range(n)], dtype=object)
    ones = np.array([Fraction(1)] * n, dtype=object)
    r1 = cg.pcg_algorithm1(lambda x: A.dot(x), b, ones, Fraction(1, 10 ** 9), 100)
    r5 = cg.pcg_algorithm5(lambda x: A.dot(x), b, ones, Fraction(1, 10 ** 9), 100)
    assert r1.iterations == r5.iterations
    assert r1.alphas == r5.alphas and r1.betas == r5.betas
    assert list(r1.x) == list(r5.x)


# ---------------------------------------------------------------- mass operator


def _mass_kronecker(p, cells, M1, dirichlet=True):
    """h^3 M (x) M (x) M from 1D assembled mass matrices (x fastest)."""
    mats = []
    for d in range(3):
        n = p * cells[d] + 1
        h = 1.0 / cells[d]
        Mg = np.zeros((n, n))
        for c in range(cells[d]):
            s = slice(p * c, p * c + p + 1)
            Mg[s, s] += M1 * h
        mats.append(sp.csr_matrix(Mg))
    Mx, My, Mz = mats
    A = sp.kron(Mz, sp.kron(My, Mx)).tocsr()
    if not dirichlet:
        return A
    bnd = fem.boundary_mask(fem.Problem(p, cells))
    keep = sp.diags((~bnd).astype(float))
    return (keep @ A @ keep + sp.diags(bnd.astype(float))).tocsr()


def test_mass_matrix_equals_kronecker_q2_exact_1d():
    # Cartesian mass matrix = Kronecker product of the exact rational Q2 1D mass matrices
    rows = {(r[0], int(r[1])): np.array([float(Fraction(t)) for t in r[2:]]) for r in _read_golden("q1_q2_1d_matrices.txt")}
    M1 = rows[("M", 2)].reshape(3, 3)
    cells = (3, 2, 4)
    A = fem.assemble(fem.Problem(2, cells, op=fem.OP_MASS))
    B = _mass_kronecker(2, cells, M1)
    assert abs(A - B).max() < 1e-14 * abs(B).max()


@pytest.mark.parametrize("p,amp,tol", [(3, 0.0, 1e-14), (4, 0.05, 1e-13), (2, 0.08, 1e-13)])
def test_mass_matrix_total_is_domain_volume(p, amp, tol):
    # without boundary rows, 1^T M 1 = |Omega| = 1: the deformation maps the unit
    # cube onto itself.  On deformed cells det J/h^3 = 1 + A (ds/dX + ds/dY + ds/dZ)
    # and each derivative term sums to zero exactly over a uniform row of cells
    # with the same Gauss rule in every cell (a sum of e^{2 pi i c/N} over c)
    A = fem.assemble(fem.Problem(p, (3, 3, 2), amp, op=fem.OP_MASS), dirichlet=False)
    one = np.ones(A.shape[0])
    assert abs(one @ (A @ one) - 1.0) < tol


@pytest.mark.parametrize("p", [1, 3, 5])
def test_quadratic_geometry_volume_is_exact(p):
    # the tri-quadratic cells tile the unit cube exactly, and since the map adds
    # the same interpolated scalar s_h to every coordinate, det J = h_x h_y h_z
    # (1 + A sum_i (d s_h / d xhat_i) / h_i) has degree <= 2 in each reference
    # coordinate: every Gauss rule here integrates it exactly, so 1^T M 1 = 1 to
    # rounding however large the deformation
    A = fem.assemble(fem.Problem(p, (3, 2, 3), 0.09, op=fem.OP_MASS, geometry_degree=2), dirichlet=False)
    one = np.ones(A.shape[0])
    assert abs(one @ (A @ one) - 1.0) < 1e-13


def test_mass_projection_reproduces_polynomial():
    # u = x(1-x) y(1-y) z(1-z) lies in Q_2 and vanishes on the boundary: the
    # discrete L2 projection (mass matrix, right-hand side by the same Gauss rule,
    # exact for this integrand) returns its nodal values
    prob = fem.Problem(2, (3, 2, 3), op=fem.OP_MASS)
    A = fem.assemble(prob)
    phi, _ = fem.reference_tables(prob.p)
    b = np.zeros(prob.n_dofs)
    ids = np.arange(prob.n_cells)
    x, _, detJ, w = fem.quadrature_geometry(prob, ids)
    u = np.prod(x * (1.0 - x), axis=-1)
    np.add.at(b, fem.local_to_global(prob, ids), (u * detJ * w[None, :]) @ phi)
    b[fem.boundary_mask(prob)] = 0.0
    xs = spla.spsolve(A.tocsc(), b)
    nx, ny, nz = prob.nodes_per_dim
    nodes = fem.gauss_lobatto_nodes(prob.p)
    coord = [np.concatenate([(c + nodes[:-1]) / n for c in range(n)] + [np.array([1.0])]) for n in prob.cells]
    Z, Y, X = np.meshgrid(coord[2], coord[1], coord[0], indexing="ij")
    exact = (X * (1 - X) * Y * (1 - Y) * Z * (1 - Z)).reshape(-1)
    np.testing.assert_allclose(xs, exact, atol=1e-14)
