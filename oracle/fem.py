"""Finite-element definitions of the oracle (plain FP64 numpy / scipy).

TEST INFRASTRUCTURE ONLY (see the package docstring).  Nothing here is tuned;
every function is the textbook definition of what it computes.

Problem (Sec. 2, Eqs. 1-5, restricted to one scalar component as in the
scalar Poisson workloads): find u_h in the continuous Q_p space on a
hexahedral mesh of the unit cube with homogeneous Dirichlet data such that
    sum_e P_e^T A_e P_e u = b                                   (Eq. 4)
with the cell matrix of the (variable-coefficient) Laplacian
    [A_e]_ij = sum_q w_q det(J_q) a(x_q) (J_q^{-T} grad phi_i)(J_q^{-T} grad phi_j)   (Eq. 5)
evaluated with the tensor-product Gauss rule of p+1 points per direction
(the "affine mesh, n_q=(p+1)^3" variant of Sec. 2.2) on a tensor-product
Lagrange basis whose p+1 nodes per direction are the Gauss-Lobatto points.

Conventions (shared with the tests, not with the GPU code):
* nodes per direction n_d = p*N_d + 1; global lexicographic id
  g = i + n_x*(j + n_y*k) with i the x index;
* cell (cx,cy,cz), local node (a,b,c) -> global (p*cx+a, p*cy+b, p*cz+c);
  local id a + (p+1)*(b + (p+1)*c);
* quadrature point (qa,qb,qc) -> local id qa + n*(qb + n*qc), n = p+1;
* Dirichlet rows are kept in the system as identity rows (Sec. 5.3, constrained
  unknowns kept in the linear system); their columns are zeroed.
"""
from __future__ import annotations

import dataclasses
import math

import numpy as np
import scipy.sparse as sp
from numpy.polynomial import legendre as npleg

# --------------------------------------------------------------------------------------
# 1D rules
# --------------------------------------------------------------------------------------


def gauss_lobatto_nodes(p: int) -> np.ndarray:
    """The p+1 Gauss-Lobatto-Legendre points on [0, 1]: both end points plus the
    p-1 roots of the derivative of the Legendre polynomial P_p (mapped from
    [-1, 1]).  These are the nodes of the 1D Lagrange basis of degree p."""
    if p < 1:
        raise ValueError("degree must be >= 1")
    inner = npleg.Legendre.basis(p).deriv().roots() if p > 1 else np.zeros(0)
    xi = np.concatenate(([-1.0], np.sort(np.real(inner)), [1.0]))
    return 0.5 * (xi + 1.0)


def gauss_rule(n: int) -> tuple[np.ndarray, np.ndarray]:
    """n-point Gauss-Legendre points and weights on [0, 1]."""
    x, w = npleg.leggauss(n)
    return 0.5 * (x + 1.0), 0.5 * w


def lagrange_values(nodes: np.ndarray, x: np.ndarray) -> np.ndarray:
    """V[q, j] = L_j(x_q) with L_j the Lagrange polynomial that is 1 at nodes[j]
    and 0 at the other nodes (product formula)."""
    nodes = np.asarray(nodes, dtype=float)
    x = np.atleast_1d(np.asarray(x, dtype=float))
    m = len(nodes)
    V = np.ones((len(x), m))
    for j in range(m):
        for k in range(m):
            if k != j:
                V[:, j] *= (x - nodes[k]) / (nodes[j] - nodes[k])
    return V


def lagrange_derivatives(nodes: np.ndarray, x: np.ndarray) -> np.ndarray:
    """D[q, j] = L_j'(x_q): derivative of the product formula by the product
    rule, sum over the dropped factor k of 1/(x_j - x_k) times the rest."""
    nodes = np.asarray(nodes, dtype=float)
    x = np.atleast_1d(np.asarray(x, dtype=float))
    m = len(nodes)
    D = np.zeros((len(x), m))
    for j in range(m):
        for k in range(m):
            if k == j:
                continue
            term = np.full(len(x), 1.0 / (nodes[j] - nodes[k]))
            for l in range(m):
                if l != j and l != k:
                    term *= (x - nodes[l]) / (nodes[j] - nodes[l])
            D[:, j] += term
    return D


def element_matrices_1d(p: int) -> tuple[np.ndarray, np.ndarray]:
    """1D reference stiffness and mass matrices on [0, 1] for the degree-p
    Gauss-Lobatto Lagrange basis, integrated with the (p+1)-point Gauss rule
    (exact for these polynomial integrands of degree <= 2p)."""
    nodes = gauss_lobatto_nodes(p)
    g, w = gauss_rule(p + 1)
    V = lagrange_values(nodes, g)
    D = lagrange_derivatives(nodes, g)
    K = D.T @ (w[:, None] * D)
    M = V.T @ (w[:, None] * V)
    return K, M


# --------------------------------------------------------------------------------------
# Mesh, geometry and coefficient
# --------------------------------------------------------------------------------------

COEF_CONSTANT = 0  # a(x) = 1
COEF_SIN_X = 1     # a(x) = 1 + 0.5 sin(pi x)

OP_LAPLACE = 0     # (a grad phi_i, grad phi_j): Eq. 5
OP_MASS = 1        # (a phi_i, phi_j): the mass operator of the bake-off family


@dataclasses.dataclass(frozen=True)
class Problem:
    """A Q_p Poisson (or mass) problem on the unit cube.

    cells = (N_x, N_y, N_z); ``amplitude`` A deforms the mesh by
    x -> X + A sin(2 pi X) sin(2 pi Y) sin(2 pi Z) on each component (A = 0 is
    the Cartesian mesh); ``coef`` selects a(x); ``op`` the operator;
    ``geometry_degree`` 0 uses that map itself, 2 its tri-quadratic
    interpolant in every cell through the 3^3 points {0, 1/2, 1}^3 of the
    reference cell (the "quadratic geometry" of Sec. 2.2)."""

    p: int
    cells: tuple[int, int, int]
    amplitude: float = 0.0
    coef: int = COEF_CONSTANT
    op: int = OP_LAPLACE
    geometry_degree: int = 0

    @property
    def nodes_per_dim(self) -> tuple[int, int, int]:
        return tuple(self.p * n + 1 for n in self.cells)

    @property
    def n_dofs(self) -> int:
        nx, ny, nz = self.nodes_per_dim
        return nx * ny * nz

    @property
    def n_cells(self) -> int:
        return int(np.prod(self.cells))


def _sine_bump(X, Y, Z):
    """s(X) = sin(2 pi X) sin(2 pi Y) sin(2 pi Z) and its gradient."""
    tp = 2.0 * math.pi
    sx, sy, sz = np.sin(tp * X), np.sin(tp * Y), np.sin(tp * Z)
    cx, cy, cz = np.cos(tp * X), np.cos(tp * Y), np.cos(tp * Z)
    s = sx * sy * sz
    grad = np.stack([tp * cx * sy * sz, tp * sx * cy * sz, tp * sx * sy * cz], axis=-1)
    return s, grad


def cell_index_arrays(prob: Problem, cell_ids: np.ndarray | None = None):
    """(cx, cy, cz) of the requested cells (default: all, x fastest)."""
    Nx, Ny, Nz = prob.cells
    if cell_ids is None:
        cell_ids = np.arange(prob.n_cells)
    cell_ids = np.asarray(cell_ids)
    cx = cell_ids % Nx
    cy = (cell_ids // Nx) % Ny
    cz = cell_ids // (Nx * Ny)
    return cx, cy, cz


def local_to_global(prob: Problem, cell_ids: np.ndarray | None = None) -> np.ndarray:
    """gid[e, loc]: the restriction P_e of Eq. 4 as an index array."""
    p = prob.p
    nx, ny, _ = prob.nodes_per_dim
    cx, cy, cz = cell_index_arrays(prob, cell_ids)
    a = np.arange(p + 1)
    la = np.tile(a, (p + 1) ** 2)
    lb = np.tile(np.repeat(a, p + 1), p + 1)
    lc = np.repeat(a, (p + 1) ** 2)
    gi = p * cx[:, None] + la[None, :]
    gj = p * cy[:, None] + lb[None, :]
    gk = p * cz[:, None] + lc[None, :]
    return gi + nx * (gj + ny * gk)


QUADRATIC_SUPPORT = np.array([0.0, 0.5, 1.0])


def quadrature_geometry(prob: Problem, cell_ids: np.ndarray | None = None, n_q1d: int | None = None):
    """Physical points, Jacobians, determinants and weights at the tensor Gauss
    points of the requested cells.

    Returns (x[e,q,3], J[e,q,3,3], detJ[e,q], w[q]).  J_ij = d x_i / d xhat_j
    of the map xhat -> X = h (c + xhat) -> x = X + A s(X) (1,1,1), or of its
    tri-quadratic interpolant (geometry_degree 2)."""
    n = prob.p + 1 if n_q1d is None else n_q1d
    g, w1 = gauss_rule(n)
    qa = np.tile(np.arange(n), n * n)
    qb = np.tile(np.repeat(np.arange(n), n), n)
    qc = np.repeat(np.arange(n), n * n)
    w = w1[qa] * w1[qb] * w1[qc]
    if prob.geometry_degree == 2:
        x, J = quadratic_geometry(quadratic_support_points(prob, cell_ids), g)
        return x, J, np.linalg.det(J), w
    if prob.geometry_degree != 0:
        raise ValueError("geometry_degree is 0 (exact map) or 2 (tri-quadratic)")
    h = np.array([1.0 / c for c in prob.cells])
    cx, cy, cz = cell_index_arrays(prob, cell_ids)
    X = h[0] * (cx[:, None] + g[qa][None, :])
    Y = h[1] * (cy[:, None] + g[qb][None, :])
    Z = h[2] * (cz[:, None] + g[qc][None, :])
    A = prob.amplitude
    s, grad_s = _sine_bump(X, Y, Z)
    x = np.stack([X, Y, Z], axis=-1) + A * s[..., None]
    dPhi = np.eye(3)[None, None] + A * np.ones(3)[None, None, :, None] * grad_s[:, :, None, :]
    J = dPhi * h[None, None, None, :]
    detJ = np.linalg.det(J)
    return x, J, detJ, w


def quadratic_support_points(prob: Problem, cell_ids: np.ndarray | None = None) -> np.ndarray:
    """pts[e, a, b, c, d]: coordinate d of the exact map at the reference point
    (s_a, s_b, s_c), s = (0, 1/2, 1), of each requested cell -- the 27 x 3
    values per cell that define the tri-quadratic geometry."""
    h = np.array([1.0 / c for c in prob.cells])
    cx, cy, cz = cell_index_arrays(prob, cell_ids)
    s3 = QUADRATIC_SUPPORT
    X = h[0] * (cx[:, None, None, None] + s3[:, None, None][None])
    Y = h[1] * (cy[:, None, None, None] + s3[None, :, None][None])
    Z = h[2] * (cz[:, None, None, None] + s3[None, None, :][None])
    X, Y, Z = np.broadcast_arrays(X, Y, Z)
    s, _ = _sine_bump(X, Y, Z)
    return np.stack([X, Y, Z], axis=-1) + prob.amplitude * s[..., None]


def quadratic_geometry(pts: np.ndarray, g: np.ndarray):
    """x[e,q,3] and J[e,q,3,3] of the tri-quadratic map
    x(xhat) = sum_abc pts[e,a,b,c] L_a(xhat_1) L_b(xhat_2) L_c(xhat_3)
    (L the quadratic Lagrange polynomials through 0, 1/2, 1) at the tensor
    points of the 1D points g (q = qa + n (qb + n qc))."""
    n = len(g)
    V = lagrange_values(QUADRATIC_SUPPORT, g)       # [q1, a]
    D = lagrange_derivatives(QUADRATIC_SUPPORT, g)  # [q1, a]
    e = pts.shape[0]
    x = np.einsum("eabcd,xa,yb,zc->ezyxd", pts, V, V, V).reshape(e, n ** 3, 3)
    j0 = np.einsum("eabcd,xa,yb,zc->ezyxd", pts, D, V, V).reshape(e, n ** 3, 3)
    j1 = np.einsum("eabcd,xa,yb,zc->ezyxd", pts, V, D, V).reshape(e, n ** 3, 3)
    j2 = np.einsum("eabcd,xa,yb,zc->ezyxd", pts, V, V, D).reshape(e, n ** 3, 3)
    return x, np.stack([j0, j1, j2], axis=-1)


def coefficient(prob: Problem, x: np.ndarray) -> np.ndarray:
    if prob.coef == COEF_CONSTANT:
        return np.ones(x.shape[:-1])
    if prob.coef == COEF_SIN_X:
        return 1.0 + 0.5 * np.sin(math.pi * x[..., 0])
    raise ValueError("unknown coefficient")


def manufactured_solution(x: np.ndarray) -> np.ndarray:
    return np.sin(math.pi * x[..., 0]) * np.sin(math.pi * x[..., 1]) * np.sin(math.pi * x[..., 2])


def manufactured_forcing(prob: Problem, x: np.ndarray) -> np.ndarray:
    """f = -div(a grad u*) for u* = sin(pi x) sin(pi y) sin(pi z); for the
    mass operator f = a u*."""
    u = manufactured_solution(x)
    if prob.op == OP_MASS:
        return coefficient(prob, x) * u
    if prob.coef == COEF_CONSTANT:
        return 3.0 * math.pi ** 2 * u
    a = coefficient(prob, x)
    # grad a = (0.5 pi cos(pi x), 0, 0); d u / d x = pi cos(pi x) sin(pi y) sin(pi z)
    return a * 3.0 * math.pi ** 2 * u - 0.5 * math.pi ** 2 * np.cos(math.pi * x[..., 0]) ** 2 * np.sin(
        math.pi * x[..., 1]) * np.sin(math.pi * x[..., 2])


# --------------------------------------------------------------------------------------
# Reference tables and element matrices (Eq. 5)
# --------------------------------------------------------------------------------------


def reference_tables(p: int, n_q1d: int | None = None):
    """phi[q, loc] and grad_phi[q, loc, d] of the tensor-product basis at the
    tensor Gauss points (x direction = local index a, fastest)."""
    n = p + 1 if n_q1d is None else n_q1d
    nodes = gauss_lobatto_nodes(p)
    g, _ = gauss_rule(n)
    V = lagrange_values(nodes, g)        # [qa, a]
    D = lagrange_derivatives(nodes, g)   # [qa, a]
    phi = np.einsum("xa,yb,zc->zyxcba", V, V, V).reshape(n ** 3, (p + 1) ** 3)
    gx = np.einsum("xa,yb,zc->zyxcba", D, V, V).reshape(n ** 3, (p + 1) ** 3)
    gy = np.einsum("xa,yb,zc->zyxcba", V, D, V).reshape(n ** 3, (p + 1) ** 3)
    gz = np.einsum("xa,yb,zc->zyxcba", V, V, D).reshape(n ** 3, (p + 1) ** 3)
    return phi, np.stack([gx, gy, gz], axis=-1)


def element_matrices(prob: Problem, cell_ids: np.ndarray | None = None, chunk: int = 256) -> np.ndarray:
    """A_e for the requested cells with full (p+1)^3 Gauss quadrature (Eq. 5):
    A_e = sum_q w_q det J_q a(x_q) (G_q J_q^{-1}) (G_q J_q^{-1})^T where row i of
    G_q is the reference gradient of phi_i at point q.  Mass operator:
    A_e = sum_q w_q det J_q a(x_q) phi(q) phi(q)^T."""
    if cell_ids is None:
        cell_ids = np.arange(prob.n_cells)
    cell_ids = np.asarray(cell_ids)
    phi, G = reference_tables(prob.p)
    nloc = G.shape[1]
    out = np.empty((len(cell_ids), nloc, nloc))
    for s in range(0, len(cell_ids), chunk):
        ids = cell_ids[s:s + chunk]
        x, J, detJ, w = quadrature_geometry(prob, ids)
        if prob.op == OP_MASS:
            c = w[None, :] * detJ * coefficient(prob, x)          # [e, q]
            out[s:s + chunk] = np.einsum("eq,qi,qj->eij", c, phi, phi)
            continue
        Jinv = np.linalg.inv(J)
        c = w[None, :] * detJ * coefficient(prob, x)              # [e, q]
        Gp = np.einsum("qid,eqdk->eiqk", G, Jinv)                # physical gradients
        Gw = Gp * c[:, None, :, None]
        e_n = len(ids)
        out[s:s + chunk] = np.matmul(Gw.reshape(e_n, nloc, -1), Gp.reshape(e_n, nloc, -1).transpose(0, 2, 1))
    return out


def cartesian_cells_identical(prob: Problem) -> bool:
    return prob.amplitude == 0.0 and prob.coef == COEF_CONSTANT


# --------------------------------------------------------------------------------------
# Assembly (Eq. 4), Dirichlet rows, right-hand side
# --------------------------------------------------------------------------------------


def boundary_mask(prob: Problem) -> np.ndarray:
    nx, ny, nz = prob.nodes_per_dim
    i = np.arange(nx)
    j = np.arange(ny)
    k = np.arange(nz)
    bi = (i == 0) | (i == nx - 1)
    bj = (j == 0) | (j == ny - 1)
    bk = (k == 0) | (k == nz - 1)
    return (bk[:, None, None] | bj[None, :, None] | bi[None, None, :]).reshape(-1)


def assemble(prob: Problem, dirichlet: bool = True) -> sp.csr_matrix:
    """Global sparse matrix sum_e P_e^T A_e P_e, duplicates summed.  With
    ``dirichlet`` the boundary rows and columns are replaced by identity rows."""
    gid = local_to_global(prob)
    if cartesian_cells_identical(prob):
        Ae = np.broadcast_to(element_matrices(prob, np.array([0]))[0], (prob.n_cells,) + (gid.shape[1],) * 2)
    else:
        Ae = element_matrices(prob)
    rows = np.repeat(gid, gid.shape[1], axis=1).reshape(-1)
    cols = np.tile(gid, (1, gid.shape[1])).reshape(-1)
    n = prob.n_dofs
    A = sp.coo_matrix((np.ascontiguousarray(Ae).reshape(-1), (rows, cols)), shape=(n, n)).tocsr()
    A.sum_duplicates()
    if not dirichlet:
        return A
    bnd = boundary_mask(prob)
    keep = sp.diags((~bnd).astype(float))
    return (keep @ A @ keep + sp.diags(bnd.astype(float))).tocsr()


def rhs(prob: Problem, chunk: int = 4096) -> np.ndarray:
    """b_i = sum_e sum_q w_q det J_q f(x_q) phi_i(xhat_q) on interior nodes
    (same Gauss rule as the operator), 0 on Dirichlet nodes."""
    phi, _ = reference_tables(prob.p)
    b = np.zeros(prob.n_dofs)
    for s in range(0, prob.n_cells, chunk):
        ids = np.arange(s, min(s + chunk, prob.n_cells))
        x, _, detJ, w = quadrature_geometry(prob, ids)
        fq = manufactured_forcing(prob, x) * detJ * w[None, :]
        be = fq @ phi                                             # [e, loc]
        np.add.at(b, local_to_global(prob, ids), be)
    b[boundary_mask(prob)] = 0.0
    return b


def diagonal(A: sp.csr_matrix) -> np.ndarray:
    return A.diagonal().copy()


def apply_rows(prob: Problem, u: np.ndarray, rows: np.ndarray) -> np.ndarray:
    """(A u)_i for the requested global rows only, computed one by one from the
    cells that contain node i (Eq. 4 restricted to one row); Dirichlet rows
    return u_i.  Works at any mesh size since no global matrix is formed."""
    p = prob.p
    nx, ny, nz = prob.nodes_per_dim
    Nx, Ny, Nz = prob.cells
    bnd_all = None
    rows = np.asarray(rows)
    out = np.empty(len(rows))
    ident = cartesian_cells_identical(prob)
    Ae0 = element_matrices(prob, np.array([0]))[0] if ident else None
    for t, g in enumerate(rows):
        i, j, k = g % nx, (g // nx) % ny, g // (nx * ny)
        if i in (0, nx - 1) or j in (0, ny - 1) or k in (0, nz - 1):
            out[t] = u[g]
            continue

        def cells_1d(idx, N):
            cs = []
            if idx % p == 0 and idx // p - 1 >= 0:
                cs.append(idx // p - 1)
            if idx // p < N:
                cs.append(idx // p)
            return cs

        acc = 0.0
        for cz in cells_1d(k, Nz):
            for cy in cells_1d(j, Ny):
                for cx in cells_1d(i, Nx):
                    e = cx + Nx * (cy + Ny * cz)
                    gid = local_to_global(prob, np.array([e]))[0]
                    Ae = Ae0 if ident else element_matrices(prob, np.array([e]))[0]
                    loc = (i - p * cx) + (p + 1) * ((j - p * cy) + (p + 1) * (k - p * cz))
                    ue = u[gid].copy()
                    gi, gj, gk = gid % nx, (gid // nx) % ny, gid // (nx * ny)
                    ue[(gi == 0) | (gi == nx - 1) | (gj == 0) | (gj == ny - 1) | (gk == 0) | (gk == nz - 1)] = 0.0
                    acc += Ae[loc] @ ue
        out[t] = acc
    del bnd_all
    return out


def diagonal_rows(prob: Problem, rows: np.ndarray) -> np.ndarray:
    """diag(A)_i for the requested rows from the cells containing node i."""
    p = prob.p
    nx, ny, nz = prob.nodes_per_dim
    Nx, Ny, Nz = prob.cells
    out = np.empty(len(rows))
    for t, g in enumerate(np.asarray(rows)):
        i, j, k = g % nx, (g // nx) % ny, g // (nx * ny)
        if i in (0, nx - 1) or j in (0, ny - 1) or k in (0, nz - 1):
            out[t] = 1.0
            continue
        acc = 0.0
        for cz in ([k // p - 1] if k % p == 0 else []) + ([k // p] if k // p < Nz else []):
            for cy in ([j // p - 1] if j % p == 0 else []) + ([j // p] if j // p < Ny else []):
                for cx in ([i // p - 1] if i % p == 0 else []) + ([i // p] if i // p < Nx else []):
                    e = cx + Nx * (cy + Ny * cz)
                    loc = (i - p * cx) + (p + 1) * ((j - p * cy) + (p + 1) * (k - p * cz))
                    acc += element_matrices(prob, np.array([e]))[0][loc, loc]
        out[t] = acc
    return out


# --------------------------------------------------------------------------------------
# Error of a discrete solution
# --------------------------------------------------------------------------------------


def l2_error(prob: Problem, u: np.ndarray, chunk: int = 4096) -> float:
    """|| u_h - u* ||_{L2(Omega)} with a (p+3)-point Gauss rule per direction on
    the physical cells."""
    nq = prob.p + 3
    phi, _ = reference_tables(prob.p, nq)
    err2 = 0.0
    for s in range(0, prob.n_cells, chunk):
        ids = np.arange(s, min(s + chunk, prob.n_cells))
        x, _, detJ, w = quadrature_geometry(prob, ids, nq)
        uh = u[local_to_global(prob, ids)] @ phi.T
        err2 += float(np.sum(w[None, :] * detJ * (uh - manufactured_solution(x)) ** 2))
    return math.sqrt(err2)
