"""Exact discrete solution of the Cartesian problem by fast diagonalisation.

TEST INFRASTRUCTURE ONLY (see the package docstring).

On a Cartesian mesh of box cells with a = 1 the element matrix of Eq. 5 is
the Kronecker sum h_x h_y h_z (K/h_x^2 (x) M (x) M + ...) of the 1D reference
matrices, so the assembled interior operator is
    A = K_z (x) M_y (x) M_x + M_z (x) K_y (x) M_x + M_z (x) M_y (x) K_x
with 1D assembled matrices K_d = assemble(K)/h_d and M_d = assemble(M) h_d
restricted to the interior nodes (lexicographic order, x fastest = last
Kronecker factor).  With the generalised eigenpairs K_d S_d = M_d S_d L_d,
S_d^T M_d S_d = I, one gets A^{-1} = S (Lx + Ly + Lz)^{-1} S^T with
S = S_z (x) S_y (x) S_x, applied axis by axis in O(n * max(n_d)) work.
"""
from __future__ import annotations

import numpy as np
import scipy.linalg as sla

from . import fem


def assembled_1d(p: int, n_cells: int) -> tuple[np.ndarray, np.ndarray]:
    """1D assembled stiffness (reference scaling, h = 1) and mass matrices on
    all p*n_cells+1 nodes."""
    K, M = fem.element_matrices_1d(p)
    n = p * n_cells + 1
    Kg = np.zeros((n, n))
    Mg = np.zeros((n, n))
    for c in range(n_cells):
        s = slice(p * c, p * c + p + 1)
        Kg[s, s] += K
        Mg[s, s] += M
    return Kg, Mg


def _eig_1d(p: int, n_cells: int):
    h = 1.0 / n_cells
    Kg, Mg = assembled_1d(p, n_cells)
    Ki = Kg[1:-1, 1:-1] / h
    Mi = Mg[1:-1, 1:-1] * h
    lam, S = sla.eigh(Ki, Mi)
    return lam, S


def solve(prob: fem.Problem, b: np.ndarray) -> np.ndarray:
    """x = A^{-1} b for the Cartesian Dirichlet problem (identity boundary
    rows: x_i = b_i there)."""
    if not fem.cartesian_cells_identical(prob) or prob.op != fem.OP_LAPLACE:
        raise ValueError("fast diagonalisation needs the Laplacian on a Cartesian mesh with a = 1")
    nx, ny, nz = prob.nodes_per_dim
    B = b.reshape(nz, ny, nx)
    x = b.copy().reshape(nz, ny, nx)
    lx, Sx = _eig_1d(prob.p, prob.cells[0])
    ly, Sy = _eig_1d(prob.p, prob.cells[1])
    lz, Sz = _eig_1d(prob.p, prob.cells[2])
    U = B[1:-1, 1:-1, 1:-1]
    # apply S^T axis by axis
    U = np.einsum("ia,kji->kja", Sx, U, optimize=True)
    U = np.einsum("jb,kja->kba", Sy, U, optimize=True)
    U = np.einsum("kc,kba->cba", Sz, U, optimize=True)
    U = U / (lz[:, None, None] + ly[None, :, None] + lx[None, None, :])
    U = np.einsum("ia,kja->kji", Sx, U, optimize=True)
    U = np.einsum("jb,kba->kja", Sy, U, optimize=True)
    U = np.einsum("kc,cba->kba", Sz, U, optimize=True)
    x[1:-1, 1:-1, 1:-1] = U
    return x.reshape(-1)


def _sparse_1d(p: int, n_cells: int):
    h = 1.0 / n_cells
    Kg, Mg = assembled_1d(p, n_cells)
    import scipy.sparse as sp
    return sp.csr_matrix(Kg / h), sp.csr_matrix(Mg * h)


def apply(prob: fem.Problem, u: np.ndarray) -> np.ndarray:
    """A u for the Cartesian Dirichlet problem from the Kronecker-sum form
    A = K_z (x) M_y (x) M_x + M_z (x) K_y (x) M_x + M_z (x) M_y (x) K_x on the
    interior nodes (boundary columns zero), identity rows on the boundary.
    Cost O(n p) with sparse 1D factors, usable at any mesh size."""
    if not fem.cartesian_cells_identical(prob) or prob.op != fem.OP_LAPLACE:
        raise ValueError("the Kronecker form needs the Laplacian on a Cartesian mesh with a = 1")
    nx, ny, nz = prob.nodes_per_dim
    Kx, Mx = _sparse_1d(prob.p, prob.cells[0])
    Ky, My = _sparse_1d(prob.p, prob.cells[1])
    Kz, Mz = _sparse_1d(prob.p, prob.cells[2])
    U = u.reshape(nz, ny, nx).copy()
    bnd = fem.boundary_mask(prob).reshape(nz, ny, nx)
    U[bnd] = 0.0

    def along(mat, X, axis):
        Xm = np.moveaxis(X, axis, 0)
        shp = Xm.shape
        Y = (mat @ Xm.reshape(shp[0], -1)).reshape(shp)
        return np.moveaxis(Y, 0, axis)

    Mx_u = along(Mx, U, 2)
    Kx_u = along(Kx, U, 2)
    MyMx = along(My, Mx_u, 1)
    out = along(Kz, MyMx, 0)
    out += along(Mz, along(Ky, Mx_u, 1) + along(My, Kx_u, 1), 0)
    out[bnd] = u.reshape(nz, ny, nx)[bnd]
    return out.reshape(-1)

