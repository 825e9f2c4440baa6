"""Conjugate-gradient iterations of the oracle.

TEST INFRASTRUCTURE ONLY (see the package docstring).

Both solvers are generic over the scalar type: ``apply_A`` maps a 1D numpy
array to A times it, ``inv_diag`` holds 1/diag(A), and every operation is an
elementwise product, a sum or a division, so that the same code runs in FP64
and in exact rationals (numpy object arrays of ``fractions.Fraction``).

Stopping rule (reading of Sec. 3.1 / Algorithm 1): the unpreconditioned
residual, ||r_{k+1}||^2 < eps^2 with eps = rtol * ||b||; squares are compared
so that no square root is needed.  The iteration count is the number of
products A p.
"""
from __future__ import annotations

import dataclasses
from typing import Callable

import numpy as np


def _dot(a, b):
    return (a * b).sum()


@dataclasses.dataclass
class CGResult:
    x: np.ndarray
    iterations: int
    converged: bool
    residual_sq_history: list  # ||r_k||^2 after each product A p (explicit in Alg. 1)
    alphas: list
    betas: list


def pcg_algorithm1(apply_A: Callable, b, inv_diag, rtol, maxit: int, x0=None) -> CGResult:
    """Algorithm 1: preconditioned CG with the point-Jacobi preconditioner
    M^{-1} = diag(A)^{-1}."""
    x = b * 0 if x0 is None else x0.copy()
    r = b - apply_A(x) if x0 is not None else b.copy()
    eps_sq = rtol * rtol * _dot(b, b)
    hist, alphas, betas = [], [], []
    if _dot(r, r) == 0:
        return CGResult(x, 0, True, hist, alphas, betas)
    z = inv_diag * r
    p = z.copy()
    e = _dot(r, z)
    k = 0
    converged = False
    while k < maxit:
        v = apply_A(p)
        alpha = e / _dot(p, v)
        x = x + alpha * p
        r = r - alpha * v
        k += 1
        gamma = _dot(r, r)
        hist.append(gamma)
        alphas.append(alpha)
        if gamma < eps_sq:
            converged = True
            break
        z = inv_diag * r
        e_new = _dot(r, z)
        beta = e_new / e
        betas.append(beta)
        p = z + beta * p
        e = e_new
    return CGResult(x, k, converged, hist, alphas, betas)


def pcg_algorithm5(apply_A: Callable, b, inv_diag, rtol, maxit: int, x0=None) -> CGResult:
    """Algorithm 5: preconditioned CG with merged vector operations.

    Per iteration k = 1, 2, ...: (odd k > 1) the delayed solution update
    x_k = x_{k-2} + alpha_{k-1} p_{k-1} + alpha_{k-2}/beta_{k-2} (p_{k-1} - M^{-1} r_{k-1});
    r_k = r_{k-1} - alpha_{k-1} v_{k-1};  p_k = M^{-1} r_k + beta_{k-1} p_{k-1};
    v_k = A p_k;  seven sums gamma, a, b, c, d, e, f;  alpha_k = d/a;
    convergence test on gamma - 2 alpha b + alpha^2 c (Eq. 8, the expansion of
    ||r_{k+1}||^2); beta_k = (d - 2 alpha e + alpha^2 f)/d (Eq. 7).
    On exit the solution is finalised according to the parity of k.
    """
    x = b * 0 if x0 is None else x0.copy()
    r = b - apply_A(x) if x0 is not None else b.copy()
    eps_sq = rtol * rtol * _dot(b, b)
    hist, alphas, betas = [], [], []
    if _dot(r, r) == 0:
        return CGResult(x, 0, True, hist, alphas, betas)
    zero = b * 0
    p = zero.copy()
    v = zero.copy()
    alpha = {0: 0 * eps_sq, -1: 0 * eps_sq}
    beta = {0: 0 * eps_sq, -1: 0 * eps_sq}
    k = 0
    converged = False
    while k < maxit:
        k += 1
        if k > 1 and k % 2 == 1:
            x = x + alpha[k - 1] * p + (alpha[k - 2] / beta[k - 2]) * (p - inv_diag * r)
        r = r - alpha[k - 1] * v
        p = inv_diag * r + beta[k - 1] * p
        v = apply_A(p)
        g_ = _dot(r, r)
        a_ = _dot(p, v)
        b_ = _dot(r, v)
        c_ = _dot(v, v)
        d_ = _dot(r, inv_diag * r)
        e_ = _dot(r, inv_diag * v)
        f_ = _dot(v, inv_diag * v)
        alpha[k] = d_ / a_
        alphas.append(alpha[k])
        gamma_next = g_ - 2 * alpha[k] * b_ + alpha[k] * alpha[k] * c_
        hist.append(gamma_next)
        if gamma_next < eps_sq:
            converged = True
            break
        beta[k] = (d_ - 2 * alpha[k] * e_ + alpha[k] * alpha[k] * f_) / d_
        betas.append(beta[k])
    # finalise x_{k+1} from the stored iterate (x_k for odd k, x_{k-1} for even k)
    if k >= 1:
        if k % 2 == 1:
            x = x + alpha[k] * p
        else:
            x = x + alpha[k] * p + (alpha[k - 1] / beta[k - 1]) * (p - inv_diag * r)
    return CGResult(x, k, converged, hist, alphas, betas)
