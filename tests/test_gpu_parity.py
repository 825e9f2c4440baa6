"""GPU parity of the CUDA path against the CPU oracle, through the C ABI.

Tolerances (stated by the workload definition): operator application in FP64
max_i |d_i| / max_i |ref_i| <= 1e-13; converged solution at rtol 1e-10 within
1e-9 (max norm, relative) of the oracle's Algorithm 1 and iteration counts
within +-1.
"""
import numpy as np
import pytest
import torch

from oracle import cg as ocg
from oracle import fastdiag, fem
from paper_2205_08909_gb300 import inputs

pytestmark = pytest.mark.gpu

OP_TOL = 1e-13
SOL_TOL = 1e-9


@pytest.fixture(scope="module")
def mfcg():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2205_08909_gb300 import build

    build.build()
    import paper_2205_08909_gb300 as m

    return m


def _oracle_problem(p, cells, amp=0.0, coef="constant"):
    return fem.Problem(p, tuple(cells), amp, fem.COEF_SIN_X if coef == "sin_x" else fem.COEF_CONSTANT)


def _gpu_problem(mfcg, p, cells, amp=0.0, coef="constant", geometry=None, **kw):
    if geometry is None:
        geometry = "deformed" if (amp != 0.0 or coef != "constant") else "affine"
    return mfcg.Problem(p, cells, amplitude=amp, geometry=geometry, coefficient=coef, **kw)


def _to_dev(prob, lex):
    return prob.from_lexicographic(torch.from_numpy(np.ascontiguousarray(lex)).cuda())


def _to_host(prob, v):
    return prob.to_lexicographic(v).cpu().numpy()


def _rel(a, ref):
    return np.abs(a - ref).max() / max(np.abs(ref).max(), 1e-300)


OPERATOR_CASES = [
    (2, (8, 8, 8), 0.0, "constant", None),
    (4, (9, 5, 6), 0.0, "constant", None),
    (1, (7, 6, 5), 0.0, "constant", (2, 3, 2)),
    (3, (5, 4, 7), 0.0, "constant", (2, 2, 3)),
    (5, (3, 4, 3), 0.0, "constant", None),
    (6, (4, 3, 3), 0.0, "constant", None),
    (7, (2, 3, 2), 0.0, "constant", (1, 2, 1)),
    (8, (2, 2, 3), 0.0, "constant", (1, 1, 2)),
    (2, (1, 1, 1), 0.0, "constant", None),
    (3, (1, 2, 1), 0.0, "constant", None),
    (2, (5, 4, 6), 0.05, "sin_x", None),
    (4, (3, 4, 3), 0.08, "constant", None),
    (6, (3, 3, 2), 0.05, "sin_x", None),
    (3, (4, 3, 5), 0.0, "sin_x", (2, 2, 2)),
]


@pytest.mark.parametrize("precision", ["fp64", "double_float"])
@pytest.mark.parametrize("p,cells,amp,coef,tile", OPERATOR_CASES)
def test_operator_diagonal_rhs_match_oracle(mfcg, p, cells, amp, coef, tile, precision):
    op = _oracle_problem(p, cells, amp, coef)
    A = fem.assemble(op)
    prob = _gpu_problem(mfcg, p, cells, amp, coef, tile=tile, precision=precision)
    assert prob.n_dofs == op.n_dofs
    u = inputs.random_vector(op.n_dofs, salt=p)
    got = _to_host(prob, prob.apply_operator(_to_dev(prob, u)))
    assert _rel(got, A @ u) <= OP_TOL
    assert _rel(_to_host(prob, prob.diagonal()), A.diagonal()) <= OP_TOL
    assert _rel(_to_host(prob, prob.rhs()), fem.rhs(op)) <= 1e-12
    prob.close()


DEFORMED_OPERATOR_CASES = [c for c in OPERATOR_CASES if c[2] != 0.0 or c[3] != "constant"]


@pytest.mark.parametrize("precision", ["fp64", "double_float"])
@pytest.mark.parametrize("p,cells,amp,coef,tile", DEFORMED_OPERATOR_CASES)
def test_final_tensor_geometry_matches_oracle(mfcg, p, cells, amp, coef, tile, precision):
    # Sec. 2.2 "final tensor" storage: the same operator as the inverse-Jacobian
    # storage, from 6 instead of 10 values per quadrature point
    op = _oracle_problem(p, cells, amp, coef)
    A = fem.assemble(op)
    prob = _gpu_problem(mfcg, p, cells, amp, coef, geometry="deformed_tensor", tile=tile, precision=precision)
    u = inputs.random_vector(op.n_dofs, salt=p)
    got = _to_host(prob, prob.apply_operator(_to_dev(prob, u)))
    assert _rel(got, A @ u) <= OP_TOL
    assert _rel(_to_host(prob, prob.diagonal()), A.diagonal()) <= OP_TOL
    assert _rel(_to_host(prob, prob.rhs()), fem.rhs(op)) <= 1e-12
    prob.close()


def test_reordering_is_a_permutation(mfcg):
    prob = mfcg.Problem(3, (5, 4, 3), tile=(2, 3, 2))
    lex = torch.arange(prob.n_dofs, dtype=torch.float64, device="cuda")
    blk = prob.from_lexicographic(lex)
    assert torch.equal(torch.sort(blk).values, lex)
    assert torch.equal(prob.to_lexicographic(blk), lex)
    prob.close()


CG_CASES = [
    (2, (8, 8, 8), 0.0, "constant"),
    (4, (5, 6, 4), 0.0, "constant"),
    (3, (3, 4, 3), 0.05, "sin_x"),
    (6, (2, 3, 2), 0.05, "sin_x"),
]


SOLVER_VARIANTS = [("fused", "fp64"), ("unfused", "fp64"), ("fused", "double_float"), ("unfused", "double_float"),
                   ("fused", "fp32_inner"), ("semi_fused", "fp64"), ("semi_fused", "double_float"),
                   ("loop_fused", "fp64"), ("loop_fused", "double_float"), ("fused", "double_float_inner")]
FIXED_VARIANTS = [v for v in SOLVER_VARIANTS if not v[1].endswith("_inner")]


@pytest.mark.parametrize("mode,precision", SOLVER_VARIANTS)
@pytest.mark.parametrize("p,cells,amp,coef", CG_CASES)
def test_cg_solution_matches_oracle(mfcg, mode, precision, p, cells, amp, coef):
    op = _oracle_problem(p, cells, amp, coef)
    A = fem.assemble(op)
    b = fem.rhs(op)
    ref = ocg.pcg_algorithm1(lambda v: A @ v, b, 1.0 / A.diagonal(), 1e-10, 5000)
    prob = _gpu_problem(mfcg, p, cells, amp, coef, mode=mode, precision=precision)
    x, info = prob.cg_solve(_to_dev(prob, b), rtol=1e-10, maxit=5000)
    assert info["converged"] == 1
    if not precision.endswith("_inner"):
        assert abs(info["iterations"] - ref.iterations) <= 1
    else:
        # defect correction: the true FP64 residual meets the tolerance
        xh = _to_host(prob, x)
        assert np.linalg.norm(b - A @ xh) < 1e-10 * np.linalg.norm(b)
        assert info["outer_cycles"] >= 1
    assert _rel(_to_host(prob, x), ref.x) <= SOL_TOL
    prob.close()


@pytest.mark.parametrize("mode,precision", [("fused", "fp64"), ("unfused", "fp64"), ("fused", "double_float"),
                                            ("fused", "fp32_inner"), ("fused", "double_float_inner")])
@pytest.mark.parametrize("p,cells,amp,coef", [c for c in CG_CASES if c[2] != 0.0])
def test_cg_with_final_tensor_geometry_matches_oracle(mfcg, mode, precision, p, cells, amp, coef):
    op = _oracle_problem(p, cells, amp, coef)
    A = fem.assemble(op)
    b = fem.rhs(op)
    ref = ocg.pcg_algorithm1(lambda v: A @ v, b, 1.0 / A.diagonal(), 1e-10, 5000)
    prob = _gpu_problem(mfcg, p, cells, amp, coef, geometry="deformed_tensor", mode=mode, precision=precision)
    x, info = prob.cg_solve(_to_dev(prob, b), rtol=1e-10, maxit=5000)
    assert info["converged"] == 1
    if not precision.endswith("_inner"):
        assert abs(info["iterations"] - ref.iterations) <= 1
    assert _rel(_to_host(prob, x), ref.x) <= SOL_TOL
    prob.close()


@pytest.mark.parametrize("mode,precision", FIXED_VARIANTS)
@pytest.mark.parametrize("maxit", [1, 2, 3, 6, 7])
def test_fixed_iterations_match_algorithm1_iterates(mfcg, mode, precision, maxit):
    # rtol = 0 runs exactly maxit iterations: checks the delayed x update and
    # the parity-dependent finalisation of Algorithm 5 for odd and even counts
    p, cells = 3, (4, 3, 5)
    op = _oracle_problem(p, cells)
    A = fem.assemble(op)
    b = inputs.boundary_zeroed(inputs.random_vector(op.n_dofs, salt=7), op.nodes_per_dim)
    ref = ocg.pcg_algorithm1(lambda v: A @ v, b, 1.0 / A.diagonal(), 0.0, maxit)
    prob = _gpu_problem(mfcg, p, cells, mode=mode, precision=precision)
    x, info = prob.cg_solve(_to_dev(prob, b), rtol=0.0, maxit=maxit)
    assert info["iterations"] == maxit
    assert _rel(_to_host(prob, x), ref.x) <= 1e-11
    prob.close()


@pytest.mark.parametrize("mode,precision", FIXED_VARIANTS)
@pytest.mark.parametrize("p,cells,amp,coef", [(2, (6, 5, 7), 0.0, "constant"), (3, (3, 4, 3), 0.05, "sin_x")])
def test_no_preconditioner_is_merged_cg_of_algorithm4(mfcg, mode, precision, p, cells, amp, coef):
    # M = I: Algorithm 5 reduces to Algorithm 4; the oracle is Algorithm 1 with M = I
    op = _oracle_problem(p, cells, amp, coef)
    A = fem.assemble(op)
    b = fem.rhs(op)
    ref = ocg.pcg_algorithm1(lambda v: A @ v, b, np.ones(op.n_dofs), 1e-10, 5000)
    prob = _gpu_problem(mfcg, p, cells, amp, coef, mode=mode, precision=precision, preconditioner="none")
    x, info = prob.cg_solve(_to_dev(prob, b), rtol=1e-10, maxit=5000)
    assert info["converged"] == 1
    assert abs(info["iterations"] - ref.iterations) <= 1
    assert _rel(_to_host(prob, x), ref.x) <= SOL_TOL
    # the diagonal entry point still returns diag(A)
    assert _rel(_to_host(prob, prob.diagonal()), A.diagonal()) <= OP_TOL
    prob.close()


def test_initial_guess_and_host_arrays(mfcg):
    p, cells = 4, (3, 4, 3)
    op = _oracle_problem(p, cells)
    A = fem.assemble(op)
    b = fem.rhs(op)
    ref = ocg.pcg_algorithm1(lambda v: A @ v, b, 1.0 / A.diagonal(), 1e-10, 5000)
    prob = mfcg.Problem(p, cells)
    x0 = inputs.boundary_zeroed(inputs.random_vector(op.n_dofs, salt=3), op.nodes_per_dim)
    x, info = prob.cg_solve(_to_dev(prob, b), _to_dev(prob, x0), rtol=1e-12, maxit=5000)
    assert info["converged"]
    assert _rel(_to_host(prob, x), ref.x) <= SOL_TOL
    # the same solve through host arrays gives bitwise the same result
    bd = _to_dev(prob, b)
    xd, _ = prob.cg_solve(bd, rtol=1e-10)
    bh = bd.cpu().pin_memory()
    xh = torch.zeros(prob.n_dofs, dtype=torch.float64).pin_memory()
    xh, info_h = prob.cg_solve_host(bh, xh, rtol=1e-10)
    assert torch.equal(xh, xd.cpu())
    prob.close()


@pytest.mark.parametrize("precision", ["fp64", "double_float"])
@pytest.mark.parametrize("p,cells,rtol,maxit", [(4, (6, 5, 4), 1e-10, 2000), (2, (9, 7, 8), 0.0, 13),
                                                (3, (4, 3, 5), 0.0, 1)])
def test_loop_fused_gives_the_unfused_iterates(mfcg, precision, p, cells, rtol, maxit):
    # loop fusion changes neither a product nor the reduction order of
    # Algorithm 1: both forms stop at the same iteration with identical x
    nn = tuple(p * c + 1 for c in cells)
    out = {}
    for mode in ("unfused", "loop_fused"):
        prob = mfcg.Problem(p, cells, mode=mode, precision=precision)
        b = _to_dev(prob, inputs.boundary_zeroed(inputs.random_vector(prob.n_dofs, salt=23), nn))
        x, info = prob.cg_solve(b, rtol=rtol, maxit=maxit)
        out[mode] = (x.cpu(), info)
        prob.close()
    (xu, iu), (xl, il) = out["unfused"], out["loop_fused"]
    assert il["iterations"] == iu["iterations"]
    assert il["converged"] == iu["converged"]
    assert il["residual_sq_est"] == iu["residual_sq_est"]
    assert torch.equal(xl, xu)


@pytest.mark.parametrize("mode,precision", SOLVER_VARIANTS)
def test_solve_is_deterministic(mfcg, mode, precision):
    prob = mfcg.Problem(4, (6, 5, 4), mode=mode, precision=precision)
    b = _to_dev(prob, inputs.boundary_zeroed(inputs.random_vector(prob.n_dofs, salt=11),
                                             (4 * 6 + 1, 4 * 5 + 1, 4 * 4 + 1)))
    x1, i1 = prob.cg_solve(b, rtol=1e-10)
    x2, i2 = prob.cg_solve(b, rtol=1e-10)
    assert i1["iterations"] == i2["iterations"]
    assert torch.equal(x1, x2)
    prob.close()


def test_degenerate_inputs(mfcg):
    prob = mfcg.Problem(2, (3, 3, 3))
    zero = torch.zeros(prob.n_dofs, dtype=torch.float64, device="cuda")
    x, info = prob.cg_solve(zero, rtol=1e-10)
    assert info["iterations"] == 0 and info["converged"] == 1 and torch.count_nonzero(x) == 0
    b = prob.rhs()
    with pytest.raises(mfcg.MfcgError) as err:
        prob.cg_solve(b, rtol=1e-14, maxit=2)
    assert err.value.status == 5
    bad = b.clone()
    bad[prob.n_dofs // 2] = float("nan")
    with pytest.raises(mfcg.MfcgError) as err:
        prob.cg_solve(bad, rtol=1e-10)
    assert err.value.status == 6
    with pytest.raises(ValueError):
        prob.apply_operator(b.float())
    prob.close()


# ----------------------------------------------------------------- full sizes


@pytest.mark.parametrize("precision", ["fp64", "double_float"])
def test_full_size_q4_64cube_operator_every_entry(mfcg, precision):
    w = inputs.WORKLOADS["q4_64cube"]
    op = _oracle_problem(w.degree, w.cells)
    prob = mfcg.Problem(w.degree, w.cells, precision=precision)
    u = inputs.random_vector(op.n_dofs, salt=64)
    got = _to_host(prob, prob.apply_operator(_to_dev(prob, u)))
    assert _rel(got, fastdiag.apply(op, u)) <= OP_TOL
    prob.close()


@pytest.mark.parametrize("mode,precision", SOLVER_VARIANTS)
def test_full_size_q4_64cube_solve(mfcg, mode, precision):
    w = inputs.WORKLOADS["q4_64cube"]
    op = _oracle_problem(w.degree, w.cells)
    prob = mfcg.Problem(w.degree, w.cells, mode=mode, precision=precision)
    b = prob.rhs()
    x, info = prob.cg_solve(b, rtol=1e-10, maxit=2000)
    assert info["converged"]
    bh = _to_host(prob, b)
    xh = _to_host(prob, x)
    xs = fastdiag.solve(op, bh)
    assert _rel(xh, xs) <= SOL_TOL
    r = bh - fastdiag.apply(op, xh)
    assert np.linalg.norm(r) <= 1.5e-10 * np.linalg.norm(bh)
    prob.close()


@pytest.mark.parametrize("geometry", ["deformed", "deformed_tensor"])
@pytest.mark.parametrize("precision", ["fp64", "double_float"])
def test_full_size_q6_48cube_deformed_operator_sampled_rows(mfcg, precision, geometry):
    w = inputs.WORKLOADS["q6_48cube_deformed"]
    op = _oracle_problem(w.degree, w.cells, w.amplitude, w.coefficient)
    prob = _gpu_problem(mfcg, w.degree, w.cells, w.amplitude, w.coefficient, geometry=geometry,
                        precision=precision)
    u = inputs.random_vector(op.n_dofs, salt=48)
    got = _to_host(prob, prob.apply_operator(_to_dev(prob, u)))
    diag = _to_host(prob, prob.diagonal())
    # rows: random ones plus nodes on tile faces, edges and corners (tiles of 2 cells)
    rng_rows = list(inputs.random_rows(op.n_dofs, 6))
    n1 = w.degree * w.cells[0] + 1
    for (i, j, k) in ((12, 12, 12), (12, 13, 14), (24, 12, 7), (1, 1, 12), (287, 12, 24)):
        rng_rows.append(i + n1 * (j + n1 * k))
    rows = np.array(rng_rows)
    ref = fem.apply_rows(op, u, rows)
    scale = np.abs(got).max()
    assert np.abs(got[rows] - ref).max() <= OP_TOL * scale
    assert np.abs(diag[rows] - fem.diagonal_rows(op, rows)).max() <= OP_TOL * np.abs(diag).max()
    prob.close()


@pytest.mark.parametrize("precision", ["fp64", "double_float"])
def test_full_size_q4_128cube_operator_every_entry(mfcg, precision):
    w = inputs.WORKLOADS["q4_128cube"]
    op = _oracle_problem(w.degree, w.cells)
    prob = mfcg.Problem(w.degree, w.cells, precision=precision)
    u = inputs.random_vector(op.n_dofs, salt=128)
    got = _to_host(prob, prob.apply_operator(_to_dev(prob, u)))
    assert _rel(got, fastdiag.apply(op, u)) <= OP_TOL
    prob.close()


def test_defect_correction_on_deformed_mesh(mfcg):
    # FP32-inner defect correction on a deformed variable-coefficient Q6 mesh
    # reaches the FP64 tolerance on its own FP64-accurate residual and the
    # solution of the fused double-float CG
    w = inputs.Workload("q6_12cube_deformed", 6, (12, 12, 12), 0.05, "sin_x")
    prob = _gpu_problem(mfcg, w.degree, w.cells, w.amplitude, w.coefficient, precision="fp32_inner")
    b = prob.rhs()
    x, info = prob.cg_solve(b, rtol=1e-10, maxit=20000)
    assert info["converged"] and info["residual_sq_est"] < 1e-20 * info["rhs_norm_sq"]
    ref = _gpu_problem(mfcg, w.degree, w.cells, w.amplitude, w.coefficient, precision="double_float")
    xr, info_r = ref.cg_solve(ref.rhs(), rtol=1e-10, maxit=20000)
    assert info_r["converged"]
    assert (x - xr).abs().max().item() <= SOL_TOL * xr.abs().max().item()
    prob.close()
    ref.close()


@pytest.mark.parametrize("precision", ["fp64", "fp32_inner", "double_float", "double_float_inner"])
def test_full_size_q4_128cube_solve(mfcg, precision):
    # the fused FP64 CG, the FP32-inner defect correction and the double-float
    # CG at 135M unknowns against the exact discrete solution by fast
    # diagonalisation
    w = inputs.WORKLOADS["q4_128cube"]
    op = _oracle_problem(w.degree, w.cells)
    prob = mfcg.Problem(w.degree, w.cells, precision=precision)
    b = prob.rhs()
    x, info = prob.cg_solve(b, rtol=1e-10, maxit=20000)
    assert info["converged"]
    if precision == "double_float_inner":
        assert info["outer_cycles"] <= 2
    bh = _to_host(prob, b)
    xh = _to_host(prob, x)
    prob.close()
    xs = fastdiag.solve(op, bh)
    assert _rel(xh, xs) <= SOL_TOL
    r = bh - fastdiag.apply(op, xh)
    # the defect correction meets the tolerance on the true FP64 residual; the
    # double-float recurrence stops at rtol on its own residual, whose true
    # counterpart sits above it by the ~2^-44 rounding of the pair arithmetic
    bound = 5e-10 if precision == "double_float" else 1.5e-10
    assert np.linalg.norm(r) <= bound * np.linalg.norm(bh)


def _q6_48_rows(op, count):
    """Random rows plus nodes on tile faces, edges and corners (tiles of 2
    cells, 12 nodes) and next to the Dirichlet boundary."""
    n1 = op.nodes_per_dim[0]
    rows = list(inputs.random_rows(op.n_dofs, count, salt=7))
    for (i, j, k) in ((12, 12, 12), (12, 13, 14), (24, 12, 7), (1, 1, 12), (287, 12, 24), (1, 1, 1),
                      (287, 287, 287), (144, 144, 12), (36, 48, 60), (11, 12, 13), (13, 11, 12)):
        rows.append(i + n1 * (j + n1 * k))
    return np.unique(np.array(rows))


def test_full_size_q6_48cube_deformed_solve(mfcg):
    # Q6 on the deformed 48^3 mesh with the variable coefficient (24.1M
    # unknowns): the fused FP64 CG to rtol 1e-10.  Its true residual is formed
    # with the FP64 operator, whose rows are checked against the oracle's
    # (sampled, >= 200 rows including tile faces, edges and corners); the
    # double-float CG and the FP32-inner defect correction reach the same
    # solution.
    w = inputs.WORKLOADS["q6_48cube_deformed"]
    op = _oracle_problem(w.degree, w.cells, w.amplitude, w.coefficient)
    prob = _gpu_problem(mfcg, w.degree, w.cells, w.amplitude, w.coefficient, true_residual=1)
    b = prob.rhs()
    x, info = prob.cg_solve(b, rtol=1e-10, maxit=20000)
    assert info["converged"]
    assert info["true_residual_sq"] <= (1.5e-10) ** 2 * info["rhs_norm_sq"]
    ax = _to_host(prob, prob.apply_operator(x))
    xh = _to_host(prob, x)
    bh = _to_host(prob, b)
    rows = _q6_48_rows(op, 220)
    assert len(rows) >= 200
    ref = fem.apply_rows(op, xh, rows)
    # A x ~ b is a sum of much larger terms of both signs: the operator's
    # rounding is measured against the size of the terms (diagonal x max |x|)
    term = np.abs(fem.diagonal_rows(op, rows)).max() * np.abs(xh).max()
    assert np.abs(ax[rows] - ref).max() <= OP_TOL * term
    # the sampled rows of the residual stay within the norm bound
    assert np.abs(bh[rows] - ref).max() <= 1.5e-10 * np.linalg.norm(bh)
    prob.close()
    for precision in ("double_float", "fp32_inner", "double_float_inner"):
        other = _gpu_problem(mfcg, w.degree, w.cells, w.amplitude, w.coefficient, precision=precision)
        xo, info_o = other.cg_solve(other.rhs(), rtol=1e-10, maxit=20000)
        assert info_o["converged"]
        assert _rel(_to_host(other, xo), xh) <= SOL_TOL
        other.close()


RANDOM_RHS_CASES = [
    (2, (6, 5, 7), 0.0, "constant"),
    (4, (4, 5, 3), 0.0, "constant"),
    (3, (3, 4, 3), 0.05, "sin_x"),
    (5, (2, 3, 2), 0.08, "constant"),
]


@pytest.mark.parametrize("mode,precision", SOLVER_VARIANTS)
@pytest.mark.parametrize("p,cells,amp,coef", RANDOM_RHS_CASES)
def test_random_rhs_solve_matches_algorithm1(mfcg, mode, precision, p, cells, amp, coef):
    # a standard-normal right-hand side (zero on the boundary) excites every
    # mode, so the solve takes many iterations and exercises the recurrences
    # of Algorithm 5 (Eqs. 7-8) throughout; iterates are compared with
    # Algorithm 1's after the same number of products A p
    op = _oracle_problem(p, cells, amp, coef)
    A = fem.assemble(op)
    b = inputs.boundary_zeroed(inputs.random_vector(op.n_dofs, salt=17 + p), op.nodes_per_dim)
    dinv = 1.0 / A.diagonal()
    ref = ocg.pcg_algorithm1(lambda v: A @ v, b, dinv, 1e-10, 5000)
    assert ref.converged and ref.iterations >= 20
    prob = _gpu_problem(mfcg, p, cells, amp, coef, mode=mode, precision=precision)
    x, info = prob.cg_solve(_to_dev(prob, b), rtol=1e-10, maxit=5000)
    assert info["converged"] == 1
    xh = _to_host(prob, x)
    if precision.endswith("_inner"):
        assert np.linalg.norm(b - A @ xh) < 1e-10 * np.linalg.norm(b)
        assert _rel(xh, ref.x) <= SOL_TOL
    else:
        assert abs(info["iterations"] - ref.iterations) <= 1
        same = ocg.pcg_algorithm1(lambda v: A @ v, b, dinv, 0.0, info["iterations"])
        assert _rel(xh, same.x) <= SOL_TOL
    prob.close()


BATCH_SPECS = [
    {"degree": 2, "cells": (8, 8, 8)},
    {"degree": 3, "cells": (3, 4, 3), "amplitude": 0.05, "coefficient": "sin_x"},
    {"degree": 6, "cells": (2, 3, 2), "amplitude": 0.05, "coefficient": "sin_x", "geometry": "deformed_tensor"},
    {"degree": 4, "cells": (5, 6, 4)},
    {"degree": 1, "cells": (7, 6, 5)},
    {"degree": 8, "cells": (2, 2, 3)},
]


@pytest.mark.parametrize("precision", ["fp64", "double_float"])
def test_batch_solve_matches_oracle_and_single_solves(mfcg, precision):
    # members converge at different iteration counts; each matches the
    # oracle's Algorithm 1 and is bitwise equal to its solve as a single problem
    batch = mfcg.Batch(BATCH_SPECS, precision=precision)
    bs, refs = [], []
    for sp, m in zip(BATCH_SPECS, batch.members):
        op = _oracle_problem(sp["degree"], sp["cells"], sp.get("amplitude", 0.0), sp.get("coefficient", "constant"))
        A = fem.assemble(op)
        b = inputs.boundary_zeroed(inputs.random_vector(op.n_dofs, salt=sp["degree"]), op.nodes_per_dim)
        refs.append(ocg.pcg_algorithm1(lambda v, A=A: A @ v, b, 1.0 / A.diagonal(), 1e-10, 5000))
        bs.append(_to_dev(m, b))
    xs, infos = batch.cg_solve(bs, rtol=1e-10, maxit=5000)
    assert len({i["iterations"] for i in infos}) > 1
    for sp, m, x, info, ref, b in zip(BATCH_SPECS, batch.members, xs, infos, refs, bs):
        assert info["converged"] == 1
        assert abs(info["iterations"] - ref.iterations) <= 1
        assert _rel(_to_host(m, x), ref.x) <= SOL_TOL
        single = _gpu_problem(mfcg, sp["degree"], sp["cells"], sp.get("amplitude", 0.0),
                              sp.get("coefficient", "constant"), geometry=sp.get("geometry"), precision=precision)
        xs1, info1 = single.cg_solve(b, rtol=1e-10, maxit=5000)
        assert info1["iterations"] == info["iterations"]
        assert torch.equal(xs1, x)
        single.close()
    # fixed iterations: every member runs exactly maxit
    xs, infos = batch.cg_solve(bs, rtol=0.0, maxit=7)
    assert all(i["iterations"] == 7 for i in infos)
    batch.close()


def test_batch_of_generated_problems(mfcg):
    # the seeded batch generator at small sizes: every member reaches rtol
    specs = inputs.batch_problems(12, max_cells=6)
    batch = mfcg.Batch(specs, precision="double_float")
    rhs = inputs.batch_rhs(specs)
    bs = [_to_dev(m, r) for m, r in zip(batch.members, rhs)]
    xs, infos = batch.cg_solve(bs, rtol=1e-8, maxit=20000)
    for m, x, b, info in zip(batch.members, xs, bs, infos):
        assert info["converged"] == 1
        r = b - m.apply_operator(x)
        assert r.norm().item() <= 2e-8 * b.norm().item()
    batch.close()


def test_autotuned_tile_solves_like_the_oracle(mfcg):
    # tile = (-1, -1, -1): setup times candidate tiles and keeps one; the
    # solution does not depend on the choice
    op = _oracle_problem(4, (6, 5, 7))
    A = fem.assemble(op)
    b = fem.rhs(op)
    ref = ocg.pcg_algorithm1(lambda v: A @ v, b, 1.0 / A.diagonal(), 1e-10, 5000)
    prob = mfcg.Problem(4, (6, 5, 7), tile=(-1, -1, -1), precision="double_float")
    x, info = prob.cg_solve(_to_dev(prob, b), rtol=1e-10, maxit=5000)
    assert info["converged"] == 1 and abs(info["iterations"] - ref.iterations) <= 1
    assert _rel(_to_host(prob, x), ref.x) <= SOL_TOL
    prob.close()


VECTOR_CASES = [
    (2, (8, 8, 8), 0.0, "constant", None),
    (4, (5, 6, 4), 0.0, "constant", None),
    (3, (3, 4, 3), 0.05, "sin_x", "deformed"),
    (6, (2, 3, 2), 0.05, "sin_x", "deformed_tensor"),
]


@pytest.mark.parametrize("precision", ["fp64", "double_float", "fp32_inner"])
@pytest.mark.parametrize("p,cells,amp,coef,geometry", VECTOR_CASES)
def test_vector_valued_operator_and_solve(mfcg, p, cells, amp, coef, geometry, precision):
    # three components, each the scalar operator (the BP4 form): operator,
    # shared diagonal and right-hand side per component, and one CG on the
    # coupled block-diagonal system against the oracle's Algorithm 1 on it
    import scipy.sparse as sp

    op = _oracle_problem(p, cells, amp, coef)
    A = fem.assemble(op)
    n = op.n_dofs
    prob = _gpu_problem(mfcg, p, cells, amp, coef, geometry=geometry, precision=precision, components=3)
    assert prob.n_dofs == 3 * n
    u = np.concatenate([inputs.random_vector(n, salt=10 + c) for c in range(3)])
    got = _to_host(prob, prob.apply_operator(_to_dev(prob, u)))
    for c in range(3):
        assert _rel(got[c * n:(c + 1) * n], A @ u[c * n:(c + 1) * n]) <= OP_TOL
    assert _rel(_to_host(prob, prob.diagonal()), np.tile(A.diagonal(), 3)) <= OP_TOL
    b1 = fem.rhs(op)
    b = np.concatenate([(c + 1) * b1 for c in range(3)])
    assert _rel(_to_host(prob, prob.rhs()), b) <= 1e-12
    A3 = sp.block_diag([A, A, A], format="csr")
    ref = ocg.pcg_algorithm1(lambda v: A3 @ v, b, 1.0 / A3.diagonal(), 1e-10, 5000)
    x, info = prob.cg_solve(_to_dev(prob, b), rtol=1e-10, maxit=5000)
    assert info["converged"] == 1
    if not precision.endswith("_inner"):
        assert abs(info["iterations"] - ref.iterations) <= 1
    else:
        xh = _to_host(prob, x)
        assert np.linalg.norm(b - A3 @ xh) < 1e-10 * np.linalg.norm(b)
    assert _rel(_to_host(prob, x), ref.x) <= SOL_TOL
    prob.close()


MASS_CASES = [
    (2, (8, 8, 8), 0.0, "constant", None),
    (5, (3, 4, 3), 0.0, "constant", (2, 2, 3)),
    (3, (3, 4, 3), 0.05, "sin_x", None),
    (6, (2, 3, 2), 0.08, "constant", None),
]


@pytest.mark.parametrize("precision", ["fp64", "double_float", "fp32_inner"])
@pytest.mark.parametrize("p,cells,amp,coef,tile", MASS_CASES)
def test_mass_operator_matches_oracle(mfcg, p, cells, amp, coef, tile, precision):
    # the mass operator (BP1): operator, diagonal and right-hand side, and the
    # Jacobi-CG solution of M x = b, against the oracle's mass matrix
    op = fem.Problem(p, tuple(cells), amp, fem.COEF_SIN_X if coef == "sin_x" else fem.COEF_CONSTANT,
                     op=fem.OP_MASS)
    A = fem.assemble(op)
    prob = _gpu_problem(mfcg, p, cells, amp, coef, tile=tile, precision=precision, operator="mass")
    u = inputs.random_vector(op.n_dofs, salt=p)
    got = _to_host(prob, prob.apply_operator(_to_dev(prob, u)))
    assert _rel(got, A @ u) <= OP_TOL
    assert _rel(_to_host(prob, prob.diagonal()), A.diagonal()) <= OP_TOL
    b = fem.rhs(op)
    assert _rel(_to_host(prob, prob.rhs()), b) <= 1e-12
    ref = ocg.pcg_algorithm1(lambda v: A @ v, b, 1.0 / A.diagonal(), 1e-10, 5000)
    x, info = prob.cg_solve(_to_dev(prob, b), rtol=1e-10, maxit=5000)
    assert info["converged"] == 1
    if not precision.endswith("_inner"):
        assert abs(info["iterations"] - ref.iterations) <= 1
    assert _rel(_to_host(prob, x), ref.x) <= SOL_TOL
    prob.close()


def test_vector_valued_mass_operator(mfcg):
    # BP2: three components of the mass operator in one CG
    import scipy.sparse as sp

    op = fem.Problem(4, (4, 3, 5), op=fem.OP_MASS)
    A = fem.assemble(op)
    prob = mfcg.Problem(4, (4, 3, 5), operator="mass", components=3, precision="double_float")
    b1 = fem.rhs(op)
    b = np.concatenate([(c + 1) * b1 for c in range(3)])
    assert _rel(_to_host(prob, prob.rhs()), b) <= 1e-12
    A3 = sp.block_diag([A, A, A], format="csr")
    ref = ocg.pcg_algorithm1(lambda v: A3 @ v, b, 1.0 / A3.diagonal(), 1e-10, 5000)
    x, info = prob.cg_solve(_to_dev(prob, b), rtol=1e-10, maxit=5000)
    assert info["converged"] == 1 and abs(info["iterations"] - ref.iterations) <= 1
    assert _rel(_to_host(prob, x), ref.x) <= SOL_TOL
    prob.close()


def test_mass_operator_rejects_final_tensor_storage(mfcg):
    with pytest.raises(mfcg.MfcgError):
        mfcg.Problem(3, (2, 2, 2), amplitude=0.05, geometry="deformed_tensor", operator="mass")


def test_batch_of_right_hand_sides_shares_operator_data(mfcg):
    # identical members (one mesh, several right-hand sides) share geometry and
    # diagonal; each solve matches the oracle and its single-problem solve
    spec = {"degree": 3, "cells": (3, 4, 3), "amplitude": 0.05, "coefficient": "sin_x"}
    specs = [spec] * 4
    batch = mfcg.Batch(specs, precision="double_float")
    op = _oracle_problem(3, (3, 4, 3), 0.05, "sin_x")
    A = fem.assemble(op)
    rhs = inputs.batch_rhs(specs)
    bs = [_to_dev(m, r) for m, r in zip(batch.members, rhs)]
    xs, infos = batch.cg_solve(bs, rtol=1e-10, maxit=5000)
    single = _gpu_problem(mfcg, 3, (3, 4, 3), 0.05, "sin_x", precision="double_float")
    for m, b, x, info, r in zip(batch.members, bs, xs, infos, rhs):
        ref = ocg.pcg_algorithm1(lambda v: A @ v, r, 1.0 / A.diagonal(), 1e-10, 5000)
        assert info["converged"] == 1 and abs(info["iterations"] - ref.iterations) <= 1
        assert _rel(_to_host(m, x), ref.x) <= SOL_TOL
        assert _rel(_to_host(m, m.diagonal()), A.diagonal()) <= OP_TOL
        x1, _ = single.cg_solve(b, rtol=1e-10, maxit=5000)
        assert torch.equal(x1, x)
    single.close()
    batch.close()


def _oracle_point_data(op):
    """The oracle's per-point geometry in the layout of MFCG_GEOM_USER:
    cells x (9 entries of J^{-1}, w det J a) x points."""
    x, J, detJ, w = fem.quadrature_geometry(op)
    Jinv = np.linalg.inv(J).reshape(J.shape[0], J.shape[1], 9)            # [e, q, 9]
    jxw = w[None, :] * detJ * fem.coefficient(op, x)                        # [e, q]
    return np.concatenate([Jinv.transpose(0, 2, 1), jxw[:, None, :]], axis=1)  # [e, 10, q]


@pytest.mark.parametrize("precision", ["fp64", "double_float"])
@pytest.mark.parametrize("p,cells,amp,coef", [(3, (3, 4, 3), 0.05, "sin_x"), (5, (2, 3, 2), 0.08, "constant"),
                                              (2, (4, 3, 5), 0.0, "constant")])
def test_user_point_data_geometry(mfcg, p, cells, amp, coef, precision):
    # the operator on per-point data supplied by the caller (here: the oracle's
    # own Jacobians and weights) equals the oracle's assembled matrix
    op = _oracle_problem(p, cells, amp, coef)
    A = fem.assemble(op)
    prob = mfcg.Problem(p, cells, geometry="user", user_data=_oracle_point_data(op), precision=precision)
    u = inputs.random_vector(op.n_dofs, salt=p)
    assert _rel(_to_host(prob, prob.apply_operator(_to_dev(prob, u))), A @ u) <= OP_TOL
    assert _rel(_to_host(prob, prob.diagonal()), A.diagonal()) <= OP_TOL
    b = fem.rhs(op)
    ref = ocg.pcg_algorithm1(lambda v: A @ v, b, 1.0 / A.diagonal(), 1e-10, 5000)
    x, info = prob.cg_solve(_to_dev(prob, b), rtol=1e-10, maxit=5000)
    assert info["converged"] == 1 and abs(info["iterations"] - ref.iterations) <= 1
    assert _rel(_to_host(prob, x), ref.x) <= SOL_TOL
    with pytest.raises(mfcg.MfcgError):
        prob.rhs()
    prob.close()


@pytest.mark.parametrize("mode,precision", [("fused", "fp64"), ("fused", "double_float"), ("semi_fused", "fp64"),
                                            ("fused", "fp32_inner")])
@pytest.mark.parametrize("maxit", [1, 2, 3, 6, 7, 0])
def test_x_update_every_iteration(mfcg, mode, precision, maxit):
    # the plain x update in every iteration gives Algorithm 1's iterates too
    # (maxit 0: run to rtol 1e-10)
    op = _oracle_problem(3, (3, 4, 3), 0.05, "sin_x")
    A = fem.assemble(op)
    b = fem.rhs(op)
    prob = _gpu_problem(mfcg, 3, (3, 4, 3), 0.05, "sin_x", mode=mode, precision=precision, x_every_iteration=True)
    if maxit == 0:
        ref = ocg.pcg_algorithm1(lambda v: A @ v, b, 1.0 / A.diagonal(), 1e-10, 5000)
        x, info = prob.cg_solve(_to_dev(prob, b), rtol=1e-10, maxit=5000)
        assert info["converged"] == 1
        if not precision.endswith("_inner"):
            assert abs(info["iterations"] - ref.iterations) <= 1
        assert _rel(_to_host(prob, x), ref.x) <= SOL_TOL
    elif not precision.endswith("_inner"):
        ref = ocg.pcg_algorithm1(lambda v: A @ v, b, 1.0 / A.diagonal(), 0.0, maxit)
        x, info = prob.cg_solve(_to_dev(prob, b), rtol=0.0, maxit=maxit)
        assert info["iterations"] == maxit
        assert _rel(_to_host(prob, x), ref.x) <= 1e-10
    prob.close()


@pytest.mark.parametrize("precision", ["fp64", "double_float", "fp32_inner"])
def test_true_residual_of_the_solution(mfcg, precision):
    # mfcg_options.true_residual: ||b - A x||^2 of the returned x with the FP64
    # operator, against the oracle's assembled matrix applied to the same x
    op = _oracle_problem(3, (3, 4, 3), 0.05, "sin_x")
    A = fem.assemble(op)
    b = fem.rhs(op)
    prob = _gpu_problem(mfcg, 3, (3, 4, 3), 0.05, "sin_x", precision=precision, true_residual=True)
    x, info = prob.cg_solve(_to_dev(prob, b), rtol=1e-10, maxit=5000)
    r = np.linalg.norm(b - A @ _to_host(prob, x))
    assert info["true_residual_sq"] >= 0.0
    assert abs(np.sqrt(info["true_residual_sq"]) - r) <= 1e-12 * np.linalg.norm(b)
    assert r <= 5e-10 * np.linalg.norm(b)
    prob.close()
    plain = _gpu_problem(mfcg, 3, (3, 4, 3), 0.05, "sin_x", precision=precision)
    _, info = plain.cg_solve(_to_dev(plain, b), rtol=1e-10, maxit=5000)
    assert info["true_residual_sq"] == -1.0
    plain.close()


@pytest.mark.parametrize("mode,precision", [("fused", "fp64"), ("fused", "double_float"), ("semi_fused", "fp64")])
def test_residual_estimate_follows_algorithm1_history(mfcg, mode, precision):
    # the Eq. 8 estimate gamma_{k+1} = gamma - 2 alpha b + alpha^2 c after k
    # iterations equals Algorithm 1's explicit ||r_k||^2 until the last
    # iterations (here far from convergence)
    p, cells = 3, (4, 3, 5)
    op = _oracle_problem(p, cells)
    A = fem.assemble(op)
    b = inputs.boundary_zeroed(inputs.random_vector(op.n_dofs, salt=11), op.nodes_per_dim)
    ref = ocg.pcg_algorithm1(lambda v: A @ v, b, 1.0 / A.diagonal(), 0.0, 12)
    prob = _gpu_problem(mfcg, p, cells, mode=mode, precision=precision)
    bd = _to_dev(prob, b)
    for k in (1, 2, 3, 5, 8, 12):
        _, info = prob.cg_solve(bd, rtol=0.0, maxit=k)
        assert abs(info["residual_sq_est"] - ref.residual_sq_history[k - 1]) <= 1e-9 * ref.residual_sq_history[k - 1]
    prob.close()


# ----------------------------------------------------------------- FP64 contractions: tensor cores / FP64 pipe


AFFINE_OPERATOR_CASES = [c for c in OPERATOR_CASES if c[2] == 0.0 and c[3] == "constant"]


@pytest.mark.parametrize("p,cells,amp,coef,tile", AFFINE_OPERATOR_CASES)
def test_fp64_pipe_sweeps_match_oracle(mfcg, p, cells, amp, coef, tile):
    # the native FP64 whole-brick sweeps (mfcg_options.fp64_contraction = FP64_PIPE)
    op = _oracle_problem(p, cells, amp, coef)
    A = fem.assemble(op)
    u = inputs.random_vector(op.n_dofs, salt=5)
    prob = _gpu_problem(mfcg, p, cells, amp, coef, tile=tile, fp64_contraction="fp64_pipe")
    got = _to_host(prob, prob.apply_operator(_to_dev(prob, u)))
    assert _rel(got, A @ u) <= OP_TOL
    prob.close()


@pytest.mark.parametrize("mode", ["fused", "unfused", "semi_fused", "loop_fused"])
def test_fp64_pipe_solve_matches_oracle(mfcg, mode):
    op = _oracle_problem(4, (5, 6, 4))
    A = fem.assemble(op)
    b = inputs.boundary_zeroed(inputs.random_vector(op.n_dofs, salt=31), op.nodes_per_dim)
    dinv = 1.0 / A.diagonal()
    ref = ocg.pcg_algorithm1(lambda v: A @ v, b, dinv, 1e-10, 5000)
    prob = _gpu_problem(mfcg, 4, (5, 6, 4), mode=mode, fp64_contraction="fp64_pipe")
    x, info = prob.cg_solve(_to_dev(prob, b), rtol=1e-10, maxit=5000)
    assert info["converged"] and abs(info["iterations"] - ref.iterations) <= 1
    same = ocg.pcg_algorithm1(lambda v: A @ v, b, dinv, 0.0, info["iterations"])
    assert _rel(_to_host(prob, x), same.x) <= SOL_TOL
    prob.close()


@pytest.mark.parametrize("p,cells", [(1, (7, 6, 5)), (2, (8, 8, 8)), (3, (5, 4, 7)), (4, (9, 5, 6)), (5, (3, 4, 3)),
                                     (7, (2, 3, 2))])
def test_tensor_core_operator_is_fp64_accurate(mfcg, p, cells):
    # inputs spanning e^-6 .. e^6 in magnitude; the tensor-core operator stays
    # within the FP64 rounding level of the oracle's FP64 CSR product (which is
    # itself about 1e-15 from the exact product of its 1D matrices), and agrees
    # with the FP64 sweeps
    op = _oracle_problem(p, cells)
    A = fem.assemble(op)
    rng = np.random.default_rng(700 + p)
    u = rng.standard_normal(op.n_dofs) * np.exp(rng.uniform(-6, 6, op.n_dofs))
    ref = A @ u
    tc = _gpu_problem(mfcg, p, cells)
    pipe = _gpu_problem(mfcg, p, cells, fp64_contraction="fp64_pipe")
    got = _to_host(tc, tc.apply_operator(_to_dev(tc, u)))
    got_pipe = _to_host(pipe, pipe.apply_operator(_to_dev(pipe, u)))
    assert _rel(got, ref) <= (5e-15 if p <= 4 else 2e-14)
    assert _rel(got, got_pipe) <= (5e-15 if p <= 4 else 2e-14)
    # Dirichlet rows are the identity, bit for bit
    bnd = fem.boundary_mask(op)
    assert np.array_equal(got[bnd], u[bnd])
    tc.close()
    pipe.close()


def test_tensor_core_operator_vector_and_mass(mfcg):
    # the tensor-core contractions serve the mass operator and the
    # vector-valued form on Cartesian meshes too
    for operator, comps in (("mass", 1), ("laplace", 3), ("mass", 3)):
        op = fem.Problem(3, (4, 3, 5), 0.0, fem.COEF_CONSTANT, fem.OP_MASS if operator == "mass" else fem.OP_LAPLACE)
        A = fem.assemble(op)
        n = op.n_dofs
        u = inputs.random_vector(n * comps, salt=77)
        tc = _gpu_problem(mfcg, 3, (4, 3, 5), operator=operator, components=comps)
        got = _to_host(tc, tc.apply_operator(_to_dev(tc, u)))
        ref = np.concatenate([A @ u[c * n:(c + 1) * n] for c in range(comps)])
        assert _rel(got, ref) <= OP_TOL
        tc.close()


# ---------------------------------------------------------------- tri-quadratic geometry (Sec. 2.2)

QUAD_CASES = [
    (1, (5, 4, 6), 0.06, "constant", None),
    (2, (5, 4, 6), 0.05, "sin_x", None),
    (3, (4, 3, 5), 0.08, "sin_x", (2, 2, 2)),
    (4, (3, 4, 3), 0.08, "constant", None),
    (5, (3, 2, 3), 0.05, "sin_x", None),
    (6, (3, 3, 2), 0.05, "sin_x", None),
    (7, (2, 3, 2), 0.07, "sin_x", (1, 2, 1)),
    (8, (2, 2, 3), 0.05, "constant", (1, 1, 2)),
    (3, (4, 3, 5), 0.0, "constant", None),
]


def _quad_oracle(p, cells, amp, coef, op=fem.OP_LAPLACE):
    return fem.Problem(p, tuple(cells), amp, fem.COEF_SIN_X if coef == "sin_x" else fem.COEF_CONSTANT, op,
                       geometry_degree=2)


@pytest.mark.parametrize("precision", ["fp64", "double_float"])
@pytest.mark.parametrize("p,cells,amp,coef,tile", QUAD_CASES)
def test_quadratic_geometry_operator_matches_oracle(mfcg, p, cells, amp, coef, tile, precision):
    # the metric computed at each point from 27 x 3 coordinates per cell
    op = _quad_oracle(p, cells, amp, coef)
    A = fem.assemble(op)
    prob = _gpu_problem(mfcg, p, cells, amp, coef, geometry="deformed_quadratic", tile=tile, precision=precision)
    u = inputs.random_vector(op.n_dofs, salt=p + 40)
    got = _to_host(prob, prob.apply_operator(_to_dev(prob, u)))
    assert _rel(got, A @ u) <= (OP_TOL if precision == "fp64" else 1e-12)
    assert _rel(_to_host(prob, prob.diagonal()), A.diagonal()) <= OP_TOL
    assert _rel(_to_host(prob, prob.rhs()), fem.rhs(op)) <= 1e-12
    prob.close()


@pytest.mark.parametrize("p,cells,amp,coef", [(2, (5, 4, 6), 0.05, "sin_x"), (5, (3, 2, 3), 0.08, "constant")])
def test_quadratic_geometry_mass_operator(mfcg, p, cells, amp, coef):
    op = _quad_oracle(p, cells, amp, coef, fem.OP_MASS)
    A = fem.assemble(op)
    prob = _gpu_problem(mfcg, p, cells, amp, coef, geometry="deformed_quadratic", operator="mass")
    u = inputs.random_vector(op.n_dofs, salt=p + 50)
    assert _rel(_to_host(prob, prob.apply_operator(_to_dev(prob, u))), A @ u) <= OP_TOL
    assert _rel(_to_host(prob, prob.diagonal()), A.diagonal()) <= OP_TOL
    assert _rel(_to_host(prob, prob.rhs()), fem.rhs(op)) <= 1e-12
    prob.close()


@pytest.mark.parametrize("mode,precision", [("fused", "fp64"), ("unfused", "fp64"), ("loop_fused", "fp64"),
                                            ("fused", "double_float"), ("fused", "fp32_inner"),
                                            ("fused", "double_float_inner")])
@pytest.mark.parametrize("p,cells,amp,coef", [(3, (4, 3, 5), 0.05, "sin_x"), (6, (2, 3, 2), 0.08, "sin_x")])
def test_quadratic_geometry_solve_matches_oracle(mfcg, mode, precision, p, cells, amp, coef):
    op = _quad_oracle(p, cells, amp, coef)
    A = fem.assemble(op)
    b = fem.rhs(op)
    ref = ocg.pcg_algorithm1(lambda v: A @ v, b, 1.0 / A.diagonal(), 1e-10, 5000)
    prob = _gpu_problem(mfcg, p, cells, amp, coef, geometry="deformed_quadratic", mode=mode, precision=precision)
    x, info = prob.cg_solve(_to_dev(prob, b), rtol=1e-10, maxit=5000)
    assert info["converged"] == 1
    xh = _to_host(prob, x)
    if precision.endswith("_inner"):
        assert np.linalg.norm(b - A @ xh) < 1e-10 * np.linalg.norm(b)
    else:
        assert abs(info["iterations"] - ref.iterations) <= 1
    assert _rel(xh, ref.x) <= SOL_TOL
    prob.close()


def test_quadratic_geometry_rejects_vector_valued_operator(mfcg):
    with pytest.raises(mfcg.MfcgError):
        mfcg.Problem(3, (2, 2, 2), amplitude=0.05, geometry="deformed_quadratic", components=3)


def test_operator_passes_stop_with_the_iterations(mfcg):
    # the unfused forms run graphs of 16 iterations; after the last iteration
    # the remaining operator passes of the graph return at once: a solve of
    # 17 iterations (two graphs) costs about 17/16 of one of 16 iterations
    # (with 15 idle operator passes it would cost about 1.7 times as much)
    prob = mfcg.Problem(4, (48, 48, 48), mode="unfused")
    b = prob.rhs()
    x = torch.zeros_like(b)
    for maxit in (16, 17):
        prob.cg_solve(b, x.zero_(), rtol=0.0, maxit=maxit)
    times = {}
    for maxit in (16, 17, 32):
        torch.cuda.synchronize()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record()
        for _ in range(3):
            prob.cg_solve(b, x.zero_(), rtol=0.0, maxit=maxit)
        e1.record()
        torch.cuda.synchronize()
        times[maxit] = e0.elapsed_time(e1)
    assert times[17] < 1.3 * times[16], times
    assert times[32] > 1.6 * times[16], times
    prob.close()
