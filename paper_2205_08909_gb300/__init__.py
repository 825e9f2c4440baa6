"""Fused matrix-free Jacobi-CG for GB300 (sm_103a).

The hot path of Kronbichler, Sashko and Munch (arXiv 2205.08909): a CG
iteration for the continuous Q_p Laplacian in which the sum-factorised
matrix-free operator evaluation (Eqs. 4-5) is fused with the vector updates
and the seven inner products of the merged PCG algorithm (Algorithm 5).  The
compute runs in the CUDA library libmfcg.so behind the C ABI of
include/mfcg.h; this package is a thin torch binding (device memory, streams).

    import torch, paper_2205_08909_gb300 as mfcg
    prob = mfcg.Problem(degree=4, cells=(64, 64, 64))
    b = prob.rhs()
    x, info = prob.cg_solve(b, rtol=1e-10)
"""
from __future__ import annotations

import ctypes

import torch

from . import _binding
from ._binding import MfcgError, SolveInfo  # noqa: F401

__all__ = ["Problem", "Batch", "MfcgError", "SolveInfo"]


def _ptr(t: torch.Tensor) -> ctypes.c_void_p:
    return ctypes.c_void_p(t.data_ptr())


class Problem:
    """One Q_p Poisson problem on the unit cube, set up on the current CUDA device.

    degree: 1..8; cells: (Nx, Ny, Nz); amplitude: sine deformation of the mesh
    (needs geometry="deformed", which stores J^{-1} and JxW per quadrature
    point, "deformed_tensor", which stores the symmetric J^{-1} JxW a J^{-T}, or
    "deformed_quadratic", the tri-quadratic interpolant of the map per cell with
    the metric computed at each point);
    geometry="user" takes those ten values per point from user_data (host array,
    cells x 10 x (degree+1)^3, cells lexicographic); x_every_iteration: update x
    in every iteration instead of Algorithm 5's delayed update;
    coefficient: "constant" (a = 1) or "sin_x"
    (a = 1 + 0.5 sin(pi x)); mode: "fused" (Algorithm 5 inside the operator
    pass), "unfused" (Algorithm 1, one kernel per vector operation),
    "loop_fused" (Algorithm 1 with loop fusion inside its vector regions) or
    "semi_fused" (Algorithm 5 as separate pre / operator / post kernels);
    preconditioner: "jacobi" or "none" (Algorithm 4);
    precision: "fp64", "double_float" (FP32 pairs, ~48 bits), "fp32_inner"
    (FP64 defect correction around an FP32 fused CG, inner_rtol per cycle) or
    "double_float_inner" (the same around the double-float fused CG, each inner
    solve to the reduction the true residual still needs);
    components: 1 (scalar) or 3 (vector-valued operator, components stored
    one after another; fused mode); operator: "laplace" (BP3/BP4) or "mass"
    (BP1/BP2; affine or geometry="deformed").
    Vectors are float64 CUDA tensors in the library's tile-blocked order.
    """

    def __init__(self, degree: int, cells, amplitude: float = 0.0, geometry: str = "affine",
                 coefficient: str = "constant", mode: str = "fused", precision: str = "fp64",
                 preconditioner: str = "jacobi", inner_rtol: float = 0.0, graph_iterations: int = 0,
                 instrument: bool = False, tile=None, components: int = 1, operator: str = "laplace",
                 user_data=None, x_every_iteration: bool = False, true_residual: bool = False,
                 fp64_contraction: str = "tensor_cores", stream: torch.cuda.Stream | None = None):
        if not torch.cuda.is_available():
            raise RuntimeError("paper_2205_08909_gb300 needs a CUDA device (no CPU fallback)")
        self._lib = _binding.load()
        self.device = torch.device("cuda", torch.cuda.current_device())
        self.stream = stream if stream is not None else torch.cuda.current_stream()
        cells = tuple(int(c) for c in (cells if hasattr(cells, "__len__") else (cells,) * 3))
        self.degree, self.cells = int(degree), cells
        mesh = _binding.Mesh(cells[0], cells[1], cells[2], float(amplitude))
        geom = _binding.Geometry(_binding.GEOM[geometry], _binding.COEF[coefficient], None)
        if geometry == "user":
            # host array of cells x 10 x (degree+1)^3 doubles (J^{-1} row-major, then w det J a)
            import numpy as np

            user = np.ascontiguousarray(user_data, dtype=np.float64)
            if user.size != cells[0] * cells[1] * cells[2] * 10 * (int(degree) + 1) ** 3:
                raise ValueError("user_data: expected cells x 10 x (degree+1)^3 values")
            geom.user_data = user.ctypes.data_as(ctypes.c_void_p)
        opt = _binding.Options()
        opt.mode = _binding.MODE[mode]
        opt.precision = _binding.PRECISION[precision]
        opt.preconditioner = _binding.PRECONDITIONER[preconditioner]
        opt.inner_rtol = float(inner_rtol)
        opt.graph_iterations = int(graph_iterations)
        opt.instrument = 1 if instrument else 0
        opt.components = int(components)
        opt.operator_kind = _binding.OPERATOR[operator]
        opt.x_update_every_iteration = 1 if x_every_iteration else 0
        opt.true_residual = 1 if true_residual else 0
        opt.fp64_contraction = _binding.FP64_CONTRACTION[fp64_contraction]
        self.components = int(components)
        if tile is not None:
            for d in range(3):
                opt.tile[d] = int(tile[d])
        handle = ctypes.c_void_p()
        _binding.check("mfcg_setup", self._lib.mfcg_setup(ctypes.byref(mesh), self.degree, ctypes.byref(geom),
                                                           ctypes.byref(opt), ctypes.c_void_p(self.stream.cuda_stream),
                                                           ctypes.byref(handle)))
        self._h = handle
        n = ctypes.c_int64()
        _binding.check("mfcg_n_dofs", self._lib.mfcg_n_dofs(self._h, ctypes.byref(n)))
        self.n_dofs = int(n.value)

    # ---------------------------------------------------------------- helpers
    def _vec(self, t: torch.Tensor, name: str) -> torch.Tensor:
        if not isinstance(t, torch.Tensor) or t.dtype != torch.float64 or t.device != self.device \
                or t.numel() != self.n_dofs or not t.is_contiguous():
            raise ValueError(f"{name}: expected a contiguous float64 tensor of {self.n_dofs} entries on {self.device}")
        return t

    def empty(self) -> torch.Tensor:
        return torch.empty(self.n_dofs, dtype=torch.float64, device=self.device)

    # ---------------------------------------------------------------- API
    def apply_operator(self, src: torch.Tensor, dst: torch.Tensor | None = None) -> torch.Tensor:
        dst = self.empty() if dst is None else dst
        _binding.check("mfcg_apply_operator", self._lib.mfcg_apply_operator(
            self._h, _ptr(self._vec(src, "src")), _ptr(self._vec(dst, "dst"))))
        return dst

    def diagonal(self, out: torch.Tensor | None = None) -> torch.Tensor:
        out = self.empty() if out is None else out
        _binding.check("mfcg_diagonal", self._lib.mfcg_diagonal(self._h, _ptr(self._vec(out, "diag"))))
        return out

    def rhs(self, out: torch.Tensor | None = None) -> torch.Tensor:
        out = self.empty() if out is None else out
        _binding.check("mfcg_rhs", self._lib.mfcg_rhs(self._h, _ptr(self._vec(out, "b"))))
        return out

    def cg_solve(self, b: torch.Tensor, x: torch.Tensor | None = None, rtol: float = 1e-10, maxit: int = 100000,
                 allow_not_converged: bool = False):
        """Solves A x = b; x (if given) is the initial guess and is overwritten.
        Returns (x, info dict)."""
        if x is None:
            x = torch.zeros(self.n_dofs, dtype=torch.float64, device=self.device)
        info = SolveInfo()
        allowed = (_binding.OK, _binding.NOT_CONVERGED) if allow_not_converged else (_binding.OK,)
        st = self._lib.mfcg_cg_solve(self._h, _ptr(self._vec(b, "b")), _ptr(self._vec(x, "x")), float(rtol),
                                     int(maxit), ctypes.byref(info))
        _binding.check("mfcg_cg_solve", st, allowed)
        return x, info.as_dict()

    def cg_solve_host(self, b: torch.Tensor, x: torch.Tensor, rtol: float = 1e-10, maxit: int = 100000,
                      allow_not_converged: bool = False):
        """The same solve with CPU float64 tensors (pinned for asynchronous copies)."""
        for t, name in ((b, "b"), (x, "x")):
            if t.device.type != "cpu" or t.dtype != torch.float64 or t.numel() != self.n_dofs or not t.is_contiguous():
                raise ValueError(f"{name}: expected a contiguous CPU float64 tensor of {self.n_dofs} entries")
        info = SolveInfo()
        allowed = (_binding.OK, _binding.NOT_CONVERGED) if allow_not_converged else (_binding.OK,)
        st = self._lib.mfcg_cg_solve_host(self._h, _ptr(b), _ptr(x), float(rtol), int(maxit), ctypes.byref(info))
        _binding.check("mfcg_cg_solve_host", st, allowed)
        return x, info.as_dict()

    def to_lexicographic(self, v: torch.Tensor, out: torch.Tensor | None = None) -> torch.Tensor:
        out = self.empty() if out is None else out
        _binding.check("mfcg_to_lexicographic", self._lib.mfcg_to_lexicographic(
            self._h, _ptr(self._vec(v, "in")), _ptr(self._vec(out, "out"))))
        return out

    def from_lexicographic(self, v: torch.Tensor, out: torch.Tensor | None = None) -> torch.Tensor:
        out = self.empty() if out is None else out
        _binding.check("mfcg_from_lexicographic", self._lib.mfcg_from_lexicographic(
            self._h, _ptr(self._vec(v, "in")), _ptr(self._vec(out, "out"))))
        return out

    def close(self) -> None:
        if getattr(self, "_h", None) and not getattr(self, "_borrowed", False):
            self._lib.mfcg_destroy(self._h)
        self._h = None

    @classmethod
    def _member(cls, lib, handle, degree: int, cells, stream) -> "Problem":
        """View of a batch member (owned by the batch)."""
        self = cls.__new__(cls)
        self._lib, self._h, self._borrowed = lib, handle, True
        self.device = torch.device("cuda", torch.cuda.current_device())
        self.stream = stream
        self.degree, self.cells = int(degree), tuple(cells)
        self.components = 1
        n = ctypes.c_int64()
        _binding.check("mfcg_n_dofs", lib.mfcg_n_dofs(handle, ctypes.byref(n)))
        self.n_dofs = int(n.value)
        return self

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()


class Batch:
    """Independent problems solved together: the fused iterations of all members
    run as one CUDA graph with one branch per member (mfcg_setup_batch).

    specs: list of dicts with keys degree, cells and optionally amplitude,
    geometry, coefficient; precision: "fp64" or "double_float".
    members[i] is a Problem view for rhs / apply_operator / reordering.
    """

    def __init__(self, specs, precision: str = "fp64", graph_iterations: int = 0,
                 stream: torch.cuda.Stream | None = None):
        if not torch.cuda.is_available():
            raise RuntimeError("paper_2205_08909_gb300 needs a CUDA device (no CPU fallback)")
        self._lib = _binding.load()
        self.stream = stream if stream is not None else torch.cuda.current_stream()
        count = len(specs)
        meshes = (_binding.Mesh * count)()
        geoms = (_binding.Geometry * count)()
        degrees = (ctypes.c_int * count)()
        cells_list = []
        for i, sp in enumerate(specs):
            c = sp["cells"]
            c = tuple(int(v) for v in (c if hasattr(c, "__len__") else (c,) * 3))
            cells_list.append(c)
            amp = float(sp.get("amplitude", 0.0))
            geometry = sp.get("geometry", "deformed" if amp != 0.0 else "affine")
            meshes[i] = _binding.Mesh(c[0], c[1], c[2], amp)
            geoms[i] = _binding.Geometry(_binding.GEOM[geometry], _binding.COEF[sp.get("coefficient", "constant")])
            degrees[i] = int(sp["degree"])
        opt = _binding.Options()
        opt.mode = _binding.MODE["fused"]
        opt.precision = _binding.PRECISION[precision]
        opt.graph_iterations = int(graph_iterations)
        handle = ctypes.c_void_p()
        _binding.check("mfcg_setup_batch", self._lib.mfcg_setup_batch(
            count, meshes, degrees, geoms, ctypes.byref(opt), ctypes.c_void_p(self.stream.cuda_stream),
            ctypes.byref(handle)))
        self._h = handle
        self.members = []
        for i in range(count):
            mh = ctypes.c_void_p()
            _binding.check("mfcg_batch_member", self._lib.mfcg_batch_member(self._h, i, ctypes.byref(mh)))
            self.members.append(Problem._member(self._lib, mh, degrees[i], cells_list[i], self.stream))

    def cg_solve(self, bs, xs=None, rtol: float = 1e-10, maxit: int = 100000, allow_not_converged: bool = False):
        """Solves every member; xs (if given) are the initial guesses and are
        overwritten.  Returns (xs, list of info dicts)."""
        count = len(self.members)
        if xs is None:
            xs = [torch.zeros(m.n_dofs, dtype=torch.float64, device=m.device) for m in self.members]
        if len(bs) != count or len(xs) != count:
            raise ValueError(f"expected {count} right-hand sides and solutions")
        bp = (ctypes.c_void_p * count)(*[_ptr(m._vec(b, "b")).value for m, b in zip(self.members, bs)])
        xp = (ctypes.c_void_p * count)(*[_ptr(m._vec(x, "x")).value for m, x in zip(self.members, xs)])
        infos = (SolveInfo * count)()
        allowed = (_binding.OK, _binding.NOT_CONVERGED) if allow_not_converged else (_binding.OK,)
        st = self._lib.mfcg_cg_solve_batch(self._h, bp, xp, float(rtol), int(maxit), infos)
        _binding.check("mfcg_cg_solve_batch", st, allowed)
        return xs, [infos[i].as_dict() for i in range(count)]

    def close(self) -> None:
        for m in getattr(self, "members", []):
            m._h = None
        if getattr(self, "_h", None):
            self._lib.mfcg_destroy_batch(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()
