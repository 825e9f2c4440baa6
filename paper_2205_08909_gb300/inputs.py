"""Seeded synthetic inputs and the named workloads (no finite-element arithmetic).

Shared by the tests and bench.py.  Random vectors are drawn with numpy's
PCG64 from fixed seeds; workloads are the scalar Q_p Poisson problems on the
unit cube with the shapes of the paper's benchmark problems.
"""
from __future__ import annotations

import dataclasses

import numpy as np

SEED_VECTORS = 220508909
SEED_RHS_BLOCK = 220508910


@dataclasses.dataclass(frozen=True)
class Workload:
    name: str
    degree: int
    cells: tuple[int, int, int]
    amplitude: float = 0.0
    coefficient: str = "constant"

    @property
    def geometry(self) -> str:
        return "deformed" if (self.amplitude != 0.0 or self.coefficient != "constant") else "affine"

    @property
    def n_dofs(self) -> int:
        n = 1
        for c in self.cells:
            n *= self.degree * c + 1
        return n


WORKLOADS = {
    "q2_8cube": Workload("q2_8cube", 2, (8, 8, 8)),
    "q4_64cube": Workload("q4_64cube", 4, (64, 64, 64)),
    "q6_48cube_deformed": Workload("q6_48cube_deformed", 6, (48, 48, 48), 0.05, "sin_x"),
    # the same deformed problem on a smaller mesh (7.2 M unknowns, about 1.5 GB of
    # vectors and geometry): the case for multi-pass profiles of its kernel
    "q6_32cube_deformed": Workload("q6_32cube_deformed", 6, (32, 32, 32), 0.05, "sin_x"),
    "q4_128cube": Workload("q4_128cube", 4, (128, 128, 128)),
}


def random_vector(n: int, seed: int = SEED_VECTORS, salt: int = 0) -> np.ndarray:
    """Standard-normal vector of length n (lexicographic node order)."""
    return np.random.Generator(np.random.PCG64([seed, salt])).standard_normal(n)


def random_rows(n: int, count: int, seed: int = SEED_VECTORS, salt: int = 1) -> np.ndarray:
    """count distinct row indices in [0, n)."""
    rng = np.random.Generator(np.random.PCG64([seed, salt]))
    return np.sort(rng.choice(n, size=min(count, n), replace=False))


def boundary_zeroed(v: np.ndarray, nodes_per_dim) -> np.ndarray:
    """Copy of v with the entries of the Dirichlet (boundary) nodes set to 0."""
    nx, ny, nz = nodes_per_dim
    out = v.copy().reshape(nz, ny, nx)
    out[0], out[-1] = 0.0, 0.0
    out[:, 0], out[:, -1] = 0.0, 0.0
    out[:, :, 0], out[:, :, -1] = 0.0, 0.0
    return out.reshape(-1)


def batch_problems(count: int = 64, seed: int = SEED_VECTORS, max_cells: int = 32) -> list[dict]:
    """Independent problems of a batch: degree ~ U{2..8}, cells per direction
    ~ U{4..max_cells} (cubes), deformation amplitude ~ U[0, 0.08] with the
    coefficient a = 1 + 0.5 sin(pi x) on deformed meshes."""
    rng = np.random.Generator(np.random.PCG64(seed))
    out = []
    for _ in range(count):
        p = int(rng.integers(2, 9))
        n = int(rng.integers(4, max_cells + 1))
        a = float(rng.uniform(0.0, 0.08))
        out.append({"degree": p, "cells": (n, n, n), "amplitude": a, "coefficient": "sin_x",
                    "geometry": "deformed_tensor"})
    return out


def batch_rhs(problems: list[dict], seed: int = SEED_RHS_BLOCK) -> list[np.ndarray]:
    """Standard-normal right-hand sides of the batch problems (lexicographic
    node order), zero on the Dirichlet nodes."""
    out = []
    for i, sp in enumerate(problems):
        dims = tuple(sp["degree"] * c + 1 for c in sp["cells"])
        v = random_vector(dims[0] * dims[1] * dims[2], seed, i)
        out.append(boundary_zeroed(v, dims))
    return out
