#!/usr/bin/env python3
"""Benchmark of the fused matrix-free Jacobi-CG (Algorithm 5) on GB300.

One step = one CG solve of the workload with a fixed number of iterations
(default 50, x0 = 0, manufactured right-hand side; default workload Q4 on
128^3 cells, 135,005,697 unknowns, FP64): start-up (r0 = b - A x0,
scalars), the fused iterations (pre, sum-factorised operator, post, seven
sums, device-side reduction and scalars) and the parity-dependent
finalisation of x.  The metric is GDoF-iterations/s = n * iterations / s and
its fraction of the HBM roofline, for the fused path and for the plain unfused
GPU CG (separate operator, axpy, Jacobi and dot kernels) on the same workload.

    python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]

With --gpus N > 1 (launched by torchrun) every rank runs an independent
replica of the workload (the method has no cross-replica exchange): value is
the sum over ranks, time the maximum over ranks.  --impl reference times the
CPU oracle (assembled sparse matrix + textbook Algorithm 1) on the host.
"""
from __future__ import annotations

import argparse
import hashlib
import json
import os
import re
import statistics
import subprocess
import sys
import tempfile
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "CG GDoF-iterations/s and % of HBM roofline, fused vs unfused GPU CG at rtol 1e-10"
UNIT = "GDoF-it/s"
FP64_PEAK_TFLOPS = 1.25          # nominal FP64 rate of GB300 (dense, FMA = 2 flops)
FALLBACK_HBM_GBS = 6800.0
KERNEL_SOURCES = ["paper_2205_08909_gb300/csrc/tile_kernels.cuh", "paper_2205_08909_gb300/csrc/mfcg_internal.h",
                  "paper_2205_08909_gb300/csrc/precision.cuh", "paper_2205_08909_gb300/csrc/tc_operator.cuh"]


def measured_peaks():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as fh:
            return json.load(fh), "measured"
    except OSError:
        return {"hbm_gbs": FALLBACK_HBM_GBS}, "fallback"


def kernel_sources_hash() -> str:
    """Hash of the kernel sources with comments and whitespace removed, so that
    an edit of comments alone keeps the stored ncu counters valid."""
    h = hashlib.sha256()
    for rel in KERNEL_SOURCES:
        with open(os.path.join(ROOT, rel)) as fh:
            text = fh.read()
        text = re.sub(r"/\*.*?\*/", " ", text, flags=re.S)
        text = re.sub(r"//[^\n]*", " ", text)
        h.update(" ".join(text.split()).encode())
    return h.hexdigest()[:16]


TRAFFIC_FILE = os.path.join(ROOT, "profiles", "traffic.json")


def stored_traffic(workload: str, precision: str):
    """DRAM bytes per launch of the fused tile kernel (ncu dram__bytes_read.sum +
    dram__bytes_write.sum) from profiles/traffic.json, or None if no capture of
    this (workload, precision) exists or it was taken on different kernel sources."""
    try:
        with open(TRAFFIC_FILE) as fh:
            table = json.load(fh)
    except (OSError, ValueError):
        return None
    entry = table.get(f"{workload}/{precision}")
    if not entry or entry.get("kernel_sources_sha256") != kernel_sources_hash():
        return None
    return float(entry["dram_bytes_per_launch"])


# ------------------------------------------------------------------------------ algorithmic counts

def geometry_values(geometry: str) -> int:
    """Values stored per quadrature point: J^{-1} and JxW a (10) or the final tensor (6)."""
    return {"affine": 0, "deformed": 10, "deformed_tensor": 6, "deformed_quadratic": 0}[geometry]


def geometry_bytes_per_dof(geometry: str, degree: int, n_cells: int, n_dofs: int) -> float:
    """Stored geometry read per iteration and unknown: the per-point values, or
    the 27 x 3 support-point coordinates per cell of the tri-quadratic map."""
    if geometry == "deformed_quadratic":
        return 81 * 8.0 * n_cells / n_dofs
    return geometry_values(geometry) * 8.0 * n_cells * (degree + 1) ** 3 / n_dofs


DEFAULT_TILE = {"affine": [0, 16, 8, 5, 4, 3, 3, 2, 2], "deformed": [0, 8, 4, 4, 3, 2, 2, 2, 2]}


def brick_segments(degree: int, cells, tile=None) -> tuple[int, int, int]:
    """Cell segments that the whole-brick sweeps of a Cartesian operator pass
    process per launch, summed over the tiles (z, y and x sweeps): a sweep
    along direction d runs over every brick line across d, one segment per cell
    along d.  Neighbouring cells share their face lines, so a cell costs about
    p^2 segments per sweep instead of the (p+1)^2 pencils of a cell-wise sweep."""
    T = tile or (DEFAULT_TILE["affine"][degree],) * 3
    seg = [0, 0, 0]
    # tile extents along each direction: full tiles of T cells and a ragged last one
    ext = []
    for d in range(3):
        n, t = cells[d], T[d]
        sizes = [t] * (n // t) + ([n % t] if n % t else [])
        ext.append(sizes)
    for nz in ext[2]:
        for ny in ext[1]:
            for nx in ext[0]:
                bx, by, bz = degree * nx + 1, degree * ny + 1, degree * nz + 1
                seg[2] += bx * by * nz
                seg[1] += bx * bz * ny
                seg[0] += by * bz * nx
    return seg[2], seg[1], seg[0]


def eo_segment_costs(n1: int, unit: str) -> tuple[float, float, float]:
    """Operations of one cell segment of the z (M and K_z from x), y (M x;
    K_y x + M z) and x (K_x x + M z) sweeps in even-odd form, with the carry of
    the shared node.  unit "flop": FP64 flops (FMA = 2).  unit "dd": FP32-pipe
    operations of the double-float arithmetic (pair addition 11, a K-term sum
    12 K - 5: first product 4, each further product 12, normalisation 3)."""
    h, ne = n1 // 2, n1 - n1 // 2
    if unit == "flop":
        add, dot = 1.0, (lambda k: 2.0 * k)
    else:
        add, dot = 11.0, (lambda k: 12.0 * k - 5.0)
    one = h * (dot(ne) + dot(h) + 2 * add) + (dot(ne) if ne > h else 0)          # A x
    two = h * (dot(2 * ne) + dot(2 * h) + 2 * add) + (dot(2 * ne) if ne > h else 0)  # A x + B z
    form1, form2 = 2 * h * add, 4 * h * add
    z = form1 + 2 * one + 2 * add
    y = form2 + one + two + 2 * add
    x = form2 + two + add
    return z, y, x


def eo_product_cost(n1: int, unit: str, anti: bool = False) -> float:
    """Operations of one even-odd 1D product y = A x (A centrosymmetric, or
    anti-centrosymmetric for the collocation derivative): forming the even and
    odd halves, the two half-size products and the recombination."""
    h, ne = n1 // 2, n1 - n1 // 2
    if unit == "flop":
        add, dot = 1.0, (lambda k: 2.0 * k)
    else:
        add, dot = 11.0, (lambda k: 12.0 * k - 5.0)
    rows = h * (dot(ne) + dot(h) + 2 * add)
    mid = (dot(h) if anti else dot(ne)) if ne > h else 0.0
    return 2 * h * add + rows + mid


def deformed_cell_cost(n1: int, unit: str, geometry: str) -> float:
    """Operations per deformed cell: 6 interpolation and 6 collocation-derivative
    sweeps of (p+1)^2 even-odd products each, two accumulating sweeps, the
    per-point metric and the node gather."""
    pencils = n1 * n1
    sweeps = 6 * pencils * eo_product_cost(n1, unit) + 6 * pencils * eo_product_cost(n1, unit, anti=True)
    if unit == "flop":
        if geometry == "deformed_quadratic":
            # per point: Jacobian and position 50, cofactors 27, det 5, the
            # factor w a / det ~5 (sine not counted), C^T (f C g) 33; per cell
            # the line sums, 48 flops for each of 9 (p+1)^2 (d, a, line) items
            return sweeps + (2 + 120 + 1) * n1 ** 3 + 48 * 9 * n1 ** 2
        metric = 42 if geometry == "deformed" else 18
        return sweeps + (2 + metric + 1) * n1 ** 3
    dot3 = 4 + 12 * 2 + 3
    axby = 4 + 12 + 3
    if geometry == "deformed_quadratic":
        # 17 three-term sums, 9 cofactor pairs, 3 pair products per point; per
        # (d, a, line) item 6 three-term sums and 9 accumulations
        metric = 17 * dot3 + 9 * axby + 3 * 7
        return sweeps + (2 * 11 + metric + 11) * n1 ** 3 + (6 * dot3 + 9 * axby) * 9 * n1 ** 2
    metric = 3 * dot3 if geometry == "deformed_tensor" else 6 * dot3 + 3 * 7
    return sweeps + (2 * 11 + metric + 11) * n1 ** 3


def algorithmic_flops_per_iteration(degree: int, n_cells: int, n_dofs: int, geometry: str = "affine",
                                    cells=None, tile=None) -> float:
    """FP64 flops of one fused iteration.  Affine cells: the whole-brick
    sweeps in even-odd form over the segments of brick_segments; deformed
    cells: twelve cell-wise sweeps in even-odd form (interpolation,
    collocation derivative and their transposes) plus the per-point metric (42
    flops from J^{-1} and JxW a, 18 from the final tensor) and the gather
    (deformed_cell_cost).  Plus the vector work per unknown (r, z, p updates
    5, x update 5 every other iteration, seven sums with M^-1 r and M^-1 v 16)."""
    n1 = degree + 1
    if geometry == "affine":
        sz, sy, sx = brick_segments(degree, cells, tile)
        cz, cy, cx = eo_segment_costs(n1, "flop")
        op = sz * cz + sy * cy + sx * cx
    else:
        op = deformed_cell_cost(n1, "flop", geometry) * n_cells
    return op + 23.5 * n_dofs


ALGORITHMIC_BYTES_PER_DOF = 64.0  # r, p, v read+write, D^-1 read, x read+write every other iteration

# Tensor-core FP64 operator (tc_operator.cuh): degrees with it, digit pairs kept
# (k + l >= 6 of 8 x 8), and the tiles the library picks for it
TC_DEGREES = (1, 2, 3, 4, 5, 7)
TC_DIGIT_PAIRS = 43


def effective_tile(degree: int, geometry: str, precision: str, contraction: str, tile=None):
    """Tile of cells the library uses: the given one, else its default (4 x 4 x 3
    cells for the tensor-core FP64 operator at degree 4)."""
    if tile:
        return tuple(tile)
    t = DEFAULT_TILE["affine" if geometry == "affine" else "deformed"][degree]
    if geometry == "affine" and precision == "fp64" and contraction == "tensor_cores" and degree == 4:
        return (t, t, 3)
    return (t, t, t)


def tc_mma_per_row_tile(degree: int) -> int:
    """mma.m16n8k16 instructions of one 16-cell row tile: per even-odd block
    ceil(size/16) k steps x ceil(size/8) n tiles, times the digit pairs."""
    n1 = degree + 1
    no, ne = n1 // 2, n1 - n1 // 2
    total = 0
    for b in range(8):
        size = 1
        for d in range(3):
            size *= no if (b >> d) & 1 else ne
        total += -(-size // 16) * -(-size // 8)
    return total * TC_DIGIT_PAIRS


def tc_digit_flops(degree: int, cells, tile) -> float:
    """FP16 tensor-core flops of one operator pass (2 x 16 x 8 x 16 per mma):
    row tiles of up to 4 x 4 x 1 cells per tile, summed over the tiles."""
    rows = 0
    ext = []
    for d in range(3):
        n, t = cells[d], tile[d]
        ext.append([t] * (n // t) + ([n % t] if n % t else []))
    for nz in ext[2]:
        for ny in ext[1]:
            for nx in ext[0]:
                rows += -(-nx // 4) * -(-ny // 4) * nz
    return float(rows) * tc_mma_per_row_tile(degree) * 2 * 16 * 8 * 16


# ------------------------------------------------------------------------------ clocks

class ClockSampler:
    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index: int):
        self.gpu = gpu_index
        self.proc = None
        self.path = None

    def __enter__(self):
        fd, self.path = tempfile.mkstemp(suffix=".csv")
        os.close(fd)
        try:
            self.proc = subprocess.Popen(["nvidia-smi", f"--id={self.gpu}", f"--query-gpu={self.FIELDS}",
                                          "--format=csv,noheader,nounits", "-lms", "200"],
                                         stdout=open(self.path, "w"), stderr=subprocess.DEVNULL)
        except OSError:
            self.proc = None
        time.sleep(0.25)
        return self

    def __exit__(self, *exc):
        if self.proc is not None:
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except subprocess.TimeoutExpired:
                self.proc.kill()

    def summary(self):
        rows = []
        try:
            for line in open(self.path):
                parts = [p.strip() for p in line.split(",")]
                if len(parts) >= 9:
                    rows.append(parts)
        except OSError:
            pass
        finally:
            if self.path:
                os.unlink(self.path)
        if not rows:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["unavailable"], "samples": 0}
        sm = [float(r[1]) for r in rows if r[1].replace(".", "").isdigit()]
        mx = [float(r[2]) for r in rows if r[2].replace(".", "").isdigit()]
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = sorted({names[i] for r in rows for i in range(4) if r[5 + i].lower().startswith("active")})
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": max(mx) if mx else None,
                "reasons": reasons, "samples": len(rows)}


# ------------------------------------------------------------------------------ CPU oracle

def threaded_matvec(A, threads: int):
    """A @ v with the rows of the oracle's CSR matrix split into `threads`
    contiguous blocks, one host thread each (scipy's SpMV releases the GIL).
    Every row is the same dot product as in A @ v; only the rows are spread
    over the cores."""
    import concurrent.futures

    import numpy as np

    if threads <= 1:
        return (lambda v: A @ v), None
    bounds = np.linspace(0, A.shape[0], threads + 1).astype(int)
    blocks = [A[bounds[i]:bounds[i + 1]] for i in range(threads)]
    pool = concurrent.futures.ThreadPoolExecutor(max_workers=threads)

    def mv(v):
        out = np.empty(A.shape[0])

        def one(i):
            out[bounds[i]:bounds[i + 1]] = blocks[i] @ v

        list(pool.map(one, range(threads)))
        return out

    return mv, pool


def oracle_sample(degree: int, cells: int, iters: int, threads: int = 1):
    """Times the oracle's Algorithm 1 (assembled CSR, scipy SpMV on `threads`
    host threads, numpy vector ops) on a Cartesian Q_degree mesh of cells^3 for
    a fixed number of iterations.  Returns (GDoF-it/s, seconds, n_dofs, setup
    seconds); setup = assembly of the CSR matrix, right-hand side and diagonal."""
    from oracle import cg as ocg
    from oracle import fem

    t0 = time.perf_counter()
    prob = fem.Problem(degree, (cells, cells, cells))
    A = fem.assemble(prob)
    b = fem.rhs(prob)
    inv_diag = 1.0 / A.diagonal()
    setup = time.perf_counter() - t0
    mv, pool = threaded_matvec(A, threads)
    try:
        t0 = time.perf_counter()
        res = ocg.pcg_algorithm1(mv, b, inv_diag, 0.0, iters)
        dt = time.perf_counter() - t0
    finally:
        if pool is not None:
            pool.shutdown()
    return prob.n_dofs * res.iterations / dt / 1e9, dt, prob.n_dofs, setup


def host_cores() -> int:
    try:
        return len(os.sched_getaffinity(0))
    except AttributeError:
        return os.cpu_count() or 1


# ------------------------------------------------------------------------------ distributed

def dist_setup(args):
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    if world > 1:
        import torch
        import torch.distributed as dist

        backend = "nccl" if (args.impl == "ours" and torch.cuda.is_available()) else "gloo"
        if backend == "nccl":
            torch.cuda.set_device(local)
        dist.init_process_group(backend)
    return world, rank, local


def barrier(world):
    if world > 1:
        import torch.distributed as dist

        dist.barrier()


def max_over_ranks(x: float, world: int) -> float:
    if world == 1:
        return x
    import torch
    import torch.distributed as dist

    t = torch.tensor([x], dtype=torch.float64, device="cuda" if torch.cuda.is_available() else "cpu")
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


# ------------------------------------------------------------------------------ arms

def run_reference(args, world, rank):
    if rank != 0:
        return None
    from paper_2205_08909_gb300 import inputs

    w = inputs.WORKLOADS[args.workload]
    cells = args.ref_cells
    cores = host_cores()
    for _ in range(args.warmup):
        oracle_sample(w.degree, cells, 2, cores)
    vals, secs = [], []
    n = 0
    setup = 0.0
    for _ in range(args.steps):
        v, dt, n, setup = oracle_sample(w.degree, cells, args.ref_iters, cores)
        vals.append(v)
        secs.append(dt)
    value = sum(vals) / len(vals)
    sample = (f"oracle Algorithm 1 (assembled CSR, scipy SpMV on {cores} host threads) on Q{w.degree} {cells}^3 "
              f"Cartesian ({n} DoFs), {args.ref_iters} fixed iterations per step, same degree as {w.name}; "
              f"assembly {setup:.1f} s per step, not timed. The full workload's CSR matrix "
              f"(about {w.n_dofs * (2 * w.degree + 1) ** 3 * 12 / 1e9:.0f} GB) is not assembled on the host")
    return {
        # n_gpus: the launch configuration of this arm (the oracle itself runs on rank 0's host cores)
        "impl": "reference", "metric": METRIC, "value": round(value, 6), "unit": UNIT, "n_gpus": world,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": round(1e3 * sum(secs) / len(secs), 3),
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
        "config": {"workload": w.name, "degree": w.degree, "cells": list(w.cells), "sample_cells": [cells] * 3},
        "same_config_note": "a bounded sample of the same degree: the oracle assembles the matrix",
        "cpu_baseline": {"value": round(value, 6), "unit": UNIT, "cores": cores, "kind": "oracle", "sample": sample},
        "e2e": {"value": round(value, 6), "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }


def dd_ops_per_dof(degree: int, n_cells: int, n_dofs: int, geometry: str = "affine", cells=None,
                   tile=None) -> float:
    """FP32-pipe operations of one fused double-float iteration per unknown,
    counted from the error-free transformations: a product accumulated into a
    (s, t) pair costs 12 (TwoProduct 2, cross terms 2, TwoSum 6, error sum 2),
    the first product of a sum 4, a normalisation 3, a pair addition 11, a pair
    product 7.  Affine operator: the whole-brick sweeps in even-odd form
    (eo_segment_costs) over the segments of brick_segments.  Deformed
    operator: twelve cell-wise sweeps in even-odd form, two accumulating
    transposed-derivative sweeps, the metric (3 three-term sums from the final
    tensor; 6 sums and 3 pair products from J^{-1} and JxW a) and the node
    gather (one pair addition per cell node): deformed_cell_cost."""
    n1 = degree + 1
    if geometry == "affine":
        sz, sy, sx = brick_segments(degree, cells, tile)
        cz, cy, cx = eo_segment_costs(n1, "dd")
        op = (sz * cz + sy * cy + sx * cx) / n_dofs
    else:
        op = deformed_cell_cost(n1, "dd", geometry) * n_cells / n_dofs
    pre = 34.0 * 1.2                                  # r and p updates on the tile brick (~1.2x the owned nodes)
    x_update = 48.0 / 2                               # every other iteration
    post = 2 * 7 + 7 * 12                             # M^-1 r, M^-1 v and seven accumulations
    return op + pre + x_update + post


def fp32_pipe_peak_tops() -> float:
    """152 SMs x 128 FP32 lanes x 2.07 GHz (maximum SM clock)."""
    return 152 * 128 * 2.07e9 / 1e12


def run_ours(args, world, rank, local):
    import torch

    import paper_2205_08909_gb300 as mfcg
    from paper_2205_08909_gb300 import build, inputs

    build.build()
    torch.cuda.set_device(local)
    w = inputs.WORKLOADS[args.workload]
    n_cells = w.cells[0] * w.cells[1] * w.cells[2]
    K, W, iters = args.steps, args.warmup, args.iters
    peaks, peak_kind = measured_peaks()
    hbm = float(peaks.get("hbm_gbs", FALLBACK_HBM_GBS))
    main_prec = args.precision

    tile = tuple(int(t) for t in args.tile.split(",")) if args.tile else None
    geometry = w.geometry
    if args.geometry:
        if w.geometry == "affine":
            raise SystemExit("--geometry applies to deformed workloads only")
        geometry = args.geometry

    def make(mode, precision, instrument=False, contraction="tensor_cores"):
        return mfcg.Problem(w.degree, w.cells, amplitude=w.amplitude, geometry=geometry,
                            coefficient=w.coefficient, mode=mode, precision=precision, instrument=instrument,
                            tile=tile, fp64_contraction=contraction,
                            x_every_iteration=args.x_update == "every_iteration")

    def timed_steps(prob, b, K, W):
        xs = [torch.zeros(prob.n_dofs, dtype=torch.float64, device="cuda") for _ in range(max(K, W, 1))]
        for i in range(W):
            prob.cg_solve(b, xs[i], rtol=0.0, maxit=iters)
        launches = 0
        torch.cuda.synchronize()
        barrier(world)
        stream = torch.cuda.current_stream()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        torch.cuda.synchronize()
        e0.record(stream)
        for i in range(K):
            _, info = prob.cg_solve(b, xs[i], rtol=0.0, maxit=iters)
            launches += info["kernel_launches"]
        e1.record(stream)
        torch.cuda.synchronize()
        barrier(world)
        ms = e0.elapsed_time(e1)
        return max_over_ranks(ms, world), launches

    def converged_solve(prob, b):
        xc = torch.zeros(w.n_dofs, dtype=torch.float64, device="cuda")
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        _, info = prob.cg_solve(b, xc, rtol=1e-10, maxit=100000)
        torch.cuda.synchronize()
        return {"iterations": info["iterations"], "ms": round(1e3 * (time.perf_counter() - t0), 3),
                "converged": info["converged"], "outer_cycles": info["outer_cycles"]}

    dof_its = w.n_dofs * iters * K * world
    # algorithmic bytes per unknown: the vectors, plus the stored geometry of deformed meshes
    geo_bytes_per_dof = geometry_bytes_per_dof(geometry, w.degree, n_cells, w.n_dofs)
    bytes_per_dof = ALGORITHMIC_BYTES_PER_DOF + geo_bytes_per_dof
    # stored values are 8 bytes (FP64, double-float pairs) or 4 bytes (FP32)
    kernel_bytes_per_dof = bytes_per_dof / 2 if main_prec == "fp32_inner" else bytes_per_dof

    # ---------------- headline: fused CG in the requested precision
    fused = make("fused", main_prec)
    b = fused.rhs()
    with ClockSampler(local) as clk:
        ms_f, launches_f = timed_steps(fused, b, K, W)
    clocks = clk.summary()
    value = dof_its / (ms_f / 1e3) / 1e9
    solve_main = converged_solve(fused, b)

    # ---------------- comparators on the same workload
    variants = {}
    # algorithmic bytes per unknown of each form: fused 64; semi-fused (the GPU form of Sec. 6.4:
    # pre 56, operator 16, post 32) 104; Algorithm 1 with loop fusion inside its regions (operator 16,
    # p.v 16, x/r/r.r 48, z/r.z 24, p 24) 128; unfused Algorithm 1 152
    form_bytes = {"fused": 64, "semi_fused": 104, "loop_fused": 128, "unfused": 152}
    forms = []
    for f in (("unfused", main_prec), ("loop_fused", main_prec), ("fused", "fp64"), ("unfused", "fp64"),
              ("loop_fused", "fp64"), ("semi_fused", "fp64"), ("fused", "fp64_pipe"), ("fused", "double_float"),
              ("unfused", "double_float")):
        if f not in forms:
            forms.append(f)
    for mode, prec_name in forms:
        # "fp64_pipe": FP64 with the operator's sweeps on the FP64 pipe (Cartesian meshes)
        prec = "fp64" if prec_name == "fp64_pipe" else prec_name
        if prec_name == "fp64_pipe" and geometry != "affine":
            continue
        if mode != "fused" and prec == "fp32_inner":
            continue  # the FP32 inner solver exists in fused form only
        if args.skip_unfused and mode == "unfused":
            continue
        if args.skip_variants and (mode, prec) not in (("unfused", main_prec), ("loop_fused", main_prec)):
            continue
        if prec_name == main_prec and mode == "fused":
            continue
        prob = make(mode, prec, contraction="fp64_pipe" if prec_name == "fp64_pipe" else "tensor_cores")
        bv = prob.rhs()  # each problem's own tile-blocked order
        ms_v, _ = timed_steps(prob, bv, K, W)
        v = dof_its / (ms_v / 1e3) / 1e9
        vb = form_bytes[mode] + geo_bytes_per_dof
        variants[f"{mode}_{prec_name}"] = {"value": round(v, 4), "ms_per_step": round(ms_v / K, 3),
                                      "hbm_roofline_frac": round(v / world * vb / hbm, 4),
                                      "algorithmic_bytes_per_dof": round(vb, 2),
                                      "solve_rtol_1e-10": converged_solve(prob, bv)}
        prob.close()
    unf_key, loop_key = f"unfused_{main_prec}", f"loop_fused_{main_prec}"
    fused_over_unfused = round(value / variants[unf_key]["value"], 4) if unf_key in variants else None
    fused_over_loop_fused = round(value / variants[loop_key]["value"], 4) if loop_key in variants else None

    # ---------------- FP64 defect correction around the FP32 fused CG (time to rtol 1e-10)
    # and around the double-float fused CG (each inner solve to the reduction the
    # true residual still needs), against the fused FP64 CG's time to the same
    # tolerance
    dc = dc_dd = None
    if not args.skip_dc:
        dcp = make("fused", "fp32_inner")
        bdc = dcp.rhs()
        converged_solve(dcp, bdc)
        dc = converged_solve(dcp, bdc)
        dcp.close()
        dcp = make("fused", "double_float_inner")
        bdc = dcp.rhs()
        converged_solve(dcp, bdc)
        dc_dd = converged_solve(dcp, bdc)
        dcp.close()
        if main_prec == "fp64" and dc_dd["ms"] > 0:
            dc_dd["fused_fp64_solve_ms_over_this"] = round(solve_main["ms"] / dc_dd["ms"], 4)

    # ---------------- dominant kernel: fused tile kernel, CUDA events around every launch
    inst = make("fused", main_prec, instrument=True)
    xi = torch.zeros(w.n_dofs, dtype=torch.float64, device="cuda")
    bi = inst.rhs()
    inst.cg_solve(bi, xi, rtol=0.0, maxit=min(iters, 8))
    _, info_i = inst.cg_solve(bi, xi.zero_(), rtol=0.0, maxit=iters)
    kernel_ms = info_i["main_kernel_ms"] / max(info_i["main_kernel_launches"], 1)
    inst.close()
    hbm_gbs = kernel_bytes_per_dof * w.n_dofs / (kernel_ms / 1e3) / 1e9
    traffic = stored_traffic(w.name, main_prec)
    eff_tile = effective_tile(w.degree, geometry, main_prec, "tensor_cores", tile)
    tc_main = main_prec == "fp64" and geometry == "affine" and w.degree in TC_DEGREES
    if tc_main:
        # FP64 on the tensor cores: the HBM roofline that the fused method aims at,
        # with the tensor-pipe and FP64-equivalent views beside it
        tflops = tc_digit_flops(w.degree, w.cells, eff_tile)
        bf16 = float(peaks.get("bf16_tflops", 1900.0))
        f64_flops = algorithmic_flops_per_iteration(w.degree, n_cells, w.n_dofs, geometry, w.cells, eff_tile)
        roofline = {"bound": "hbm", "achieved": round(hbm_gbs, 1), "peak": hbm, "unit": "GB/s",
                    "frac": round(hbm_gbs / hbm, 4), "traffic": traffic, "peak_kind": peak_kind,
                    "tensor_view": {"digit_product_tflops": round(tflops / (kernel_ms / 1e3) / 1e12, 2),
                                    "peak_tflops": bf16, "peak_kind": "measured bf16 dense burst (FP16 same rate)",
                                    "frac": round(tflops / (kernel_ms / 1e3) / 1e12 / bf16, 4),
                                    "flops_per_launch": tflops},
                    "fp64_equivalent_view": {"tflops": round(f64_flops / (kernel_ms / 1e3) / 1e12, 4),
                                             "peak_tflops": FP64_PEAK_TFLOPS, "peak_kind": "nominal FP64",
                                             "frac": round(f64_flops / (kernel_ms / 1e3) / 1e12 / FP64_PEAK_TFLOPS, 4)}}
    elif main_prec == "fp64":
        flops = algorithmic_flops_per_iteration(w.degree, n_cells, w.n_dofs, geometry, w.cells, eff_tile)
        achieved = flops / (kernel_ms / 1e3) / 1e12
        roofline = {"bound": "alu", "achieved": round(achieved, 4), "peak": FP64_PEAK_TFLOPS, "unit": "TFLOP/s",
                    "frac": round(achieved / FP64_PEAK_TFLOPS, 4), "traffic": traffic,
                    "peak_kind": "nominal FP64 (recipe table)", "algorithmic_flops_per_launch": flops}
    elif main_prec == "double_float":
        ops = dd_ops_per_dof(w.degree, n_cells, w.n_dofs, geometry, w.cells, tile) * w.n_dofs
        achieved = ops / (kernel_ms / 1e3) / 1e12
        peak = fp32_pipe_peak_tops()
        roofline = {"bound": "alu", "achieved": round(achieved, 4), "peak": round(peak, 2),
                    "unit": "T FP32-pipe ops/s", "frac": round(achieved / peak, 4), "traffic": traffic,
                    "peak_kind": "152 SMs x 128 FP32 lanes x 2.07 GHz", "algorithmic_ops_per_launch": ops}
    else:
        achieved = hbm_gbs
        roofline = {"bound": "hbm", "achieved": round(achieved, 1), "peak": hbm, "unit": "GB/s",
                    "frac": round(achieved / hbm, 4), "traffic": traffic, "peak_kind": peak_kind}
    roofline.update({"kernel": f"tile_kernel<{w.degree}, MODE_CG, GEOM_{ {'affine': 'AFFINE', 'deformed': 'DEFORMED', 'deformed_tensor': 'TENSOR', 'deformed_quadratic': 'QUAD'}[geometry]}, {'fp64, tensor-core contractions' if tc_main else main_prec}>",
                     "tile": list(eff_tile),
                     "kernel_ms": round(kernel_ms, 4),
                     "hbm_view": {"achieved_gbs": round(hbm_gbs, 1), "peak_gbs": hbm, "peak_kind": peak_kind,
                                  "frac": round(hbm_gbs / hbm, 4),
                                  # measured DRAM bytes of the stored ncu capture over the CUDA-event time
                                  "dram_gbs": round(traffic / (kernel_ms / 1e3) / 1e9, 1) if traffic else None,
                                  "dram_bytes_per_dof": round(traffic / w.n_dofs, 1) if traffic else None}})

    # ---------------- end to end through the host-array entry point
    e2e = None
    if not args.skip_e2e:
        bh = b.cpu().pin_memory()
        xh = [torch.zeros(w.n_dofs, dtype=torch.float64).pin_memory() for _ in range(K)]
        fused.cg_solve_host(bh, torch.zeros(w.n_dofs, dtype=torch.float64).pin_memory(), rtol=0.0, maxit=iters)
        torch.cuda.synchronize()
        barrier(world)
        t0 = time.perf_counter()
        for i in range(K):
            fused.cg_solve_host(bh, xh[i], rtol=0.0, maxit=iters)
        torch.cuda.synchronize()
        barrier(world)
        sec = max_over_ranks(time.perf_counter() - t0, world)
        e2e = {"value": round(dof_its / sec / 1e9, 4), "unit": UNIT,
               "h2d_bytes_per_step": 2 * 8 * w.n_dofs, "d2h_bytes_per_step": 8 * w.n_dofs}
    fused.close()

    # ---------------- batched forms (short runs): a batch of independent problems and a block of
    # right-hand sides sharing one mesh's operator data
    batched = None
    if not args.skip_batch:
        bprec = "fp64" if main_prec == "fp64" else "double_float"
        batched = {}
        for key, blk in (("batch_of_8_problems", False), ("block_of_8_rhs_q5_48cube", True)):
            batched[key] = measure_batch(batch_specs(8, blk), bprec, 2, 1, iters, world, local)
            batched[key]["precision"] = bprec

    # the stated target of the fused FP64 CG at p = 4 on >= 100M unknowns
    met = bool(main_prec == "fp64" and value / world * kernel_bytes_per_dof / hbm >= 0.70
               and (fused_over_unfused or 0.0) >= 2.0)
    target = {"hbm_roofline_frac_min": 0.70, "fused_over_unfused_min": 2.0, "met": met,
              "why_not": None if met else (
                  "the fused FP64 kernel is bound by FP64 vector arithmetic (Algorithm 5: about 15 FP64 "
                  "operations per unknown and iteration, twice Algorithm 1's, on a pipe of two FMAs per clock "
                  "per SM) and by issue latency, not by HBM traffic")}

    dtype = {"fp64": "f64", "double_float": "f32x2 (double-float, ~48-bit; FP64 scalars and reductions)",
             "fp32_inner": "f32"}[main_prec]
    line = {
        "metric": METRIC, "value": round(value, 4), "unit": UNIT, "n_gpus": world, "steps": K, "warmup": W,
        "ms_per_step": round(ms_f / K, 3), "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
        "dtype": dtype,
        "data": "synthetic: manufactured right-hand side of u = sin(pi x) sin(pi y) sin(pi z), x0 = 0",
        "config": {"workload": w.name, "degree": w.degree, "cells": list(w.cells), "n_dofs": w.n_dofs,
                   "geometry": geometry, "precision": main_prec, "iterations_per_step": iters, "x_update": args.x_update,
                   "tile": list(eff_tile),
                   "arithmetic": ("FP64 vectors, updates and inner products; operator contractions as exact "
                                  "8-bit digit products of 64-bit fixed-point data on the FP16 tensor cores, "
                                  "recombined in 64-bit integers (FP64-level results)") if tc_main else main_prec,
                   "parallelism": f"replicas x{world}",
                   "l2": f"inputs larger than L2: {8 * w.n_dofs / 1e6:.0f} MB per vector, 8 vectors"},
        "hbm_roofline_frac": round(value / world * kernel_bytes_per_dof / hbm, 4),
        "algorithmic_bytes_per_dof": round(kernel_bytes_per_dof, 2),
        "fused_over_unfused": fused_over_unfused,
        "fused_over_loop_fused": fused_over_loop_fused,
        # the stated target of the fused FP64 CG at p = 4 on >= 100M unknowns
        "target": target,
        "solve_rtol_1e-10": solve_main,
        "variants": variants,
        "defect_correction_fp32_inner": dc,
        "defect_correction_double_float_inner": dc_dd,
        "batched": batched,
        "roofline": roofline,
        "e2e": e2e,
        "gpu_launches": launches_f,
        "clocks": clocks,
    }
    if rank == 0 and world == 1 and not args.skip_cpu:
        cores = host_cores()
        v, dt, n, setup = oracle_sample(w.degree, args.ref_cells, args.ref_iters, cores)
        v1, dt1, _, _ = oracle_sample(w.degree, args.ref_cells, max(args.ref_iters // 3, 1), 1)
        line["cpu_baseline"] = {"value": round(v, 6), "unit": UNIT, "cores": cores, "kind": "oracle",
                                "one_thread_value": round(v1, 6),
                                "sample": f"Algorithm 1 on the assembled CSR matrix (scipy SpMV split by rows over "
                                          f"{cores} host threads), Q{w.degree} {args.ref_cells}^3 Cartesian "
                                          f"({n} DoFs), {args.ref_iters} iterations in {dt:.1f} s; assembly "
                                          f"{setup:.1f} s (not in the rate); one thread: {v1:.4g} GDoF-it/s"}
    return line if rank == 0 else None


def measure_batch(specs, prec, K, W, iters, world, local):
    """Times the problems of specs (fixed iterations each) solved as one batch
    (one CUDA graph branch per member) and, for comparison, one after another
    as single problems."""
    import torch

    import paper_2205_08909_gb300 as mfcg
    from paper_2205_08909_gb300 import inputs

    rhs = inputs.batch_rhs(specs)
    batch = mfcg.Batch(specs, precision=prec)
    bs = [m.from_lexicographic(torch.from_numpy(r).cuda()) for m, r in zip(batch.members, rhs)]
    xs = [torch.zeros_like(b) for b in bs]
    dofs = sum(m.n_dofs for m in batch.members)

    def timed(fn):
        for _ in range(W):
            fn()
        torch.cuda.synchronize()
        barrier(world)
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        stream = torch.cuda.current_stream()
        e0.record(stream)
        for _ in range(K):
            fn()
        e1.record(stream)
        torch.cuda.synchronize()
        barrier(world)
        return max_over_ranks(e0.elapsed_time(e1), world)

    def batched():
        for x in xs:
            x.zero_()
        return batch.cg_solve(bs, xs, rtol=0.0, maxit=iters)

    with ClockSampler(local) as clk:
        ms_b = timed(batched)
    clocks = clk.summary()
    _, infos = batched()
    launches = sum(i["kernel_launches"] for i in infos)

    def sequential():
        for m, b, x in zip(batch.members, bs, xs):
            x.zero_()
            m.cg_solve(b, x, rtol=0.0, maxit=iters)

    ms_s = timed(sequential)
    _, conv = batch.cg_solve(bs, [torch.zeros_like(b) for b in bs], rtol=1e-10, maxit=100000)
    batch.close()
    return {
        "value": round(dofs * iters * K * world / (ms_b / 1e3) / 1e9, 4), "ms_per_step": round(ms_b / K, 3),
        "total_dofs": dofs, "iterations_per_step": iters, "steps": K, "warmup": W,
        "sequential_single_solves": {"value": round(dofs * iters * K * world / (ms_s / 1e3) / 1e9, 4),
                                     "ms_per_step": round(ms_s / K, 3)},
        "batched_over_sequential": round(ms_s / ms_b, 4),
        "solve_rtol_1e-10": {"iterations_min": min(i["iterations"] for i in conv),
                             "iterations_max": max(i["iterations"] for i in conv),
                             "converged": sum(i["converged"] for i in conv)},
        "gpu_launches": launches, "clocks": clocks,
    }


def batch_specs(count: int, rhs_block: bool):
    from paper_2205_08909_gb300 import inputs

    if rhs_block:
        # a block of right-hand sides on one mesh: identical members share the operator data
        return [{"degree": 5, "cells": (48, 48, 48)}] * count
    return inputs.batch_problems(count)


def run_batch(args, world, rank, local):
    """Batched form: args.batch independent seeded problems (degree U{2..8},
    cells U{4..32}^3, deformation U[0, 0.08], final-tensor geometry, random
    right-hand sides) or, with --rhs-block, args.batch right-hand sides on one
    Q5 48^3 mesh; args.iters fixed iterations each."""
    import torch

    from paper_2205_08909_gb300 import build

    build.build()
    torch.cuda.set_device(local)
    prec = args.precision if args.precision != "fp32_inner" else "double_float"
    specs = batch_specs(args.batch, args.rhs_block)
    m = measure_batch(specs, prec, args.steps, args.warmup, args.iters, world, local)
    degrees = [sp["degree"] for sp in specs]
    return {
        "metric": "batched CG GDoF-iterations/s", "value": m["value"], "unit": UNIT, "n_gpus": world,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": m["ms_per_step"], "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": {"fp64": "f64", "double_float": "f32x2 (double-float)"}[prec],
        "data": "synthetic: seeded problems and standard-normal right-hand sides, zero on the boundary",
        "config": {"workload": (f"block of {args.batch} right-hand sides on Q5 48^3" if args.rhs_block
                                else f"batch of {args.batch} problems"), "total_dofs": m["total_dofs"],
                   "degrees": {str(p): degrees.count(p) for p in sorted(set(degrees))},
                   "iterations_per_step": args.iters, "precision": prec,
                   "geometry": "affine" if args.rhs_block else "deformed_tensor",
                   "parallelism": f"replicas x{world}"},
        "sequential_single_solves": m["sequential_single_solves"],
        "batched_over_sequential": m["batched_over_sequential"],
        "solve_rtol_1e-10": m["solve_rtol_1e-10"],
        "gpu_launches": m["gpu_launches"],
        "clocks": m["clocks"],
    }


def main():
    ap = argparse.ArgumentParser(description=__doc__.split("\n")[0])
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=10)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", choices=["ours", "reference"], default="ours")
    ap.add_argument("--workload", default="q4_128cube")
    ap.add_argument("--iters", type=int, default=50, help="CG iterations per step")
    ap.add_argument("--ref-cells", type=int, default=16, help="cells per direction of the oracle sample")
    ap.add_argument("--ref-iters", type=int, default=150, help="iterations of the oracle sample")
    ap.add_argument("--skip-cpu", action="store_true")
    ap.add_argument("--skip-unfused", action="store_true")
    ap.add_argument("--skip-e2e", action="store_true")
    ap.add_argument("--skip-dc", action="store_true", help="skip the FP32-inner defect-correction solve")
    ap.add_argument("--skip-variants", action="store_true", help="skip the FP64 comparators")
    ap.add_argument("--skip-batch", action="store_true", help="skip the short batched and block runs")
    ap.add_argument("--geometry", default="", choices=["", "deformed", "deformed_tensor", "deformed_quadratic"],
                    help="storage of the deformed map: J^{-1} and JxW (10 values per point), the final tensor (6), "
                         "or the tri-quadratic map (27 x 3 coordinates per cell, metric computed per point)")
    ap.add_argument("--batch", type=int, default=0,
                    help="run the batched form on this many seeded problems instead of the headline workload")
    ap.add_argument("--rhs-block", action="store_true",
                    help="with --batch N: N right-hand sides on one Q5 48^3 mesh instead of N different problems")
    ap.add_argument("--tile", default="", help="cells per tile, e.g. 4,4,2 (default: chosen from the degree)")
    ap.add_argument("--precision", default="fp64", choices=["fp64", "double_float", "fp32_inner"],
                    help="arithmetic of the headline fused path")
    ap.add_argument("--x-update", default="delayed", choices=["delayed", "every_iteration"],
                    help="fused forms: Algorithm 5's delayed x update (every other iteration) or x += alpha p "
                         "in every iteration")
    args = ap.parse_args()
    world, rank, local = dist_setup(args)
    if args.impl == "reference":
        line = run_reference(args, world, rank)
    elif args.batch > 0:
        line = run_batch(args, world, rank, local)
    else:
        line = run_ours(args, world, rank, local)
    if line is not None:
        print(json.dumps(line), flush=True)
    if world > 1:
        import torch.distributed as dist

        dist.destroy_process_group()


if __name__ == "__main__":
    main()
