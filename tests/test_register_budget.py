"""Register budgets of the fused-iteration kernels (CPU: nvcc -Xptxas -v).

With 256 threads per CTA and 65,536 registers per SM, two resident CTAs need
at most 128 registers per thread and three at most 85.  The double-float and
FP64 tiles of degree 4 and 5 are meant to run two CTAs per SM (their node
bricks allow it), the FP32 tiles and the tail kernel three.  These checks
compile the degree-4 and degree-5 translation units for sm_103a with the
library's own flags and read the register counts that ptxas reports, so that a
change of launch bounds or of a kernel body that pushes a kernel past its
budget fails here instead of showing up as a slowdown on the GPU.
"""
import concurrent.futures
import os
import re
import shutil
import subprocess

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
CSRC = os.path.join(ROOT, "paper_2205_08909_gb300", "csrc")
ARCH = ["-gencode", "arch=compute_103a,code=sm_103a"]
FLAGS = ["-O3", "-std=c++17", "-Xptxas", "-v"]

# template arguments: tile_kernel<P, MODE, GEOM, PREC, NC>, tail_kernel<P, MODE, PREC>
MODE_OPERATOR, MODE_CG = 0, 1
AFFINE, DEFORMED, TENSOR = 0, 1, 2
F64, DD, F32 = 0, 1, 2
TWO_CTAS, THREE_CTAS = 128, 85


def _nvcc():
    for cand in (shutil.which("nvcc"), "/usr/local/cuda/bin/nvcc"):
        if cand and os.path.exists(cand):
            return cand
    return None


def _parse(text):
    """{(kind, template args): (registers, spill store bytes)} from ptxas -v."""
    out, cur, spill = {}, None, 0
    for line in text.splitlines():
        m = re.search(r"Compiling entry function '_ZN4mfcg\d+(tile|tail)_kernelI((?:Li\d+E)+)E", line)
        if m:
            cur = (m.group(1), tuple(int(v) for v in re.findall(r"Li(\d+)E", m.group(2))))
            spill = 0
            continue
        m = re.search(r"(\d+) bytes spill stores", line)
        if cur and m:
            spill = int(m.group(1))
        m = re.search(r"Used (\d+) registers", line)
        if cur and m:
            out[cur] = (int(m.group(1)), spill)
            cur = None
    return out


@pytest.fixture(scope="module")
def usage(tmp_path_factory):
    nvcc = _nvcc()
    if nvcc is None:
        pytest.skip("nvcc not available")
    tmp = tmp_path_factory.mktemp("regs")

    def compile_one(p):
        src = os.path.join(CSRC, f"tile_p{p}.cu")
        res = subprocess.run([nvcc, *ARCH, *FLAGS, "-c", src, "-o", str(tmp / f"p{p}.o")],
                             capture_output=True, text=True)
        assert res.returncode == 0, res.stderr[-2000:]
        return _parse(res.stdout + res.stderr)

    with concurrent.futures.ThreadPoolExecutor(max_workers=2) as ex:
        parts = list(ex.map(compile_one, (4, 5)))
    merged = {}
    for part in parts:
        merged.update(part)
    return merged


@pytest.mark.slow
@pytest.mark.parametrize("P", [4, 5])
def test_fused_tiles_fit_two_ctas_per_sm(usage, P):
    for prec in (F64, DD):
        regs, spill = usage[("tile", (P, MODE_CG, AFFINE, prec, 1))]
        # a few bytes of spill are the compiler's choice for a tighter target
        assert regs <= TWO_CTAS and spill <= 16, (P, prec, regs, spill)
    for geom in (DEFORMED, TENSOR):
        regs, _ = usage[("tile", (P, MODE_CG, geom, DD, 1))]
        assert regs <= TWO_CTAS, (P, geom, regs)
    # the operator pass of the unfused and semi-fused comparators and of A x0
    regs, _ = usage[("tile", (P, MODE_OPERATOR, AFFINE, DD, 1))]
    assert regs <= TWO_CTAS, (P, regs)


@pytest.mark.slow
@pytest.mark.parametrize("P", [4, 5])
def test_fp32_tiles_and_tail_fit_three_ctas_per_sm(usage, P):
    for geom in (AFFINE, DEFORMED, TENSOR):
        for nc in (1, 3):
            regs, _ = usage[("tile", (P, MODE_CG, geom, F32, nc))]
            assert regs <= THREE_CTAS, (P, geom, nc, regs)
    for prec in (F64, DD, F32):
        regs, _ = usage[("tail", (P, MODE_CG, prec))]
        assert regs <= THREE_CTAS, (P, prec, regs)
