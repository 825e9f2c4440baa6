"""CPU tests of the host-side logic and of the C ABI library (no GPU needed)."""
import ctypes
import os
import subprocess

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def test_numbering_shell_and_tail_enumeration(tmp_path):
    exe = tmp_path / "numbering_check"
    src = os.path.join(ROOT, "tests", "cpp", "numbering_check.cpp")
    cuda_inc = "/usr/local/cuda/include"
    subprocess.run(["g++", "-std=c++17", "-O1", f"-I{cuda_inc}", src, "-o", str(exe)], check=True)
    out = subprocess.run([str(exe)], capture_output=True, text=True)
    assert out.returncode == 0, out.stdout + out.stderr
    assert out.stdout.startswith("ok")


def _lib():
    from paper_2205_08909_gb300 import build
    build.build()
    from paper_2205_08909_gb300 import _binding
    return _binding


def test_library_exports_every_declared_symbol():
    b = _lib()
    lib = ctypes.CDLL(b.LIB_PATH)
    names = b.declared_functions()
    assert len(names) >= 10
    for name in names:
        assert hasattr(lib, name), name


def test_status_strings_without_gpu():
    b = _lib()
    lib = b.load()
    for code in range(8):
        assert lib.mfcg_status_string(code)
    assert b"unknown" in lib.mfcg_status_string(99)


def test_setup_rejects_invalid_arguments_before_touching_the_gpu():
    b = _lib()
    lib = b.load()
    h = ctypes.c_void_p()
    mesh = b.Mesh(4, 4, 4, 0.0)
    geom = b.Geometry(0, 0)
    assert lib.mfcg_setup(None, 2, ctypes.byref(geom), None, None, ctypes.byref(h)) == 1
    assert lib.mfcg_setup(ctypes.byref(mesh), 9, ctypes.byref(geom), None, None, ctypes.byref(h)) == 2
    assert lib.mfcg_setup(ctypes.byref(mesh), 0, ctypes.byref(geom), None, None, ctypes.byref(h)) == 2
    bad = b.Mesh(0, 4, 4, 0.0)
    assert lib.mfcg_setup(ctypes.byref(bad), 2, ctypes.byref(geom), None, None, ctypes.byref(h)) == 1
    deformed_affine = b.Mesh(4, 4, 4, 0.05)
    assert lib.mfcg_setup(ctypes.byref(deformed_affine), 2, ctypes.byref(geom), None, None, ctypes.byref(h)) == 1
    too_big = b.Mesh(4, 4, 4, 0.2)
    g2 = b.Geometry(1, 0)
    assert lib.mfcg_setup(ctypes.byref(too_big), 2, ctypes.byref(g2), None, None, ctypes.byref(h)) == 1
    assert lib.mfcg_n_dofs(None, None) == 1
    assert lib.mfcg_destroy(None) == 0


def test_binding_structs_match_the_c_header(tmp_path):
    """The ctypes mirrors of mfcg_mesh, mfcg_geometry, mfcg_options and
    mfcg_solve_info have the header's size and field offsets."""
    from paper_2205_08909_gb300 import _binding as b

    structs = {"mfcg_mesh": b.Mesh, "mfcg_geometry": b.Geometry, "mfcg_options": b.Options,
               "mfcg_solve_info": b.SolveInfo}
    lines = ["#include <stddef.h>", "#include <stdio.h>", '#include "mfcg.h"', "int main(void) {"]
    for cname, py in structs.items():
        lines.append(f'  printf("{cname} size %zu\\n", sizeof({cname}));')
        for field, _ in py._fields_:
            lines.append(f'  printf("{cname} {field} %zu\\n", offsetof({cname}, {field}));')
    lines += ["  return 0;", "}"]
    src = tmp_path / "layout.c"
    src.write_text("\n".join(lines) + "\n")
    exe = tmp_path / "layout"
    subprocess.run(["gcc", "-std=c11", f"-I{os.path.join(ROOT, 'include')}", str(src), "-o", str(exe)], check=True)
    out = subprocess.run([str(exe)], capture_output=True, text=True, check=True).stdout.split("\n")
    got = {tuple(ln.split()[:2]): int(ln.split()[2]) for ln in out if ln.strip()}
    for cname, py in structs.items():
        assert got[(cname, "size")] == ctypes.sizeof(py), cname
        for field, _ in py._fields_:
            assert got[(cname, field)] == getattr(py, field).offset, (cname, field)
