"""The allocation-free operator entry point, mfcg_apply_operator_static.

It serves callers that cannot allocate device memory (programs whose device
memory belongs to their own pool allocator, loops that must not call
cudaMalloc/cudaFree because those calls can synchronise the device).  Its
scratch is a fixed array in device memory shared by all calls, so this file
runs last: two calls in a row must reproduce the regular entry point,
whatever earlier tests left in that array.
"""
import ctypes

import pytest
import torch

from paper_2205_08909_gb300 import inputs

pytestmark = pytest.mark.gpu

OP_TOL = 1e-13  # the operator tolerance of the other GPU tests


@pytest.fixture(scope="module")
def lib():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2205_08909_gb300 import _binding, build

    build.build()
    lib = _binding.load()
    lib.mfcg_apply_operator_static.argtypes = [ctypes.POINTER(_binding.Mesh), ctypes.c_int, ctypes.c_void_p,
                                               ctypes.c_void_p, ctypes.c_void_p]
    lib.mfcg_apply_operator_static.restype = ctypes.c_int
    return lib


@pytest.mark.parametrize("degree,cells", [(2, (8, 8, 8)), (4, (9, 5, 6)), (4, (32, 32, 32)), (6, (4, 3, 5)),
                                          (1, (7, 6, 5)), (8, (2, 3, 2))])
def test_static_operator_matches_regular_entry_point_twice(lib, degree, cells):
    import paper_2205_08909_gb300 as mfcg
    from paper_2205_08909_gb300 import _binding

    prob = mfcg.Problem(degree, cells)
    src = torch.from_numpy(inputs.random_vector(prob.n_dofs, salt=99)).cuda()
    ref = prob.apply_operator(src)
    mesh = _binding.Mesh(cells[0], cells[1], cells[2], 0.0)
    stream = ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)
    scale = ref.abs().max().item()
    for _ in range(2):
        dst = torch.full_like(src, float("nan"))
        st = lib.mfcg_apply_operator_static(ctypes.byref(mesh), degree, ctypes.c_void_p(src.data_ptr()),
                                            ctypes.c_void_p(dst.data_ptr()), stream)
        assert st == 0
        torch.cuda.synchronize()
        assert (dst - ref).abs().max().item() <= OP_TOL * scale
    prob.close()


def test_static_operator_rejects_meshes_beyond_its_scratch(lib):
    from paper_2205_08909_gb300 import _binding

    big = _binding.Mesh(128, 128, 128, 0.0)
    dummy = torch.zeros(8, dtype=torch.float64, device="cuda")
    other = torch.zeros(8, dtype=torch.float64, device="cuda")
    st = lib.mfcg_apply_operator_static(ctypes.byref(big), 4, ctypes.c_void_p(dummy.data_ptr()),
                                        ctypes.c_void_p(other.data_ptr()), None)
    assert st == 8
    assert b"scratch" in lib.mfcg_status_string(st)
    deformed = _binding.Mesh(4, 4, 4, 0.05)
    assert lib.mfcg_apply_operator_static(ctypes.byref(deformed), 4, ctypes.c_void_p(dummy.data_ptr()),
                                          ctypes.c_void_p(other.data_ptr()), None) == 1
