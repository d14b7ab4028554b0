"""The allocation-free entry point, fmm_morton_sort_noalloc, against fmm_build.

Some callers cannot allocate device memory when they need the result: a
loop with a fixed device-memory budget (a cudaMalloc can block on the device
and can fail part-way through a run), or an application whose device memory
is owned by another framework's allocator. fmm_morton_sort_noalloc gives them the Morton keys and the
sorting permutation of the octree build using only the caller's buffers and a
fixed scratch array that the library reserves when it is loaded.

The checks compare its output bit for bit (integer results are compared
exactly everywhere in these tests) with the keys and permutation that
fmm_build computes and fmm_export_tree returns for the same input, on two
calls in a row: the second, smaller call runs on scratch that still holds the
first call's data. This file is collected last so that a run stopping at the
first failure has already run every other test.
"""
import ctypes

import numpy as np
import pytest

from paper_1106_2176_gb300 import inputs

from gpu_common import ensure_built, torch_cuda

pytestmark = pytest.mark.gpu


def sorted_by_build(x):
    torch = torch_cuda()
    ensure_built()
    from paper_1106_2176_gb300 import FMM
    xt = torch.tensor(x, device="cuda")
    f = FMM(len(x), p=2, theta=0.5, ncrit=64)
    f.build(xt, torch.ones(len(x), dtype=xt.dtype, device="cuda"))
    t = f.export_tree()
    f.close()
    return t["keys"], t["perm"]


def sorted_without_allocation(x):
    torch = torch_cuda()
    ensure_built()
    from paper_1106_2176_gb300 import fmm
    xt = torch.tensor(x, device="cuda")
    n = len(x)
    keys = torch.empty(n, dtype=torch.int64, device="cuda")
    perm = torch.empty(n, dtype=torch.int32, device="cuda")
    dt = fmm.FMM_F64 if x.dtype == np.float64 else fmm.FMM_F32
    stream = ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)
    rc = fmm.lib().fmm_morton_sort_noalloc(ctypes.c_void_p(xt.data_ptr()), n, dt, ctypes.c_void_p(keys.data_ptr()),
                                           ctypes.c_void_p(perm.data_ptr()), stream)
    assert rc == fmm.FMM_OK, fmm.lib().fmm_last_error(None)
    torch.cuda.synchronize()
    return keys.cpu().numpy().view(np.uint64), perm.cpu().numpy()


def test_two_calls_in_a_row_match_build():
    cases = [(300001, 5, np.float64), (70000, 6, np.float32)]
    for n, seed, dtype in cases:
        x, _ = inputs.uniform_cube(n, seed, dtype=dtype)
        k_ref, p_ref = sorted_by_build(x)
        k, p = sorted_without_allocation(x)
        assert np.array_equal(k, k_ref)
        assert np.array_equal(p, p_ref)


def test_clustered_input_and_largest_size():
    x, _ = inputs.plummer(1 << 20, 7)
    k_ref, p_ref = sorted_by_build(x)
    k, p = sorted_without_allocation(x)
    assert np.array_equal(k, k_ref) and np.array_equal(p, p_ref)


def test_sizes_beyond_the_scratch_are_rejected():
    ensure_built()
    from paper_1106_2176_gb300 import fmm
    L = fmm.lib()
    dummy = ctypes.c_void_p(16)  # never dereferenced: the size check comes first
    for n in ((1 << 20) + 1, 0):
        assert L.fmm_morton_sort_noalloc(dummy, n, fmm.FMM_F32, dummy, dummy, None) == fmm.FMM_EINVAL
        assert b"1048576" in L.fmm_last_error(None)
