"""The C-ABI library builds, loads and exports every entry point include/fmm.h
declares; argument checks that need no GPU."""
import ctypes
import os

import pytest

from paper_1106_2176_gb300 import _build, fmm

from conftest import gpu_available


@pytest.fixture(scope="module")
def L():
    _build.build()
    return fmm.lib()


def test_header_declares_the_boundary():
    names = fmm.declared_symbols()
    for required in ("fmm_create", "fmm_build", "fmm_evaluate", "fmm_destroy", "fmm_set_precision",
                     "fmm_set_stream", "fmm_get_stats", "fmm_export_tree", "fmm_last_error"):
        assert required in names


def test_library_exports_every_declared_symbol(L):
    for name in fmm.declared_symbols():
        assert hasattr(L, name), name


def test_library_is_sm103a_only():
    # the build passes one -gencode: compute_103a -> sm_103a
    assert _build.ARCH == ["-gencode", "arch=compute_103a,code=sm_103a"]


@pytest.mark.parametrize("args", [(0, 8, 0.5, 64), (100, 0, 0.5, 64), (100, 21, 0.5, 64),
                                  (100, 8, 0.0, 64), (100, 8, 1.0, 64), (100, 8, float("nan"), 64),
                                  (100, 8, 0.5, 0)])
def test_create_rejects_bad_arguments(L, args):
    h = ctypes.c_void_p()
    rc = L.fmm_create(*args, ctypes.byref(h))
    assert rc == fmm.FMM_EINVAL and not h.value
    assert L.fmm_last_error(None)


def test_null_handle_is_rejected(L):
    assert L.fmm_build(None, None, None, 1, 0) == fmm.FMM_EINVAL
    assert L.fmm_evaluate(None, None, None) == fmm.FMM_EINVAL
    assert L.fmm_destroy(None) == fmm.FMM_EINVAL


@pytest.mark.skipif(gpu_available(), reason="checks the no-device path")
def test_create_without_device_fails_cleanly(L):
    h = ctypes.c_void_p()
    rc = L.fmm_create(1000, 8, 0.5, 64, ctypes.byref(h))
    assert rc in (fmm.FMM_ENODEV, fmm.FMM_ECUDA) and not h.value


def test_measurement_entry_points_check_arguments(L):
    out = ctypes.c_double()
    # unknown kind, reps out of range, bad MMA width, NULL output: rejected
    # before any device call
    assert L.fmm_measure_peak(7, 0, 3, ctypes.byref(out)) == fmm.FMM_EINVAL
    assert L.fmm_measure_peak(fmm.FMM_PEAK_FP32_FMA, 0, 0, ctypes.byref(out)) == fmm.FMM_EINVAL
    assert L.fmm_measure_peak(fmm.FMM_PEAK_TF32_MMA, 64, 3, ctypes.byref(out)) == fmm.FMM_EINVAL
    assert L.fmm_measure_peak(fmm.FMM_PEAK_FP32_FMA, 0, 3, None) == fmm.FMM_EINVAL
    assert L.fmm_get_stats_mean(None, 1, None) == fmm.FMM_EINVAL


def test_batch_entry_points_check_arguments(L):
    # NULL arrays, nsys < 1, NULL batch or outputs, bad pass: rejected before
    # any device call
    b = ctypes.c_void_p(1234)
    assert L.fmm_batch_create(None, 1, None, None, ctypes.byref(b)) == fmm.FMM_EINVAL
    assert b.value is None
    arr = (ctypes.c_void_p * 1)(None)
    assert L.fmm_batch_create(arr, 0, arr, arr, ctypes.byref(b)) == fmm.FMM_EINVAL
    assert L.fmm_batch_create(arr, 1, arr, arr, None) == fmm.FMM_EINVAL
    assert L.fmm_batch_create(arr, 1, arr, arr, ctypes.byref(b)) == fmm.FMM_EINVAL
    assert L.fmm_batch_evaluate(None, None) == fmm.FMM_EINVAL
    e, k = ctypes.c_int(), ctypes.c_int64()
    assert L.fmm_batch_status(None, ctypes.byref(e), ctypes.byref(k)) == fmm.FMM_EINVAL
    i = [ctypes.c_int() for _ in range(4)]
    assert L.fmm_batch_items(None, 0, 0, *[ctypes.byref(v) for v in i]) == fmm.FMM_EINVAL
    assert L.fmm_batch_withhold(None, 0, 0) == fmm.FMM_EINVAL
    assert L.fmm_batch_destroy(None) == fmm.FMM_EINVAL
    assert b"fmm_batch" in L.fmm_last_error(None)


def test_m2l_pool_setter_checks_arguments(L):
    assert L.fmm_set_m2l_pool(None, 512) == fmm.FMM_EINVAL


def test_m2l_lattice_setter_checks_arguments(L):
    assert L.fmm_set_m2l_lattice(None, 1) == fmm.FMM_EINVAL
    assert b"fmm_set_m2l_lattice" in L.fmm_last_error(None)


def test_stats_layout_matches_the_header():
    # the ctypes mirror of fmm_stats lists the header's fields in order
    import re
    hdr = open(os.path.join(os.path.dirname(__file__), "..", "include", "fmm.h")).read()
    body = hdr[hdr.index("typedef struct {\n    int64_t n;  "):]
    body = body[:body.index("} fmm_stats;")]
    names = re.findall(r"\b(\w+)(?:\[\d+\])?\s*[;,]", re.sub(r"/\*.*?\*/", "", body, flags=re.S))
    assert names == [f[0] for f in fmm.fmm_stats._fields_]
