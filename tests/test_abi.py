"""Host-side checks of the C ABI that need no GPU: the library builds, loads,
exports every function include/pppm.h declares, and validates arguments."""
import ctypes
import os
import re

import pytest

from paper_2504_15508_gb300 import _native as N

HEADER = os.path.join(os.path.dirname(os.path.dirname(os.path.abspath(__file__))), "include", "pppm.h")


def _declared_functions():
    src = open(HEADER).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    return sorted(set(re.findall(r"\b(pppm_\w+)\s*\(", src)))


def test_header_functions_exported(pppm_lib):
    names = _declared_functions()
    assert "pppm_create" in names and "pppm_compute" in names
    for name in names:
        assert hasattr(pppm_lib, name), name
    # the binding declares signatures for exactly what the header declares
    assert set(N.SIGNATURES) == set(names)


def _create(lib, box=(10.0, 10.0, 10.0), mesh=(32, 32, 32), order=5, beta=0.4, prec=N.PPPM_FP32):
    b = (ctypes.c_double * 3)(*box)
    m = (ctypes.c_int * 3)(*mesh)
    h = ctypes.c_void_p()
    rc = lib.pppm_create(b, m, order, beta, prec, ctypes.byref(h))
    if rc == N.PPPM_OK:
        lib.pppm_destroy(h)
    return rc


def test_create_validates_arguments(pppm_lib):
    L = pppm_lib
    assert _create(L, mesh=(32, 32, 7)) == N.PPPM_ERR_BAD_MESH      # 7 is not 2^a 3^b 5^c
    assert _create(L, mesh=(4, 32, 32)) == N.PPPM_ERR_BAD_MESH      # smaller than the order
    assert _create(L, mesh=(4096, 32, 32)) == N.PPPM_ERR_BAD_MESH   # too large
    assert _create(L, order=1) == N.PPPM_ERR_BAD_ORDER
    assert _create(L, order=8) == N.PPPM_ERR_BAD_ORDER
    assert _create(L, box=(10.0, -1.0, 10.0)) == N.PPPM_ERR_BAD_BOX
    assert _create(L, box=(10.0, float("nan"), 10.0)) == N.PPPM_ERR_BAD_BOX
    assert _create(L, beta=0.0) == N.PPPM_ERR_INVALID_ARG
    assert _create(L, prec=3) == N.PPPM_ERR_INVALID_ARG
    assert L.pppm_create(None, None, 5, 0.4, 1, None) == N.PPPM_ERR_INVALID_ARG


def test_create_without_device_reports_cuda_error(pppm_lib):
    import torch
    if torch.cuda.is_available():
        pytest.skip("a GPU is present")
    assert _create(pppm_lib) == N.PPPM_ERR_CUDA


def test_null_plan_calls_are_rejected(pppm_lib):
    L = pppm_lib
    assert L.pppm_compute(None, None, None, None, 0, None, None, None) == N.PPPM_ERR_INVALID_ARG
    assert L.pppm_status(None) == N.PPPM_ERR_INVALID_ARG
    assert L.pppm_reserve(None, 10) == N.PPPM_ERR_INVALID_ARG
    L.pppm_destroy(None)
    for code in range(-8, 1):
        assert N.strerror(code) != "unknown error"


def test_corrector_calls_validate_arguments(pppm_lib):
    from oracle import mlp
    L = pppm_lib
    assert L.pppm_corr_nparams() == mlp.N_PARAMS == 7491
    h = ctypes.c_void_p()
    assert L.pppm_corr_create(None, ctypes.byref(h)) == N.PPPM_ERR_INVALID_ARG
    assert L.pppm_corr_create(None, None) == N.PPPM_ERR_INVALID_ARG
    assert L.pppm_set_potential(None, 1) == N.PPPM_ERR_INVALID_ARG
    assert L.pppm_set_dependent_launch(None, 1) == N.PPPM_ERR_INVALID_ARG
    assert L.pppm_corr_set_weights(None, None, 1.0, 1.0) == N.PPPM_ERR_INVALID_ARG
    assert L.pppm_corr_get_weights(None, None, None, None) == N.PPPM_ERR_INVALID_ARG
    assert L.pppm_corr_features(None, None, None, None, None, 0, None, None) == N.PPPM_ERR_INVALID_ARG
    assert L.pppm_corr_forward(None, None, None, 0, None) == N.PPPM_ERR_INVALID_ARG
    assert L.pppm_corr_apply(None, None, None, None, None, 0, None, None, None) == N.PPPM_ERR_INVALID_ARG
    assert L.pppm_corr_grad(None, None, None, None, 1, None, 1, None, None) == N.PPPM_ERR_INVALID_ARG
    assert L.pppm_corr_train_step(None, None, None, None, 1, None, 1, 1e-3, None) == N.PPPM_ERR_INVALID_ARG
    assert L.pppm_corr_calibrate(None, None, None, None, None, 1, None) == N.PPPM_ERR_INVALID_ARG
    assert L.pppm_corr_targets(None, None, None, None, None, 0, None) == N.PPPM_ERR_INVALID_ARG
    assert L.pppm_corr_get_scales(None, None, None) == N.PPPM_ERR_INVALID_ARG
    assert L.pppm_corr_save(None, b"x") == N.PPPM_ERR_INVALID_ARG
    assert L.pppm_corr_load(None, b"x") == N.PPPM_ERR_INVALID_ARG
    L.pppm_corr_destroy(None)


def test_wc_fold_validates_arguments(pppm_lib):
    L = pppm_lib
    assert L.pppm_wc_fold(None, 5, 0, None, None, None, None, None, None, None, None) == N.PPPM_ERR_INVALID_ARG
    assert L.pppm_wc_fold_f32(None, -1, 0, None, None, None, None, None, None, None, None) == N.PPPM_ERR_INVALID_ARG
    assert L.pppm_wc_fold(None, 0, 0, None, None, None, None, None, None, None, None) == N.PPPM_OK


def test_graph_calls_validate_arguments(pppm_lib):
    L = pppm_lib
    h = ctypes.c_void_p()
    assert L.pppm_graph_create(None, None, None, None, 1, None, None, None, ctypes.byref(h)) == N.PPPM_ERR_INVALID_ARG
    assert L.pppm_graph_create_f32(None, None, None, None, 1, None, None, None, None) == N.PPPM_ERR_INVALID_ARG
    assert L.pppm_graph_launch(None, None, None, None) == N.PPPM_ERR_INVALID_ARG
    assert L.pppm_graph_launch_f32(None, None, None, None) == N.PPPM_ERR_INVALID_ARG
    L.pppm_graph_destroy(None)


def test_batch_set_dft_validates(pppm_lib):
    assert pppm_lib.pppm_batch_set_dft(None, 18) == N.PPPM_ERR_INVALID_ARG


def test_batch_set_quantized_validates(pppm_lib):
    assert pppm_lib.pppm_batch_set_quantized(None, 4, 1e7) == N.PPPM_ERR_INVALID_ARG


def test_wait_hooks_validate_arguments(pppm_lib):
    assert pppm_lib.pppm_set_wait_limit(None, 10) == N.PPPM_ERR_INVALID_ARG
    assert pppm_lib.pppm_batch_set_wait_probe(None, 1) == N.PPPM_ERR_INVALID_ARG


def test_corrector_feature_sets_validate_arguments(pppm_lib):
    h = ctypes.c_void_p()
    assert pppm_lib.pppm_corr_create_features(None, N.PPPM_CORR_STATED, ctypes.byref(h)) == N.PPPM_ERR_INVALID_ARG
    assert pppm_lib.pppm_corr_param_count(None) == N.PPPM_ERR_INVALID_ARG
    assert pppm_lib.pppm_corr_feature_width(None) == N.PPPM_ERR_INVALID_ARG


def test_batch_set_launch_validates(pppm_lib):
    assert pppm_lib.pppm_batch_set_launch(None, N.PPPM_BATCH_STAGED) == N.PPPM_ERR_INVALID_ARG


def test_corrector_forward_options_validate_arguments(pppm_lib):
    assert pppm_lib.pppm_corr_set_forward(None, N.PPPM_FORWARD_TCGEN05) == N.PPPM_ERR_INVALID_ARG
    assert pppm_lib.pppm_corr_set_wait_limit(None, 10) == N.PPPM_ERR_INVALID_ARG
    assert pppm_lib.pppm_corr_forward(None, None, None, 1, None) == N.PPPM_ERR_INVALID_ARG
