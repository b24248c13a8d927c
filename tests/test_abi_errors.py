"""Error behaviour of the C ABI as include/ds.h states it, on the CPU:
invalid arguments are refused (DS_ERR_INVALID_ARG, with a message from
ds_last_error) before any CUDA call, NULL handles are harmless, and a valid
request on a host without a GPU fails with DS_ERR_CUDA: there is no CPU
fallback."""
import ctypes

import numpy as np
import pytest

torch = pytest.importorskip("torch")


@pytest.fixture(scope="module")
def ds():
    from paper_2310_07551_gb300 import ds as _ds
    try:
        _ds.lib()
    except ImportError as e:
        pytest.skip(str(e))
    return _ds


def last_error(ds):
    return ds.lib().ds_last_error().decode()


def test_invalid_grids_and_arguments_are_refused(ds):
    L = ds.lib()
    out = ctypes.c_void_p()
    A = np.zeros(64)
    for d, n, msg in [(1, (8,), "d must be"), (5, (8, 8, 8, 8), "d must be"), (2, (8, 1), "n_mu")]:
        g = ds.make_grid(n) if len(n) <= 4 else ds.Grid()
        g.d = d
        assert L.ds_phi_setup(ctypes.byref(g), A.ctypes.data, 0, 1e-3, ctypes.byref(out), None) == \
            ds.DS_ERR_INVALID_ARG
        assert msg in last_error(ds)
    g = ds.make_grid((8, 8))
    assert L.ds_phi_setup(ctypes.byref(g), A.ctypes.data, 0, 0.0, ctypes.byref(out), None) == \
        ds.DS_ERR_INVALID_ARG
    assert "tau" in last_error(ds)
    assert L.ds_phi_setup_ex(ctypes.byref(g), A.ctypes.data, 0, 1e-3, 99, ctypes.byref(out), None) == \
        ds.DS_ERR_INVALID_ARG
    assert "scheme" in last_error(ds)
    big = ds.make_grid((128, 64))   # 8192 points: above the dense scheme's limit
    assert L.ds_phi_setup_ex(ctypes.byref(big), A.ctypes.data, 0, 1e-3, ds.SCHEMES["exprk3_dense"],
                             ctypes.byref(out), None) == ds.DS_ERR_UNSUPPORTED
    assert L.ds_tucker(ctypes.byref(g), None, None, None, 0, 0, None) == ds.DS_ERR_INVALID_ARG
    assert L.ds_batch_create(0, None, None, None, None, 0, ctypes.byref(out)) == ds.DS_ERR_INVALID_ARG


def test_null_handles(ds):
    L = ds.lib()
    i = ctypes.c_int()
    i64 = ctypes.c_int64()
    f2 = (ctypes.c_float * 2)()
    f16 = (ctypes.c_float * 16)()
    fa, fb = ctypes.c_float(), ctypes.c_float()
    refused = [
        L.ds_step(None, None, None),
        L.ds_integrate(None, None, 1, None),
        L.ds_plan_sync(None, None, 0),
        L.ds_plan_tuning_ex(None, 0, 0, ctypes.byref(i), ctypes.byref(i64), ctypes.byref(i), f16),
        L.ds_plan_streamk_times(None, 0, 0, f2),
        L.ds_plan_tile_order(None, 0, 0, ctypes.byref(i), f2),
        L.ds_plan_set_tile_order(None, 0, 0, 1),
        L.ds_plan_set_tiles(None, 0, 0, 256, 1),
        L.ds_plan_fusion(None, 0, ctypes.byref(i), ctypes.byref(fa), ctypes.byref(fb)),
        L.ds_plan_set_fusion(None, 0, 1),
        L.ds_batch_integrate(None, None, 1, None),
        L.ds_batch_fusion(None, 0, ctypes.byref(i), ctypes.byref(fa), ctypes.byref(fb)),
        L.ds_batch_tile_order(None, 0, ctypes.byref(i), f2),
        L.ds_batch_set_fusion(None, 0, 1),
    ]
    assert all(r == ds.DS_ERR_INVALID_ARG for r in refused), refused
    assert L.ds_plan_kernels_per_step(None) == -1
    assert L.ds_batch_kernels_per_step(None) == -1
    assert L.ds_plan_destroy(None) == ds.DS_OK
    assert L.ds_batch_destroy(None) == ds.DS_OK
    assert L.ds_phi_set_destroy(None) == ds.DS_OK


@pytest.mark.skipif(torch.cuda.is_available(), reason="checks the behaviour without a GPU")
def test_valid_request_without_gpu_fails_loudly(ds):
    L = ds.lib()
    g = ds.make_grid((8, 8))
    X = np.zeros(64)
    Y = np.zeros(64)
    Ls = (ctypes.c_void_p * 2)(np.eye(8).ctypes.data, np.eye(8).ctypes.data)
    assert L.ds_tucker(ctypes.byref(g), X.ctypes.data, Y.ctypes.data, Ls, 0, 0, None) == ds.DS_ERR_CUDA
    assert "no CUDA device" in last_error(ds)
