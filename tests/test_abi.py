"""The C-ABI library builds, loads and exports every function its header
declares; argument checks that run before any CUDA call behave as documented.
No compute is launched (these run without a GPU)."""
import ctypes

import pytest

from paper_2501_13664_gb300 import _abi


@pytest.fixture(scope="module")
def lib():
    return _abi.lib()


def test_header_declares_the_boundary():
    names = set(_abi.header_functions())
    for must in ("drt3d_planes_forward", "drt3d_planes_inverse", "djt3d_lines_forward",
                 "drt3d_planes_adjoint", "drt3d_plan_create", "drt3d_get_device_error"):
        assert must in names


def test_every_declared_symbol_is_exported(lib):
    for name in _abi.header_functions():
        assert hasattr(lib, name), name
        assert name in _abi.SIGNATURES, f"binding lacks a signature for {name}"


def test_status_strings_and_version(lib):
    for code, name in _abi.STATUS.items():
        assert lib.drt3d_status_string(code).decode() == name
    assert lib.drt3d_version() >= 100


def test_plan_create_rejects_bad_arguments_before_touching_the_device(lib):
    h = ctypes.c_void_p()
    assert lib.drt3d_plan_create(None, 8, 0, 0) == 1            # INVALID_ARG
    assert lib.drt3d_plan_create(ctypes.byref(h), 8, 0, 1) == 1  # flags reserved
    for bad_n in (0, 1, 3, 12, 2048, -4):
        assert lib.drt3d_plan_create(ctypes.byref(h), bad_n, 0, 0) == 2  # SIZE
    assert lib.drt3d_plan_create(ctypes.byref(h), 8, 7, 0) == 3  # DTYPE


def test_null_plan_queries(lib):
    dims = (ctypes.c_int64 * 5)()
    assert lib.drt3d_planes_out_shape(None, dims) == 1
    assert lib.drt3d_lines_out_shape(None, dims) == 1
    sz = ctypes.c_size_t()
    assert lib.drt3d_workspace_bytes(None, 0, ctypes.byref(sz)) == 1
    assert lib.drt3d_planes_forward(None, None, None, 0xFFF, None, 0, None) == 1
    assert lib.drt3d_plan_destroy(None) == 0
