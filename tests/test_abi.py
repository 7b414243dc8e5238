"""CPU checks of the C-ABI library: it builds, loads, exports every symbol
include/evx.h declares, and its host-side argument validation works
(no CUDA work is issued by any call made here)."""
import ctypes
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
HEADERS = [os.path.join(ROOT, "include", h) for h in ("evx.h", "evx_nn.h")]


@pytest.fixture(scope="module")
def lib():
    from paper_2507_21748_gb300.build import build_lib
    path = build_lib()
    return ctypes.CDLL(path)


def declared_functions():
    names = set()
    for h in HEADERS:
        text = re.sub(r"/\*.*?\*/", "", open(h).read(), flags=re.S)
        names |= set(re.findall(r"\b(evx_\w+)\s*\(", text))
    return sorted(names)


def test_header_declares_entry_points():
    names = declared_functions()
    for required in ("evx_grid_create", "evx_ch_step", "evx_ch_adjoint", "evx_energy"):
        assert required in names


def test_exports_every_declared_symbol(lib):
    missing = [n for n in declared_functions() if not hasattr(lib, n)]
    assert not missing, missing


def test_binding_lists_every_declared_symbol():
    import paper_2507_21748_gb300.evx as evx
    import paper_2507_21748_gb300.surrogate as sur
    assert sorted(evx.EXPORTS + sur.NN_EXPORTS) == declared_functions()


class Params(ctypes.Structure):
    _fields_ = [("dt", ctypes.c_double), ("M", ctypes.c_double), ("kappa", ctypes.c_double),
                ("h", ctypes.c_double)]


@pytest.mark.parametrize("shape", [(7, 8, 8), (8, 8, 6), (14, 8, 8), (8, 2048, 8), (8, 8, 10 * 7)])
def test_bad_sizes_rejected(lib, shape):
    lib.evx_grid_create.argtypes = [ctypes.c_int] * 3 + [Params, ctypes.c_void_p,
                                                         ctypes.POINTER(ctypes.c_void_p)]
    lib.evx_last_error.restype = ctypes.c_char_p
    lib.evx_last_error.argtypes = [ctypes.c_void_p]
    h = ctypes.c_void_p(123)
    s = lib.evx_grid_create(*shape, Params(0.1, 1, 1, 1), None, ctypes.byref(h))
    assert s == 2  # EVX_ERR_SIZE
    assert h.value is None
    assert b"unsupported" in lib.evx_last_error(None)


def test_bad_params_rejected(lib):
    lib.evx_grid_create.argtypes = [ctypes.c_int] * 3 + [Params, ctypes.c_void_p,
                                                         ctypes.POINTER(ctypes.c_void_p)]
    h = ctypes.c_void_p()
    for p in (Params(-0.1, 1, 1, 1), Params(0.1, -1, 1, 1), Params(0.1, 1, 1, 0),
              Params(float("nan"), 1, 1, 1)):
        assert lib.evx_grid_create(8, 8, 8, p, None, ctypes.byref(h)) == 1  # EVX_ERR_ARG


def test_null_arguments(lib):
    lib.evx_grid_create.argtypes = [ctypes.c_int] * 3 + [Params, ctypes.c_void_p, ctypes.c_void_p]
    assert lib.evx_grid_create(8, 8, 8, Params(0.1, 1, 1, 1), None, None) == 1
    lib.evx_ch_step.argtypes = [ctypes.c_void_p, ctypes.c_int]
    assert lib.evx_ch_step(None, 1) == 1
    lib.evx_energy.argtypes = [ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p]
    assert lib.evx_energy(None, None, None) == 1
    assert lib.evx_grid_destroy(None) == 0


def test_model_and_engine_entry_points_reject_bad_arguments(lib):
    """Host-side argument checks of the model and engine calls (no device work)."""
    lib.evx_set_model.argtypes = [ctypes.c_void_p, ctypes.c_int]
    lib.evx_get_model.argtypes = [ctypes.c_void_p]
    lib.evx_get_model.restype = ctypes.c_int
    lib.evx_step.argtypes = [ctypes.c_void_p, ctypes.c_int]
    assert lib.evx_set_model(None, 1) == 1   # EVX_ERR_ARG
    assert lib.evx_get_model(None) == -1
    assert lib.evx_step(None, 1) == 1
    lib.evx_nn_set_conv_engine.argtypes = [ctypes.c_int]
    lib.evx_nn_conv_engine.restype = ctypes.c_int
    assert lib.evx_nn_set_conv_engine(7) == 1
    assert lib.evx_nn_set_conv_engine(1) == 0 and lib.evx_nn_conv_engine() == 1
    assert lib.evx_nn_set_conv_engine(0) == 0 and lib.evx_nn_conv_engine() == 0
    vp, i = ctypes.c_void_p, ctypes.c_int
    lib.evx_nn_conv3d.argtypes = [vp] * 6 + [i] * 7 + [vp]
    assert lib.evx_nn_conv3d(None, None, None, None, None, None, 1, 1, 2, 64, 32, 32, 0, None) == 1
    one = ctypes.c_void_p(16)  # never dereferenced: the size check comes first
    assert lib.evx_nn_conv3d(one, one, None, one, None, None, 1, 1, 3, 64, 32, 32, 0, None) == 2  # Y odd
    assert lib.evx_nn_conv3d(one, one, None, one, None, None, 1, 1, 2, 48, 32, 32, 0, None) == 2  # Z % 64


def test_checkpoint_and_query_entry_points_reject_null(lib):
    """evx_save / evx_load / evx_step_count / evx_get_params validate their
    arguments on the host before touching a grid or a file."""
    vp = ctypes.c_void_p
    lib.evx_save.argtypes = [vp, ctypes.c_char_p]
    lib.evx_load.argtypes = [vp, ctypes.c_char_p]
    lib.evx_step_count.argtypes = [vp, vp]
    lib.evx_get_params.argtypes = [vp, vp]
    assert lib.evx_save(None, b"/nonexistent/x") == 1
    assert lib.evx_load(None, b"/nonexistent/x") == 1
    assert lib.evx_step_count(None, None) == 1
    assert lib.evx_get_params(None, None) == 1
