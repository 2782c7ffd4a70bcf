"""CPU-only checks of the C-ABI library: it builds for sm_103a, loads, exports
every entry point include/glrm.h declares, and rejects bad arguments on the
host before touching a GPU."""
import ctypes
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def lib():
    from paper_1410_0342_gb300 import build
    path = build.build()
    return ctypes.CDLL(path)


def declared_functions():
    names = []
    for h in sorted(os.listdir(os.path.join(ROOT, "include"))):
        if h.endswith(".h"):
            text = open(os.path.join(ROOT, "include", h)).read()
            text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
            names += re.findall(r"\b(glrm_\w+)\s*\(", text)
    return sorted(set(names))


def test_header_declares_entry_points():
    names = declared_functions()
    for n in ("glrm_create", "glrm_set_observed", "glrm_set_factors", "glrm_get_factors",
              "glrm_sweep", "glrm_objective", "glrm_grad", "glrm_grad_at", "glrm_predict",
              "glrm_get_state", "glrm_set_state", "glrm_last_error", "glrm_destroy",
              "glrm_set_offset", "glrm_column_stats", "glrm_set_column_scale", "glrm_proxprox_sweep",
              "glrm_embed_losses", "glrm_embed_size", "glrm_embed_features", "glrm_decode_features",
              "glrm_set_reg_weights", "glrm_certificate", "glrm_regularization_path", "glrm_svd_init"):
        assert n in names


def test_every_declared_symbol_is_exported(lib):
    for name in declared_functions():
        assert hasattr(lib, name), name


def _create(lib, m, n, k, losses, rx=(0, 0.0), ry=(0, 0.0), prec=1):
    class L(ctypes.Structure):
        _fields_ = [("kind", ctypes.c_int32), ("levels", ctypes.c_int32),
                    ("param", ctypes.c_double)]
    arr = (L * max(1, len(losses)))(*[L(x[0], x[2], x[1]) for x in losses])
    h = ctypes.c_void_p()
    lib.glrm_create.restype = ctypes.c_int
    lib.glrm_global_error.restype = ctypes.c_char_p
    rc = lib.glrm_create(ctypes.c_int64(m), ctypes.c_int64(n), ctypes.c_int32(k), arr,
                         ctypes.c_int32(rx[0]), ctypes.c_double(rx[1]), ctypes.c_int32(ry[0]),
                         ctypes.c_double(ry[1]), ctypes.c_int32(prec), None, ctypes.byref(h))
    return rc, lib.glrm_global_error().decode()


def test_host_argument_validation(lib):
    ok = [(0, 0.0, 0)] * 3
    assert _create(lib, 4, 3, 0, ok)[0] == -2       # k < 1
    assert _create(lib, 4, 3, 65, ok)[0] == -2      # k > 64
    assert _create(lib, 0, 3, 2, ok)[0] == -2       # m < 1
    assert _create(lib, 4, 3, 2, ok, prec=7)[0] == -1
    rc, msg = _create(lib, 4, 3, 2, [(0, 0.0, 0), (9, 0.0, 0), (0, 0.0, 0)])
    assert rc == -1 and "column 1" in msg
    rc, msg = _create(lib, 4, 3, 2, [(1, 0.0, 0)] * 3)     # Huber threshold 0
    assert rc == -1 and "Huber" in msg
    rc, msg = _create(lib, 4, 3, 2, [(4, 0.0, 1)] * 3)     # ordinal with 1 level
    assert rc == -1 and "ordinal" in msg
    assert _create(lib, 4, 3, 2, ok, rx=(5, 0.0))[0] == -1
    assert _create(lib, 4, 3, 2, ok, rx=(1, -1.0))[0] == -1


def test_null_handle_calls_fail_cleanly(lib):
    lib.glrm_sweep.restype = ctypes.c_int
    assert lib.glrm_sweep(None, 1, None) == -1
    lib.glrm_objective.restype = ctypes.c_int
    assert lib.glrm_objective(None, None) == -1
    lib.glrm_destroy(None)
