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
              "glrm_set_reg_weights", "glrm_certificate", "glrm_regularization_path", "glrm_svd_init",
              "glrm_set_observed_csr", "glrm_set_observed_csr_host"):
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


def test_null_handle_calls_of_the_method_pieces(lib):
    """Every handle entry point of the method pieces around the sweep rejects
    a null handle on the host (GLRM_ERR_ARG) without touching a GPU."""
    p = ctypes.c_void_p
    calls = [
        ("glrm_set_offset", [p, ctypes.c_int32], (None, 1)),
        ("glrm_column_stats", [p, p, p], (None, None, None)),
        ("glrm_set_column_scale", [p, p], (None, None)),
        ("glrm_set_reg_weights", [p, ctypes.c_double, ctypes.c_double], (None, 0.1, 0.1)),
        ("glrm_certificate", [p, ctypes.c_int32, ctypes.c_double, p, p], (None, 10, 1e-9, None, None)),
        ("glrm_regularization_path", [p, ctypes.c_int32, p, ctypes.c_int32, ctypes.c_double, ctypes.c_int32, p, p,
                                      p, ctypes.c_int32], (None, 1, None, 1, 1e-6, 1, None, None, None, 0)),
        ("glrm_svd_init", [p, ctypes.c_int32, ctypes.c_int32, ctypes.c_uint64, p], (None, 8, 4, 1, None)),
        ("glrm_decode_features", [p, ctypes.c_int32, p, ctypes.c_int64, p, p, p], (None, 1, None, 0, None, None, None)),
        ("glrm_proxprox_sweep", [p, ctypes.c_int32, ctypes.c_double, ctypes.c_int32, p], (None, 1, 1.0, 1, None)),
    ]
    for name, argtypes, args in calls:
        f = getattr(lib, name)
        f.restype = ctypes.c_int
        f.argtypes = argtypes
        assert f(*args) == -1, name


class _Feature(ctypes.Structure):
    _fields_ = [("kind", ctypes.c_int32), ("levels", ctypes.c_int32)]


class _Loss(ctypes.Structure):
    _fields_ = [("kind", ctypes.c_int32), ("levels", ctypes.c_int32), ("param", ctypes.c_double)]


def test_embed_losses_on_the_host(lib):
    """Block widths (scalar 1, categorical d, ordinal d - 1), the scalar
    features' losses kept, the hinge loss on every block column; bad
    descriptors rejected."""
    f = lib.glrm_embed_losses
    f.restype = ctypes.c_int
    f.argtypes = [ctypes.c_int32, ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p]
    feats = (_Feature * 4)(_Feature(0, 0), _Feature(1, 3), _Feature(2, 4), _Feature(0, 0))
    sl = (_Loss * 4)(_Loss(1, 0, 0.5), _Loss(0, 0, 0.0), _Loss(0, 0, 0.0), _Loss(6, 0, 0.3))
    D = ctypes.c_int64()
    assert f(4, ctypes.cast(feats, ctypes.c_void_p), ctypes.cast(sl, ctypes.c_void_p), None, ctypes.byref(D)) == 0
    assert D.value == 1 + 3 + 3 + 1
    out = (_Loss * D.value)()
    assert f(4, ctypes.cast(feats, ctypes.c_void_p), ctypes.cast(sl, ctypes.c_void_p),
             ctypes.cast(out, ctypes.c_void_p), None) == 0
    assert [o.kind for o in out] == [1, 2, 2, 2, 2, 2, 2, 6]
    assert out[0].param == 0.5 and out[7].param == 0.3
    for bad in ((1, 1), (2, 1), (3, 4), (1, 70000)):
        fb = (_Feature * 1)(_Feature(*bad))
        assert f(1, ctypes.cast(fb, ctypes.c_void_p), ctypes.cast(sl, ctypes.c_void_p), None, ctypes.byref(D)) == -1
