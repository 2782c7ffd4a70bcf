"""Python binding of libglrm (C ABI in include/glrm.h).

Argument marshalling only: every function here passes pointers and sizes to
the CUDA library of the same name; all arithmetic runs in its kernels.  Device
buffers are torch CUDA tensors; PyTorch supplies memory and the stream.  If
the library is missing the import of this module fails loudly: there is no
CPU fallback.
"""
from __future__ import annotations

import ctypes
import os

import numpy as np
import torch

GLRM_OK = 0
GLRM_ERR_ARG, GLRM_ERR_RANGE, GLRM_ERR_OMEGA, GLRM_ERR_NONFINITE = -1, -2, -3, -4
GLRM_ERR_CUDA, GLRM_ERR_TIMEOUT, GLRM_ERR_STATE, GLRM_ERR_NOMEM = -5, -6, -7, -8
GLRM_LOSS_QUAD, GLRM_LOSS_HUBER, GLRM_LOSS_HINGE, GLRM_LOSS_LOGISTIC, GLRM_LOSS_ORDINAL_HINGE = range(5)
GLRM_LOSS_L1, GLRM_LOSS_QUANTILE = 5, 6
GLRM_REG_ZERO, GLRM_REG_QUAD, GLRM_REG_L1, GLRM_REG_NONNEG = range(4)
GLRM_FP64, GLRM_FP32, GLRM_BF16 = 0, 1, 2
GLRM_PATH_AUTO, GLRM_PATH_CHUNKED, GLRM_PATH_FUSED, GLRM_PATH_BLOCKED = 0, 1, 2, 3
GLRM_PATH_MASKED, GLRM_PATH_MASKED_SPLIT, GLRM_PATH_DENSE = 4, 5, 6

_LIB_PATH = os.path.join(os.path.dirname(os.path.abspath(__file__)), "lib", "libglrm.so")


class GLRMError(RuntimeError):
    def __init__(self, code: int, msg: str):
        super().__init__(f"libglrm error {code}: {msg}")
        self.code = code


class glrm_loss(ctypes.Structure):
    _fields_ = [("kind", ctypes.c_int32), ("levels", ctypes.c_int32), ("param", ctypes.c_double)]


class glrm_feature(ctypes.Structure):
    _fields_ = [("kind", ctypes.c_int32), ("levels", ctypes.c_int32)]


GLRM_FEATURE_SCALAR, GLRM_FEATURE_CATEGORICAL, GLRM_FEATURE_ORDINAL = 0, 1, 2


def _load():
    if not os.path.exists(_LIB_PATH):
        raise ImportError(f"libglrm.so not built ({_LIB_PATH}); run __graft_entry__.build()")
    lib = ctypes.CDLL(_LIB_PATH)
    p, i32, i64, f64 = ctypes.c_void_p, ctypes.c_int32, ctypes.c_int64, ctypes.c_double
    sig = {
        "glrm_create": [i64, i64, i32, p, i32, f64, i32, f64, i32, p, p],
        "glrm_set_observed": [p, i64, p, p, p, p, p, p],
        "glrm_set_observed_host": [p, i64, p, p, p, p, p, p],
        "glrm_set_dense": [p, p, i64],
        "glrm_set_observed_csr": [p, i64, p, p, p],
        "glrm_set_observed_csr_host": [p, i64, p, p, p],
        "glrm_set_dense_host": [p, p, i64],
        "glrm_set_factors": [p, p, p],
        "glrm_get_factors": [p, p, p],
        "glrm_set_factors_host": [p, p, p],
        "glrm_get_factors_host": [p, p, p],
        "glrm_reset_steps": [p],
        "glrm_embed_losses": [i32, p, p, p, p],
        "glrm_set_reg_weights": [p, f64, f64],
        "glrm_svd_init": [p, i32, i32, ctypes.c_uint64, p],
        "glrm_certificate": [p, i32, f64, p, p],
        "glrm_regularization_path": [p, i32, p, i32, f64, i32, p, p, p, i32],
        "glrm_embed_size": [i32, p, p, p, p, p],
        "glrm_embed_features": [i32, p, i64, i64, p, p, p, p, p, p, i32, p, p, p, p, p, p, p],
        "glrm_decode_features": [p, i32, p, i64, p, p, p],
        "glrm_set_offset": [p, i32],
        "glrm_column_stats": [p, p, p],
        "glrm_set_column_scale": [p, p],
        "glrm_sweep": [p, i32, p],
        "glrm_sweep_until": [p, i32, f64, f64, i32, p, p],
        "glrm_last_accepts": [p, p],
        "glrm_objective": [p, p],
        "glrm_objective_at": [p, p, p, p],
        "glrm_grad_at": [p, p, p, p, p, i32, p],
        "glrm_grad": [p, p, p],
        "glrm_predict": [p, i64, p, p, p, i32],
        "glrm_als_sweep": [p, i32, p],
        "glrm_proxprox_sweep": [p, i32, f64, i32, p],
        "glrm_get_state": [p, p, p],
        "glrm_set_state": [p, p, ctypes.c_size_t],
        "glrm_timing_enable": [p, i32],
        "glrm_timing_read": [p, i32, p, p, p, p],
        "glrm_launch_count": [p, p],
        "glrm_set_path": [p, i32, i32],
        "glrm_get_path": [p, p],
        "glrm_objective_noalloc": [i64, i64, i32, i64, p, p, p, p, i32, f64, i32, f64, p, p, p, p],
        "glrm_batch_create": [i32, p, p, p, p, p, p, p, p, p],
        "glrm_batch_set_factors": [p, p, p],
        "glrm_batch_get_factors": [p, p, p],
        "glrm_batch_set_steps": [p, p, p],
        "glrm_batch_get_steps": [p, p, p],
        "glrm_batch_sweep": [p, i32, p, i32],
        "glrm_batch_autotune": [p, i32, p, p],
        "glrm_batch_set_wait_limit": [p, i64],
        "glrm_tc_gemm_bf16": [p, p, p, i32, i32, i32, p],
        "glrm_wait_selftest": [i64, i32, p],
        "glrm_fma_peak": [i32, p, p, p],
    }
    for name, args in sig.items():
        fn = getattr(lib, name)
        fn.argtypes = args
        fn.restype = ctypes.c_int
    lib.glrm_last_error.argtypes = [p]
    lib.glrm_last_error.restype = ctypes.c_char_p
    lib.glrm_global_error.argtypes = []
    lib.glrm_global_error.restype = ctypes.c_char_p
    lib.glrm_destroy.argtypes = [p]
    lib.glrm_destroy.restype = None
    lib.glrm_batch_last_error.argtypes = [p]
    lib.glrm_batch_last_error.restype = ctypes.c_char_p
    lib.glrm_batch_destroy.argtypes = [p]
    lib.glrm_batch_destroy.restype = None
    return lib


_lib = _load()


def library():
    """The loaded ctypes library (for tests that check exported symbols)."""
    return _lib


def _ptr(t):
    if t is None:
        return None
    if isinstance(t, torch.Tensor):
        if not t.is_contiguous():
            raise ValueError("tensor must be contiguous")
        return ctypes.c_void_p(t.data_ptr())
    if isinstance(t, np.ndarray):
        if not t.flags["C_CONTIGUOUS"]:
            raise ValueError("array must be C-contiguous")
        return t.ctypes.data_as(ctypes.c_void_p)
    return t


def _check(rc: int, h=None):
    if rc != GLRM_OK:
        msg = (_lib.glrm_last_error(h) if h else _lib.glrm_global_error()) or b""
        raise GLRMError(rc, msg.decode(errors="replace"))


def dtype_of(precision: int) -> torch.dtype:
    return torch.float64 if precision == GLRM_FP64 else torch.float32


# ------------------------------------------------------- same-name wrappers

def glrm_create(m, n, k, col_loss, rx, ry, precision=GLRM_FP32, stream=None):
    """col_loss: sequence of (kind, param, levels) per column, or arrays
    (kind[n], param[n], levels[n]).  rx, ry: (kind, weight).  stream: a
    torch.cuda.Stream (default: the current stream)."""
    if isinstance(col_loss, tuple) and len(col_loss) == 3 and hasattr(col_loss[0], "__len__"):
        kinds, params, levels = (np.asarray(a) for a in col_loss)
    else:
        arr = np.asarray(col_loss, dtype=np.float64).reshape(-1, 3)
        kinds, params, levels = arr[:, 0], arr[:, 1], arr[:, 2]
    losses = (glrm_loss * n)()
    for j in range(n):
        losses[j] = glrm_loss(int(kinds[j]), int(levels[j]), float(params[j]))
    if stream is None:
        stream = torch.cuda.current_stream()
    h = ctypes.c_void_p()
    _check(_lib.glrm_create(m, n, k, ctypes.cast(losses, ctypes.c_void_p), int(rx[0]),
                            float(rx[1]), int(ry[0]), float(ry[1]), precision,
                            ctypes.c_void_p(stream.cuda_stream), ctypes.byref(h)))
    return h


def glrm_set_observed(h, nnz, csr_rowptr, csr_colidx, csr_val, csc_colptr, csc_rowidx, csc_val):
    _check(_lib.glrm_set_observed(h, nnz, _ptr(csr_rowptr), _ptr(csr_colidx), _ptr(csr_val),
                                  _ptr(csc_colptr), _ptr(csc_rowidx), _ptr(csc_val)), h)


def glrm_set_observed_host(h, nnz, csr_rowptr, csr_colidx, csr_val, csc_colptr, csc_rowidx,
                           csc_val):
    _check(_lib.glrm_set_observed_host(h, nnz, _ptr(csr_rowptr), _ptr(csr_colidx),
                                       _ptr(csr_val), _ptr(csc_colptr), _ptr(csc_rowidx),
                                       _ptr(csc_val)), h)


def glrm_set_observed_csr(h, nnz, csr_rowptr, csr_colidx, csr_val):
    _check(_lib.glrm_set_observed_csr(h, nnz, _ptr(csr_rowptr), _ptr(csr_colidx), _ptr(csr_val)), h)


def glrm_set_observed_csr_host(h, nnz, csr_rowptr, csr_colidx, csr_val):
    _check(_lib.glrm_set_observed_csr_host(h, nnz, _ptr(csr_rowptr), _ptr(csr_colidx), _ptr(csr_val)), h)


def glrm_set_dense(h, A, lda=None):
    """A: m x n float32 CUDA tensor (rows contiguous; lda = its row stride)."""
    if lda is None:
        lda = A.stride(0) if isinstance(A, torch.Tensor) else A.shape[1]
    _check(_lib.glrm_set_dense(h, ctypes.c_void_p(A.data_ptr()), int(lda)), h)


def glrm_set_dense_host(h, A, lda=None):
    """A: m x n float32 host array or CPU tensor (pinned memory copies faster)."""
    if lda is None:
        lda = A.stride(0) if isinstance(A, torch.Tensor) else A.shape[1]
    ptr = ctypes.c_void_p(A.data_ptr()) if isinstance(A, torch.Tensor) else _ptr(A)
    _check(_lib.glrm_set_dense_host(h, ptr, int(lda)), h)


def glrm_set_factors(h, X, Yt):
    _check(_lib.glrm_set_factors(h, _ptr(X), _ptr(Yt)), h)


def glrm_get_factors(h, X, Yt):
    _check(_lib.glrm_get_factors(h, _ptr(X), _ptr(Yt)), h)


def glrm_set_factors_host(h, X, Yt):
    _check(_lib.glrm_set_factors_host(h, _ptr(X), _ptr(Yt)), h)


def glrm_get_factors_host(h, X, Yt):
    _check(_lib.glrm_get_factors_host(h, _ptr(X), _ptr(Yt)), h)


def glrm_set_offset(h, on=True):
    _check(_lib.glrm_set_offset(h, 1 if on else 0), h)


def glrm_column_stats(h, mu, sigma2):
    """mu, sigma2: float64 device tensors of n values."""
    _check(_lib.glrm_column_stats(h, _ptr(mu), _ptr(sigma2)), h)


def glrm_set_column_scale(h, w=None):
    """w: n positive finite weights (host), or None to remove them."""
    if w is None:
        _check(_lib.glrm_set_column_scale(h, None), h)
        return
    arr = np.ascontiguousarray(np.asarray(w, dtype=np.float64))
    _check(_lib.glrm_set_column_scale(h, _ptr(arr)), h)


def glrm_svd_init(h, kp, oversample=8, power_iters=4, seed=1410034200):
    """Sec. 7.5 initialisation; returns the kp singular values used."""
    sv = np.empty(max(kp, 1))
    _check(_lib.glrm_svd_init(h, int(oversample), int(power_iters), int(seed), _ptr(sv)), h)
    return sv[:kp]


def glrm_set_reg_weights(h, rx_weight, ry_weight):
    _check(_lib.glrm_set_reg_weights(h, float(rx_weight), float(ry_weight)), h)


def glrm_certificate(h, max_iters=1000, tol=1e-10):
    """(norm, iterations) of the optimality certificate (Sec. 7.6)."""
    nrm = ctypes.c_double()
    it = ctypes.c_int32()
    _check(_lib.glrm_certificate(h, int(max_iters), float(tol), ctypes.byref(nrm), ctypes.byref(it)), h)
    return nrm.value, it.value


def glrm_regularization_path(h, gammas, max_sweeps, rtol, window=1, cert_iters=0):
    """(objectives, sweeps, certificates or None) per weight (Sec. 8.1)."""
    g = np.ascontiguousarray(np.asarray(gammas, dtype=np.float64))
    obj = np.empty(g.size)
    sw = np.empty(g.size, dtype=np.int32)
    cert = np.empty(g.size) if cert_iters > 0 else None
    _check(_lib.glrm_regularization_path(h, g.size, _ptr(g), int(max_sweeps), float(rtol), int(window), _ptr(obj),
                                         _ptr(sw), _ptr(cert) if cert is not None else None, int(cert_iters)), h)
    return obj, sw, cert


def _features(fkind, flevels):
    fkind = np.asarray(fkind)
    flevels = np.asarray(flevels)
    arr = (glrm_feature * len(fkind))()
    for j in range(len(fkind)):
        arr[j] = glrm_feature(int(fkind[j]), int(flevels[j]))
    return arr


def glrm_embed_losses(fkind, flevels, scalar_loss):
    """scalar_loss: arrays (kind[nf], param[nf], levels[nf]) of the scalar
    features.  Returns (kind, param, levels) of the embedded columns."""
    nf = len(fkind)
    feats = _features(fkind, flevels)
    sl = (glrm_loss * nf)()
    for j in range(nf):
        sl[j] = glrm_loss(int(scalar_loss[0][j]), int(scalar_loss[2][j]), float(scalar_loss[1][j]))
    D = ctypes.c_int64()
    _check(_lib.glrm_embed_losses(nf, ctypes.cast(feats, ctypes.c_void_p), ctypes.cast(sl, ctypes.c_void_p),
                                  None, ctypes.byref(D)))
    out = (glrm_loss * D.value)()
    _check(_lib.glrm_embed_losses(nf, ctypes.cast(feats, ctypes.c_void_p), ctypes.cast(sl, ctypes.c_void_p),
                                  ctypes.cast(out, ctypes.c_void_p), None))
    return (np.array([o.kind for o in out], np.int32), np.array([o.param for o in out]),
            np.array([o.levels for o in out], np.int32))


def glrm_embed_size(fkind, flevels, colptr, stream=None):
    D = ctypes.c_int64()
    nnz = ctypes.c_int64()
    st = ctypes.c_void_p((stream or torch.cuda.current_stream()).cuda_stream)
    _check(_lib.glrm_embed_size(len(fkind), ctypes.cast(_features(fkind, flevels), ctypes.c_void_p), _ptr(colptr),
                                ctypes.byref(D), ctypes.byref(nnz), st))
    return D.value, nnz.value


def glrm_embed_features(fkind, flevels, m, nnz, rowptr, featidx, val, colptr, rowidx, cval, precision,
                        e_rowptr, e_colidx, e_val, e_colptr, e_rowidx, e_cval, stream=None):
    st = ctypes.c_void_p((stream or torch.cuda.current_stream()).cuda_stream)
    _check(_lib.glrm_embed_features(len(fkind), ctypes.cast(_features(fkind, flevels), ctypes.c_void_p), m, nnz,
                                    _ptr(rowptr), _ptr(featidx), _ptr(val), _ptr(colptr), _ptr(rowidx), _ptr(cval),
                                    precision, _ptr(e_rowptr), _ptr(e_colidx), _ptr(e_val), _ptr(e_colptr),
                                    _ptr(e_rowidx), _ptr(e_cval), st))


def glrm_decode_features(h, fkind, flevels, rows, feats, out):
    _check(_lib.glrm_decode_features(h, len(fkind), ctypes.cast(_features(fkind, flevels), ctypes.c_void_p),
                                     rows.numel(), _ptr(rows), _ptr(feats), _ptr(out)), h)


def glrm_reset_steps(h):
    _check(_lib.glrm_reset_steps(h), h)


def glrm_sweep(h, nsweeps, history=True):
    """Returns the per-sweep objective (numpy float64) when history is True."""
    if history:
        out = np.empty(nsweeps, dtype=np.float64)
        _check(_lib.glrm_sweep(h, nsweeps, _ptr(out)), h)
        return out
    _check(_lib.glrm_sweep(h, nsweeps, None), h)
    return None


def glrm_sweep_until(h, max_sweeps, rtol, f_ref=float("nan"), window=1):
    """Sweeps until the device-side convergence test passes; returns the
    objectives of the sweeps run (numpy float64)."""
    ran = ctypes.c_int32(0)
    out = np.empty(max_sweeps, dtype=np.float64)
    _check(_lib.glrm_sweep_until(h, int(max_sweeps), float(rtol), float(f_ref), int(window),
                                 ctypes.byref(ran), _ptr(out)), h)
    return out[:ran.value].copy()


def glrm_last_accepts(h):
    out = np.zeros(2, dtype=np.int64)
    _check(_lib.glrm_last_accepts(h, _ptr(out)), h)
    return out


def glrm_objective(h) -> float:
    out = np.zeros(1, dtype=np.float64)
    _check(_lib.glrm_objective(h, _ptr(out)), h)
    return float(out[0])


def glrm_objective_at(h, X, Yt, out):
    _check(_lib.glrm_objective_at(h, _ptr(X), _ptr(Yt), _ptr(out)), h)


def glrm_grad_at(h, X, Yt, GX, GYt, include_reg=True, scale=None):
    """scale: optional CUDA float64 tensor (one element) multiplying both gradients."""
    _check(_lib.glrm_grad_at(h, _ptr(X), _ptr(Yt), _ptr(GX), _ptr(GYt), int(bool(include_reg)),
                             _ptr(scale)), h)


def glrm_grad(h, GX, GYt):
    """Loss part of the gradient at the handle's factors into GX (m x k), GYt (n x k)."""
    _check(_lib.glrm_grad(h, _ptr(GX), _ptr(GYt)), h)


def glrm_predict(h, rows, cols, out, decode=True):
    _check(_lib.glrm_predict(h, int(rows.numel()), _ptr(rows), _ptr(cols), _ptr(out),
                             int(bool(decode))), h)


def glrm_als_sweep(h, nsweeps, history=True):
    if history:
        out = np.empty(nsweeps, dtype=np.float64)
        _check(_lib.glrm_als_sweep(h, nsweeps, _ptr(out)), h)
        return out
    _check(_lib.glrm_als_sweep(h, nsweeps, None), h)
    return None


def glrm_proxprox_sweep(h, nsweeps, alpha, inner, history=True):
    if history:
        out = np.empty(nsweeps, dtype=np.float64)
        _check(_lib.glrm_proxprox_sweep(h, nsweeps, float(alpha), int(inner), _ptr(out)), h)
        return out
    _check(_lib.glrm_proxprox_sweep(h, nsweeps, float(alpha), int(inner), None), h)
    return None


def glrm_get_state(h) -> bytes:
    n = ctypes.c_size_t(0)
    _check(_lib.glrm_get_state(h, None, ctypes.byref(n)), h)
    buf = ctypes.create_string_buffer(n.value)
    _check(_lib.glrm_get_state(h, buf, ctypes.byref(n)), h)
    return buf.raw[:n.value]


def glrm_set_state(h, state: bytes):
    buf = ctypes.create_string_buffer(state, len(state))
    _check(_lib.glrm_set_state(h, buf, len(state)), h)


def glrm_set_path(h, xstep_path, ystep_path):
    _check(_lib.glrm_set_path(h, int(xstep_path), int(ystep_path)), h)


def glrm_get_path(h):
    out = np.zeros(2, np.int32)
    _check(_lib.glrm_get_path(h, _ptr(out)), h)
    return int(out[0]), int(out[1])


def glrm_timing_enable(h, on=True):
    _check(_lib.glrm_timing_enable(h, int(bool(on))), h)


def glrm_timing_read(h, max_kernels=64):
    """{kernel name: (total ms, launches)} recorded since timing was enabled."""
    names = ctypes.create_string_buffer(32 * max_kernels)
    ms = np.zeros(max_kernels, np.float64)
    cnt = np.zeros(max_kernels, np.int64)
    q = ctypes.c_int32(0)
    _check(_lib.glrm_timing_read(h, max_kernels, names, _ptr(ms), _ptr(cnt), ctypes.byref(q)), h)
    out = {}
    for i in range(q.value):
        nm = names.raw[32 * i:32 * (i + 1)].split(b"\0", 1)[0].decode()
        out[nm] = (float(ms[i]), int(cnt[i]))
    return out


def glrm_launch_count(h) -> int:
    out = ctypes.c_int64(0)
    _check(_lib.glrm_launch_count(h, ctypes.byref(out)), h)
    return int(out.value)


def glrm_objective_noalloc(m, n, k, nnz, csr_rowptr, csr_colidx, csr_val, col_loss_dev, rx, ry, X,
                           Yt, out, stream=None):
    """Objective without device allocation (see include/glrm.h); every
    argument is a CUDA tensor, col_loss_dev the raw bytes of n glrm_loss."""
    if stream is None:
        stream = torch.cuda.current_stream()
    _check(_lib.glrm_objective_noalloc(m, n, k, nnz, _ptr(csr_rowptr), _ptr(csr_colidx), _ptr(csr_val),
                                       _ptr(col_loss_dev), int(rx[0]), float(rx[1]), int(ry[0]),
                                       float(ry[1]), _ptr(X), _ptr(Yt), _ptr(out),
                                       ctypes.c_void_p(stream.cuda_stream)))


def glrm_tc_gemm_bf16(A, B, D, stream=None):
    """D = A B^T on the tensor cores; A (M x K) and B (N x K) bf16 CUDA tensors,
    D (M x N) float32."""
    if stream is None:
        stream = torch.cuda.current_stream()
    M, K = A.shape
    N = B.shape[0]
    _check(_lib.glrm_tc_gemm_bf16(_ptr(A), _ptr(B), _ptr(D), M, N, K,
                                  ctypes.c_void_p(stream.cuda_stream)))


def glrm_wait_selftest(attempts, arm, stream=None):
    """Bounded-wait self-test; raises GLRMError(GLRM_ERR_TIMEOUT) when the wait ran out."""
    if stream is None:
        stream = torch.cuda.current_stream()
    _check(_lib.glrm_wait_selftest(int(attempts), int(bool(arm)), ctypes.c_void_p(stream.cuda_stream)))


def glrm_fma_peak(iters=8192, stream=None):
    """(FP32 FMA TFLOP/s measured on the current device, SM count)."""
    if stream is None:
        stream = torch.cuda.current_stream()
    tf = ctypes.c_double(0.0)
    sms = ctypes.c_int32(0)
    _check(_lib.glrm_fma_peak(int(iters), ctypes.byref(tf), ctypes.byref(sms),
                              ctypes.c_void_p(stream.cuda_stream)))
    return tf.value, sms.value


def glrm_destroy(h):
    if h:
        _lib.glrm_destroy(h)


# ------------------------------------------------------------ batched form

GLRM_BATCH_PROXGRAD, GLRM_BATCH_ALS = 0, 1
GLRM_BATCH_GRAPH, GLRM_BATCH_STREAM, GLRM_BATCH_PER_INSTANCE = 0, 1, 2


class glrm_batch_instance(ctypes.Structure):
    _fields_ = [("m", ctypes.c_int64), ("n", ctypes.c_int64), ("k", ctypes.c_int32),
                ("method", ctypes.c_int32), ("loss", glrm_loss), ("rx_kind", ctypes.c_int32),
                ("ry_kind", ctypes.c_int32), ("rx_weight", ctypes.c_double),
                ("ry_weight", ctypes.c_double), ("nnz", ctypes.c_int64)]


def _bcheck(rc, b=None):
    if rc != GLRM_OK:
        msg = _lib.glrm_batch_last_error(b) or b""
        raise GLRMError(rc, msg.decode(errors="replace"))


class Batch:
    """A glrm_batch_t over a workloads.Batch (device tensors)."""

    def __init__(self, wb, methods, rx=(GLRM_REG_QUAD, 0.1), ry=(GLRM_REG_QUAD, 0.1),
                 huber_delta=1.0, stream=None):
        self.count = wb.count
        arr = (glrm_batch_instance * self.count)()
        for s in range(self.count):
            kind = int(wb.kind[s])
            arr[s] = glrm_batch_instance(int(wb.m[s]), int(wb.n[s]), int(wb.k[s]), int(methods[s]),
                                         glrm_loss(kind, 0, huber_delta if kind == 1 else 0.0),
                                         int(rx[0]), int(ry[0]), float(rx[1]), float(ry[1]),
                                         int(wb.nnz[s]))
        if stream is None:
            stream = torch.cuda.current_stream()
        self.wb = wb
        self.b = ctypes.c_void_p()
        rc = _lib.glrm_batch_create(self.count, ctypes.cast(arr, ctypes.c_void_p), _ptr(wb.rowptr),
                                    _ptr(wb.colidx), _ptr(wb.val), _ptr(wb.colptr), _ptr(wb.rowidx),
                                    _ptr(wb.cval), ctypes.c_void_p(stream.cuda_stream),
                                    ctypes.byref(self.b))
        if rc != GLRM_OK:
            msg = (_lib.glrm_batch_last_error(self.b) if self.b else _lib.glrm_batch_last_error(None)) or b""
            if self.b:
                _lib.glrm_batch_destroy(self.b)
                self.b = None
            raise GLRMError(rc, msg.decode(errors="replace"))
        _bcheck(_lib.glrm_batch_set_factors(self.b, _ptr(wb.X0), _ptr(wb.Yt0)), self.b)

    def sweep(self, nsweeps, mode=GLRM_BATCH_GRAPH, history=True):
        if history:
            out = np.empty((nsweeps, self.count), np.float64)
            _bcheck(_lib.glrm_batch_sweep(self.b, nsweeps, _ptr(out), mode), self.b)
            return out
        _bcheck(_lib.glrm_batch_sweep(self.b, nsweeps, None, mode), self.b)
        return None

    def factors(self):
        X = torch.empty_like(self.wb.X0)
        Yt = torch.empty_like(self.wb.Yt0)
        _bcheck(_lib.glrm_batch_get_factors(self.b, _ptr(X), _ptr(Yt)), self.b)
        return X, Yt

    def set_factors(self, X, Yt):
        _bcheck(_lib.glrm_batch_set_factors(self.b, _ptr(X), _ptr(Yt)), self.b)

    def steps(self):
        ax = torch.empty(int(self.wb.m.sum()), dtype=torch.float32, device=self.wb.X0.device)
        ay = torch.empty(int(self.wb.n.sum()), dtype=torch.float32, device=self.wb.X0.device)
        _bcheck(_lib.glrm_batch_get_steps(self.b, _ptr(ax), _ptr(ay)), self.b)
        return ax, ay

    def set_steps(self, ax, ay):
        _bcheck(_lib.glrm_batch_set_steps(self.b, _ptr(ax), _ptr(ay)), self.b)

    def set_wait_limit(self, polls):
        _bcheck(_lib.glrm_batch_set_wait_limit(self.b, int(polls)), self.b)

    def autotune(self, reps=3):
        tx = np.zeros(32, np.int32)
        ty = np.zeros(32, np.int32)
        _bcheck(_lib.glrm_batch_autotune(self.b, reps, _ptr(tx), _ptr(ty)), self.b)
        return tx, ty

    def close(self):
        if self.b:
            _lib.glrm_batch_destroy(self.b)
            self.b = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


# ----------------------------------------------------------- convenience

class GLRM:
    """Owns one handle.  ``table`` is anything with the fields of
    workloads.Table (m, n, k, CSR/CSC arrays, per-column losses, rx, ry)."""

    def __init__(self, m, n, k, col_loss, rx, ry, precision=GLRM_FP32, device=None,
                 stream=None):
        self.m, self.n, self.k, self.precision = int(m), int(n), int(k), precision
        self.device = torch.device(device) if device is not None else torch.device("cuda")
        self.dtype = dtype_of(precision)
        with torch.cuda.device(self.device):
            self.h = glrm_create(self.m, self.n, self.k, col_loss, rx, ry, precision, stream)

    @classmethod
    def from_table(cls, t, precision=GLRM_FP32, device=None, stream=None, factors=True):
        g = cls(t.m, t.n, t.k, (t.loss_kind, t.loss_param, t.loss_levels), t.rx, t.ry,
                precision, device, stream)
        g.set_observed_table(t)
        if factors:
            g.set_factors(torch.as_tensor(t.X0, dtype=g.dtype, device=g.device),
                          torch.as_tensor(t.Yt0, dtype=g.dtype, device=g.device))
        return g

    @classmethod
    def from_dense_table(cls, t, device=None, stream=None, factors=True):
        """A workloads.DenseTable, or a fully observed workloads.Table (nnz ==
        m n, CSR rows complete), given to the dense form."""
        g = cls(t.m, t.n, t.k, (t.loss_kind, t.loss_param, t.loss_levels), t.rx, t.ry,
                GLRM_FP32, device, stream)
        if hasattr(t, "A"):
            src = t.A
        else:
            if int(t.colidx.size) != t.m * t.n:
                raise ValueError("the table is not fully observed")
            src = np.asarray(t.val).reshape(t.m, t.n)
        A = torch.as_tensor(src, dtype=torch.float32, device=g.device)
        g.set_dense(A)
        if factors:
            g.set_factors(torch.as_tensor(t.X0, dtype=g.dtype, device=g.device),
                          torch.as_tensor(t.Yt0, dtype=g.dtype, device=g.device))
        return g

    @classmethod
    def from_feature_table(cls, t, precision=GLRM_FP32, device=None, stream=None, factors=True):
        """A workloads.FeatureTable: embedded on the device (glrm_embed_features)
        into its Boolean block columns and given to a model of sum d_j columns."""
        dev = torch.device(device) if device is not None else torch.device("cuda")
        dt = dtype_of(precision)
        i32 = torch.int32
        src = [torch.as_tensor(np.asarray(a), dtype=ty, device=dev) for a, ty in
               ((t.rowptr, i32), (t.featidx, i32), (t.val, dt), (t.colptr, i32), (t.rowidx, i32), (t.cval, dt))]
        with torch.cuda.device(dev):
            D, ennz = glrm_embed_size(t.fkind, t.flevels, src[3], stream)
            out = [torch.empty(t.m + 1, dtype=i32, device=dev), torch.empty(max(ennz, 1), dtype=i32, device=dev),
                   torch.empty(max(ennz, 1), dtype=dt, device=dev), torch.empty(D + 1, dtype=i32, device=dev),
                   torch.empty(max(ennz, 1), dtype=i32, device=dev), torch.empty(max(ennz, 1), dtype=dt, device=dev)]
            glrm_embed_features(t.fkind, t.flevels, t.m, t.nnz, *src, precision, *out, stream=stream)
            losses = glrm_embed_losses(t.fkind, t.flevels, (t.loss_kind, t.loss_param, t.loss_levels))
        g = cls(t.m, D, t.k, losses, t.rx, t.ry, precision, dev, stream)
        g.fkind, g.flevels = np.asarray(t.fkind), np.asarray(t.flevels)
        with torch.cuda.device(dev):
            glrm_set_observed(g.h, ennz, *out)
        if factors:
            g.set_factors(torch.as_tensor(t.X0, dtype=dt, device=dev), torch.as_tensor(t.Yt0, dtype=dt, device=dev))
        return g

    def decode_features(self, rows, feats):
        out = torch.empty(rows.numel(), dtype=self.dtype, device=self.device)
        glrm_decode_features(self.h, self.fkind, self.flevels, rows.to(torch.int32).contiguous(),
                             feats.to(torch.int32).contiguous(), out)
        return out

    def set_dense(self, A):
        with torch.cuda.device(self.device):
            glrm_set_dense(self.h, A)

    def set_observed_table(self, t):
        dev, dt = self.device, self.dtype
        i32 = torch.int32
        arrs = [torch.as_tensor(np.asarray(t.rowptr), dtype=i32, device=dev),
                torch.as_tensor(np.asarray(t.colidx), dtype=i32, device=dev),
                torch.as_tensor(np.asarray(t.val), dtype=dt, device=dev),
                torch.as_tensor(np.asarray(t.colptr), dtype=i32, device=dev),
                torch.as_tensor(np.asarray(t.rowidx), dtype=i32, device=dev),
                torch.as_tensor(np.asarray(t.cval), dtype=dt, device=dev)]
        with torch.cuda.device(self.device):
            glrm_set_observed(self.h, int(t.colidx.size), *arrs)

    def set_factors(self, X, Yt):
        glrm_set_factors(self.h, X.contiguous() if X is not None else None,
                         Yt.contiguous() if Yt is not None else None)

    def factors(self):
        X = torch.empty(self.m, self.k, dtype=self.dtype, device=self.device)
        Yt = torch.empty(self.n, self.k, dtype=self.dtype, device=self.device)
        glrm_get_factors(self.h, X, Yt)
        return X, Yt

    def sweep(self, nsweeps, history=True):
        return glrm_sweep(self.h, nsweeps, history)

    def sweep_until(self, max_sweeps, rtol, f_ref=float("nan"), window=1):
        return glrm_sweep_until(self.h, max_sweeps, rtol, f_ref, window)

    def als_sweep(self, nsweeps, history=True):
        return glrm_als_sweep(self.h, nsweeps, history)

    def proxprox_sweep(self, nsweeps, alpha, inner, history=True):
        return glrm_proxprox_sweep(self.h, nsweeps, alpha, inner, history)

    def objective(self):
        return glrm_objective(self.h)

    def svd_init(self, oversample=8, power_iters=4, seed=1410034200, offset=None):
        """offset: None keeps the handle's setting."""
        if offset is not None:
            self.set_offset(offset)
            self._offset = bool(offset)
        kp = self.k - 1 if getattr(self, "_offset", False) else self.k
        return glrm_svd_init(self.h, kp, oversample, power_iters, seed)

    def certificate(self, max_iters=1000, tol=1e-10):
        return glrm_certificate(self.h, max_iters, tol)

    def set_reg_weights(self, rx_weight, ry_weight):
        glrm_set_reg_weights(self.h, rx_weight, ry_weight)

    def regularization_path(self, gammas, max_sweeps, rtol, window=1, cert_iters=0):
        return glrm_regularization_path(self.h, gammas, max_sweeps, rtol, window, cert_iters)

    def set_offset(self, on=True):
        glrm_set_offset(self.h, on)
        self._offset = bool(on)

    def column_stats(self):
        """(mu, sigma2) per column, float64 on the device (Sec. 4.3)."""
        mu = torch.empty(self.n, dtype=torch.float64, device=self.device)
        s2 = torch.empty(self.n, dtype=torch.float64, device=self.device)
        glrm_column_stats(self.h, mu, s2)
        return mu, s2

    def set_column_scale(self, w=None):
        glrm_set_column_scale(self.h, None if w is None else
                              (w.detach().cpu().numpy() if isinstance(w, torch.Tensor) else w))

    def accepts(self):
        return glrm_last_accepts(self.h)

    def grad(self):
        """Loss part of the gradient at the current factors: (GX, GYt)."""
        GX = torch.empty(self.m, self.k, dtype=self.dtype, device=self.device)
        GYt = torch.empty(self.n, self.k, dtype=self.dtype, device=self.device)
        glrm_grad(self.h, GX, GYt)
        return GX, GYt

    def predict(self, rows, cols, decode=True):
        out = torch.empty(rows.numel(), dtype=self.dtype, device=self.device)
        glrm_predict(self.h, rows.to(torch.int32).contiguous(), cols.to(torch.int32).contiguous(),
                     out, decode)
        return out

    def state(self) -> bytes:
        return glrm_get_state(self.h)

    def load_state(self, s: bytes):
        glrm_set_state(self.h, s)

    def close(self):
        if self.h:
            glrm_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass
