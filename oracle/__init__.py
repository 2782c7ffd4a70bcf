"""FP64 CPU oracle for the GLRM alternating proximal-gradient method.

TEST INFRASTRUCTURE ONLY: the tests, the smoke check and the CPU-baseline leg
of the benchmark use it to check and time the CUDA library.  It shares no code
with that library and never imports it.

The arithmetic lives in ``glrm_oracle.c`` (plain C, double precision, loops in
index order); this module compiles it with gcc and marshals numpy arrays to it.
Every function follows the passage of Udell et al., "Generalized Low Rank
Models" (arXiv 1410.0342), cited in its docstring.

The observed set is passed as coordinate triples (row, col, value) sorted by
row then column; the oracle builds its own row and column lists from them.
Factors are X (m x k) and Yt = Y^T (n x k), both row-major float64.

Parity status of each function (the pins live in tests/test_oracle_*.py):
  loss / dloss / decode / reg / prox   pinned (closed forms, brute force,
                                       finite differences, Huber identity)
  objective / gradient                 pinned (brute-force loops, finite
                                       differences)
  gradient_abs                         pinned (brute-force loops; equals the
                                       gradient where every term is >= 0)
  gradient_variation                   pinned (closed form for quadratic loss,
                                       the hinge's unit jump at its kink)
  proxgrad                             pinned (qPCA closed form, Eckart-Young,
                                       monotone objective, single-row brute force,
                                       one 2 x 2 sweep followed by hand: Gauss-Seidel
                                       order and both step-rule branches; empty
                                       row / column: alpha = 1, x <- prox(x))
  als                                  pinned (normal equations vs numpy.linalg,
                                       qPCA closed form)
  column_stats                         pinned (quadratic: mean and sample variance;
                                       l1: median; quantile: the alpha-quantile;
                                       logistic log-odds; hinge two-label minimum;
                                       the smallest point of a flat bottom; brute
                                       force over a grid)
  offset                               pinned (objective by hand; k = 1: the
                                       offset row converges to the column mean)
  col_scale (weighted losses)          pinned (objective and gradient by hand; the
                                       sweep's invariance under weights c with
                                       regulariser weights c and steps alpha / c)
  mloss / mgrad / mdecode              pinned (hand values, sums of the scalar hinge
                                       over the block, finite differences, brute-
                                       force decoding with ties)
  FeatureProblem objective / proxgrad  pinned (cell-by-cell sum; scalar features
                                       follow the plain sweep exactly; a block
                                       follows its Boolean columns' sweep exactly)
  entry_derivs / certificate           pinned (the qPCA closed forms: s_{k+1} / w
                                       holding at rank 5 and failing at rank 4;
                                       invariance under X T, Y T^-T)
  svd_init                             pinned (an exactly low-rank table plus
                                       column offsets reproduced; invariance under
                                       affine encodings of a quadratic column)
  proxprox                             pinned (fixed points: the least-squares
                                       solution for r = 0, the closed form
                                       ((1 + 2 alpha gamma) G + gamma I) x = b
                                       for gamma ||x||^2, the NNLS optimality
                                       conditions of the envelope for x >= 0)
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading

import numpy as np

LOSS_QUAD, LOSS_HUBER, LOSS_HINGE, LOSS_LOGISTIC, LOSS_ORDINAL = 0, 1, 2, 3, 4
LOSS_L1, LOSS_QUANTILE = 5, 6
REG_ZERO, REG_QUAD, REG_L1, REG_NONNEG = 0, 1, 2, 3
FEAT_SCALAR, FEAT_CATEGORICAL, FEAT_ORDINAL_MD = 0, 1, 2

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "glrm_oracle.c")
_LIBDIR = os.path.join(_HERE, "lib")
_LIB = os.path.join(_LIBDIR, "libglrm_oracle.so")
_lock = threading.Lock()
_lib = None


def build(force: bool = False) -> str:
    """Compile the oracle with gcc (-O2, OpenMP) into oracle/lib/."""
    os.makedirs(_LIBDIR, exist_ok=True)
    if force or not os.path.exists(_LIB) or os.path.getmtime(_LIB) < os.path.getmtime(_SRC):
        tmp = _LIB + f".tmp{os.getpid()}"
        subprocess.check_call(["gcc", "-O2", "-std=c11", "-fPIC", "-shared", "-fopenmp",
                               "-o", tmp, _SRC, "-lm"])
        os.replace(tmp, _LIB)
    return _LIB


def _load():
    global _lib
    with _lock:
        if _lib is not None:
            return _lib
        lib = ctypes.CDLL(build())
        d, i32, i64 = ctypes.c_double, ctypes.c_int, ctypes.c_int64
        p = ctypes.c_void_p
        lib.oracle_loss.restype = d
        lib.oracle_loss.argtypes = [i32, d, i32, d, d]
        lib.oracle_dloss.restype = d
        lib.oracle_dloss.argtypes = [i32, d, i32, d, d]
        lib.oracle_decode.restype = d
        lib.oracle_decode.argtypes = [i32, i32, d]
        lib.oracle_reg.restype = d
        lib.oracle_reg.argtypes = [i32, d, i32, p]
        lib.oracle_prox.restype = None
        lib.oracle_prox.argtypes = [i32, d, d, i32, p, p]
        lib.oracle_objective.restype = d
        lib.oracle_objective.argtypes = [i64, i64, i32, i64, p, p, p, p, p, p,
                                         i32, d, i32, d, i32, p, p, p, i32]
        lib.oracle_gradient.restype = i32
        lib.oracle_gradient.argtypes = [i64, i64, i32, i64, p, p, p, p, p, p, p, p, p, p, p, i32]
        lib.oracle_gradient_abs.restype = i32
        lib.oracle_gradient_abs.argtypes = [i64, i64, i32, i64, p, p, p, p, p, p, p, p, p, p, i32]
        lib.oracle_gradient_variation.restype = i32
        lib.oracle_gradient_variation.argtypes = [i64, i64, i32, i64, p, p, p, p, p, p, p, p, d, p,
                                                  p, i32]
        lib.oracle_proxgrad.restype = i32
        lib.oracle_proxgrad.argtypes = [i64, i64, i32, i64, p, p, p, p, p, p, i32, d, i32, d, i32,
                                        p, p, p, p, p, i32, p, p, i32]
        lib.oracle_als.restype = i32
        lib.oracle_als.argtypes = [i64, i64, i32, i64, p, p, p, d, p, p, i32, p, i32]
        lib.oracle_proxprox.restype = i32
        lib.oracle_proxprox.argtypes = [i64, i64, i32, i64, p, p, p, i32, d, i32, d, d, i32, p, p, i32,
                                        p, i32]
        lib.oracle_column_stats.restype = i32
        lib.oracle_column_stats.argtypes = [i64, i64, i64, p, p, p, p, p, p, p, p, i32]
        lib.oracle_entry_derivs.restype = i32
        lib.oracle_entry_derivs.argtypes = [i64, i32, p, p, p, p, p, p, p, p, p, p]
        lib.oracle_feature_dim.restype = i32
        lib.oracle_feature_dim.argtypes = [i32, i32]
        lib.oracle_mloss.restype = d
        lib.oracle_mloss.argtypes = [i32, i32, p, d]
        lib.oracle_mgrad.restype = None
        lib.oracle_mgrad.argtypes = [i32, i32, p, d, p]
        lib.oracle_mdecode.restype = d
        lib.oracle_mdecode.argtypes = [i32, i32, p]
        lib.oracle_mobjective.restype = d
        lib.oracle_mobjective.argtypes = [i64, i64, i32, i64, p, p, p, p, p, p, p, p, i32, d, i32, d, p, p, i32]
        lib.oracle_mproxgrad.restype = i32
        lib.oracle_mproxgrad.argtypes = [i64, i64, i32, i64, p, p, p, p, p, p, p, p, i32, d, i32, d, p, p, p, p,
                                         i32, p, p, i32]
        lib.oracle_num_threads.restype = i32
        lib.oracle_num_threads.argtypes = [i32]
        _lib = lib
        return lib


def _ptr(a: np.ndarray):
    return a.ctypes.data_as(ctypes.c_void_p)


def _c(a, dtype):
    return np.ascontiguousarray(a, dtype=dtype)


# ----------------------------------------------------------------- entrywise

def loss(kind: int, u: float, a: float, param: float = 1.0, levels: int = 0) -> float:
    """L(u, a): eq. qpca, Huber (Sec. 4.3), hinge and logistic (Sec. 5.2), eq. ord-pca,
    l1 and quantile (Sec. 4.2, robust and quantile PCA; param = alpha)."""
    return _load().oracle_loss(kind, param, levels, float(u), float(a))


def dloss(kind: int, u: float, a: float, param: float = 1.0, levels: int = 0) -> float:
    """dL/du, 0 at kinks (gradient form of Sec. 7.2)."""
    return _load().oracle_dloss(kind, param, levels, float(u), float(a))


def decode(kind: int, u: float, levels: int = 0) -> float:
    """argmin_a L(u, a) over the loss's domain (Sec. 5.3)."""
    return _load().oracle_decode(kind, levels, float(u))


def reg(kind: int, w: float, x) -> float:
    """r(x) for zero / gamma||x||^2 / lambda||x||_1 / nonnegativity indicator (Sec. 3)."""
    x = _c(x, np.float64)
    return _load().oracle_reg(kind, w, x.size, _ptr(x))


def prox(kind: int, w: float, alpha: float, z) -> np.ndarray:
    """prox_{alpha r}(z) (Sec. 7.2, definition of the proximal operator)."""
    z = _c(z, np.float64)
    out = np.empty_like(z)
    _load().oracle_prox(kind, w, alpha, z.size, _ptr(z), _ptr(out))
    return out


def feature_dim(fkind: int, levels: int) -> int:
    """Width d_j of a feature's block of Y (Sec. 6): 1 scalar, d categorical, d - 1 ordinal."""
    return int(_load().oracle_feature_dim(fkind, levels))


def mloss(fkind: int, levels: int, u, a: float) -> float:
    """Multi-dimensional loss L(u, a), u in R^{d_j} (Sec. 6: one-vs-all categorical, eq. ord-mpca)."""
    u = _c(u, np.float64)
    return _load().oracle_mloss(fkind, levels, _ptr(u), float(a))


def mgrad(fkind: int, levels: int, u, a: float) -> np.ndarray:
    u = _c(u, np.float64)
    g = np.empty_like(u)
    _load().oracle_mgrad(fkind, levels, _ptr(u), float(a), _ptr(g))
    return g


def mdecode(fkind: int, levels: int, u) -> float:
    """Categorical: argmax_l u_l; ordinal: argmin_a L(u, a) over every level (Sec. 6, Sec. 5.3)."""
    u = _c(u, np.float64)
    return _load().oracle_mdecode(fkind, levels, _ptr(u))


# ------------------------------------------------------------------- problem

class Problem:
    """Data of one GLRM (eq. gpca): Omega as sorted (row, col, value) triples,
    per-column losses and the row / column regularisers."""

    def __init__(self, m, n, k, rows, cols, vals, loss_kind, loss_param, loss_levels,
                 rx=(REG_ZERO, 0.0), ry=(REG_ZERO, 0.0), offset=False, col_scale=None):
        self.m, self.n, self.k = int(m), int(n), int(k)
        self.rows = _c(rows, np.int32)
        self.cols = _c(cols, np.int32)
        self.vals = _c(vals, np.float64)
        self.nnz = int(self.rows.size)
        self.loss_kind = _c(np.broadcast_to(loss_kind, (self.n,)), np.int32)
        self.loss_param = _c(np.broadcast_to(loss_param, (self.n,)), np.float64)
        self.loss_levels = _c(np.broadcast_to(loss_levels, (self.n,)), np.int32)
        self.rx = (int(rx[0]), float(rx[1]))
        self.ry = (int(ry[0]), float(ry[1]))
        # offset (Sec. 3.4): the last coordinate of X is held at 1, that of Y
        # is not penalised
        self.offset = bool(offset)
        # per-column loss weights w_j (the scaled losses w_j L_j of Sec. 4.3)
        self.col_scale = None if col_scale is None else _c(np.broadcast_to(col_scale, (self.n,)), np.float64)

    @classmethod
    def from_csr(cls, m, n, k, rowptr, colidx, vals, **kw):
        rowptr = np.asarray(rowptr, dtype=np.int64)
        rows = np.repeat(np.arange(m, dtype=np.int32), np.diff(rowptr))
        return cls(m, n, k, rows, colidx, vals, **kw)

    def row_counts(self) -> np.ndarray:
        return np.bincount(self.rows, minlength=self.m).astype(np.int64)

    def col_counts(self) -> np.ndarray:
        return np.bincount(self.cols, minlength=self.n).astype(np.int64)

    def initial_alphas(self):
        """alpha_i = 1 / max(n_i, 1) and alpha_j = 1 / max(m_j, 1) (Sec. 7.2)."""
        ax = 1.0 / np.maximum(self.row_counts(), 1).astype(np.float64)
        ay = 1.0 / np.maximum(self.col_counts(), 1).astype(np.float64)
        return ax, ay

    def _common(self):
        return (self.m, self.n, self.k, self.nnz, _ptr(self.rows), _ptr(self.cols),
                _ptr(self.vals))

    def _scale(self):
        return None if self.col_scale is None else _ptr(self.col_scale)

    def _losses(self):
        return (_ptr(self.loss_kind), _ptr(self.loss_param), _ptr(self.loss_levels))

    def objective(self, X, Yt, nthreads: int = 0) -> float:
        """sum_Omega L + sum_i r(x_i) + sum_j rt(y_j) (eq. gpca)."""
        X = _c(X, np.float64)
        Yt = _c(Yt, np.float64)
        return _load().oracle_objective(*self._common(), *self._losses(), *self.rx, *self.ry,
                                        int(self.offset), self._scale(), _ptr(X), _ptr(Yt), nthreads)

    def gradient(self, X, Yt, nthreads: int = 0):
        """Loss part of the gradient: G_X = R Y^T and G_Y^T = R^T X over Omega (Sec. 7.2)."""
        X = _c(X, np.float64)
        Yt = _c(Yt, np.float64)
        GX = np.empty_like(X)
        GYt = np.empty_like(Yt)
        rc = _load().oracle_gradient(*self._common(), *self._losses(), self._scale(), _ptr(X), _ptr(Yt),
                                     _ptr(GX), _ptr(GYt), nthreads)
        if rc:
            raise ValueError(f"oracle_gradient failed ({rc})")
        return GX, GYt

    def gradient_abs(self, X, Yt, nthreads: int = 0):
        """Per gradient coordinate, the sum of the magnitudes of its terms:
        sum_{j in Omega_i} |L'| |y_j| and sum_{i in Omega_j} |L'| |x_i| (the
        scale of the rounding error of any summation of the gradient)."""
        X = _c(X, np.float64)
        Yt = _c(Yt, np.float64)
        SX = np.empty_like(X)
        SYt = np.empty_like(Yt)
        rc = _load().oracle_gradient_abs(*self._common(), *self._losses(), _ptr(X), _ptr(Yt),
                                         _ptr(SX), _ptr(SYt), nthreads)
        if rc:
            raise ValueError(f"oracle_gradient_abs failed ({rc})")
        return SX, SYt

    def gradient_variation(self, X, Yt, u_rel: float, nthreads: int = 0):
        """Per gradient coordinate, how far it can move when every product
        x_i . y_j is off by at most u_rel * sum_c |x_ic y_jc|: sum over the
        coordinate's entries of (L'(u + delta) - L'(u - delta)) |w| (L' is
        nondecreasing for the convex losses here)."""
        X = _c(X, np.float64)
        Yt = _c(Yt, np.float64)
        VX = np.empty_like(X)
        VYt = np.empty_like(Yt)
        rc = _load().oracle_gradient_variation(*self._common(), *self._losses(), _ptr(X),
                                               _ptr(Yt), float(u_rel), _ptr(VX), _ptr(VYt),
                                               nthreads)
        if rc:
            raise ValueError(f"oracle_gradient_variation failed ({rc})")
        return VX, VYt

    def proxgrad(self, X, Yt, nsweeps: int, alpha_x=None, alpha_y=None, nthreads: int = 0):
        """Alternating proximal-gradient sweeps with the step-size safeguard
        (Algorithm 2, Sec. 7.2).  Returns (X, Yt, alpha_x, alpha_y, history,
        accepts) with history[t] the objective after sweep t and accepts[t] the
        (rows, columns) accepted in sweep t."""
        X = np.array(X, dtype=np.float64, order="C")
        Yt = np.array(Yt, dtype=np.float64, order="C")
        if alpha_x is None or alpha_y is None:
            alpha_x, alpha_y = self.initial_alphas()
        alpha_x = np.array(alpha_x, dtype=np.float64)
        alpha_y = np.array(alpha_y, dtype=np.float64)
        hist = np.empty(nsweeps, dtype=np.float64)
        acc = np.empty(2 * nsweeps, dtype=np.int64)
        rc = _load().oracle_proxgrad(*self._common(), *self._losses(), *self.rx, *self.ry,
                                     int(self.offset), self._scale(), _ptr(X), _ptr(Yt), _ptr(alpha_x),
                                     _ptr(alpha_y),
                                     nsweeps,
                                     _ptr(hist), _ptr(acc), nthreads)
        if rc:
            raise ValueError(f"oracle_proxgrad failed ({rc})")
        return X, Yt, alpha_x, alpha_y, hist, acc.reshape(nsweeps, 2)

    def als(self, X, Yt, gamma: float, nsweeps: int, nthreads: int = 0):
        """Alternating exact minimisation for quadratic loss + gamma||.||^2
        (Algorithm 1; Sec. 2.4).  Returns (X, Yt, history)."""
        X = np.array(X, dtype=np.float64, order="C")
        Yt = np.array(Yt, dtype=np.float64, order="C")
        hist = np.empty(nsweeps, dtype=np.float64)
        rc = _load().oracle_als(*self._common(), gamma, _ptr(X), _ptr(Yt), nsweeps, _ptr(hist),
                                nthreads)
        if rc:
            raise ValueError(f"oracle_als failed ({rc})")
        return X, Yt, hist

    def column_stats(self, nthreads: int = 0):
        """(mu, sigma2) per column (Sec. 4.3, "Offsets and scaling"): mu_j
        minimises sum_i L_j(mu, A_ij) over the column's observed entries and
        sigma2_j = sum_i L_j(mu_j, A_ij) / (n_j - 1)."""
        mu = np.empty(self.n)
        s2 = np.empty(self.n)
        rc = _load().oracle_column_stats(self.m, self.n, self.nnz, _ptr(self.rows), _ptr(self.cols),
                                         _ptr(self.vals), *self._losses(), _ptr(mu), _ptr(s2), nthreads)
        if rc:
            raise ValueError(f"oracle_column_stats failed ({rc})")
        return mu, s2

    def entry_derivs(self, X, Yt):
        """w_j L_j'(x_i . y_j, A_ij) per observed entry (rows, then columns)."""
        X = _c(X, np.float64)
        Yt = _c(Yt, np.float64)
        out = np.empty(self.nnz)
        _load().oracle_entry_derivs(self.nnz, self.k, _ptr(self.rows), _ptr(self.cols), _ptr(self.vals),
                                    *self._losses(), self._scale(), _ptr(X), _ptr(Yt), _ptr(out))
        return out

    def certificate(self, X, Yt, rank_rtol: float = 1e-10):
        """||(1/gamma) G + U V^T||_2 (Sec. 7.6, eq. convex-certificate) for the
        quadratic regulariser w (||X||^2 + ||Y||^2) of this problem: with
        ||Z||_* = inf 1/2 (||X||^2 + ||Y||^2) over X Y = Z (Sec. 7.6's lemma)
        the convex problem is L(Z) + 2 w ||Z||_*, so gamma = 2 w.  G is the
        m x n loss gradient (zero off Omega), U V^T the product of the
        singular vectors of Z = X Y with singular values above rank_rtol
        times the largest.  Dense numpy (library SVD and matrix 2-norm): for
        small problems."""
        if self.rx[0] != REG_QUAD or self.ry[0] != REG_QUAD or self.rx[1] != self.ry[1] or self.rx[1] <= 0:
            raise ValueError("the certificate needs one quadratic regulariser weight on X and Y")
        gamma = 2.0 * self.rx[1]
        X = np.asarray(X, np.float64)
        Yt = np.asarray(Yt, np.float64)
        G = np.zeros((self.m, self.n))
        G[self.rows, self.cols] = self.entry_derivs(X, Yt)
        U, sv, Vt = np.linalg.svd(X @ Yt.T, full_matrices=False)
        r = int(np.sum(sv > rank_rtol * sv[0])) if sv.size and sv[0] > 0 else 0
        M = G / gamma + U[:, :r] @ Vt[:r]
        return float(np.linalg.norm(M, 2))

    def svd_init(self, offset: bool = False):
        """SVD initialisation (Sec. 7.5): the scaled table
        A~_ij = m / (sigma_j m_j) (A_ij - mu_j) on Omega (0 elsewhere; a column
        without a finite sigma_j > 0 is 0 and takes sigma_j = 1), its top k'
        singular triples (k' = k - 1 with the offset, else k; numpy's dense
        SVD), X = U S^1/2, Y = S^1/2 V^T diag(sigma), and with the offset X's
        last column 1 and Y's last row mu (0 where undefined).  Returns
        (X, Yt, S[:k'])."""
        kp = self.k - 1 if offset else self.k
        mu, s2 = self.column_stats()
        sg = np.sqrt(s2)
        valid = np.isfinite(sg) & (sg > 0)
        mj = self.col_counts().astype(np.float64)
        fac = np.where(valid, self.m / (np.where(valid, sg, 1.0) * np.maximum(mj, 1.0)), 0.0)
        At = np.zeros((self.m, self.n))
        At[self.rows, self.cols] = fac[self.cols] * (self.vals - np.nan_to_num(mu)[self.cols])
        U, S, Vt = np.linalg.svd(At, full_matrices=False)
        X = np.zeros((self.m, self.k))
        Yt = np.zeros((self.n, self.k))
        r = np.sqrt(S[:kp])
        X[:, :kp] = U[:, :kp] * r
        Yt[:, :kp] = Vt[:kp].T * r * np.where(valid, sg, 1.0)[:, None]
        if offset:
            X[:, self.k - 1] = 1.0
            Yt[:, self.k - 1] = np.nan_to_num(mu)
        return X, Yt, S[:kp]

    def proxprox(self, X, Yt, alpha: float, inner: int, nsweeps: int, nthreads: int = 0):
        """Alternating prox-prox sweeps for quadratic loss (Sec. 7.2 prox-prox
        update, Sec. 7.3 cached factorisation) with the problem's regularisers:
        each row, then each column, takes `inner` updates
        v <- prox_{alpha r}((2 alpha G + I)^{-1} (2 alpha b + v)).  Returns
        (X, Yt, history)."""
        X = np.array(X, dtype=np.float64, order="C")
        Yt = np.array(Yt, dtype=np.float64, order="C")
        hist = np.empty(nsweeps, dtype=np.float64)
        rc = _load().oracle_proxprox(*self._common(), *self.rx, *self.ry, float(alpha), int(inner),
                                     _ptr(X), _ptr(Yt), nsweeps, _ptr(hist), nthreads)
        if rc:
            raise ValueError(f"oracle_proxprox failed ({rc})")
        return X, Yt, hist


class FeatureProblem:
    """A table of features (eq. mpca, Sec. 6): Omega as sorted (row, feature,
    value) triples, per feature its kind (FEAT_*), label / level count and,
    for scalar features, its loss.  Y has d = sum_j d_j columns, feature j's
    block first[j] .. first[j+1]-1; Yt is d x k."""

    def __init__(self, m, nf, k, rows, feats, vals, fkind, flevels, loss_kind, loss_param, loss_levels,
                 rx=(REG_ZERO, 0.0), ry=(REG_ZERO, 0.0)):
        self.m, self.nf, self.k = int(m), int(nf), int(k)
        self.rows = _c(rows, np.int32)
        self.feats = _c(feats, np.int32)
        self.vals = _c(vals, np.float64)
        self.nnz = int(self.rows.size)
        self.fkind = _c(np.broadcast_to(fkind, (self.nf,)), np.int32)
        self.flevels = _c(np.broadcast_to(flevels, (self.nf,)), np.int32)
        self.loss_kind = _c(np.broadcast_to(loss_kind, (self.nf,)), np.int32)
        self.loss_param = _c(np.broadcast_to(loss_param, (self.nf,)), np.float64)
        self.loss_levels = _c(np.broadcast_to(loss_levels, (self.nf,)), np.int32)
        self.rx = (int(rx[0]), float(rx[1]))
        self.ry = (int(ry[0]), float(ry[1]))
        dims = np.array([feature_dim(int(a), int(b)) for a, b in zip(self.fkind, self.flevels)], np.int64)
        self.first = np.concatenate([[0], np.cumsum(dims)]).astype(np.int64)
        self.d = int(self.first[-1])

    def _args(self):
        return (self.m, self.nf, self.k, self.nnz, _ptr(self.rows), _ptr(self.feats), _ptr(self.vals),
                _ptr(self.fkind), _ptr(self.flevels), _ptr(self.loss_kind), _ptr(self.loss_param),
                _ptr(self.loss_levels), *self.rx, *self.ry)

    def initial_alphas(self):
        """1 / max(count, 1), count = scalar loss terms: sum of d_j over a row's
        features; feature j's observation count for each column of its block."""
        dims = np.diff(self.first)
        rowterms = np.bincount(self.rows, weights=dims[self.feats], minlength=self.m)
        fcount = np.bincount(self.feats, minlength=self.nf).astype(np.float64)
        ax = 1.0 / np.maximum(rowterms, 1.0)
        ay = 1.0 / np.maximum(np.repeat(fcount, dims), 1.0)
        return ax, ay

    def objective(self, X, Yt, nthreads: int = 0) -> float:
        X = _c(X, np.float64)
        Yt = _c(Yt, np.float64)
        return _load().oracle_mobjective(*self._args(), _ptr(X), _ptr(Yt), nthreads)

    def proxgrad(self, X, Yt, nsweeps: int, alpha_x=None, alpha_y=None, nthreads: int = 0):
        """Sweeps of Algorithm 2 on eq. mpca; returns (X, Yt, alpha_x, alpha_y,
        history, accepts) like Problem.proxgrad (accepts: rows, columns of Y)."""
        X = np.array(X, dtype=np.float64, order="C")
        Yt = np.array(Yt, dtype=np.float64, order="C")
        if alpha_x is None or alpha_y is None:
            alpha_x, alpha_y = self.initial_alphas()
        alpha_x = np.array(alpha_x, dtype=np.float64)
        alpha_y = np.array(alpha_y, dtype=np.float64)
        hist = np.empty(nsweeps)
        acc = np.empty(2 * nsweeps, dtype=np.int64)
        rc = _load().oracle_mproxgrad(*self._args(), _ptr(X), _ptr(Yt), _ptr(alpha_x), _ptr(alpha_y),
                                      nsweeps, _ptr(hist), _ptr(acc), nthreads)
        if rc:
            raise ValueError(f"oracle_mproxgrad failed ({rc})")
        return X, Yt, alpha_x, alpha_y, hist, acc.reshape(nsweeps, 2)


def num_threads(nthreads: int = 0) -> int:
    """Threads the oracle's OpenMP loops use (after setting them, if > 0)."""
    return _load().oracle_num_threads(nthreads)
