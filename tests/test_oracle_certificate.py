"""Pins of the oracle's global optimality certificate (Sec. 7.6, eq.
convex-certificate) and of the regularisation path by homotopy (Sec. 8.1).

For quadratic loss on a fully observed table and the regulariser
w (||X||^2 + ||Y||^2), the optimum of the unconstrained problem
||A - Z||^2 + 2 w ||Z||_* is Z = U (S - w)_+ V^T (the closed form of Sec. 2.4
and Appendix A).  At the rank-k solution that keeps every singular value
above w, G = 2 (Z - A) = -2 U min(S, w) V^T, so
    (1/(2w)) G + U_k V_k^T = -U diag(min(s_i, w)/w [s_i <= w]) V^T
and the certificate is max_{s_i <= w} s_i / w < 1.  A rank-k solution that
drops a singular value s_{k+1} > w has certificate s_{k+1} / w > 1."""
import numpy as np
import pytest

from paper_1410_0342_gb300 import workloads as W

RQ = 1


def qpca_problem(o, t, k, w):
    return o.Problem.from_csr(t.m, t.n, k, t.rowptr, t.colidx, t.val, loss_kind=t.loss_kind,
                              loss_param=t.loss_param, loss_levels=t.loss_levels, rx=(RQ, w), ry=(RQ, w))


def optimum(A, k, w):
    U, s, Vt = np.linalg.svd(A, full_matrices=False)
    r = np.sqrt(np.maximum(s[:k] - w, 0.0))
    return U[:, :k] * r, Vt[:k].T * r, s


def test_certificate_closed_form_holds(oracle_mod):
    t = W.qpca_dense(m=200, n=100, k=5, seed=7)
    A = t.val.reshape(t.m, t.n)
    X, Yt, s = optimum(A, 5, 5.0)
    p = qpca_problem(oracle_mod, t, 5, 5.0)
    assert p.certificate(X, Yt) == pytest.approx(s[5] / 5.0, rel=1e-10)
    assert p.certificate(X, Yt) < 1.0


def test_certificate_closed_form_fails_for_too_small_rank(oracle_mod):
    t = W.qpca_dense(m=200, n=100, k=5, seed=7)
    A = t.val.reshape(t.m, t.n)
    X, Yt, s = optimum(A, 4, 5.0)
    p = qpca_problem(oracle_mod, t, 4, 5.0)
    assert p.certificate(X, Yt) == pytest.approx(s[4] / 5.0, rel=1e-10)
    assert p.certificate(X, Yt) > 1.0


def test_certificate_depends_on_z_only(oracle_mod):
    """(X T, Y T^-T) has the same product: the same certificate."""
    t = W.qpca_dense(m=60, n=40, k=3, seed=9)
    p = qpca_problem(oracle_mod, t, 3, 0.5)
    rng = np.random.default_rng(9)
    X, Yt = t.X0, t.Yt0
    T = rng.normal(size=(3, 3)) + 3 * np.eye(3)
    c1 = p.certificate(X, Yt)
    c2 = p.certificate(X @ T, Yt @ np.linalg.inv(T).T)
    assert c2 == pytest.approx(c1, rel=1e-9)


def test_path_reaches_each_closed_form(oracle_mod):
    """Homotopy over decreasing weights, warm-started, step sizes reset per
    weight: each weight's objective reaches its closed-form optimum
    ||A||^2 - sum_{i<=k} ((s_i - w)_+)^2.  (The path starts below s_1: above
    it the factors decay towards (0, 0), a stationary point of every weight,
    from which smaller weights recover only slowly.)"""
    t = W.qpca_dense(m=200, n=100, k=5, seed=7)
    A = t.val.reshape(t.m, t.n)
    s = np.linalg.svd(A, compute_uv=False)
    X, Yt = t.X0, t.Yt0
    for w in (160.0, 40.0, 10.0):
        p = qpca_problem(oracle_mod, t, 5, w)
        X, Yt, _, _, hist, _ = p.proxgrad(X, Yt, 300)
        fstar = float(np.sum(A * A) - np.sum(np.maximum(s[:5] - w, 0.0) ** 2))
        assert hist[-1] == pytest.approx(fstar, rel=1e-9)
        # and the certificate of the converged factors is the closed form
        assert p.certificate(X, Yt) == pytest.approx(max(s[s <= w]) / w, rel=1e-4)
