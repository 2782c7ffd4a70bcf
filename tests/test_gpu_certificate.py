"""The optimality certificate (Sec. 7.6) and the regularisation path
(Sec. 8.1) on the GPU: the certificate against its closed form at the qPCA
optimum (holding at rank 5, failing at rank 4) and against the oracle's dense
computation on mixed-loss tables; the path against the oracle replaying the
same sweep counts, each weight's closed-form optimum and certificate."""
import numpy as np
import pytest
import torch

from paper_1410_0342_gb300 import workloads as W

from gpu_parity import oracle_problem

pytestmark = pytest.mark.gpu

RQ = 1


@pytest.fixture(scope="module")
def G():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1410_0342_gb300 import build
    build.build()
    from paper_1410_0342_gb300 import glrm
    return glrm


def _table(t, k, w):
    return W.Table(t.name, t.m, t.n, k, t.rowptr, t.colidx, t.val, t.colptr, t.rowidx, t.cval, t.loss_kind,
                   t.loss_param, t.loss_levels, (RQ, w), (RQ, w), t.X0[:, :k], t.Yt0[:, :k])


@pytest.mark.parametrize("k,prec", [(5, 0), (4, 0), (5, 1)])
def test_certificate_closed_form(G, k, prec):
    t = _table(W.qpca_dense(m=200, n=100, k=5, seed=7), k, 5.0)
    A = t.val.reshape(t.m, t.n)
    U, s, Vt = np.linalg.svd(A, full_matrices=False)
    r = np.sqrt(np.maximum(s[:k] - 5.0, 0.0))
    g = G.GLRM.from_table(t, precision=prec)
    g.set_factors(torch.as_tensor(U[:, :k] * r, dtype=g.dtype, device="cuda"),
                  torch.as_tensor(Vt[:k].T * r, dtype=g.dtype, device="cuda"))
    val, it = g.certificate(max_iters=3000, tol=1e-13)
    want = s[k] / 5.0  # the largest singular value left out
    assert val == pytest.approx(want, rel=1e-6 if prec == 0 else 1e-4), (val, want, it)
    assert (val < 1.0) == (k == 5)


@pytest.mark.parametrize("seed,loss", [(1, "mixed"), (2, "huber"), (3, "logistic")])
def test_certificate_matches_oracle(G, oracle_mod, seed, loss):
    if loss == "mixed":
        t = W.small_mixed(m=400, n=90, k=6, p_obs=0.5, seed=700 + seed, rx=(RQ, 0.3), ry=(RQ, 0.3), nkinds=7)
    else:
        kind = {"huber": 1, "logistic": 3}[loss]
        t = W.small_mixed(m=400, n=90, k=6, p_obs=0.5, seed=700 + seed, rx=(RQ, 0.3), ry=(RQ, 0.3), nkinds=7)
        t = W.Table(t.name, t.m, t.n, t.k, t.rowptr, t.colidx, t.val if kind == 1 else np.sign(t.val) + (t.val == 0),
                    t.colptr, t.rowidx, t.cval if kind == 1 else np.sign(t.cval) + (t.cval == 0),
                    np.full(t.n, kind, np.int32), np.ones(t.n), np.zeros(t.n, np.int32), t.rx, t.ry, t.X0, t.Yt0)
    g = G.GLRM.from_table(t, precision=G.GLRM_FP64)
    g.sweep(30)
    X, Yt = (a.cpu().numpy() for a in g.factors())
    val, it = g.certificate(max_iters=20000, tol=1e-14)
    want = oracle_problem(oracle_mod, t).certificate(X, Yt)
    assert val <= want * (1 + 1e-12)  # power iteration approaches the norm from below
    assert val == pytest.approx(want, rel=1e-5), (val, want, it)


def test_certificate_with_column_weights(G, oracle_mod):
    t = W.small_mixed(m=300, n=60, k=4, p_obs=0.6, seed=710, rx=(RQ, 0.2), ry=(RQ, 0.2), nkinds=7)
    w = np.random.default_rng(3).uniform(0.5, 2.0, size=t.n)
    g = G.GLRM.from_table(t, precision=G.GLRM_FP64)
    g.set_column_scale(w)
    g.sweep(20)
    X, Yt = (a.cpu().numpy() for a in g.factors())
    val, _ = g.certificate(max_iters=20000, tol=1e-14)
    want = oracle_problem(oracle_mod, t, col_scale=w).certificate(X, Yt)
    assert val == pytest.approx(want, rel=1e-5)


def test_certificate_arguments(G):
    t = W.small_mixed(m=50, n=20, k=3, seed=711)  # l1 / nonnegativity regularisers
    g = G.GLRM.from_table(t)
    with pytest.raises(G.GLRMError):
        g.certificate()
    t2 = _table(W.qpca_dense(m=40, n=30, k=3, seed=3), 3, 0.5)
    g2 = G.GLRM.from_table(t2)
    g2.set_offset(True)
    with pytest.raises(G.GLRMError):
        g2.certificate()


def test_regularization_path_matches_oracle(G, oracle_mod):
    """FP64 path over decreasing weights: the oracle runs the same number of
    sweeps per weight from the same warm start (steps reset per weight);
    objectives to 1e-9; every weight reaches its closed form; the
    certificates are the closed forms max_{s_i <= w} s_i / w."""
    t = _table(W.qpca_dense(m=200, n=100, k=5, seed=7), 5, 1.0)
    A = t.val.reshape(t.m, t.n)
    s = np.linalg.svd(A, compute_uv=False)
    gammas = [160.0, 40.0, 10.0]
    g = G.GLRM.from_table(t, precision=G.GLRM_FP64)
    obj, sweeps, cert = g.regularization_path(gammas, max_sweeps=2000, rtol=1e-13, window=5, cert_iters=5000)
    X, Yt = t.X0, t.Yt0
    for w, f, ns, c in zip(gammas, obj, sweeps, cert):
        p = oracle_mod.Problem.from_csr(t.m, t.n, 5, t.rowptr, t.colidx, t.val, loss_kind=t.loss_kind,
                                        loss_param=t.loss_param, loss_levels=t.loss_levels, rx=(RQ, w), ry=(RQ, w))
        X, Yt, _, _, hist, _ = p.proxgrad(X, Yt, int(ns))
        assert f == pytest.approx(hist[-1], rel=1e-9)
        fstar = float(np.sum(A * A) - np.sum(np.maximum(s[:5] - w, 0.0) ** 2))
        assert f == pytest.approx(fstar, rel=1e-8)
        assert c == pytest.approx(max(s[s <= w]) / w, rel=1e-4)
    Xg, Yg = (a.cpu().numpy() for a in g.factors())
    np.testing.assert_allclose(Xg @ Yg.T, X @ Yt.T, rtol=0, atol=1e-6 * np.abs(X @ Yt.T).max())


def test_certificate_tall_table(G, oracle_mod):
    """6,000 x 24: columns of 6,000 entries take the chunked products (chunk
    partials summed per column in chunk order); the closed form at the qPCA
    optimum and the oracle at other factors."""
    t = _table(W.qpca_dense(m=6000, n=24, k=3, seed=17), 3, 2.0)
    A = t.val.reshape(t.m, t.n)
    U, s, Vt = np.linalg.svd(A, full_matrices=False)
    r = np.sqrt(np.maximum(s[:3] - 2.0, 0.0))
    g = G.GLRM.from_table(t, precision=G.GLRM_FP64)
    g.set_factors(torch.as_tensor(U[:, :3] * r, dtype=g.dtype, device="cuda"),
                  torch.as_tensor(Vt[:3].T * r, dtype=g.dtype, device="cuda"))
    val, _ = g.certificate(max_iters=5000, tol=1e-14)
    assert val == pytest.approx(s[3] / 2.0, rel=1e-6)
    g.set_factors(torch.as_tensor(t.X0, dtype=g.dtype, device="cuda"),
                  torch.as_tensor(t.Yt0, dtype=g.dtype, device="cuda"))
    g.sweep(3)
    X, Yt = (a.cpu().numpy() for a in g.factors())
    val, _ = g.certificate(max_iters=20000, tol=1e-14)
    assert val == pytest.approx(oracle_problem(oracle_mod, t).certificate(X, Yt), rel=1e-5)
