"""Offsets and scaling (Sec. 3.4 and Sec. 4.3, "Offsets and scaling") on the
GPU against the FP64 oracle: the column statistics mu_j, sigma2_j of every
loss kind (sparse and dense tables, empty and single-entry columns), sweeps
with the offset on every kernel path, and sweeps, objective and gradient with
per-column loss weights w_j = 1 / sigma2_j."""
import numpy as np
import pytest
import torch

from paper_1410_0342_gb300 import workloads as W

from gpu_parity import (assert_grad_close, decode_state, grad_bounds, oracle_problem, subset_table,
                        synced_sweeps)

pytestmark = pytest.mark.gpu

Q, HU, HI, LO, OR, L1, QT = 0, 1, 2, 3, 4, 5, 6
RZ, RQ, RL1, RNN = 0, 1, 2, 3


@pytest.fixture(scope="module")
def G():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1410_0342_gb300 import build
    build.build()
    from paper_1410_0342_gb300 import glrm
    return glrm


def _sum_S(o, t, mu):
    """sum_j S_j(mu_j) by the oracle: the objective of the k = 1 model
    x_i = 1, y_j = mu_j with no regulariser."""
    t1 = W.Table(t.name, t.m, t.n, 1, t.rowptr, t.colidx, t.val, t.colptr, t.rowidx, t.cval,
                 t.loss_kind, t.loss_param, t.loss_levels, (RZ, 0.0), (RZ, 0.0),
                 np.ones((t.m, 1)), np.zeros((t.n, 1)))
    p = oracle_problem(o, t1)
    return p.objective(np.ones((t.m, 1)), np.nan_to_num(np.asarray(mu, np.float64))[:, None])


def rounded(t, dtype):
    """The table with its values rounded to the model's element type (what
    the handle holds), in FP64."""
    r = lambda v: np.asarray(v).astype(dtype).astype(np.float64)
    return W.Table(t.name, t.m, t.n, t.k, t.rowptr, t.colidx, r(t.val), t.colptr, t.rowidx, r(t.cval),
                   t.loss_kind, t.loss_param, t.loss_levels, t.rx, t.ry, t.X0, t.Yt0)


def check_stats(o, t, mu, s2, fp64=False):
    """sigma2 of every column equal to the oracle's (both are minima of S_j,
    which is flat at its minimiser), mu of every column (the smallest
    minimiser), sum_j S_j(mu_j) at the oracle's minimum, NaN exactly where
    the oracle has NaN.  The oracle reads the
    values the handle holds (rounded to its element type)."""
    if not fp64:
        t = rounded(t, np.float32)
    mu = mu.cpu().numpy()
    s2 = s2.cpu().numpy()
    mo, so = oracle_problem(o, t).column_stats()
    np.testing.assert_array_equal(np.isnan(mu), np.isnan(mo))
    np.testing.assert_array_equal(np.isnan(s2), np.isnan(so))
    f = ~np.isnan(so)
    np.testing.assert_allclose(s2[f], so[f], rtol=1e-9, atol=1e-12)
    # every kind: both take the smallest minimiser where the minimisers form
    # an interval (the flat-bottomed hinge, ordinal, l1 and quantile sums)
    f = ~np.isnan(mo)
    err = np.abs(mu[f] - mo[f])
    assert np.all(err <= 1e-6 * (1 + np.abs(mo[f]))), err.max()
    assert _sum_S(o, t, mu) <= _sum_S(o, t, mo) * (1 + 1e-12) + 1e-12


@pytest.mark.parametrize("prec", [1, 0])
def test_column_stats_sparse(G, oracle_mod, prec):
    t = W.small_mixed(m=2500, n=70, k=3, p_obs=0.4, seed=601, nkinds=7)
    rows = t.rows()
    # column 0 empty, column 7 a single entry, column 14 two entries
    keep = ~((t.colidx == 0) | ((t.colidx == 7) & (rows > rows[t.colidx == 7].min())) |
             ((t.colidx == 14) & (rows > np.sort(rows[t.colidx == 14])[1])))
    t = subset_table(t, keep)
    g = G.GLRM.from_table(t, precision=prec)
    mu, s2 = g.column_stats()
    torch.cuda.synchronize()
    assert np.isnan(mu[0].item()) and np.isnan(s2[0].item())
    assert np.isnan(s2[7].item()) and not np.isnan(mu[7].item())
    check_stats(oracle_mod, t, mu, s2, fp64=prec == G.GLRM_FP64)


def test_column_stats_long_columns(G, oracle_mod):
    """Columns of 20000 entries: the warp strides many times per bisection step."""
    t = W.small_mixed(m=40000, n=14, k=2, p_obs=0.5, seed=602, nkinds=7)
    g = G.GLRM.from_table(t)
    mu, s2 = g.column_stats()
    check_stats(oracle_mod, t, mu, s2)


def test_column_stats_dense(G, oracle_mod):
    """A fully observed table on the dense form (the 32-column CTA kernel),
    with a ragged last block of columns."""
    t = W.small_mixed(m=3001, n=77, k=4, p_obs=1.0, seed=603, nkinds=7)
    assert t.nnz == t.m * t.n
    g = G.GLRM.from_dense_table(t)
    assert tuple(G.glrm_get_path(g.h)) == (G.GLRM_PATH_DENSE, G.GLRM_PATH_DENSE)
    mu, s2 = g.column_stats()
    check_stats(oracle_mod, t, mu, s2)


def _offset_init(t, mu=None):
    X0 = t.X0.copy()
    X0[:, -1] = 1.0
    Yt0 = t.Yt0.copy()
    if mu is not None:
        Yt0[:, -1] = np.nan_to_num(mu)
    return W.Table(t.name, t.m, t.n, t.k, t.rowptr, t.colidx, t.val, t.colptr, t.rowidx, t.cval,
                   t.loss_kind, t.loss_param, t.loss_levels, t.rx, t.ry,
                   X0.astype(np.float32), Yt0.astype(np.float32))


@pytest.mark.parametrize("paths", [(1, 1), (2, 2), (3, 3), (4, 4), (5, 5), (6, 6)])
def test_offset_paths_match_oracle(G, oracle_mod, paths):
    """Offset on every kernel path (6: the dense form of a sparse table), from
    the initialisation of Sec. 7.5 (x_ik = 1, y_jk = mu_j)."""
    t = W.small_mixed(m=1303, n=140, k=8, p_obs=0.5, seed=610, nkinds=7, rx=(RQ, 0.1), ry=(RL1, 0.05))
    mo, _ = oracle_problem(oracle_mod, t).column_stats()
    t = _offset_init(t, mo)
    g = G.GLRM.from_table(t)
    g.set_offset(True)
    G.glrm_set_path(g.h, *paths)
    synced_sweeps(g, oracle_mod, t, 6, offset=True)


def test_offset_from_unset_coordinate(G, oracle_mod):
    """x_ik != 1 at the start: objective +inf, the first X-step sets it to 1
    (every row step accepted), then the sweeps follow the oracle."""
    t = W.small_mixed(m=900, n=60, k=5, p_obs=0.5, seed=611, nkinds=7, rx=(RQ, 0.1), ry=(RNN, 0.0))
    g = G.GLRM.from_table(t)
    g.set_offset(True)
    assert g.objective() == np.inf
    synced_sweeps(g, oracle_mod, t, 4, offset=True)
    X, _ = g.factors()
    assert torch.all(X[:, -1] == 1.0)


def test_offset_fp64_and_grad(G, oracle_mod):
    t = _offset_init(W.small_mixed(m=700, n=50, k=4, p_obs=0.6, seed=612, nkinds=7, rx=(RQ, 0.2),
                                   ry=(RQ, 0.3)))
    g = G.GLRM.from_table(t, precision=G.GLRM_FP64)
    g.set_offset(True)
    hist = g.sweep(10)
    p = oracle_problem(oracle_mod, t, offset=True)
    _, _, _, _, oh, _ = p.proxgrad(t.X0, t.Yt0, 10)
    np.testing.assert_allclose(hist, oh, rtol=1e-9)
    X, Yt = g.factors()
    assert abs(g.objective() - p.objective(X.cpu().numpy(), Yt.cpu().numpy())) < 1e-10 * abs(oh[-1])
    # the loss gradient does not depend on the offset; with the regulariser the
    # held coordinate contributes 0 and y's last coordinate is unpenalised
    GX = torch.empty_like(X)
    GY = torch.empty_like(Yt)
    G.glrm_grad_at(g.h, X, Yt, GX, GY, True)
    gx, gy = p.gradient(X.cpu().numpy(), Yt.cpu().numpy())
    gx[:, :-1] += 2 * 0.2 * X.cpu().numpy()[:, :-1]
    gy[:, :-1] += 2 * 0.3 * Yt.cpu().numpy()[:, :-1]
    np.testing.assert_allclose(GX.cpu().numpy(), gx, rtol=1e-9, atol=1e-9)
    np.testing.assert_allclose(GY.cpu().numpy(), gy, rtol=1e-9, atol=1e-9)


def test_offset_refused_by_als_and_proxprox(G):
    t = W.qpca_dense(m=50, n=30, k=3, seed=3)
    g = G.GLRM.from_table(t)
    g.set_offset(True)
    with pytest.raises(G.GLRMError):
        g.als_sweep(1)
    with pytest.raises(G.GLRMError):
        g.proxprox_sweep(1, 1.0, 2)
    g.set_offset(False)
    g.als_sweep(1)


def _weights(s2):
    s2 = np.asarray(s2, np.float64)
    return np.where(np.isfinite(s2) & (s2 > 0), 1.0 / np.where(s2 > 0, s2, 1.0), 1.0)


@pytest.mark.parametrize("paths", [(1, 1), (2, 2), (4, 4), (6, 6)])
def test_scaled_losses_match_oracle(G, oracle_mod, paths):
    """w_j = 1 / sigma2_j from the GPU's own statistics (the standardised GLRM
    of Sec. 4.3, with the offset); the weighted half-steps run on the dense
    form where it was asked for (6), else on the chunked path."""
    t = W.small_mixed(m=1303, n=140, k=8, p_obs=0.5, seed=620, nkinds=7, rx=(RQ, 0.1), ry=(RQ, 0.1))
    g = G.GLRM.from_table(t)
    G.glrm_set_path(g.h, *paths)
    mu, s2 = g.column_stats()
    w = _weights(s2.cpu().numpy())
    t = _offset_init(t, mu.cpu().numpy())
    g.set_factors(torch.as_tensor(t.X0, device=g.device), torch.as_tensor(t.Yt0, device=g.device))
    g.set_offset(True)
    g.set_column_scale(w)
    want = G.GLRM_PATH_DENSE if paths == (6, 6) else G.GLRM_PATH_CHUNKED
    assert tuple(G.glrm_get_path(g.h)) == (want, want)
    synced_sweeps(g, oracle_mod, t, 6, offset=True, col_scale=w)
    g.set_column_scale(None)
    synced_sweeps(g, oracle_mod, t, 2, offset=True)


def test_scaled_fp64_objective_and_gradient(G, oracle_mod):
    t = W.small_mixed(m=800, n=64, k=5, p_obs=0.5, seed=621, nkinds=7, rx=(RQ, 0.2), ry=(RQ, 0.2))
    w = np.random.default_rng(5).uniform(0.25, 4.0, size=t.n)
    g = G.GLRM.from_table(t, precision=G.GLRM_FP64)
    g.set_column_scale(w)
    p = oracle_problem(oracle_mod, t, col_scale=w)
    hist = g.sweep(8)
    _, _, _, _, oh, _ = p.proxgrad(t.X0, t.Yt0, 8)
    np.testing.assert_allclose(hist, oh, rtol=1e-9)
    X, Yt = g.factors()
    GX, GY = g.grad()
    gx, gy = p.gradient(X.cpu().numpy(), Yt.cpu().numpy())
    np.testing.assert_allclose(GX.cpu().numpy(), gx, rtol=1e-9, atol=1e-9)
    np.testing.assert_allclose(GY.cpu().numpy(), gy, rtol=1e-9, atol=1e-9)


def test_scale_arguments(G):
    t = W.qpca_dense(m=40, n=20, k=3, seed=4)
    g = G.GLRM.from_table(t)
    for bad in (np.zeros(t.n), np.full(t.n, np.inf), -np.ones(t.n)):
        with pytest.raises(G.GLRMError):
            g.set_column_scale(bad)
    g.set_column_scale(np.ones(t.n))
    with pytest.raises(G.GLRMError):
        g.als_sweep(1)
    with pytest.raises(G.GLRMError):
        g.proxprox_sweep(1, 1.0, 2)
    b = G.GLRM.from_table(t, precision=G.GLRM_BF16)
    with pytest.raises(G.GLRMError):
        b.set_column_scale(np.ones(t.n))



@pytest.mark.parametrize("m,n,k", [(1000, 301, 20), (129, 65, 16)])
def test_scaled_dense_table_matches_oracle(G, oracle_mod, m, n, k):
    """Weighted losses on a fully observed table (the tensor-core form, every
    loss kind, ragged against the 128-row tiles and 64-wide chunks): sweeps
    from a state shared with the oracle, then objective and gradient at the
    factors reached.  The oracle's gradient bounds are of the unweighted
    terms: a row coordinate's terms carry weights up to max w, a column's its
    own w_j."""
    t = W.small_mixed(m=m, n=n, k=k, p_obs=1.0, seed=622 + k, nkinds=7, rx=(RQ, 0.1), ry=(RQ, 0.1))
    w = np.random.default_rng(k).uniform(0.25, 4.0, size=n)
    g = G.GLRM.from_dense_table(t)
    g.set_column_scale(w)
    assert tuple(G.glrm_get_path(g.h)) == (G.GLRM_PATH_DENSE, G.GLRM_PATH_DENSE)
    synced_sweeps(g, oracle_mod, t, 6, col_scale=w)
    X, Yt = g.factors()
    Xd = X.double().cpu().numpy()
    Yd = Yt.double().cpu().numpy()
    p = oracle_problem(oracle_mod, t, col_scale=w)
    of = p.objective(Xd, Yd)
    assert abs(g.objective() - of) <= 1e-5 * abs(of), (g.objective(), of)
    GX = torch.empty_like(X)
    GY = torch.empty_like(Yt)
    G.glrm_grad_at(g.h, X, Yt, GX, GY, False)
    oGX, oGY = p.gradient(Xd, Yd)
    sX, sY, vX, vY = grad_bounds(oracle_problem(oracle_mod, t), Xd, Yd)
    assert_grad_close(GX.cpu().numpy(), oGX, sX * w.max(), vX * w.max(), what="GX")
    assert_grad_close(GY.cpu().numpy(), oGY, sY * w[:, None], vY * w[:, None], what="GYt")
    g.set_column_scale(None)
    synced_sweeps(g, oracle_mod, t, 2)
