"""SVD initialisation (Sec. 7.5) on the GPU against the oracle's dense-SVD
construction: the initial product X Y (independent of the singular vectors'
signs) and the singular values, with and without the offset, FP64 and FP32,
on a noisy low-rank table with missing entries, a mixed-loss table and an
exactly low-rank table that the offset model reproduces."""
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


def _rounded(t, prec):
    if prec == 0:
        return t
    r = lambda v: np.asarray(v).astype(np.float32).astype(np.float64)
    return W.Table(t.name, t.m, t.n, t.k, t.rowptr, t.colidx, r(t.val), t.colptr, t.rowidx, r(t.cval),
                   t.loss_kind, t.loss_param, t.loss_levels, t.rx, t.ry, t.X0, t.Yt0)


def _compare(G, o, t, prec, offset, rtol, power_iters=6):
    g = G.GLRM.from_table(t, precision=prec)
    sv = g.svd_init(power_iters=power_iters, offset=offset)
    X, Yt = (a.cpu().numpy().astype(np.float64) for a in g.factors())
    Xo, Yo, So = oracle_problem(o, _rounded(t, prec), offset=offset).svd_init(offset=offset)
    np.testing.assert_allclose(sv, So, rtol=rtol)
    Z, Zo = X @ Yt.T, Xo @ Yo.T
    assert np.linalg.norm(Z - Zo) <= rtol * np.linalg.norm(Zo)
    if offset:
        assert np.all(X[:, -1] == 1.0)
    return g


@pytest.mark.parametrize("prec,offset", [(0, False), (0, True), (1, True)])
def test_svd_init_completion_table(G, oracle_mod, prec, offset):
    """Noisy rank-5 quadratic table, 30% missing: a clear gap after the 5th
    singular value."""
    from gpu_parity import subset_table
    t = W.qpca_dense(m=400, n=150, k=5, seed=11, noise=0.05)
    keep = np.random.default_rng(11).random(t.nnz) < 0.7
    t = subset_table(t, keep)
    if offset:  # rank 5 plus the offset
        t = W.Table(t.name, t.m, t.n, 6, t.rowptr, t.colidx, t.val, t.colptr, t.rowidx, t.cval, t.loss_kind,
                    t.loss_param, t.loss_levels, t.rx, t.ry, np.zeros((t.m, 6)), np.zeros((t.n, 6)))
    _compare(G, oracle_mod, t, prec, offset, 1e-6 if prec == 0 else 2e-4)


def test_svd_init_mixed_table(G, oracle_mod):
    t = W.small_mixed(m=600, n=80, k=5, p_obs=0.6, seed=12, nkinds=7, rx=(RQ, 0.1), ry=(RQ, 0.1))
    _compare(G, oracle_mod, t, 0, True, 1e-5, power_iters=20)


def test_svd_init_reproduces_a_low_rank_table(G, oracle_mod):
    rng = np.random.default_rng(13)
    m, n, r = 300, 40, 3
    A = rng.normal(size=(m, r)) @ rng.normal(size=(r, n)) + rng.normal(size=n) * 4
    rowptr = np.arange(m + 1, dtype=np.int64) * n
    colidx = np.tile(np.arange(n, dtype=np.int32), m)
    colptr, rowidx, cval = W.csc_from_csr(m, n, rowptr, colidx, A.reshape(-1))
    t = W.Table("lowrank", m, n, r + 1, rowptr, colidx, A.reshape(-1), colptr, rowidx, cval,
                np.zeros(n, np.int32), np.ones(n), np.zeros(n, np.int32), (RQ, 0.1), (RQ, 0.1),
                np.zeros((m, r + 1)), np.zeros((n, r + 1)))
    g = G.GLRM.from_table(t, precision=G.GLRM_FP64)
    G.glrm_set_path(g.h, 1, 1)  # the sparse form: the initialisation reads the observed set
    g.svd_init(offset=True)
    X, Yt = (a.cpu().numpy() for a in g.factors())
    np.testing.assert_allclose(X @ Yt.T, A, rtol=0, atol=1e-6 * np.abs(A).max())


def test_svd_init_then_sweeps(G, oracle_mod):
    """The initial model is where the sweeps start: after it, synced sweeps
    follow the oracle as from any other start, and its objective after 10
    sweeps is below that of the random start."""
    from gpu_parity import synced_sweeps
    t = W.small_mixed(m=1000, n=120, k=6, p_obs=0.5, seed=14, nkinds=7, rx=(RQ, 0.1), ry=(RQ, 0.1))
    g0 = G.GLRM.from_table(t)
    f_rand = g0.sweep(10)[-1]
    g = G.GLRM.from_table(t)
    g.svd_init(offset=True)
    synced_sweeps(g, oracle_mod, t, 3, offset=True)
    f_svd = g.sweep(7)[-1]
    assert f_svd < f_rand


def test_svd_init_tall_table(G, oracle_mod):
    """8,000 x 30 with 60% observed: the Y-side products take the chunked form
    (columns of about 4,800 entries)."""
    from gpu_parity import subset_table
    t = W.qpca_dense(m=8000, n=30, k=4, seed=18, noise=0.05)
    t = subset_table(t, np.random.default_rng(18).random(t.nnz) < 0.6)
    _compare(G, oracle_mod, t, 0, False, 1e-6)
