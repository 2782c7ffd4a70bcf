"""Failure handling without a GPU fault: a device-side wait that runs out
returns GLRM_ERR_TIMEOUT and leaves the context usable; an ALS system that is
not numerically positive definite is reported, not turned into NaN factors;
FP64 ALS pivots far outside the float range still factorise exactly."""
import numpy as np
import pytest
import torch

from paper_1410_0342_gb300 import workloads as W

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def G():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1410_0342_gb300 import build
    build.build()
    from paper_1410_0342_gb300 import glrm
    return glrm


def test_wait_limit_expires_and_context_survives(G, oracle_mod):
    # an armed barrier completes within the limit
    G.glrm_wait_selftest(1000, arm=True)
    # a barrier nothing arrives on: the bounded wait runs out after 200 attempts
    for _ in range(2):
        with pytest.raises(G.GLRMError) as e:
            G.glrm_wait_selftest(200, arm=False)
        assert e.value.code == G.GLRM_ERR_TIMEOUT
    # the context is usable afterwards: a sweep still matches the oracle
    t = W.small_mixed(m=300, n=50, k=8, seed=5)
    g = G.GLRM.from_table(t)
    h = g.sweep(2)
    p = oracle_mod.Problem.from_csr(t.m, t.n, t.k, t.rowptr, t.colidx, t.val, loss_kind=t.loss_kind,
                                    loss_param=t.loss_param, loss_levels=t.loss_levels, rx=t.rx,
                                    ry=t.ry)
    *_, oh, _ = p.proxgrad(t.X0, t.Yt0, 2)
    assert np.isfinite(h).all() and abs(h[0] - oh[0]) / abs(oh[0]) < 1e-5
    G.glrm_wait_selftest(1000, arm=True)


def test_als_pivot_failure_is_reported(G, oracle_mod):
    """FP32 Gram matrices of factors equal to 1e20 overflow to Inf: every pivot
    is infinite, the sweep returns GLRM_ERR_NONFINITE and the factors are kept;
    after new factors the same handle fits normally."""
    t = W.batch_instance(0, m_range=(200, 200), n_range=(60, 60), ks=(8,))
    g = G.GLRM.from_table(t)
    # both factors huge: the X-step's Gram (of Y) and the Y-step's (of X) overflow
    g.set_factors(torch.full((t.m, t.k), 1e20, dtype=torch.float32, device="cuda"),
                  torch.full((t.n, t.k), 1e20, dtype=torch.float32, device="cuda"))
    X0, Y0 = g.factors()
    with pytest.raises(G.GLRMError) as e:
        g.als_sweep(1)
    assert e.value.code == G.GLRM_ERR_NONFINITE
    X1, Y1 = g.factors()
    assert torch.equal(X0, X1) and torch.equal(Y0, Y1)
    g.set_factors(torch.as_tensor(t.X0, dtype=torch.float32, device="cuda"),
                  torch.as_tensor(t.Yt0, dtype=torch.float32, device="cuda"))
    h = g.als_sweep(5)
    p = oracle_mod.Problem.from_csr(t.m, t.n, t.k, t.rowptr, t.colidx, t.val, loss_kind=t.loss_kind,
                                    loss_param=t.loss_param, loss_levels=t.loss_levels, rx=t.rx,
                                    ry=t.ry)
    *_, oh = p.als(t.X0, t.Yt0, 0.1, 5)
    assert (np.abs(h - oh) / oh).max() < 1e-4


def test_als_fp64_pivots_beyond_float_range(G, oracle_mod):
    """FP64 model, data scaled by 1e40 and factors by 1e20: Gram pivots near
    1e42 are beyond the float range of the reciprocal square root's seed, yet
    the factorisation (exponent-scaled seed, Newton refinement) matches the
    oracle's sqrt-based Cholesky to 1e-9."""
    t = W.qpca_dense(m=120, n=70, k=4, seed=17)
    s = 1e40
    t2 = W.Table(t.name, t.m, t.n, t.k, t.rowptr, t.colidx, t.val * s, t.colptr, t.rowidx,
                 t.cval * s, t.loss_kind, t.loss_param, t.loss_levels, t.rx, t.ry, t.X0 * 1e20,
                 t.Yt0 * 1e20)
    g = G.GLRM.from_table(t2, precision=G.GLRM_FP64)
    h = g.als_sweep(6)
    p = oracle_mod.Problem.from_csr(t2.m, t2.n, t2.k, t2.rowptr, t2.colidx, t2.val,
                                    loss_kind=t2.loss_kind, loss_param=t2.loss_param,
                                    loss_levels=t2.loss_levels, rx=t2.rx, ry=t2.ry)
    *_, oh = p.als(t2.X0, t2.Yt0, 0.1, 6)
    assert np.isfinite(h).all()
    assert (np.abs(h - oh) / oh).max() < 1e-9
