"""The kernel paths of a half-step (chunked, fused, blocked, masked tiles
with the whole other factor or panel by panel) against the FP64 oracle on the
same tables, and the automatic choice on shapes that select each of them."""
import numpy as np
import pytest
import torch

from paper_1410_0342_gb300 import workloads as W

from gpu_parity import synced_sweeps

pytestmark = pytest.mark.gpu

RZ, RQ, RL1, RNN = 0, 1, 2, 3


@pytest.fixture(scope="module")
def G():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1410_0342_gb300 import build
    build.build()
    from paper_1410_0342_gb300 import glrm
    return glrm


def oracle_hist(o, t, nsweeps):
    p = o.Problem.from_csr(t.m, t.n, t.k, t.rowptr, t.colidx, t.val, loss_kind=t.loss_kind,
                           loss_param=t.loss_param, loss_levels=t.loss_levels, rx=t.rx, ry=t.ry)
    return p.proxgrad(t.X0, t.Yt0, nsweeps)


PATHS = [(1, 1), (2, 2), (3, 3), (2, 3), (3, 1), (1, 2), (4, 4), (5, 5), (4, 1), (1, 5), (5, 4)]


@pytest.mark.parametrize("paths", PATHS)
@pytest.mark.parametrize("k", [4, 7, 20, 32])
def test_paths_match_oracle_fp32(G, oracle_mod, paths, k):
    t = W.small_mixed(m=1303, n=150, k=k, p_obs=0.5, seed=200 + k)
    g = G.GLRM.from_table(t)
    G.glrm_set_path(g.h, *paths)
    got = G.glrm_get_path(g.h)
    for want, have in zip(paths, got):
        # a masked request runs panel by panel when the factor does not fit whole
        assert have == want or (want == G.GLRM_PATH_MASKED and have == G.GLRM_PATH_MASKED_SPLIT)
    synced_sweeps(g, oracle_mod, t, 8)


@pytest.mark.parametrize("paths", [(1, 1), (2, 2), (3, 3), (4, 4), (5, 5)])
def test_paths_match_oracle_fp64(G, oracle_mod, paths):
    t = W.qpca_dense(m=300, n=140, k=6, seed=5)
    g = G.GLRM.from_table(t, precision=G.GLRM_FP64)
    G.glrm_set_path(g.h, *paths)
    hist = g.sweep(40)
    acc = g.accepts()
    X, Yt, ax, ay, ohist, oacc = oracle_hist(oracle_mod, t, 40)
    assert (np.abs(hist - ohist) / np.abs(ohist)).max() < 1e-9
    assert tuple(acc) == tuple(oacc[-1])


def test_path_switch_keeps_state(G):
    """Switching paths mid-fit continues the same fit (same factors and steps)."""
    t = W.small_mixed(m=900, n=80, k=12, seed=9)
    g1 = G.GLRM.from_table(t)
    h1 = g1.sweep(8)
    g2 = G.GLRM.from_table(t)
    G.glrm_set_path(g2.h, 1, 1)
    h2a = g2.sweep(4)
    G.glrm_set_path(g2.h, 4, 5)
    h2b = g2.sweep(4)
    h2 = np.concatenate([h2a, h2b])
    assert (np.abs(h1 - h2) / np.abs(h1)).max() < 1e-5


def test_auto_path_choice(G):
    # dense: masked tiles; Y^T fits whole, X only panel by panel
    t = W.small_mixed(m=6000, n=64, k=16, p_obs=0.7, seed=3)
    g = G.GLRM.from_table(t)
    assert G.glrm_get_path(g.h) == (G.GLRM_PATH_MASKED, G.GLRM_PATH_MASKED_SPLIT)
    # sparse with a large X: chunked Y-step
    t2 = W.small_mixed(m=60000, n=3000, k=8, p_obs=0.002, seed=4)
    g2 = G.GLRM.from_table(t2)
    assert G.glrm_get_path(g2.h) == (G.GLRM_PATH_FUSED, G.GLRM_PATH_CHUNKED)
    # k > 32: chunked only
    t3 = W.small_mixed(m=300, n=40, k=40, seed=5)
    g3 = G.GLRM.from_table(t3)
    assert G.glrm_get_path(g3.h) == (G.GLRM_PATH_CHUNKED, G.GLRM_PATH_CHUNKED)
    with pytest.raises(G.GLRMError):
        G.glrm_set_path(g3.h, G.GLRM_PATH_FUSED, G.GLRM_PATH_AUTO)
    assert G.glrm_get_path(g3.h) == (G.GLRM_PATH_CHUNKED, G.GLRM_PATH_CHUNKED)


def test_sparse_chunked_matches_oracle(G, oracle_mod):
    t = W.small_mixed(m=20000, n=900, k=8, p_obs=0.004, seed=6)
    g = G.GLRM.from_table(t)
    synced_sweeps(g, oracle_mod, t, 6)
