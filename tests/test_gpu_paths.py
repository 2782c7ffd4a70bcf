"""The kernel paths of a half-step (chunked, fused, blocked, masked tiles
with the whole other factor or panel by panel) against the FP64 oracle on the
same tables, and the automatic choice on shapes that select each of them."""
import numpy as np
import pytest
import torch

from paper_1410_0342_gb300 import workloads as W

from gpu_parity import subset_table, synced_sweeps

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
    G.glrm_set_path(g1.h, G.GLRM_PATH_MASKED, G.GLRM_PATH_MASKED_SPLIT)
    h1 = g1.sweep(8)
    g2 = G.GLRM.from_table(t)
    G.glrm_set_path(g2.h, 1, 1)
    h2a = g2.sweep(4)
    G.glrm_set_path(g2.h, 4, 5)
    h2b = g2.sweep(4)
    h2 = np.concatenate([h2a, h2b])
    assert (np.abs(h1 - h2) / np.abs(h1)).max() < 1e-5


def test_auto_path_choice(G):
    # 70% observed: stored densely, tensor-core form (FP32); FP64 stays sparse
    t = W.small_mixed(m=6000, n=64, k=16, p_obs=0.7, seed=3)
    g = G.GLRM.from_table(t)
    assert G.glrm_get_path(g.h) == (G.GLRM_PATH_DENSE, G.GLRM_PATH_DENSE)
    g64 = G.GLRM.from_table(t, precision=G.GLRM_FP64)
    assert G.glrm_get_path(g64.h) == (G.GLRM_PATH_MASKED, G.GLRM_PATH_MASKED_SPLIT)
    # 33% observed: masked tiles; Y^T fits whole, X only panel by panel
    t1 = W.small_mixed(m=6000, n=64, k=16, p_obs=0.33, seed=3)
    g1 = G.GLRM.from_table(t1)
    assert G.glrm_get_path(g1.h) == (G.GLRM_PATH_MASKED, G.GLRM_PATH_MASKED_SPLIT)
    # sparse with a large X: chunked Y-step
    t2 = W.small_mixed(m=60000, n=3000, k=8, p_obs=0.002, seed=4)
    g2 = G.GLRM.from_table(t2)
    assert G.glrm_get_path(g2.h) == (G.GLRM_PATH_FUSED, G.GLRM_PATH_CHUNKED)
    # k > 32 below the dense threshold: chunked only
    t3 = W.small_mixed(m=300, n=40, k=40, p_obs=0.3, seed=5)
    g3 = G.GLRM.from_table(t3)
    assert G.glrm_get_path(g3.h) == (G.GLRM_PATH_CHUNKED, G.GLRM_PATH_CHUNKED)
    with pytest.raises(G.GLRMError):
        G.glrm_set_path(g3.h, G.GLRM_PATH_FUSED, G.GLRM_PATH_AUTO)
    assert G.glrm_get_path(g3.h) == (G.GLRM_PATH_CHUNKED, G.GLRM_PATH_CHUNKED)


def test_sparse_chunked_matches_oracle(G, oracle_mod):
    t = W.small_mixed(m=20000, n=900, k=8, p_obs=0.004, seed=6)
    g = G.GLRM.from_table(t)
    synced_sweeps(g, oracle_mod, t, 6)


@pytest.mark.parametrize("paths", [(4, 4), (5, 5)])
def test_masked_tiles_of_a_tall_table(G, oracle_mod, paths):
    """Masked tiles whose other dimension takes more than 48 KB of bitmap to
    count (the Y-step's 400,003 rows: the pair counts of its tiles from a
    bitmap in opt-in shared memory), against the oracle."""
    t = W.completion(m=400_003, n=700, k=8, per_row=6)
    g = G.GLRM.from_table(t)
    G.glrm_set_path(g.h, *paths)
    # the Y-step's 22 tiles are too few for the GPU's warps: split either way
    assert tuple(G.glrm_get_path(g.h)) == (paths[0], G.GLRM_PATH_MASKED_SPLIT)
    synced_sweeps(g, oracle_mod, t, 3)


@pytest.mark.parametrize("p_obs,k", [(0.55, 12), (0.45, 33), (0.9, 5)])
def test_dense_path_with_missing_cells(G, oracle_mod, p_obs, k):
    """An observed set stored densely (NaN at the missing cells): synced
    sweeps against the oracle, including empty rows and columns."""
    t = W.small_mixed(m=1501, n=130, k=k, p_obs=p_obs, seed=300 + k)
    keep = ~np.isin(t.rows(), [0, 17, t.m - 1]) & (t.colidx != 5)
    t = subset_table(t, keep)
    g = G.GLRM.from_table(t)
    G.glrm_set_path(g.h, G.GLRM_PATH_DENSE, G.GLRM_PATH_DENSE)
    assert G.glrm_get_path(g.h) == (G.GLRM_PATH_DENSE, G.GLRM_PATH_DENSE)
    synced_sweeps(g, oracle_mod, t, 6)


def test_dense_path_switch_and_als(G, oracle_mod):
    """Switching between the dense and the sparse paths keeps the fit; ALS
    still runs on an observed set stored densely."""
    t = W.small_mixed(m=800, n=60, k=6, p_obs=0.6, seed=21, rx=(RQ, 0.1), ry=(RQ, 0.1))
    g = G.GLRM.from_table(t)
    assert G.glrm_get_path(g.h) == (G.GLRM_PATH_DENSE, G.GLRM_PATH_DENSE)
    synced_sweeps(g, oracle_mod, t, 2)
    G.glrm_set_path(g.h, G.GLRM_PATH_CHUNKED, G.GLRM_PATH_MASKED)
    synced_sweeps(g, oracle_mod, t, 2)
    G.glrm_set_path(g.h, G.GLRM_PATH_AUTO, G.GLRM_PATH_AUTO)
    assert G.glrm_get_path(g.h) == (G.GLRM_PATH_DENSE, G.GLRM_PATH_DENSE)
    synced_sweeps(g, oracle_mod, t, 2)
    q = W.qpca_dense(m=300, n=90, k=4, seed=22)
    gq = G.GLRM.from_table(q)
    assert G.glrm_get_path(gq.h) == (G.GLRM_PATH_DENSE, G.GLRM_PATH_DENSE)
    X0, Y0 = gq.factors()
    hist = gq.als_sweep(30)
    p = oracle_mod.Problem.from_csr(q.m, q.n, q.k, q.rowptr, q.colidx, q.val, loss_kind=q.loss_kind,
                                    loss_param=q.loss_param, loss_levels=q.loss_levels, rx=q.rx, ry=q.ry)
    *_, ohist = p.als(X0.double().cpu().numpy(), Y0.double().cpu().numpy(), 0.1, 30)
    assert (np.abs(hist - ohist) / ohist).max() < 1e-4
    with pytest.raises(G.GLRMError):
        G.glrm_set_path(gq.h, G.GLRM_PATH_DENSE, G.GLRM_PATH_CHUNKED)


@pytest.mark.parametrize("m,nsweeps", [(20000, 5), (100000, 2)])
def test_benchmark_table_dense_path_matches_oracle(G, oracle_mod, m, nsweeps):
    """The benchmark's own table recipe (W.mixed: 60% observed, contiguous
    blocks of 500 Huber, 300 hinge and 200 ordinal columns, l1 on X,
    nonnegativity on Y, k = 20) on the path the benchmark times: stored
    densely with NaN at the missing cells, 16-column loss groups of one kind,
    cost-planned work items split across the tile's chunks.  At m = 100,000
    this is the exact launch configuration of the benchmark; synced sweeps
    against the oracle, objectives within 1e-5, factors and steps compared."""
    t = W.mixed(m=m)
    g = G.GLRM.from_table(t)
    assert G.glrm_get_path(g.h) == (G.GLRM_PATH_DENSE, G.GLRM_PATH_DENSE)
    rels = synced_sweeps(g, oracle_mod, t, nsweeps)
    assert rels.max() < 1e-5


@pytest.mark.parametrize("paths", [(1, 1), (2, 2), (3, 3), (4, 4), (4, 5), (6, 6)])
def test_l1_and_quantile_losses_on_every_path(G, oracle_mod, paths):
    """Columns cycling through all seven loss kinds (quadratic, Huber, hinge,
    logistic, ordinal hinge, l1, quantile with alpha = 0.3) on every kernel
    path, the dense form included: synced sweeps against the oracle."""
    t = W.small_mixed(m=1303, n=140, k=12, p_obs=0.5, seed=407, nkinds=7)
    g = G.GLRM.from_table(t)
    G.glrm_set_path(g.h, *paths)
    synced_sweeps(g, oracle_mod, t, 6)
