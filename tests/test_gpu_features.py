"""Tables of multi-dimensional features (Sec. 6, eq. mpca) on the GPU: the
embedding of categorical and ordinal features into their blocks' Boolean
columns against the tests' own expansion (bit-exact), sweeps of the embedded
model against the oracle's block model (eq. mpca written with the block
losses, not with the embedding) on several kernel paths, and the imputation
of labels against the oracle (exact on dyadic factors, where every product
is exact; elsewhere up to near-ties)."""
import numpy as np
import pytest
import torch

from paper_1410_0342_gb300 import workloads as W

from gpu_parity import synced_sweeps
from test_oracle_features import expand_to_hinge

pytestmark = pytest.mark.gpu

SC, CAT, ORD = 0, 1, 2
RZ, RQ, RL1, RNN = 0, 1, 2, 3


@pytest.fixture(scope="module")
def G():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1410_0342_gb300 import build
    build.build()
    from paper_1410_0342_gb300 import glrm
    return glrm


def fproblem(o, t):
    return o.FeatureProblem(t.m, t.nf, t.k, t.rows(), t.featidx, t.val, t.fkind, t.flevels, t.loss_kind,
                            t.loss_param, t.loss_levels, rx=t.rx, ry=t.ry)


def embed(G, t, precision):
    dt = G.dtype_of(precision)
    i32 = torch.int32
    src = [torch.as_tensor(np.asarray(a), dtype=ty, device="cuda") for a, ty in
           ((t.rowptr, i32), (t.featidx, i32), (t.val, dt), (t.colptr, i32), (t.rowidx, i32), (t.cval, dt))]
    D, ennz = G.glrm_embed_size(t.fkind, t.flevels, src[3])
    out = [torch.full((t.m + 1,), -7, dtype=i32, device="cuda"), torch.full((ennz,), -7, dtype=i32, device="cuda"),
           torch.full((ennz,), 7.0, dtype=dt, device="cuda"), torch.full((D + 1,), -7, dtype=i32, device="cuda"),
           torch.full((ennz,), -7, dtype=i32, device="cuda"), torch.full((ennz,), 7.0, dtype=dt, device="cuda")]
    G.glrm_embed_features(t.fkind, t.flevels, t.m, t.nnz, *src, precision, *out)
    return D, ennz, [a.cpu().numpy() for a in out]


@pytest.mark.parametrize("prec", [1, 0])
def test_embedding_is_the_expansion(G, prec):
    t = W.features_mixed(m=700, n_real=3, n_bool=2, n_cat=4, n_ord=4, classes=5, levels=6, k=4, seed=41)
    D, ennz, (rp, ci, v, cp, ri, cv) = embed(G, t, prec)
    R, C, V, kinds, params, levs, D0 = expand_to_hinge(t)
    assert D == D0 and ennz == R.size
    rowptr = np.concatenate([[0], np.cumsum(np.bincount(R, minlength=t.m))])
    np.testing.assert_array_equal(rp, rowptr)
    np.testing.assert_array_equal(ci, C)
    vt = np.float64 if prec == 0 else np.float32
    np.testing.assert_array_equal(v, V.astype(vt))
    colptr, rowidx, cval = W.csc_from_csr(t.m, D, rowptr, C, V)
    np.testing.assert_array_equal(cp, colptr)
    np.testing.assert_array_equal(ri, rowidx)
    np.testing.assert_array_equal(cv, np.asarray(cval).astype(vt))
    k2, p2, l2 = G.glrm_embed_losses(t.fkind, t.flevels, (t.loss_kind, t.loss_param, t.loss_levels))
    np.testing.assert_array_equal(k2, kinds)
    np.testing.assert_array_equal(p2, params)
    np.testing.assert_array_equal(l2, levs)


@pytest.mark.parametrize("paths", [(1, 1), (2, 2), (4, 4), (5, 5), (6, 6)])
def test_feature_sweeps_match_block_oracle_fp32(G, oracle_mod, paths):
    t = W.features_mixed(m=1500, n_real=4, n_bool=3, n_cat=4, n_ord=4, classes=5, levels=6, k=8, seed=42,
                         rx=(RL1, 0.05), ry=(RQ, 0.1))
    g = G.GLRM.from_feature_table(t)
    G.glrm_set_path(g.h, *paths)
    synced_sweeps(g, oracle_mod, None, 6, problem=fproblem(oracle_mod, t))


def test_feature_sweeps_fp64_free_running(G, oracle_mod):
    t = W.features_mixed(m=600, n_real=3, n_bool=2, n_cat=3, n_ord=3, classes=4, levels=5, k=5, seed=43,
                         rx=(RQ, 0.1), ry=(RQ, 0.1))
    g = G.GLRM.from_feature_table(t, precision=G.GLRM_FP64)
    hist = g.sweep(15)
    acc = g.accepts()
    *_, oh, oacc = fproblem(oracle_mod, t).proxgrad(t.X0, t.Yt0, 15)
    np.testing.assert_allclose(hist, oh, rtol=1e-9)
    assert tuple(acc) == tuple(oacc[-1])


def test_census_like_table_auto_path(G, oracle_mod):
    """Contiguous groups of features (real, Boolean, categorical, ordinal)
    at 20,000 rows; the automatic path choice."""
    t = W.features_mixed(m=20000, n_real=10, n_bool=8, n_cat=8, n_ord=6, classes=6, levels=7, k=10, seed=44,
                         cyclic=False, rx=(RL1, 0.02), ry=(RQ, 0.05))
    g = G.GLRM.from_feature_table(t)
    synced_sweeps(g, oracle_mod, None, 3, problem=fproblem(oracle_mod, t))


def _all_pairs(t):
    rows = np.repeat(np.arange(t.m), t.nf).astype(np.int32)
    feats = np.tile(np.arange(t.nf), t.m).astype(np.int32)
    return rows, feats


def _oracle_decode(o, t, X, Yt, rows, feats):
    first = np.concatenate([[0], np.cumsum(t.widths())])
    out = np.empty(rows.size)
    for r, (i, j) in enumerate(zip(rows, feats)):
        u = np.asarray(X[i], np.float64) @ np.asarray(Yt[first[j]:first[j + 1]], np.float64).T
        if t.fkind[j] == SC:
            out[r] = o.decode(int(t.loss_kind[j]), float(u[0]), int(t.loss_levels[j]))
        else:
            out[r] = o.mdecode(int(t.fkind[j]), int(t.flevels[j]), u)
    return out


@pytest.mark.parametrize("prec", [1, 0])
def test_decode_exact_on_dyadic_factors(G, oracle_mod, prec):
    """Factor entries in {-1, -1/2, 0, 1/2, 1}: every product and every sum of
    the ordinal rule is exact in FP32 and FP64 alike, equal maxima and minima
    are common, and the labels must agree exactly, ties included."""
    t = W.features_mixed(m=300, n_real=2, n_bool=2, n_cat=4, n_ord=4, classes=5, levels=6, k=4, seed=45)
    g = G.GLRM.from_feature_table(t, precision=prec)
    rng = np.random.default_rng(45)
    X = rng.integers(-2, 3, size=(t.m, t.k)) / 2.0
    Yt = rng.integers(-2, 3, size=(g.n, t.k)) / 2.0
    g.set_factors(torch.as_tensor(X, dtype=g.dtype, device="cuda"), torch.as_tensor(Yt, dtype=g.dtype, device="cuda"))
    rows, feats = _all_pairs(t)
    got = g.decode_features(torch.as_tensor(rows, device="cuda"), torch.as_tensor(feats, device="cuda")).cpu().numpy()
    want = _oracle_decode(oracle_mod, t, X, Yt, rows, feats)
    np.testing.assert_array_equal(got.astype(np.float64), want)
    blocks = t.fkind[feats] != SC
    assert len(np.unique(want[blocks])) > 3


def test_decode_after_fit(G, oracle_mod):
    """After 20 sweeps: the labels of every (row, feature) pair agree with the
    oracle's decoding of the same factors (products in FP64 there, FP32 here)
    on all but 0.1% of the block features' pairs (near-ties), real features
    to FP32 rounding."""
    t = W.features_mixed(m=800, n_real=2, n_bool=2, n_cat=4, n_ord=4, classes=5, levels=6, k=6, seed=46)
    g = G.GLRM.from_feature_table(t)
    g.sweep(20)
    X, Yt = (a.cpu().numpy().astype(np.float64) for a in g.factors())
    rows, feats = _all_pairs(t)
    got = g.decode_features(torch.as_tensor(rows, device="cuda"), torch.as_tensor(feats, device="cuda")).cpu().numpy()
    want = _oracle_decode(oracle_mod, t, X, Yt, rows, feats)
    blocks = t.fkind[feats] != SC
    bad = blocks & (got != want)
    assert bad.sum() <= max(2, int(1e-3 * blocks.sum())), bad.sum()
    # real features decode to u itself: FP32 rounding of the product
    real = (t.fkind[feats] == SC) & (t.loss_kind[feats] == W.LOSS_HUBER)
    np.testing.assert_allclose(got[real], want[real], rtol=1e-5, atol=1e-5)


def test_embed_rejects_bad_labels(G):
    t = W.features_mixed(m=100, n_real=1, n_bool=1, n_cat=1, n_ord=1, classes=4, levels=5, k=3, seed=47)
    j = int(np.nonzero(t.fkind == CAT)[0][0])
    for bad in (0.0, 5.0, 2.5):
        val = t.val.copy()
        cval = t.cval.copy()
        e = int(np.nonzero(t.featidx == j)[0][0])
        val[e] = bad
        r = t.rows()[e]
        q = t.colptr[j] + int(np.nonzero(t.rowidx[t.colptr[j]:t.colptr[j + 1]] == r)[0][0])
        cval[q] = bad
        t2 = W.FeatureTable(t.name, t.m, t.nf, t.k, t.rowptr, t.featidx, val, t.colptr, t.rowidx, cval, t.fkind,
                            t.flevels, t.loss_kind, t.loss_param, t.loss_levels, t.rx, t.ry, t.X0, t.Yt0)
        with pytest.raises(G.GLRMError) as ei:
            embed(G, t2, 1)
        assert ei.value.code == G.GLRM_ERR_OMEGA
    fi = t.featidx.copy()
    fi[0] = t.nf
    t3 = W.FeatureTable(t.name, t.m, t.nf, t.k, t.rowptr, fi, t.val, t.colptr, t.rowidx, t.cval, t.fkind,
                        t.flevels, t.loss_kind, t.loss_param, t.loss_levels, t.rx, t.ry, t.X0, t.Yt0)
    with pytest.raises(G.GLRMError):
        embed(G, t3, 1)
    # bad descriptors
    with pytest.raises(G.GLRMError):
        G.glrm_embed_losses([CAT], [1], ([0], [0.0], [0]))
