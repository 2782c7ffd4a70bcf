"""Pins of the oracle's multi-dimensional losses (Sec. 6, eq. mpca): the
one-vs-all categorical loss and the multi-dimensional ordinal loss
(eq. ord-mpca) against hand values and against sums of the scalar hinge loss
over the block's columns (the separability the paper states for one-vs-all),
their gradients against central differences, the imputations against
brute force, the objective cell by cell, and the block sweep against the
scalar sweep: a table of scalar features only must give the plain model's
trajectory, and a categorical (ordinal) feature the trajectory of its d
(d - 1) Boolean hinge columns."""
import numpy as np
import pytest

from paper_1410_0342_gb300 import workloads as W

Q, HU, HI = 0, 1, 2
SC, CAT, ORD = 0, 1, 2
RZ, RQ, RL1, RNN = 0, 1, 2, 3


def test_categorical_loss_by_hand(oracle_mod):
    o = oracle_mod
    u = [2.0, -3.0, 0.5]
    # a = 1: (1 - 2)_+ + (1 - 3)_+ + (1 + 0.5)_+
    assert o.mloss(CAT, 3, u, 1) == pytest.approx(1.5)
    # a = 3: (1 + 2)_+ + (1 - 3)_+ + (1 - 0.5)_+
    assert o.mloss(CAT, 3, u, 3) == pytest.approx(3.5)
    np.testing.assert_array_equal(o.mgrad(CAT, 3, u, 3), [1.0, 0.0, -1.0])
    assert o.mdecode(CAT, 3, u) == 1.0


def test_ordinal_md_loss_by_hand(oracle_mod):
    o = oracle_mod
    u = [0.5, 0.2, -2.0]  # 4 levels, thresholds a' = 1, 2, 3
    # a = 2: a > 1 -> (1 - 0.5)_+; a <= 2, 3 -> (1 + 0.2)_+ + (1 - 2)_+
    assert o.mloss(ORD, 4, u, 2) == pytest.approx(1.7)
    # a = 4: every threshold passed: (1 - 0.5) + (1 - 0.2) + (1 + 2)
    assert o.mloss(ORD, 4, u, 4) == pytest.approx(4.3)
    np.testing.assert_array_equal(o.mgrad(ORD, 4, u, 2), [-1.0, 1.0, 0.0])
    # levels 1..4 cost 2.7, 1.7, 1.3, 4.3
    assert o.mdecode(ORD, 4, u) == 3.0
    assert o.feature_dim(ORD, 4) == 3 and o.feature_dim(CAT, 4) == 4 and o.feature_dim(SC, 0) == 1


@pytest.mark.parametrize("fkind,d", [(CAT, 2), (CAT, 5), (ORD, 2), (ORD, 6)])
def test_block_loss_is_a_sum_of_hinge_losses(oracle_mod, fkind, d):
    """One-vs-all: label a gives +1 to column a and -1 to the others; ordinal:
    threshold a' gets +1 when a > a', else -1.  The block loss is the sum of
    the scalar hinge (1 - b u)_+ over its columns, and so is its gradient."""
    o = oracle_mod
    rng = np.random.default_rng(d + 10 * fkind)
    w = o.feature_dim(fkind, d)
    for _ in range(40):
        u = rng.normal(scale=1.5, size=w)
        for a in range(1, d + 1):
            if fkind == CAT:
                b = np.where(np.arange(1, d + 1) == a, 1.0, -1.0)
            else:
                b = np.where(a > np.arange(1, d), 1.0, -1.0)
            want = sum(o.loss(HI, u[l], b[l]) for l in range(w))
            assert o.mloss(fkind, d, u, a) == pytest.approx(want, rel=1e-14, abs=1e-14)
            gw = [o.dloss(HI, u[l], b[l]) for l in range(w)]
            np.testing.assert_array_equal(o.mgrad(fkind, d, u, a), gw)


@pytest.mark.parametrize("fkind,d", [(CAT, 4), (ORD, 5)])
def test_block_gradient_central_differences(oracle_mod, fkind, d):
    o = oracle_mod
    rng = np.random.default_rng(7)
    w = o.feature_dim(fkind, d)
    h = 1e-6
    for _ in range(30):
        u = rng.normal(scale=2.0, size=w)
        if np.min(np.abs(np.abs(u) - 1.0)) < 1e-3:  # too close to a kink
            continue
        a = int(rng.integers(1, d + 1))
        g = o.mgrad(fkind, d, u, a)
        for l in range(w):
            e = np.zeros(w)
            e[l] = h
            fd = (o.mloss(fkind, d, u + e, a) - o.mloss(fkind, d, u - e, a)) / (2 * h)
            assert g[l] == pytest.approx(fd, abs=1e-6)


def test_decode_brute_force(oracle_mod):
    """Categorical: the first largest u_l.  Ordinal: no level has a smaller
    loss, and a level of equal loss is not smaller (ties to the lower level);
    strongly positive u passes every threshold, strongly negative none."""
    o = oracle_mod
    rng = np.random.default_rng(8)
    for _ in range(200):
        u = np.round(rng.normal(scale=1.5, size=5) * 4) / 4  # quarter steps: exact ties happen
        assert o.mdecode(CAT, 5, u) == float(np.argmax(u) + 1)
        a = int(o.mdecode(ORD, 6, u))
        costs = [o.mloss(ORD, 6, u, b) for b in range(1, 7)]
        assert costs[a - 1] == min(costs) and costs.index(min(costs)) == a - 1
    assert o.mdecode(ORD, 6, np.full(5, 3.0)) == 6.0
    assert o.mdecode(ORD, 6, np.full(5, -3.0)) == 1.0


def _fproblem(o, t, rx=None, ry=None):
    return o.FeatureProblem(t.m, t.nf, t.k, t.rows(), t.featidx, t.val, t.fkind, t.flevels, t.loss_kind,
                            t.loss_param, t.loss_levels, rx=rx or t.rx, ry=ry or t.ry)


def test_feature_objective_cell_by_cell(oracle_mod):
    o = oracle_mod
    t = W.features_mixed(m=40, n_real=3, n_bool=2, n_cat=3, n_ord=3, classes=4, levels=5, k=3, seed=31,
                         rx=(RL1, 0.2), ry=(RQ, 0.3))
    p = _fproblem(o, t)
    first = np.concatenate([[0], np.cumsum(t.widths())])
    rows = t.rows()
    X, Yt = t.X0, t.Yt0
    tot = 0.0
    for e in range(t.nnz):
        i, j, a = rows[e], t.featidx[e], t.val[e]
        u = X[i] @ Yt[first[j]:first[j + 1]].T
        if t.fkind[j] == SC:
            tot += o.loss(int(t.loss_kind[j]), float(u[0]), a, float(t.loss_param[j]), int(t.loss_levels[j]))
        else:
            tot += o.mloss(int(t.fkind[j]), int(t.flevels[j]), u, a)
    tot += 0.2 * np.abs(X).sum() + 0.3 * np.sum(Yt * Yt)
    assert p.objective(X, Yt) == pytest.approx(tot, rel=1e-12)


def test_scalar_features_follow_the_plain_sweep(oracle_mod):
    """Only scalar features: the block sweep is the plain sweep of Sec. 7.2."""
    o = oracle_mod
    t = W.small_mixed(m=60, n=25, k=4, seed=32, rx=(RL1, 0.1), ry=(RNN, 0.0), nkinds=7)
    p1 = o.Problem.from_csr(t.m, t.n, t.k, t.rowptr, t.colidx, t.val, loss_kind=t.loss_kind,
                            loss_param=t.loss_param, loss_levels=t.loss_levels, rx=t.rx, ry=t.ry)
    pf = o.FeatureProblem(t.m, t.n, t.k, t.rows(), t.colidx, t.val, SC, 0, t.loss_kind, t.loss_param,
                          t.loss_levels, rx=t.rx, ry=t.ry)
    for a, b in zip(pf.initial_alphas(), p1.initial_alphas()):
        np.testing.assert_array_equal(a, b)
    r1 = p1.proxgrad(t.X0, t.Yt0, 8)
    rf = pf.proxgrad(t.X0, t.Yt0, 8)
    for a, b in zip(rf[:5], r1[:5]):
        np.testing.assert_allclose(a, b, rtol=1e-12, atol=1e-12)
    np.testing.assert_array_equal(rf[5], r1[5])


def expand_to_hinge(t):
    """The table with every categorical / ordinal feature replaced by its
    block's Boolean columns (+-1 as in the separability above): (rowptr,
    colidx, val, loss kinds) of the expanded scalar table."""
    widths = t.widths()
    first = np.concatenate([[0], np.cumsum(widths)])
    rows = t.rows()
    R, C, V = [], [], []
    for e in range(t.nnz):
        i, j, a = rows[e], t.featidx[e], t.val[e]
        if t.fkind[j] == SC:
            R.append(i); C.append(first[j]); V.append(a)
            continue
        for l in range(widths[j]):
            lab = l + 1
            b = (1.0 if lab == a else -1.0) if t.fkind[j] == CAT else (1.0 if a > lab else -1.0)
            R.append(i); C.append(first[j] + l); V.append(b)
    D = int(first[-1])
    kinds = np.full(D, HI, np.int32)
    params = np.zeros(D)
    levs = np.zeros(D, np.int32)
    for j in range(t.nf):
        if t.fkind[j] == SC:
            kinds[first[j]] = t.loss_kind[j]
            params[first[j]] = t.loss_param[j]
            levs[first[j]] = t.loss_levels[j]
    return np.array(R), np.array(C), np.array(V), kinds, params, levs, D


def test_blocks_follow_their_boolean_columns(oracle_mod):
    """A categorical (ordinal) feature is fitted as its d (d - 1) Boolean
    hinge columns: same step sizes, same factors and objective sweep by
    sweep, same accept counts."""
    o = oracle_mod
    t = W.features_mixed(m=150, n_real=3, n_bool=2, n_cat=3, n_ord=3, classes=4, levels=5, k=4, seed=33,
                         rx=(RQ, 0.1), ry=(RQ, 0.1))
    pf = _fproblem(o, t)
    R, C, V, kinds, params, levs, D = expand_to_hinge(t)
    pe = o.Problem(t.m, D, t.k, R, C, V, kinds, params, levs, rx=t.rx, ry=t.ry)
    for a, b in zip(pf.initial_alphas(), pe.initial_alphas()):
        np.testing.assert_allclose(a, b, rtol=1e-15)
    rf = pf.proxgrad(t.X0, t.Yt0, 10)
    re = pe.proxgrad(t.X0, t.Yt0, 10)
    for a, b in zip(rf[:5], re[:5]):
        np.testing.assert_allclose(a, b, rtol=1e-11, atol=1e-11)
    np.testing.assert_array_equal(rf[5], re[5])


def test_feature_sweep_monotone(oracle_mod):
    o = oracle_mod
    t = W.features_mixed(m=300, k=5, seed=34, rx=(RL1, 0.05), ry=(RNN, 0.0))
    p = _fproblem(o, t)
    *_, hist, _ = p.proxgrad(t.X0, np.abs(t.Yt0), 25)
    assert np.all(np.diff(hist) <= 1e-12 * np.abs(hist[1:]))
