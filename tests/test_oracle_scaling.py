"""Pins of the oracle's offsets and scaling (Sec. 3.4 and Sec. 4.3, "Offsets
and scaling"): the column statistics against their closed forms (mean and
sample variance, median, quantile, the logistic log-odds, the hinge's
two-label minimum) and brute force over candidate points; the offset model's
objective summed by hand and its trivial case (k = 1: the offset converges to
the column mean); the weighted losses against a hand sum and an invariance of
the whole sweep (weights c with regulariser weights c and steps alpha / c give
the unweighted trajectory with c times its objective).

The oracle finds mu_j by golden-section search on S_j's values, which places
a smooth minimiser only to about the square root of the rounding unit times
the column's scale (near the minimum S changes quadratically); S_j(mu_j), and
so sigma2_j, is accurate to rounding.  MU_TOL is that resolution."""
import numpy as np
import pytest

from paper_1410_0342_gb300 import workloads as W

Q, HU, HI, LO, OR, L1, QT = 0, 1, 2, 3, 4, 5, 6
RZ, RQ, RL1, RNN = 0, 1, 2, 3
MU_TOL = 1e-6


def _columns(o, cols_vals, kind, param=1.0, levels=0):
    """A problem whose column j holds the values cols_vals[j] (one row per value)."""
    m = max(len(v) for v in cols_vals)
    rows, cols, vals = [], [], []
    for j, v in enumerate(cols_vals):
        for i, a in enumerate(v):
            rows.append(i)
            cols.append(j)
            vals.append(a)
    order = np.lexsort((np.array(cols), np.array(rows)))
    return o.Problem(m, len(cols_vals), 1, np.array(rows)[order], np.array(cols)[order],
                     np.array(vals, dtype=np.float64)[order], kind, param, levels)


def test_column_stats_quadratic_mean_and_variance(oracle_mod):
    o = oracle_mod
    rng = np.random.default_rng(1)
    cols = [rng.normal(3.0, 2.0, size=c) for c in (2, 5, 17, 40)]
    mu, s2 = _columns(o, cols, Q).column_stats()
    for j, v in enumerate(cols):
        assert mu[j] == pytest.approx(np.mean(v), abs=MU_TOL)
        assert s2[j] == pytest.approx(np.var(v, ddof=1), rel=1e-10)


def test_column_stats_l1_median(oracle_mod):
    o = oracle_mod
    rng = np.random.default_rng(2)
    cols = [rng.normal(size=c) for c in (1, 3, 9, 31)]  # odd counts: the median is unique
    mu, s2 = _columns(o, cols, L1).column_stats()
    for j, v in enumerate(cols):
        assert mu[j] == pytest.approx(np.median(v), abs=1e-11)
        if len(v) > 1:
            assert s2[j] == pytest.approx(np.sum(np.abs(v - np.median(v))) / (len(v) - 1), rel=1e-10)
        else:
            assert np.isnan(s2[j])


@pytest.mark.parametrize("alpha", [0.1, 0.3, 0.77])
def test_column_stats_quantile(oracle_mod, alpha):
    """The pinball sum is piecewise linear and convex, so its minimum is taken
    at a data point: brute force over the data points gives min S, and
    mu lies between the lower and upper alpha-quantiles of the column."""
    o = oracle_mod
    rng = np.random.default_rng(3)
    cols = [rng.normal(size=c) for c in (7, 20, 33)]
    mu, s2 = _columns(o, cols, QT, param=alpha).column_stats()
    for j, v in enumerate(cols):
        S = lambda x: float(np.sum(np.where(v > x, alpha * (v - x), (1 - alpha) * (x - v))))
        best = min(S(a) for a in v)
        assert S(mu[j]) == pytest.approx(best, rel=1e-10, abs=1e-12)
        assert s2[j] == pytest.approx(best / (len(v) - 1), rel=1e-10, abs=1e-12)
        srt = np.sort(v)
        c = len(v)
        # S'(x+) = #{a <= x} - alpha c >= 0 and S'(x-) = #{a < x} - alpha c <= 0
        lo_q = srt[int(np.ceil(alpha * c)) - 1]
        hi_q = srt[min(int(np.floor(alpha * c)), c - 1)]
        assert lo_q - 1e-9 <= mu[j] <= hi_q + 1e-9


def test_column_stats_logistic_log_odds(oracle_mod):
    """sum log(1 + exp(-a mu)) over p c labels +1 and (1-p) c labels -1 is
    minimised at mu = log(p / (1 - p))."""
    o = oracle_mod
    cols = [[1.0] * 3 + [-1.0] * 7, [1.0] * 12 + [-1.0] * 4, [1.0, -1.0]]
    mu, s2 = _columns(o, cols, LO).column_stats()
    for j, v in enumerate(cols):
        p = np.mean(np.array(v) > 0)
        assert mu[j] == pytest.approx(np.log(p / (1 - p)), abs=MU_TOL)
        Smin = len(v) * (-(p * np.log(p) + (1 - p) * np.log(1 - p)))  # the label entropy
        assert s2[j] == pytest.approx(Smin / (len(v) - 1), rel=1e-10)


def test_column_stats_hinge_two_labels(oracle_mod):
    """n+ labels +1, n- labels -1: S(mu) = n+ (1 - mu)_+ + n- (1 + mu)_+ has
    its minimum 2 min(n+, n-) at mu = 1 when n+ > n- (at -1 when n- > n+)."""
    o = oracle_mod
    cols = [[1.0] * 5 + [-1.0] * 2, [1.0] * 1 + [-1.0] * 4]
    mu, s2 = _columns(o, cols, HI).column_stats()
    assert mu[0] == pytest.approx(1.0, abs=1e-9)
    assert mu[1] == pytest.approx(-1.0, abs=1e-9)
    assert s2[0] == pytest.approx(2 * 2 / 6, rel=1e-9)
    assert s2[1] == pytest.approx(2 * 1 / 4, rel=1e-9)


@pytest.mark.parametrize("kind,param,levels,gen", [
    (HU, 0.7, 0, lambda r, c: r.standard_t(2, size=c)),
    (OR, 1.0, 5, lambda r, c: r.integers(1, 6, size=c).astype(float)),
])
def test_column_stats_brute_force_grid(oracle_mod, kind, param, levels, gen):
    """Huber and ordinal columns: S(mu) is not above the minimum of S over a
    fine grid of the column's range (Huber: also the first-order condition)."""
    o = oracle_mod
    rng = np.random.default_rng(4)
    cols = [gen(rng, c) for c in (6, 25)]
    mu, s2 = _columns(o, cols, kind, param, levels).column_stats()
    for j, v in enumerate(cols):
        S = lambda x: sum(o.loss(kind, x, a, param, levels) for a in v)
        grid = np.linspace(v.min() - 1, v.max() + 1, 4001)
        best = min(S(x) for x in grid)
        assert S(mu[j]) <= best + 1e-9 * max(1.0, abs(best))
        assert s2[j] == pytest.approx(S(mu[j]) / (len(v) - 1), rel=1e-12)
        if kind == HU:
            d = np.clip(mu[j] - v, -param, param).sum()
            assert abs(d) < MU_TOL * len(v)


def test_column_stats_empty_and_single(oracle_mod):
    o = oracle_mod
    p = o.Problem(3, 3, 1, np.array([0, 1, 2]), np.array([0, 0, 2]), np.array([1.0, 2.0, 5.0]), Q, 1.0, 0)
    mu, s2 = p.column_stats()
    assert mu[0] == pytest.approx(1.5) and s2[0] == pytest.approx(0.5)
    assert np.isnan(mu[1]) and np.isnan(s2[1])
    assert mu[2] == pytest.approx(5.0) and np.isnan(s2[2])


def _offset_problem(o, t, offset=True, col_scale=None, rx=None, ry=None):
    return o.Problem.from_csr(t.m, t.n, t.k, t.rowptr, t.colidx, t.val, loss_kind=t.loss_kind,
                              loss_param=t.loss_param, loss_levels=t.loss_levels,
                              rx=rx or t.rx, ry=ry or t.ry, offset=offset, col_scale=col_scale)


def test_offset_objective_by_hand(oracle_mod):
    """With the offset the last coordinate of X enters through the indicator
    of x_ik = 1 and the last of Y is not regularised."""
    o = oracle_mod
    t = W.small_mixed(m=12, n=9, k=4, seed=8, rx=(RQ, 0.25), ry=(RL1, 0.5), nkinds=7)
    p = _offset_problem(o, t)
    X = t.X0.copy()
    X[:, -1] = 1.0
    Yt = t.Yt0
    rows = t.rows()
    tot = 0.0
    for e in range(t.nnz):
        i, j = rows[e], t.colidx[e]
        tot += o.loss(int(t.loss_kind[j]), float(X[i] @ Yt[j]), t.val[e], float(t.loss_param[j]),
                      int(t.loss_levels[j]))
    tot += 0.25 * np.sum(X[:, :-1] ** 2) + 0.5 * np.abs(Yt[:, :-1]).sum()
    assert p.objective(X, Yt) == pytest.approx(tot, rel=1e-12)
    X[3, -1] = 0.5
    assert p.objective(X, Yt) == np.inf


def test_offset_k1_converges_to_column_mean(oracle_mod):
    """k = 1 with the offset: x_i = 1 after the first X-step and y_j is an
    unregularised scalar fitted to column j under quadratic loss, i.e. the
    column mean (the trivial case of the k+1 construction)."""
    o = oracle_mod
    rng = np.random.default_rng(9)
    t = W.small_mixed(m=30, n=8, k=1, seed=9, rx=(RQ, 0.3), ry=(RQ, 0.3))
    vals = rng.normal(2.0, 1.5, size=t.nnz)
    p = o.Problem.from_csr(t.m, t.n, 1, t.rowptr, t.colidx, vals, loss_kind=Q, loss_param=1.0,
                           loss_levels=0, rx=(RQ, 0.3), ry=(RQ, 0.3), offset=True)
    X0 = rng.normal(size=(t.m, 1))
    Yt0 = np.zeros((t.n, 1))
    X, Yt, *_ = p.proxgrad(X0, Yt0, 200)
    assert np.all(X == 1.0)
    cols = p.cols
    for j in range(t.n):
        # the accept test compares objective values, which resolve y_j only
        # to about the square root of the rounding unit
        assert Yt[j, 0] == pytest.approx(vals[cols == j].mean(), abs=MU_TOL)


def test_weighted_objective_and_gradient_by_hand(oracle_mod):
    o = oracle_mod
    t = W.small_mixed(m=11, n=10, k=3, seed=12, rx=(RQ, 0.2), ry=(RQ, 0.1), nkinds=7)
    w = np.random.default_rng(12).uniform(0.2, 3.0, size=t.n)
    p = _offset_problem(o, t, offset=False, col_scale=w)
    p1 = _offset_problem(o, t, offset=False)
    X, Yt = t.X0, t.Yt0
    rows = t.rows()
    tot = 0.0
    GX = np.zeros_like(X)
    GYt = np.zeros_like(Yt)
    for e in range(t.nnz):
        i, j, a = rows[e], t.colidx[e], t.val[e]
        u = float(X[i] @ Yt[j])
        kd, pr, lv = int(t.loss_kind[j]), float(t.loss_param[j]), int(t.loss_levels[j])
        tot += w[j] * o.loss(kd, u, a, pr, lv)
        d = w[j] * o.dloss(kd, u, a, pr, lv)
        GX[i] += d * Yt[j]
        GYt[j] += d * X[i]
    tot += 0.2 * np.sum(X * X) + 0.1 * np.sum(Yt * Yt)
    assert p.objective(X, Yt) == pytest.approx(tot, rel=1e-12)
    gx, gy = p.gradient(X, Yt)
    np.testing.assert_allclose(gx, GX, rtol=1e-12, atol=1e-12)
    np.testing.assert_allclose(gy, GYt, rtol=1e-12, atol=1e-12)
    # a column's gradient is exactly w_j times its unweighted one
    _, gy1 = p1.gradient(X, Yt)
    np.testing.assert_allclose(gy, gy1 * w[:, None], rtol=1e-14, atol=0)


def test_weighted_sweep_invariance(oracle_mod):
    """Weights c on every column with regulariser weights c lambda and steps
    alpha / c: every gradient step, prox and accept test of the sweep is the
    unweighted one (x - (alpha/c)(c g) = x - alpha g; prox of (alpha/c) c
    lambda r; c f_new <= c f_old), so the factors follow the unweighted
    trajectory and the objective is c times it."""
    o = oracle_mod
    c = 4.0  # a power of two: the scaling is exact in floating point
    t = W.small_mixed(m=16, n=12, k=3, seed=13, rx=(RQ, 0.2), ry=(RL1, 0.1), nkinds=7)
    p1 = _offset_problem(o, t, offset=True)
    pc = _offset_problem(o, t, offset=True, col_scale=np.full(t.n, c), rx=(RQ, 0.2 * c), ry=(RL1, 0.1 * c))
    ax, ay = p1.initial_alphas()
    X1, Y1, ax1, ay1, h1, acc1 = p1.proxgrad(t.X0, t.Yt0, 6, ax, ay)
    Xc, Yc, axc, ayc, hc, accc = pc.proxgrad(t.X0, t.Yt0, 6, ax / c, ay / c)
    np.testing.assert_allclose(Xc, X1, rtol=1e-12, atol=1e-13)
    np.testing.assert_allclose(Yc, Y1, rtol=1e-12, atol=1e-13)
    np.testing.assert_allclose(hc, c * h1, rtol=1e-12)
    np.testing.assert_array_equal(accc, acc1)
    np.testing.assert_allclose(axc * c, ax1, rtol=1e-14)


def test_column_stats_smallest_minimiser(oracle_mod):
    """Where the minimisers form an interval mu_j is its smallest point: the
    lower median of an even count (l1), the lower alpha-quantile, -1 for a
    hinge column with as many +1 as -1 labels (S flat on [-1, 1])."""
    o = oracle_mod
    rng = np.random.default_rng(21)
    v = np.sort(rng.normal(size=10))
    mu, _ = _columns(o, [v], L1).column_stats()
    assert mu[0] == pytest.approx(v[4], abs=1e-12)
    alpha = 0.3  # alpha c = 3 for c = 10: every x in [v_3, v_4] (1-based) minimises
    mu, _ = _columns(o, [v], QT, param=alpha).column_stats()
    assert mu[0] == pytest.approx(v[2], abs=1e-12)
    mu, s2 = _columns(o, [[1.0] * 3 + [-1.0] * 3], HI).column_stats()
    assert mu[0] == pytest.approx(-1.0, abs=1e-12)
    assert s2[0] == pytest.approx(6.0 / 5.0)
