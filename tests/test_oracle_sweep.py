"""Pins of the oracle's objective, gradient, proximal-gradient sweep and
alternating-minimisation sweep against what the paper fixes: the quadratically
regularised PCA closed form (eq. pca-reg-soln; Appendix A), Eckart-Young
(Sec. 2.4), X^T X = Y Y^T at stationary points (Appendix A), the monotone
objective the step-size safeguard guarantees (Sec. 7.2), finite-difference
gradients and the l1 optimality conditions."""
import numpy as np
import pytest

from paper_1410_0342_gb300 import workloads as W

Q, HU, HI, LO, OR = 0, 1, 2, 3, 4
RZ, RQ, RL1, RNN = 0, 1, 2, 3


def _problem(o, t: W.Table, rx=None, ry=None):
    return o.Problem.from_csr(t.m, t.n, t.k, t.rowptr, t.colidx, t.val, loss_kind=t.loss_kind,
                              loss_param=t.loss_param, loss_levels=t.loss_levels,
                              rx=rx or t.rx, ry=ry or t.ry)


def qpca_optimum(A, k, gamma):
    """min ||A - XY||_F^2 + gamma(||X||^2 + ||Y||^2) = ||A||^2 - sum_{i<=k} ((s_i - gamma)_+)^2."""
    s = np.linalg.svd(A, compute_uv=False)
    return float(np.sum(A * A) - np.sum(np.maximum(s[:k] - gamma, 0.0) ** 2))


def test_objective_matches_matrix_form(oracle_mod):
    """Fully observed quadratic problem: the entry sum equals the matrix form."""
    o = oracle_mod
    t = W.qpca_dense(m=23, n=17, k=3, seed=7)
    p = _problem(o, t)
    A = t.val.reshape(t.m, t.n)
    X, Yt = t.X0, t.Yt0
    ref = np.sum((A - X @ Yt.T) ** 2) + 0.1 * np.sum(X * X) + 0.1 * np.sum(Yt * Yt)
    assert p.objective(X, Yt) == pytest.approx(ref, rel=1e-13)


@pytest.mark.parametrize("nkinds", [5, 7])
def test_objective_brute_force_mixed(oracle_mod, nkinds):
    """Every loss kind and regulariser, summed cell by cell over a dense mask."""
    o = oracle_mod
    t = W.small_mixed(m=13, n=11, k=3, seed=3, rx=(RL1, 0.2), ry=(RQ, 0.3), nkinds=nkinds)
    p = _problem(o, t)
    rows = t.rows()
    X, Yt = t.X0, t.Yt0
    tot = 0.0
    for e in range(t.nnz):
        i, j, a = rows[e], t.colidx[e], t.val[e]
        u = float(X[i] @ Yt[j])
        tot += o.loss(int(t.loss_kind[j]), u, a, float(t.loss_param[j]), int(t.loss_levels[j]))
    tot += 0.2 * np.abs(X).sum() + 0.3 * np.sum(Yt * Yt)
    assert p.objective(X, Yt) == pytest.approx(tot, rel=1e-12)


def test_gradient_matches_finite_differences(oracle_mod):
    """Loss part of the gradient against central differences of the loss part
    of the objective (zero regularisers), away from kinks."""
    o = oracle_mod
    t = W.small_mixed(m=9, n=10, k=3, seed=5, rx=(RZ, 0.0), ry=(RZ, 0.0))
    # drop the kinked losses' kinks by using smooth kinds only
    kinds = np.array([Q, HU, LO, Q, HU, LO, Q, HU, LO, Q], dtype=np.int32)
    rows = t.rows()
    vals = t.val.copy()
    for e in range(t.nnz):
        if kinds[t.colidx[e]] == LO:
            vals[e] = 1.0 if vals[e] > 0 else -1.0
    p = o.Problem(t.m, t.n, t.k, rows, t.colidx, vals, kinds, np.full(t.n, 0.7), 0)
    X, Yt = t.X0.copy(), t.Yt0.copy()
    GX, GYt = p.gradient(X, Yt)
    h = 1e-6
    for i in range(t.m):
        for c in range(t.k):
            Xp, Xm = X.copy(), X.copy()
            Xp[i, c] += h
            Xm[i, c] -= h
            fd = (p.objective(Xp, Yt) - p.objective(Xm, Yt)) / (2 * h)
            assert GX[i, c] == pytest.approx(fd, abs=2e-5, rel=1e-5)
    for j in range(t.n):
        for c in range(t.k):
            Yp, Ym = Yt.copy(), Yt.copy()
            Yp[j, c] += h
            Ym[j, c] -= h
            fd = (p.objective(X, Yp) - p.objective(X, Ym)) / (2 * h)
            assert GYt[j, c] == pytest.approx(fd, abs=2e-5, rel=1e-5)


def test_proxgrad_reaches_qpca_closed_form(oracle_mod):
    """Sweeps on the 200x100, k=5, gamma=0.1 qPCA table reach the closed-form
    optimum (unique local minimum, Appendix A) and X^T X = Y Y^T there."""
    o = oracle_mod
    t = W.qpca_dense()
    p = _problem(o, t)
    A = t.val.reshape(t.m, t.n)
    fstar = qpca_optimum(A, t.k, 0.1)
    X, Yt, ax, ay, hist, acc = p.proxgrad(t.X0, t.Yt0, 3000)
    assert np.all(np.diff(hist) <= 1e-9 * np.abs(hist[1:]))
    assert (hist[-1] - fstar) / fstar < 1e-8
    np.testing.assert_allclose(X.T @ X, Yt.T @ Yt, atol=1e-4 * np.abs(X.T @ X).max())


def test_proxgrad_eckart_young(oracle_mod):
    """gamma = 0: the optimum is the truncated-SVD error sum_{i>k} s_i^2."""
    o = oracle_mod
    t = W.qpca_dense(m=40, n=30, k=3, seed=11)
    p = _problem(o, t, rx=(RZ, 0.0), ry=(RZ, 0.0))
    A = t.val.reshape(t.m, t.n)
    s = np.linalg.svd(A, compute_uv=False)
    ey = float(np.sum(s[t.k:] ** 2))
    *_, hist, _ = p.proxgrad(t.X0, t.Yt0, 6000)
    assert (hist[-1] - ey) / ey < 1e-6


def test_proxgrad_monotone_mixed(oracle_mod):
    """The safeguard rejects increasing steps, so the objective never rises
    (Sec. 7.2); nonnegativity holds on Y after the first sweep."""
    o = oracle_mod
    t = W.small_mixed()
    p = _problem(o, t)
    X, Yt, ax, ay, hist, acc = p.proxgrad(t.X0, t.Yt0, 60)
    assert np.all(np.isfinite(hist))
    assert np.all(np.diff(hist) <= 1e-12 * np.abs(hist[1:]))
    assert Yt.min() >= 0.0
    assert acc[0, 1] == t.n  # first Y-step leaves an infinite objective: all accepted
    # the returned objective is the objective of the returned factors
    assert p.objective(X, Yt) == pytest.approx(hist[-1], rel=1e-13)


def test_proxgrad_thread_count_invariant(oracle_mod):
    o = oracle_mod
    t = W.small_mixed(m=120, n=50, seed=9)
    p = _problem(o, t)
    r1 = p.proxgrad(t.X0, t.Yt0, 7, nthreads=1)
    r4 = p.proxgrad(t.X0, t.Yt0, 7, nthreads=4)
    for a, b in zip(r1, r4):
        np.testing.assert_array_equal(a, b)


def test_proxgrad_step_rule_single_row(oracle_mod):
    """A single fully observed row: the X-step of the first sweep can be
    followed by hand (gradient, prox of gamma||x||^2, accept test, alpha
    update), and the result must match the oracle's."""
    o = oracle_mod
    rng = np.random.default_rng(4)
    k, n = 3, 6
    Yt = rng.normal(size=(n, k))
    a = rng.normal(size=n)
    x = rng.normal(size=(1, k))
    p = o.Problem(1, n, k, np.zeros(n, np.int32), np.arange(n, dtype=np.int32), a,
                  np.full(n, Q), 0.0, 0, rx=(RQ, 0.2), ry=(RZ, 0.0))
    # the expected X-step: g = sum 2(u - a) y_j; z = x - g/n; prox; accept test
    alpha = 1.0 / n
    u = Yt @ x[0]
    g = (2 * (u - a)) @ Yt
    xp = (x[0] - alpha * g) / (1 + 2 * alpha * 0.2)
    fo = np.sum((u - a) ** 2) + 0.2 * x[0] @ x[0]
    fn = np.sum((Yt @ xp - a) ** 2) + 0.2 * xp @ xp
    X1, Yt1, ax, ay, hist, acc = p.proxgrad(x, Yt, 1)
    if fn <= fo:
        np.testing.assert_allclose(X1[0], xp, rtol=1e-13)
        assert ax[0] == pytest.approx(alpha * 1.05)
    else:
        np.testing.assert_array_equal(X1[0], x[0])
        assert ax[0] == pytest.approx(alpha * 0.7)


def test_proxgrad_l1_optimality(oracle_mod):
    """At convergence with l1 on X, every row meets 0 in g_i + lambda d|x_i|:
    g_ic = -lambda sign(x_ic) where x_ic != 0 and |g_ic| <= lambda where 0."""
    o = oracle_mod
    t = W.qpca_dense(m=30, n=20, k=3, seed=13)
    lam = 2.0
    p = _problem(o, t, rx=(RL1, lam), ry=(RQ, 0.1))
    X, Yt, *_ = p.proxgrad(t.X0, t.Yt0, 20000)
    GX, _ = p.gradient(X, Yt)
    nz = np.abs(X) > 1e-9
    assert nz.any() and (~nz).any()
    np.testing.assert_allclose(GX[nz], -lam * np.sign(X[nz]), atol=1e-4)
    assert np.all(np.abs(GX[~nz]) <= lam + 1e-4)


def test_als_normal_equations(oracle_mod):
    """One ALS sweep: each x_i solves (sum y_j y_j^T + gamma I) x = sum a_ij y_j
    (Sec. 2.4) with the old Y; each y_j then solves its equations with the new X."""
    o = oracle_mod
    t = W.small_mixed(m=15, n=12, k=4, seed=21, p_obs=0.6)
    gamma = 0.3
    rows = t.rows()
    p = o.Problem(t.m, t.n, t.k, rows, t.colidx, t.val, np.full(t.n, Q), 0.0, 0,
                  rx=(RQ, gamma), ry=(RQ, gamma))
    X1, Yt1, hist = p.als(t.X0, t.Yt0, gamma, 1)
    for i in range(t.m):
        sel = rows == i
        Yi = t.Yt0[t.colidx[sel]]
        G = Yi.T @ Yi + gamma * np.eye(t.k)
        np.testing.assert_allclose(X1[i], np.linalg.solve(G, Yi.T @ t.val[sel]), rtol=1e-10,
                                   atol=1e-12)
    for j in range(t.n):
        sel = t.colidx == j
        Xj = X1[rows[sel]]
        G = Xj.T @ Xj + gamma * np.eye(t.k)
        np.testing.assert_allclose(Yt1[j], np.linalg.solve(G, Xj.T @ t.val[sel]), rtol=1e-10,
                                   atol=1e-12)


def test_als_reaches_qpca_closed_form(oracle_mod):
    o = oracle_mod
    t = W.qpca_dense()
    p = _problem(o, t)
    A = t.val.reshape(t.m, t.n)
    fstar = qpca_optimum(A, t.k, 0.1)
    X, Yt, hist = p.als(t.X0, t.Yt0, 0.1, 5000)
    assert np.all(np.diff(hist) <= 1e-10 * np.abs(hist[1:]))
    assert (hist[-1] - fstar) / fstar < 1e-9


def test_proxgrad_one_sweep_by_hand(oracle_mod):
    """One full sweep (Algorithm 2, Sec. 7.2) of a 2 x 2 table with cell (1, 1)
    missing, k = 1, quadratic loss (u - a)^2, no regularisers, followed by hand
    in exact dyadic arithmetic.  Steps start at alpha = 1/n_i: 1/2 and 1 for
    the rows, 1/2 and 1 for the columns.

    X-step against y = (-1/2, 3/2):
      row 0 (a = 1/2, 1/4): u = (5/8, -15/8), g = 2 (1/8 (-1/2) - 17/8 (3/2))
        = -13/2, x+ = -5/4 + 13/4 = 2; f_old = 290/64 < f_new = 628/64:
        rejected, x stays -5/4, alpha = 1/2 * 0.7.
      row 1 (a = -1): u = 7/8, g = 2 (15/8)(-1/2) = -15/8, x+ = 1/8;
        f_new = 225/256 <= f_old = 225/64: accepted, alpha = 1.05.
    Y-step against the NEW x = (-5/4, 1/8) (Gauss-Seidel):
      column 0 (a = 1/2, -1): u = (5/8, -1/16), g = 2 (1/8 (-5/4) + 15/16 (1/8))
        = -5/64, y+ = -1/2 + 5/128 = -59/128; f_new = 937309/2^20 <=
        f_old = 937984/2^20: accepted, alpha = 1/2 * 1.05.
      column 1 (a = 1/4): u = -15/8, g = 85/16, y+ = -61/16; f_new =
        83521/4096 > f_old = 289/64: rejected, alpha = 0.7.
    A Jacobi sweep (Y-step against the old x = (-5/4, -7/4)) would reject
    column 0 and keep y_0 = -1/2, so this pins the order of the half-steps
    as well as both branches of the step-size rule."""
    o = oracle_mod
    rows = np.array([0, 0, 1], np.int32)
    cols = np.array([0, 1, 0], np.int32)
    vals = np.array([0.5, 0.25, -1.0])
    p = o.Problem(2, 2, 1, rows, cols, vals, Q, 0.0, 0, rx=(RZ, 0.0), ry=(RZ, 0.0))
    X0 = np.array([[-1.25], [-1.75]])
    Yt0 = np.array([[-0.5], [1.5]])
    ax0, ay0 = p.initial_alphas()
    np.testing.assert_array_equal(ax0, [0.5, 1.0])
    np.testing.assert_array_equal(ay0, [0.5, 1.0])
    X1, Yt1, ax, ay, hist, acc = p.proxgrad(X0, Yt0, 1)
    np.testing.assert_array_equal(X1[:, 0], [-1.25, 0.125])
    np.testing.assert_array_equal(Yt1[:, 0], [-59.0 / 128.0, 1.5])
    np.testing.assert_allclose(ax, [0.5 * 0.7, 1.05], rtol=1e-15)
    np.testing.assert_allclose(ay, [0.5 * 1.05, 0.7], rtol=1e-15)
    assert tuple(acc[0]) == (1, 1)
    # objective of eq. gpca at the new factors: column 0's two terms + column 1's
    assert hist[0] == 937309.0 / 2**20 + (-1.25 * 1.5 - 0.25) ** 2


def test_proxgrad_empty_row_and_column(oracle_mod):
    """A row and a column with no observed entries (Sec. 7.2 with n_i = 0):
    their step starts at alpha = 1 / max(0, 1) = 1, the gradient is zero, so
    the update is x <- prox_{alpha r}(x): soft thresholding at alpha lambda for
    l1 on X, shrinkage by 1 / (1 + 2 alpha gamma) for gamma ||y||^2 on Y.  Both
    lower r, so both are accepted and alpha becomes 1.05."""
    o = oracle_mod
    lam, gam = 0.5, 0.25
    # 2 x 2 with row 1 and column 1 empty: the only entry is (0, 0)
    p = o.Problem(2, 2, 3, np.array([0], np.int32), np.array([0], np.int32), np.array([0.3]),
                  Q, 0.0, 0, rx=(RL1, lam), ry=(RQ, gam))
    ax0, ay0 = p.initial_alphas()
    np.testing.assert_array_equal(ax0, [1.0, 1.0])
    np.testing.assert_array_equal(ay0, [1.0, 1.0])
    X0 = np.array([[0.2, -0.1, 0.4], [0.75, -0.25, 0.1]])
    Yt0 = np.array([[0.3, 0.6, -0.2], [1.0, -2.0, 0.5]])
    X1, Yt1, ax, ay, hist, acc = p.proxgrad(X0, Yt0, 1)
    np.testing.assert_array_equal(X1[1], [0.25, 0.0, 0.0])  # soft threshold at 1 * 0.5
    np.testing.assert_array_equal(Yt1[1], Yt0[1] / (1.0 + 2.0 * gam))
    assert ax[1] == 1.05 and ay[1] == 1.05


def test_gradient_abs_brute_force(oracle_mod):
    """sum |L'| |w| per gradient coordinate, cell by cell over the entries; and
    where every term is nonnegative (hinge with a = -1 and u > -1, so L' = 1,
    and nonnegative factors) it equals the gradient itself."""
    o = oracle_mod
    t = W.small_mixed(m=11, n=9, k=3, seed=8, rx=(RZ, 0.0), ry=(RZ, 0.0))
    p = _problem(o, t)
    rows = t.rows()
    SX, SY = p.gradient_abs(t.X0, t.Yt0)
    bx = np.zeros_like(SX)
    by = np.zeros_like(SY)
    for e in range(t.nnz):
        i, j, a = rows[e], t.colidx[e], t.val[e]
        d = abs(o.dloss(int(t.loss_kind[j]), float(t.X0[i] @ t.Yt0[j]), a, float(t.loss_param[j]),
                        int(t.loss_levels[j])))
        bx[i] += d * np.abs(t.Yt0[j])
        by[j] += d * np.abs(t.X0[i])
    np.testing.assert_allclose(SX, bx, rtol=1e-13, atol=1e-15)
    np.testing.assert_allclose(SY, by, rtol=1e-13, atol=1e-15)
    rng = np.random.default_rng(2)
    X = rng.uniform(0.1, 1.0, size=(6, 2))
    Yt = rng.uniform(0.1, 1.0, size=(5, 2))
    r, c = np.nonzero(rng.random((6, 5)) < 0.7)
    q = o.Problem(6, 5, 2, r.astype(np.int32), c.astype(np.int32), -np.ones(r.size), HI, 0.0, 0)
    GX, GY = q.gradient(X, Yt)
    SX, SY = q.gradient_abs(X, Yt)
    np.testing.assert_allclose(SX, GX, rtol=1e-14)
    np.testing.assert_allclose(SY, GY, rtol=1e-14)


def test_gradient_variation_closed_forms(oracle_mod):
    """Quadratic loss: L'(u + d) - L'(u - d) = 4 d, so the variation is
    sum 4 u_rel (sum_c |x_c y_c|) |w|.  Hinge with a = 1: a product exactly at
    the kink u = 1 gives the unit jump (0 - (-1)) times |w|; products more than
    delta away from it give 0."""
    o = oracle_mod
    rng = np.random.default_rng(3)
    X = rng.normal(size=(4, 3))
    Yt = rng.normal(size=(5, 3))
    r, c = np.nonzero(rng.random((4, 5)) < 0.8)
    r, c = r.astype(np.int32), c.astype(np.int32)
    q = o.Problem(4, 5, 3, r, c, rng.normal(size=r.size), Q, 0.0, 0)
    VX, VY = q.gradient_variation(X, Yt, 1e-3)
    ex = np.zeros_like(X)
    ey = np.zeros_like(Yt)
    for i, j in zip(r, c):
        d = 1e-3 * np.sum(np.abs(X[i] * Yt[j]))
        ex[i] += 4 * d * np.abs(Yt[j])
        ey[j] += 4 * d * np.abs(X[i])
    np.testing.assert_allclose(VX, ex, rtol=1e-9)
    np.testing.assert_allclose(VY, ey, rtol=1e-9)
    # hinge: row 0 sits on the kink (u = 1) for column 0, far from it for column 1
    Xh = np.array([[1.0, 0.0]])
    Yh = np.array([[1.0, 0.5], [3.0, 2.0]])
    h = o.Problem(1, 2, 2, np.array([0, 0], np.int32), np.array([0, 1], np.int32),
                  np.array([1.0, 1.0]), HI, 0.0, 0)
    VX, VY = h.gradient_variation(Xh, Yh, 1e-6)
    np.testing.assert_allclose(VX[0], np.abs(Yh[0]), rtol=1e-15)
    np.testing.assert_allclose(VY[0], np.abs(Xh[0]), rtol=1e-15)
    assert not VY[1].any()


def _one_row(o, rng, n=9, k=3, reg=(RZ, 0.0)):
    Yt = rng.normal(size=(n, k))
    a = rng.normal(size=n)
    p = o.Problem(1, n, k, np.zeros(n, np.int32), np.arange(n, dtype=np.int32), a, Q, 0.0, 0,
                  rx=reg, ry=(RZ, 0.0))
    return p, Yt, a, Yt.T @ Yt, Yt.T @ a


def test_proxprox_fixed_point_least_squares(oracle_mod):
    """r = 0: the prox-prox update's fixed point (Sec. 7.2) is the exact
    least-squares solution G x = b of the row problem (the Y-step that
    follows does not touch the returned row)."""
    o = oracle_mod
    rng = np.random.default_rng(21)
    p, Yt, a, G, b = _one_row(o, rng)
    X, *_ = p.proxprox(rng.normal(size=(1, 3)), Yt, alpha=0.5, inner=4000, nsweeps=1)
    np.testing.assert_allclose(X[0], np.linalg.solve(G, b), rtol=1e-9)


def test_proxprox_fixed_point_quadratic_regulariser(oracle_mod):
    """r = gamma ||x||^2: x = prox_{alpha r}(prox_{alpha f}(x)) with
    prox_{alpha f}(x) = (2 alpha G + I)^{-1}(2 alpha b + x) and prox_{alpha r}
    = scaling by 1 / (1 + 2 alpha gamma) holds exactly when
    ((1 + 2 alpha gamma) G + gamma I) x = b (derived by substituting one into
    the other).  That is the minimiser of the Moreau envelope of f plus r,
    which differs from the minimiser of f + r, (G + gamma I) x = b, unless
    alpha -> 0."""
    o = oracle_mod
    rng = np.random.default_rng(22)
    gam, al = 0.7, 0.4
    p, Yt, a, G, b = _one_row(o, rng, reg=(RQ, gam))
    X, *_ = p.proxprox(rng.normal(size=(1, 3)), Yt, alpha=al, inner=4000, nsweeps=1)
    np.testing.assert_allclose(X[0], np.linalg.solve((1 + 2 * al * gam) * G + gam * np.eye(3), b),
                               rtol=1e-9)
    assert np.abs(X[0] - np.linalg.solve(G + gam * np.eye(3), b)).max() > 1e-3


def test_proxprox_fixed_point_nonnegative(oracle_mod):
    """r = indicator of x >= 0: the update is a projected gradient step on the
    Moreau envelope M(x) = f(P x) + ||x - P x||^2 / (2 alpha), P x =
    prox_{alpha f}(x), so its fixed point minimises M over x >= 0; an
    independent bounded quasi-Newton solve of that problem agrees."""
    from scipy import optimize
    o = oracle_mod
    rng = np.random.default_rng(23)
    al = 0.3
    p, Yt, a, G, b = _one_row(o, rng, n=12, k=4, reg=(RNN, 0.0))
    X, *_ = p.proxprox(np.abs(rng.normal(size=(1, 4))), Yt, alpha=al, inner=20000, nsweeps=1)
    Mi = np.linalg.inv(2 * al * G + np.eye(4))

    def env(x):
        px = Mi @ (2 * al * b + x)
        return np.sum((Yt @ px - a) ** 2) + np.sum((x - px) ** 2) / (2 * al)

    res = optimize.minimize(env, np.ones(4), method="L-BFGS-B", bounds=[(0, None)] * 4,
                            options={"ftol": 1e-15, "gtol": 1e-12, "maxiter": 10000})
    assert X[0].min() >= 0.0 and (X[0] == 0.0).any()
    np.testing.assert_allclose(X[0], res.x, atol=2e-5)
