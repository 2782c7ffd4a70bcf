"""GPU parity of the proximal-gradient sweep, objective, gradient, imputation
and ALS against the FP64 oracle, on the same seeded inputs.

Tolerances: FP64 path: objectives after a fixed number of sweeps within 1e-9
relative and identical accept counts.  FP32 path: each sweep from a state
shared with the oracle within 1e-5 relative (near-tie accept / reject flips
allowed on at most 1% of rows, see gpu_parity.py); objectives after a fixed
number of free-running sweeps within 1e-4 on tables large enough that a flip
does not move the total.  FP32 gradients element by element within 1e-5
relative plus the FP32 summation bound of their terms (gpu_parity.assert_grad_close),
empty rows and columns exactly zero;
Omega handling and decoded Boolean / ordinal values bit-exact."""
import numpy as np
import pytest
import torch

from paper_1410_0342_gb300 import workloads as W

from gpu_parity import assert_grad_close, grad_bounds, synced_sweeps

pytestmark = pytest.mark.gpu

Q, HU, HI, LO, OR = 0, 1, 2, 3, 4
RZ, RQ, RL1, RNN = 0, 1, 2, 3


@pytest.fixture(scope="module")
def G():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1410_0342_gb300 import build
    build.build()
    from paper_1410_0342_gb300 import glrm
    return glrm


def oracle_problem(o, t, rx=None, ry=None):
    return o.Problem.from_csr(t.m, t.n, t.k, t.rowptr, t.colidx, t.val, loss_kind=t.loss_kind,
                              loss_param=t.loss_param, loss_levels=t.loss_levels,
                              rx=rx or t.rx, ry=ry or t.ry)


def relerr(a, b):
    a, b = np.asarray(a, np.float64), np.asarray(b, np.float64)
    return np.abs(a - b) / np.maximum(np.abs(b), 1e-300)


def test_fp64_qpca_matches_oracle(G, oracle_mod):
    t = W.qpca_dense()
    g = G.GLRM.from_table(t, precision=G.GLRM_FP64)
    hist = g.sweep(100)
    acc = g.accepts()
    X, Yt, ax, ay, ohist, oacc = oracle_problem(oracle_mod, t).proxgrad(t.X0, t.Yt0, 100)
    assert relerr(hist, ohist).max() < 1e-9
    assert tuple(acc) == tuple(oacc[-1])
    Xg, Ytg = g.factors()
    np.testing.assert_allclose(Xg.cpu().numpy(), X, rtol=1e-7, atol=1e-9)
    np.testing.assert_allclose(Ytg.cpu().numpy(), Yt, rtol=1e-7, atol=1e-9)


def test_fp64_reaches_qpca_closed_form(G):
    t = W.qpca_dense()
    g = G.GLRM.from_table(t, precision=G.GLRM_FP64)
    hist = g.sweep(3000)
    A = t.val.reshape(t.m, t.n)
    s = np.linalg.svd(A, compute_uv=False)
    fstar = float(np.sum(A * A) - np.sum(np.maximum(s[:t.k] - 0.1, 0) ** 2))
    assert (hist[-1] - fstar) / fstar < 1e-8


@pytest.mark.parametrize("k", [6, 8, 19, 20, 33, 50, 64])
def test_fp32_mixed_matches_oracle(G, oracle_mod, k):
    t = W.small_mixed(m=211, n=57, k=k, seed=100 + k)
    g = G.GLRM.from_table(t)
    synced_sweeps(g, oracle_mod, t, 12)


def test_fp32_free_running_objective(G, oracle_mod):
    """20 free-running sweeps of quadratic-loss matrix completion (20,000 x
    400, 40 entries per row, k = 16): objectives within 1e-4 of the oracle's.
    (With piecewise-linear losses the FP32 and FP64 trajectories part after
    near-tie flips; those tables are checked sweep by sweep instead.)"""
    t = W.completion(m=20000, n=400, k=16, per_row=40, seed=78)
    g = G.GLRM.from_table(t)
    hist = g.sweep(20)
    *_, ohist, _ = oracle_problem(oracle_mod, t).proxgrad(t.X0, t.Yt0, 20)
    assert relerr(hist, ohist).max() < 1e-4


def test_fp32_multichunk_segments(G, oracle_mod):
    """Columns of ~1500 entries (two chunks and a ragged tail) and rows with
    zero entries."""
    t = W.small_mixed(m=3001, n=130, k=20, p_obs=0.5, seed=31, rx=(RQ, 0.1), ry=(RL1, 0.02))
    rowptr = t.rowptr.copy()
    # empty rows 0, 17 and the last; empty column 5
    keep = np.ones(t.nnz, bool)
    rows = t.rows()
    keep &= ~np.isin(rows, [0, 17, t.m - 1])
    keep &= t.colidx != 5
    t2 = _subset(t, keep)
    g = G.GLRM.from_table(t2)
    synced_sweeps(g, oracle_mod, t2, 10)


def _subset(t, keep):
    rows = t.rows()[keep]
    cols = t.colidx[keep]
    vals = t.val[keep]
    rowptr = np.zeros(t.m + 1, np.int64)
    np.cumsum(np.bincount(rows, minlength=t.m), out=rowptr[1:])
    colptr, rowidx, cval = W.csc_from_csr(t.m, t.n, rowptr, cols, vals)
    return W.Table(t.name, t.m, t.n, t.k, rowptr, cols, vals, colptr, rowidx, cval,
                   t.loss_kind, t.loss_param, t.loss_levels, t.rx, t.ry, t.X0, t.Yt0)


def test_objective_and_gradient_match_oracle(G, oracle_mod):
    """Objective and gradient at caller factors (glrm_objective_at,
    glrm_grad_at) and at the model's factors (glrm_grad), element by element,
    on a table with empty rows and an empty column (their loss gradient is
    exactly zero)."""
    t = W.small_mixed(m=1500, n=90, k=20, seed=41, rx=(RQ, 0.1), ry=(RL1, 0.05))
    keep = ~np.isin(t.rows(), [0, 700, t.m - 1]) & (t.colidx != 13)
    t = _subset(t, keep)
    g = G.GLRM.from_table(t)
    X = torch.as_tensor(t.X0, dtype=torch.float32, device="cuda")
    Yt = torch.as_tensor(t.Yt0, dtype=torch.float32, device="cuda")
    out = torch.zeros(1, dtype=torch.float64, device="cuda")
    G.glrm_objective_at(g.h, X, Yt, out)
    p = oracle_problem(oracle_mod, t)
    # the oracle evaluates at the same float32-rounded factors
    Xd, Yd = X.double().cpu().numpy(), Yt.double().cpu().numpy()
    assert relerr(out.item(), p.objective(Xd, Yd)) < 1e-5
    GX = torch.empty_like(X)
    GY = torch.empty_like(Yt)
    G.glrm_grad_at(g.h, X, Yt, GX, GY, include_reg=False)
    oGX, oGY = p.gradient(Xd, Yd)
    sX, sY, vX, vY = grad_bounds(p, Xd, Yd)
    assert_grad_close(GX.cpu().numpy(), oGX, sX, vX, what="GX")
    assert_grad_close(GY.cpu().numpy(), oGY, sY, vY, what="GYt")
    for i in (0, 700, t.m - 1):
        assert not GX[i].any()
    assert not GY[13].any()
    # glrm_grad: the same at the handle's own factors
    GX2, GY2 = g.grad()
    assert torch.equal(GX2, GX) and torch.equal(GY2, GY)
    G.glrm_grad_at(g.h, X, Yt, GX, GY, include_reg=True)
    rgx = oGX + 2 * 0.1 * Xd
    rgy = oGY + 0.05 * np.sign(Yd)
    assert_grad_close(GX.cpu().numpy(), rgx, sX + 2 * 0.1 * np.abs(Xd), vX, what="GX + reg")
    assert_grad_close(GY.cpu().numpy(), rgy, sY + 0.05, vY, what="GYt + reg")


def test_decode_bit_exact(G, oracle_mod):
    """Decoded values equal the oracle's decode of the same u, including the
    half-integer ties of the ordinal hinge and u = 0 for Boolean columns."""
    t = W.small_mixed(m=300, n=60, k=6, seed=51)
    g = G.GLRM.from_table(t)
    g.sweep(5)
    rng = np.random.default_rng(0)
    rows = torch.as_tensor(rng.integers(0, t.m, 20000), dtype=torch.int32, device="cuda")
    cols = torch.as_tensor(rng.integers(0, t.n, 20000), dtype=torch.int32, device="cuda")
    u = g.predict(rows, cols, decode=False).cpu().numpy()
    dec = g.predict(rows, cols, decode=True).cpu().numpy()
    c = cols.cpu().numpy()
    for e in range(u.size):
        j = c[e]
        ref = oracle_mod.decode(int(t.loss_kind[j]), float(u[e]), int(t.loss_levels[j]))
        assert dec[e] == np.float32(ref), (e, j, u[e], dec[e], ref)
    # exact ties through a handle whose factors produce chosen u values
    k = 1
    n = 8
    us = np.array([0.0, -0.0, 1.5, 2.5, 3.5, 6.5, 2.4999998, 2.5000002], np.float32)
    kinds = np.array([HI, LO, OR, OR, OR, OR, OR, OR])
    gg = G.GLRM(1, n, k, (kinds, np.zeros(n), np.where(kinds == OR, 7, 0)), (RZ, 0.0), (RZ, 0.0))
    tt = W.Table("ties", 1, n, k, np.array([0, n]), np.arange(n, dtype=np.int32),
                 np.where(kinds == OR, 1.0, 1.0), np.arange(n + 1), np.zeros(n, np.int32),
                 np.ones(n), kinds, np.zeros(n), np.where(kinds == OR, 7, 0), (RZ, 0.0),
                 (RZ, 0.0), np.ones((1, 1)), us.reshape(n, 1).astype(np.float64))
    gg.set_observed_table(tt)
    gg.set_factors(torch.ones(1, 1, device="cuda"), torch.as_tensor(us.reshape(n, 1), device="cuda"))
    r = torch.zeros(n, dtype=torch.int32, device="cuda")
    cc = torch.arange(n, dtype=torch.int32, device="cuda")
    d = gg.predict(r, cc).cpu().numpy()
    for j in range(n):
        ref = oracle_mod.decode(int(kinds[j]), float(us[j]), 7)
        assert d[j] == np.float32(ref), (j, us[j], d[j], ref)


def test_deterministic_and_resumable(G):
    t = W.small_mixed(m=800, n=70, k=12, seed=61)
    g1 = G.GLRM.from_table(t)
    h1 = g1.sweep(10)
    g2 = G.GLRM.from_table(t)
    h2a = g2.sweep(4)
    st = g2.state()
    g3 = G.GLRM.from_table(t, factors=False)
    g3.load_state(st)
    h3 = g3.sweep(6)
    np.testing.assert_array_equal(h1, np.concatenate([h2a, h3]))
    X1, Y1 = g1.factors()
    X3, Y3 = g3.factors()
    assert torch.equal(X1, X3) and torch.equal(Y1, Y3)


def test_als_matches_oracle(G, oracle_mod):
    t = W.qpca_dense()
    g = G.GLRM.from_table(t, precision=G.GLRM_FP64)
    hist = g.als_sweep(30)
    X, Yt, ohist = oracle_problem(oracle_mod, t).als(t.X0, t.Yt0, 0.1, 30)
    assert relerr(hist, ohist).max() < 1e-9
    # missing data, FP32 Gram accumulation, k = 16 (ALS has no accept / reject
    # branch, so free-running trajectories stay together)
    t2 = W.batch_instance(0, m_range=(400, 400), n_range=(120, 120), ks=(16,))
    g2 = G.GLRM.from_table(t2)
    h2 = g2.als_sweep(10)
    *_, oh2 = oracle_problem(oracle_mod, t2).als(t2.X0, t2.Yt0, 0.1, 10)
    assert relerr(h2, oh2).max() < 1e-4


def test_als_rejects_non_quadratic(G):
    t = W.small_mixed(m=50, n=20, k=4)
    g = G.GLRM.from_table(t)
    with pytest.raises(G.GLRMError) as e:
        g.als_sweep(1)
    assert e.value.code == G.GLRM_ERR_ARG


def _omega_tensors(t, dt=torch.float32):
    i32 = torch.int32
    return [torch.as_tensor(t.rowptr, dtype=i32, device="cuda"),
            torch.as_tensor(t.colidx, dtype=i32, device="cuda"),
            torch.as_tensor(t.val, dtype=dt, device="cuda"),
            torch.as_tensor(t.colptr, dtype=i32, device="cuda"),
            torch.as_tensor(t.rowidx, dtype=i32, device="cuda"),
            torch.as_tensor(t.cval, dtype=dt, device="cuda")]


@pytest.mark.parametrize("fault", ["ptr", "range", "dup", "unsorted", "cross", "value", "nan",
                                   "domain"])
def test_observed_set_validation(G, fault):
    t = W.small_mixed(m=40, n=15, k=4, seed=71)
    g = G.GLRM(t.m, t.n, t.k, (t.loss_kind, t.loss_param, t.loss_levels), t.rx, t.ry)
    a = _omega_tensors(t)
    if fault == "ptr":
        a[0][3] = a[0][4] + 1
    elif fault == "range":
        a[1][5] = t.n
    elif fault == "dup":
        r = int(np.argmax(np.diff(t.rowptr) >= 2))
        a[1][int(t.rowptr[r]) + 1] = a[1][int(t.rowptr[r])]
    elif fault == "unsorted":
        r = int(np.argmax(np.diff(t.rowptr) >= 2))
        b = int(t.rowptr[r])
        a[1][b], a[1][b + 1] = a[1][b + 1].clone(), a[1][b].clone()
    elif fault == "cross":
        a[4][0] = (a[4][0] + 1) % t.m
    elif fault == "value":
        a[5][3] += 1.0
    elif fault == "nan":
        a[2][2] = float("nan")
    elif fault == "domain":
        # an ordinal column (kind 4 every fifth column) gets level 0 in both orientations
        j = 4
        q = int(t.colptr[j])
        i = int(t.rowidx[q])
        e = int(t.rowptr[i]) + int(np.searchsorted(t.colidx[t.rowptr[i]:t.rowptr[i + 1]], j))
        a[2][e] = 0.0
        a[5][q] = 0.0
    with pytest.raises(G.GLRMError) as e:
        G.glrm_set_observed(g.h, t.nnz, *a)
    expect = G.GLRM_ERR_NONFINITE if fault == "nan" else G.GLRM_ERR_OMEGA
    assert e.value.code == expect
    with pytest.raises(G.GLRMError) as e:
        g.sweep(1)
    assert e.value.code == G.GLRM_ERR_STATE
    # a valid set afterwards works
    G.glrm_set_observed(g.h, t.nnz, *_omega_tensors(t))
    assert np.isfinite(g.sweep(1)).all()


@pytest.mark.parametrize("fault", [None, "unsorted", "dup", "range", "value", "cross"])
def test_observed_set_validation_long_columns(G, oracle_mod, fault):
    """A tall table (20,000 x 6, 90% observed): the CSC's columns hold about
    18,000 entries each, so its checks and digest split every column into
    pieces of about 1,024 entries; faults sit on a piece boundary or deep in a
    column.  The valid table sweeps in step with the oracle."""
    t = W.small_mixed(m=20000, n=6, k=4, p_obs=0.9, seed=73)
    g = G.GLRM(t.m, t.n, t.k, (t.loss_kind, t.loss_param, t.loss_levels), t.rx, t.ry)
    if fault is None:
        G.glrm_set_observed(g.h, t.nnz, *_omega_tensors(t))
        g.set_factors(torch.as_tensor(t.X0, dtype=torch.float32, device="cuda"),
                      torch.as_tensor(t.Yt0, dtype=torch.float32, device="cuda"))
        synced_sweeps(g, oracle_mod, t, 2, rtol=1e-5)
        return
    a = _omega_tensors(t)
    j = 2
    sb, se = int(t.colptr[j]), int(t.colptr[j + 1])
    pieces = max(1, min(1024, (t.nnz // t.n + 1023) // 1024))
    per = -(-(se - sb) // pieces)
    q = sb + per  # first entry of the column's second piece
    assert pieces > 1 and sb < q - 1 and q + 3 * per < se
    if fault == "unsorted":
        a[4][q - 1], a[4][q] = a[4][q].clone(), a[4][q - 1].clone()
    elif fault == "dup":
        a[4][q] = a[4][q - 1]
    elif fault == "range":
        a[4][q + 3 * per] = t.m
    elif fault == "value":
        a[5][q + 2 * per + 5] += 1.0
    elif fault == "cross":
        # a row index moved to an unobserved row, order kept: only the digests see it
        gaps = np.nonzero(np.diff(t.rowidx[sb:se]) >= 2)[0]
        a[4][sb + int(gaps[len(gaps) // 2])] += 1
    with pytest.raises(G.GLRMError) as e:
        G.glrm_set_observed(g.h, t.nnz, *a)
    assert e.value.code == G.GLRM_ERR_OMEGA
    G.glrm_set_observed(g.h, t.nnz, *_omega_tensors(t))
    assert np.isfinite(g.sweep(1)).all()


def test_host_entry_points(G, oracle_mod):
    t = W.small_mixed(m=120, n=40, k=5, seed=81)
    g = G.GLRM(t.m, t.n, t.k, (t.loss_kind, t.loss_param, t.loss_levels), t.rx, t.ry)
    G.glrm_set_observed_host(g.h, t.nnz, t.rowptr.astype(np.int32), t.colidx,
                             t.val.astype(np.float32), t.colptr.astype(np.int32), t.rowidx,
                             t.cval.astype(np.float32))
    G.glrm_set_factors_host(g.h, t.X0.astype(np.float32), t.Yt0.astype(np.float32))
    synced_sweeps(g, oracle_mod, t, 5)
    X = np.empty((t.m, t.k), np.float32)
    Y = np.empty((t.n, t.k), np.float32)
    G.glrm_get_factors_host(g.h, X, Y)
    Xd, Yd = g.factors()
    np.testing.assert_array_equal(X, Xd.cpu().numpy())
    np.testing.assert_array_equal(Y, Yd.cpu().numpy())


@pytest.mark.parametrize("prec,reg,tol", [(0, (RQ, 0.1), 1e-9), (0, (RL1, 0.05), 1e-9),
                                          (0, (RNN, 0.0), 1e-9), (1, (RQ, 0.1), 1e-4),
                                          (1, (RNN, 0.0), 1e-4)])
def test_proxprox_matches_oracle(G, oracle_mod, prec, reg, tol):
    """Prox-prox sweeps (Sec. 7.2 update, Sec. 7.3 cached factorisation) on a
    30%-missing quadratic-loss table with the given regulariser on both
    factors: objectives after each of 6 sweeps (3 updates per row / column,
    alpha = 0.5) and the final factors against the oracle's (no accept /
    reject branch, so FP32 trajectories stay with the FP64 ones)."""
    import dataclasses
    t = W.batch_instance(0, m_range=(400, 400), n_range=(120, 120), ks=(8,))
    t = dataclasses.replace(t, rx=reg, ry=reg)
    g = G.GLRM.from_table(t, precision=prec)
    h = g.proxprox_sweep(6, 0.5, 3)
    X, Yt, oh = oracle_problem(oracle_mod, t).proxprox(t.X0, t.Yt0, 0.5, 3, 6)
    assert np.isfinite(h).all()
    assert relerr(h, oh).max() < tol, relerr(h, oh)
    Xg, Yg = g.factors()
    np.testing.assert_allclose(Xg.double().cpu().numpy(), X, rtol=tol * 10, atol=tol * 10)
    np.testing.assert_allclose(Yg.double().cpu().numpy(), Yt, rtol=tol * 10, atol=tol * 10)


def test_proxprox_rejects_non_quadratic(G):
    t = W.small_mixed(m=50, n=20, k=4)
    g = G.GLRM.from_table(t)
    with pytest.raises(G.GLRMError) as e:
        g.proxprox_sweep(1, 0.5, 2)
    assert e.value.code == G.GLRM_ERR_ARG
