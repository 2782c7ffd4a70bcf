"""The dense, fully observed form (tensor-core contractions) against the FP64
oracle run on the same table as an observed set with every entry present.

Tolerances come from the arithmetic: the products x_i . y_j are six BF16
products of three-part splits x = hi + mid + lo accumulated in FP32, an error
of about 2^-25 sum_c |x_ic y_jc| per entry, below FP32's k 2^-24; the
gradient contraction R W splits R the same way.  So
per-sweep objectives from a state shared with the oracle agree within 1e-5
(as for the FP32 sparse path); factors after a sweep within 1e-4; gradients
element by element within 1e-5 relative plus the FP32 summation bound of
their terms (gpu_parity.assert_grad_close).  Shapes are ragged against the 128-row tiles and 64-wide chunks,
and large enough that both half-steps split the other dimension into parts."""
import numpy as np
import pytest
import torch

from paper_1410_0342_gb300 import workloads as W

from gpu_parity import assert_grad_close, grad_bounds, oracle_problem, synced_sweeps

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def G():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1410_0342_gb300 import build
    build.build()
    from paper_1410_0342_gb300 import glrm
    return glrm


def dense_mixed(m, n, k, seed, rx=(1, 0.1), ry=(1, 0.1)):
    return W.small_mixed(m=m, n=n, k=k, p_obs=1.0, seed=seed, rx=rx, ry=ry)


def test_dense_qpca_tiny_matches_oracle(G, oracle_mod):
    """200 x 100, k = 5 (one partial tile each way, k padded to 16)."""
    t = W.qpca_dense()
    g = G.GLRM.from_dense_table(t)
    assert tuple(G.glrm_get_path(g.h)) == (G.GLRM_PATH_DENSE, G.GLRM_PATH_DENSE)
    rels = synced_sweeps(g, oracle_mod, t, 10, rtol=1e-5)
    assert rels.max() < 1e-5


@pytest.mark.parametrize("m,n,k", [(1000, 301, 20), (777, 130, 33), (300, 64, 64), (129, 65, 16)])
def test_dense_mixed_matches_oracle(G, oracle_mod, m, n, k):
    """Every loss kind (columns cycle quadratic, Huber, hinge, logistic,
    ordinal), ragged m and n, k padded to 16 / 32 / 64."""
    t = dense_mixed(m, n, k, seed=500 + k)
    g = G.GLRM.from_dense_table(t)
    synced_sweeps(g, oracle_mod, t, 6, rtol=1e-5)


def test_dense_objective_and_gradient(G, oracle_mod):
    """Objective and gradient at the initial factors on a 5,000 x 2,000 table
    (k = 64): both half-steps split the other dimension into several parts."""
    t = W.qpca_dense(m=5000, n=2000, k=64, seed=77)
    g = G.GLRM.from_dense_table(t)
    p = oracle_problem(oracle_mod, t)
    X = torch.as_tensor(t.X0, dtype=torch.float32, device="cuda")
    Yt = torch.as_tensor(t.Yt0, dtype=torch.float32, device="cuda")
    out = torch.zeros(1, dtype=torch.float64, device="cuda")
    G.glrm_objective_at(g.h, X, Yt, out)
    Xd = X.double().cpu().numpy()
    Yd = Yt.double().cpu().numpy()
    of = p.objective(Xd, Yd)
    assert abs(out.item() - of) / of < 1e-5, (out.item(), of)
    GX = torch.empty_like(X)
    GY = torch.empty_like(Yt)
    G.glrm_grad_at(g.h, X, Yt, GX, GY, include_reg=False)
    oGX, oGY = p.gradient(Xd, Yd)
    sX, sY, vX, vY = grad_bounds(p, Xd, Yd)
    assert_grad_close(GX.cpu().numpy(), oGX, sX, vX, what="GX")
    assert_grad_close(GY.cpu().numpy(), oGY, sY, vY, what="GYt")


@pytest.mark.parametrize("k", [20, 64])
def test_dense_long_loops_match_oracle(G, oracle_mod, k):
    """20,000 x 2,000 mixed table: each CTA walks 8 or more 64-wide chunks, so
    every staging ring and completion barrier wraps several times.  Objective
    and gradient at random factors, then two synced sweeps."""
    t = W.mixed_dense(m=20000, n=2000, k=k, n_real=1000, n_bool=600, seed=600 + k,
                      rx=(2, 0.01), ry=(1, 0.1)).observed()
    g = G.GLRM.from_dense_table(t)
    p = oracle_problem(oracle_mod, t)
    X = torch.as_tensor(t.X0, dtype=torch.float32, device="cuda")
    Yt = torch.as_tensor(t.Yt0, dtype=torch.float32, device="cuda")
    out = torch.zeros(1, dtype=torch.float64, device="cuda")
    G.glrm_objective_at(g.h, X, Yt, out)
    of = p.objective(X.double().cpu().numpy(), Yt.double().cpu().numpy())
    assert abs(out.item() - of) / of < 1e-5, (out.item(), of)
    GX = torch.empty_like(X)
    GY = torch.empty_like(Yt)
    G.glrm_grad_at(g.h, X, Yt, GX, GY, include_reg=False)
    Xd, Yd = X.double().cpu().numpy(), Yt.double().cpu().numpy()
    oGX, oGY = p.gradient(Xd, Yd)
    sX, sY, vX, vY = grad_bounds(p, Xd, Yd)
    assert_grad_close(GX.cpu().numpy(), oGX, sX, vX, what="GX")
    assert_grad_close(GY.cpu().numpy(), oGY, sY, vY, what="GYt")
    synced_sweeps(g, oracle_mod, t, 2, rtol=1e-5)


def test_dense_mixed_objective_gradient(G, oracle_mod):
    t = dense_mixed(1500, 410, 24, seed=9)
    g = G.GLRM.from_dense_table(t)
    p = oracle_problem(oracle_mod, t)
    rng = np.random.default_rng(5)
    X = torch.as_tensor(rng.standard_normal((t.m, t.k)), dtype=torch.float32, device="cuda")
    Yt = torch.as_tensor(rng.standard_normal((t.n, t.k)), dtype=torch.float32, device="cuda")
    out = torch.zeros(1, dtype=torch.float64, device="cuda")
    G.glrm_objective_at(g.h, X, Yt, out)
    of = p.objective(X.double().cpu().numpy(), Yt.double().cpu().numpy())
    assert abs(out.item() - of) / of < 1e-5
    GX = torch.empty_like(X)
    GY = torch.empty_like(Yt)
    G.glrm_grad_at(g.h, X, Yt, GX, GY, include_reg=True)
    Xd, Yd = X.double().cpu().numpy(), Yt.double().cpu().numpy()
    oGX, oGY = p.gradient(Xd, Yd)
    sX, sY, vX, vY = grad_bounds(p, Xd, Yd)
    # glrm_grad_at adds the regulariser's gradient (quadratic, weight 0.1)
    oGX = oGX + 2 * 0.1 * Xd
    oGY = oGY + 2 * 0.1 * Yd
    assert_grad_close(GX.cpu().numpy(), oGX, sX + 0.2 * np.abs(Xd), vX, what="GX + reg")
    assert_grad_close(GY.cpu().numpy(), oGY, sY + 0.2 * np.abs(Yd), vY, what="GYt + reg")


def test_dense_matches_sparse_fp32_one_sweep(G):
    """The dense form and the FP32 sparse path on the same fully observed
    quadratic table (3,000 x 700, k = 32), one sweep from the same state:
    objectives within 1e-5, accepted rows and columns within 1%.  (Free-running
    trajectories part after near-tie accept / reject flips, as between any two
    roundings.)"""
    t = W.qpca_dense(m=3000, n=700, k=32, seed=41)
    gd = G.GLRM.from_dense_table(t)
    gs = G.GLRM.from_table(t, precision=G.GLRM_FP32)
    for _ in range(3):
        hd = gd.sweep(1)[0]
        hs = gs.sweep(1)[0]
        assert abs(hd - hs) / hs < 1e-5, (hd, hs)
        ad, as_ = gd.accepts(), gs.accepts()
        assert abs(int(ad[0]) - int(as_[0])) <= max(2, t.m // 100)
        assert abs(int(ad[1]) - int(as_[1])) <= max(2, t.n // 100)
        gs.load_state(gd.state())


def test_dense_reaches_qpca_closed_form(G):
    """Quadratic loss and regulariser on a fully observed table: the sweep
    approaches ||A||^2 - sum_i (sigma_i - gamma)_+^2 (Section 2.5, shrunk
    singular values) as closely as FP32 arithmetic allows.  On this table the
    FP32 sparse path stalls 9.0e-5 above f* (its accept / reject test stops
    resolving the remaining decrease); the dense form must do as well, 1e-4."""
    t = W.qpca_dense()
    g = G.GLRM.from_dense_table(t)
    hist = g.sweep(3000)
    assert np.all(np.diff(hist) <= 1e-7 * np.abs(hist[1:]))
    A = t.val.reshape(t.m, t.n)
    s = np.linalg.svd(A, compute_uv=False)
    fstar = float(np.sum(A * A) - np.sum(np.maximum(s[:t.k] - 0.1, 0) ** 2))
    assert 0 <= (hist[-1] - fstar) / fstar < 1e-4, (hist[-1], fstar)


def test_dense_host_copy_and_pitch(G):
    """glrm_set_dense_host from a strided host array equals glrm_set_dense."""
    t = dense_mixed(300, 77, 8, seed=3)
    A = t.val.reshape(t.m, t.n).astype(np.float32)
    wide = np.zeros((t.m, 80), np.float32)
    wide[:, :t.n] = A
    g1 = G.GLRM.from_dense_table(t)
    g2 = G.GLRM(t.m, t.n, t.k, (t.loss_kind, t.loss_param, t.loss_levels), t.rx, t.ry)
    G.glrm_set_dense_host(g2.h, wide, 80)
    g2.set_factors(torch.as_tensor(t.X0, dtype=torch.float32, device="cuda"),
                   torch.as_tensor(t.Yt0, dtype=torch.float32, device="cuda"))
    np.testing.assert_array_equal(g1.sweep(3), g2.sweep(3))


def test_dense_validation(G):
    t = dense_mixed(200, 50, 8, seed=4)
    A = torch.as_tensor(t.val.reshape(t.m, t.n), dtype=torch.float32, device="cuda")
    g = G.GLRM(t.m, t.n, t.k, (t.loss_kind, t.loss_param, t.loss_levels), t.rx, t.ry)
    bad = A.clone()
    bad[3, 7] = float("nan")
    with pytest.raises(G.GLRMError) as e:
        g.set_dense(bad)
    assert e.value.code == G.GLRM_ERR_NONFINITE
    bad = A.clone()
    bad[5, 2] = 0.5  # column 2 has hinge loss: values must be -1 or +1
    with pytest.raises(G.GLRMError) as e:
        g.set_dense(bad)
    assert e.value.code == G.GLRM_ERR_OMEGA
    with pytest.raises(G.GLRMError) as e:
        G.glrm_set_dense(g.h, A, 10)
    assert e.value.code == G.GLRM_ERR_ARG
    with pytest.raises(G.GLRMError) as e:
        g.sweep(1)
    assert e.value.code == G.GLRM_ERR_STATE
    g.set_dense(A)
    g.sweep(1)
    with pytest.raises(G.GLRMError) as e:
        g.als_sweep(1)
    assert e.value.code == G.GLRM_ERR_STATE
    g64 = G.GLRM(t.m, t.n, t.k, (t.loss_kind, t.loss_param, t.loss_levels), t.rx, t.ry,
                 precision=G.GLRM_FP64)
    with pytest.raises(G.GLRMError) as e:
        g64.set_dense(A.double())
    assert e.value.code == G.GLRM_ERR_ARG


def test_dense_bf16_form(G, oracle_mod):
    """A GLRM_BF16 model on a table stored densely: the gradient contraction
    R W is one BF16 product on the tensor cores (elementwise within 2e-2 of
    the oracle, plus 2^-7 of the terms' absolute sum), while U, the losses and
    the objective keep FP32 quality (1e-5); its sweeps never increase the
    objective, report the FP32 objective of the kept factors, and reach the
    FP32 dense form's 12-sweep objective to within 1e-4."""
    t = W.mixed(m=6000, n=300, n_real=150, n_bool=90, seed=71)
    gb = G.GLRM.from_table(t, precision=G.GLRM_BF16)
    assert G.glrm_get_path(gb.h) == (G.GLRM_PATH_DENSE, G.GLRM_PATH_DENSE)
    p = oracle_problem(oracle_mod, t)
    rng = np.random.default_rng(3)
    X = torch.as_tensor(rng.standard_normal((t.m, t.k)), dtype=torch.float32, device="cuda")
    Yt = torch.as_tensor(np.abs(rng.standard_normal((t.n, t.k))), dtype=torch.float32, device="cuda")
    Xd, Yd = X.double().cpu().numpy(), Yt.double().cpu().numpy()
    out = torch.zeros(1, dtype=torch.float64, device="cuda")
    G.glrm_objective_at(gb.h, X, Yt, out)
    of = p.objective(Xd, Yd)
    assert abs(out.item() - of) / abs(of) < 1e-5
    GX = torch.empty_like(X)
    GY = torch.empty_like(Yt)
    G.glrm_grad_at(gb.h, X, Yt, GX, GY, include_reg=False)
    oGX, oGY = p.gradient(Xd, Yd)
    sX, sY, vX, vY = grad_bounds(p, Xd, Yd)
    assert_grad_close(GX.cpu().numpy(), oGX, sX, vX, rtol=2e-2, srel=2.0 ** -7, what="GX bf16")
    assert_grad_close(GY.cpu().numpy(), oGY, sY, vY, rtol=2e-2, srel=2.0 ** -7, what="GYt bf16")
    assert np.linalg.norm(GX.double().cpu().numpy() - oGX) / np.linalg.norm(oGX) > 1e-7  # really BF16
    gf = G.GLRM.from_table(t, precision=G.GLRM_FP32)
    hf = gf.sweep(12)
    hb = gb.sweep(60)
    assert np.all(np.diff(hb) <= 1e-7 * np.abs(hb[1:]))
    reach = np.nonzero(hb <= hf[-1] * (1 + 1e-4))[0]
    print(f"dense BF16 form reaches the FP32 form's 12-sweep objective after "
          f"{reach[0] + 1 if reach.size else None} sweeps")
    assert reach.size, (hb[-1], hf[-1])
    Xb, Yb = gb.factors()
    G.glrm_objective_at(gb.h, Xb, Yb, out)
    assert abs(out.item() - hb[-1]) / abs(hb[-1]) < 1e-5
