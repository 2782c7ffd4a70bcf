"""The BF16 form: gradient passes on BF16 copies of the other factor with
FP32 accumulation and FP32 loss derivatives (FP32 rows for a segment retrying
after a rejected step); candidates evaluated on FP32 rows, so the accept /
reject test and the objective are those of the FP32 form.  Checked against the FP64 oracle (gradient
element by element within 2e-2, objectives and sampled predictions of a
row-reduced completion table) and against the plain FP32 sweep (objective
accuracy)."""
import numpy as np
import pytest
import torch

from paper_1410_0342_gb300 import workloads as W

from gpu_parity import U_REL_BF16, assert_grad_close, grad_bounds

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def G():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1410_0342_gb300 import build
    build.build()
    from paper_1410_0342_gb300 import glrm
    return glrm


def oracle_problem(o, t):
    return o.Problem.from_csr(t.m, t.n, t.k, t.rowptr, t.colidx, t.val, loss_kind=t.loss_kind,
                              loss_param=t.loss_param, loss_levels=t.loss_levels, rx=t.rx, ry=t.ry)


@pytest.mark.parametrize("k", [16, 64])
def test_bf16_gradient_within_2e2(G, oracle_mod, k):
    t = W.completion(m=8000, n=600, k=k, per_row=60, seed=60 + k)
    g = G.GLRM.from_table(t, precision=G.GLRM_BF16)
    assert G.glrm_get_path(g.h) == (G.GLRM_PATH_CHUNKED, G.GLRM_PATH_CHUNKED)
    X = torch.as_tensor(t.X0, dtype=torch.float32, device="cuda")
    Yt = torch.as_tensor(t.Yt0, dtype=torch.float32, device="cuda")
    GX = torch.empty_like(X)
    GY = torch.empty_like(Yt)
    G.glrm_grad_at(g.h, X, Yt, GX, GY, include_reg=False)
    p = oracle_problem(oracle_mod, t)
    Xd, Yd = X.double().cpu().numpy(), Yt.double().cpu().numpy()
    oGX, oGY = p.gradient(Xd, Yd)
    sX, sY, vX, vY = grad_bounds(p, Xd, Yd, U_REL_BF16)
    # element by element: 2e-2 relative plus 2^-7 of the terms' absolute sum
    # (two BF16 roundings, 2^-9 relative each, in every product of the sum)
    for a, b, sc, v, nm in ((GX, oGX, sX, vX, "GX"), (GY, oGY, sY, vY, "GYt")):
        assert_grad_close(a.cpu().numpy(), b, sc, v, rtol=2e-2, srel=2.0 ** -7, what=nm)
        rel = np.linalg.norm(a.double().cpu().numpy() - b) / np.linalg.norm(b)
        assert rel > 1e-7  # it really ran on BF16 copies


def test_bf16_reaches_fp32_objective_small_table(G, oracle_mod):
    """20,000 x 400, k = 64, 40 entries per row, compared with the FP32 sweep
    at the same objective accuracy: the BF16 form never increases the
    objective, the objective it reports is the FP32 objective of the factors
    it keeps (candidates and decisions are evaluated on FP32 rows), and it
    reaches the FP32 form's 20-sweep objective to within 1e-4 (the FP32 form
    itself is within 1e-4 of the FP64 oracle there).  On this small,
    underdetermined table (40 entries per row, k = 64) its BF16 gradients take
    more sweeps to get there; the count is printed."""
    t = W.completion(m=20000, n=400, k=64, per_row=40, seed=79)
    gb = G.GLRM.from_table(t, precision=G.GLRM_BF16)
    gf = G.GLRM.from_table(t, precision=G.GLRM_FP32)
    hf = gf.sweep(20)
    hb = gb.sweep(200)
    *_, oh, _ = oracle_problem(oracle_mod, t).proxgrad(t.X0, t.Yt0, 20)
    assert abs(hf[-1] - oh[-1]) / oh[-1] < 1e-4, (hf[-1], oh[-1])
    assert np.all(np.diff(hb) <= 1e-7 * np.abs(hb[1:]))
    reach = np.nonzero(hb <= hf[-1] * (1 + 1e-4))[0]
    print(f"BF16 form reaches the FP32 form's 20-sweep objective after {reach[0] + 1 if reach.size else None} sweeps")
    assert reach.size, (hb[-1], hf[-1])
    X, Yt = gb.factors()
    out = torch.zeros(1, dtype=torch.float64, device="cuda")
    G.glrm_objective_at(gb.h, X, Yt, out)
    assert abs(out.item() - hb[-1]) / hb[-1] < 1e-5


def test_bf16_matches_fp32_objective_midsize(G):
    """200,000 x 20,000, k = 64, 200 entries per row (the completion workload
    at a fifth of its rows): objectives of the BF16 and FP32 forms after 10
    sweeps from the same start within 1e-4."""
    t = W.completion(m=200_000, n=20_000, k=64, per_row=200, seed=81)
    gb = G.GLRM.from_table(t, precision=G.GLRM_BF16)
    hb = gb.sweep(10)
    gb.close()
    gf = G.GLRM.from_table(t, precision=G.GLRM_FP32)
    hf = gf.sweep(10)
    assert np.all(np.diff(hb) <= 1e-7 * np.abs(hb[1:]))
    assert (np.abs(hb - hf) / hf).max() < 1e-4, np.abs(hb - hf) / hf


def test_completion_sample_against_oracle(G, oracle_mod):
    """The completion workload at 1/20 of its rows (50,000 x 20,000, k = 64,
    200 entries per row, quadratic loss, gamma = 0.05): FP32 and BF16 forms
    after 6 free-running sweeps against the FP64 oracle's 6 sweeps from the
    same start (quadratic loss: no kinks, so the trajectories stay together).
    Objectives within 1e-4 relative; predictions u = x_i . y_j on a seeded
    sample of 10^6 cells (observed or not) compared with the oracle's
    factors: relative RMS error printed, bounded by 1e-4 (FP32) and 1e-2
    (BF16: the gathered rows carry 2^-9 relative rounding)."""
    t = W.completion(m=50_000, n=20_000, k=64, per_row=200, seed=83)
    T = 6
    p = oracle_problem(oracle_mod, t)
    Xo, Yo, *_, oh, _ = p.proxgrad(t.X0, t.Yt0, T)
    rng = np.random.default_rng(1410034203)
    ri = rng.integers(0, t.m, 1_000_000)
    ci = rng.integers(0, t.n, 1_000_000)
    uo = np.einsum("ek,ek->e", Xo[ri], Yo[ci])
    rows = torch.as_tensor(ri, dtype=torch.int32, device="cuda")
    cols = torch.as_tensor(ci, dtype=torch.int32, device="cuda")
    for prec, bound in ((G.GLRM_FP32, 1e-4), (G.GLRM_BF16, 1e-2)):
        g = G.GLRM.from_table(t, precision=prec)
        h = g.sweep(T)
        rel = np.abs(h - oh) / oh
        assert rel.max() < 1e-4, (prec, rel)
        u = g.predict(rows, cols, decode=False).double().cpu().numpy()
        err = np.sqrt(np.mean((u - uo) ** 2) / np.mean(uo ** 2))
        print(f"precision {prec}: objective rel diff {rel.max():.2e}, prediction rel RMS {err:.2e}")
        assert err < bound, (prec, err)
        g.close()
