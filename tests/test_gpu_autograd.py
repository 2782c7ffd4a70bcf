"""The differentiable form: GLRMObjective forward / backward against the FP64
oracle, torch.autograd.gradcheck in FP64, central finite differences
(h = 1e-3, FP64) on seeded coordinates, and a torch optimizer loop against
the same loop driven by the oracle's gradient."""
import numpy as np
import pytest
import torch

from paper_1410_0342_gb300 import workloads as W

from gpu_parity import assert_grad_close, grad_bounds

pytestmark = pytest.mark.gpu

RQ = 1


@pytest.fixture(scope="module")
def G():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1410_0342_gb300 import build
    build.build()
    from paper_1410_0342_gb300 import glrm
    return glrm


@pytest.fixture(scope="module")
def AG(G):
    from paper_1410_0342_gb300 import autograd
    return autograd


def oracle_problem(o, t):
    return o.Problem.from_csr(t.m, t.n, t.k, t.rowptr, t.colidx, t.val, loss_kind=t.loss_kind,
                              loss_param=t.loss_param, loss_levels=t.loss_levels, rx=t.rx, ry=t.ry)


def test_forward_backward_match_oracle_logistic_table(G, AG, oracle_mod):
    """The differentiation workload: m = 50,000, n = 2,000, k = 32, logistic loss,
    20% missing, gamma = 0.1."""
    t = W.logistic_bool()
    g = G.GLRM.from_table(t, factors=False)
    X = torch.as_tensor(t.X0, dtype=torch.float32, device="cuda").requires_grad_()
    Yt = torch.as_tensor(t.Yt0, dtype=torch.float32, device="cuda").requires_grad_()
    F = AG.glrm_objective(X, Yt, g)
    F.backward()
    p = oracle_problem(oracle_mod, t)
    Xd, Yd = X.detach().double().cpu().numpy(), Yt.detach().double().cpu().numpy()
    ref = p.objective(Xd, Yd)
    assert abs(F.item() - ref) / abs(ref) < 1e-5
    gx, gy = p.gradient(Xd, Yd)
    sx, sy, vx, vy = grad_bounds(p, Xd, Yd)
    gx += 2 * 0.1 * Xd
    gy += 2 * 0.1 * Yd
    # element by element: 1e-5 relative plus the FP32 summation bound
    assert_grad_close(X.grad.cpu().numpy(), gx, sx + 0.2 * np.abs(Xd), vx, what="dF/dX")
    assert_grad_close(Yt.grad.cpu().numpy(), gy, sy + 0.2 * np.abs(Yd), vy, what="dF/dYt")


def test_backward_scales_with_incoming_derivative(G, AG):
    t = W.logistic_bool(m=700, n=90, k=8, seed=5)
    g = G.GLRM.from_table(t, factors=False)
    X = torch.as_tensor(t.X0, dtype=torch.float32, device="cuda").requires_grad_()
    Yt = torch.as_tensor(t.Yt0, dtype=torch.float32, device="cuda").requires_grad_()
    AG.glrm_objective(X, Yt, g).backward()
    gx1, gy1 = X.grad.clone(), Yt.grad.clone()
    X.grad = None
    Yt.grad = None
    (-2.5 * AG.glrm_objective(X, Yt, g)).backward()
    torch.testing.assert_close(X.grad, -2.5 * gx1, rtol=1e-6, atol=1e-6)
    torch.testing.assert_close(Yt.grad, -2.5 * gy1, rtol=1e-6, atol=1e-6)


def test_gradcheck_fp64(G, AG):
    t = W.logistic_bool(m=37, n=23, k=4, p_obs=0.7, seed=6)
    g = G.GLRM.from_table(t, precision=G.GLRM_FP64, factors=False)
    X = torch.as_tensor(t.X0, dtype=torch.float64, device="cuda").requires_grad_()
    Yt = torch.as_tensor(t.Yt0, dtype=torch.float64, device="cuda").requires_grad_()
    assert torch.autograd.gradcheck(lambda a, b: AG.glrm_objective(a, b, g), (X, Yt),
                                    eps=1e-6, atol=1e-6, rtol=1e-5)


def test_central_differences_fp64(G, AG, oracle_mod):
    """FP32 GPU gradient against central differences (h = 1e-3) of the FP64
    objective on 256 seeded coordinates of X and Y."""
    t = W.logistic_bool(m=3000, n=400, k=32, seed=7)
    g = G.GLRM.from_table(t, factors=False)
    X = torch.as_tensor(t.X0, dtype=torch.float32, device="cuda").requires_grad_()
    Yt = torch.as_tensor(t.Yt0, dtype=torch.float32, device="cuda").requires_grad_()
    AG.glrm_objective(X, Yt, g).backward()
    p = oracle_problem(oracle_mod, t)
    Xd, Yd = X.detach().double().cpu().numpy(), Yt.detach().double().cpu().numpy()
    gx, gy = X.grad.double().cpu().numpy(), Yt.grad.double().cpu().numpy()
    rng = np.random.default_rng(8)
    h = 1e-3
    scale = max(np.abs(gx).max(), np.abs(gy).max())
    for which, M, gm in (("X", Xd, gx), ("Y", Yd, gy)):
        for _ in range(128):
            i, c = int(rng.integers(0, M.shape[0])), int(rng.integers(0, M.shape[1]))
            Mp, Mm = M.copy(), M.copy()
            Mp[i, c] += h
            Mm[i, c] -= h
            if which == "X":
                fd = (p.objective(Mp, Yd) - p.objective(Mm, Yd)) / (2 * h)
            else:
                fd = (p.objective(Xd, Mp) - p.objective(Xd, Mm)) / (2 * h)
            assert abs(gm[i, c] - fd) <= 1e-4 * max(abs(fd), 1e-2 * scale), (which, i, c, gm[i, c], fd)


def test_optimizer_loop_matches_oracle_loop(G, AG, oracle_mod):
    """30 plain gradient steps through torch.optim.SGD against the same steps
    taken with the oracle's FP64 gradient."""
    t = W.logistic_bool(m=4000, n=500, k=16, seed=9)
    g = G.GLRM.from_table(t, factors=False)
    X = torch.nn.Parameter(torch.as_tensor(t.X0, dtype=torch.float32, device="cuda"))
    Yt = torch.nn.Parameter(torch.as_tensor(t.Yt0, dtype=torch.float32, device="cuda"))
    lr = 1e-3
    opt = torch.optim.SGD([X, Yt], lr=lr)
    hist = []
    for _ in range(30):
        opt.zero_grad()
        F = AG.glrm_objective(X, Yt, g)
        F.backward()
        opt.step()
        hist.append(F.item())
    p = oracle_problem(oracle_mod, t)
    Xo = t.X0.astype(np.float32).astype(np.float64)
    Yo = t.Yt0.astype(np.float32).astype(np.float64)
    ohist = []
    for _ in range(30):
        ohist.append(p.objective(Xo, Yo))
        gx, gy = p.gradient(Xo, Yo)
        gx += 2 * 0.1 * Xo
        gy += 2 * 0.1 * Yo
        Xo, Yo = Xo - lr * gx, Yo - lr * gy
    hist, ohist = np.array(hist), np.array(ohist)
    assert hist[-1] < 0.9 * hist[0]
    assert (np.abs(hist - ohist) / ohist).max() < 1e-4
