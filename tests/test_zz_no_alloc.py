"""The allocation-free objective (glrm_objective_noalloc) against the FP64
oracle and the handle's objective (glrm_objective_at) on the same data, two
calls in a row.

Callers that cannot allocate device memory where they need the objective (a
CUDA graph capture in progress, a host pool owning all device memory) use
this entry point: its scratch is a fixed device array inside the library.
This file is named to run last so that a failure here stops a run only after
every other test has run."""
import numpy as np
import pytest
import torch

from paper_1410_0342_gb300 import workloads as W

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def G():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1410_0342_gb300 import build
    build.build()
    from paper_1410_0342_gb300 import glrm
    return glrm


def _loss_bytes(t):
    rec = np.zeros(t.n, dtype=[("kind", "<i4"), ("levels", "<i4"), ("param", "<f8")])
    rec["kind"] = t.loss_kind
    rec["levels"] = t.loss_levels
    rec["param"] = t.loss_param
    return torch.from_numpy(rec.view(np.uint8).copy()).cuda()


def _inputs(t):
    dev = "cuda"
    return (torch.as_tensor(t.rowptr, dtype=torch.int32, device=dev),
            torch.as_tensor(t.colidx, dtype=torch.int32, device=dev),
            torch.as_tensor(t.val, dtype=torch.float32, device=dev),
            _loss_bytes(t),
            torch.as_tensor(t.X0, dtype=torch.float32, device=dev),
            torch.as_tensor(t.Yt0, dtype=torch.float32, device=dev))


def test_noalloc_matches_oracle_and_handle_twice(G, oracle_mod):
    """Two calls in a row: each equals the FP64 oracle's objective at the same
    FP32-rounded factors within 1e-5 relative (FP32 loss terms, FP64 sums) and
    the handle's glrm_objective_at, and the two calls agree bit for bit."""
    t = W.small_mixed(m=5003, n=217, k=20, p_obs=0.45, seed=91, rx=(1, 0.1), ry=(2, 0.05))
    g = G.GLRM.from_table(t)
    rowptr, colidx, val, losses, X, Yt = _inputs(t)
    ref = torch.zeros(1, dtype=torch.float64, device="cuda")
    G.glrm_objective_at(g.h, X, Yt, ref)
    p = oracle_mod.Problem.from_csr(t.m, t.n, t.k, t.rowptr, t.colidx, t.val, loss_kind=t.loss_kind,
                                    loss_param=t.loss_param, loss_levels=t.loss_levels, rx=t.rx,
                                    ry=t.ry)
    want = p.objective(X.double().cpu().numpy(), Yt.double().cpu().numpy())
    outs = []
    for _ in range(2):
        out = torch.full((1,), float("nan"), dtype=torch.float64, device="cuda")
        G.glrm_objective_noalloc(t.m, t.n, t.k, t.nnz, rowptr, colidx, val, losses, t.rx, t.ry, X,
                                 Yt, out)
        torch.cuda.synchronize()
        outs.append(out.item())
    r = ref.item()
    for v in outs:
        assert np.isfinite(v)
        assert abs(v - want) / abs(want) < 1e-5, (v, want)
        assert abs(v - r) / abs(r) < 1e-5, (v, r)
    assert outs[0] == outs[1]  # a fixed summation order


def test_noalloc_malformed_inputs_give_nan(G):
    """A row range reaching past nnz, a column index out of range and a loss
    descriptor of unknown kind each turn the result into NaN; no read leaves
    the caller's arrays (the row range is checked against nnz before use)."""
    t = W.small_mixed(m=300, n=40, k=6, seed=93, rx=(1, 0.1), ry=(2, 0.05))
    rowptr, colidx, val, losses, X, Yt = _inputs(t)
    out = torch.zeros(1, dtype=torch.float64, device="cuda")

    def run(rp=rowptr, ci=colidx, ls=losses):
        out.fill_(0.0)
        G.glrm_objective_noalloc(t.m, t.n, t.k, t.nnz, rp, ci, val, ls, t.rx, t.ry, X, Yt, out)
        torch.cuda.synchronize()
        return out.item()

    assert np.isfinite(run())
    rp = rowptr.clone()
    rp[-1] = t.nnz + 5          # last row claims entries beyond nnz
    assert np.isnan(run(rp=rp))
    rp = rowptr.clone()
    rp[7] = rp[8] + 1           # row 7 runs backwards
    assert np.isnan(run(rp=rp))
    ci = colidx.clone()
    ci[3] = t.n                 # column index out of range
    assert np.isnan(run(ci=ci))
    ls = losses.clone()
    ls[16 * int(t.colidx[0])] = 9  # unknown loss kind in a column that row 0 uses
    assert np.isnan(run(ls=ls))
    assert np.isfinite(run())


def test_noalloc_rejects_bad_arguments(G):
    dummy = torch.zeros(16, dtype=torch.int32, device="cuda")
    out = torch.zeros(1, dtype=torch.float64, device="cuda")
    with pytest.raises(G.GLRMError) as e:
        G.glrm_objective_noalloc(1 << 20, 1, 4, 0, dummy, dummy, dummy, dummy, (0, 0.0),
                                 (0, 0.0), dummy, dummy, out)
    assert e.value.code == G.GLRM_ERR_RANGE
    with pytest.raises(G.GLRMError) as e:
        G.glrm_objective_noalloc(4, 4, 4, 1 << 31, dummy, dummy, dummy, dummy, (0, 0.0),
                                 (0, 0.0), dummy, dummy, out)
    assert e.value.code == G.GLRM_ERR_RANGE
    with pytest.raises(G.GLRMError) as e:
        G.glrm_objective_noalloc(4, 4, 4, 0, dummy, dummy, dummy, dummy, (1, -0.5),
                                 (0, 0.0), dummy, dummy, out)
    assert e.value.code == G.GLRM_ERR_ARG
