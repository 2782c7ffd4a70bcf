"""The allocation-free objective (glrm_objective_noalloc) against the handle's
objective (glrm_objective_at) on the same data, two calls in a row.

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


def test_noalloc_matches_handle_objective_twice(G):
    t = W.small_mixed(m=5003, n=217, k=20, p_obs=0.45, seed=91, rx=(1, 0.1), ry=(2, 0.05))
    g = G.GLRM.from_table(t)
    X = torch.as_tensor(t.X0, dtype=torch.float32, device="cuda")
    Yt = torch.as_tensor(t.Yt0, dtype=torch.float32, device="cuda")
    ref = torch.zeros(1, dtype=torch.float64, device="cuda")
    G.glrm_objective_at(g.h, X, Yt, ref)
    rowptr = torch.as_tensor(t.rowptr, dtype=torch.int32, device="cuda")
    colidx = torch.as_tensor(t.colidx, dtype=torch.int32, device="cuda")
    val = torch.as_tensor(t.val, dtype=torch.float32, device="cuda")
    losses = _loss_bytes(t)
    outs = []
    for _ in range(2):
        out = torch.full((1,), float("nan"), dtype=torch.float64, device="cuda")
        G.glrm_objective_noalloc(t.m, t.n, t.k, rowptr, colidx, val, losses, t.rx, t.ry, X, Yt, out)
        torch.cuda.synchronize()
        outs.append(out.item())
    r = ref.item()
    for v in outs:
        assert np.isfinite(v)
        assert abs(v - r) / abs(r) < 1e-5, (v, r)
    assert outs[0] == outs[1]  # a fixed summation order


def test_noalloc_rejects_sizes_beyond_scratch(G):
    t = W.small_mixed(m=50, n=20, k=4, seed=92)
    dummy = torch.zeros(16, dtype=torch.int32, device="cuda")
    out = torch.zeros(1, dtype=torch.float64, device="cuda")
    with pytest.raises(G.GLRMError) as e:
        G.glrm_objective_noalloc(1 << 20, 1, 4, dummy, dummy, dummy, dummy, (0, 0.0),
                                 (0, 0.0), dummy, dummy, out)
    assert e.value.code == G.GLRM_ERR_RANGE
