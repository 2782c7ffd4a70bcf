"""The batched form: many instances of uneven size in one set of launches,
against the FP64 oracle instance by instance (ALS instances free-running,
proximal-gradient instances one sweep at a time from a shared state), the
three launch modes giving identical results, the autotuner keeping the fit
state, and validation of the batched observed sets."""
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


def small_batch(count=24, **kw):
    kw.setdefault("m_range", (50, 700))
    kw.setdefault("n_range", (20, 160))
    return W.batch_torch(count, device="cuda", **kw)


def methods_of(wb, G):
    return [G.GLRM_BATCH_ALS if s % 2 == 0 else G.GLRM_BATCH_PROXGRAD for s in range(wb.count)]


def instance_arrays(wb, s):
    """Instance s's CSR arrays and initial factors as numpy (float64)."""
    m, n, k = int(wb.m[s]), int(wb.n[s]), int(wb.k[s])
    rp0 = int(np.sum(wb.m[:s] + 1))
    e0 = int(np.sum(wb.nnz[:s]))
    x0 = int(np.sum(wb.m[:s] * wb.k[:s]))
    y0 = int(np.sum(wb.n[:s] * wb.k[:s]))
    rowptr = wb.rowptr[rp0:rp0 + m + 1].cpu().numpy().astype(np.int64)
    colidx = wb.colidx[e0:e0 + int(wb.nnz[s])].cpu().numpy()
    val = wb.val[e0:e0 + int(wb.nnz[s])].double().cpu().numpy()
    return m, n, k, rowptr, colidx, val, (x0, y0), (int(np.sum(wb.m[:s])), int(np.sum(wb.n[:s])))


def oracle_for(o, wb, s):
    m, n, k, rowptr, colidx, val, _, _ = instance_arrays(wb, s)
    kind = int(wb.kind[s])
    return o.Problem.from_csr(m, n, k, rowptr, colidx, val, loss_kind=kind,
                              loss_param=1.0 if kind == 1 else 0.0, loss_levels=0,
                              rx=(1, 0.1), ry=(1, 0.1))


def split_factors(wb, s, X, Yt):
    m, n, k, *_, (x0, y0), _ = instance_arrays(wb, s)
    return (X[x0:x0 + m * k].reshape(m, k).double().cpu().numpy(),
            Yt[y0:y0 + n * k].reshape(n, k).double().cpu().numpy())


def check_batch(G, o, wb, meth, T, autotune=False):
    """Every instance against the oracle: ALS instances free-running for T
    sweeps (no accept / reject branch, so the trajectories stay together)
    within 1e-4; proximal-gradient instances one sweep at a time from the
    batch's own state within 1e-5."""
    B = G.Batch(wb, meth)
    if autotune:
        B.autotune(reps=2)
    X0, Y0 = B.factors()
    hist = []
    states = []
    for _ in range(T):
        X, Yt = B.factors()
        ax, ay = B.steps()
        states.append((X, Yt, ax, ay))
        hist.append(B.sweep(1)[0])
    hist = np.array(hist)
    for s in range(wb.count):
        p = oracle_for(o, wb, s)
        if meth[s] == G.GLRM_BATCH_ALS:
            Xs, Ys = split_factors(wb, s, X0, Y0)
            *_, oh = p.als(Xs, Ys, 0.1, T)
            rel = np.abs(hist[:, s] - oh) / np.abs(oh)
            assert rel.max() < 1e-4, (s, rel)
        else:
            _, _, _, _, _, _, _, (r0, c0) = instance_arrays(wb, s)
            for t in range(T):
                X, Yt, ax, ay = states[t]
                Xs, Ys = split_factors(wb, s, X, Yt)
                m, n = int(wb.m[s]), int(wb.n[s])
                axs = ax[r0:r0 + m].double().cpu().numpy()
                ays = ay[c0:c0 + n].double().cpu().numpy()
                *_, oh, _ = p.proxgrad(Xs, Ys, 1, axs, ays)
                assert abs(hist[t, s] - oh[0]) / abs(oh[0]) < 1e-5, (s, t, hist[t, s], oh[0])
    B.close()


def test_batch_matches_oracle(G, oracle_mod):
    wb = small_batch()
    check_batch(G, oracle_mod, wb, methods_of(wb, G), 4)


def test_batch_workload_sizes_match_oracle(G, oracle_mod):
    """The first 128 instances of the 4,096-instance workload itself (m up to
    5,000, n up to 500, k in {4, 8, 16}, every size class), with the work-item
    table autotuned first as the benchmark does."""
    wb = W.batch_torch(128, device="cuda")
    assert int(wb.m.max()) > 4000 and int(wb.n.max()) > 400 and set(wb.k.tolist()) == {4, 8, 16}
    check_batch(G, oracle_mod, wb, methods_of(wb, G), 3, autotune=True)


def test_launch_modes_agree(G):
    wb = small_batch(count=16)
    meth = methods_of(wb, G)
    out = []
    for mode in (G.GLRM_BATCH_GRAPH, G.GLRM_BATCH_STREAM, G.GLRM_BATCH_PER_INSTANCE):
        B = G.Batch(wb, meth)
        out.append((B.sweep(3, mode=mode), B.factors()))
        B.close()
    for h, (X, Y) in out[1:]:
        np.testing.assert_array_equal(h, out[0][0])
        assert torch.equal(X, out[0][1][0]) and torch.equal(Y, out[0][1][1])


def test_graph_replay_repeats(G):
    """A captured graph is replayed (same nsweeps) and continues the fit."""
    wb = small_batch(count=8)
    meth = methods_of(wb, G)
    B1 = G.Batch(wb, meth)
    h1 = np.concatenate([B1.sweep(2), B1.sweep(2)])
    B2 = G.Batch(wb, meth)
    h2 = B2.sweep(4, mode=G.GLRM_BATCH_STREAM)
    np.testing.assert_array_equal(h1, h2)


def test_autotune_keeps_state(G):
    wb = small_batch(count=20)
    meth = methods_of(wb, G)
    B = G.Batch(wb, meth)
    B.sweep(1)
    X, Yt = B.factors()
    tx, ty = B.autotune(reps=2)
    assert set(np.unique(tx)) <= {1, 2, 4, 8} and set(np.unique(ty)) <= {1, 2, 4, 8}
    X2, Yt2 = B.factors()
    assert torch.equal(X, X2) and torch.equal(Yt, Yt2)
    h_after = B.sweep(2)
    B2 = G.Batch(wb, meth)
    B2.sweep(1)
    h_ref = B2.sweep(2)
    # tiles change only how rows are grouped into work items, not any result
    np.testing.assert_array_equal(h_after, h_ref)


def test_batch_validation(G):
    wb = small_batch(count=4)
    meth = methods_of(wb, G)
    # the split of the entries between instances 1 and 2 is off by one (the
    # total stays the same, so every copy stays inside the caller's arrays)
    bad = W.Batch(**{f: getattr(wb, f) for f in wb.__dataclass_fields__})
    bad.nnz = wb.nnz.copy()
    bad.nnz[1] -= 1
    bad.nnz[2] += 1
    with pytest.raises(G.GLRMError) as e:
        G.Batch(bad, meth)
    assert e.value.code in (G.GLRM_ERR_OMEGA, G.GLRM_ERR_ARG)
    bad2 = W.Batch(**{f: getattr(wb, f) for f in wb.__dataclass_fields__})
    bad2.colidx = wb.colidx.clone()
    bad2.colidx[3] = 10**6
    with pytest.raises(G.GLRMError) as e:
        G.Batch(bad2, meth)
    assert e.value.code == G.GLRM_ERR_OMEGA


def test_wait_limit_expiry_returns_timeout(G, oracle_mod):
    """The one-launch queue: with a wait limit of 0 polls, an item whose
    dependencies are not complete when it is taken gives up at once.  The
    Y-step items are handed out while the X-step items of their instances
    still run (the GPU holds thousands of warps and the batch a few hundred
    items), so the call returns GLRM_ERR_TIMEOUT, and does not hang.  With the
    default limit, batches fit normally and the graph and stream modes agree
    bit for bit."""
    wb = small_batch(count=64, m_range=(50, 400))
    meth = methods_of(wb, G)
    B = G.Batch(wb, meth)
    B.set_wait_limit(0)
    timed_out = False
    for _ in range(5):
        B.set_factors(wb.X0, wb.Yt0)
        try:
            B.sweep(3, mode=G.GLRM_BATCH_STREAM)
        except G.GLRMError as e:
            assert e.code == G.GLRM_ERR_TIMEOUT, e
            timed_out = True
            break
    assert timed_out
    B.close()
    B1 = G.Batch(wb, meth)
    B1.set_wait_limit(1 << 24)
    h1 = B1.sweep(3, mode=G.GLRM_BATCH_GRAPH)
    B2 = G.Batch(wb, meth)
    h2 = B2.sweep(3, mode=G.GLRM_BATCH_STREAM)
    np.testing.assert_array_equal(h1, h2)
    assert np.isfinite(h1).all()
