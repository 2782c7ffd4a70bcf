"""The device-side convergence test (glrm_sweep_until): the sweeps it runs
are the sweeps of glrm_sweep, and it stops at the first sweep whose FP64
objective meets the test, both for a relative decrease and for the distance
to a reference objective (the qPCA closed form, Appendix A)."""
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


def first_rel_decrease(F0, hist, rtol, w):
    """First sweep t >= w with F_{t-w} - F_t <= w rtol |F_t| (F_0 = F0)."""
    F = np.concatenate([[F0], hist])
    for t in range(w, len(F)):
        if F[t - w] - F[t] <= w * rtol * abs(F[t]):
            return t
    return None


@pytest.mark.parametrize("prec,window", [("fp32", 1), ("fp64", 1), ("bf16", 1), ("fp32", 5)])
def test_relative_decrease_stop(G, prec, window):
    t = W.small_mixed(m=3000, n=120, k=8, p_obs=0.5, seed=17, rx=(1, 0.1), ry=(2, 0.02))
    P = {"fp32": G.GLRM_FP32, "fp64": G.GLRM_FP64, "bf16": G.GLRM_BF16}[prec]
    ref = G.GLRM.from_table(t, precision=P)
    F0 = ref.objective()
    hist_ref = ref.sweep(400)
    rtol = 1e-4
    want = first_rel_decrease(F0, hist_ref, rtol, window)
    assert want is not None and want > 3
    g = G.GLRM.from_table(t, precision=P)
    h = g.sweep_until(400, rtol, window=window)
    assert len(h) == want
    np.testing.assert_array_equal(h, hist_ref[:want])
    # a second call continues the same fit (the captured graph is replayed);
    # an unreachable reference objective lets the sweep limit stop it
    h2 = g.sweep_until(5, 0.0, -1e300)
    np.testing.assert_array_equal(h2, hist_ref[want:want + 5])


def test_reference_objective_stop_qpca(G):
    """FP64 qPCA table: sweep until within 1e-6 of the closed-form optimum
    ||A||^2 - sum_{i<=k} ((s_i - gamma)_+)^2."""
    t = W.qpca_dense()
    A = t.val.reshape(t.m, t.n)
    s = np.linalg.svd(A, compute_uv=False)
    fstar = float(np.sum(A * A) - np.sum(np.maximum(s[:t.k] - 0.1, 0) ** 2))
    g = G.GLRM.from_table(t, precision=G.GLRM_FP64)
    h = g.sweep_until(5000, 1e-6, fstar)
    assert (h[-1] - fstar) / fstar <= 1e-6
    assert len(h) < 5000 and (h[-2] - fstar) / fstar > 1e-6
    ref = G.GLRM.from_table(t, precision=G.GLRM_FP64)
    np.testing.assert_array_equal(ref.sweep(len(h)), h)


def test_sweep_limit_and_arguments(G):
    t = W.small_mixed(m=500, n=60, k=6, seed=18, rx=(1, 0.1), ry=(1, 0.1))
    g = G.GLRM.from_table(t)
    assert len(g.sweep_until(7, 0.0, -1e300)) == 7   # an unreachable reference: the limit stops it
    for bad in ((0, 1e-4, 1), (5, -1.0, 1), (5, 1e-4, 0)):
        with pytest.raises(G.GLRMError) as e:
            g.sweep_until(bad[0], bad[1], window=bad[2])
        assert e.value.code == G.GLRM_ERR_ARG
