"""Omega from its CSR arrays alone (glrm_set_observed_csr[_host]): the CSC
orientation built on the device must be the one the caller would have
given, so a handle set up that way sweeps bitwise like one given both
orientations (same step sizes, same objective history), on the sparse
paths, the dense form of a sparse table and tables whose count table needs
row blocks of several rows; malformed CSR arrays are rejected as before."""
import numpy as np
import pytest
import torch

from paper_1410_0342_gb300 import workloads as W

from gpu_parity import subset_table

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def G():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1410_0342_gb300 import build
    build.build()
    from paper_1410_0342_gb300 import glrm
    return glrm


def _twins(G, t, prec, host, paths=None):
    a = G.GLRM.from_table(t, precision=prec)
    b = G.GLRM(t.m, t.n, t.k, (t.loss_kind, t.loss_param, t.loss_levels), t.rx, t.ry, prec)
    dt = np.float64 if prec == G.GLRM_FP64 else np.float32
    arrs = [np.ascontiguousarray(np.asarray(t.rowptr), np.int32), np.ascontiguousarray(t.colidx, np.int32),
            np.ascontiguousarray(t.val, dt)]
    if host:
        G.glrm_set_observed_csr_host(b.h, t.nnz, *arrs)
    else:
        G.glrm_set_observed_csr(b.h, t.nnz, *[torch.as_tensor(x, device="cuda") for x in arrs])
    b.set_factors(torch.as_tensor(t.X0, dtype=b.dtype, device="cuda"),
                  torch.as_tensor(t.Yt0, dtype=b.dtype, device="cuda"))
    if paths:
        G.glrm_set_path(a.h, *paths)
        G.glrm_set_path(b.h, *paths)
    assert tuple(G.glrm_get_path(a.h)) == tuple(G.glrm_get_path(b.h))
    return a, b


@pytest.mark.parametrize("prec,host,paths", [(1, True, None), (1, False, (1, 1)), (0, True, None),
                                             (1, False, (4, 4)), (1, True, (2, 3))])
def test_csr_only_sweeps_bitwise(G, prec, host, paths):
    t = W.small_mixed(m=1500, n=130, k=8, p_obs=0.5, seed=901, nkinds=7)
    rows = t.rows()
    t = subset_table(t, ~((rows == 7) | (t.colidx == 3)))  # an empty row and an empty column
    a, b = _twins(G, t, prec, host, paths)
    ha, hb = a.sweep(6), b.sweep(6)
    np.testing.assert_array_equal(ha, hb)
    Xa, Ya = a.factors()
    Xb, Yb = b.factors()
    assert torch.equal(Xa, Xb) and torch.equal(Ya, Yb)


def test_csr_only_dense_form_and_row_blocks(G):
    """The benchmark recipe at 20,000 rows (dense form, count table in row
    blocks of one row) and a completion table of 100,000 x 20,000 (row blocks
    of 30 rows)."""
    t = W.mixed(m=20000)
    a, b = _twins(G, t, 1, True)
    np.testing.assert_array_equal(a.sweep(3), b.sweep(3))
    tc = W.completion(m=100_000, k=16)
    a, b = _twins(G, tc, 1, False)
    np.testing.assert_array_equal(a.sweep(2), b.sweep(2))


@pytest.mark.parametrize("table,host", [("small", True), ("small", False), ("mixed20k", True)])
def test_csr_only_dense_form_csc(G, table, host):
    """On the dense form the CSC entries are read from the dense table's
    tiles; the dense sweeps never read them, so they are checked through what
    does: the column statistics and sweeps on the sparse paths after a path
    switch, bitwise against a handle given both orientations (ragged rows and
    columns, an empty row and an empty column; the 20,000-row table comes
    over from the host in two pieces, its dense table scattered per piece)."""
    if table == "small":
        t = W.small_mixed(m=3001, n=301, k=8, p_obs=0.6, seed=903, nkinds=7)
        rows = t.rows()
        t = subset_table(t, ~((rows == 11) | (t.colidx == 300)))
    else:
        t = W.mixed(m=20000)
    a, b = _twins(G, t, 1, host)
    assert tuple(G.glrm_get_path(b.h)) == (G.GLRM_PATH_DENSE, G.GLRM_PATH_DENSE)
    np.testing.assert_array_equal(a.sweep(2), b.sweep(2))
    for x, y in zip(a.column_stats(), b.column_stats()):
        assert torch.equal(x.nan_to_num(-7.0), y.nan_to_num(-7.0))
    for paths in ((1, 1), (2, 3)):
        G.glrm_set_path(a.h, *paths)
        G.glrm_set_path(b.h, *paths)
        np.testing.assert_array_equal(a.sweep(2), b.sweep(2))
    Xa, Ya = a.factors()
    Xb, Yb = b.factors()
    assert torch.equal(Xa, Xb) and torch.equal(Ya, Yb)


def test_csr_only_wide_tables(G):
    """Column counts beyond what shared memory holds (n = 50,000: the count and
    scatter passes on global counters) and a host-piped build of a table whose
    counters take the opt-in shared memory (n = 20,000) with a ragged last row
    block."""
    tw = W.completion(m=3000, n=50_000, k=8, per_row=40)
    a, b = _twins(G, tw, 1, True)
    np.testing.assert_array_equal(a.sweep(2), b.sweep(2))
    tc = W.completion(m=70_001, n=20_000, k=8, per_row=30)
    a, b = _twins(G, tc, 1, True)
    np.testing.assert_array_equal(a.sweep(2), b.sweep(2))


def test_csr_only_rejects_bad_arrays(G):
    t = W.small_mixed(m=200, n=40, k=4, seed=902)
    b = G.GLRM(t.m, t.n, t.k, (t.loss_kind, t.loss_param, t.loss_levels), t.rx, t.ry, G.GLRM_FP32)
    rp = np.ascontiguousarray(np.asarray(t.rowptr), np.int32)
    ci = np.ascontiguousarray(t.colidx, np.int32)
    v = np.ascontiguousarray(t.val, np.float32)
    bad = ci.copy()
    bad[0], bad[1] = bad[1], bad[0]  # columns of row 0 out of order
    with pytest.raises(G.GLRMError) as ei:
        G.glrm_set_observed_csr_host(b.h, t.nnz, rp, bad, v)
    assert ei.value.code == G.GLRM_ERR_OMEGA
    bad = ci.copy()
    bad[5] = t.n
    with pytest.raises(G.GLRMError):
        G.glrm_set_observed_csr_host(b.h, t.nnz, rp, bad, v)
    vb = v.copy()
    vb[3] = np.nan
    with pytest.raises(G.GLRMError):
        G.glrm_set_observed_csr_host(b.h, t.nnz, rp, ci, vb)
    G.glrm_set_observed_csr_host(b.h, t.nnz, rp, ci, v)  # and a good set afterwards
    b.sweep(1)
