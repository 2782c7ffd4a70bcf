"""Helpers shared by the GPU parity tests (not a test module).

The FP32 sweep and the FP64 oracle take the same accept / reject decisions
except at near-ties, where rounding can flip one (a step whose row objective
barely changes).  A flip swaps two almost equal objectives but sends the two
trajectories apart afterwards, so FP32 parity is checked one sweep at a time
from a shared state: the oracle restarts every sweep from the GPU's factors
and step sizes, and the objectives after that sweep must agree."""
import struct

import numpy as np

from paper_1410_0342_gb300 import workloads as W


def decode_state(buf: bytes, m: int, n: int, k: int, dtype=np.float32):
    """(X, Yt, alpha_x, alpha_y, sweeps) from a glrm_get_state buffer."""
    hdr = struct.unpack("<8q", buf[:64])
    assert hdr[2] == m and hdr[3] == n and hdr[4] == k
    es = np.dtype(dtype).itemsize
    off = 64
    X = np.frombuffer(buf, dtype, m * k, off).reshape(m, k)
    off += m * k * es
    Yt = np.frombuffer(buf, dtype, n * k, off).reshape(n, k)
    off += n * k * es
    ax = np.frombuffer(buf, dtype, m, off)
    off += m * es
    ay = np.frombuffer(buf, dtype, n, off)
    return X, Yt, ax, ay, hdr[6]


def oracle_problem(o, t, rx=None, ry=None):
    return o.Problem.from_csr(t.m, t.n, t.k, t.rowptr, t.colidx, t.val, loss_kind=t.loss_kind,
                              loss_param=t.loss_param, loss_levels=t.loss_levels,
                              rx=rx or t.rx, ry=ry or t.ry)


def synced_sweeps(g, o, t, nsweeps, rtol=1e-5, max_flip_frac=0.01):
    """Run nsweeps GPU sweeps; before each, hand the GPU state to the oracle
    and run the same sweep there.  Checks per sweep: objective within rtol,
    accepted row / column counts within max(2, max_flip_frac) of each other,
    X after the sweep equal (to FP32 accuracy) on all but the flipped rows.
    Returns the per-sweep relative objective differences."""
    p = oracle_problem(o, t)
    rels = []
    for _ in range(nsweeps):
        X, Yt, ax, ay, _ = decode_state(g.state(), t.m, t.n, t.k)
        h = g.sweep(1)[0]
        acc = g.accepts()
        Xo, Yo, _, _, oh, oacc = p.proxgrad(X.astype(np.float64), Yt.astype(np.float64), 1,
                                            ax.astype(np.float64), ay.astype(np.float64))
        rel = abs(h - oh[0]) / abs(oh[0])
        rels.append(rel)
        assert rel < rtol, (rel, h, oh[0])
        for a, b, cnt in ((acc[0], oacc[0, 0], t.m), (acc[1], oacc[0, 1], t.n)):
            assert abs(int(a) - int(b)) <= max(2, int(max_flip_frac * cnt)), (acc, oacc)
        Xg, _, _, _, _ = decode_state(g.state(), t.m, t.n, t.k)
        scale = np.maximum(np.abs(Xo).max(axis=1), 1e-3)
        bad = (np.abs(Xg - Xo).max(axis=1) / scale) > 1e-4
        assert bad.mean() <= max_flip_frac + 2.0 / len(bad), bad.sum()
    return np.array(rels)


def subset_table(t, keep):
    """The table restricted to the entries where keep (a CSR-order mask) is set."""
    rows = t.rows()[keep]
    cols = t.colidx[keep]
    vals = t.val[keep]
    rowptr = np.zeros(t.m + 1, np.int64)
    np.cumsum(np.bincount(rows, minlength=t.m), out=rowptr[1:])
    colptr, rowidx, cval = W.csc_from_csr(t.m, t.n, rowptr, cols, vals)
    return W.Table(t.name, t.m, t.n, t.k, rowptr, cols, vals, colptr, rowidx, cval,
                   t.loss_kind, t.loss_param, t.loss_levels, t.rx, t.ry, t.X0, t.Yt0)
