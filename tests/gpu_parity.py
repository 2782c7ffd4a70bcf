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


def oracle_problem(o, t, rx=None, ry=None, offset=False, col_scale=None):
    return o.Problem.from_csr(t.m, t.n, t.k, t.rowptr, t.colidx, t.val, loss_kind=t.loss_kind,
                              loss_param=t.loss_param, loss_levels=t.loss_levels,
                              rx=rx or t.rx, ry=ry or t.ry, offset=offset, col_scale=col_scale)


def _flipped(got, want, tol=1e-4):
    """Rows of got that differ from want by more than tol of the row's scale
    (an accept / reject decision taken the other way, or its consequence)."""
    scale = np.maximum(np.abs(want).max(axis=1), 1e-3)
    return (np.abs(np.asarray(got, np.float64) - want).max(axis=1) / scale) > tol


def synced_sweeps(g, o, t, nsweeps, rtol=1e-5, max_flip_frac=0.01, offset=False, col_scale=None, problem=None):
    """Run nsweeps GPU sweeps; before each, hand the GPU state to the oracle
    and run the same sweep there.  Checks per sweep: objective within rtol,
    accepted row / column counts within max(2, max_flip_frac) of each other,
    X and Yt after the sweep equal (to 1e-4 of each row's scale) and both
    step-size arrays equal (to FP32 rounding, 1e-6) on all but the rows /
    columns whose decision flipped.  Returns the per-sweep relative objective
    differences.  offset / col_scale: the oracle's model of a handle with
    glrm_set_offset / glrm_set_column_scale.  problem: an oracle problem to
    use instead (a FeatureProblem for a model of an embedded feature table);
    the sizes are the handle's."""
    p = problem if problem is not None else oracle_problem(o, t, offset=offset, col_scale=col_scale)
    m, n, k = g.m, g.n, g.k
    rels = []
    for _ in range(nsweeps):
        X, Yt, ax, ay, _ = decode_state(g.state(), m, n, k)
        h = g.sweep(1)[0]
        acc = g.accepts()
        Xo, Yo, axo, ayo, oh, oacc = p.proxgrad(X.astype(np.float64), Yt.astype(np.float64), 1,
                                                ax.astype(np.float64), ay.astype(np.float64))
        rel = abs(h - oh[0]) / abs(oh[0])
        rels.append(rel)
        assert rel < rtol, (rel, h, oh[0])
        for a, b, cnt in ((acc[0], oacc[0, 0], m), (acc[1], oacc[0, 1], n)):
            assert abs(int(a) - int(b)) <= max(2, int(max_flip_frac * cnt)), (acc, oacc)
        Xg, Yg, axg, ayg, _ = decode_state(g.state(), m, n, k)
        for F, Fo, a, ao, cnt, what in ((Xg, Xo, axg, axo, m, "X"), (Yg, Yo, ayg, ayo, n, "Yt")):
            bad = _flipped(F, Fo)
            sbad = np.abs(np.asarray(a, np.float64) - ao) > 1e-6 * np.abs(ao)
            allowed = max(2, int(max_flip_frac * cnt))
            assert bad.sum() <= allowed, (what, bad.sum(), allowed)
            assert sbad.sum() <= allowed, (what + " steps", sbad.sum(), allowed)
    return np.array(rels)


# Rounding bound of a product x_i . y_j relative to sum_c |x_ic y_jc|: an FP32
# dot product of k <= 64 terms (k 2^-24 <= 2^-18); the BF16 form's products
# of two BF16-rounded rows (2^-9 each, with margin).
U_REL_FP32 = 2.0 ** -18
U_REL_BF16 = 2.0 ** -7


def grad_bounds(p, X, Yt, u_rel=U_REL_FP32):
    """(SX, SYt, VX, VYt): per gradient coordinate the absolute sum of its
    terms and the variation of its terms when every product is off by its
    rounding bound (oracle gradient_abs, gradient_variation)."""
    SX, SY = p.gradient_abs(X, Yt)
    VX, VY = p.gradient_variation(X, Yt, u_rel)
    return SX, SY, VX, VY


def assert_grad_close(got, want, scale, slack=0.0, rtol=1e-5, srel=16 * 2.0 ** -24,
                      what="gradient"):
    """Element by element: |got - want| <= rtol |want| + srel scale + slack.
    scale is the sum of the magnitudes of the coordinate's terms (oracle
    gradient_abs), and srel scale the rounding bound of an FP32 summation of
    them (16 units of 2^-24 of their absolute sum), needed where the terms
    cancel.  slack (oracle gradient_variation) covers the products' own
    rounding: a product within its rounding bound of a kink of the loss may
    take either one-sided derivative, a smooth loss's derivative moves by
    about 2 L'' times that bound.  A coordinate without terms (an empty row or
    column) must match exactly."""
    got = np.asarray(got, np.float64)
    want = np.asarray(want, np.float64)
    err = np.abs(got - want)
    bound = rtol * np.abs(want) + srel * np.asarray(scale, np.float64) + np.asarray(slack, np.float64)
    bad = err > bound
    if bad.any():
        q = np.unravel_index(np.argmax(err - bound), err.shape)
        raise AssertionError(f"{what}: {int(bad.sum())} of {bad.size} values beyond the bound; "
                             f"worst at {q}: got {got[q]!r}, want {want[q]!r}, bound {bound[q]:.3g}")


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
