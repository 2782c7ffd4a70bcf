"""Seeded synthetic GLRM workloads.

This module only draws data: latent factors, observed sets, table values and
initial factors.  It holds none of the fitting method's arithmetic and is the
one piece of code that both the CUDA library's tests and the FP64 oracle's
tests use, so that both sides see identical inputs.

The shapes follow the paper's synthetic experiments (Udell et al., "Generalized
Low Rank Models"): Gaussian low-rank tables with noise (Sec. 6.1 mixed data,
Sec. 7.3 qPCA convergence), entries observed uniformly at random, Boolean data
as signs of a noisy low-rank matrix (Sec. 6.1), and Spark's random sparse
matrices with a fixed count of nonzeros per row (Sec. 9.3), scaled up.

Every table is returned as ``Table``: Omega in CSR (rowptr, colidx, val) and
CSC (colptr, rowidx, val) int32/float32 form plus per-column loss kinds,
parameters and level counts, the regularisers and the initial factors.
"""
from __future__ import annotations

import dataclasses

import numpy as np

LOSS_QUAD, LOSS_HUBER, LOSS_HINGE, LOSS_LOGISTIC, LOSS_ORDINAL = 0, 1, 2, 3, 4
LOSS_L1, LOSS_QUANTILE = 5, 6
REG_ZERO, REG_QUAD, REG_L1, REG_NONNEG = 0, 1, 2, 3

BASE_SEED = 1410034200


@dataclasses.dataclass
class Table:
    name: str
    m: int
    n: int
    k: int
    rowptr: np.ndarray      # int64 [m+1]
    colidx: np.ndarray      # int32 [nnz]
    val: np.ndarray         # float64 [nnz], CSR order
    colptr: np.ndarray      # int64 [n+1]
    rowidx: np.ndarray      # int32 [nnz]
    cval: np.ndarray        # float64 [nnz], CSC order
    loss_kind: np.ndarray   # int32 [n]
    loss_param: np.ndarray  # float64 [n]
    loss_levels: np.ndarray  # int32 [n]
    rx: tuple
    ry: tuple
    X0: np.ndarray          # float64 [m, k] initial X
    Yt0: np.ndarray         # float64 [n, k] initial Y^T

    @property
    def nnz(self) -> int:
        return int(self.colidx.size)

    def rows(self) -> np.ndarray:
        """Row index of every entry in CSR order."""
        return np.repeat(np.arange(self.m, dtype=np.int32), np.diff(self.rowptr))


def rng_for(seed: int) -> np.random.Generator:
    return np.random.Generator(np.random.PCG64(seed))


def csc_from_csr(m, n, rowptr, colidx, val):
    """Reorder CSR entries by column (stable, so rows stay ascending)."""
    order = np.argsort(colidx, kind="stable")
    rows = np.repeat(np.arange(m, dtype=np.int32), np.diff(rowptr))
    colptr = np.zeros(n + 1, dtype=np.int64)
    np.cumsum(np.bincount(colidx, minlength=n), out=colptr[1:])
    return colptr, rows[order].astype(np.int32), val[order]


def omega_bernoulli(m: int, n: int, p: float, rng: np.random.Generator, block: int = 4096):
    """Each cell observed independently with probability p; CSR with sorted columns."""
    counts = np.empty(m, dtype=np.int64)
    cols = []
    for r0 in range(0, m, block):
        r1 = min(m, r0 + block)
        mask = rng.random((r1 - r0, n)) < p
        counts[r0:r1] = mask.sum(axis=1)
        cols.append(np.nonzero(mask)[1].astype(np.int32))
    rowptr = np.zeros(m + 1, dtype=np.int64)
    np.cumsum(counts, out=rowptr[1:])
    colidx = np.concatenate(cols) if cols else np.zeros(0, dtype=np.int32)
    return rowptr, colidx


def omega_fixed_per_row(m: int, n: int, r: int, rng: np.random.Generator, block: int = 65536):
    """Exactly r distinct columns per row, each r-subset equally likely:
    draw columns with replacement, keep the first r distinct in draw order."""
    assert r <= n
    draw = r + max(16, int(3 * np.sqrt(r * r * r / max(n, 1))) + 8)
    rowptr = np.arange(m + 1, dtype=np.int64) * r
    colidx = np.empty(m * r, dtype=np.int32)
    for r0 in range(0, m, block):
        r1 = min(m, r0 + block)
        rows = r1 - r0
        out = np.empty((rows, r), dtype=np.int32)
        todo = np.arange(rows)
        while todo.size:
            d = rng.integers(0, n, size=(todo.size, draw), dtype=np.int64)
            order = np.argsort(d, axis=1, kind="stable")
            sd = np.take_along_axis(d, order, axis=1)
            dup_sorted = np.zeros_like(sd, dtype=bool)
            dup_sorted[:, 1:] = sd[:, 1:] == sd[:, :-1]
            dup = np.empty_like(dup_sorted)
            np.put_along_axis(dup, order, dup_sorted, axis=1)
            keep = ~dup
            ok = keep.sum(axis=1) >= r
            good = todo[ok]
            if good.size:
                kk = keep[ok]
                pos = np.cumsum(kk, axis=1)
                sel = kk & (pos <= r)
                vals = d[ok][sel].reshape(good.size, r)
                out[good] = np.sort(vals, axis=1).astype(np.int32)
            todo = todo[~ok]
        colidx[r0 * r:r1 * r] = out.reshape(-1)
    return rowptr, colidx


def sampled_products(X0: np.ndarray, Y0t: np.ndarray, rowptr, colidx, chunk: int = 1 << 22):
    """(X0 Y0)_ij for the observed entries in CSR order, to synthesise data."""
    m = X0.shape[0]
    rows = np.repeat(np.arange(m, dtype=np.int64), np.diff(rowptr))
    out = np.empty(colidx.size, dtype=np.float64)
    for e0 in range(0, colidx.size, chunk):
        e1 = min(colidx.size, e0 + chunk)
        out[e0:e1] = np.einsum("ek,ek->e", X0[rows[e0:e1]], Y0t[colidx[e0:e1]])
    return out


def _finish(name, m, n, k, rowptr, colidx, val, kind, param, levels, rx, ry, rng, init_std=1.0):
    colptr, rowidx, cval = csc_from_csr(m, n, rowptr, colidx, val)
    X0 = rng.standard_normal((m, k)) * init_std
    Yt0 = rng.standard_normal((n, k)) * init_std
    return Table(name, m, n, k, rowptr, colidx.astype(np.int32), val.astype(np.float64),
                 colptr, rowidx, cval.astype(np.float64),
                 np.asarray(kind, dtype=np.int32), np.asarray(param, dtype=np.float64),
                 np.asarray(levels, dtype=np.int32), rx, ry, X0, Yt0)


# --------------------------------------------------------------- the tables

def qpca_dense(m=200, n=100, k=5, gamma=0.1, noise=0.1, seed=BASE_SEED + 1, name="qpca_dense"):
    """Fully observed A = X0 Y0 + N(0, noise^2), quadratic loss, gamma||.||^2
    on both factors (the paper's qPCA experiment shape, Sec. 7.3)."""
    rng = rng_for(seed)
    X0 = rng.standard_normal((m, k))
    Y0 = rng.standard_normal((k, n))
    A = X0 @ Y0 + noise * rng.standard_normal((m, n))
    rowptr = np.arange(m + 1, dtype=np.int64) * n
    colidx = np.tile(np.arange(n, dtype=np.int32), m)
    return _finish(name, m, n, k, rowptr, colidx, A.reshape(-1),
                   np.full(n, LOSS_QUAD), np.zeros(n), np.zeros(n),
                   (REG_QUAD, gamma), (REG_QUAD, gamma), rng)


def mixed(m=100_000, n=1000, k=20, n_real=500, n_bool=300, levels=7, p_obs=0.6,
          seed=BASE_SEED + 2, name="mixed", lam=0.01):
    """Mixed-type table (Sec. 6.1 shape, scaled up): real columns with Huber
    loss (Laplace(0, 0.5) noise, 1% of entries with noise x20), Boolean columns
    sign(X0 Y0 + N(0, 0.5^2)) with hinge loss, ordinal columns binned at the
    column's empirical septiles with the ordinal hinge; cells observed with
    probability p_obs; l1 (lambda) on X, nonnegativity on Y."""
    rng = rng_for(seed)
    n_ord = n - n_real - n_bool
    assert n_ord >= 0
    X0 = rng.standard_normal((m, k))
    Y0t = rng.standard_normal((n, k))
    rowptr, colidx = omega_bernoulli(m, n, p_obs, rng)
    u = sampled_products(X0, Y0t, rowptr, colidx)
    val = np.empty_like(u)
    real = colidx < n_real
    boo = (colidx >= n_real) & (colidx < n_real + n_bool)
    ordi = colidx >= n_real + n_bool
    nr = int(real.sum())
    noise = rng.laplace(0.0, 0.5, size=nr)
    outl = rng.random(nr) < 0.01
    noise[outl] *= 20.0
    val[real] = u[real] + noise
    z = u[boo] + 0.5 * rng.standard_normal(int(boo.sum()))
    val[boo] = np.where(z >= 0.0, 1.0, -1.0)
    if n_ord:
        # septile edges of each ordinal column of X0 Y0 over all m rows
        ocols = np.arange(n_real + n_bool, n)
        edges = np.empty((n_ord, levels - 1))
        qs = np.arange(1, levels) / levels
        for c0 in range(0, n_ord, 64):
            c1 = min(n_ord, c0 + 64)
            full = X0 @ Y0t[ocols[c0:c1]].T
            edges[c0:c1] = np.quantile(full, qs, axis=0).T
        oc = colidx[ordi] - (n_real + n_bool)
        uo = u[ordi]
        lev = np.ones(uo.size)
        for q in range(levels - 1):
            lev += uo > edges[oc, q]
        val[ordi] = lev
    kind = np.concatenate([np.full(n_real, LOSS_HUBER), np.full(n_bool, LOSS_HINGE),
                           np.full(n_ord, LOSS_ORDINAL)])
    param = np.concatenate([np.full(n_real, 1.0), np.zeros(n_bool), np.zeros(n_ord)])
    lv = np.concatenate([np.zeros(n_real), np.zeros(n_bool), np.full(n_ord, levels)])
    return _finish(name, m, n, k, rowptr, colidx, val, kind, param, lv,
                   (REG_L1, lam), (REG_NONNEG, 0.0), rng)


def completion(m=1_000_000, n=20_000, k=64, per_row=200, gamma=0.05, noise=0.1,
               seed=BASE_SEED + 3, name="completion"):
    """Matrix completion: exactly per_row uniform columns per row,
    A = X0 Y0 + N(0, noise^2) with X0, Y0 entries of variance 1/sqrt(k),
    quadratic loss, gamma||.||^2 on both factors."""
    rng = rng_for(seed)
    sd = k ** -0.25
    X0 = rng.standard_normal((m, k)) * sd
    Y0t = rng.standard_normal((n, k)) * sd
    rowptr, colidx = omega_fixed_per_row(m, n, per_row, rng)
    val = sampled_products(X0, Y0t, rowptr, colidx) + noise * rng.standard_normal(colidx.size)
    return _finish(name, m, n, k, rowptr, colidx, val, np.full(n, LOSS_QUAD), np.zeros(n),
                   np.zeros(n), (REG_QUAD, gamma), (REG_QUAD, gamma), rng, init_std=sd)


def logistic_bool(m=50_000, n=2000, k=32, p_obs=0.8, gamma=0.1, seed=BASE_SEED + 4,
                  name="logistic"):
    """Boolean table A_ij = +1 with probability sigma(x0_i . y0_j), else -1;
    cells observed with probability p_obs; logistic loss, gamma||.||^2."""
    rng = rng_for(seed)
    X0 = rng.standard_normal((m, k))
    Y0t = rng.standard_normal((n, k))
    rowptr, colidx = omega_bernoulli(m, n, p_obs, rng)
    u = sampled_products(X0, Y0t, rowptr, colidx)
    prob = 1.0 / (1.0 + np.exp(-u))
    val = np.where(rng.random(u.size) < prob, 1.0, -1.0)
    return _finish(name, m, n, k, rowptr, colidx, val, np.full(n, LOSS_LOGISTIC), np.zeros(n),
                   np.zeros(n), (REG_QUAD, gamma), (REG_QUAD, gamma), rng)


def batch_instance(s: int, seed=BASE_SEED + 5, m_range=(50, 5000), n_range=(20, 500),
                   ks=(4, 8, 16), p_obs=0.7, gamma=0.1, noise=0.2):
    """Instance s of the batched workload: m, n uniform in their ranges, k
    uniform over ks; even s quadratic loss, odd s Huber (delta = 1); A =
    X0 Y0 + N(0, noise^2); cells observed with probability p_obs."""
    rng = rng_for(seed + s)
    m = int(rng.integers(m_range[0], m_range[1] + 1))
    n = int(rng.integers(n_range[0], n_range[1] + 1))
    k = int(ks[int(rng.integers(0, len(ks)))])
    X0 = rng.standard_normal((m, k))
    Y0t = rng.standard_normal((n, k))
    rowptr, colidx = omega_bernoulli(m, n, p_obs, rng)
    val = sampled_products(X0, Y0t, rowptr, colidx) + noise * rng.standard_normal(colidx.size)
    kind = LOSS_QUAD if s % 2 == 0 else LOSS_HUBER
    return _finish(f"batch{s}", m, n, k, rowptr, colidx, val, np.full(n, kind),
                   np.full(n, 1.0 if kind == LOSS_HUBER else 0.0), np.zeros(n),
                   (REG_QUAD, gamma), (REG_QUAD, gamma), rng)


def small_mixed(m=97, n=41, k=6, p_obs=0.55, seed=BASE_SEED + 20, rx=(REG_L1, 0.05),
                ry=(REG_NONNEG, 0.0), levels=5, nkinds=5, alpha=0.3):
    """A small mixed table for parity on ragged shapes: column j takes loss
    kind j mod nkinds (5: quadratic, Huber, hinge, logistic, ordinal hinge;
    7: also l1 and the quantile loss with the given alpha)."""
    rng = rng_for(seed)
    X0 = rng.standard_normal((m, k))
    Y0t = rng.standard_normal((n, k))
    rowptr, colidx = omega_bernoulli(m, n, p_obs, rng)
    u = sampled_products(X0, Y0t, rowptr, colidx)
    kinds = np.arange(n) % nkinds
    val = np.empty_like(u)
    ke = kinds[colidx]
    val[ke == LOSS_QUAD] = u[ke == LOSS_QUAD] + 0.1 * rng.standard_normal(int((ke == 0).sum()))
    sel = ke == LOSS_HUBER
    val[sel] = u[sel] + rng.laplace(0.0, 0.5, int(sel.sum()))
    for kk in (LOSS_HINGE, LOSS_LOGISTIC):
        sel = ke == kk
        val[sel] = np.where(u[sel] + 0.5 * rng.standard_normal(int(sel.sum())) >= 0, 1.0, -1.0)
    sel = ke == LOSS_ORDINAL
    val[sel] = np.clip(np.round(u[sel] / 2.0 + (levels + 1) / 2.0), 1, levels)
    for kk in (LOSS_L1, LOSS_QUANTILE):
        sel = ke == kk
        val[sel] = u[sel] + rng.laplace(0.0, 0.5, int(sel.sum()))
    param = np.where(kinds == LOSS_HUBER, 1.0, np.where(kinds == LOSS_QUANTILE, alpha, 0.0))
    lv = np.where(kinds == LOSS_ORDINAL, levels, 0)
    return _finish("small_mixed", m, n, k, rowptr, colidx, val, kinds, param, lv, rx, ry, rng)


# ------------------------------------------------------------- dense tables

@dataclasses.dataclass
class DenseTable:
    """A fully observed table: A (m x n, row-major float32), column losses,
    regularisers and the initial factors."""
    name: str
    m: int
    n: int
    k: int
    A: np.ndarray           # float32 [m, n]
    loss_kind: np.ndarray   # int32 [n]
    loss_param: np.ndarray  # float64 [n]
    loss_levels: np.ndarray  # int32 [n]
    rx: tuple
    ry: tuple
    X0: np.ndarray          # float64 [m, k]
    Yt0: np.ndarray         # float64 [n, k]

    def observed(self) -> Table:
        """The same data as an observed set with every entry present (CSR and
        CSC); for the oracle on small tables."""
        rowptr = np.arange(self.m + 1, dtype=np.int64) * self.n
        colidx = np.tile(np.arange(self.n, dtype=np.int32), self.m)
        val = self.A.astype(np.float64).reshape(-1)
        colptr, rowidx, cval = csc_from_csr(self.m, self.n, rowptr, colidx, val)
        return Table(self.name, self.m, self.n, self.k, rowptr, colidx, val, colptr, rowidx, cval,
                     self.loss_kind, self.loss_param, self.loss_levels, self.rx, self.ry,
                     self.X0, self.Yt0)


def mixed_dense(m=100_000, n=1000, k=20, n_real=500, n_bool=300, levels=7, seed=BASE_SEED + 6,
                name="mixed_dense", lam=0.01, block=8192, rx=None, ry=None):
    """The mixed-type table's recipe with every cell observed: Huber columns
    (Laplace(0, 0.5) noise, 1% of entries x20), hinge columns
    sign(X0 Y0 + N(0, 0.5^2)), ordinal columns binned at the column's
    empirical septiles of X0 Y0 (estimated on the first 20,000 rows); l1
    (lambda) on X, nonnegativity on Y unless rx / ry say otherwise.  Generated
    in row blocks."""
    rng = rng_for(seed)
    n_ord = n - n_real - n_bool
    assert n_ord >= 0
    X0 = rng.standard_normal((m, k))
    Y0t = rng.standard_normal((n, k))
    ocols = np.arange(n_real + n_bool, n)
    qs = np.arange(1, levels) / levels
    sample = X0[:min(m, 20000)] @ Y0t[ocols].T
    edges = np.quantile(sample, qs, axis=0).T if n_ord else np.zeros((0, levels - 1))
    A = np.empty((m, n), dtype=np.float32)
    for r0 in range(0, m, block):
        r1 = min(m, r0 + block)
        u = X0[r0:r1] @ Y0t.T
        noise = rng.laplace(0.0, 0.5, size=(r1 - r0, n_real))
        noise[rng.random((r1 - r0, n_real)) < 0.01] *= 20.0
        A[r0:r1, :n_real] = u[:, :n_real] + noise
        z = u[:, n_real:n_real + n_bool] + 0.5 * rng.standard_normal((r1 - r0, n_bool))
        A[r0:r1, n_real:n_real + n_bool] = np.where(z >= 0.0, 1.0, -1.0)
        if n_ord:
            uo = u[:, n_real + n_bool:]
            lev = np.ones(uo.shape)
            for q in range(levels - 1):
                lev += uo > edges[:, q][None, :]
            A[r0:r1, n_real + n_bool:] = lev
    kind = np.concatenate([np.full(n_real, LOSS_HUBER), np.full(n_bool, LOSS_HINGE),
                           np.full(n_ord, LOSS_ORDINAL)]).astype(np.int32)
    param = np.concatenate([np.full(n_real, 1.0), np.zeros(n_bool), np.zeros(n_ord)])
    lv = np.concatenate([np.zeros(n_real), np.zeros(n_bool), np.full(n_ord, levels)]).astype(np.int32)
    Xi = rng.standard_normal((m, k))
    Yi = rng.standard_normal((n, k))
    return DenseTable(name, m, n, k, A, kind, param, lv, rx or (REG_L1, lam), ry or (REG_NONNEG, 0.0), Xi, Yi)


# ------------------------------------------------------------ batched tables

@dataclasses.dataclass
class Batch:
    """Concatenated instances: per-instance sizes and losses, CSR / CSC arrays
    with instance-local indices, initial factors (torch tensors on `device`)."""
    m: np.ndarray          # int64 [count]
    n: np.ndarray          # int64 [count]
    k: np.ndarray          # int32 [count]
    kind: np.ndarray       # int32 [count] loss of every column of the instance
    nnz: np.ndarray        # int64 [count]
    rowptr: object         # int32 [sum(m+1)], instance-local entry offsets
    colidx: object         # int32 [sum nnz]
    val: object            # float32 [sum nnz]
    colptr: object         # int32 [sum(n+1)]
    rowidx: object         # int32 [sum nnz]
    cval: object           # float32 [sum nnz]
    X0: object             # float32 [sum m*k]
    Yt0: object            # float32 [sum n*k]

    @property
    def count(self) -> int:
        return int(self.m.size)


def batch_instance_torch(s: int, device, seed=BASE_SEED + 5, m_range=(50, 5000),
                         n_range=(20, 500), ks=(4, 8, 16), p_obs=0.7, noise=0.2):
    """Instance s of the batched workload drawn with torch generators on
    `device` (sizes from a CPU generator, data from a device generator, both
    seeded with seed + s): m, n uniform in their ranges, k uniform over ks;
    even s quadratic loss, odd s Huber; A = X0 Y0 + N(0, noise^2); cells
    observed with probability p_obs.  Returns host-side metadata and device
    tensors (CSR, CSC, initial factors)."""
    import torch
    cg = torch.Generator().manual_seed(seed + s)
    m = int(torch.randint(m_range[0], m_range[1] + 1, (1,), generator=cg))
    n = int(torch.randint(n_range[0], n_range[1] + 1, (1,), generator=cg))
    k = int(ks[int(torch.randint(0, len(ks), (1,), generator=cg))])
    dg = torch.Generator(device=device).manual_seed(seed + s)
    kw = dict(generator=dg, device=device)
    X0 = torch.randn(m, k, **kw)
    Y0t = torch.randn(n, k, **kw)
    mask = torch.rand(m, n, **kw) < p_obs
    A = X0 @ Y0t.T + noise * torch.randn(m, n, **kw)
    rc = mask.nonzero()
    rows, cols = rc[:, 0], rc[:, 1]
    rowptr = torch.zeros(m + 1, dtype=torch.int64, device=device)
    rowptr[1:] = torch.cumsum(torch.bincount(rows, minlength=m), 0)
    cr = mask.T.nonzero()
    colptr = torch.zeros(n + 1, dtype=torch.int64, device=device)
    colptr[1:] = torch.cumsum(torch.bincount(cr[:, 0], minlength=n), 0)
    Xi = torch.randn(m, k, **kw)
    Yi = torch.randn(n, k, **kw)
    return dict(m=m, n=n, k=k, kind=LOSS_QUAD if s % 2 == 0 else LOSS_HUBER,
                rowptr=rowptr.to(torch.int32), colidx=cols.to(torch.int32),
                val=A[rows, cols].float(), colptr=colptr.to(torch.int32),
                rowidx=cr[:, 1].to(torch.int32), cval=A[cr[:, 1], cr[:, 0]].float(),
                X0=Xi.float(), Yt0=Yi.float())


def batch_torch(count=4096, device="cuda", **kw) -> Batch:
    """The batched workload: `count` instances from batch_instance_torch,
    concatenated."""
    import torch
    parts = [batch_instance_torch(s, device, **kw) for s in range(count)]
    cat = lambda key: torch.cat([p[key].reshape(-1) for p in parts])
    return Batch(m=np.array([p["m"] for p in parts], np.int64),
                 n=np.array([p["n"] for p in parts], np.int64),
                 k=np.array([p["k"] for p in parts], np.int32),
                 kind=np.array([p["kind"] for p in parts], np.int32),
                 nnz=np.array([int(p["colidx"].numel()) for p in parts], np.int64),
                 rowptr=cat("rowptr"), colidx=cat("colidx"), val=cat("val"),
                 colptr=cat("colptr"), rowidx=cat("rowidx"), cval=cat("cval"),
                 X0=cat("X0"), Yt0=cat("Yt0"))


# ------------------------------------------------------ tables of features

FEAT_SCALAR, FEAT_CATEGORICAL, FEAT_ORDINAL_MD = 0, 1, 2


@dataclasses.dataclass
class FeatureTable:
    """A table of features (the multi-dimensional model of Sec. 6): Omega
    over (row, feature) in CSR and CSC form, per feature its kind (FEAT_*),
    its label / level count and, for scalar features, its loss.  Feature j
    owns a block of Y of width 1 (scalar), d (categorical, d labels) or d - 1
    (ordinal, d levels); Yt0 holds the initial blocks one after another
    (sum of the widths rows of k)."""
    name: str
    m: int
    nf: int
    k: int
    rowptr: np.ndarray      # int64 [m+1]
    featidx: np.ndarray     # int32 [nnz]
    val: np.ndarray         # float64 [nnz]: real values, +-1, or labels / levels 1..d
    colptr: np.ndarray      # int64 [nf+1]
    rowidx: np.ndarray      # int32 [nnz]
    cval: np.ndarray        # float64 [nnz]
    fkind: np.ndarray       # int32 [nf]
    flevels: np.ndarray     # int32 [nf]
    loss_kind: np.ndarray   # int32 [nf] (scalar features)
    loss_param: np.ndarray  # float64 [nf]
    loss_levels: np.ndarray  # int32 [nf]
    rx: tuple
    ry: tuple
    X0: np.ndarray          # float64 [m, k]
    Yt0: np.ndarray         # float64 [sum of block widths, k]

    @property
    def nnz(self) -> int:
        return int(self.featidx.size)

    def rows(self) -> np.ndarray:
        return np.repeat(np.arange(self.m, dtype=np.int32), np.diff(self.rowptr))

    def widths(self) -> np.ndarray:
        return np.where(self.fkind == FEAT_CATEGORICAL, self.flevels,
                        np.where(self.fkind == FEAT_ORDINAL_MD, self.flevels - 1, 1)).astype(np.int64)


def features_mixed(m=2000, n_real=6, n_bool=4, n_cat=5, n_ord=5, classes=4, levels=5, k=6, p_obs=0.6,
                   seed=BASE_SEED + 30, rx=(REG_QUAD, 0.1), ry=(REG_QUAD, 0.1), cyclic=True,
                   name="features_mixed"):
    """A census-like table of mixed features (Sec. 6's categorical and
    ordinal embeddings beside scalar columns): real features with Huber loss
    (X0 y + Laplace(0, 0.5)), Boolean features with hinge loss (sign of
    X0 y + N(0, 0.5^2)), categorical features with `classes` labels (argmax of
    X0 W + Gumbel noise, W k x classes) and ordinal features with `levels`
    levels (X0 w + N(0, 0.5^2) binned at its empirical quantiles).  Cells are
    observed with probability p_obs.  cyclic: the kinds alternate feature by
    feature, else they come in contiguous groups."""
    rng = rng_for(seed)
    kinds = [0] * n_real + [1] * n_bool + [2] * n_cat + [3] * n_ord
    if cyclic:
        # the i-th feature of every kind, then the (i+1)-th, ...
        keys = [i * 4 + g for g, cnt in enumerate((n_real, n_bool, n_cat, n_ord)) for i in range(cnt)]
        order = np.argsort(np.array(keys), kind="stable")
        kinds = [kinds[o] for o in order]
    nf = len(kinds)
    X0 = rng.standard_normal((m, k))
    rowptr, featidx = omega_bernoulli(m, nf, p_obs, rng)
    rows = np.repeat(np.arange(m, dtype=np.int32), np.diff(rowptr))
    val = np.empty(featidx.size)
    fkind = np.zeros(nf, np.int32)
    flev = np.zeros(nf, np.int32)
    lkind = np.zeros(nf, np.int32)
    lparam = np.zeros(nf)
    llev = np.zeros(nf, np.int32)
    # the entries of each feature in ascending order (the same set and order
    # as a boolean mask, without a pass over all entries per feature)
    by_feat = np.argsort(featidx, kind="stable")
    starts = np.concatenate([[0], np.cumsum(np.bincount(featidx, minlength=nf))])
    for j, kd in enumerate(kinds):
        sel = by_feat[starts[j]:starts[j + 1]]
        r = rows[sel]
        if kd == 0:
            u = X0[r] @ rng.standard_normal(k)
            val[sel] = u + rng.laplace(0.0, 0.5, r.size)
            lkind[j], lparam[j] = LOSS_HUBER, 1.0
        elif kd == 1:
            u = X0[r] @ rng.standard_normal(k)
            val[sel] = np.where(u + 0.5 * rng.standard_normal(r.size) >= 0, 1.0, -1.0)
            lkind[j] = LOSS_HINGE
        elif kd == 2:
            S = X0[r] @ rng.standard_normal((k, classes)) + rng.gumbel(size=(r.size, classes))
            val[sel] = np.argmax(S, axis=1) + 1.0
            fkind[j], flev[j] = FEAT_CATEGORICAL, classes
        else:
            s = X0 @ rng.standard_normal(k) + 0.5 * rng.standard_normal(m)
            edges = np.quantile(s, np.linspace(0, 1, levels + 1)[1:-1])
            val[sel] = np.searchsorted(edges, s[r]) + 1.0
            fkind[j], flev[j] = FEAT_ORDINAL_MD, levels
    widths = np.where(fkind == FEAT_CATEGORICAL, flev, np.where(fkind == FEAT_ORDINAL_MD, flev - 1, 1))
    colptr, rowidx, cval = csc_from_csr(m, nf, rowptr, featidx, val)
    Yt0 = rng.standard_normal((int(widths.sum()), k))
    X0i = rng.standard_normal((m, k))
    return FeatureTable(name, m, nf, k, rowptr, featidx.astype(np.int32), val.astype(np.float64), colptr,
                        rowidx, cval.astype(np.float64), fkind, flev, lkind, lparam, llev, rx, ry, X0i, Yt0)
