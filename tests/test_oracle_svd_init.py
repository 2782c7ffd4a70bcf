"""Pins of the oracle's SVD initialisation (Sec. 7.5): an exactly low-rank
table (plus column offsets) is reproduced by the initial model with the
offset, and the initial X does not depend on the affine encoding of a
quadratic-loss column (Boolean (0, 1) vs (-1, 1); ordinal (1, 2, 3) vs
(-5, 0, 5)), as the paper says of its scaling."""
import numpy as np
import pytest

Q = 0


def _full_problem(o, A, k, kinds=Q):
    m, n = A.shape
    rows = np.repeat(np.arange(m), n)
    cols = np.tile(np.arange(n), m)
    return o.Problem(m, n, k, rows, cols, A.reshape(-1), kinds, 1.0, 0)


def test_low_rank_table_is_reproduced_with_offset(oracle_mod):
    rng = np.random.default_rng(5)
    m, n, r = 60, 25, 3
    A = rng.normal(size=(m, r)) @ rng.normal(size=(r, n)) + rng.normal(size=n) * 4
    p = _full_problem(oracle_mod, A, r + 1)
    X, Yt, S = p.svd_init(offset=True)
    assert np.all(X[:, -1] == 1.0)
    np.testing.assert_allclose(X @ Yt.T, A, rtol=0, atol=1e-6 * np.abs(A).max())
    # without the offset the same rank cannot absorb the column means
    p2 = _full_problem(oracle_mod, A, r)
    X2, Yt2, _ = p2.svd_init(offset=False)
    assert np.abs(X2 @ Yt2.T - A).max() > 1e-2 * np.abs(A).max()


def _x_gram(X):
    return X @ X.T


def test_affine_encodings_give_the_same_x(oracle_mod):
    rng = np.random.default_rng(6)
    m, n = 80, 12
    L = rng.normal(size=(m, 3)) @ rng.normal(size=(3, n))
    A1 = L.copy()
    A1[:, 0] = (L[:, 0] > 0).astype(float)            # Boolean as (0, 1)
    A1[:, 1] = np.digitize(L[:, 1], [-0.5, 0.5]) + 1   # ordinal as (1, 2, 3)
    A2 = A1.copy()
    A2[:, 0] = 2 * A1[:, 0] - 1                        # Boolean as (-1, 1)
    A2[:, 1] = 5 * A1[:, 1] - 10                       # ordinal as (-5, 0, 5)
    mask = rng.random((m, n)) < 0.7
    def prob(A):
        rows, cols = np.nonzero(mask)
        return oracle_mod.Problem(m, n, 3, rows, cols, A[rows, cols], Q, 1.0, 0)
    X1, Y1, S1 = prob(A1).svd_init()
    X2, Y2, S2 = prob(A2).svd_init()
    np.testing.assert_allclose(S1, S2, rtol=1e-6)
    np.testing.assert_allclose(_x_gram(X1), _x_gram(X2), rtol=0, atol=1e-6 * np.abs(_x_gram(X1)).max())
    # an encoding that is not affine changes it
    A3 = A1.copy()
    A3[:, 1] = np.choose((A1[:, 1] - 1).astype(int), [0.0, 1.0, 10.0])
    X3, _, _ = prob(A3).svd_init()
    assert np.abs(_x_gram(X3) - _x_gram(X1)).max() > 1e-3 * np.abs(_x_gram(X1)).max()
