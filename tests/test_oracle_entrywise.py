"""Pins of the oracle's entrywise pieces against what the paper and the
mathematics fix: loss derivatives against finite differences of the loss,
the Huber infimal-convolution identity (Sec. 4.3), the logistic loss against
-log(sigma), the ordinal hinge against the hinge (d = 2) and its integer-point
closed form, decoding against brute force and the derived threshold rule
(Sec. 5.3), and every prox against a direct 1-D minimisation (Sec. 7.2)."""
import math

import numpy as np
import pytest
from scipy import optimize, special

Q, HU, HI, LO, OR = 0, 1, 2, 3, 4
L1, QT = 5, 6
RZ, RQ, RL1, RNN = 0, 1, 2, 3


def _fd(o, kind, u, a, param, levels, h=1e-6):
    return (o.loss(kind, u + h, a, param, levels) - o.loss(kind, u - h, a, param, levels)) / (2 * h)


@pytest.mark.parametrize("kind,param,levels,avals", [
    (Q, 0.0, 0, [-1.3, 0.0, 2.5]),
    (HU, 1.0, 0, [-2.0, 0.3, 1.7]),
    (HU, 0.4, 0, [-2.0, 0.3, 1.7]),
    (HI, 0.0, 0, [-1.0, 1.0]),
    (LO, 0.0, 0, [-1.0, 1.0]),
    (OR, 0.0, 7, [1, 2, 4, 7]),
    (L1, 0.0, 0, [-1.3, 0.0, 2.5]),
    (QT, 0.2, 0, [-1.3, 0.0, 2.5]),
    (QT, 0.85, 0, [-1.3, 0.0, 2.5]),
])
def test_derivative_matches_finite_difference(oracle_mod, kind, param, levels, avals):
    o = oracle_mod
    rng = np.random.default_rng(0)
    for a in avals:
        for u in rng.uniform(-6, 9, size=60):
            # stay away from kinks: Huber |u-a| = delta, hinge au = 1, ordinal u = integer
            if kind == HU and abs(abs(u - a) - param) < 1e-3:
                continue
            if kind == HI and abs(a * u - 1) < 1e-3:
                continue
            if kind == OR and abs(u - round(u)) < 1e-3:
                continue
            if kind in (L1, QT) and abs(u - a) < 1e-3:
                continue
            assert o.dloss(kind, u, a, param, levels) == pytest.approx(
                _fd(o, kind, u, a, param, levels), abs=1e-6, rel=1e-6)


def test_kink_subgradient_is_zero_term(oracle_mod):
    o = oracle_mod
    # hinge at a u = 1: the term is inactive
    assert o.dloss(HI, 1.0, 1.0) == 0.0
    assert o.dloss(HI, -1.0, -1.0) == 0.0
    # ordinal at u = a: every term inactive
    for a in range(1, 8):
        assert o.dloss(OR, float(a), a, 0.0, 7) == 0.0
        assert o.loss(OR, float(a), a, 0.0, 7) == 0.0


def test_huber_is_infimal_convolution(oracle_mod):
    """huber(x) = inf { |s| + n^2/2 : x = n + s } (Sec. 4.3, Huber PCA)."""
    o = oracle_mod
    for x in np.linspace(-4, 4, 41):
        res = optimize.minimize_scalar(lambda s: abs(s) + 0.5 * (x - s) ** 2,
                                       bounds=(-10, 10), method="bounded",
                                       options={"xatol": 1e-12})
        assert o.loss(HU, x, 0.0, 1.0) == pytest.approx(res.fun, abs=1e-8)


def test_huber_delta_scaling(oracle_mod):
    """huber_delta(x) = delta^2 huber_1(x / delta): the threshold-delta reading
    is the paper's function rescaled."""
    o = oracle_mod
    for d in (0.25, 0.5, 2.0):
        for x in np.linspace(-5, 5, 23):
            assert o.loss(HU, x, 0.0, d) == pytest.approx(d * d * o.loss(HU, x / d, 0.0, 1.0),
                                                          rel=1e-13, abs=1e-15)


def test_logistic_is_negative_log_sigmoid(oracle_mod):
    o = oracle_mod
    for a in (-1.0, 1.0):
        for u in np.linspace(-40, 40, 161):
            ref = -special.log_expit(a * u)
            assert o.loss(LO, u, a) == pytest.approx(ref, rel=1e-12, abs=1e-300)
            # derivative: -a (1 - sigma(a u)) = -a sigma(-a u)
            assert o.dloss(LO, u, a) == pytest.approx(-a * special.expit(-a * u), rel=1e-12,
                                                     abs=1e-300)


def test_ordinal_two_levels_is_scaled_hinge(oracle_mod):
    """With d = 2 the ordinal hinge is half the hinge loss at 2u - 3 with
    level l coded as 2l - 3 in {-1, +1}."""
    o = oracle_mod
    for lev in (1, 2):
        for u in np.linspace(-3, 5, 33):
            assert o.loss(OR, u, lev, 0.0, 2) == pytest.approx(
                0.5 * o.loss(HI, 2 * u - 3, 2 * lev - 3), abs=1e-14)


def test_ordinal_integer_points(oracle_mod):
    """At an integer u = b the ordinal hinge sums 1 + 2 + ... + |a - b|."""
    o = oracle_mod
    d = 7
    for a in range(1, d + 1):
        for b in range(-2, d + 3):
            t = abs(a - b)
            if b < 1:
                # below level 1 the terms a' < a keep growing, terms a' > a vanish
                expect = sum(1 - b + ap for ap in range(1, a))
            elif b > d:
                expect = sum(1 + b - ap for ap in range(a + 1, d + 1))
            else:
                expect = t * (t + 1) / 2
            assert o.loss(OR, float(b), a, 0.0, d) == pytest.approx(expect, abs=1e-12)


def test_decode_rules(oracle_mod):
    """Decoding (Sec. 5.3): real losses return u; Boolean losses sign(u) with
    sign(0) = +1; ordinal argmin equals 1 + #{a in 1..d-1 : u > a + 1/2}, the
    rule that follows from L(u, a+1) - L(u, a) = (1 + a - u)_+ - (u - a)_+."""
    o = oracle_mod
    grid = np.concatenate([np.linspace(-3, 10, 521), np.arange(-2, 11) + 0.5,
                           np.arange(-2, 11, dtype=float), [0.0, -0.0]])
    grid = np.concatenate([grid, np.nextafter(grid, np.inf), np.nextafter(grid, -np.inf)])
    for u in grid:
        assert o.decode(Q, u) == u
        assert o.decode(HU, u) == u
        assert o.decode(HI, u) == (1.0 if u >= 0 else -1.0)
        assert o.decode(LO, u) == (1.0 if u >= 0 else -1.0)
        for d in (2, 5, 7):
            rule = 1 + sum(1 for a in range(1, d) if u > a + 0.5)
            assert o.decode(OR, u, d) == rule
            # brute force in exact-enough arithmetic: every level's loss
            vals = [o.loss(OR, u, a, 0.0, d) for a in range(1, d + 1)]
            assert vals[int(o.decode(OR, u, d)) - 1] == min(vals)


def _brute_prox(rfun, alpha, z):
    out = np.empty_like(z)
    for c, zc in enumerate(z):
        res = optimize.minimize_scalar(lambda x: alpha * rfun(x) + 0.5 * (x - zc) ** 2,
                                       bounds=(zc - 20, zc + 20), method="bounded",
                                       options={"xatol": 1e-12})
        out[c] = res.x
    return out


@pytest.mark.parametrize("alpha", [0.01, 0.3, 2.0])
def test_prox_is_argmin(oracle_mod, alpha):
    """prox_{alpha r}(z) = argmin_x alpha r(x) + ||x - z||^2 / 2 (Sec. 7.2),
    coordinate by coordinate since all four regularisers are separable."""
    o = oracle_mod
    rng = np.random.default_rng(1)
    z = rng.normal(0, 2, size=9)
    z[0] = 0.0
    w = 0.7
    cases = {
        RZ: lambda x: 0.0,
        RQ: lambda x: w * x * x,
        RL1: lambda x: w * abs(x),
        RNN: lambda x: 0.0 if x >= 0 else 1e30,
    }
    for kind, rfun in cases.items():
        got = o.prox(kind, w, alpha, z)
        ref = _brute_prox(rfun, alpha, z)
        np.testing.assert_allclose(got, ref, atol=2e-6)


def test_reg_values(oracle_mod):
    o = oracle_mod
    x = np.array([0.5, -1.5, 2.0])
    assert o.reg(RZ, 3.0, x) == 0.0
    assert o.reg(RQ, 0.1, x) == pytest.approx(0.1 * np.dot(x, x))
    assert o.reg(RL1, 0.1, x) == pytest.approx(0.1 * np.abs(x).sum())
    assert math.isinf(o.reg(RNN, 0.0, x))
    assert o.reg(RNN, 0.0, np.abs(x)) == 0.0


def test_l1_and_quantile_closed_forms(oracle_mod):
    """l1: |a - u| (Sec. 4.2, robust PCA); quantile: alpha (a - u)_+ +
    (1 - alpha) (u - a)_+ (Sec. 4.2, quantile PCA), which at alpha = 1/2 is
    half the l1 loss; at the kink u = a both take the zero subgradient; both
    decode to u."""
    o = oracle_mod
    rng = np.random.default_rng(7)
    for u, a in rng.normal(0, 2, size=(50, 2)):
        assert o.loss(L1, u, a) == pytest.approx(abs(a - u), rel=1e-15)
        assert o.loss(QT, u, a, 0.5) == pytest.approx(0.5 * abs(a - u), rel=1e-15)
        al = 0.3
        want = al * (a - u) if a > u else (1 - al) * (u - a)
        assert o.loss(QT, u, a, al) == pytest.approx(want, rel=1e-15)
    assert o.dloss(L1, 1.25, 1.25) == 0.0 and o.dloss(QT, -0.5, -0.5, 0.3) == 0.0
    assert o.decode(L1, 3.7) == 3.7 and o.decode(QT, -2.25) == -2.25


@pytest.mark.parametrize("alpha", [0.2, 0.5, 0.9])
def test_quantile_loss_minimiser_is_the_quantile(oracle_mod, alpha):
    """The scalene loss performs quantile regression (Sec. 4.2): over a
    constant prediction mu, sum_i L(mu, a_i) is minimised at the alpha-quantile
    of the a_i -- the order statistic a_(ceil(alpha n)) -- which brute force
    over a fine grid confirms."""
    o = oracle_mod
    rng = np.random.default_rng(11)
    a = rng.normal(0, 1, size=101)
    total = lambda mu: sum(o.loss(QT, float(mu), float(ai), alpha) for ai in a)
    q = np.sort(a)[int(np.ceil(alpha * a.size)) - 1]
    grid = np.linspace(a.min() - 0.5, a.max() + 0.5, 4001)
    best = min(total(g) for g in grid)
    assert total(q) <= best + 1e-12
    # and strictly better than moving off it in either direction
    assert total(q - 0.05) > total(q) and total(q + 0.05) > total(q)
