"""Pins of the oracle's adaptive cubature (Genz-Malik rule and the subdivision passes)
against exact integrals: polynomial exactness of both rules, the fourth difference,
closed-form integrals and the box's closed form through every sector."""
import itertools
import math

import mpmath as mp
import numpy as np
import pytest

import workloads as W
from oracle import cuhre as C, pipeline as P


def _monomial_integral(k, lo, hi):
    return float(np.prod([(b ** (e + 1) - a ** (e + 1)) / (e + 1) for e, a, b in zip(k, lo, hi)]))


@pytest.mark.parametrize("n", [2, 3, 4, 6])
def test_rule_degrees(n):
    """Every monomial of total degree <= 7 is integrated exactly by I7 and every one
    of degree <= 5 by I5 (and then err = 0), on an off-centre box; x_1^8 is not."""
    rng = np.random.default_rng(n)
    lo = rng.uniform(-0.7, 0.2, n)
    hi = lo + rng.uniform(0.3, 1.1, n)
    c, h = (lo + hi) / 2, (hi - lo) / 2
    exps = [k for k in itertools.product(range(8), repeat=n) if sum(k) <= 7]
    if n == 6:
        exps = [exps[i] for i in rng.choice(len(exps), 300, replace=False)]
    K = np.array(exps)
    f = lambda X: np.prod(X[:, None, :] ** K[None, :, :], axis=2)
    I7, I5, err, _ = C.apply_rule(f, c, h)
    for i, k in enumerate(exps):
        ex = _monomial_integral(k, lo, hi)
        scale = _monomial_integral([2 * e for e in k], np.zeros(n), np.maximum(np.abs(lo), np.abs(hi))) ** 0.5
        scale = max(scale, float(np.prod(hi - lo)))
        assert abs(I7[i] - ex) <= 1e-13 * scale, (k, I7[i], ex)
        if sum(k) <= 5:
            assert abs(I5[i] - ex) <= 1e-13 * scale, (k, I5[i], ex)
            assert err[i] <= 2e-13 * scale
    k8 = (8,) + (0,) * (n - 1)
    I7, _, _, _ = C.apply_rule(lambda X: X[:, 0] ** 8, c, h)
    assert abs(I7[0] - _monomial_integral(k8, lo, hi)) > 1e-8


def test_weights_and_points():
    """Point counts 1 + 4n + 2n(n-1) + 2^n, all strictly inside the box."""
    for n in range(2, 9):
        groups = C.rule_points(n)
        assert sum(len(g) for g in groups) == 1 + 4 * n + 2 * n * (n - 1) + 2 ** n
        assert max(np.max(np.abs(np.stack(g))) for g in groups) < 1.0


def test_fourth_difference_and_axis():
    """The fourth difference vanishes for cubics along an axis, not for quartics; the
    split goes across the quartic coordinate even when a quadratic is larger."""
    c, h = np.array([0.4, 0.5, 0.6]), np.array([0.3, 0.2, 0.25])
    _, _, _, dif = C.apply_rule(lambda X: 5 * X[:, 0] ** 3 - X[:, 1] ** 2 + 7 * X[:, 2] * X[:, 0], c, h)
    assert np.max(dif) < 1e-13
    _, _, _, dif = C.apply_rule(lambda X: 10 * X[:, 0] ** 2 + X[:, 2] ** 4, c, h)
    assert dif[2, 0] > 1e-4 and dif[0, 0] < 1e-12 and C.split_axis(dif, h) == 2
    # no fourth difference anywhere: the widest side
    assert C.split_axis(np.zeros((3, 1)), h) == 0
    assert C.split_axis(np.zeros((3, 1)), np.array([0.1, 0.3, 0.3])) == 1


@pytest.mark.parametrize("dim", [2, 3, 5])
def test_adaptive_closed_forms(dim):
    """Exponential and Genz product-peak integrands: the estimate meets the tolerance
    and the reported error bounds the true error."""
    rng = np.random.default_rng(dim)
    a = rng.uniform(-2, 2, dim)
    r = C.cuhre(lambda X: np.exp(X @ a), dim, rel_tol=1e-9)
    ex = float(np.prod([(math.exp(x) - 1) / x for x in a]))
    assert r.converged and abs(r.value[0] - ex) <= max(r.error[0], 1e-14) and r.error[0] <= 1e-9 * abs(ex)
    cc = rng.uniform(2, 5, dim)
    w = rng.uniform(0.2, 0.8, dim)
    f = lambda X: np.prod(1.0 / (cc ** -2.0 + (X - w) ** 2), axis=1)
    ex = float(np.prod(cc * (np.arctan(cc * (1 - w)) + np.arctan(cc * w))))
    r = C.cuhre(f, dim, rel_tol=1e-7 if dim < 5 else 1e-5, max_passes=60)
    assert r.converged and abs(r.value[0] - ex) <= r.error[0]


def test_vector_valued_and_one_dimension():
    """A vector integrand: each result meets its own tolerance; dim 1 through the
    dummy second coordinate."""
    f = lambda X: np.stack([np.sqrt(X[:, 0]), np.log(X[:, 0]) ** 2, np.cos(3 * X[:, 0])], axis=1)
    r = C.cuhre(f, 1, rel_tol=1e-8, max_passes=80)
    ex = [2.0 / 3.0, 2.0, math.sin(3.0) / 3.0]
    assert r.converged
    for o in range(3):
        assert abs(r.value[o] - ex[o]) <= max(r.error[o], 1e-15), o
        assert r.error[o] <= 1e-8 * abs(ex[o])


def test_box_through_all_sectors():
    """Every sector unit of the box by the cubature, assembled with the prefactor:
    2/eps^2 - ln2/eps - 2 pi^2/3 at s = -1, t = -2 within the summed errors."""
    pr = P.feynman_problem(W.box())
    val, err = {}, {}
    for u in pr.units:
        r = C.cuhre(u.f_numpy, u.dim, rel_tol=1e-7, max_passes=60)
        val[u.order] = val.get(u.order, 0.0) + r.value[0]
        err[u.order] = err.get(u.order, 0.0) + r.error[0]
    R, _ = P.assemble(pr, val, {K: 0.0 for K in err})
    q, c = pr.prefactor
    E = {n: sum(abs(float(ci)) * err.get(n - (i - q), 0.0) for i, ci in enumerate(c)) for n in R}
    exact = {-2: 2.0, -1: -math.log(2.0), 0: -2 * math.pi ** 2 / 3}
    for n, v in exact.items():
        assert abs(R[n] - v) <= E[n] + 1e-12, (n, R[n], v, E[n])
        assert E[n] < 1e-5


def test_bubble_unit_against_quadrature():
    """A 1-D sector unit (subtracted, with logarithms) against mpmath's quadrature."""
    pr = P.feynman_problem(W.bubble())
    for u in pr.units[:4]:
        r = C.cuhre(u.f_numpy, u.dim, rel_tol=1e-10, max_passes=80)
        with mp.workdps(30):
            ex = float(mp.quad(lambda t: u.f_mp([t], 30), [0, 1]))
        assert abs(r.value[0] - ex) <= max(r.error[0], 1e-14), (u.sector, u.order)
