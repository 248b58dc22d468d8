"""Seeded, synthetic workload definitions shared by the oracle and the GPU path.

This module holds input data only: propagator lists, kinematic points, exponents,
and the seeded generator of the synthetic stress suite.  It contains none of the
method's arithmetic (no Symanzik polynomials, no sector decomposition, no
subtraction, no expansion, no integration).  Both ``oracle`` and the product
package read their problem definitions from here so that they integrate the same
integrals; neither imports the other.

Momenta are written as polynomials over symbols: a loop momentum ``k1``, an
external momentum ``p1`` and so on.  A product of two momentum symbols stands for
their Minkowski scalar product.  Each propagator is given as ``-E_i`` in the
notation of the Feynman integral definition (Sec. 1, Eq. 1 of the paper; the
``UF`` input convention of Sec. 4.3), i.e. ``-k1**2`` for a massless line.

Kinematics are given as a mapping from a pair of external momentum names to the
value of their scalar product.
"""
from __future__ import annotations

import dataclasses
import numpy as np

__all__ = [
    "FeynmanProblem", "DirectProblem", "DirectFactor",
    "bubble", "box", "box_physical", "box_paper_example", "double_box", "double_box_alt_routing",
    "stress_suite", "STRESS_SEED", "higher_pole_suite",
]


@dataclasses.dataclass(frozen=True)
class FeynmanProblem:
    """A scalar Feynman integral: loop momenta, propagators (-E_i) and kinematics.

    ``propagators`` are strings in Python syntax over the momentum symbols,
    ``indices`` the integer powers a_i, ``kinematics`` maps sorted pairs of
    external momentum names (``("p1", "p2")``) to the scalar product value, and
    ``order`` is the highest power of epsilon requested in the final result.
    """
    name: str
    loop_momenta: tuple
    external_momenta: tuple
    propagators: tuple
    indices: tuple
    kinematics: dict
    order: int


def _kin(pairs):
    out = {}
    for (a, b), v in pairs.items():
        out[tuple(sorted((a, b)))] = v
    return out


def bubble(order: int = 2) -> FeynmanProblem:
    """One-loop massless bubble, a1 = a2 = 1, Euclidean p^2 = -1."""
    return FeynmanProblem(
        name="bubble",
        loop_momenta=("k",), external_momenta=("p",),
        propagators=("-k**2", "-(k+p)**2"),
        indices=(1, 1),
        kinematics=_kin({("p", "p"): -1}),
        order=order)


def _box_kin(S, T):
    # p1^2 = p2^2 = p4^2 = 0, p1.p2 = -S/2, p2.p4 = -T/2, p1.p4 = (S+T)/2,
    # the kinematic substitution of the box example in Sec. 4.3 of the paper.
    from fractions import Fraction as Fr
    S, T = Fr(S), Fr(T)
    return _kin({("p1", "p1"): 0, ("p2", "p2"): 0, ("p4", "p4"): 0,
                 ("p1", "p2"): -S / 2, ("p2", "p4"): -T / 2, ("p1", "p4"): (S + T) / 2})


def box(order: int = 0, S=1, T=2) -> FeynmanProblem:
    """One-loop massless on-shell box, a_i = 1, with s = -S, t = -T.

    The default S = 1, T = 2 is the Euclidean point s = -1, t = -2.
    """
    return FeynmanProblem(
        name="box",
        loop_momenta=("k",), external_momenta=("p1", "p2", "p4"),
        propagators=("-k**2", "-(k+p1)**2", "-(k+p1+p2)**2", "-(k+p1+p2+p4)**2"),
        indices=(1, 1, 1, 1),
        kinematics=_box_kin(S, T),
        order=order)


def box_physical(order: int = 0, s=3, t=-1) -> FeynmanProblem:
    """The massless box at a physical point s > 0, t < 0 (F changes sign: contour deformation)."""
    p = box(order=order, S=-s, T=-t)
    return dataclasses.replace(p, name="box_physical")


def box_paper_example() -> FeynmanProblem:
    """The box of the worked example in Sec. 4.3 (S = 3, T = 1)."""
    p = box(order=0, S=3, T=1)
    return dataclasses.replace(p, name="box_S3_T1")


def double_box(order: int = 0, S=1, T=1) -> FeynmanProblem:
    """Two-loop massless planar double box (ladder routing), a_i = 1, s = -S, t = -T."""
    return FeynmanProblem(
        name="double_box",
        loop_momenta=("k1", "k2"), external_momenta=("p1", "p2", "p4"),
        propagators=("-k1**2", "-(k1+p1)**2", "-(k1+p1+p2)**2", "-(k1-k2)**2",
                     "-k2**2", "-(k2+p1+p2)**2", "-(k2+p1+p2+p4)**2"),
        indices=(1,) * 7,
        kinematics=_box_kin(S, T),
        order=order)


def double_box_alt_routing(order: int = 0, S=1, T=1) -> FeynmanProblem:
    """The same planar double box with loop momenta relabelled (k1 -> -k1 - p1 - p2, k2 -> -k2 - p1 - p2).

    U and F depend only on the graph, so both routings give the same polynomials.
    """
    return FeynmanProblem(
        name="double_box_alt",
        loop_momenta=("k1", "k2"), external_momenta=("p1", "p2", "p4"),
        propagators=("-(k1+p1+p2)**2", "-(k1+p2)**2", "-k1**2", "-(k1-k2)**2",
                     "-(k2+p1+p2)**2", "-k2**2", "-(k2-p4)**2"),
        indices=(1,) * 7,
        kinematics=_box_kin(S, T),
        order=order)


# ---------------------------------------------------------------------------
# Direct integrands (the SDEvaluateDirect input form of Sec. 4.3)
# ---------------------------------------------------------------------------

@dataclasses.dataclass(frozen=True)
class DirectFactor:
    """A polynomial raised to the power n + m*eps.

    ``terms`` is a tuple of (coefficient, exponent-tuple) pairs; coefficients are
    floats (exactly representable binary64 numbers), exponents non-negative ints.
    """
    terms: tuple
    n: int
    m: int


@dataclasses.dataclass(frozen=True)
class DirectProblem:
    """An integrand  prod_i x_i^{k_i} * prod_f P_f^{n_f + m_f eps} * log(P_1)^j  over [0,1]^dim.

    ``orders`` lists the powers of epsilon whose coefficients are wanted.
    """
    name: str
    dim: int
    monomial: tuple
    factors: tuple
    log_power: int
    orders: tuple


def higher_pole_suite():
    """Direct integrands with a pole of order 2 in one variable (t^{-2+eps}), the case
    the Taylor subtraction of order p >= 1 covers: x^{-2+eps}/(1+x); the separable
    x1^{-2+eps}(1+x1)^-1 x2^{-1+eps}(1+x2)^-1; and a non-separable 2-dimensional one."""
    F = DirectFactor
    one_plus = lambda dim, j: F(((1.0, (0,) * dim), (1.0, tuple(int(i == j) for i in range(dim)))), -1, 0)
    eps_pow = lambda dim, j, m: F(((1.0, tuple(int(i == j) for i in range(dim))),), 0, m)
    return (
        DirectProblem("pole2_1d", 1, (-2,), (eps_pow(1, 0, 1), one_plus(1, 0)), 0, (-1, 0, 1, 2)),
        DirectProblem("pole2_separable", 2, (-2, -1), (eps_pow(2, 0, 1), eps_pow(2, 1, 1), one_plus(2, 0),
                                                      one_plus(2, 1)), 0, (-2, -1, 0, 1)),
        DirectProblem("pole2_mixed", 2, (-2, -1), (eps_pow(2, 0, 1), eps_pow(2, 1, 2),
                                                   F(((1.0, (0, 0)), (0.5, (1, 0)), (0.25, (0, 1)), (0.3, (1, 1))),
                                                     -2, 1)), 0, (-2, -1, 0, 1)),
    )


STRESS_SEED = 1511036140


def _monomials_up_to_degree3(dim):
    """Exponent tuples of total degree 1..3 in ``dim`` variables, in a fixed order."""
    out = []
    for deg in (1, 2, 3):
        def rec(i, left, cur):
            if i == dim - 1:
                out.append(tuple(cur + [left]))
                return
            for k in range(left, -1, -1):
                rec(i + 1, left - k, cur + [k])
        rec(0, deg, [])
    return out


def stress_suite(n_units: int = 10_000, seed: int = STRESS_SEED, orders=(0, 1, 2), all_orders: bool = False):
    """The seeded synthetic stress suite.

    Each integrand has dim uniform in 3..8, monomial exponents k_i in {0..3},
    two polynomials with 5..40 distinct monomials of total degree <= 3 (at most
    all of them when there are fewer) and coefficients
    uniform in [0.1, 1] (one term is always the constant monomial so that P >= 0.1
    on the unit cube), exponents n + m*eps with n, m uniform in {-2..2}, and
    log(P1)^j with j in {0, 1, 2}.  Coefficients are rounded to binary64.  Each
    integrand contributes one unit: the coefficient of eps^K with K drawn
    uniformly from ``orders`` (the lowest order when the integrand does not
    depend on eps); with ``all_orders`` it contributes the coefficients of every
    order in ``orders`` instead (the same integrands: the order is still drawn).
    Returns a list of DirectProblem.
    """
    rng = np.random.Generator(np.random.PCG64(seed))
    out = []
    for u in range(n_units):
        dim = int(rng.integers(3, 9))
        mono = tuple(int(v) for v in rng.integers(0, 4, size=dim))
        factors = []
        monos = _monomials_up_to_degree3(dim)
        for _ in range(2):
            nterms = min(int(rng.integers(5, 41)), len(monos) + 1)
            pick = rng.choice(len(monos), size=nterms - 1, replace=False)
            exps = [tuple([0] * dim)] + [monos[i] for i in sorted(pick)]
            coefs = rng.uniform(0.1, 1.0, size=len(exps))
            terms = tuple((float(c), e) for c, e in zip(coefs, exps))
            n = int(rng.integers(-2, 3))
            m = int(rng.integers(-2, 3))
            factors.append(DirectFactor(terms=terms, n=n, m=m))
        j = int(rng.integers(0, 3))
        K = int(orders[int(rng.integers(0, len(orders)))])
        eps_free = all(f.m == 0 for f in factors)
        if eps_free:
            K = min(orders)          # higher coefficients of an eps-free integrand vanish
        Ks = (min(orders),) if eps_free else tuple(orders)
        out.append(DirectProblem(name=f"stress{u}", dim=dim, monomial=mono,
                                 factors=tuple(factors), log_power=j, orders=Ks if all_orders else (K,)))
    return out
