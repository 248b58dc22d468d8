"""Units, evaluation and assembly (oracle).

A unit is one (sector, eps order K) pair, integrated on its own, as in the
paper's integrand database whose keys carry the eps order and the sector number
(Sec. 4.7).  Per order, sector results are summed and their errors combined in
the mean-square norm, sqrt(sum sigma^2) (Sec. 4.3); the prefactor series is then
multiplied in (Eq. 2).
"""
from __future__ import annotations

import dataclasses
import itertools
import math

import numpy as np
import sympy as sp
import mpmath as mp

from . import sectors as S
from .uf import symanzik
from .prefactor import prefactor_series, combine


@dataclasses.dataclass
class Unit:
    sector: int                 # index into the sector list
    order: int                  # eps order K of the parametric integral
    variables: tuple            # original indices; dimension i of the cube <-> variables[i]
    expr: object                # sympy expression in t-symbols
    complex: bool = False       # deformed contour: complex values
    term: tuple = None          # separately integrable term: the variables whose pole term it is
    _np: object = None
    _mp: object = None

    @property
    def dim(self):
        return len(self.variables)

    def f_numpy(self, X):
        """Evaluate in float64 (complex128 for a deformed contour) at points X of shape (n, dim)."""
        if self._np is None:
            syms = [S.tsym(j) for j in self.variables]
            self._np = sp.lambdify(syms, self.expr, modules="numpy")
        cols = [X[:, i] for i in range(self.dim)]
        if self.complex:
            cols = [c.astype(np.complex128) for c in cols]
        with np.errstate(all="ignore"):
            v = self._np(*cols)
        dt = np.complex128 if self.complex else np.float64
        return np.broadcast_to(np.asarray(v, dtype=dt), (X.shape[0],)).copy()

    def f_mp(self, x, dps=50):
        """Evaluate at one point with mpmath at ``dps`` digits (x given as exact binary64)."""
        if self._mp is None:
            syms = [S.tsym(j) for j in self.variables]
            self._mp = sp.lambdify(syms, self.expr, modules="mpmath")
        with mp.workdps(dps):
            return self._mp(*[mp.mpf(float(v)) for v in x])


@dataclasses.dataclass
class Problem:
    name: str
    sectors: list
    units: list
    prefactor: tuple          # (q, coeffs)
    int_orders: tuple         # orders K of the parametric integral
    out_orders: tuple         # orders n of the final result


def _term_units(i, s, K):
    """The separately integrable terms of unit (sector i, order K): one unit per subset
    T of the singular variables, over the variables not in T (the term is constant
    along those; a term over no variable keeps the first one)."""
    units = []
    Sv = S.singular_vars(s)
    for r in range(len(Sv) + 1):
        for T in itertools.combinations(Sv, r):
            e = S.unit_integrand(s, K, term=T)
            if e == 0:
                continue
            var = tuple(j for j in s.variables if j not in T) or (s.variables[0],)
            units.append(Unit(i, K, var, e, term=tuple(T)))
    return units


def feynman_problem(problem, strategy="M", lam=None, separate_terms=False):
    """Units of a Feynman integral.  ``lam``: a contour-deformation parameter per
    sector (callable sector -> lam or None, or one number for every sector whose F
    has a coefficient that is not positive).  ``separate_terms``: one unit per
    separately integrable term of every real sector and order (``_term_units``)."""
    U, F, xs = symanzik(problem)
    L = len(problem.loop_momenta)
    prim = S.primary_sectors(U, F, xs, problem.indices, L)
    secs = [s for p in prim for s in S.decompose(p, strategy)]
    kmin = min(S.min_order(s) for s in secs)
    q0, _ = prefactor_series(problem.indices, L, 0)
    khi = problem.order + q0
    pre = prefactor_series(problem.indices, L, problem.order - kmin)
    units = []
    for i, s in enumerate(secs):
        if callable(lam):
            ls = lam(s)
        elif lam is not None and any(c <= 0 for c in s.polys[-1][0].coeffs()):
            ls = lam
        else:
            ls = None
        for K in range(max(kmin, S.min_order(s)), khi + 1):
            if separate_terms and ls is None:
                units += _term_units(i, s, K)
                continue
            e = S.unit_integrand(s, K, ls)
            if e != 0:
                units.append(Unit(i, K, s.variables, e, complex=ls is not None))
    int_orders = tuple(range(kmin, khi + 1))
    out_orders = tuple(range(kmin - pre[0], problem.order + 1))
    return Problem(problem.name, secs, units, pre, int_orders, out_orders)


def direct_problem(problem):
    sec = S.direct_sector(problem)
    secs = S.decompose(sec, "M")
    units = []
    for i, s in enumerate(secs):
        for K in problem.orders:
            if K < S.min_order(s):
                continue
            e = S.unit_integrand(s, K)
            if e != 0:
                units.append(Unit(i, K, s.variables, e))
    return Problem(problem.name, secs, units, (0, [mp.mpf(1)]), tuple(problem.orders), tuple(problem.orders))


def sum_orders(prob, unit_values, unit_errors=None):
    """Per eps order: sum over sectors; errors in the mean-square norm."""
    val = {K: 0.0 for K in prob.int_orders}
    err = {K: 0.0 for K in prob.int_orders}
    for i, u in enumerate(prob.units):
        val[u.order] += unit_values[i]
        if unit_errors is not None:
            err[u.order] += unit_errors[i] ** 2
    return val, {K: math.sqrt(e) for K, e in err.items()}


def assemble(prob, val, err):
    """Multiply the prefactor series in; sigma_n = sqrt(sum c_m^2 sigma_{n-m}^2)."""
    R = combine(prob.prefactor, prob.int_orders, val, prob.out_orders)
    q, coeffs = prob.prefactor
    E = {}
    for n in prob.out_orders:
        s = 0.0
        for i, c in enumerate(coeffs):
            K = n - (i - q)
            if K in err:
                s += float(c) ** 2 * err[K] ** 2
        E[n] = math.sqrt(s)
    return {n: float(v) for n, v in R.items()}, E


def _absify(e):
    """Condition-scaled magnitude M of an expression (the per-point tolerance scale).

    Sums: the sum of the magnitudes of the terms; products: the product of the
    magnitudes of the factors; a power b^x: |b|^x (1 + |x| (M(b)/|b| - 1)); a
    logarithm log b: |log b| + M(b)/|b|; numbers and variables: their absolute
    value.  This is first-order forward error propagation: a relative error
    r = c u M(b)/|b| of b becomes |x| r in b^x and an absolute error r in log b,
    so |f_computed - f| <= c u M(x) bounds the rounding error of any evaluation
    order of f (u the unit roundoff, c of the order of the expression depth),
    and M >= |f| everywhere.  Where no base cancels (M(b) = |b|) a power adds
    nothing and a logarithm adds 1.  M is what the per-point tolerances scale
    with where the pole-subtraction differences cancel.
    """
    if e.is_Add:
        return sp.Add(*[_absify(a) for a in e.args])
    if e.is_Mul:
        return sp.Mul(*[_absify(a) for a in e.args])
    if e.is_Pow:
        b, x = e.args
        mb, ab = _absify(b), sp.Abs(b)
        if mb == ab:
            return sp.Pow(ab, x)
        return sp.Pow(ab, x) * (1 + sp.Abs(x) * (mb / ab - 1))
    if isinstance(e, sp.log):
        b = e.args[0]
        mb, ab = _absify(b), sp.Abs(b)
        return sp.Abs(e) + (1 if mb == ab else mb / ab)
    return sp.Abs(e)


def magnitude_numpy(unit, X):
    """M(x) of ``_absify`` at points X (n, dim), float64."""
    if getattr(unit, "_abs", None) is None:
        syms = [S.tsym(j) for j in unit.variables]
        unit._abs = sp.lambdify(syms, _absify(unit.expr), modules="numpy")
    with np.errstate(all="ignore"):
        v = unit._abs(*[X[:, i] for i in range(unit.dim)])
    return np.broadcast_to(np.abs(np.asarray(v)).astype(np.float64), (X.shape[0],)).copy()
