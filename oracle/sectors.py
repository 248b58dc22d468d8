"""Sector decomposition, pole subtraction and epsilon expansion (oracle, sympy).

The paper's program summary splits the method into the sector decomposition,
the pole resolution with epsilon expansion, and the numerical integration of
the result (Sec. 1 defers the algorithmic detail to the earlier FIESTA papers,
and Sec. 4.4 ``STRATEGY`` names the decomposition strategies).  This module is
the textbook Binoth-Heinrich procedure written out plainly:

1. Primary sectors (Eq. 2 with the delta function): for each l, the region where
   x_l is the largest parameter; x_l = 1 and x_j = t_j in [0,1] for j != l.  The
   integrand of Eq. 2 is homogeneous of degree -n in x, so the delta function
   integrates to 1 in each region.
2. Iterated decomposition: while a polynomial factor (after pulling out its
   monomial factor) has no constant term, pick a set S of variables whose
   vanishing makes it vanish and split the cube into |S| subsectors, t_k the
   largest of S: t_j -> t_k t_j for j in S \\ {k}, Jacobian t_k^{|S|-1}.
   Strategy "X" (the Binoth-Heinrich heuristic): the smallest such S,
   lexicographically first among those of that size.  "Xrev": the
   lexicographically last smallest S, subsectors in decreasing k.  "M": the S on
   which a polynomial without constant term vanishes to the highest order
   (order = min over its monomials of the sum of the exponents of the variables
   in S), ties to the smaller S, then lexicographically first.  "R": as "M" but
   looking only at the last polynomial (F) and ranking by order / |S|.  X loops
   forever on the planar double box; M and R terminate on every workload here.
   All are valid decompositions; their sector sums must agree.
3. Pole subtraction: a variable with exponent t^{-1-p+b eps} (p >= 0) is split as
      int_0^1 t^{-1-p+b eps} G dt = int_0^1 t^{-1-p+b eps} [G - sum_{k<=p} t^k G^(k)(0)/k!] dt
                                   + sum_{k<=p} G^(k)(0) / (k! (k - p + b eps)).
4. Epsilon expansion: t^{b eps} = exp(b eps log t) and
   prod P_i^{a_i + c_i eps} = prod P_i^{a_i} exp(eps sum c_i log P_i) are expanded,
   the coefficient of eps^K collected, giving the integrand of unit (sector, K).

Exponents are kept exactly as integer pairs (c, b) meaning c + b*eps.
"""
from __future__ import annotations

import dataclasses
import itertools
import math
from fractions import Fraction

import sympy as sp

EPS_MAX_DEPTH = 64


@dataclasses.dataclass
class Sector:
    primary: int                 # 1-based index l of the primary sector (0 for direct input)
    variables: tuple             # original 1-based indices of the integration variables, ascending
    coef: sp.Rational
    mono: dict                   # j -> (c_j, b_j): factor t_j^{c_j + b_j eps}
    polys: list                  # [(sympy Poly in t-symbols, (a0, a1))] factor P^{a0 + a1 eps}
    log_factor: tuple = ()       # ((poly index, power),) extra log(P)^power factors (direct input)
    path: tuple = ()             # decomposition history, for comparisons


def tsym(j):
    return sp.Symbol(f"t{j}")


def _factor_monomials(sec: Sector):
    """Pull the monomial gcd out of every polynomial into the t-exponents."""
    new = []
    for P, (a0, a1) in sec.polys:
        gens = P.gens
        monoms = P.monoms()
        mins = [min(m[i] for m in monoms) for i in range(len(gens))]
        if any(mins):
            div = sp.Integer(1)
            for g, e in zip(gens, mins):
                div *= g ** e
            q, r = sp.div(P, sp.Poly(div, *gens))
            assert r.is_zero
            P = q
            for g, e in zip(gens, mins):
                if e:
                    j = int(str(g)[1:])
                    c, b = sec.mono[j]
                    sec.mono[j] = (c + e * a0, b + e * a1)
        new.append((P, (a0, a1)))
    sec.polys = new


def _has_constant(P):
    return P.as_expr().subs({g: 0 for g in P.gens}) != 0


def _vanishes(P, S):
    return sp.expand(P.as_expr().subs({tsym(j): 0 for j in S})) == 0


def _order(P, S):
    """Vanishing order of P on the coordinate subspace t_j = 0 (j in S)."""
    return min(sum(m[P.gens.index(tsym(j))] for j in S) for m in P.monoms())


def _choose_set(sec: Sector, strategy: str):
    """The set S of the next split; returns (S, reverse-subsector-order)."""
    bad = [P for P, _ in sec.polys if not _has_constant(P)]
    vs = list(sec.variables)
    if strategy in ("X", "Xrev"):
        for size in range(1, len(vs) + 1):
            cands = [S for S in itertools.combinations(vs, size)
                     if any(_vanishes(P, S) for P in bad)]
            if cands:
                return (cands[0], False) if strategy == "X" else (cands[-1], True)
        raise RuntimeError("no vanishing set found")
    if strategy in ("M", "R"):
        best = None
        for size in range(1, len(vs) + 1):
            for S in itertools.combinations(vs, size):
                pool = bad
                if strategy == "R":
                    # R: prefer the last polynomial (F) while it lacks a constant term
                    pool = [bad[-1]]
                for P in pool:
                    if not _vanishes(P, S):
                        continue
                    o = _order(P, S)
                    key = (-o, size, S) if strategy == "M" else (-Fraction(o, size), size, S)
                    if best is None or key < best[0]:
                        best = (key, S)
        if best is None:
            raise RuntimeError("no vanishing set found")
        return best[1], False
    raise ValueError(f"unknown strategy {strategy}")


def _split(sec: Sector, S, k):
    """Subsector where t_k is the largest of S: t_j -> t_k t_j for j in S, j != k."""
    tk = tsym(k)
    subs = {tsym(j): tk * tsym(j) for j in S if j != k}
    polys = []
    for P, ex in sec.polys:
        e = sp.expand(P.as_expr().subs(subs, simultaneous=True))
        polys.append((sp.Poly(e, *P.gens), ex))
    mono = dict(sec.mono)
    ck, bk = mono[k]
    for j in S:
        if j != k:
            c, b = sec.mono[j]
            ck += c
            bk += b
    ck += len(S) - 1          # Jacobian t_k^{|S|-1}
    mono[k] = (ck, bk)
    return Sector(sec.primary, sec.variables, sec.coef, mono, polys,
                  sec.log_factor, sec.path + ((tuple(S), k),))


def decompose(sec: Sector, strategy="M", depth=0):
    """Iterated decomposition; returns the list of resolved sectors in a fixed order."""
    if depth > EPS_MAX_DEPTH:
        raise RuntimeError("sector decomposition did not terminate")
    _factor_monomials(sec)
    if all(_has_constant(P) for P, _ in sec.polys):
        return [sec]
    S, rev = _choose_set(sec, strategy)
    out = []
    for k in (sorted(S, reverse=True) if rev else sorted(S)):
        out.extend(decompose(_split(sec, S, k), strategy, depth + 1))
    return out


def primary_sectors(U, F, xs, indices, loops):
    """Primary sectors of Eq. 2: x_l = 1, x_j = t_j; exponents of U and F from d = 4 - 2 eps."""
    n = len(xs)
    A = sum(indices)
    L = loops
    # U^{A-(L+1)d/2}: A - 2(L+1) + (L+1) eps;  F^{-(A - L d/2)}: -(A - 2L) - L eps
    aU = (A - 2 * (L + 1), L + 1)
    aF = (-(A - 2 * L), -L)
    out = []
    for l in range(1, n + 1):
        var = tuple(j for j in range(1, n + 1) if j != l)
        gens = [tsym(j) for j in var]
        subs = {xs[l - 1]: 1}
        subs.update({xs[j - 1]: tsym(j) for j in var})
        Ul = sp.Poly(sp.expand(U.subs(subs, simultaneous=True)), *gens)
        Fl = sp.Poly(sp.expand(F.subs(subs, simultaneous=True)), *gens)
        mono = {j: (indices[j - 1] - 1, 0) for j in var}
        out.append(Sector(l, var, sp.Integer(1), mono, [(Ul, aU), (Fl, aF)]))
    return out


def direct_sector(problem):
    """A DirectProblem as a single sector over [0,1]^dim (variables 1..dim)."""
    var = tuple(range(1, problem.dim + 1))
    gens = [tsym(j) for j in var]
    polys = []
    for f in problem.factors:
        e = sum(sp.Float(c, 30) * sp.Mul(*[g ** k for g, k in zip(gens, ex)]) for c, ex in f.terms)
        e = sum(sp.Rational(Fraction(c)) * sp.Mul(*[g ** k for g, k in zip(gens, ex)]) for c, ex in f.terms)
        polys.append((sp.Poly(e, *gens), (f.n, f.m)))
    mono = {j: (problem.monomial[j - 1], 0) for j in var}
    logf = ((0, problem.log_power),) if problem.log_power else ()
    return Sector(0, var, sp.Integer(1), mono, polys, logf)


# ---------------------------------------------------------------------------
# Pole subtraction and epsilon expansion
# ---------------------------------------------------------------------------

def _series_mul(a, b, kmax):
    """Multiply two truncated Laurent series given as {power: coeff}."""
    out = {}
    for i, x in a.items():
        for j, y in b.items():
            if i + j <= kmax:
                out[i + j] = out.get(i + j, 0) + x * y
    return out


def singular_vars(sec: Sector):
    S = []
    for j in sec.variables:
        c, b = sec.mono[j]
        if c <= -1:
            if b == 0:
                raise ValueError(f"unregulated singularity in t{j}")
            S.append(j)
    return tuple(S)


def min_order(sec: Sector):
    return -len(singular_vars(sec))


def deformation(sec: Sector, lam, poly_index=-1):
    """Contour deformation of the sector variables (physical kinematics).

    With F the sector's polynomial ``sec.polys[poly_index]``, z_j = t_j - i lam
    t_j (1 - t_j) dF/dt_j; the deformation vanishes on the faces t_j = 0, 1, so the
    integral over the cube is unchanged (Cauchy) while Im F(z) <= 0 for small lam
    enforces the F - i0 prescription of the propagators (Sec. 1, Eq. 1).  Returns
    (z, w, detJ): z_j, w_j = z_j / t_j = 1 - i lam (1 - t_j) dF/dt_j, det dz/dt.
    """
    t = [tsym(j) for j in sec.variables]
    F = sec.polys[poly_index][0].as_expr()
    z, w = {}, {}
    for j, tj in zip(sec.variables, t):
        dF = sp.diff(F, tj)
        w[j] = 1 - sp.I * lam * (1 - tj) * dF
        z[j] = tj * w[j]
    J = sp.Matrix([[sp.diff(z[j], tk) for tk in t] for j in sec.variables])
    return z, w, sp.expand(J.det())


def unit_integrand(sec: Sector, K: int, lam=None, term=None):
    """The sympy expression of the eps^K coefficient of the subtracted sector integrand.

    Variables not integrated analytically keep their t-dependence; variables whose
    pole term was taken appear not at all (the integrand is constant along them).
    The expression is a sum over the subsets T of the singular variables whose pole
    term is taken; each such term is integrable on its own (the paper's SeparateTerms
    option, Sec. 4.4, hands them to the integrator one by one): ``term`` = T (a tuple
    of variables, a subset of ``singular_vars``) keeps that term only.
    With ``lam`` the contour is deformed (``deformation``): the integrand
    prod_j z_j^{c_j + b_j eps} G(z) det J equals prod_j t_j^{c_j + b_j eps} times
    [prod_j w_j^{c_j + b_j eps} G(z) det J], and the bracket takes the place of G
    in the subtraction and the expansion; the result is complex.
    """
    S = singular_vars(sec)
    if K < -len(S):
        return sp.Integer(0)
    wanted = None if term is None else tuple(sorted(term))
    t = {j: tsym(j) for j in sec.variables}
    # G_n = prod P^{a0} * extra logs * L^n / n!,  L = sum a1 log P
    G0 = sp.Integer(1)
    Lsum = sp.Integer(0)
    if lam is not None:
        z, w, detJ = deformation(sec, lam)
        zsub = {t[j]: z[j] for j in sec.variables}
        G0 = detJ
        for j in sec.variables:
            c, b = sec.mono[j]
            G0 = G0 * w[j] ** c
            if b:
                Lsum = Lsum + b * sp.log(w[j])
    else:
        zsub = {}
    for P, (a0, a1) in sec.polys:
        e = P.as_expr().subs(zsub, simultaneous=True) if zsub else P.as_expr()
        G0 = G0 * e ** a0
        if a1:
            Lsum = Lsum + a1 * sp.log(e)
    for idx, power in sec.log_factor:
        e = sec.polys[idx][0].as_expr()
        e = e.subs(zsub, simultaneous=True) if zsub else e
        G0 = G0 * sp.log(e) ** power
    # highest eps power any factor may need: K plus the poles it can multiply
    nmax = K + len(S)
    Gn = [G0 * Lsum ** n / math.factorial(n) for n in range(nmax + 1)]

    total = sp.Integer(0)
    for r in range(len(S) + 1):
        for T in itertools.combinations(S, r):
            if wanted is not None and tuple(sorted(T)) != wanted:
                continue
            rest = [j for j in S if j not in T]
            ptuples = [range(-sec.mono[j][0]) for j in T]   # k = 0..p_j  (p_j = -1 - c_j)
            for ks in itertools.product(*ptuples):
                # coefficient series prod_{j in T} 1/(k! (k - p + b eps))
                coef = {0: sp.Integer(1)}
                for j, k in zip(T, ks):
                    c, b = sec.mono[j]
                    p = -1 - c
                    if k == p:
                        s = {-1: sp.Rational(1, math.factorial(p) * b)}
                    else:
                        q = k - p
                        s = {m: sp.Rational(1, math.factorial(k) * q) * sp.Rational(-b, q) ** m
                             for m in range(0, K + len(S) + 2)}
                    coef = _series_mul(coef, s, K + len(S))
                # t^{b eps} series for the non-analytic variables
                for j in sec.variables:
                    if j in T:
                        continue
                    c, b = sec.mono[j]
                    if b:
                        s = {m: (b * sp.log(t[j])) ** m / math.factorial(m)
                             for m in range(0, K + len(S) + 2)}
                        coef = _series_mul(coef, s, K + len(S))
                # operator on G_n
                def op(g):
                    for j, k in zip(T, ks):
                        g = sp.diff(g, t[j], k).subs(t[j], 0) if k else g.subs(t[j], 0)
                    for j in rest:
                        p = -1 - sec.mono[j][0]
                        taylor = sum(t[j] ** k / math.factorial(k) *
                                     (sp.diff(g, t[j], k).subs(t[j], 0) if k else g.subs(t[j], 0))
                                     for k in range(p + 1))
                        g = g - taylor
                    return g
                term = sp.Integer(0)
                for m, cm in coef.items():
                    n = K - m
                    if 0 <= n <= nmax and cm != 0:
                        term += cm * op(Gn[n])
                if term == 0:
                    continue
                mon = sp.Integer(1)
                for j in sec.variables:
                    if j in T:
                        continue
                    mon *= t[j] ** sec.mono[j][0]
                total += mon * term
    return sec.coef * total
