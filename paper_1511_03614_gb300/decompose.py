"""Primary and iterated sector decomposition (host preprocessor).

Primary sectors follow Eq. 2 of the paper: in the region where x_l is the
largest Feynman parameter, x_l = 1 and x_j = t_j in [0,1]; homogeneity of the
integrand (degree -n) makes the delta function integrate to one.  Iterated
splits resolve each polynomial into monomial x (polynomial with a non-zero
constant term): for a chosen variable set S on which a polynomial vanishes, the
cube splits into |S| pieces, t_k the largest of S, t_j -> t_k t_j (j in S, j != k)
with Jacobian t_k^{|S|-1}.

The paper defers the choice of S to the earlier FIESTA papers (Sec. 4.4,
``STRATEGY``).  Rules implemented (all give valid decompositions; the sum over
sectors does not depend on the rule):

* ``X``    smallest vanishing S, lexicographically first (Binoth-Heinrich);
* ``Xrev`` smallest vanishing S, lexicographically last, pieces in decreasing k;
* ``M``    the S of highest vanishing order of a polynomial without constant
           term (order = lowest total degree in the variables of S), then the
           smaller S, then lexicographically first;  the default, because X does
           not terminate on the planar double box;
* ``R``    like M but on the last polynomial only, ranked by order / |S|.

Exponents of the monomial prefactor are kept as pairs (c, b) meaning c + b eps.
"""
from __future__ import annotations

import dataclasses
import itertools
from fractions import Fraction

from .poly import has_constant, vanishes_on, order_on, min_exponents, divide_monomial

MAX_DEPTH = 64


@dataclasses.dataclass
class Sector:
    primary: int
    variables: tuple          # original 1-based indices, ascending; dimension i <-> variables[i]
    coef: Fraction
    mono: dict                # j -> (c, b)
    polys: list               # [(poly dict over all n positions, (a0, a1))]
    log_factor: tuple = ()    # ((poly index, power),)
    path: tuple = ()


def _normalize(sec):
    polys = []
    mono = dict(sec.mono)
    for p, (a0, a1) in sec.polys:
        e = min_exponents(p)
        if any(e):
            p = divide_monomial(p, e)
            for pos, k in enumerate(e):
                if k:
                    c, b = mono[pos + 1]
                    mono[pos + 1] = (c + k * a0, b + k * a1)
        polys.append((p, (a0, a1)))
    return dataclasses.replace(sec, mono=mono, polys=polys)


def _pick(sec, strategy):
    pos = [j - 1 for j in sec.variables]      # exponent positions of the sector variables
    bad = [p for p, _ in sec.polys if not has_constant(p)]
    if strategy in ("X", "Xrev"):
        for size in range(1, len(pos) + 1):
            found = [S for S in itertools.combinations(pos, size) if any(vanishes_on(p, S) for p in bad)]
            if found:
                S = found[0] if strategy == "X" else found[-1]
                return S, strategy == "Xrev"
        raise RuntimeError("no vanishing variable set")
    if strategy in ("M", "R"):
        pool = bad if strategy == "M" else [bad[-1]]
        best = None
        for size in range(1, len(pos) + 1):
            for S in itertools.combinations(pos, size):
                for p in pool:
                    if vanishes_on(p, S):
                        o = order_on(p, S)
                        rank = -o if strategy == "M" else -Fraction(o, size)
                        key = (rank, size, S)
                        if best is None or key < best:
                            best = key
        if best is None:
            raise RuntimeError("no vanishing variable set")
        return best[2], False
    raise ValueError(f"unknown strategy {strategy!r}")


def _blow_up(sec, S, k):
    """Piece of S where position k is the largest: t_j -> t_k t_j for j in S \\ {k}."""
    polys = []
    for p, ex in sec.polys:
        q = {}
        for m, c in p.items():
            mm = list(m)
            mm[k] = sum(m[j] for j in S)
            mm = tuple(mm)
            q[mm] = q.get(mm, 0) + c
        polys.append(({m: c for m, c in q.items() if c}, ex))
    mono = dict(sec.mono)
    ck, bk = mono[k + 1]
    for j in S:
        if j != k:
            c, b = sec.mono[j + 1]
            ck, bk = ck + c, bk + b
    mono[k + 1] = (ck + len(S) - 1, bk)
    return dataclasses.replace(sec, mono=mono, polys=polys,
                               path=sec.path + ((tuple(j + 1 for j in S), k + 1),))


def iterate(sec, strategy="M"):
    out = []
    stack = [(sec, 0)]
    # depth-first, pieces in the order the strategy gives
    def rec(s, depth):
        if depth > MAX_DEPTH:
            raise RuntimeError("sector decomposition did not terminate")
        s = _normalize(s)
        if all(has_constant(p) for p, _ in s.polys):
            out.append(s)
            return
        S, rev = _pick(s, strategy)
        for k in (sorted(S, reverse=True) if rev else sorted(S)):
            rec(_blow_up(s, S, k), depth + 1)
    rec(sec, 0)
    return out


def primary(U, F, n, indices, loops):
    A = sum(indices)
    L = loops
    aU = (A - 2 * (L + 1), L + 1)          # U^{A-(L+1)d/2}, d = 4 - 2 eps
    aF = (2 * L - A, -L)                   # F^{-(A-L d/2)}
    out = []
    for l in range(1, n + 1):
        var = tuple(j for j in range(1, n + 1) if j != l)

        def restrict(p):
            q = {}
            for m, c in p.items():
                mm = list(m)
                mm[l - 1] = 0
                mm = tuple(mm)
                q[mm] = q.get(mm, 0) + c
            return {m: c for m, c in q.items() if c}
        mono = {j: (indices[j - 1] - 1, 0) for j in var}
        out.append(Sector(l, var, Fraction(1), mono, [(restrict(U), aU), (restrict(F), aF)]))
    return out


def decompose_feynman(U, F, n, indices, loops, strategy="M"):
    return [s for p in primary(U, F, n, indices, loops) for s in iterate(p, strategy)]


def direct_sector(problem):
    dim = problem.dim
    var = tuple(range(1, dim + 1))
    polys = []
    for f in problem.factors:
        p = {}
        for c, e in f.terms:
            p[tuple(e)] = p.get(tuple(e), 0) + Fraction(c)
        polys.append(({m: c for m, c in p.items() if c}, (f.n, f.m)))
    mono = {j: (problem.monomial[j - 1], 0) for j in var}
    logf = ((0, problem.log_power),) if problem.log_power else ()
    return Sector(0, var, Fraction(1), mono, polys, logf)


def singular(sec):
    out = []
    for j in sec.variables:
        c, b = sec.mono[j]
        if c <= -1:
            if b == 0:
                raise ValueError(f"unregulated endpoint singularity in t{j}")
            out.append(j)
    return tuple(out)
