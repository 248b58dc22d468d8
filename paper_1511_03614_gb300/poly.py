"""Sparse multivariate polynomials with exact rational coefficients.

A polynomial is a dict mapping exponent tuples to ``fractions.Fraction`` (or
float for numerically given input).  Variables are positional: exponent tuple
position i is variable i of whatever numbering the caller uses.
"""
from __future__ import annotations

from fractions import Fraction


def padd(a, b):
    out = dict(a)
    for m, c in b.items():
        v = out.get(m, 0) + c
        if v:
            out[m] = v
        else:
            out.pop(m, None)
    return out


def pscale(a, s):
    return {m: c * s for m, c in a.items() if c * s} if s else {}


def pmul(a, b):
    out = {}
    for m1, c1 in a.items():
        for m2, c2 in b.items():
            m = tuple(x + y for x, y in zip(m1, m2))
            v = out.get(m, 0) + c1 * c2
            if v:
                out[m] = v
            else:
                out.pop(m, None)
    return out


def pconst(c, n):
    return {tuple([0] * n): Fraction(c)} if c else {}


def pvar(i, n):
    e = [0] * n
    e[i] = 1
    return {tuple(e): Fraction(1)}


def min_exponents(p):
    n = len(next(iter(p)))
    return [min(m[i] for m in p) for i in range(n)]


def divide_monomial(p, e):
    return {tuple(x - y for x, y in zip(m, e)): c for m, c in p.items()}


def has_constant(p):
    n = len(next(iter(p)))
    return tuple([0] * n) in p


def vanishes_on(p, S):
    """True if p is identically zero when every variable in S is set to 0."""
    return all(any(m[j] for j in S) for m in p)


def order_on(p, S):
    """Lowest total degree in the variables of S over the monomials of p."""
    return min(sum(m[j] for j in S) for m in p)


def det(mat):
    """Determinant of a small square matrix of polynomials (Laplace expansion)."""
    n = len(mat)
    if n == 1:
        return mat[0][0]
    out = {}
    for j in range(n):
        if not mat[0][j]:
            continue
        minor = [row[:j] + row[j + 1:] for row in mat[1:]]
        term = pmul(mat[0][j], det(minor))
        out = padd(out, term if j % 2 == 0 else pscale(term, -1))
    return out


def adjugate(mat):
    n = len(mat)
    if n == 1:
        return [[pconst(1, len(next(iter(mat[0][0]))) if mat[0][0] else 0)]]
    adj = [[None] * n for _ in range(n)]
    for i in range(n):
        for j in range(n):
            minor = [row[:j] + row[j + 1:] for k, row in enumerate(mat) if k != i]
            c = det(minor)
            adj[j][i] = c if (i + j) % 2 == 0 else pscale(c, -1)
    return adj


def pderiv(p, i):
    """Derivative with respect to exponent position i."""
    out = {}
    for m, c in p.items():
        if m[i]:
            mm = list(m)
            mm[i] -= 1
            mm = tuple(mm)
            out[mm] = out.get(mm, 0) + c * m[i]
    return {m: c for m, c in out.items() if c}
