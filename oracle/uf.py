"""Symanzik polynomials U and F (oracle, sympy).

Eq. 2 ("Alpha") of the paper writes a Feynman integral as a Feynman-parameter
integral of U^{A-(l+1)d/2} / F^{A-l d/2}; Sec. 4.3 (``UF``) builds U and F from
loop momenta, propagators given as -E_i and kinematic substitutions.

Textbook construction used here: with propagators P_i = -E_i,

    sum_i x_i P_i = -( k^T M k + 2 Q.k + J ),

M an l x l matrix of linear forms in x, Q a vector of linear combinations of
external momenta, J a scalar.  Then U = det M and
F = Q^T adj(M) Q - J det M, after the scalar products of external momenta are
replaced by their kinematic values.
"""
from __future__ import annotations

import itertools
import sympy as sp


def symanzik(problem):
    """Return (U, F, xs) as sympy expressions in the Feynman parameters xs = (x1..xn)."""
    loop = [sp.Symbol(k) for k in problem.loop_momenta]
    ext = [sp.Symbol(p) for p in problem.external_momenta]
    table = {str(s): s for s in loop + ext}
    props = [sp.sympify(s, locals=table) for s in problem.propagators]
    n = len(props)
    xs = sp.symbols(f"x1:{n + 1}")
    total = sp.expand(sum(x * p for x, p in zip(xs, props)))
    # total = -(k^T M k + 2 Q.k + J); read M, Q, J off the polynomial in momenta.
    neg = sp.expand(-total)
    poly = sp.Poly(neg, *loop)
    L = len(loop)
    M = sp.zeros(L, L)
    Q = [sp.Integer(0)] * L
    J = sp.Integer(0)
    for monom, coeff in poly.terms():
        deg = sum(monom)
        if deg == 2:
            idx = [i for i, e in enumerate(monom) for _ in range(e)]
            a, b = idx
            if a == b:
                M[a, a] += coeff
            else:
                M[a, b] += coeff / 2
                M[b, a] += coeff / 2
        elif deg == 1:
            a = monom.index(1)
            Q[a] += coeff / 2
        elif deg == 0:
            J += coeff
        else:
            raise ValueError("propagators must be quadratic in loop momenta")
    for i in range(L):
        for j in range(L):
            if M[i, j].free_symbols - set(xs):
                raise ValueError("masses/kinematics inside quadratic part are not supported")
    U = sp.expand(M.det())
    adj = M.adjugate()
    quad = sp.Integer(0)
    for a in range(L):
        for b in range(L):
            quad += Q[a] * adj[a, b] * Q[b]
    Fmom = sp.expand(quad - J * U)
    F = _substitute_kinematics(Fmom, ext, problem.kinematics)
    return U, sp.expand(F), xs


def _substitute_kinematics(expr, ext, kin):
    """Replace each product of two external momenta by its scalar-product value."""
    if not ext:
        return expr
    poly = sp.Poly(expr, *ext)
    out = sp.Integer(0)
    names = [str(e) for e in ext]
    for monom, coeff in poly.terms():
        if sum(monom) == 0:
            out += coeff
            continue
        if sum(monom) != 2:
            raise ValueError("F must be quadratic in external momenta")
        idx = [i for i, e in enumerate(monom) for _ in range(e)]
        key = tuple(sorted((names[idx[0]], names[idx[1]])))
        if key not in kin:
            raise ValueError(f"missing kinematic value for {key}")
        out += coeff * sp.Rational(sp.nsimplify(kin[key]))
    return out
