"""Symanzik polynomials U and F of a Feynman integral (Eq. 2 of the paper; the
``UF`` constructor of Sec. 4.3).

Propagators are given as -E_i, each of the form  s * (linear combination of
momenta)**2 [+ constant].  With P_i = -E_i,

    sum_i x_i P_i = -( sum_ab M_ab k_a.k_b + 2 sum_a Q_a.k_a + J ),

and U = det M, F = Q^T adj(M) Q - J U with external scalar products replaced by
their kinematic values.
"""
from __future__ import annotations

import re
from fractions import Fraction

from .poly import padd, pmul, pscale, pvar, det, adjugate

_TERM = re.compile(r"\s*([+-]?)\s*(\d*)\s*\*?\s*([A-Za-z_]\w*)")


def _lincomb(text):
    """'k1+p1-2*p2' -> {'k1': 1, 'p1': 1, 'p2': -2}."""
    out = {}
    pos = 0
    text = text.strip()
    while pos < len(text):
        m = _TERM.match(text, pos)
        if not m or m.end() == pos:
            raise ValueError(f"cannot parse momentum combination {text!r}")
        sign = -1 if m.group(1) == "-" else 1
        mult = int(m.group(2)) if m.group(2) else 1
        out[m.group(3)] = out.get(m.group(3), 0) + sign * mult
        pos = m.end()
    return {k: v for k, v in out.items() if v}


_PROP = re.compile(r"^\s*([+-]?)\s*(?:\((.*)\)|([A-Za-z_]\w*))\s*\*\*\s*2\s*(?:([+-])\s*(\S+))?\s*$")


def parse_propagator(text):
    """'-(k+p1)**2' -> (sign, {'k': 1, 'p1': 1}, constant)."""
    m = _PROP.match(text)
    if not m:
        raise ValueError(f"unsupported propagator form {text!r}")
    sign = -1 if m.group(1) == "-" else 1
    comb = _lincomb(m.group(2) if m.group(2) is not None else m.group(3))
    const = Fraction(0)
    if m.group(4):
        const = Fraction(m.group(5)) * (1 if m.group(4) == "+" else -1)
    return sign, comb, const


def symanzik(problem):
    """Return (U, F) as polynomials (dicts) in x_1..x_n (exponent position i <-> x_{i+1})."""
    loop = list(problem.loop_momenta)
    ext = list(problem.external_momenta)
    props = [parse_propagator(p) for p in problem.propagators]
    n = len(props)
    L = len(loop)
    kin = {tuple(sorted(k)): Fraction(v) for k, v in problem.kinematics.items()}

    def sp(a, b):
        return kin[tuple(sorted((a, b)))]

    M = [[{} for _ in range(L)] for _ in range(L)]
    # Q_a as {external name: polynomial in x}
    Q = [dict() for _ in range(L)]
    J = {}
    for i, (s, comb, const) in enumerate(props):
        xi = pvar(i, n)
        al = [comb.get(k, 0) for k in loop]
        be = {e: comb.get(e, 0) for e in ext if comb.get(e, 0)}
        for a in range(L):
            for b in range(L):
                if al[a] and al[b]:
                    M[a][b] = padd(M[a][b], pscale(xi, -s * al[a] * al[b]))
            if al[a]:
                for e, v in be.items():
                    Q[a][e] = padd(Q[a].get(e, {}), pscale(xi, -s * al[a] * v))
        ext2 = Fraction(0)
        for e1, v1 in be.items():
            for e2, v2 in be.items():
                ext2 += v1 * v2 * sp(e1, e2)
        J = padd(J, pscale(xi, -(s * ext2 + const)))
    U = det(M)
    adj = adjugate(M)
    quad = {}
    for a in range(L):
        for b in range(L):
            for e1, q1 in Q[a].items():
                for e2, q2 in Q[b].items():
                    v = sp(e1, e2)
                    if v:
                        quad = padd(quad, pscale(pmul(pmul(q1, adj[a][b]), q2), v))
    F = padd(quad, pscale(pmul(J, U), -1))
    return U, F
