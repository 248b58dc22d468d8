"""The integrand text format of the paper's integration workers (Sec. 4.6).

An expression is a sequence of ';'-terminated lines closed by a line '|':
the number of variables, the number of intermediate functions f[1..m], one line
per intermediate function, and the final expression.  Expressions use + - * /,
brackets, decimal numbers, x[i], f[i], p[expr, exponent] (power), l[expr]
(natural log), P (pi), G (Euler's gamma) and PolyGamma[n, m] for integer
arguments.  Example from the paper: ``1; 0; x[1]+0.2; |`` integrates x + 0.2 over
[0, 1].  The result is one unit over [0,1]^n, lowered to the register bytecode.
"""
from __future__ import annotations

import math
import re

from .ir import Graph
from . import bytecode as B
from .prefactor import zeta
from .preprocess import Prepared, Unit

EULER_GAMMA = 0.57721566490153286061

_TOK = re.compile(r"\s*(?:(\d+\.\d*(?:[eE][+-]?\d+)?|\.\d+(?:[eE][+-]?\d+)?|\d+(?:[eE][+-]?\d+)?)|"
                  r"(PolyGamma|[A-Za-z]+)|(.))")


def _tokens(s):
    out = []
    pos = 0
    s = s.strip()
    while pos < len(s):
        m = _TOK.match(s, pos)
        if not m:
            raise ValueError(f"bad character at {pos} in {s!r}")
        if m.group(1) is not None:
            out.append(("num", float(m.group(1))))
        elif m.group(2) is not None:
            out.append(("id", m.group(2)))
        elif m.group(3) is not None and not m.group(3).isspace():
            out.append(("op", m.group(3)))
        pos = m.end()
    return out


def polygamma(n, m):
    """psi^(n)(m) for integers n >= 1, m >= 1: (-1)^(n+1) n! (zeta(n+1) - sum_{k<m} k^-(n+1))."""
    return (-1) ** (n + 1) * math.factorial(n) * (zeta(n + 1) - sum(k ** -(n + 1) for k in range(1, m)))


class _Parser:
    def __init__(self, g, toks, nvars, funcs):
        self.g, self.t, self.i, self.nvars, self.funcs = g, toks, 0, nvars, funcs

    def peek(self):
        return self.t[self.i] if self.i < len(self.t) else (None, None)

    def take(self, kind=None, val=None):
        tok = self.peek()
        if tok[0] is None or (kind and tok[0] != kind) or (val is not None and tok[1] != val):
            raise ValueError(f"expected {val or kind}, got {tok}")
        self.i += 1
        return tok

    def expr(self):
        v = self.term()
        while self.peek() in (("op", "+"), ("op", "-")):
            op = self.take()[1]
            r = self.term()
            v = self.g.add(v, r) if op == "+" else self.g.sub(v, r)
        return v

    def term(self):
        v = self.unary()
        while self.peek() in (("op", "*"), ("op", "/")):
            op = self.take()[1]
            r = self.unary()
            v = self.g.mul(v, r) if op == "*" else self.g.div(v, r)
        return v

    def unary(self):
        if self.peek() == ("op", "-"):
            self.take()
            return self.g.neg(self.unary())
        if self.peek() == ("op", "+"):
            self.take()
            return self.unary()
        return self.atom()

    def _index(self):
        self.take("op", "[")
        k = self.take("num")[1]
        self.take("op", "]")
        if k != int(k):
            raise ValueError("index must be an integer")
        return int(k)

    def atom(self):
        kind, val = self.peek()
        if kind == "num":
            self.take()
            return self.g.c(val)
        if kind == "op" and val == "(":
            self.take()
            v = self.expr()
            self.take("op", ")")
            return v
        if kind == "id":
            self.take()
            if val == "x":
                k = self._index()
                if not 1 <= k <= self.nvars:
                    raise ValueError(f"x[{k}] out of range")
                return self.g.x(k - 1)
            if val == "f":
                k = self._index()
                if k not in self.funcs:
                    raise ValueError(f"f[{k}] used before it is defined")
                return self.funcs[k]
            if val == "P":
                return self.g.c(math.pi)
            if val == "G":
                return self.g.c(EULER_GAMMA)
            if val == "l":
                self.take("op", "[")
                v = self.expr()
                self.take("op", "]")
                return self.g.log(v)
            if val == "p":
                self.take("op", "[")
                base = self.expr()
                self.take("op", ",")
                ex = self.expr()
                self.take("op", "]")
                e = self.g.const_value(ex)
                if e is None or e != int(e):
                    raise ValueError("p[expr, exponent] needs an integer constant exponent")
                return self.g.powi(base, int(e))
            if val == "PolyGamma":
                self.take("op", "[")
                n = self.take("num")[1]
                self.take("op", ",")
                m = self.take("num")[1]
                self.take("op", "]")
                return self.g.c(polygamma(int(n), int(m)))
        raise ValueError(f"unexpected token {kind} {val!r}")


def parse(text, name="text"):
    """Parse one integrand in the paper's text format into a single-unit Prepared."""
    body = text.strip()
    if not body.endswith("|"):
        raise ValueError("expression must end with a line '|'")
    lines = [l.strip() for l in body[:-1].split(";")]
    lines = [l for l in lines if l]
    if len(lines) < 3:
        raise ValueError("need the number of variables, of functions and an expression")
    nvars, nfun = int(lines[0]), int(lines[1])
    if len(lines) != 3 + nfun:
        raise ValueError(f"expected {nfun} function lines")
    if not 1 <= nvars <= 8:
        raise ValueError("1..8 variables supported")
    g = Graph()
    funcs = {}
    for k in range(nfun):
        funcs[k + 1] = _Parser(g, _tokens(lines[2 + k]), nvars, funcs).expr()
    p = _Parser(g, _tokens(lines[-1]), nvars, funcs)
    out = p.expr()
    if p.i != len(p.t):
        raise ValueError("trailing tokens in expression")
    prog = B.emit(g, out, nvars)
    return Prepared(name, [Unit(0, 0, nvars, prog, 0)], (0, [1.0]), (0,), (0,), [])
