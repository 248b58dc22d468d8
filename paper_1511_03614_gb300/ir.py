"""Expression DAG with hash-consing, the intermediate form between the
expanded sector integrands and the register bytecode.

The paper's integrator turns each integrand string into a list of quadruples
(operator, first operand, second operand, result) and loops over them per point
(Sec. 2.1); this DAG is the common-subexpression-free form from which such a
straight-line list is emitted.
"""
from __future__ import annotations

import math


class Graph:
    """Nodes are tuples (kind, args...); ``ids`` maps a node to its index."""

    def __init__(self):
        self.nodes = []
        self.ids = {}

    def _add(self, node):
        i = self.ids.get(node)
        if i is None:
            i = len(self.nodes)
            self.nodes.append(node)
            self.ids[node] = i
        return i

    # leaves
    def x(self, j):
        return self._add(("x", j))

    def c(self, v):
        v = float(v)
        if v == 0.0:
            v = 0.0                      # fold -0.0
        return self._add(("c", v))

    def const_value(self, i):
        n = self.nodes[i]
        return n[1] if n[0] == "c" else None

    # arithmetic with folding of neutral elements
    def add(self, a, b):
        ca, cb = self.const_value(a), self.const_value(b)
        if ca is not None and cb is not None:
            return self.c(ca + cb)
        if ca == 0.0:
            return b
        if cb == 0.0:
            return a
        if a > b:
            a, b = b, a
        return self._add(("add", a, b))

    def sub(self, a, b):
        ca, cb = self.const_value(a), self.const_value(b)
        if ca is not None and cb is not None:
            return self.c(ca - cb)
        if cb == 0.0:
            return a
        if ca == 0.0:
            return self.neg(b)
        if a == b:
            return self.c(0.0)
        return self._add(("sub", a, b))

    def mul(self, a, b):
        ca, cb = self.const_value(a), self.const_value(b)
        if ca is not None and cb is not None:
            return self.c(ca * cb)
        if ca == 0.0 or cb == 0.0:
            return self.c(0.0)
        if ca == 1.0:
            return b
        if cb == 1.0:
            return a
        if ca == -1.0:
            return self.neg(b)
        if cb == -1.0:
            return self.neg(a)
        if a > b:
            a, b = b, a
        return self._add(("mul", a, b))

    def fma(self, a, b, acc):
        """a*b + acc"""
        if self.const_value(acc) == 0.0:
            return self.mul(a, b)
        ca, cb = self.const_value(a), self.const_value(b)
        if ca == 0.0 or cb == 0.0:
            return acc
        if ca == 1.0:
            return self.add(b, acc)
        if cb == 1.0:
            return self.add(a, acc)
        if ca is not None and cb is None:
            a, b = b, a
        return self._add(("fma", a, b, acc))

    def div(self, a, b):
        cb = self.const_value(b)
        if cb is not None:
            return self.mul(a, self.c(1.0 / cb)) if cb in (1.0, 2.0, 4.0, 0.5, 0.25, -1.0) else \
                self._add(("div", a, b))
        return self._add(("div", a, b))

    def inv(self, a):
        ca = self.const_value(a)
        if ca is not None:
            return self.c(1.0 / ca)
        return self._add(("inv", a))

    def neg(self, a):
        ca = self.const_value(a)
        if ca is not None:
            return self.c(-ca)
        n = self.nodes[a]
        if n[0] == "neg":
            return n[1]
        return self._add(("neg", a))

    def powi(self, a, n):
        if n == 0:
            return self.c(1.0)
        if n == 1:
            return a
        ca = self.const_value(a)
        if ca is not None:
            return self.c(ca ** n)
        if n == 2:
            return self.mul(a, a)
        if n == -1:
            return self.inv(a)
        return self._add(("powi", a, int(n)))

    def log(self, a):
        ca = self.const_value(a)
        if ca is not None:
            return self.c(math.log(ca))
        return self._add(("log", a))

    def atan2(self, y, x):
        cy, cx = self.const_value(y), self.const_value(x)
        if cy is not None and cx is not None:
            return self.c(math.atan2(cy, cx))
        return self._add(("atan2", y, x))

    def sum(self, items):
        out = self.c(0.0)
        for i in items:
            out = self.add(out, i)
        return out

    def prod(self, items):
        out = self.c(1.0)
        for i in items:
            out = self.mul(out, i)
        return out


# ---------------------------------------------------------------------------
# Complex values as pairs (re, im) of real nodes.  A constant zero imaginary part
# folds away, so purely real computations cost nothing extra.
# ---------------------------------------------------------------------------

def cconst(g, re, im=0.0):
    return (g.c(re), g.c(im))


def creal(g, x):
    return (x, g.c(0.0))


def cadd(g, x, y):
    return (g.add(x[0], y[0]), g.add(x[1], y[1]))


def csub(g, x, y):
    return (g.sub(x[0], y[0]), g.sub(x[1], y[1]))


def cmul(g, x, y):
    return (g.sub(g.mul(x[0], y[0]), g.mul(x[1], y[1])), g.fma(x[0], y[1], g.mul(x[1], y[0])))


def cscale(g, x, r):
    """complex x times real node r"""
    return (g.mul(x[0], r), g.mul(x[1], r))


def cfma(g, x, y, acc):
    """x * y + acc"""
    re = g.sub(g.fma(x[0], y[0], acc[0]), g.mul(x[1], y[1]))
    im = g.fma(x[0], y[1], g.fma(x[1], y[0], acc[1]))
    return (re, im)


def cinv(g, x):
    if g.const_value(x[1]) == 0.0:
        return (g.inv(x[0]), g.c(0.0))
    d = g.fma(x[0], x[0], g.mul(x[1], x[1]))
    r = g.inv(d)
    return (g.mul(x[0], r), g.neg(g.mul(x[1], r)))


def cpowi(g, x, n):
    if g.const_value(x[1]) == 0.0:
        return (g.powi(x[0], n), g.c(0.0))
    if n == 0:
        return cconst(g, 1.0)
    m = abs(n)
    out, base = None, x
    while m:
        if m & 1:
            out = base if out is None else cmul(g, out, base)
        m >>= 1
        if m:
            base = cmul(g, base, base)
    return cinv(g, out) if n < 0 else out


def clog(g, x):
    """Principal logarithm; a value with a constant zero imaginary part is taken as positive."""
    if g.const_value(x[1]) == 0.0:
        return (g.log(x[0]), g.c(0.0))
    m2 = g.fma(x[0], x[0], g.mul(x[1], x[1]))
    return (g.mul(g.log(m2), g.c(0.5)), g.atan2(x[1], x[0]))
