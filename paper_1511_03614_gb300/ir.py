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
