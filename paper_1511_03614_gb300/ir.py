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
        if ca is not None and cb is not None:
            return self.add(self.c(ca * cb), acc)
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
        """a^n for an integer n.  Exponents up to 16 in magnitude become products
        (a^2k from a^k squared, a^(k+1) = a^k a; shared through the hash-consing), a
        negative one the same products of 1/a, so every power of one base shares a
        single reciprocal; larger exponents keep the POWI instruction."""
        n = int(n)
        if n == 0:
            return self.c(1.0)
        if n == 1:
            return a
        ca = self.const_value(a)
        if ca is not None:
            return self.c(ca ** n)
        if n < 0 and -n <= 16:
            return self.powi(self.inv(a), -n)
        if n == -1:
            return self.inv(a)
        if 2 <= n <= 16:
            h = self.powi(a, n // 2)
            sq = self.mul(h, h)
            return sq if n % 2 == 0 else self.mul(sq, a)
        return self._add(("powi", a, n))

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


def _children(n):
    k = n[0]
    if k in ("add", "sub", "mul", "div", "atan2"):
        return (n[1], n[2])
    if k == "fma":
        return (n[1], n[2], n[3])
    if k in ("neg", "log", "inv"):
        return (n[1],)
    if k == "powi":
        return (n[1],)
    return ()


def contract(g, outs, allow=None):
    """Fused multiply-add contraction of the nodes reachable from ``outs``: a product
    used only by one sum becomes the multiply of a fused multiply-add there,
    a*b + c -> fma(a, b, c) and c - a*k -> fma(a, -k, c) for a constant k.  The
    value changes only by the rounding of the product that is no longer made; the
    operation count of every such pair halves.  ``allow(sum_node, product_node,
    other_node)`` (original node ids) can veto a contraction.  Returns the new
    result nodes (in the same graph)."""
    nodes = g.nodes
    order, seen, stack = [], set(), list(outs)
    while stack:                                  # post-order over the live nodes
        i = stack[-1]
        if i in seen:
            stack.pop()
            continue
        pend = [a for a in _children(nodes[i]) if a not in seen]
        if pend:
            stack.extend(pend)
            continue
        seen.add(i)
        order.append(i)
        stack.pop()
    uses = {}
    for i in order:
        for a in _children(nodes[i]):
            uses[a] = uses.get(a, 0) + 1
    for o in outs:
        uses[o] = uses.get(o, 0) + 1
    new = {}

    def single_mul(orig):
        n = nodes[orig]
        return n[0] == "mul" and uses.get(orig, 0) == 1

    def ok(i, m, other):
        return allow is None or allow(i, m, other)

    for i in order:
        n = nodes[i]
        k = n[0]
        ch = [new[a] for a in _children(n)]
        if k == "add":
            a, b = n[1], n[2]
            cands = [(m, o) for m, o in ((a, b), (b, a)) if single_mul(m) and ok(i, m, o)]
            if cands:
                m, other = cands[0]
                mm = nodes[new[m]]
                if mm[0] == "mul":
                    new[i] = g.fma(mm[1], mm[2], new[other])
                    continue
            new[i] = g.add(ch[0], ch[1])
        elif k == "sub":
            a, b = n[1], n[2]
            mm = nodes[new[b]]
            if single_mul(b) and ok(i, b, a) and mm[0] == "mul" and (g.const_value(mm[1]) is not None or
                                                                   g.const_value(mm[2]) is not None):
                x, kc = (mm[2], mm[1]) if g.const_value(mm[1]) is not None else (mm[1], mm[2])
                new[i] = g.fma(x, g.c(-g.const_value(kc)), new[a])
                continue
            new[i] = g.sub(ch[0], ch[1])
        elif k == "mul":
            new[i] = g.mul(ch[0], ch[1])
        elif k == "fma":
            new[i] = g.fma(ch[0], ch[1], ch[2])
        elif k == "div":
            new[i] = g.div(ch[0], ch[1])
        elif k == "atan2":
            new[i] = g.atan2(ch[0], ch[1])
        elif k == "neg":
            new[i] = g.neg(ch[0])
        elif k == "log":
            new[i] = g.log(ch[0])
        elif k == "inv":
            new[i] = g.inv(ch[0])
        elif k == "powi":
            new[i] = g._add(("powi", ch[0], n[2]))
        else:
            new[i] = i
    return [new[o] for o in outs]


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
