"""Pole subtraction and epsilon expansion of a resolved sector into the
straight-line integrand of each unit (sector, eps order K).

The paper's summary names this step "pole resolution and epsilon expansion"
and leaves its detail to the earlier FIESTA papers.  A resolved sector is

    coef * prod_j t_j^{c_j + b_j eps} * G(t, eps),   G = prod_i P_i^{a_i + a'_i eps} * extra logs,

with every P_i(0) != 0.  For the variables S with c_j = -1 the standard
subtraction at t_j = 0 gives

    int_0^1 t^{-1+b eps} G dt = int_0^1 t^{-1+b eps} (G - G|_{t=0}) dt + G|_{t=0} / (b eps).

Writing G = sum_N eps^N G_N with G_N = prod P_i^{a_i} * logs * L^N / N!,
L = sum_i a'_i log P_i, and t^{b eps} = sum_m (b log t)^m eps^m / m!, the
coefficient of eps^K is

    f_K = coef * prod_{j not in S} t_j^{c_j}
          * sum_{T subset S} prod_{j in T} 1/b_j * prod_{j in S\\T} 1/t_j
          * sum_{m=0}^{K+|T|} lambda_T^m / m! * D_{T, K+|T|-m},

    lambda_T = sum_{j not in T} b_j log t_j,
    D_{T,N}  = sum_{Z subset S\\T} (-1)^{|Z|} G_N evaluated with t_{T u Z} = 0.

T are the variables integrated analytically (their pole term); the integrand is
constant along them.
"""
from __future__ import annotations

import itertools
import math

from .ir import Graph
from .decompose import singular


def _subsets(seq):
    seq = tuple(seq)
    for r in range(len(seq) + 1):
        for c in itertools.combinations(seq, r):
            yield c


class _SectorEval:
    """Shared pieces of one sector's integrands inside one Graph."""

    def __init__(self, g: Graph, sec):
        self.g = g
        self.sec = sec
        self.pos = {j: i for i, j in enumerate(sec.variables)}   # variable -> x index
        self.S = singular(sec)
        self._pow = {}
        self._mono = {}
        self._corner = {}
        self._logt = {}

    def t(self, j):
        return self.g.x(self.pos[j])

    def tpow(self, j, e):
        key = (j, e)
        if key not in self._pow:
            if e == 1:
                self._pow[key] = self.t(j)
            elif e % 2 == 0:
                h = self.tpow(j, e // 2)
                self._pow[key] = self.g.mul(h, h)
            else:
                self._pow[key] = self.g.mul(self.tpow(j, e - 1), self.t(j))
        return self._pow[key]

    def monomial(self, m):
        """t^m for an exponent tuple over all positions (position j-1 <-> variable j)."""
        key = tuple(m)
        if key not in self._mono:
            out = self.g.c(1.0)
            for p, e in enumerate(m):
                if e:
                    out = self.g.mul(out, self.tpow(p + 1, e))
            self._mono[key] = out
        return self._mono[key]

    def poly_at(self, i, W):
        """P_i with the variables W set to 0, as a node (monomials grouped by their support in S)."""
        key = ("P", i, W)
        if key in self._corner:
            return self._corner[key]
        p = self.sec.polys[i][0]
        Sset = set(self.S)
        groups = {}
        for m, c in p.items():
            supp = tuple(sorted(j for j in Sset if m[j - 1]))
            if any(j in W for j in supp):
                continue
            groups.setdefault(supp, []).append((m, c))
        parts = []
        for supp in sorted(groups):
            gkey = ("Q", i, supp)
            if gkey not in self._corner:
                acc = self.g.c(0.0)
                for m, c in sorted(groups[supp]):
                    acc = self.g.fma(self.monomial(m), self.g.c(float(c)), acc)
                self._corner[gkey] = acc
            parts.append(self._corner[gkey])
        node = self.g.sum(parts)
        self._corner[key] = node
        return node

    def logpoly_at(self, i, W):
        key = ("logP", i, W)
        if key not in self._corner:
            self._corner[key] = self.g.log(self.poly_at(i, W))
        return self._corner[key]

    def G_at(self, N, W):
        """G_N with t_W = 0."""
        key = ("G", N, W)
        if key in self._corner:
            return self._corner[key]
        g = self.g
        if N == 0:
            out = g.c(1.0)
            for i, (p, (a0, a1)) in enumerate(self.sec.polys):
                if a0:
                    out = g.mul(out, g.powi(self.poly_at(i, W), a0))
            for i, power in self.sec.log_factor:
                out = g.mul(out, g.powi(self.logpoly_at(i, W), power))
        else:
            L = g.c(0.0)
            for i, (p, (a0, a1)) in enumerate(self.sec.polys):
                if a1:
                    L = g.fma(self.logpoly_at(i, W), g.c(float(a1)), L)
            if g.const_value(L) == 0.0:
                out = g.c(0.0)
            else:
                out = g.mul(g.mul(self.G_at(N - 1, W), L), g.c(1.0 / N))
        self._corner[key] = out
        return out

    def D(self, T, N):
        """sum over Z subset S\\T of (-1)^|Z| G_N(t_{T u Z} = 0), by successive differences."""
        key = ("D", T, N)
        if key in self._corner:
            return self._corner[key]
        rest = [j for j in self.S if j not in T]

        def diff(k, W):
            if k == len(rest):
                return self.G_at(N, tuple(sorted(W)))
            j = rest[k]
            return self.g.sub(diff(k + 1, W), diff(k + 1, W + (j,)))
        out = diff(0, tuple(T))
        self._corner[key] = out
        return out

    def logt(self, j):
        if j not in self._logt:
            self._logt[j] = self.g.log(self.t(j))
        return self._logt[j]

    def unit(self, K):
        """Node of f_K; None when f_K is identically zero."""
        g = self.g
        sec = self.sec
        S = self.S
        total = g.c(0.0)
        for T in _subsets(S):
            top = K + len(T)
            if top < 0:
                continue
            lam = g.c(0.0)
            for j in sec.variables:
                b = sec.mono[j][1]
                if j not in T and b:
                    lam = g.fma(self.logt(j), g.c(float(b)), lam)
            inner = g.c(0.0)
            lam_pow = g.c(1.0)
            for m in range(0, top + 1):
                if m:
                    if g.const_value(lam) == 0.0:
                        break
                    lam_pow = g.mul(g.mul(lam_pow, lam), g.c(1.0 / m))
                Dn = self.D(T, top - m)
                if g.const_value(Dn) == 0.0:
                    continue
                inner = g.fma(lam_pow, Dn, inner)
            if g.const_value(inner) == 0.0:
                continue
            fac = 1.0
            for j in T:
                fac /= sec.mono[j][1]
            term = g.mul(inner, g.c(fac))
            for j in S:
                if j not in T:
                    term = g.mul(term, g.inv(self.t(j)))
            total = g.add(total, term)
        if g.const_value(total) == 0.0:
            return None
        mono = g.c(float(sec.coef))
        for j in sec.variables:
            if j in S:
                continue
            c = sec.mono[j][0]
            if c:
                mono = g.mul(mono, g.powi(self.t(j), c))
        return g.mul(total, mono)


def unit_graph(sec, K):
    """(Graph, output node) for the unit (sec, K), or None if f_K == 0."""
    g = Graph()
    ev = _SectorEval(g, sec)
    out = ev.unit(K)
    if out is None:
        return None
    return g, out


def min_order(sec):
    return -len(singular(sec))


def sector_graph(sec, orders):
    """(Graph, result nodes) with the integrands of every order in ``orders`` of one
    sector in a single graph (shared subexpressions); identically-zero orders give a
    constant 0 result."""
    g = Graph()
    ev = _SectorEval(g, sec)
    outs = []
    for K in orders:
        node = ev.unit(K) if K >= -len(ev.S) else None
        outs.append(g.c(0.0) if node is None else node)
    return g, outs
