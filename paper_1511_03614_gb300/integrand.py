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

    def __init__(self, g: Graph, sec, variables=None):
        self.g = g
        self.sec = sec
        # variable -> x index (a separate term is a function of fewer variables)
        self.pos = {j: i for i, j in enumerate(variables if variables is not None else sec.variables)}
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

    def _pow_at(self, i, W, e):
        """P_i^e with t_W = 0 for an integer e."""
        return self.g.powi(self.poly_at(i, W), int(e))

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
                    out = g.mul(out, self._pow_at(i, W, a0) if float(a0).is_integer()
                                else g.powi(self.poly_at(i, W), a0))
            for i, power in self.sec.log_factor:
                out = g.mul(out, g.powi(self.logpoly_at(i, W), power))
        else:
            L = self.L_at(W)
            if g.const_value(L) == 0.0:
                out = g.c(0.0)
            else:
                out = g.mul(g.mul(self.G_at(N - 1, W), L), g.c(1.0 / N))
        self._corner[key] = out
        return out

    def L_at(self, W):
        """L = sum_i a'_i log P_i at t_W = 0.  With integer a'_i (integer indices in
        d = 4 - 2 eps) this is one logarithm, log prod_i P_i^a'_i, instead of one per
        polynomial: the P_i are positive and bounded away from 0 and infinity on the
        cube (each has a constant term, all coefficients positive when F > 0), so the
        product stays in range, and its rounding error (a few u, relative) becomes the
        same absolute error in L as the sum of logarithms carries."""
        key = ("L", W)
        if key in self._corner:
            return self._corner[key]
        g = self.g
        terms = [(i, a1) for i, (p, (a0, a1)) in enumerate(self.sec.polys) if a1]
        if terms and not self.sec.log_factor and all(float(a1).is_integer() for _, a1 in terms) and \
                all(c > 0 for p, _ in self.sec.polys for c in p.values()):
            prod = g.c(1.0)
            for i, a1 in terms:
                prod = g.mul(prod, self._pow_at(i, W, a1))
            L = g.log(prod)
        else:
            L = g.c(0.0)
            for i, a1 in terms:
                L = g.fma(self.logpoly_at(i, W), g.c(float(a1)), L)
        self._corner[key] = L
        return L

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

    def unit(self, K, only=None):
        """Node of f_K (with ``only`` = T: of its T term alone); None when it is
        identically zero."""
        if any(self.sec.mono[j][0] < -1 for j in self.S):
            return self._unit_general(K, only)
        g = self.g
        sec = self.sec
        S = self.S
        total = g.c(0.0)
        for T in _subsets(S):
            if only is not None and tuple(sorted(T)) != tuple(sorted(only)):
                continue
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


    # -- poles of higher order: Taylor subtraction of order p_j in t_j --------------------
    #
    # For t^{-1-p+b eps} G the subtraction at t = 0 keeps the Taylor polynomial of G of
    # degree p:  int_0^1 t^{-1-p+b eps} G = int_0^1 t^{-1-p+b eps} (G - sum_{k<=p} t^k G_k)
    # + sum_{k<=p} G_k / (k - p + b eps),  G_k the k-th Taylor coefficient at t = 0.  Over
    # several singular variables the pole terms T (with their coefficient orders k_T) and
    # the remainders of the others multiply out; the Taylor coefficients of G_N are taken
    # from truncated multivariate power series of the polynomials (products, the series
    # inverse and the series logarithm).  p = 0 everywhere is the corner form above.

    def _poly_series(self, i, spec):
        """Series of P_i in the variables of ``spec`` with order >= 1 (truncated at those
        orders), the variables of order 0 set to 0: {multi-index: node}."""
        V = [j for j in sorted(spec) if spec[j] >= 1]
        zero = {j for j in spec if spec[j] == 0}
        p = self.sec.polys[i][0]
        groups = {}
        for m, c in p.items():
            if any(m[j - 1] for j in zero):
                continue
            idx = tuple(m[j - 1] for j in V)
            if any(e > spec[j] for e, j in zip(idx, V)):
                continue
            rest = tuple(0 if (q + 1) in V else e for q, e in enumerate(m))
            groups.setdefault(idx, []).append((rest, c))
        out = {}
        for idx, terms in sorted(groups.items()):
            acc = self.g.c(0.0)
            for rest, c in sorted(terms):
                acc = self.g.fma(self.monomial(rest), self.g.c(float(c)), acc)
            out[idx] = acc
        return V, out

    @staticmethod
    def _indices(V, spec):
        return sorted(itertools.product(*[range(spec[j] + 1) for j in V]), key=lambda m: (sum(m), m))

    def _smul(self, A, B, V, spec):
        g = self.g
        out = {}
        for m in self._indices(V, spec):
            acc = g.c(0.0)
            for l, a in A.items():
                r = tuple(x - y for x, y in zip(m, l))
                if min(r, default=0) < 0 or r not in B:
                    continue
                acc = g.fma(a, B[r], acc)
            if g.const_value(acc) != 0.0:
                out[m] = acc
        return out

    def _sinv(self, A, V, spec):
        g = self.g
        z = tuple(0 for _ in V)
        b0 = g.inv(A[z])
        out = {z: b0}
        for m in self._indices(V, spec):
            if m == z:
                continue
            acc = g.c(0.0)
            for l, a in A.items():
                if l == z:
                    continue
                r = tuple(x - y for x, y in zip(m, l))
                if min(r, default=0) < 0 or r not in out:
                    continue
                acc = g.fma(a, out[r], acc)
            if g.const_value(acc) != 0.0:
                out[m] = g.neg(g.mul(acc, b0))
        return out

    def _spow(self, A, a, V, spec):
        z = tuple(0 for _ in V)
        if a < 0:
            A, a = self._sinv(A, V, spec), -a
        out = {z: self.g.c(1.0)}
        for _ in range(int(a)):
            out = self._smul(out, A, V, spec)
        return out

    def _slog(self, A, V, spec):
        g = self.g
        z = tuple(0 for _ in V)
        inv0 = g.inv(A[z])
        u = {m: g.mul(a, inv0) for m, a in A.items() if m != z}
        out = {z: g.log(A[z])}
        power = dict(u)
        for n in range(1, sum(spec[j] for j in V) + 1):
            for m, v in power.items():
                out[m] = g.fma(v, g.c((-1.0) ** (n + 1) / n), out.get(m, g.c(0.0)))
            power = self._smul(power, u, V, spec)
        return out

    def G_coeff(self, N, spec):
        """The Taylor coefficient of G_N of order spec[j] in each variable j of ``spec``
        (order 0: G_N at t_j = 0)."""
        key = ("GC", N, tuple(sorted(spec.items())))
        if key in self._corner:
            return self._corner[key]
        if all(k == 0 for k in spec.values()):
            out = self.G_at(N, tuple(sorted(spec)))
            self._corner[key] = out
            return out
        g = self.g
        V = [j for j in sorted(spec) if spec[j] >= 1]
        z = tuple(0 for _ in V)
        G = {z: g.c(1.0)}
        L = {}
        for i, (p, (a0, a1)) in enumerate(self.sec.polys):
            _, Pi = self._poly_series(i, spec)
            if a0:
                G = self._smul(G, self._spow(Pi, a0, V, spec), V, spec)
            if a1:
                Li = self._slog(Pi, V, spec)
                for m, v in Li.items():
                    L[m] = g.fma(v, g.c(float(a1)), L.get(m, g.c(0.0)))
        for i, power in self.sec.log_factor:
            _, Pi = self._poly_series(i, spec)
            G = self._smul(G, self._spow(self._slog(Pi, V, spec), power, V, spec), V, spec)
        for n in range(1, N + 1):
            G = {m: g.mul(v, g.c(1.0 / n)) for m, v in self._smul(G, L, V, spec).items()}
        out = G.get(tuple(spec[j] for j in V), g.c(0.0))
        self._corner[key] = out
        return out

    def _unit_general(self, K, only):
        g = self.g
        sec = self.sec
        S = self.S
        p = {j: -1 - sec.mono[j][0] for j in S}
        nmax = K + len(S)

        def smul(a, b):
            out = {}
            for i, x in a.items():
                for j, y in b.items():
                    if i + j <= nmax:
                        out[i + j] = g.fma(x, y, out.get(i + j, g.c(0.0)))
            return out

        total = g.c(0.0)
        for T in _subsets(S):
            if only is not None and tuple(sorted(T)) != tuple(sorted(only)):
                continue
            rest = [j for j in S if j not in T]
            for ks in itertools.product(*[range(p[j] + 1) for j in T]):
                coef = {0: g.c(1.0)}
                for j, k in zip(T, ks):
                    b = sec.mono[j][1]
                    if k == p[j]:
                        s = {-1: g.c(1.0 / (math.factorial(k) * b))}
                    else:
                        q = k - p[j]
                        s = {m: g.c((1.0 / (math.factorial(k) * q)) * (-b / q) ** m) for m in range(0, nmax + 2)}
                    coef = smul(coef, s)
                for j in sec.variables:
                    b = sec.mono[j][1]
                    if j in T or not b:
                        continue
                    lt = g.mul(self.logt(j), g.c(float(b)))
                    s, pw = {0: g.c(1.0)}, g.c(1.0)
                    for m in range(1, nmax + 2):
                        pw = g.mul(pw, g.mul(lt, g.c(1.0 / m)))
                        s[m] = pw
                    coef = smul(coef, s)
                term = g.c(0.0)
                for m, cm in sorted(coef.items()):
                    n = K - m
                    if not 0 <= n <= nmax or g.const_value(cm) == 0.0:
                        continue
                    # remainders of the rest: sum over Z subset rest and orders k_Z of
                    # (-1)^|Z| prod_{j in Z} t_j^k_j  x  the Taylor coefficient
                    op = g.c(0.0)
                    for Z in _subsets(rest):
                        for kz in itertools.product(*[range(p[j] + 1) for j in Z]):
                            spec = {j: k for j, k in zip(T, ks)}
                            spec.update({j: k for j, k in zip(Z, kz)})
                            c = self.G_coeff(n, spec)
                            if g.const_value(c) == 0.0:
                                continue
                            fac = g.c((-1.0) ** len(Z))
                            for j, k in zip(Z, kz):
                                if k:
                                    fac = g.mul(fac, self.tpow(j, k))
                            op = g.fma(fac, c, op)
                    term = g.fma(cm, op, term)
                if g.const_value(term) == 0.0:
                    continue
                for j, k in zip(T, ks):                   # d^k/dt^k at 0 = k! x coefficient
                    if k:
                        term = g.mul(term, g.c(float(math.factorial(k))))
                for j in rest:
                    term = g.mul(term, g.powi(self.t(j), sec.mono[j][0]))
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


def term_subsets(sec):
    """The subsets T of the singular variables: the separately integrable terms of a
    sector (the paper's SeparateTerms option, Sec. 4.4)."""
    return list(_subsets(singular(sec)))


def term_variables(sec, T):
    """The variables a T term depends on (it is constant along T); at least one."""
    return tuple(j for j in sec.variables if j not in T) or (sec.variables[0],)


def term_graph(sec, orders, T):
    """(Graph, result nodes) of the T term of every order in ``orders`` of one sector,
    over the variables ``term_variables(sec, T)``; zero orders give constant 0."""
    g = Graph()
    ev = _SectorEval(g, sec, term_variables(sec, T))
    outs = []
    for K in orders:
        node = ev.unit(K, only=T) if K >= -len(ev.S) else None
        outs.append(g.c(0.0) if node is None else node)
    return g, outs


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


def mixed_graph(secs, orders):
    """(Graph, result nodes) summing the integrands of several sectors of the same
    dimension over the common unit cube, every order in ``orders`` (the paper's
    MixSectors option, Sec. 4.4: fewer, longer integrands; the integral of the sum is
    the sum of the sector integrals).  Sector j's variables are the coordinates
    x_0..x_{d-1} in its own order; an order below a sector's lowest contributes 0."""
    dims = {len(s.variables) for s in secs}
    if len(dims) != 1:
        raise ValueError("mixed sectors must have one dimension")
    g = Graph()
    evs = [_SectorEval(g, s) for s in secs]
    outs = []
    for K in orders:
        nodes = [ev.unit(K) for ev in evs if K >= -len(ev.S)]
        nodes = [n for n in nodes if n is not None]
        acc = g.c(0.0) if not nodes else nodes[0]
        for n in nodes[1:]:
            acc = g.add(acc, n)
        outs.append(acc)
    return g, outs


# ---------------------------------------------------------------------------
# Physical kinematics: contour deformation
# ---------------------------------------------------------------------------

from .ir import cconst, cadd, csub, cmul, cscale, cinv, cpowi, clog  # noqa: E402
from .poly import pderiv  # noqa: E402


class _ComplexSectorEval:
    """The sector integrand on a deformed contour.

    With F the sector's last polynomial (the second Symanzik polynomial after the
    monomial factor is pulled out), the variables move to
    z_j = t_j - i lam t_j (1 - t_j) dF/dt_j.  The deformation vanishes on the faces
    t_j = 0, 1, so the integral over the cube is unchanged, and Im F(z) <= 0 for small
    lam realises the F - i0 prescription of the propagators.  Writing
    z_j = t_j w_j, the integrand prod z_j^{c_j + b_j eps} G(z) det(dz/dt) is
    prod t_j^{c_j + b_j eps} times G~ = prod w_j^{c_j + b_j eps} G(z) det(dz/dt),
    and G~ takes the place of G in the subtraction and expansion of ``_SectorEval``.
    All quantities are (re, im) pairs of real graph nodes.
    """

    def __init__(self, g, sec, lam):
        self.g = g
        self.sec = sec
        self.lam = float(lam)
        self.pos = {j: i for i, j in enumerate(sec.variables)}
        self.S = singular(sec)
        F = sec.polys[-1][0]
        self.D1 = {j: pderiv(F, j - 1) for j in sec.variables}
        self.D2 = {(j, k): pderiv(self.D1[j], k - 1) for j in sec.variables for k in sec.variables}
        self._c = {}

    def t(self, j):
        return self.g.x(self.pos[j])

    def _tpow(self, j, e):
        key = ("tp", j, e)
        if key not in self._c:
            g = self.g
            if e == 1:
                self._c[key] = self.t(j)
            elif e % 2 == 0:
                h = self._tpow(j, e // 2)
                self._c[key] = g.mul(h, h)
            else:
                self._c[key] = g.mul(self._tpow(j, e - 1), self.t(j))
        return self._c[key]

    def rpoly(self, p, W):
        """Real polynomial p at t with t_W = 0."""
        g = self.g
        acc = g.c(0.0)
        for m, c in sorted(p.items()):
            if any(m[j - 1] for j in W):
                continue
            mono = g.c(1.0)
            for q, e in enumerate(m):
                if e:
                    mono = g.mul(mono, self._tpow(q + 1, e))
            acc = g.fma(mono, g.c(float(c)), acc)
        return acc

    def w(self, j, W):
        key = ("w", j, W)
        if key not in self._c:
            g = self.g
            one_minus_t = g.c(1.0) if j in W else g.sub(g.c(1.0), self.t(j))
            im = g.mul(g.mul(one_minus_t, self.rpoly(self.D1[j], W)), g.c(-self.lam))
            self._c[key] = (g.c(1.0), im)
        return self._c[key]

    def zpow(self, j, e, W):
        """z_j^e at the corner W (z_j = 0 for j in W)."""
        key = ("zp", j, e, W)
        if key not in self._c:
            g = self.g
            if j in W:
                self._c[key] = cconst(g, 0.0)
            elif e == 1:
                wj = self.w(j, W)
                self._c[key] = (self.t(j), g.mul(self.t(j), wj[1]))
            elif e % 2 == 0:
                h = self.zpow(j, e // 2, W)
                self._c[key] = cmul(g, h, h)
            else:
                self._c[key] = cmul(g, self.zpow(j, e - 1, W), self.zpow(j, 1, W))
        return self._c[key]

    def cpoly(self, i, W):
        key = ("P", i, W)
        if key not in self._c:
            g = self.g
            acc = cconst(g, 0.0)
            for m, c in sorted(self.sec.polys[i][0].items()):
                if any(m[j - 1] for j in W):
                    continue
                mono = cconst(g, 1.0)
                for q, e in enumerate(m):
                    if e:
                        mono = cmul(g, mono, self.zpow(q + 1, e, W))
                acc = cadd(g, acc, cscale(g, mono, g.c(float(c))))
            self._c[key] = acc
        return self._c[key]

    def detJ(self, W):
        """det(dz/dt) = det(I - i lam M), M_jk = delta_jk (1 - 2 t_j) D_j + t_j (1 - t_j) D_jk,
        by Gaussian elimination without pivoting (the matrix is close to the identity)."""
        key = ("J", W)
        if key in self._c:
            return self._c[key]
        g = self.g
        V = list(self.sec.variables)
        d = len(V)
        A = [[None] * d for _ in range(d)]
        for a, j in enumerate(V):
            tj = g.c(0.0) if j in W else self.t(j)
            tt = g.mul(tj, g.sub(g.c(1.0), tj))
            for b, k in enumerate(V):
                m = g.mul(tt, self.rpoly(self.D2[(j, k)], W))
                if a == b:
                    m = g.fma(g.sub(g.c(1.0), g.mul(tj, g.c(2.0))), self.rpoly(self.D1[j], W), m)
                A[a][b] = (g.c(1.0 if a == b else 0.0), g.mul(m, g.c(-self.lam)))
        det = cconst(g, 1.0)
        for k in range(d):
            piv = A[k][k]
            det = cmul(g, det, piv)
            if k + 1 == d:
                break
            ip = cinv(g, piv)
            for i in range(k + 1, d):
                f = cmul(g, A[i][k], ip)
                for jj in range(k + 1, d):
                    A[i][jj] = csub(g, A[i][jj], cmul(g, f, A[k][jj]))
        self._c[key] = det
        return det

    def G_at(self, N, W):
        key = ("G", N, W)
        if key in self._c:
            return self._c[key]
        g = self.g
        sec = self.sec
        if N == 0:
            out = self.detJ(W)
            for j in sec.variables:
                c = sec.mono[j][0]
                if c:
                    out = cmul(g, out, cpowi(g, self.w(j, W), c))
            for i, (p, (a0, a1)) in enumerate(sec.polys):
                if a0:
                    out = cmul(g, out, cpowi(g, self.cpoly(i, W), a0))
            for i, power in sec.log_factor:
                out = cmul(g, out, cpowi(g, clog(g, self.cpoly(i, W)), power))
        else:
            L = cconst(g, 0.0)
            for i, (p, (a0, a1)) in enumerate(sec.polys):
                if a1:
                    L = cadd(g, L, cscale(g, clog(g, self.cpoly(i, W)), g.c(float(a1))))
            for j in sec.variables:
                b = sec.mono[j][1]
                if b:
                    L = cadd(g, L, cscale(g, clog(g, self.w(j, W)), g.c(float(b))))
            out = cscale(g, cmul(g, self.G_at(N - 1, W), L), g.c(1.0 / N))
        self._c[key] = out
        return out

    def D(self, T, N):
        key = ("D", T, N)
        if key in self._c:
            return self._c[key]
        rest = [j for j in self.S if j not in T]

        def diff(k, W):
            if k == len(rest):
                return self.G_at(N, tuple(sorted(W)))
            j = rest[k]
            return csub(self.g, diff(k + 1, W), diff(k + 1, W + (j,)))
        out = diff(0, tuple(T))
        self._c[key] = out
        return out

    def logt(self, j):
        key = ("lt", j)
        if key not in self._c:
            self._c[key] = self.g.log(self.t(j))
        return self._c[key]

    def unit(self, K):
        g = self.g
        sec = self.sec
        S = self.S
        total = cconst(g, 0.0)
        for T in _subsets(S):
            top = K + len(T)
            if top < 0:
                continue
            lam = g.c(0.0)
            for j in sec.variables:
                b = sec.mono[j][1]
                if j not in T and b:
                    lam = g.fma(self.logt(j), g.c(float(b)), lam)
            inner = cconst(g, 0.0)
            lam_pow = g.c(1.0)
            for m in range(0, top + 1):
                if m:
                    if g.const_value(lam) == 0.0:
                        break
                    lam_pow = g.mul(g.mul(lam_pow, lam), g.c(1.0 / m))
                Dn = self.D(T, top - m)
                inner = cadd(g, inner, cscale(g, Dn, lam_pow))
            fac = 1.0
            for j in T:
                fac /= sec.mono[j][1]
            term = cscale(g, inner, g.c(fac))
            for j in S:
                if j not in T:
                    term = cscale(g, term, g.inv(self.t(j)))
            total = cadd(g, total, term)
        mono = g.c(float(sec.coef))
        for j in sec.variables:
            if j in S:
                continue
            c = sec.mono[j][0]
            if c:
                mono = g.mul(mono, g.powi(self.t(j), c))
        return cscale(g, total, mono)


def sector_graph_complex(sec, orders, lam):
    """(Graph, [re_K0, im_K0, re_K1, im_K1, ...]) of a sector on the deformed contour."""
    g = Graph()
    ev = _ComplexSectorEval(g, sec, lam)
    outs = []
    for K in orders:
        if K < -len(ev.S):
            outs += [g.c(0.0), g.c(0.0)]
        else:
            re, im = ev.unit(K)
            outs += [re, im]
    return g, outs


def choose_lambda(sec, lam_max=1.0, n_points=2000, seed=0):
    """Largest lam in lam_max * 2^-k (k = 0..12) with Im F(z) <= 0 and Re w_j > 0 at
    random points of the cube, or None when F has only positive coefficients (no
    deformation needed)."""
    import numpy as np
    F = sec.polys[-1][0]
    if all(c > 0 for c in F.values()):
        return None
    rng = np.random.default_rng(seed)
    var = sec.variables
    X = rng.uniform(1e-6, 1 - 1e-6, size=(n_points, len(var)))

    def ev_poly(p, Z):
        out = np.zeros(Z.shape[0], dtype=Z.dtype)
        for m, c in p.items():
            term = np.full(Z.shape[0], float(c), dtype=Z.dtype)
            for q, e in enumerate(m):
                if e:
                    term = term * Z[:, var.index(q + 1)] ** e
            out = out + term
        return out
    D = np.stack([ev_poly(pderiv(F, j - 1), X) for j in var], axis=1)
    for k in range(13):
        lam = lam_max * 2.0 ** -k
        Z = X - 1j * lam * X * (1 - X) * D
        if np.all(np.imag(ev_poly(F, Z)) <= 0.0):
            return lam
    raise ValueError("no contour deformation parameter keeps Im F <= 0")
