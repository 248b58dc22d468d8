"""Host preprocessor: problem -> units (sector, eps order) -> register programs.

Step a0 of the hot path; not timed.  For a Feynman integral it builds U and F
(Eq. 2, the ``UF`` constructor of Sec. 4.3), decomposes into sectors, subtracts
the poles and expands in eps, and lowers every unit to bytecode.  A unit is the
integrand of one sector at one power of eps, the unit of work of the paper's
integrand database (Sec. 4.7: keys carry the eps order and the sector number).
"""
from __future__ import annotations

import dataclasses
import math

from . import decompose as D
from . import integrand as I
from . import bytecode as B
from . import prefactor as PF
from .symanzik import symanzik


@dataclasses.dataclass
class Unit:
    sector: int
    order: int                # eps order of the (first) result
    dim: int
    program: B.Program
    rng_key: int
    n_out: int = 1            # results: orders order .. order + n_out - 1 (fused multi-order unit)


@dataclasses.dataclass
class Prepared:
    name: str
    units: list
    prefactor: tuple          # (q, coeffs): c(eps) = sum coeffs[i] eps^(i-q)
    int_orders: tuple         # eps orders of the parametric integral
    out_orders: tuple         # eps orders of the assembled result
    sectors: list

    def flops_per_point(self):
        """Mean arithmetic operations per point over the units (see Program.flops)."""
        return sum(u.program.flops() for u in self.units) / max(len(self.units), 1)


def _units_for(sectors, orders_of):
    units = []
    for si, sec in enumerate(sectors):
        for K in orders_of(sec):
            r = I.unit_graph(sec, K)
            if r is None:
                continue
            g, out = r
            prog = B.emit(g, out, len(sec.variables))
            units.append(Unit(si, K, len(sec.variables), prog, len(units)))
    return units


MAX_OUT = 6


def _fused_units(sectors, orders_of):
    """One unit per sector whose program returns every eps order of the sector: the
    orders share the polynomial values, logarithms and corner terms (one evaluation
    of U, F and the subtraction corners per point instead of one per order)."""
    units = []
    for si, sec in enumerate(sectors):
        Ks = list(orders_of(sec))
        if not Ks:
            continue
        if len(Ks) > MAX_OUT:
            raise ValueError(f"a fused unit holds at most {MAX_OUT} orders")
        g, outs = I.sector_graph(sec, Ks)
        prog = B.emit(g, outs, len(sec.variables))
        units.append(Unit(si, Ks[0], len(sec.variables), prog, len(units), n_out=len(Ks)))
    return units


def prepare_feynman(problem, strategy="M", fuse_orders=False):
    """Units of a Feynman integral; with ``fuse_orders`` one unit per sector carries all
    its eps orders (a vector-valued integrand with one Vegas grid)."""
    U, F = symanzik(problem)
    n = len(problem.propagators)
    L = len(problem.loop_momenta)
    secs = D.decompose_feynman(U, F, n, problem.indices, L, strategy)
    kmin = min(I.min_order(s) for s in secs)
    q0, _ = PF.series(problem.indices, L, 0)
    khi = problem.order + q0
    orders_of = lambda s: range(max(kmin, I.min_order(s)), khi + 1)
    units = (_fused_units if fuse_orders else _units_for)(secs, orders_of)
    pre = PF.series(problem.indices, L, problem.order - kmin)
    return Prepared(problem.name, units, pre, tuple(range(kmin, khi + 1)),
                    tuple(range(kmin - pre[0], problem.order + 1)), secs)


def prepare_direct(problems, name="direct"):
    """One Prepared holding every unit of a list of DirectProblem (no prefactor)."""
    units = []
    secs = []
    orders = set()
    for prob in problems:
        for sec in D.iterate(D.direct_sector(prob), "M"):
            si = len(secs)
            secs.append(sec)
            for K in prob.orders:
                if K < I.min_order(sec):
                    continue
                r = I.unit_graph(sec, K)
                if r is None:
                    continue
                g, out = r
                prog = B.emit(g, out, len(sec.variables))
                units.append(Unit(si, K, len(sec.variables), prog, len(units)))
                orders.add(K)
    orders = tuple(sorted(orders))
    return Prepared(name, units, (0, [1.0]), orders, orders, secs)


def assemble(prep, values, errors, correlated=None):
    """Step a6: R_n = sum_m c_m I_{n-m}.

    With one unit per (sector, order) the I_K are independent and
    sigma_n^2 = sum_m c_m^2 sigma_{n-m}^2.  Fused units evaluate all orders of a
    sector at the same points, so I_K of different K are correlated; then the
    bound sigma_n <= sum_m |c_m| sigma_{n-m}, valid for any correlation, is used.
    ``values``/``errors`` map eps orders of the parametric integral to sums over
    sectors (errors combined in the mean-square norm, Sec. 4.3).
    """
    if correlated is None:
        correlated = any(getattr(u, "n_out", 1) > 1 for u in prep.units)
    q, c = prep.prefactor
    R, E = {}, {}
    for n in prep.out_orders:
        v, e2, e1 = 0.0, 0.0, 0.0
        for i, ci in enumerate(c):
            K = n - (i - q)
            if K in values:
                v += ci * values[K]
                e2 += (ci * errors[K]) ** 2
                e1 += abs(ci) * errors[K]
        R[n] = v
        E[n] = e1 if correlated else math.sqrt(e2)
    return R, E
