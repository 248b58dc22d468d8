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
    cplx: bool = False        # deformed contour: results are (re, im) pairs, orders order .. order + n_out/2 - 1
    lam: float = None         # the deformation parameter of a complex unit
    sectors: tuple = None     # mixed units: the sectors whose integrands the program sums
    term: tuple = None        # separate-term units: the variables whose pole term it is


@dataclasses.dataclass
class Prepared:
    name: str
    units: list
    prefactor: tuple          # (q, coeffs): c(eps) = sum coeffs[i] eps^(i-q)
    int_orders: tuple         # eps orders of the parametric integral
    out_orders: tuple         # eps orders of the assembled result
    sectors: list
    lams: list = None         # per sector: contour-deformation parameter, None when F > 0

    @property
    def complex(self):
        return any(u.cplx for u in self.units)

    def flops_per_point(self):
        """Mean arithmetic operations per point over the units (see Program.flops)."""
        return sum(u.program.flops() for u in self.units) / max(len(self.units), 1)


def _real_units(si, sec, Ks, fuse):
    """Units of a sector with F > 0: one per order, or one fused unit for all orders."""
    if fuse:
        if len(Ks) > MAX_OUT:
            raise ValueError(f"a fused unit holds at most {MAX_OUT} orders")
        g, outs = I.sector_graph(sec, Ks)
        return [Unit(si, Ks[0], len(sec.variables), B.emit(g, outs, len(sec.variables)), 0,
                     n_out=len(Ks))]
    units = []
    for K in Ks:
        r = I.unit_graph(sec, K)
        if r is None:
            continue
        g, out = r
        units.append(Unit(si, K, len(sec.variables), B.emit(g, out, len(sec.variables)), 0))
    return units


def _term_units(si, sec, Ks, fuse):
    """Units of a sector with F > 0, one per separately integrable term (the paper's
    SeparateTerms, Sec. 4.4): the term of a subset T of the singular variables is
    constant along T, so it is integrated over the remaining variables only.  Fused:
    one unit per term carrying the orders where it is non-zero; else one per (term,
    order)."""
    units = []
    for T in I.term_subsets(sec):
        var = I.term_variables(sec, T)
        d = len(var)
        if fuse:
            g, outs = I.term_graph(sec, Ks, T)
            nz = [k for k, o in enumerate(outs) if g.const_value(o) != 0.0]
            if not nz:
                continue
            lo, hi = nz[0], nz[-1]
            if hi - lo + 1 > MAX_OUT:
                raise ValueError(f"a fused unit holds at most {MAX_OUT} orders")
            units.append(Unit(si, Ks[lo], d, B.emit(g, outs[lo:hi + 1], d), 0, n_out=hi - lo + 1, term=tuple(T)))
        else:
            for K in Ks:
                g, outs = I.term_graph(sec, [K], T)
                if g.const_value(outs[0]) == 0.0:
                    continue
                units.append(Unit(si, K, d, B.emit(g, outs[0], d), 0, term=tuple(T)))
    return units


def _complex_units(si, sec, Ks, fuse, lam):
    """Units of a sector on the deformed contour: each order gives a (re, im) pair of
    results; fused while the pairs fit MAX_OUT results, else one unit per order."""
    groups = [Ks] if fuse and 2 * len(Ks) <= MAX_OUT else [[K] for K in Ks]
    units = []
    for grp in groups:
        g, outs = I.sector_graph_complex(sec, grp, lam)
        units.append(Unit(si, grp[0], len(sec.variables), B.emit(g, outs, len(sec.variables)), 0,
                          n_out=2 * len(grp), cplx=True, lam=lam))
    return units


MAX_OUT = 6


def _sector_lambda(sec, lam, lam_max):
    """None when every coefficient of F is positive (no deformation needed)."""
    if all(c > 0 for c in sec.polys[-1][0].values()):
        return None
    if callable(lam):
        return lam(sec)
    if lam is not None:
        return float(lam)
    return I.choose_lambda(sec, lam_max)


def _mix_units(secs, real, Ks_of, group, max_slots=72):
    """Mixed units (the paper's MixSectors): consecutive real sectors of equal
    dimension, up to ``group`` at a time, as one program summing their fused
    integrands.  A group also closes when its program would need more than
    ``max_slots`` slots (the slot file lives in shared memory, per thread)."""

    def build(run):
        lo = min(Ks_of(secs[i])[0] for i in run)
        hi = max(Ks_of(secs[i])[-1] for i in run)
        Ks = list(range(lo, hi + 1))
        if len(Ks) > MAX_OUT:
            return None
        g, outs = I.mixed_graph([secs[i] for i in run], Ks)
        d = len(secs[run[0]].variables)
        prog = B.emit(g, outs, d)
        if len(run) > 1 and prog.n_slots > max_slots:
            return None
        return Unit(run[0], Ks[0], d, prog, 0, n_out=len(Ks), sectors=tuple(run))

    def build_one(i):
        u = build([i])
        if u is None:
            raise ValueError(f"a fused unit holds at most {MAX_OUT} orders")
        return u

    units, run, best = [], [], None
    for i in real:
        if not Ks_of(secs[i]):
            continue
        if run and (len(run) == group or len(secs[i].variables) != len(secs[run[0]].variables)):
            units.append(best)
            run, best = [], None
        trial = build(run + [i]) if run else build_one(i)
        if trial is None:                  # the group is full: start a new one with i
            units.append(best)
            run, best = [i], build_one(i)
        else:
            run, best = run + [i], trial
    if best is not None:
        units.append(best)
    return units


def prepare_feynman(problem, strategy="M", fuse_orders=False, lam=None, lam_max=1.0, mix_sectors=1,
                    separate_terms=False):
    """Units of a Feynman integral; with ``fuse_orders`` one unit per sector carries all
    its eps orders (a vector-valued integrand with one Vegas grid).

    Sectors whose F has a coefficient that is not positive (physical kinematics) are
    integrated on a deformed contour (``integrand.sector_graph_complex``) with complex
    results; ``lam`` fixes the deformation parameter (a number, or a callable of the
    sector), else it is chosen per sector by ``integrand.choose_lambda`` up to lam_max.
    A sector where no parameter keeps Im F <= 0 raises ValueError.
    ``mix_sectors`` > 1 sums that many consecutive real sectors of equal dimension into
    one program with all their orders (the paper's MixSectors; implies fused orders).
    ``separate_terms`` gives every real sector one unit per separately integrable term
    (the paper's SeparateTerms, ``_term_units``); it excludes ``mix_sectors``.
    """
    if separate_terms and mix_sectors > 1:
        raise ValueError("separate_terms and mix_sectors exclude each other")
    U, F = symanzik(problem)
    n = len(problem.propagators)
    L = len(problem.loop_momenta)
    secs = D.decompose_feynman(U, F, n, problem.indices, L, strategy)
    kmin = min(I.min_order(s) for s in secs)
    q0, _ = PF.series(problem.indices, L, 0)
    khi = problem.order + q0
    units, lams = [], []
    Ks_of = lambda s: list(range(max(kmin, I.min_order(s)), khi + 1))
    for si, sec in enumerate(secs):
        Ks = Ks_of(sec)
        lm = _sector_lambda(sec, lam, lam_max)
        lams.append(lm)
        if not Ks:
            continue
        if lm is None:
            if separate_terms:
                units += _term_units(si, sec, Ks, fuse_orders)
            elif mix_sectors <= 1:
                units += _real_units(si, sec, Ks, fuse_orders)
        else:
            units += _complex_units(si, sec, Ks, fuse_orders, lm)
    if mix_sectors > 1:
        units = _mix_units(secs, [i for i, l in enumerate(lams) if l is None], Ks_of, mix_sectors) + units
    for k, u in enumerate(units):
        u.rng_key = k
    pre = PF.series(problem.indices, L, problem.order - kmin)
    return Prepared(problem.name, units, pre, tuple(range(kmin, khi + 1)),
                    tuple(range(kmin - pre[0], problem.order + 1)), secs, lams)


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
    sectors (errors combined in the mean-square norm, Sec. 4.3).  Complex values
    (deformed contour) come with errors complex(sigma_re, sigma_im); the prefactor
    series is real, so the real and imaginary parts are assembled separately.
    """
    if any(isinstance(v, complex) for v in values.values()):
        part = lambda d, f: {K: f(x) for K, x in d.items()}
        Rr, Er = assemble(prep, part(values, lambda z: complex(z).real), part(errors, lambda z: complex(z).real),
                          correlated)
        Ri, Ei = assemble(prep, part(values, lambda z: complex(z).imag), part(errors, lambda z: complex(z).imag),
                          correlated)
        return ({n: complex(Rr[n], Ri[n]) for n in Rr}, {n: complex(Er[n], Ei[n]) for n in Er})
    if correlated is None:
        correlated = any((u.n_out // 2 if u.cplx else u.n_out) > 1 for u in prep.units)
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
