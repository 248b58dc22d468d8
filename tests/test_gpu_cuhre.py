"""GPU parity of the adaptive cubature: per region against the oracle's rule, whole
runs against the oracle's passes, and integrals against closed forms."""
import functools
import math

import numpy as np
import pytest

import workloads as W
from oracle import cuhre as OC, pipeline as P

from gpu_common import need_gpu, feynman, integrator, stress

pytestmark = pytest.mark.gpu


def _oracle_vector_f(prep_unit, orc_units):
    """The oracle's integrand of a (possibly fused or complex) unit as an (m, n_out) function."""
    by = {(u.sector, u.order): u for u in orc_units}
    u = prep_unit
    if u.cplx:
        parts = [by.get((u.sector, u.order + k)) for k in range(u.n_out // 2)]

        def f(X):
            cols = []
            for o in parts:
                v = o.f_numpy(X) if o is not None else np.zeros(X.shape[0], complex)
                cols += [np.real(v), np.imag(v)]
            return np.stack(cols, axis=1)
        return f
    parts = [by.get((u.sector, u.order + k)) for k in range(u.n_out)]

    def f(X):
        return np.stack([o.f_numpy(X) if o is not None else np.zeros(X.shape[0]) for o in parts], axis=1)
    return f


def _check_regions(integ, prep, orc_units, idx):
    checked = 0
    for i in idx:
        u = prep.units[i]
        cen, half, val, err, ax = integ.cuhre_regions(i)
        f = _oracle_vector_f(u, orc_units)
        g = f if u.dim >= 2 else (lambda X, f=f: f(X[:, :1]))
        for k in range(len(cen)):
            I7, I5, e, dif = OC.apply_rule(g, cen[k], half[k])
            n = cen.shape[1]
            pts = np.concatenate([np.stack(gr) for gr in OC.rule_points(n)]) * half[k] + cen[k]
            V = float(np.prod(2 * half[k]))
            scale = 4 * V * np.max(np.abs(g(pts)), axis=0) + 1e-300
            assert np.all(np.abs(val[k] - I7) <= 1e-12 * scale), (i, k, val[k], I7)
            assert np.all(np.abs(err[k] - e) <= 1e-12 * scale), (i, k, err[k], e)
            s = np.sort(dif.sum(axis=1))
            if len(s) < 2 or s[-1] - s[-2] > 1e-9 * s[-1]:
                assert ax[k] == OC.split_axis(dif, half[k]), (i, k)
            checked += 1
    return checked


@pytest.mark.parametrize("name,passes", [("box", 3), ("bubble", 6)])
def test_cuhre_regions_match_oracle_rule(name, passes):
    """After a few passes, every live region's I7, |I7 - I5| and split axis equal the
    oracle's rule applied to the same region (fused units, all results)."""
    need_gpu()
    from paper_1511_03614_gb300 import prepare_feynman, Integrator
    prep = prepare_feynman(getattr(W, name)(), fuse_orders=True)
    integ = Integrator(prep)
    integ.cuhre(rel_tol=1e-12, max_passes=passes)
    orc = P.feynman_problem(getattr(W, name)())
    assert _check_regions(integ, prep, orc.units, range(len(prep.units))) > 20


def test_cuhre_complex_regions_match_oracle_rule():
    need_gpu()
    from paper_1511_03614_gb300 import prepare_feynman, Integrator
    prep = prepare_feynman(W.box_physical(), fuse_orders=True)
    integ = Integrator(prep)
    integ.cuhre(rel_tol=1e-12, max_passes=3)
    orc = P.feynman_problem(W.box_physical(), lam=prep.lams[0])
    assert _check_regions(integ, prep, orc.units, range(len(prep.units))) > 20


def test_cuhre_runs_match_oracle_passes():
    """Whole runs on random polynomial-log integrands (dims 3..8): the oracle's passes
    give the same value (to 1e-11 relative) and, where no split decision is a
    near tie, the same region count and pass count."""
    need_gpu()
    probs, prep, integ = stress(24)
    res = integ.cuhre(rel_tol=1e-5, abs_tol=1e-14, max_passes=12, max_regions=1 << 20)
    same_tree = 0
    for k, prob in enumerate(probs):
        o = P.direct_problem(prob).units[0]
        r = OC.cuhre(o.f_numpy, prob.dim, rel_tol=1e-5, abs_tol=1e-14, max_passes=12)
        g = res.per_unit[k]
        if g["n_regions"] == r.n_regions and g["passes"] == r.passes:
            same_tree += 1
            assert g["converged"] == r.converged
            assert g["n_points"] == r.n_evals
            assert abs(g["value"] - r.value[0]) <= max(1e-11 * abs(r.value[0]), 1e-14), (k, g, r.value)
        else:
            assert abs(g["value"] - r.value[0]) <= g["error"] + r.error[0], (k, g, r.value, r.error)
    assert same_tree >= 0.9 * len(probs)


def test_cuhre_box_closed_form():
    """All box units to 1e-8 relative: the assembled series within its error bound of
    2/eps^2 - ln2/eps - 2 pi^2/3; deterministic (two calls agree bit for bit)."""
    need_gpu()
    from paper_1511_03614_gb300 import prepare_feynman, Integrator
    integ = Integrator(prepare_feynman(W.box(), fuse_orders=True))
    r1 = integ.cuhre(rel_tol=1e-8)
    r2 = integ.cuhre(rel_tol=1e-8)
    exact = {-2: 2.0, -1: -math.log(2.0), 0: -2 * math.pi ** 2 / 3}
    for n, v in exact.items():
        assert abs(r1.assembled[n] - v) <= r1.assembled_errors[n] + 1e-12, (n, r1.assembled[n], v)
        assert r1.assembled_errors[n] < 1e-6
        assert r1.assembled[n] == r2.assembled[n]
    assert all(d["converged"] for d in r1.per_unit)


def test_cuhre_bubble_closed_form():
    """1-D units through the dummy coordinate: 1/eps + 2 + (4 - pi^2/12) eps + ..."""
    need_gpu()
    integ = integrator("bubble")
    r = integ.cuhre(rel_tol=1e-10)
    z3 = 1.2020569031595942
    exact = {-1: 1.0, 0: 2.0, 1: 4 - math.pi ** 2 / 12, 2: 8 - math.pi ** 2 / 6 - 7 * z3 / 3}
    for n, v in exact.items():
        assert abs(r.assembled[n] - v) <= r.assembled_errors[n] + 1e-12, (n, r.assembled[n], v)


def test_cuhre_physical_box():
    """Deformed contour: the continued closed form within the error bound, re and im."""
    need_gpu()
    import mpmath as mp
    from paper_1511_03614_gb300 import prepare_feynman, Integrator
    integ = Integrator(prepare_feynman(W.box_physical(), fuse_orders=True))
    r = integ.cuhre(rel_tol=1e-7)
    s, t = mp.mpf(3), mp.mpf(-1)
    with mp.workdps(30):
        Ls, Lt = mp.log(s) - 1j * mp.pi, mp.log(-t)

        def g(e):
            cg = mp.exp(mp.euler * e) * mp.gamma(1 + e) * mp.gamma(1 - e) ** 2 / mp.gamma(1 - 2 * e)
            return cg / (s * t) * (2 * (mp.exp(-e * Ls) + mp.exp(-e * Lt)) - e ** 2 * ((Ls - Lt) ** 2 + mp.pi ** 2))
        c = mp.taylor(g, 0, 2, method="quad", radius=0.25)
    for n in (-2, -1, 0):
        v = complex(c[n + 2])
        a, e = r.assembled[n], r.assembled_errors[n]
        assert abs(a.real - v.real) <= e.real + 1e-12 and abs(a.imag - v.imag) <= e.imag + 1e-12, (n, a, v, e)


def test_cuhre_region_cap_and_bad_options():
    """A region cap stops the run with finite, unconverged estimates; bad options are
    rejected before any launch."""
    need_gpu()
    from paper_1511_03614_gb300._native import FiestaError
    integ = integrator("box")
    r = integ.cuhre(rel_tol=1e-14, max_regions=200)
    assert all(np.isfinite(d["value"]) for d in r.per_unit)
    assert not all(d["converged"] for d in r.per_unit)
    assert sum(d["n_regions"] for d in r.per_unit) <= 200
    with pytest.raises(FiestaError):
        integ.cuhre(rel_tol=0.0, abs_tol=0.0)
    with pytest.raises(FiestaError):
        integ.cuhre(threads=48)
