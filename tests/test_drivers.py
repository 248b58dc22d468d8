"""The accuracy loop's host arithmetic in the library (no GPU): fiesta_assemble and
fiesta_allocate_points against the same formulas written out here in numpy, and the
Python drivers as pure marshalling (they return what the library wrote)."""
import contextlib
import ctypes as C
import math
import types

import numpy as np
import pytest

import workloads as W
from paper_1511_03614_gb300 import prepare_feynman, build


@pytest.fixture(scope="module")
def lib():
    build.build()
    from paper_1511_03614_gb300 import _native as N
    return N.load()


def _series(orders, parts, vals, sigs, pre, q, out, linear, correlated):
    """The assembled series written out: per-order sums over records, then
    R_n = sum_i c_i I_(n - (i - q))."""
    res = {}
    for n in out:
        tot = [0.0, 0.0]
        e1, e2 = [0.0, 0.0], [0.0, 0.0]
        for i, c in enumerate(pre):
            K = n - (i - q)
            for p in (0, 1):
                sel = (orders == K) & (parts == p)
                I = vals[sel].sum()
                E = sigs[sel].sum() if linear else math.sqrt((sigs[sel] ** 2).sum())
                tot[p] += c * I
                e1[p] += abs(c) * E
                e2[p] += (c * E) ** 2
        lin = linear or correlated
        res[n] = (tot, [e1[p] if lin else math.sqrt(e2[p]) for p in (0, 1)])
    return res


@pytest.mark.parametrize("linear,correlated,cplx", [(False, False, False), (False, True, True), (True, False, False)])
def test_assemble_matches_the_written_out_series(lib, linear, correlated, cplx):
    from paper_1511_03614_gb300 import _native as N
    rng = np.random.default_rng(7)
    n = 40
    orders = rng.integers(-3, 1, n).astype(np.int32)
    parts = (rng.integers(0, 2, n) if cplx else np.zeros(n)).astype(np.int32)
    vals = rng.normal(size=n)
    sigs = rng.uniform(0.01, 0.1, n)
    pre = np.array([1.0, -0.57, 0.98, -0.3])
    q, out = 1, list(range(-4, 1))
    o = N.AccuracyOptions()
    o.pre, o.n_pre, o.pre_q, o.correlated, o.out_lo = pre.ctypes.data_as(C.POINTER(C.c_double)), len(pre), q, \
        int(correlated), out[0]
    o.target, o.floor = 1e-3, 1e-2
    val, err, vim, eim = (np.zeros(len(out)) for _ in range(4))
    ratio = C.c_double()
    dp = lambda a: a.ctypes.data_as(C.POINTER(C.c_double))
    ip = lambda a: a.ctypes.data_as(C.POINTER(C.c_int32))
    assert lib.fiesta_assemble(C.byref(o), n, ip(orders), ip(parts), dp(vals), dp(sigs), int(linear), len(out),
                               dp(val), dp(err), dp(vim), dp(eim), C.byref(ratio)) == 0
    ref = _series(orders, parts, vals, sigs, pre, q, out, linear, correlated)
    big = max(math.hypot(*ref[m][0]) for m in out)
    worst = 0.0
    for i, m in enumerate(out):
        (re, im), (ere, eim_) = ref[m]
        assert math.isclose(val[i], re, rel_tol=1e-13, abs_tol=1e-14)
        assert math.isclose(vim[i], im, rel_tol=1e-13, abs_tol=1e-14)
        assert math.isclose(err[i], ere, rel_tol=1e-13) and math.isclose(eim[i], eim_, rel_tol=1e-13, abs_tol=1e-300)
        worst = max(worst, math.hypot(ere, eim_) / (1e-3 * max(math.hypot(re, im), 1e-2 * big)))
    assert math.isclose(ratio.value, worst, rel_tol=1e-12)


def test_allocate_points_neyman(lib):
    """Neyman allocation: a unit with four times the variance gets twice the points;
    the total cost is that of the uniform allocation; the clamp keeps every unit within
    [0.01, 64] x points."""
    from paper_1511_03614_gb300.api import allocate_points
    prep = prepare_feynman(W.box())
    nu = len(prep.units)
    values = {-2: 2.0, -1: -0.69, 0: -6.58}
    sig = np.full(nu, 1e-3)
    n_used = np.full(nu, 1e6)
    N1 = allocate_points(prep, sig, n_used, values, 1e-4, 1e-2, 100_000)
    cost = np.array([len(u.program.code) + 4 * u.dim + 8 for u in prep.units], dtype=float)
    assert abs(np.sum(N1 * cost) / (100_000 * cost.sum()) - 1) < 1e-3
    sig2 = sig.copy()
    sig2[3] *= 2.0
    N2 = allocate_points(prep, sig2, n_used, values, 1e-4, 1e-2, 100_000)
    ratio = (N2[3] / N2[4]) / (N1[3] / N1[4])
    assert abs(ratio - 2.0) < 0.01, ratio
    sig3 = sig.copy()
    sig3[5] *= 1e6
    N3 = allocate_points(prep, sig3, n_used, values, 1e-4, 1e-2, 100_000)
    assert int(np.argmax(N3)) == 5 and N3.min() == 1000 and N3.max() <= 64 * 100_000   # the lower clamp binds


def test_drivers_only_marshal(lib):
    """run_to_accuracy, run_to_accuracy_rqmc, run_flow and run_cuhre_to_accuracy return
    what fiesta_integrate_to_accuracy wrote, untouched: the loop and its arithmetic are
    in the library."""
    from paper_1511_03614_gb300 import api, _native as N
    prep = prepare_feynman(W.box())
    calls = []

    def fake(ctx, opts, state, n, val, err, vim, eim, uv, us):
        o, st = opts._obj, state._obj
        calls.append((o.method, o.proposal, o.max_calls))
        for i in range(n):
            val[i], err[i] = 10.0 + i, 0.5 + i
        for k in range(sum(u.n_out for u in prep.units)):
            uv[k], us[k] = -k, 1e-3 * k
        st.iterations, st.converged, st.gpu_ms, st.points, st.ratio = 7, 1, 1234.0, 99, 0.25
        return 0

    integ = types.SimpleNamespace(prep=prep, ctx=None, device=None, lib=types.SimpleNamespace(
        fiesta_integrate_to_accuracy=fake), _torch=types.SimpleNamespace(cuda=types.SimpleNamespace(
            device=lambda d: contextlib.nullcontext())))
    outs = tuple(prep.out_orders)
    for run, kw, method in ((api.run_to_accuracy, {}, 0), (api.run_to_accuracy_rqmc, {}, 1),
                            (api.run_flow, {}, 0), (api.run_cuhre_to_accuracy, {}, 2)):
        r = run(integ, **kw)
        assert r["values"] == {m: 10.0 + i for i, m in enumerate(outs)}
        assert r["errors"] == {m: 0.5 + i for i, m in enumerate(outs)}
        assert r["gpu_s"] == 1.234 and r["points"] == 99 and r["converged"] and r["ratio"] == 0.25
        assert list(r["unit_values"][:3]) == [0.0, -1.0, -2.0]
        assert calls[-1][0] == method
    assert calls[2][1] == N.PROPOSAL["flow"]
