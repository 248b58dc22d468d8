"""GPU parity of the kernel variants the large workloads run, through the C ABI.

* Fused double-box units (one program per sector returning all its eps orders,
  Sec. 4.3's per-order integrands evaluated at shared points): per point against
  the oracle's per-order integrands, and same-point sums with the per-thread sums
  of the evaluation kernel forced into registers and into shared memory.
* Mixed units (the paper's MixSectors option, Sec. 4.4: several sectors summed
  into one integrand): per point against the sum of the oracle's sector
  integrands, and the box integrated from mixed units against its closed form.
* The stress set: per point on 120 units covering every dimension 3..8 and the
  longest programs of the 10 000.
"""
import math

import numpy as np
import pytest

import workloads as W
from oracle import pipeline as P, vegas as V

from gpu_common import need_gpu, feynman, feynman_fused, sample_points, reference, Parity, C_SCALED, UROUND

pytestmark = pytest.mark.gpu

MIN_STRICT_SHARE = {"fp64": 0.4, "fp32": 0.15}
_INTEG = {}


def _integ(prep):
    from paper_1511_03614_gb300 import Integrator
    if id(prep) not in _INTEG:
        _INTEG[id(prep)] = (prep, Integrator(prep))
    return _INTEG[id(prep)][1]


def _dbox_fused_sample(n_total=40, seed=31):
    """The fused double-box units with the most slots and the longest programs, filled
    up to ``n_total`` with a random sample of the rest."""
    prep = feynman_fused("double_box")
    n = len(prep.units)
    by_slots = sorted(range(n), key=lambda i: -prep.units[i].program.n_slots)[:5]
    by_len = sorted(range(n), key=lambda i: -len(prep.units[i].program.code))[:5]
    top = set(by_slots) | set(by_len)
    rng = np.random.default_rng(seed)
    rest = [i for i in range(n) if i not in top]
    idx = sorted(top | set(rng.choice(rest, max(n_total - len(top), 0), replace=False).tolist()))
    return prep, idx


@pytest.mark.parametrize("precision", ["fp64", "fp32"])
def test_fused_double_box_points(precision):
    need_gpu()
    prep, idx = _dbox_fused_sample()
    assert len(idx) >= 40
    _, orc = feynman("double_box")
    by = {(u.sector, u.order): u for u in orc.units}
    integ = _integ(prep)
    rng = np.random.default_rng(32)
    par = Parity("double_box-fused", precision)
    for i in idx:
        u = prep.units[i]
        X = sample_points(u.dim, rng, 16, n_log=16, n_edge=8)
        f = integ.eval_batch(i, X, precision)
        for k in range(u.n_out):
            o = by[(u.sector, u.order + k)]
            par.check(f[:, k], reference(o, X), P.magnitude_numpy(o, X), X, (int(i), k))
    par.finish(MIN_STRICT_SHARE[precision])


@pytest.mark.parametrize("precision", ["fp64", "fp32"])
def test_fused_six_orders_points(precision):
    """The largest fused unit: the box expanded to eps^3 carries six orders (the most a
    unit holds) in most sectors; every result per point against the oracle's integrand
    of its sector and order."""
    need_gpu()
    from paper_1511_03614_gb300 import prepare_feynman
    prob = W.box(order=3)
    prep = prepare_feynman(prob, fuse_orders=True)
    assert max(u.n_out for u in prep.units) == 6
    by = {(u.sector, u.order): u for u in P.feynman_problem(prob).units}
    integ = _integ(prep)
    rng = np.random.default_rng(38)
    par = Parity("box-eps3-fused", precision)
    for i, u in enumerate(prep.units):
        X = sample_points(u.dim, rng, 24, n_log=16, n_edge=8)
        f = integ.eval_batch(i, X, precision)
        for k in range(u.n_out):
            o = by[(u.sector, u.order + k)]
            par.check(f[:, k], reference(o, X), P.magnitude_numpy(o, X), X, (i, k))
    par.finish(MIN_STRICT_SHARE[precision])


@pytest.mark.parametrize("accumulate,threads", [("registers", 256), ("shared", 128)])
def test_fused_double_box_same_point_sums(accumulate, threads):
    """Iteration 0 on the uniform grid, every fused unit at once: each result's mean
    equals the oracle's Vegas estimate of that sector and order at the same Philox
    points, with the kernel's per-thread sums in registers (the variant the double-box
    benchmark runs) and in shared memory.  Both means are binary64 sums of values that
    each err by at most C_SCALED u M (the per-point bar), so they may differ by twice
    that summed: 2 C_SCALED u mean(M |J|).  Double-box units cancel strongly (mean(M J)
    reaches 1.7e5 mean|v| on the eps^0 result of a 4-subtraction sector)."""
    need_gpu()
    prep, idx = _dbox_fused_sample(n_total=16, seed=33)
    _, orc = feynman("double_box")
    by = {(u.sector, u.order): u for u in orc.units}
    integ = _integ(prep)
    N = 8192
    res = integ.integrate(n_iter=1, points=N, seed=13, adapt=False, accumulate=accumulate, threads=threads,
                          points_per_thread=16)
    assert res.stats["threads"][0] == threads
    for i in idx:
        u = prep.units[i]
        U = V.philox.uniforms(13, u.rng_key, 0, 0, N, u.dim)
        X, J, _ = V.vegas_map(V.uniform_grid(u.dim), U)
        for k in range(u.n_out):
            o = by[(u.sector, u.order + k)]
            m, _ = integ.iterations(i, 1, k)
            v = o.f_numpy(X) * J
            bound = 2 * C_SCALED * UROUND["fp64"] * np.mean(P.magnitude_numpy(o, X) * np.abs(J))
            assert abs(m[0] - np.mean(v)) <= bound, (int(i), k, m[0], np.mean(v), bound)


def test_slot_groups_same_point_sums():
    """With the launch shape left to the autotuner, the fused double box's binary64 units
    run in two launches per iteration, split by slot count (the units whose slot files
    fit 512-thread blocks, and the rest); every sampled unit of both groups has the
    oracle's Vegas estimate at the same Philox points, within the bar of the test above."""
    need_gpu()
    prep, idx = _dbox_fused_sample(n_total=16, seed=35)
    _, orc = feynman("double_box")
    by = {(u.sector, u.order): u for u in orc.units}
    integ = _integ(prep)
    N = 50000          # both groups hold at least 512 * 16 points per SM: the split pays
    res = integ.integrate(n_iter=1, points=N, seed=14, adapt=False)
    assert res.stats["eval_groups"] == 2 and res.stats["wide_threads"][0] > 0, res.stats
    slots = [prep.units[i].program.n_slots for i in idx]
    assert min(slots) <= 40 < max(slots)
    for i in idx:
        u = prep.units[i]
        U = V.philox.uniforms(14, u.rng_key, 0, 0, N, u.dim)
        X, J, _ = V.vegas_map(V.uniform_grid(u.dim), U)
        for k in range(u.n_out):
            o = by[(u.sector, u.order + k)]
            m, _ = integ.iterations(i, 1, k)
            v = o.f_numpy(X) * J
            bound = 2 * C_SCALED * UROUND["fp64"] * np.mean(P.magnitude_numpy(o, X) * np.abs(J))
            assert abs(m[0] - np.mean(v)) <= bound, (int(i), k, m[0], np.mean(v), bound)


def test_mixed_units_points():
    """MixSectors programs: per point, the sum of the oracle's integrands of the sectors
    the unit mixes (box: 3 sectors per program; double box: 4, a sample of 8 units)."""
    need_gpu()
    for name, mix, n_units in (("box", 3, None), ("double_box", 4, 8)):
        prep = feynman_fused(name, mix)
        _, orc = feynman(name)
        by = {(u.sector, u.order): u for u in orc.units}
        integ = _integ(prep)
        rng = np.random.default_rng(34)
        mixed = [i for i, u in enumerate(prep.units) if u.sectors and len(u.sectors) > 1]
        assert mixed
        idx = mixed if n_units is None else rng.choice(mixed, n_units, replace=False)
        par = Parity(f"{name}-mix{mix}", "fp64")
        for i in idx:
            u = prep.units[i]
            X = sample_points(u.dim, rng, 16, n_log=16, n_edge=8)
            f = integ.eval_batch(int(i), X)
            for k in range(u.n_out):
                parts = [by[(s, u.order + k)] for s in u.sectors if (s, u.order + k) in by]
                ref = sum(reference(o, X) for o in parts)
                M = sum(P.magnitude_numpy(o, X) for o in parts)
                par.check(f[:, k], ref, M, X, (int(i), k))
        par.finish(0.3)


def test_mixed_units_box_closed_form():
    """The box integrated from programs that mix three sectors each: every order within
    3 standard errors (the correlated bound of fused units) of the closed form."""
    need_gpu()
    prep = feynman_fused("box", 3)
    assert any(u.sectors and len(u.sectors) == 3 for u in prep.units)
    res = _integ(prep).integrate(n_iter=10, points=1_000_000, seed=2)
    exact = {-2: 2.0, -1: -math.log(2.0), 0: -2 * math.pi ** 2 / 3}
    for n, v in exact.items():
        s = res.assembled_errors[n]
        assert 0 < s < 2e-3
        assert abs(res.assembled[n] - v) < 3 * s, (n, res.assembled[n], v, s)


def _stress_sample():
    from paper_1511_03614_gb300 import prepare_direct
    probs = W.stress_suite()
    prep = prepare_direct(probs)
    rng = np.random.default_rng(35)
    idx = []
    for d in range(3, 9):
        of_d = [i for i, u in enumerate(prep.units) if u.dim == d]
        longest = sorted(of_d, key=lambda i: -len(prep.units[i].program.code))[:5]
        rest = [i for i in of_d if i not in longest]
        idx += longest + rng.choice(rest, 15, replace=False).tolist()
    return probs, prep, sorted(idx)


@pytest.mark.parametrize("precision", ["fp64", "fp32"])
def test_stress_all_orders_points(precision):
    """The stress integrands expanded to every order eps^0..eps^2 (one unit per
    coefficient): per point against the oracle's expansion of the same integrands."""
    need_gpu()
    from paper_1511_03614_gb300 import prepare_direct
    probs = W.stress_suite(40, all_orders=True)
    prep = prepare_direct(probs, "stress")
    assert len(prep.units) == sum(len(p.orders) for p in probs) > 100
    integ = _integ(prep)
    rng = np.random.default_rng(37)
    par = Parity("stress-all-orders", precision)
    oracle_units = {}
    for k, p in enumerate(probs):
        for o in P.direct_problem(p).units:
            oracle_units[(k, o.order)] = o
    for i, u in enumerate(prep.units):
        o = oracle_units[(u.sector, u.order)]
        X = sample_points(u.dim, rng, 8, n_log=4, n_edge=4)
        f = integ.eval_batch(i, X, precision)
        par.check(f, reference(o, X), P.magnitude_numpy(o, X), X, i)
    par.finish(MIN_STRICT_SHARE[precision])


@pytest.mark.parametrize("precision", ["fp64", "fp32"])
def test_stress_points(precision):
    need_gpu()
    global _STRESS
    if "_STRESS" not in globals():
        _STRESS = _stress_sample()
    probs, prep, idx = _STRESS
    assert len(idx) >= 100 and {prep.units[i].dim for i in idx} == set(range(3, 9))
    integ = _integ(prep)
    rng = np.random.default_rng(36)
    par = Parity("stress", precision)
    for i in idx:
        u = prep.units[i]
        o = P.direct_problem(probs[i]).units[0]
        X = sample_points(u.dim, rng, 16, n_log=8, n_edge=8)
        f = integ.eval_batch(int(i), X, precision)
        par.check(f, reference(o, X), P.magnitude_numpy(o, X), X, int(i))
    par.finish(MIN_STRICT_SHARE[precision])
