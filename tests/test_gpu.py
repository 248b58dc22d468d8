"""GPU parity tests: the CUDA path (through the C ABI) against the oracle."""
import math

import mpmath as mp
import numpy as np
import pytest

import workloads as W
from oracle import pipeline as P, vegas as V, quadrature as Q

from gpu_common import need_gpu, feynman, integrator, stress, sample_points, reference, Parity

pytestmark = pytest.mark.gpu

# The per-point bar (scaled on every point, strictly relative on the well-conditioned
# points with all t_j >= 2^-20) is defined and justified in gpu_common.Parity.
MIN_STRICT_SHARE = {"fp64": 0.4, "fp32": 0.15}


def _check_points(prep, orc, idx, precision, rng, label, n_random=48, n_log=32):
    integ = integrator_for(prep)
    par = Parity(label, precision)
    for i in idx:
        u, o = prep.units[i], orc.units[i]
        X = sample_points(u.dim, rng, n_random, n_log=n_log)
        f = integ.eval_batch(i, X, precision)
        par.check(f, reference(o, X), P.magnitude_numpy(o, X), X, (label, int(i)))
    return par.finish(MIN_STRICT_SHARE[precision])


_INTEG = {}


def integrator_for(prep):
    from paper_1511_03614_gb300 import Integrator
    key = id(prep)
    if key not in _INTEG:
        _INTEG[key] = Integrator(prep)
    return _INTEG[key]


@pytest.mark.parametrize("precision", ["fp64", "fp32"])
@pytest.mark.parametrize("name", ["bubble", "box"])
def test_eval_batch_parity_all_units(name, precision):
    need_gpu()
    prep, orc = feynman(name)
    _check_points(prep, orc, range(len(prep.units)), precision, np.random.default_rng(10), name)


@pytest.mark.parametrize("precision", ["fp64", "fp32"])
def test_eval_batch_parity_double_box_sample(precision):
    need_gpu()
    prep, orc = feynman("double_box")
    rng = np.random.default_rng(11)
    idx = rng.choice(len(prep.units), 12, replace=False)
    _check_points(prep, orc, idx, precision, rng, "double_box")


def test_eval_batch_device_pointers():
    torch = need_gpu()
    prep, orc = feynman("box")
    integ = integrator("box")
    rng = np.random.default_rng(12)
    X = rng.uniform(size=(1000, 3))
    f_host = integ.eval_batch(5, X)
    f_dev = integ.eval_batch(5, torch.tensor(X, device="cuda")).cpu().numpy()
    assert np.array_equal(f_host, f_dev)


@pytest.mark.parametrize("name", ["bubble", "box"])
def test_same_points_first_iteration(name):
    """Iteration 0 on the uniform grid: GPU sum(v) vs the oracle's on the same Philox points."""
    need_gpu()
    prep, orc = feynman(name)
    integ = integrator(name)
    N = 20000
    integ.integrate(n_iter=1, points=N, seed=7, adapt=False)
    for i, (u, o) in enumerate(zip(prep.units, orc.units)):
        m, _ = integ.iterations(i, 1)
        r = V.integrate_unit(o.f_numpy, o.dim, 1, N, 7, u.rng_key, adapt=False)
        I, var, sv, sv2 = r.iters[0]
        U = V.philox.uniforms(7, u.rng_key, 0, 0, N, o.dim)
        X, J, _ = V.vegas_map(r.grids[0], U)
        absum = np.sum(np.abs(o.f_numpy(X) * J)) / N
        assert abs(m[0] - I) <= 1e-11 * absum, (i, m[0], I)


def test_vegas_iterations_follow_oracle():
    """Three adapted iterations: means follow the oracle's through the refined grids."""
    need_gpu()
    prep, orc = feynman("box")
    integ = integrator("box")
    N = 16384
    integ.integrate(n_iter=3, points=N, seed=3, adapt=True)
    for i in (0, 5, 17, len(prep.units) - 1):
        u, o = prep.units[i], orc.units[i]
        m, _ = integ.iterations(i, 3)
        r = V.integrate_unit(o.f_numpy, o.dim, 3, N, 3, u.rng_key)
        for it in range(3):
            assert abs(m[it] - r.iters[it][0]) <= 1e-9 * (abs(r.iters[it][0]) + math.sqrt(r.iters[it][1])), (i, it)
        g = integ.get_grid(i)
        g_or = V.refine(r.grids[1], r.hists[1])
        assert np.max(np.abs(g - g_or)) < 1e-9


def test_refine_parity():
    need_gpu()
    integ = integrator("bubble")
    rng = np.random.default_rng(4)
    for dim in (1, 3, 8):
        n = 5
        grids = np.stack([V.uniform_grid(dim) for _ in range(n)])
        grids[:, :, 1:-1] = np.sort(rng.uniform(size=(n, dim, 127)), axis=2)
        hists = rng.uniform(size=(n, dim, 128)) ** 6
        hists[0, 0, 5:] = 0.0                         # sparse histogram
        got = integ.refine(grids, hists, 1.5)
        for k in range(n):
            ref = V.refine(grids[k], hists[k], 1.5)
            assert np.max(np.abs(got[k] - ref)) < 1e-12


def test_bubble_closed_form():
    need_gpu()
    integ = integrator("bubble")
    res = integ.integrate(n_iter=10, points=100_000, seed=1)
    z3 = float(mp.zeta(3))
    exact = {-1: 1.0, 0: 2.0, 1: 4 - math.pi ** 2 / 12, 2: 8 - math.pi ** 2 / 6 - 7 * z3 / 3}
    for n, v in exact.items():
        s = res.assembled_errors[n]
        assert 0 < s < 1e-3
        assert abs(res.assembled[n] - v) < 4 * s, (n, res.assembled[n], v, s)


def test_box_closed_form():
    need_gpu()
    integ = integrator("box")
    res = integ.integrate(n_iter=10, points=1_000_000, seed=2)
    exact = {-2: 2.0, -1: -math.log(2.0), 0: -2 * math.pi ** 2 / 3}
    for n, v in exact.items():
        s = res.assembled_errors[n]
        assert 0 < s < 2e-3
        assert abs(res.assembled[n] - v) < 4 * s, (n, res.assembled[n], v, s)


def test_fp32_box_within_errors():
    need_gpu()
    integ = integrator("box")
    r64 = integ.integrate(n_iter=6, points=400_000, seed=5, precision="fp64")
    r32 = integ.integrate(n_iter=6, points=400_000, seed=5, precision="fp32")
    for n in r64.assembled:
        s = math.hypot(r64.assembled_errors[n], r32.assembled_errors[n])
        assert abs(r64.assembled[n] - r32.assembled[n]) < 3 * s + 1e-6


def test_linear_text_integrand():
    """The paper's worker example x[1]+0.2 integrates to 0.7 (Sec. 4.6)."""
    need_gpu()
    from paper_1511_03614_gb300 import parse_text, Integrator
    integ = Integrator(parse_text("1;\n0;\nx[1]+0.2;\n|"))
    res = integ.integrate(n_iter=5, points=100_000, seed=9)
    assert abs(res.values[0] - 0.7) < 4 * res.errors[0] and res.errors[0] < 1e-4


def test_stress_sobol_same_points():
    need_gpu()
    probs, prep, integ = stress(64)
    N = 4096
    integ.integrate(n_iter=1, points=N, seed=11, rng="sobol", adapt=False)
    for k in range(0, 64, 4):
        orc = P.direct_problem(probs[k])
        o = orc.units[0]
        m, _ = integ.iterations(k, 1)
        r = V.integrate_unit(o.f_numpy, o.dim, 1, N, 11, prep.units[k].rng_key, rng="sobol", adapt=False)
        U = V.sobol.uniforms(11, prep.units[k].rng_key, 0, 0, N, o.dim)
        X, J, _ = V.vegas_map(r.grids[0], U)
        absum = np.mean(np.abs(o.f_numpy(X) * J))
        assert abs(m[0] - r.iters[0][0]) <= 1e-11 * absum, k


def test_deterministic_without_adaptation():
    need_gpu()
    integ = integrator("box")
    a = integ.integrate(n_iter=2, points=50_000, seed=21, adapt=False)
    b = integ.integrate(n_iter=2, points=50_000, seed=21, adapt=False)
    assert [u["value"] for u in a.per_unit] == [u["value"] for u in b.per_unit]


def test_adapted_runs_reproduce_to_rounding():
    """Adapted runs repeat up to the summation order of the grid histogram: each block
    sums its points' v^2 into shared-memory bins with binary64 atomics and adds them to
    the unit's histogram in the order the blocks finish, so grid edges can differ in
    their last bits between runs; the repeated run's per-unit values agree far below
    their statistical errors."""
    need_gpu()
    integ = integrator("box")
    a = integ.integrate(n_iter=5, points=50_000, seed=21)
    b = integ.integrate(n_iter=5, points=50_000, seed=21)
    for ua, ub in zip(a.per_unit, b.per_unit):
        assert abs(ua["value"] - ub["value"]) <= 1e-10 * abs(ua["value"]) + 1e-6 * ua["sigma"], (ua, ub)


def test_timeout_returns_cleanly():
    need_gpu()
    from paper_1511_03614_gb300._native import FiestaError
    integ = integrator("box")
    with pytest.raises(FiestaError) as e:
        integ.integrate(n_iter=1, points=50_000_000, seed=1, timeout_ms=1)
    assert e.value.code == -4
    res = integ.integrate(n_iter=2, points=10_000, seed=1)     # context still usable
    assert math.isfinite(res.values[0])


def test_nonfinite_samples_are_reported():
    """Fault injection on the host: a NaN constant in one unit's program."""
    need_gpu()
    from paper_1511_03614_gb300 import parse_text, Integrator
    from paper_1511_03614_gb300._native import FiestaError
    prep = parse_text("1; 0; x[1]*0.5 + 1.0; |")
    prep.units[0].program.consts[:] = np.nan
    integ = Integrator(prep)
    with pytest.raises(FiestaError) as e:
        integ.integrate(n_iter=1, points=1000)
    assert e.value.code == -5 and "unit 0" in str(e.value)


def test_table_log_within_one_ulp():
    """The interpreter's binary64 log (Tang's table method) against the exact value:
    within 1 ulp, the accuracy bound CUDA documents for its own log."""
    need_gpu()
    from paper_1511_03614_gb300 import parse_text, Integrator
    rng = np.random.default_rng(13)
    x = np.concatenate([np.exp(rng.uniform(-690, 0, 4000)), 1 - rng.uniform(0, 1e-3, 500),
                        rng.uniform(0.5, 1, 2000), [2.0 ** -1022, 0.7071067811865476, 0.70710671, 1.0]])
    for text, scale in (("1; 0; l[x[1]]; |", 1.0), ("1; 0; l[x[1]*1e300]; |", 1e300)):
        integ = Integrator(parse_text(text))
        got = integ.eval_batch(0, x[:, None])
        arg = x * scale
        with mp.workdps(40):
            ref = [mp.log(mp.mpf(float(a))) for a in arg]
        ulps = [abs(mp.mpf(float(g)) - r) / math.ulp(float(r)) if float(r) != 0 else abs(g) for g, r in zip(got, ref)]
        assert max(ulps) <= 1.0, max(ulps)


def test_reciprocal_within_one_ulp():
    """The interpreter's binary64 reciprocal (Newton-Raphson refinement of the hardware's
    approximate reciprocal) against the exact value: within 1 ulp over the whole
    exponent range, both signs, and IEEE results for zero, subnormal and overflowing
    arguments (the cases that take the IEEE division)."""
    need_gpu()
    from paper_1511_03614_gb300 import parse_text, Integrator
    rng = np.random.default_rng(17)
    x = np.concatenate([np.exp(rng.uniform(-740, 0, 6000)), rng.uniform(0.5, 1, 2000),
                        [2.0 ** -1022, 2.0 ** -1021, 2.0 ** -1020, 1.0, 0.75, 1 - 2.0 ** -53]])
    for text, scale in (("1; 0; p[x[1],-1]; |", 1.0), ("1; 0; p[x[1]*1e300,-1]; |", 1e300),
                        ("1; 0; p[x[1]*-3.0,-1]; |", -3.0), ("1; 0; p[x[1]*1.7976931348623157e308,-1]; |",
                                                            1.7976931348623157e308)):
        integ = Integrator(parse_text(text))
        got = integ.eval_batch(0, x[:, None])
        arg = x * scale
        with np.errstate(divide="ignore", over="ignore"):
            ieee = 1.0 / arg
        special = ~np.isfinite(ieee) | (np.abs(arg) < 2.0 ** -1021) | (np.abs(arg) >= 2.0 ** 1022)
        assert np.array_equal(got[special], ieee[special])
        with mp.workdps(40):
            ulps = [float(abs(mp.mpf(float(g)) - 1 / mp.mpf(float(a))) / math.ulp(float(r)))
                    for g, a, r in zip(got[~special], arg[~special], ieee[~special])]
        assert max(ulps) <= 1.0, max(ulps)
    integ = Integrator(parse_text("1; 0; p[x[1],-1]; |"))
    z = np.array([[0.0], [5e-324], [2.0 ** -1030]])
    with np.errstate(divide="ignore"):
        assert np.array_equal(integ.eval_batch(0, z), 1.0 / z[:, 0])


def test_precision_probe_and_auto_mode():
    """The per-unit binary32 probe and FIESTA_AUTO: box results stay within errors of the closed form."""
    need_gpu()
    prep, _ = feynman("box")
    integ = integrator("box")
    em, ex = integ.precision_probe(n_points=16384, seed=4)
    em2, ex2 = integ.precision_probe(n_points=16384, seed=4)
    assert np.array_equal(em, em2) and np.array_equal(ex, ex2)          # deterministic
    assert np.all(em < 1e-5) and np.all(np.isfinite(ex))
    res = integ.integrate(n_iter=6, points=400_000, seed=4, precision="auto", fp32_budget=1e-6)
    exact = {-2: 2.0, -1: -math.log(2.0), 0: -2 * math.pi ** 2 / 3}
    for n, v in exact.items():
        s = res.assembled_errors[n]
        assert abs(res.assembled[n] - v) < 4 * s + 1e-6, (n, res.assembled[n], v, s)
    used = [u["precision"] for u in res.per_unit]
    assert used.count("fp32") == res.stats["units_fp32"]
    for u in res.per_unit:
        assert (u["precision"] == "fp32") == (u["fp32_error"] <= 1e-6)
        assert u["fp32_error"] < 1e-5


def test_block_shape_does_not_change_the_points():
    """Autotuned and fixed launch shapes evaluate the same point streams."""
    need_gpu()
    integ = integrator("box")
    a = integ.integrate(n_iter=1, points=300_000, seed=8, adapt=False, threads=128, points_per_thread=16)
    b = integ.integrate(n_iter=1, points=300_000, seed=8, adapt=False, threads=0, points_per_thread=0)
    c = integ.integrate(n_iter=1, points=300_000, seed=8, adapt=False, threads=64, points_per_thread=32)
    for x, y, z in zip(a.per_unit, b.per_unit, c.per_unit):
        scale = abs(x["value"]) + x["sigma"] * 1e3
        assert abs(x["value"] - y["value"]) <= 1e-12 * scale
        assert abs(x["value"] - z["value"]) <= 1e-12 * scale


def test_stress_low_dim_against_gauss_legendre():
    """Three-dimensional stress integrands (smooth, P >= 0.1): Sobol estimate vs a
    tensor Gauss-Legendre rule of the oracle's integrand."""
    need_gpu()
    probs, prep, integ = stress(64)
    res = integ.integrate(n_iter=1, points=1 << 18, seed=12, rng="sobol", adapt=False)
    xg, wg = np.polynomial.legendre.leggauss(24)
    xg, wg = (xg + 1) / 2, wg / 2
    checked = 0
    for k, prob in enumerate(probs):
        if prob.dim != 3:
            continue
        o = P.direct_problem(prob).units[0]
        X = np.stack(np.meshgrid(xg, xg, xg, indexing="ij"), -1).reshape(-1, 3)
        Wt = np.einsum("i,j,k->ijk", wg, wg, wg).ravel()
        truth = float(np.sum(Wt * o.f_numpy(X)))
        r = res.per_unit[k]
        assert abs(r["value"] - truth) <= 3 * r["sigma"] + 1e-9 * abs(truth), (k, r["value"], truth, r["sigma"])
        checked += 1
    assert checked >= 3


def test_checkpoint_resume_continues_the_same_streams(tmp_path):
    """An interrupted run resumed from its checkpoint gives the uninterrupted run's results."""
    need_gpu()
    from paper_1511_03614_gb300 import Integrator
    from paper_1511_03614_gb300.api import run_to_accuracy
    prep, _ = feynman("bubble")
    full = run_to_accuracy(Integrator(prep), target=1e-12, points=50_000, max_iters=6, seed=5)
    ck = str(tmp_path / "bubble.ck")
    run_to_accuracy(Integrator(prep), target=1e-12, points=50_000, max_iters=6, seed=5, checkpoint=ck, stop_after=2)
    resumed = run_to_accuracy(Integrator(prep), target=1e-12, points=50_000, max_iters=6, seed=5, resume=ck)
    assert resumed["iterations"] == full["iterations"] == 6
    d = np.abs(resumed["unit_values"] - full["unit_values"])
    assert np.all(d <= 1e-9 * (np.abs(full["unit_values"]) + full["unit_sigmas"]))


def test_double_box_strategy_invariance():
    """Sector sums do not depend on the decomposition strategy (M: 293 sectors, R: 313)."""
    need_gpu()
    import workloads as W
    from paper_1511_03614_gb300 import prepare_feynman, Integrator
    res = {}
    for strat in ("M", "R"):
        prep = prepare_feynman(W.double_box(), strategy=strat)
        res[strat] = Integrator(prep).integrate(n_iter=6, points=200_000, seed=3, precision="fp32")
    assert len(prepare_feynman(W.double_box(), strategy="R").sectors) != len(prepare_feynman(W.double_box()).sectors)
    for n in res["M"].assembled:
        s = math.hypot(res["M"].assembled_errors[n], res["R"].assembled_errors[n])
        assert abs(res["M"].assembled[n] - res["R"].assembled[n]) < 4 * s, (n, res["M"].assembled[n], res["R"].assembled[n], s)


def test_fused_units_match_oracle_and_closed_form():
    """Fused multi-order units: per point and per same-point iteration against the
    oracle's per-order units, and the box closed form."""
    need_gpu()
    import workloads as W
    from paper_1511_03614_gb300 import prepare_feynman, Integrator
    prep = prepare_feynman(W.box(), fuse_orders=True)
    _, orc = feynman("box")
    by = {(u.sector, u.order): u for u in orc.units}
    integ = Integrator(prep)
    rng = np.random.default_rng(21)
    par = Parity("box-fused", "fp64")
    for i, u in enumerate(prep.units):
        X = sample_points(u.dim, rng, 32, n_log=16)
        f = integ.eval_batch(i, X)
        for k in range(u.n_out):
            o = by[(u.sector, u.order + k)]
            par.check(f[:, k], reference(o, X), P.magnitude_numpy(o, X), X, (i, k))
    par.finish(MIN_STRICT_SHARE["fp64"])
    N = 20000
    integ.integrate(n_iter=1, points=N, seed=9, adapt=False)
    for i, u in enumerate(prep.units):
        for k in range(u.n_out):
            o = by[(u.sector, u.order + k)]
            m, _ = integ.iterations(i, 1, k)
            r = V.integrate_unit(o.f_numpy, o.dim, 1, N, 9, u.rng_key, adapt=False)
            U = V.philox.uniforms(9, u.rng_key, 0, 0, N, o.dim)
            X, J, _ = V.vegas_map(r.grids[0], U)
            absum = np.mean(np.abs(o.f_numpy(X) * J))
            assert abs(m[0] - r.iters[0][0]) <= 1e-11 * absum
    res = integ.integrate(n_iter=10, points=1_000_000, seed=2)
    assert len(res.per_unit) == sum(u.n_out for u in prep.units)
    exact = {-2: 2.0, -1: -math.log(2.0), 0: -2 * math.pi ** 2 / 3}
    for n, v in exact.items():
        s = res.assembled_errors[n]
        assert abs(res.assembled[n] - v) < 4 * s, (n, res.assembled[n], v, s)


def test_graph_replay_matches_direct_launches():
    """The iteration loop replayed as a CUDA graph gives what direct launches give."""
    need_gpu()
    integ = integrator("box")
    kw = dict(n_iter=3, points=100_000, seed=31, adapt=False)
    a = integ.integrate(graph=False, **kw)
    b = integ.integrate(graph=True, **kw)       # captured
    c = integ.integrate(graph=True, **kw)       # replayed
    for x, y, z in zip(a.per_unit, b.per_unit, c.per_unit):
        assert x["value"] == y["value"] == z["value"] and x["sigma"] == y["sigma"] == z["sigma"]
    assert b.stats["eval_ms"] > 0 and c.stats["eval_ms"] > 0


def test_whole_unit_items_same_points():
    """With many more units than resident blocks (1300 stress integrands on 152 SMs) a work
    item is a whole unit: the same Sobol points and sums as the oracle, and the same
    means as the chunked schedule of a small slice of the same units."""
    need_gpu()
    probs, prep, integ = stress(1300)
    N = 4096
    integ.integrate(n_iter=1, points=N, seed=17, rng="sobol", adapt=False)
    whole = {k: integ.iterations(k, 1)[0][0] for k in range(0, 1300, 97)}
    for k in list(whole)[:8]:
        o = P.direct_problem(probs[k]).units[0]
        r = V.integrate_unit(o.f_numpy, o.dim, 1, N, 17, prep.units[k].rng_key, rng="sobol", adapt=False)
        U = V.sobol.uniforms(17, prep.units[k].rng_key, 0, 0, N, o.dim)
        X, J, _ = V.vegas_map(r.grids[0], U)
        absum = np.mean(np.abs(o.f_numpy(X) * J))
        assert abs(whole[k] - r.iters[0][0]) <= 1e-11 * absum, k
    integ.integrate(n_iter=1, points=N, seed=17, rng="sobol", adapt=False, units=(0, 98), assemble_result=False)
    for k in (0, 97):
        m = integ.iterations(k, 1)[0][0]
        assert abs(m - whole[k]) <= 1e-13 * abs(m) + 1e-300, k
