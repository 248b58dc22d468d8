"""Per-unit point counts (fiesta_options.unit_points) and the variance-driven
allocation of the accuracy driver."""
import math

import numpy as np
import pytest

from oracle import vegas as V

from gpu_common import need_gpu, feynman, integrator

pytestmark = pytest.mark.gpu


def test_unit_points_same_points_as_oracle():
    """Units run with different point counts: each unit's iteration 0 equals the
    oracle's Vegas on its own number of Philox points (same streams), and the
    per-unit records report those counts."""
    need_gpu()
    prep, orc = feynman("box")
    integ = integrator("box")
    rng = np.random.default_rng(5)
    npts = rng.integers(3000, 40000, len(prep.units))
    res = integ.integrate(n_iter=1, points=20000, seed=9, adapt=False, unit_points=npts)
    assert [d["n_points"] for d in res.per_unit] == list(npts)
    assert res.stats["points"] == int(npts.sum())
    for i in (0, 3, 11, 20, len(prep.units) - 1):
        u, o = prep.units[i], orc.units[i]
        m, _ = integ.iterations(i, 1)
        r = V.integrate_unit(o.f_numpy, o.dim, 1, int(npts[i]), 9, u.rng_key, adapt=False)
        U = V.philox.uniforms(9, u.rng_key, 0, 0, int(npts[i]), o.dim)
        X, J, _ = V.vegas_map(r.grids[0], U)
        absum = np.mean(np.abs(o.f_numpy(X) * J))
        assert abs(m[0] - r.iters[0][0]) <= 1e-11 * absum, i


def test_equal_unit_points_change_nothing():
    """unit_points all equal to points_per_iter gives bit-identical results (without
    grid adaptation, whose shared-memory histogram sums are not order-deterministic)."""
    need_gpu()
    integ = integrator("box")
    n = len(integ.prep.units)
    a = integ.integrate(n_iter=3, points=30000, seed=4, adapt=False)
    b = integ.integrate(n_iter=3, points=30000, seed=4, adapt=False, unit_points=np.full(n, 30000))
    assert a.values == b.values and a.errors == b.errors


def test_allocation_reaches_target():
    """The accuracy driver with allocation converges to the box's closed form (every
    order within 4 sigma) and moves points between units."""
    need_gpu()
    from paper_1511_03614_gb300 import prepare_feynman, Integrator
    import workloads as W
    from paper_1511_03614_gb300.api import run_to_accuracy, allocate_points
    integ = Integrator(prepare_feynman(W.box()))
    r = run_to_accuracy(integ, target=3e-4, points=200_000, max_iters=60, allocate=True)
    assert r["converged"]
    exact = {-2: 2.0, -1: -math.log(2.0), 0: -2 * math.pi ** 2 / 3}
    for n, v in exact.items():
        assert abs(r["values"][n] - v) < 4 * r["errors"][n] + 1e-9, n
    sig = r["unit_sigmas"]
    N = allocate_points(integ.prep, sig, np.full(len(integ.prep.units), 1e6),
                        {K: 1.0 for K in (-2, -1, 0)}, 1e-4, 1e-2, 200_000)
    assert N.max() > 2 * N.min()


def test_rqmc_replicates_reach_the_closed_form():
    """Randomised QMC on adapted grids: Sobol replicates with independent digital
    shifts give unbiased unit estimates whose spread is the error; the box's closed
    form within 4 sigma at a 1e-5 target."""
    need_gpu()
    from paper_1511_03614_gb300 import prepare_feynman, Integrator
    import workloads as W
    from paper_1511_03614_gb300.api import run_to_accuracy_rqmc
    integ = Integrator(prepare_feynman(W.box(), fuse_orders=True))
    r = run_to_accuracy_rqmc(integ, target=1e-5, points=1 << 16, replicates=8)
    assert r["converged"]
    exact = {-2: 2.0, -1: -math.log(2.0), 0: -2 * math.pi ** 2 / 3}
    for n, v in exact.items():
        assert abs(r["values"][n] - v) < 4 * r["errors"][n] + 1e-12, (n, r["values"][n], v, r["errors"][n])


def test_vegas_loop_combines_every_counted_iteration():
    """fiesta_integrate_to_accuracy one call at a time (max_calls = 1): after each call the
    running sums hold exactly the inverse-variance sums of every iteration but the first
    (skip = 1), the per-iteration results being those fiesta_iterations reports for the
    call; the returned unit values and sigmas are swi / sw and sqrt(1 / sw)."""
    need_gpu()
    from paper_1511_03614_gb300 import prepare_feynman, Integrator
    from paper_1511_03614_gb300.api import integrate_to_accuracy, _records
    import workloads as W
    integ = Integrator(prepare_feynman(W.bubble()))
    recs = _records(integ.prep)
    sw, swi = np.zeros(len(recs)), np.zeros(len(recs))
    state = None
    for call in range(3):
        res, state = integrate_to_accuracy(integ, state, method="vegas", target=1e-12, points=20_000,
                                           iters_per_call=2, max_iters=6, skip=1, max_calls=1, seed=3)
        for k, (u, o) in enumerate(recs):
            m, v = integ.iterations(u, 2, o)
            for j in range(2):
                if 2 * call + j >= 1:
                    sw[k] += 1.0 / v[j]
                    swi[k] += m[j] / v[j]
        assert state[0].iterations == 2 * (call + 1)
        assert np.allclose(state[1]["sw"], sw, rtol=1e-13, atol=0) and np.allclose(state[1]["swi"], swi, rtol=1e-12)
    assert np.allclose(res["unit_values"], swi / sw, rtol=1e-12)
    assert np.allclose(res["unit_sigmas"], np.sqrt(1.0 / sw), rtol=1e-12)


def test_rqmc_loop_uses_the_replicate_spread():
    """One round of FIESTA_METHOD_RQMC: each result's estimate is the mean of its
    replicates and its variance their sample variance over the replicate count."""
    need_gpu()
    from paper_1511_03614_gb300 import prepare_feynman, Integrator
    from paper_1511_03614_gb300.api import integrate_to_accuracy, _records
    import workloads as W
    integ = Integrator(prepare_feynman(W.box(), fuse_orders=True))
    recs = _records(integ.prep)
    res, state = integrate_to_accuracy(integ, method="rqmc", target=1e-12, points=1 << 12, replicates=8,
                                       adapt_iters=2, max_iters=1, seed=5)
    for k, (u, o) in enumerate(recs):
        m, _ = integ.iterations(u, 8, o)
        var = np.var(m, ddof=1) / 8
        assert math.isclose(res["unit_values"][k], np.mean(m), rel_tol=1e-12, abs_tol=1e-15)
        assert math.isclose(res["unit_sigmas"][k], math.sqrt(var), rel_tol=1e-9)
    assert state[0].points_per_replicate == 1 << 12


@pytest.mark.parametrize("name", ["box", "box_physical"])
def test_rqmc_assembles_each_replicate(name):
    """One round of FIESTA_METHOD_RQMC on fused units: each assembled order's value is
    the mean over the replicates of the series assembled from that replicate's results
    (through the prefactor), and its error their spread over sqrt(replicates), so the
    correlation between a fused unit's orders enters as measured."""
    need_gpu()
    from paper_1511_03614_gb300 import prepare_feynman, Integrator
    from paper_1511_03614_gb300.api import integrate_to_accuracy, _records
    import workloads as W
    prep = prepare_feynman(getattr(W, name)(), fuse_orders=True)
    integ = Integrator(prep)
    recs = _records(prep)
    R = 8
    res, _ = integrate_to_accuracy(integ, method="rqmc", target=1e-12, points=1 << 12, replicates=R,
                                   adapt_iters=2, max_iters=1, seed=7)
    q, c = prep.prefactor
    orders = list(prep.out_orders)
    A = np.zeros((R, len(orders)), dtype=complex)
    for j in range(R):
        I = {}
        for (u, o) in recs:
            unit = prep.units[u]
            m, _ = integ.iterations(u, R, o)
            K = unit.order + (o // 2 if unit.cplx else o)
            I[K] = I.get(K, 0) + (1j * m[j] if unit.cplx and o % 2 else m[j])
        for a, n in enumerate(orders):
            A[j, a] = sum(ci * I.get(n - (i - q), 0) for i, ci in enumerate(c))
    for a, n in enumerate(orders):
        mean, err = res["values"][n], res["errors"][n]
        for part in (np.real, np.imag):
            x = part(A[:, a])
            if np.all(x == 0):
                continue
            assert math.isclose(part(mean), np.mean(x), rel_tol=1e-11, abs_tol=1e-13), (n, part(mean), np.mean(x))
            assert math.isclose(part(err), math.sqrt(np.var(x, ddof=1) / R), rel_tol=1e-8), (n, part(err))


def test_flow_proposal_in_fiesta_integrate():
    """fiesta_options.proposal = FLOW: iterations drawn from the units' flows, trained
    between iterations; the box's closed form within 4 sigma of the combined result."""
    need_gpu()
    from paper_1511_03614_gb300 import prepare_feynman, Integrator
    import workloads as W
    integ = Integrator(prepare_feynman(W.box(), fuse_orders=True))
    res = integ.integrate(n_iter=6, points=400_000, seed=4, precision="fp32", proposal="flow",
                          flow_train_steps=10, skip_first=True)
    exact = {-2: 2.0, -1: -math.log(2.0), 0: -2 * math.pi ** 2 / 3}
    for n, v in exact.items():
        s = res.assembled_errors[n]
        assert 0 < s < 5e-3 and abs(res.assembled[n] - v) < 4 * s, (n, res.assembled[n], v, s)
    assert res.stats["kernels_launched"] > 6
