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
