"""Poles of order 2 (t^{-2+eps}: Taylor subtraction of order 1) on the GPU, through the
C ABI: per point against the oracle, and integrals against closed forms."""
import mpmath as mp
import numpy as np
import pytest

import workloads as W
from oracle import pipeline as P

from gpu_common import need_gpu, sample_points, reference, Parity

pytestmark = pytest.mark.gpu


def _beta(s):
    """int_0^1 t^(s-1)/(1+t) dt."""
    return (mp.digamma((s + 1) / 2) - mp.digamma(s / 2)) / 2


def test_higher_pole_points():
    need_gpu()
    from paper_1511_03614_gb300 import prepare_direct, Integrator
    par = Parity("pole2", "fp64")
    rng = np.random.default_rng(61)
    for prob in W.higher_pole_suite():
        prep = prepare_direct([prob])
        orc = P.direct_problem(prob)
        by = {(u.sector, u.order): u for u in orc.units}
        integ = Integrator(prep)
        for i, u in enumerate(prep.units):
            o = by[(u.sector, u.order)]
            X = sample_points(u.dim, rng, 32, n_log=32, n_edge=8)
            par.check(integ.eval_batch(i, X), reference(o, X), P.magnitude_numpy(o, X), X, (prob.name, u.order))
        integ.close()
    par.finish(0.3)


@pytest.mark.parametrize("which", [0, 1])
def test_higher_pole_integrals_match_closed_forms(which):
    """x^{-2+eps}/(1+x): beta(-1+eps); the separable two-dimensional integrand:
    beta(-1+eps) beta(eps); every requested order within 4 sigma."""
    need_gpu()
    from paper_1511_03614_gb300 import prepare_direct, Integrator
    prob = W.higher_pole_suite()[which]
    lead = 1 if which == 0 else 2
    with mp.workdps(30):
        c = mp.taylor(lambda e: e ** lead * _beta(-1 + e) * (_beta(e) if which else 1), 0, 5, method="quad",
                      radius=0.2)
    res = Integrator(prepare_direct([prob])).integrate(n_iter=10, points=1_000_000, seed=3)
    for K in prob.orders:
        v, s = res.values[K], res.errors[K]
        exact = float(c[K + lead])
        assert abs(v - exact) < 4 * s + 1e-12, (K, v, exact, s)
