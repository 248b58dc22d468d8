"""GPU edge cases of the sampling path: an empty evaluation batch, the smallest point
count, point counts that leave a ragged last work item, and an integrand of zero
variance (the degenerate case of the Vegas iteration statistics)."""
import numpy as np
import pytest

from oracle import vegas as V

from gpu_common import need_gpu, feynman, integrator

pytestmark = pytest.mark.gpu


def test_empty_batch():
    need_gpu()
    integ = integrator("box")
    f = integ.eval_batch(0, np.empty((0, 3)))
    assert f.shape == (0,)


@pytest.mark.parametrize("N", [2, 3, 1023, 4097, 12289])
def test_ragged_point_counts_match_oracle(N):
    """Iteration 0 on the uniform grid with point counts that are not a multiple of a
    work item: mean and variance against the oracle's Vegas on the same Philox points."""
    need_gpu()
    prep, orc = feynman("box")
    integ = integrator("box")
    integ.integrate(n_iter=1, points=N, seed=11, adapt=False)
    for i in (0, 7, len(prep.units) - 1):
        u, o = prep.units[i], orc.units[i]
        m, v = integ.iterations(i, 1)
        r = V.integrate_unit(o.f_numpy, o.dim, 1, N, 11, u.rng_key, adapt=False)
        I, var, sv, sv2 = r.iters[0]
        U = V.philox.uniforms(11, u.rng_key, 0, 0, N, o.dim)
        X, J, _ = V.vegas_map(r.grids[0], U)
        absum = np.sum(np.abs(o.f_numpy(X) * J)) / N
        assert abs(m[0] - I) <= 1e-11 * absum, (N, i, m[0], I)
        # the variance is a difference of two sums; compare at the scale of its terms
        assert abs(v[0] - var) <= 1e-9 * sv2 / N / (N - 1), (N, i, v[0], var)


def test_zero_variance_integrand_is_exact():
    """A constant integrand: every v is the same value on the uniform grid, so the
    iteration's mean is exact and its variance zero; the unit then counts as exact."""
    need_gpu()
    from paper_1511_03614_gb300 import parse_text, Integrator
    integ = Integrator(parse_text("4; 0; 2.5; |"))
    res = integ.integrate(n_iter=1, points=4096, seed=3, adapt=False)
    m, v = integ.iterations(0, 1)
    assert m[0] == 2.5 and v[0] == 0.0
    assert res.values[0] == 2.5 and res.errors[0] == 0.0
    res = integ.integrate(n_iter=3, points=3000, seed=3)
    assert abs(res.values[0] - 2.5) <= 1e-14 and res.errors[0] <= 1e-14
