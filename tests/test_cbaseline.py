"""The timed CPU baseline (compiled C++ from the oracle's expression trees) does the
work of the oracle it is generated from: same integrand values, the same Philox
points bit for bit, the same Vegas iteration and refinement."""
import numpy as np
import pytest

import workloads as W
from oracle import pipeline as P, vegas as V, philox

pytestmark = pytest.mark.skipif(__import__("shutil").which("g++") is None, reason="needs g++")


@pytest.fixture(scope="module")
def box_baseline():
    from oracle.cbaseline import Baseline
    orc = P.feynman_problem(W.box())
    return orc, Baseline(orc.units)


def test_values_match_the_oracle(box_baseline):
    orc, b = box_baseline
    rng = np.random.default_rng(3)
    for k, u in enumerate(orc.units):
        X = np.concatenate([rng.uniform(size=(64, u.dim)), np.exp2(-rng.uniform(0, 30, size=(16, u.dim)))])
        f, ref, M = b.eval(k, X), u.f_numpy(X), P.magnitude_numpy(u, X)
        ok = np.isfinite(ref)
        assert np.all(np.abs(f[ok] - ref[ok]) <= 64 * 2.0 ** -53 * M[ok]), k


def test_philox_points_are_the_oracles(box_baseline):
    _, b = box_baseline
    for dim in (1, 3, 6, 8):
        assert np.array_equal(b.uniforms(11, 9, 4, 2 ** 32 - 5, 300, dim), philox.uniforms(11, 9, 4, 2 ** 32 - 5, 300, dim))


def test_vegas_iteration_and_refinement_match_the_oracle(box_baseline):
    orc, b = box_baseline
    N = 8192
    b.grids[:] = np.concatenate([V.uniform_grid(u.dim).ravel() for u in orc.units])
    m, v, bad = b.iterate(N, seed=5, iteration=0)
    assert not bad.any()
    for k in (0, 7, len(orc.units) - 1):
        u = orc.units[k]
        r = V.integrate_unit(u.f_numpy, u.dim, 2, N, 5, k)
        I, var, _, _ = r.iters[0]
        assert abs(m[k] - I) <= 1e-12 * abs(I) and abs(v[k] - var) <= 1e-9 * var
        assert np.allclose(b.histogram(k), r.hists[0], rtol=1e-12, atol=0)
    b.refine()
    for k in (0, 7):
        u = orc.units[k]
        r = V.integrate_unit(u.f_numpy, u.dim, 2, N, 5, k)
        assert np.max(np.abs(b.grid(k) - r.grids[1])) < 1e-12
