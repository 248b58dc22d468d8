"""GPU tests of the double-double path (the extended precision used near the
boundary of the cube): arithmetic pins on cancelling expressions, sector
integrands at boundary points against 50-digit values, and the mixed
integration mode."""
import math

import mpmath as mp
import numpy as np
import pytest

import workloads as W
from oracle import pipeline as P

from gpu_common import need_gpu, feynman, integrator

pytestmark = pytest.mark.gpu

# expressions whose binary64 evaluation cancels for small x[1], with their exact
# values as functions of (x1, x2) evaluated in mpmath
CASES = [
    ("(l[1+x[1]]-x[1]+x[1]*x[1]/2-x[1]*x[1]*x[1]/3)/(x[1]*x[1]*x[1]*x[1])",
     lambda a, b: (mp.log(1 + a) - a + a ** 2 / 2 - a ** 3 / 3) / a ** 4),
    ("(1/(1+x[1])-1+x[1])/(x[1]*x[1])", lambda a, b: (1 / (1 + a) - 1 + a) / a ** 2),
    ("(p[1+x[1],5]-1-5*x[1])/(x[1]*x[1])", lambda a, b: ((1 + a) ** 5 - 1 - 5 * a) / a ** 2),
    ("(p[1+x[1],-3]-1+3*x[1])/(x[1]*x[1])", lambda a, b: ((1 + a) ** -3 - 1 + 3 * a) / a ** 2),
    ("(l[x[2]+x[1]]-l[x[2]])/x[1]", lambda a, b: (mp.log(b + a) - mp.log(b)) / a),
    ("l[x[1]]*x[2]", lambda a, b: mp.log(a) * b),
]


def _exact(fn, X):
    with mp.workdps(60):
        return np.array([float(fn(mp.mpf(float(a)), mp.mpf(float(b)))) for a, b in X])


def test_dd_arithmetic_on_cancelling_expressions():
    """Every case to 1e-13 relative for x[1] in (1e-5, 0.1), where binary64 loses up
    to all digits on the first cases (their cancellation amplifies the rounding
    error by up to 1/x^3); logarithms over most of the binary64 range."""
    need_gpu()
    from paper_1511_03614_gb300 import parse_text, Integrator
    rng = np.random.default_rng(41)
    X = np.stack([10.0 ** rng.uniform(-5, -1, 200), rng.uniform(0.05, 1.0, 200)], axis=1)
    worst64 = 0.0
    for text, fn in CASES:
        integ = Integrator(parse_text(f"2;\n0;\n{text};\n|"))
        ref = _exact(fn, X)
        f = integ.eval_batch(0, X, "dd")
        rel = np.abs(f - ref) / np.abs(ref)
        assert rel.max() < 1e-13, (text, rel.max())
        f64 = integ.eval_batch(0, X, "fp64")
        worst64 = max(worst64, float(np.max(np.abs(f64 - ref) / np.abs(ref))))
        integ.close()
    assert worst64 > 1e-3            # the cases do defeat binary64
    # log from subnormal to huge arguments: (log(x) - log(x(1+2^-40)))*2^40 = -1 + 2^-41 - ...
    integ = Integrator(parse_text("2;\n0;\n(l[x[1]*x[2]]-l[x[1]*x[2]*(1+1/1099511627776)])*1099511627776;\n|"))
    Y = np.stack([10.0 ** rng.uniform(-280, 0, 100), 10.0 ** rng.uniform(-20, 0, 100)], axis=1)
    f = integ.eval_batch(0, Y, "dd")
    with mp.workdps(60):
        e = float(-mp.log(1 + mp.mpf(2) ** -40) * mp.mpf(2) ** 40)
    assert np.max(np.abs(f - e)) < 1e-12 * abs(e)
    integ.close()


@pytest.mark.parametrize("name", ["box", "double_box"])
def test_dd_sector_units_at_the_boundary(name):
    """Sector integrands at points with one coordinate in (1e-14, 1e-6): double-double
    matches a 50-digit evaluation of the oracle's expression to 1e-13 relative at
    every point, where binary64 is off by more than 1e-4 (up to tens of per cent on
    the double box: the subtraction terms cancel)."""
    need_gpu()
    prep, orc = feynman(name)
    from paper_1511_03614_gb300 import Integrator
    integ = Integrator(prep)
    rng = np.random.default_rng(42)
    idx = range(len(prep.units)) if len(prep.units) < 40 else rng.choice(len(prep.units), 16, replace=False)
    worst_dd, worst_64 = 0.0, 0.0
    for i in idx:
        u, o = prep.units[i], orc.units[i]
        X = rng.uniform(0.1, 0.9, size=(16, u.dim))
        for k in range(16):
            X[k, rng.integers(u.dim)] = 10.0 ** rng.uniform(-14, -6)
        with mp.workdps(50):
            ref = np.array([float(o.f_mp(x, 50)) for x in X])
        ok = ref != 0
        fdd = integ.eval_batch(i, X, "dd")
        f64 = integ.eval_batch(i, X, "fp64")
        rd = np.abs(fdd[ok] - ref[ok]) / np.abs(ref[ok])
        r6 = np.abs(f64[ok] - ref[ok]) / np.abs(ref[ok])
        worst_dd = max(worst_dd, float(rd.max(initial=0)))
        worst_64 = max(worst_64, float(r6.max(initial=0)))
        assert np.all(np.abs(fdd[~ok]) < 1e-25)
    assert worst_dd < 1e-13, worst_dd
    assert worst_64 > 1e-4          # binary64 at the same points


def test_mixed_integration():
    """small_x: points near the boundary in double-double, the rest in binary64; the
    same point streams give the binary64 result within its error, the closed form of
    the box within 4 sigma, and a nonzero count of double-double points."""
    need_gpu()
    integ = integrator("box")
    r64 = integ.integrate(n_iter=5, points=200_000, seed=3)
    rmx = integ.integrate(n_iter=5, points=200_000, seed=3, small_x=1e-4)
    assert rmx.stats["points_ext"] > 0 and r64.stats["points_ext"] == 0
    exact = {-2: 2.0, -1: -math.log(2.0), 0: -2 * math.pi ** 2 / 3}
    for n, v in exact.items():
        assert abs(rmx.assembled[n] - r64.assembled[n]) < 0.1 * rmx.assembled_errors[n] + 1e-12
        assert abs(rmx.assembled[n] - v) < 4 * rmx.assembled_errors[n]


def test_dd_rejects_complex_units():
    need_gpu()
    from paper_1511_03614_gb300 import prepare_feynman, Integrator
    from paper_1511_03614_gb300._native import FiestaError
    integ = Integrator(prepare_feynman(W.box_physical()))
    with pytest.raises(FiestaError):
        integ.eval_batch(0, np.full((4, integ.prep.units[0].dim), 0.5), "dd")
    with pytest.raises(FiestaError):
        integ.integrate(n_iter=1, points=1000, small_x=1e-6)


def test_fp32_with_binary64_near_the_boundary():
    """small_x32 with the binary32 body: points near the boundary run in binary64 (the
    subtraction differences there stay binary64); results within errors of binary64,
    the promoted points counted; on the double box the AUTO probe then accepts more
    units for binary32 than without promotion."""
    need_gpu()
    integ = integrator("box")
    r64 = integ.integrate(n_iter=5, points=200_000, seed=3)
    r32 = integ.integrate(n_iter=5, points=200_000, seed=3, precision="fp32", small_x32=1e-3)
    assert r32.stats["points_ext"] > 0
    for n in r64.assembled:
        s = math.hypot(r64.assembled_errors[n], r32.assembled_errors[n])
        assert abs(r64.assembled[n] - r32.assembled[n]) < 3 * s + 1e-6
    from paper_1511_03614_gb300 import Integrator
    prep, _ = feynman("double_box")
    integ = Integrator(prep)
    integ.integrate(n_iter=3, points=20000, seed=1)        # adapt the grids
    a = integ.integrate(n_iter=1, points=20000, seed=2, precision="auto", reset_grid=False, adapt=False)
    b = integ.integrate(n_iter=1, points=20000, seed=2, precision="auto", reset_grid=False, adapt=False,
                        small_x32=1e-2)
    assert b.stats["units_fp32"] > a.stats["units_fp32"], (a.stats["units_fp32"], b.stats["units_fp32"])
