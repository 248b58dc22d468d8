"""GPU parity of the deformed-contour (complex) path: the massless box at the
physical point s = 3, t = -1, where F changes sign inside the cube."""
import functools
import math

import mpmath as mp
import numpy as np
import pytest

import workloads as W
from oracle import pipeline as P

from gpu_common import need_gpu, sample_points

pytestmark = pytest.mark.gpu

TOL = {"fp64": 1e-12, "fp32": 1e-5}


@functools.lru_cache(maxsize=None)
def _prepared(fuse, lam=None):
    from paper_1511_03614_gb300 import prepare_feynman, Integrator
    prep = prepare_feynman(W.box_physical(), fuse_orders=fuse, lam=lam)
    return prep, Integrator(prep)


@functools.lru_cache(maxsize=None)
def _oracle(lam):
    return P.feynman_problem(W.box_physical(), lam=lam)


@functools.lru_cache(maxsize=None)
def _continued_box():
    """Laurent coefficients eps^-2..eps^0 of the one-loop massless box at s = 3, t = -1:
    the Euclidean closed form continued with log(-s - i0) = log s - i pi."""
    s, t = mp.mpf(3), mp.mpf(-1)
    with mp.workdps(30):
        Ls = mp.log(s) - 1j * mp.pi
        Lt = mp.log(-t)

        def g(e):
            cg = mp.exp(mp.euler * e) * mp.gamma(1 + e) * mp.gamma(1 - e) ** 2 / mp.gamma(1 - 2 * e)
            return cg / (s * t) * (2 * (mp.exp(-e * Ls) + mp.exp(-e * Lt)) - e ** 2 * ((Ls - Lt) ** 2 + mp.pi ** 2))
        c = mp.taylor(g, 0, 2, method="quad", radius=0.25)
    return {n: complex(c[n + 2]) for n in (-2, -1, 0)}


@pytest.mark.parametrize("precision", ["fp64", "fp32"])
@pytest.mark.parametrize("fuse", [False, True])
def test_complex_eval_parity(fuse, precision):
    """Per point, real and imaginary parts against a 50-digit evaluation of the
    oracle's deformed integrand, within tol * M(x) (M the condition-scaled magnitude)."""
    need_gpu()
    prep, integ = _prepared(fuse)
    orc = _oracle(prep.lams[0])
    assert all(l == prep.lams[0] for l in prep.lams)
    by = {(u.sector, u.order): u for u in orc.units}
    rng = np.random.default_rng(31)
    for i, u in enumerate(prep.units):
        X = sample_points(u.dim, rng, 40)
        f = integ.eval_batch(i, X, precision)
        f = f[:, None] if f.ndim == 1 else f
        for k in range(u.n_out // 2):
            o = by[(u.sector, u.order + k)]
            with mp.workdps(50):
                ref = np.array([complex(o.f_mp(x, 50)) for x in X])
            M = np.maximum(P.magnitude_numpy(o, X), np.abs(ref))
            err = np.abs(f[:, k] - ref)
            assert np.all(err <= TOL[precision] * np.maximum(M, 1e-300)), (i, k, np.max(err / M))


def test_complex_eval_device_tensor():
    """Device input gives a complex128 device tensor equal to the host-array call."""
    torch = need_gpu()
    prep, integ = _prepared(True)
    X = np.random.default_rng(32).uniform(size=(1000, prep.units[0].dim))
    a = integ.eval_batch(0, X)
    b = integ.eval_batch(0, torch.tensor(X, device="cuda"))
    assert b.is_cuda and b.dtype == torch.complex128 and b.shape == a.shape
    assert np.array_equal(b.cpu().numpy(), a)


@pytest.mark.parametrize("fuse", [False, True])
def test_physical_box_matches_continuation(fuse):
    """Vegas on the deformed contour: every order within 4 sigma of the continued
    closed form, separately in the real and the imaginary part."""
    need_gpu()
    prep, integ = _prepared(fuse)
    res = integ.integrate(n_iter=8, points=500_000, seed=7)
    exact = _continued_box()
    for n, v in exact.items():
        r, e = res.assembled[n], res.assembled_errors[n]
        assert isinstance(r, complex)
        assert abs(r.real - v.real) < 4 * e.real + 1e-6, (n, r, v, e)
        assert abs(r.imag - v.imag) < 4 * e.imag + 1e-6, (n, r, v, e)
        assert abs(e) < 3e-3 * max(abs(v), 1.0), (n, e)
    assert {d["part"] for d in res.per_unit} == {0, 1}


def test_cauchy_invariance_on_gpu():
    """The integral does not depend on the deformation parameter (Cauchy's theorem):
    lam = 1/4 and the automatic choice agree within the combined errors."""
    need_gpu()
    _, a = _prepared(True)
    _, b = _prepared(True, 0.25)
    ra = a.integrate(n_iter=6, points=400_000, seed=3)
    rb = b.integrate(n_iter=6, points=400_000, seed=4)
    for n in ra.assembled:
        d = ra.assembled[n] - rb.assembled[n]
        ea, eb = ra.assembled_errors[n], rb.assembled_errors[n]
        assert abs(d.real) < 4 * math.hypot(ea.real, eb.real) + 1e-6, n
        assert abs(d.imag) < 4 * math.hypot(ea.imag, eb.imag) + 1e-6, n


def test_complex_run_to_accuracy():
    """The accuracy driver combines (re, im) records per order."""
    need_gpu()
    from paper_1511_03614_gb300.api import run_to_accuracy
    _, integ = _prepared(True)
    r = run_to_accuracy(integ, target=1e-3, points=400_000, max_iters=40, seed=11)
    assert r["converged"]
    exact = _continued_box()
    for n, v in exact.items():
        assert abs(r["values"][n] - v) < 5 * abs(r["errors"][n]) + 1e-6, n
