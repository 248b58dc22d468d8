"""SeparateTerms (the paper's option of Sec. 4.4: the integrator receives each
integrable term of a sector separately) on the GPU, through the C ABI: per point
against the oracle's terms, and the box from its separate terms against the closed
form."""
import math

import numpy as np
import pytest

import workloads as W
from oracle import pipeline as P, sectors as OS

from gpu_common import need_gpu, feynman, sample_points, reference, Parity

pytestmark = pytest.mark.gpu


def _term_unit(orc, u, k):
    sec = orc.sectors[u.sector]
    var = tuple(j for j in sec.variables if j not in u.term) or (sec.variables[0],)
    return P.Unit(u.sector, u.order + k, var, OS.unit_integrand(sec, u.order + k, term=u.term))


@pytest.mark.parametrize("name,fuse,n_units", [("box", False, None), ("double_box", True, 24)])
def test_separate_terms_points(name, fuse, n_units):
    need_gpu()
    from paper_1511_03614_gb300 import prepare_feynman, Integrator
    prep = prepare_feynman(getattr(W, name)(), fuse_orders=fuse, separate_terms=True)
    _, orc = feynman(name)
    integ = Integrator(prep)
    rng = np.random.default_rng(51)
    idx = range(len(prep.units)) if n_units is None else rng.choice(len(prep.units), n_units, replace=False)
    par = Parity(f"{name}-terms", "fp64")
    for i in idx:
        u = prep.units[int(i)]
        X = sample_points(u.dim, rng, 16, n_log=16, n_edge=8)
        f = integ.eval_batch(int(i), X)
        f = f[:, None] if f.ndim == 1 else f
        for k in range(u.n_out):
            o = _term_unit(orc, u, k)
            par.check(f[:, k], reference(o, X), P.magnitude_numpy(o, X), X, (int(i), k))
    par.finish(0.4)
    integ.close()


@pytest.mark.parametrize("fuse", [False, True])
def test_separate_terms_box_closed_form(fuse):
    """The box from its separately integrated terms (48 units of 1-2 dimensions, or 28
    fused ones): every order within 3 standard errors of the closed form."""
    need_gpu()
    from paper_1511_03614_gb300 import prepare_feynman, Integrator
    prep = prepare_feynman(W.box(), fuse_orders=fuse, separate_terms=True)
    assert max(u.dim for u in prep.units) < 3
    res = Integrator(prep).integrate(n_iter=10, points=500_000, seed=6)
    exact = {-2: 2.0, -1: -math.log(2.0), 0: -2 * math.pi ** 2 / 3}
    for n, v in exact.items():
        s = res.assembled_errors[n]
        assert 0 < s < 2e-3 and abs(res.assembled[n] - v) < 3 * s, (n, res.assembled[n], v, s)
