"""Host logic of the accuracy drivers (no GPU): a stand-in integrator returns, for
every unit result, known true values plus seeded Gaussian noise of a known size, so
the drivers' combination of iterations, replicates and orders can be checked
exactly against the statistics of that noise."""
import math
import types

import numpy as np

import workloads as W
from paper_1511_03614_gb300 import prepare_feynman
from paper_1511_03614_gb300.api import run_to_accuracy, run_to_accuracy_rqmc, _record_key


class FakeIntegrator:
    """integrate() draws per-iteration means m = truth + s / sqrt(N) * z for every
    (unit, result); iterations() hands them back; variances are s^2 / N."""

    def __init__(self, prep, seed=0, spread=1.0):
        self.prep = prep
        self.rng = np.random.default_rng(seed)
        self.truth = {}
        self.spread = {}
        for k, u in enumerate(prep.units):
            for o in range(u.n_out):
                self.truth[(k, o)] = float(k + 1) * (1 if o % 2 == 0 else -0.5)
                self.spread[(k, o)] = spread * (1.0 + 0.1 * k)
        self.last = {}
        self.calls = []

    def integrate(self, n_iter, points, unit_points=None, **kw):
        self.calls.append(dict(n_iter=n_iter, points=points, unit_points=unit_points, **kw))
        self.last = {}
        total = 0
        for k, u in enumerate(self.prep.units):
            N = points if unit_points is None else int(unit_points[k])
            for o in range(u.n_out):
                s = self.spread[(k, o)] / math.sqrt(N)
                m = self.truth[(k, o)] + s * self.rng.standard_normal(n_iter)
                self.last[(k, o)] = (m, np.full(n_iter, s * s))
            total += N * n_iter * u.n_out
        return types.SimpleNamespace(stats=dict(gpu_ms=1.0, unit_points=total))

    def iterations(self, unit, n_iter, out=0):
        m, v = self.last[(unit, out)]
        return m[:n_iter].copy(), v[:n_iter].copy()

    def exact(self):
        """The per-order sums of the true unit values."""
        out = {}
        for k, u in enumerate(self.prep.units):
            for o in range(u.n_out):
                K, part = _record_key(u, o)
                out[K] = out.get(K, 0.0) + self.truth[(k, o)]
        return out


def test_run_to_accuracy_combines_iterations_and_orders():
    """Inverse-variance combination over calls, sums per order, prefactor assembly:
    the result sits within 4 sigma of the assembled truth and sigma matches the
    noise actually injected."""
    prep = prepare_feynman(W.box())
    fake = FakeIntegrator(prep, seed=1)
    r = run_to_accuracy(fake, target=1e-3, points=10_000, iters_per_call=2, max_iters=40)
    from paper_1511_03614_gb300.preprocess import assemble
    R, _ = assemble(prep, fake.exact(), {K: 0.0 for K in fake.exact()})
    for n in R:
        assert abs(r["values"][n] - R[n]) < 4 * r["errors"][n], n
    # the reported unit sigmas are the injected noise over the iterations used
    used = r["iterations"] - 1
    k0 = fake.spread[(0, 0)] / math.sqrt(10_000 * used)
    assert abs(r["unit_sigmas"][0] / k0 - 1) < 1e-9


def test_allocation_moves_points_to_noisy_units():
    """With allocation, the units with the largest injected spread get the most
    points, and the total per iteration stays nu * points (cost-weighted)."""
    prep = prepare_feynman(W.box())
    fake = FakeIntegrator(prep, seed=2)
    fake.spread[(31, 0)] = 50.0                  # one very noisy unit
    run_to_accuracy(fake, target=1e-4, points=10_000, iters_per_call=2, max_iters=6, allocate=True)
    alloc = [c["unit_points"] for c in fake.calls if c["unit_points"] is not None]
    assert alloc, "allocation was never applied"
    N = alloc[-1]
    assert int(np.argmax(N)) == 31


def test_rqmc_replicate_statistics():
    """The RQMC driver's error is the spread of the replicate means over sqrt(R);
    values within 4 sigma of the truth; the sequence length doubles per round."""
    prep = prepare_feynman(W.box(), fuse_orders=True)
    fake = FakeIntegrator(prep, seed=3, spread=0.05)
    r = run_to_accuracy_rqmc(fake, target=1e-6, points=1 << 10, replicates=8, max_points=1 << 14)
    ns = [c["points"] for c in fake.calls[1:]]
    assert ns == [1 << (10 + i) for i in range(len(ns))]
    from paper_1511_03614_gb300.preprocess import assemble
    R, _ = assemble(prep, fake.exact(), {K: 0.0 for K in fake.exact()})
    for n in R:
        assert abs(r["values"][n] - R[n]) < 4 * r["errors"][n], n
