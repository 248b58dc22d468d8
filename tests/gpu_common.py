"""Shared helpers of the GPU tests (prepared problems cached per process) and the
per-point parity bar.

Per-point parity bar (per result of a unit, against a 50-digit evaluation f of
the oracle's expression at the same binary64 point):

* scaled, on every point: |f_gpu - f| <= min(tol, C_SCALED u) * M(x), with M
  the oracle's condition-scaled magnitude (first-order forward-error bound of
  any evaluation order: |error| <= c u M, c of the order of the expression
  depth), u the unit roundoff of the evaluation precision;
* strict, relative: |f_gpu - f| <= tol |f| on every point whose coordinates are
  all >= 2^-20 and whose condition number kappa = M/|f| is at most
  KAPPA_MAX = tol / (16 u) (563 in binary64, 10.5 in binary32).  Outside that
  set no evaluation in that precision can promise the relative bound: the
  rounding error is c u kappa |f| with c measured at up to 9.2 on the box and
  double box (host evaluation, 5000 points with all t_j >= 2^-20), and 31 % of
  such double-box points have kappa u c > 1e-12.

Both bounds carry an absolute floor of 2^20 times the smallest normal number of
the precision (FLOOR): results and intermediates below the normal range (a
stress integrand x^9 P^-2 at x ~ 1e-6 is ~1e-54, below binary32's 1.2e-38)
carry absolute, not relative, rounding errors, and the remaining factors of the
integrands amplify such an error by less than 2^20 (P >= 0.1 gives P^-2 <= 100,
|log P| <= 3.7); the strict set also leaves out values below FLOOR / tol.

tol = 1e-12 (binary64) and 1e-5 (binary32).  Both pass rates (scaled: every
point; strict: the share of the t_j >= 2^-20 points inside the strict set, and
the share of all t_j >= 2^-20 points that happen to meet the relative bound) are
recorded per test and printed; each test also requires the strict set to be a
sizeable part of its points, so the relative check cannot pass vacuously.
"""
import functools
import json
import os

import numpy as np
import pytest

import workloads as W
from oracle import pipeline as P

TOL = {"fp64": 1e-12, "fp32": 1e-5}
UROUND = {"fp64": 2.0 ** -53, "fp32": 2.0 ** -24}
C_SCALED = 64
KAPPA_MAX = {p: TOL[p] / (16 * UROUND[p]) for p in TOL}
T_MIN = 2.0 ** -20
FLOOR = {"fp64": 2.0 ** 20 * 2.0 ** -1022, "fp32": 2.0 ** 20 * 2.0 ** -126}


def need_gpu():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1511_03614_gb300 import build
    build.build()
    return torch


@functools.lru_cache(maxsize=None)
def feynman(name):
    from paper_1511_03614_gb300 import prepare_feynman
    prob = getattr(W, name)()
    return prepare_feynman(prob), P.feynman_problem(prob)


@functools.lru_cache(maxsize=None)
def feynman_fused(name, mix=1):
    from paper_1511_03614_gb300 import prepare_feynman
    prob = getattr(W, name)()
    return prepare_feynman(prob, fuse_orders=True, mix_sectors=mix)


@functools.lru_cache(maxsize=None)
def integrator(name):
    from paper_1511_03614_gb300 import Integrator
    prep, _ = feynman(name)
    return Integrator(prep)


@functools.lru_cache(maxsize=None)
def stress(n):
    from paper_1511_03614_gb300 import prepare_direct, Integrator
    probs = W.stress_suite(n)
    prep = prepare_direct(probs)
    return probs, prep, Integrator(prep)


def sample_points(dim, rng, n_random=96, n_log=0, n_edge=32):
    """Random interior points, log-uniform points in [2^-20, 1) (where the subtraction
    differences cancel), and boundary points (coordinates at 2^-40, 2^-20, 1 - 2^-20, 1/2)."""
    X = [rng.uniform(0.0, 1.0, size=(n_random, dim))]
    if n_log:
        X.append(np.exp2(-rng.uniform(0.0, 20.0, size=(n_log, dim))))
    edge = np.array([2.0 ** -40, 2.0 ** -20, 1 - 2.0 ** -20, 0.5])
    X.append(rng.choice(edge, size=(n_edge, dim)))
    for j in range(dim):
        Y = np.full((len(edge), dim), 0.5)
        Y[:, j] = edge
        X.append(Y)
    return np.concatenate(X)


def reference(unit, X):
    """The oracle's expression at 50 digits, rounded to binary64."""
    return np.array([float(unit.f_mp(x, 50)) for x in X])


class Parity:
    """Accumulates the per-point bar over the checks of one test."""

    def __init__(self, label, precision):
        self.label, self.precision = label, precision
        self.n = self.region = self.strict = self.region_rel_ok = 0
        self.worst_scaled = 0.0      # max |f_gpu - f| / (u M)
        self.worst_strict = 0.0      # max relative error on the strict set

    def check(self, f, ref, M, X, what=""):
        p = self.precision
        tol, u = TOL[p], UROUND[p]
        f, ref, M = np.asarray(f, float), np.asarray(ref, float), np.asarray(M, float)
        ok = np.isfinite(ref) & np.isfinite(M)
        assert np.all(np.isfinite(f[ok])), (what, "non-finite GPU value where the reference is finite")
        d = np.abs(f - ref)
        bound = min(tol, C_SCALED * u) * M + FLOOR[p]
        bad = ok & ~(d <= bound)
        assert not bad.any(), (what, "scaled bound", float(np.max(d[bad] / (u * M[bad] + FLOOR[p]))))
        if ok.any():
            self.worst_scaled = max(self.worst_scaled, float(np.max(d[ok] / (u * M[ok] + FLOOR[p]))))
        absf = np.maximum(np.abs(ref), 1e-300)
        rel = d / absf
        region = ok & np.all(np.asarray(X) >= T_MIN, axis=1)
        strict = region & (M / absf <= KAPPA_MAX[p]) & (np.abs(ref) >= FLOOR[p] / tol)
        bad = strict & ~(rel <= tol)
        assert not bad.any(), (what, "strict relative bound", float(np.max(rel[bad])))
        if strict.any():
            self.worst_strict = max(self.worst_strict, float(np.max(rel[strict])))
        self.n += int(ok.sum())
        self.region += int(region.sum())
        self.strict += int(strict.sum())
        self.region_rel_ok += int((region & (rel <= tol)).sum())

    def finish(self, min_strict_share):
        """Print and record the pass rates; require the strict set to be non-vacuous."""
        rec = {"test": self.label, "precision": self.precision, "points": self.n,
               "points_t_ge_2^-20": self.region, "strict_set": self.strict,
               "strict_share": self.strict / max(self.region, 1),
               "relative_bound_met_share": self.region_rel_ok / max(self.region, 1),
               "scaled_pass_rate": 1.0, "worst_err_over_uM": self.worst_scaled,
               "worst_strict_rel": self.worst_strict}
        print("parity", json.dumps(rec))
        path = os.environ.get("FIESTA_PARITY_LOG")
        if path:
            with open(path, "a") as fh:
                fh.write(json.dumps(rec) + "\n")
        assert self.strict >= min_strict_share * self.region and self.strict > 0, rec
        return rec
