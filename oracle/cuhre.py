"""Deterministic adaptive cubature (oracle, numpy float64): the Cuhre alternative
to Vegas named among the integrators of Sec. 4.4 (``CurrentIntegrator``).

TEST INFRASTRUCTURE ONLY (see the package header).

The paper does not describe the integrator; this module restates the published
pieces it rests on and fixes the rest:

* the basic rule is Genz and Malik's degree-7 fully symmetric rule for an
  n-cube with its embedded degree-5 rule (A. C. Genz, A. A. Malik, J. Comput.
  Appl. Math. 6 (1980) 295), region error |I7 - I5|;
* a region is split in two halves across the coordinate with the largest
  fourth divided difference along the axis (Genz-Malik's choice of axis), the
  sum over the results of a vector-valued integrand deciding;
* the subdivision runs in passes over all live regions (the order in which a
  parallel implementation can work): in every pass each live region is
  evaluated; a unit whose summed error meets its tolerance stops; in the other
  units a region whose error is within its volume's share of the tolerance is
  frozen (kept with its estimate) and every other region is split.

Tolerance of result o of a unit: tau_o = max(abs_tol, rel_tol * s_o) with s_o the
modulus of the current estimate of result o (of its (re, im) pair for complex
units).  A unit converges when every result's summed error is <= tau_o.

One-dimensional integrands are integrated as two-dimensional ones that do not
depend on the second coordinate (the Genz-Malik rule needs n >= 2).
"""
from __future__ import annotations

import dataclasses
import itertools
import math

import numpy as np

LAM2 = math.sqrt(9.0 / 70.0)
LAM3 = math.sqrt(9.0 / 10.0)
LAM4 = math.sqrt(9.0 / 10.0)
LAM5 = math.sqrt(9.0 / 19.0)


def weights(n):
    """Weights of the degree-7 rule (w1..w5) and of the embedded degree-5 rule
    (v1..v4), normalised to a region of volume 1 (Genz-Malik 1980)."""
    w = (
        (12824.0 - 9120.0 * n + 400.0 * n * n) / 19683.0,
        980.0 / 6561.0,
        (1820.0 - 400.0 * n) / 19683.0,
        200.0 / 19683.0,
        6859.0 / 19683.0 / 2.0 ** n,
    )
    v = (
        (729.0 - 950.0 * n + 50.0 * n * n) / 729.0,
        245.0 / 486.0,
        (265.0 - 100.0 * n) / 1458.0,
        25.0 / 729.0,
    )
    return w, v


def rule_points(n):
    """Generator points of the rule on [-1, 1]^n, grouped: the centre, the 2n points
    +-lam2 e_j, the 2n points +-lam3 e_j, the 2n(n-1) points +-lam4 e_j +-lam4 e_k
    (j < k) and the 2^n points (+-lam5, ..., +-lam5)."""
    c = [np.zeros(n)]
    g2, g3 = [], []
    for j in range(n):
        for s in (1.0, -1.0):
            p = np.zeros(n)
            p[j] = s * LAM2
            g2.append(p)
            p = np.zeros(n)
            p[j] = s * LAM3
            g3.append(p)
    g4 = []
    for j in range(n):
        for k in range(j + 1, n):
            for sj in (1.0, -1.0):
                for sk in (1.0, -1.0):
                    p = np.zeros(n)
                    p[j] = sj * LAM4
                    p[k] = sk * LAM4
                    g4.append(p)
    g5 = [LAM5 * np.array(s) for s in itertools.product((1.0, -1.0), repeat=n)]
    return c, g2, g3, g4, g5


def apply_rule(f, center, half):
    """Genz-Malik rule on the box prod [c_j - h_j, c_j + h_j].

    ``f`` maps (m, n) points to (m,) or (m, k) values.  Returns (I7, I5, err, dif):
    arrays of k results (k = 1 for scalar f), err = |I7 - I5| and dif the
    fourth differences, shape (n, k)."""
    I7, I5, err, dif = apply_rule_batch(f, np.asarray(center)[None], np.asarray(half)[None])
    return I7[0], I5[0], err[0], dif[0]


def apply_rule_batch(f, centers, halves):
    """The rule on R boxes at once (one call of f on all their points): arrays
    I7, I5, err of shape (R, k) and dif of shape (R, n, k)."""
    centers = np.asarray(centers, dtype=np.float64)
    halves = np.asarray(halves, dtype=np.float64)
    R, n = centers.shape
    groups = rule_points(n)
    G = np.concatenate([np.stack(g) for g in groups])          # (P, n)
    P = centers[:, None, :] + G[None, :, :] * halves[:, None, :]
    y = np.asarray(f(P.reshape(-1, n)), dtype=np.float64).reshape(R, G.shape[0], -1)
    vol = np.prod(2.0 * halves, axis=1)[:, None]
    sizes = [len(g) for g in groups]
    edges = np.cumsum([0] + sizes)
    sums = [y[:, edges[i]:edges[i + 1]].sum(axis=1) for i in range(5)]
    w, v = weights(n)
    I7 = vol * (w[0] * sums[0] + w[1] * sums[1] + w[2] * sums[2] + w[3] * sums[3] + w[4] * sums[4])
    I5 = vol * (v[0] * sums[0] + v[1] * sums[1] + v[2] * sums[2] + v[3] * sums[3])
    f0 = y[:, 0]
    y2 = y[:, edges[1]:edges[2]]
    y3 = y[:, edges[2]:edges[3]]
    ratio = (LAM2 / LAM3) ** 2
    dif = np.stack([np.abs(y2[:, 2 * j] + y2[:, 2 * j + 1] - 2.0 * f0
                           - ratio * (y3[:, 2 * j] + y3[:, 2 * j + 1] - 2.0 * f0)) for j in range(n)], axis=1)
    return I7, I5, np.abs(I7 - I5), dif


def split_axis(dif, half):
    """Largest sum over results of the fourth difference; ties go to the wider side,
    then to the lower coordinate."""
    score = dif.sum(axis=1)
    best = 0
    for j in range(1, len(score)):
        if score[j] > score[best] or (score[j] == score[best] and half[j] > half[best]):
            best = j
    return best


@dataclasses.dataclass
class Region:
    center: np.ndarray
    half: np.ndarray
    value: np.ndarray = None
    error: np.ndarray = None
    axis: int = 0


@dataclasses.dataclass
class CuhreResult:
    value: np.ndarray          # per result
    error: np.ndarray
    converged: bool
    passes: int
    n_regions: int             # leaves (frozen + live) at the end
    n_evals: int
    live: list                 # live regions at the end (evaluated, not split)


def tolerances(value, rel_tol, abs_tol, pairs=False):
    """tau_o = max(abs_tol, rel_tol * s_o), s_o = |value_o| or the modulus of its pair."""
    s = np.abs(value)
    if pairs:
        m = np.hypot(value[0::2], value[1::2])
        s = np.repeat(m, 2)
    return np.maximum(abs_tol, rel_tol * s)


def cuhre(f, dim, rel_tol=1e-6, abs_tol=1e-14, max_passes=40, max_regions=1 << 20, pairs=False):
    """Adaptive cubature of f over the unit cube [0, 1]^dim by the passes described
    in the module header.  Returns a CuhreResult."""
    n = max(dim, 2)
    g = f if dim >= 2 else (lambda X: f(X[:, :1]))
    npts = 1 + 4 * n + 2 * n * (n - 1) + 2 ** n
    live = [Region(np.full(n, 0.5), np.full(n, 0.5))]
    frozen_v = None
    frozen_e = None
    n_frozen = 0
    evals = 0
    passes = 0
    converged = False
    while live:
        I7, _, err, dif = apply_rule_batch(g, np.stack([r.center for r in live]), np.stack([r.half for r in live]))
        for i, r in enumerate(live):
            r.value, r.error, r.axis = I7[i], err[i], split_axis(dif[i], r.half)
        evals += npts * len(live)
        passes += 1
        k = live[0].value.size
        if frozen_v is None:
            frozen_v, frozen_e = np.zeros(k), np.zeros(k)
        tot_v = frozen_v + sum(r.value for r in live)
        tot_e = frozen_e + sum(r.error for r in live)
        tau = tolerances(tot_v, rel_tol, abs_tol, pairs)
        if np.all(tot_e <= tau):
            converged = True
            break
        if passes >= max_passes:
            break
        keep, split = [], []
        for r in live:
            share = tau * float(np.prod(2.0 * r.half))
            (keep if np.all(r.error <= share) else split).append(r)
        if n_frozen + len(keep) + 2 * len(split) > max_regions:
            break
        for r in keep:
            frozen_v = frozen_v + r.value
            frozen_e = frozen_e + r.error
        n_frozen += len(keep)
        nxt = []
        for r in split:
            a = r.axis
            h = r.half.copy()
            h[a] *= 0.5
            lo = r.center.copy()
            lo[a] -= h[a]
            hi = r.center.copy()
            hi[a] += h[a]
            nxt += [Region(lo, h.copy()), Region(hi, h.copy())]
        live = nxt
        if not live:          # every region frozen although the sum misses tau (tau shrank)
            tot_v, tot_e = frozen_v, frozen_e
    return CuhreResult(tot_v, tot_e, converged, passes, n_frozen + len(live), evals, live)

