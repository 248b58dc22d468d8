"""VEGAS adaptive Monte Carlo (oracle, numpy float64).

The paper's default integrator is Cuba's Vegas (Sec. 4.4, ``CurrentIntegrator``)
whose internals it does not describe; this is G. P. Lepage's published algorithm
(J. Comput. Phys. 27 (1978) 192) with the constants this project fixes:

* a separable grid of NB bins per coordinate, edges 0 = g_0 < ... < g_NB = 1;
* map of a uniform u: y = u NB, i = floor(y), x = g_i + (y - i)(g_{i+1} - g_i),
  Jacobian factor NB (g_{i+1} - g_i) per coordinate;
* per iteration with N points: I = sum(v)/N, var = (sum(v^2)/N - I^2)/(N-1),
  v = f(x) J;
* histogram: d_i = sum of v^2 over the points whose coordinate falls in bin i;
* refinement: 3-point smoothing (2-point at the two end bins), normalisation,
  damping w_i = ((1 - r_i)/ln(1/r_i))^alpha (w = 0 for r = 0, w = 1 for r = 1),
  then new edges that split sum(w) into NB equal parts by linear interpolation
  inside the old bins;
* iterations combined with inverse-variance weights, chi^2/dof reported.
"""
from __future__ import annotations

import dataclasses
import math

import numpy as np

from . import philox, sobol

NB_DEFAULT = 128
ALPHA_DEFAULT = 1.5


def uniform_grid(dim, nb=NB_DEFAULT):
    return np.tile(np.linspace(0.0, 1.0, nb + 1), (dim, 1))


def vegas_map(grid, U):
    """Map uniforms U (n, dim) through the grid; returns x, J, bin indices."""
    dim, nb1 = grid.shape
    nb = nb1 - 1
    y = U * nb
    i = np.minimum(np.floor(y).astype(np.int64), nb - 1)
    X = np.empty_like(U)
    J = np.ones(U.shape[0])
    for j in range(dim):
        g0 = grid[j, i[:, j]]
        dlt = grid[j, i[:, j] + 1] - g0
        X[:, j] = g0 + (y[:, j] - i[:, j]) * dlt
        J *= nb * dlt
    return X, J, i


def refine(grid, hist, alpha=ALPHA_DEFAULT):
    """One Lepage refinement of every coordinate's edges from the v^2 histogram."""
    dim, nb1 = grid.shape
    nb = nb1 - 1
    out = grid.copy()
    for j in range(dim):
        d = hist[j]
        s = np.empty(nb)
        s[0] = (d[0] + d[1]) / 2.0
        s[-1] = (d[-2] + d[-1]) / 2.0
        s[1:-1] = (d[:-2] + d[1:-1] + d[2:]) / 3.0
        tot = s.sum()
        if not (tot > 0.0) or not math.isfinite(tot):
            continue
        r = s / tot
        w = np.zeros(nb)
        for i in range(nb):
            if r[i] <= 0.0:
                w[i] = 0.0
            elif r[i] >= 1.0:
                w[i] = 1.0
            else:
                w[i] = ((1.0 - r[i]) / math.log(1.0 / r[i])) ** alpha
        W = 0.0
        for i in range(nb):
            W += w[i]
        delta = W / nb
        g = grid[j]
        i = 0
        acc = w[0]
        for k in range(1, nb):
            target = k * delta
            while acc < target and i < nb - 1:
                i += 1
                acc += w[i]
            if w[i] > 0.0:
                out[j, k] = g[i] + (target - (acc - w[i])) / w[i] * (g[i + 1] - g[i])
            else:
                out[j, k] = g[i + 1]
        out[j, 0] = 0.0
        out[j, nb] = 1.0
    return out


@dataclasses.dataclass
class UnitResult:
    value: float
    sigma: float
    chi2_dof: float
    iters: list            # [(I, var, sum_v, sum_v2)]
    grids: list            # grid used in each iteration
    hists: list


def combine_iterations(iters, skip_first=False):
    its = iters[1:] if (skip_first and len(iters) > 1) else iters
    zero = [I for I, var, *_ in its if var <= 0.0]
    if zero:
        return float(np.mean(zero)), 0.0, 0.0
    w = np.array([1.0 / var for _, var, *_ in its])
    I = np.array([I for I, *_ in its])
    val = float((w * I).sum() / w.sum())
    sig = float(math.sqrt(1.0 / w.sum()))
    chi2 = float(((I - val) ** 2 * w).sum() / (len(its) - 1)) if len(its) > 1 else 0.0
    return val, sig, chi2


def integrate_unit(f, dim, n_iter, n_points, seed, unit_key, rng="philox",
                   nb=NB_DEFAULT, alpha=ALPHA_DEFAULT, chunk=1 << 18, adapt=True,
                   grid=None, skip_first=False):
    """Plain Vegas on one unit with the project's point streams.

    ``f`` maps an (n, dim) array to n float64 values.  Returns a UnitResult.
    """
    gen = philox.uniforms if rng == "philox" else sobol.uniforms
    grid = uniform_grid(dim, nb) if grid is None else grid.copy()
    iters, grids, hists = [], [], []
    for it in range(n_iter):
        sv = 0.0
        sv2 = 0.0
        hist = np.zeros((dim, nb))
        for first in range(0, n_points, chunk):
            cnt = min(chunk, n_points - first)
            U = gen(seed, unit_key, it, first, cnt, dim)
            X, J, bins = vegas_map(grid, U)
            v = f(X) * J
            sv += float(np.sum(v))
            sv2 += float(np.sum(v * v))
            for j in range(dim):
                np.add.at(hist[j], bins[:, j], v * v)
        I = sv / n_points
        var = max((sv2 / n_points - I * I) / (n_points - 1), 0.0) if n_points > 1 else 0.0
        iters.append((I, var, sv, sv2))
        grids.append(grid.copy())
        hists.append(hist)
        if adapt and it + 1 < n_iter:
            grid = refine(grid, hist, alpha)
    val, sig, chi2 = combine_iterations(iters, skip_first)
    return UnitResult(val, sig, chi2, iters, grids, hists)
