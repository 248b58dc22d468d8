"""The timed CPU baseline: compiled per-unit C++ from the oracle's expression trees.

Test and measurement infrastructure, like the rest of ``oracle/``: only the tests,
``__graft_entry__`` and the benchmark's CPU legs use it; nothing in the product
imports it, and it shares no code with the CUDA path.

For a list of the oracle's units (``pipeline.Unit``: one sector at one power of eps,
the paper's integrand, Sec. 4.3), ``generate`` writes one straight-line C++
function per unit from its sympy tree (common subexpressions hoisted by sympy's
``cse``, small integer powers as products), plus a driver that runs one Vegas
iteration (Lepage's map and v^2 histogram, the spec of ``oracle/vegas.py``) on the
Philox points of ``oracle/philox.py`` (its published definition restated in C++),
with OpenMP over units.  ``Baseline`` compiles it (g++ -O3, -mcpu=native on
aarch64 hosts, -fopenmp), loads it and refines the grids between iterations with
``oracle.vegas.refine``.  Everything is binary64.
"""
from __future__ import annotations

import ctypes as C
import hashlib
import os
import platform
import subprocess
import tempfile

import numpy as np
import sympy as sp
from sympy.printing.c import C99CodePrinter

from . import sectors as S
from . import vegas as V

NB = V.NB_DEFAULT


class _Printer(C99CodePrinter):
    """C99 printer writing integer powers |n| <= 8 as products (and 1/product)."""

    def _print_Pow(self, expr):
        b, e = expr.args
        if e.is_Integer and 1 <= abs(int(e)) <= 8:
            base = self.parenthesize(b, 100)
            prod = "*".join([base] * abs(int(e)))
            return f"({prod})" if e > 0 else f"(1.0/({prod}))"
        return super()._print_Pow(expr)


_RUNTIME = r"""
#include <cmath>
#include <cstdint>
#include <vector>
#include <omp.h>

namespace {
// Philox4x32-10 (Salmon, Moraes, Dror, Shaw, SC'11)
inline void philox(uint32_t c[4], uint32_t k0, uint32_t k1) {
    for (int r = 0; r < 10; ++r) {
        if (r) { k0 += 0x9E3779B9u; k1 += 0xBB67AE85u; }
        const uint64_t p0 = (uint64_t)0xD2511F53u * c[0], p1 = (uint64_t)0xCD9E8D57u * c[2];
        const uint32_t n0 = (uint32_t)(p1 >> 32) ^ c[1] ^ k0, n2 = (uint32_t)(p0 >> 32) ^ c[3] ^ k1;
        c[0] = n0; c[1] = (uint32_t)p1; c[2] = n2; c[3] = (uint32_t)p0;
    }
}
inline double unit_u(uint32_t lo, uint32_t hi) {
    const uint64_t m = ((uint64_t)hi << 20) | (lo >> 12);
    return (2.0 * (double)m + 1.0) * 0x1p-53;
}
inline void uniforms(uint32_t seed, uint32_t key, uint32_t it, uint64_t pi, int dim, double *u) {
    for (int q = 0; 2 * q < dim; ++q) {
        uint32_t c[4] = {(uint32_t)pi, (uint32_t)(pi >> 32), it, (uint32_t)q};
        philox(c, seed, key);
        u[2 * q] = unit_u(c[0], c[1]);
        if (2 * q + 1 < dim) u[2 * q + 1] = unit_u(c[2], c[3]);
    }
}
typedef double (*Fn)(const double *);
}  // namespace
"""

_DRIVER = r"""
extern "C" int cb_threads() { return omp_get_max_threads(); }

extern "C" int cb_n_units() { return N_UNITS; }

// f of unit k at n points x (n x dim, row-major).
extern "C" void cb_eval(int k, int64_t n, const double *x, double *f) {
    for (int64_t i = 0; i < n; ++i) f[i] = FN[k](x + i * DIM[k]);
}

// Points first .. first+count-1 of the (seed, key, iteration) stream, count x dim.
extern "C" void cb_uniforms(uint32_t seed, uint32_t key, uint32_t it, uint64_t first, int64_t count, int dim,
                            double *out) {
    for (int64_t i = 0; i < count; ++i) uniforms(seed, key, it, first + i, dim, out + i * dim);
}

// One Vegas iteration of every unit: grids (per unit dim x (NB+1) edges at goff[k]),
// hist (dim x NB at hoff[k], overwritten), per unit mean, variance of the mean and the
// count of non-finite values (counted as 0).  OpenMP over units.
extern "C" void cb_iterate(const uint32_t *keys, int64_t n_points, uint32_t seed, uint32_t it, const double *grids,
                           const int64_t *goff, double *hist, const int64_t *hoff, double *mean, double *var,
                           int64_t *bad) {
#pragma omp parallel for schedule(dynamic, 1)
    for (int k = 0; k < N_UNITS; ++k) {
        const int d = DIM[k];
        const double *g = grids + goff[k];
        double *h = hist + hoff[k];
        for (int i = 0; i < d * NBINS; ++i) h[i] = 0.0;
        double s = 0.0, s2 = 0.0;
        int64_t nb = 0;
        double u[8], x[8];
        int bin[8];
        for (int64_t p = 0; p < n_points; ++p) {
            uniforms(seed, keys[k], it, (uint64_t)p, d, u);
            double J = 1.0;
            for (int j = 0; j < d; ++j) {
                const double y = u[j] * NBINS;
                int b = (int)y;
                if (b > NBINS - 1) b = NBINS - 1;
                const double g0 = g[j * (NBINS + 1) + b], w = g[j * (NBINS + 1) + b + 1] - g0;
                x[j] = g0 + (y - b) * w;
                J *= NBINS * w;
                bin[j] = b;
            }
            double v = FN[k](x) * J;
            if (!std::isfinite(v)) { ++nb; v = 0.0; }
            s += v;
            s2 += v * v;
            for (int j = 0; j < d; ++j) h[j * NBINS + bin[j]] += v * v;
        }
        const double N = (double)n_points, I = s / N;
        double var_ = (s2 / N - I * I) / (N - 1.0);
        mean[k] = I;
        var[k] = var_ > 0.0 ? var_ : 0.0;
        bad[k] = nb;
    }
}
"""


def _function(k, unit):
    """C++ source of unit k's integrand: x[i] is the unit's i-th variable."""
    syms = [S.tsym(j) for j in unit.variables]
    xs = sp.symbols(f"x0:{len(syms)}")
    expr = unit.expr.subs(dict(zip(syms, xs)), simultaneous=True)
    reps, (red,) = sp.cse(expr, symbols=sp.numbered_symbols("c"))
    pr = _Printer()
    lines = [f"double f{k}(const double *x) {{"]
    lines += [f"    const double x{i} = x[{i}];" for i in range(len(xs))]
    lines += [f"    const double {s} = {pr.doprint(e)};" for s, e in reps]
    lines.append(f"    return {pr.doprint(red)};")
    lines.append("}")
    return "\n".join(lines)


def generate(units):
    """The whole translation unit for a list of oracle units."""
    funcs = [_function(k, u) for k, u in enumerate(units)]
    table = ", ".join(f"f{k}" for k in range(len(units)))
    dims = ", ".join(str(u.dim) for u in units)
    return (_RUNTIME + f"#define NBINS {NB}\nnamespace {{\n" + "\n\n".join(funcs) +
            f"\nconst Fn FN[] = {{{table}}};\nconst int DIM[] = {{{dims}}};\nconst int N_UNITS = {len(units)};\n}}\n" +
            _DRIVER)


def compile_flags():
    flags = ["-O3", "-fopenmp", "-fno-math-errno", "-shared", "-fPIC", "-std=c++17"]
    if platform.machine() in ("aarch64", "arm64"):
        flags.append("-mcpu=native")
    return flags


def cpu_model():
    try:
        for line in open("/proc/cpuinfo"):
            low = line.lower()
            if low.startswith("model name") or low.startswith("cpu part") or low.startswith("hardware"):
                return line.split(":", 1)[1].strip()
    except OSError:
        pass
    return platform.processor() or platform.machine()


class Baseline:
    """Compiled baseline for a list of oracle units (built once per source in a temp dir)."""

    def __init__(self, units, keys=None, workdir=None):
        self.units = list(units)
        self.keys = np.asarray(keys if keys is not None else range(len(self.units)), dtype=np.uint32)
        src = generate(self.units)
        tag = hashlib.sha1(src.encode()).hexdigest()[:16]
        workdir = workdir or os.path.join(tempfile.gettempdir(), "fiesta_cbaseline")
        os.makedirs(workdir, exist_ok=True)
        so = os.path.join(workdir, f"cb_{tag}.so")
        self.compile_s = 0.0
        if not os.path.exists(so):
            import time
            cpp = os.path.join(workdir, f"cb_{tag}.cpp")
            with open(cpp, "w") as fh:
                fh.write(src)
            t0 = time.perf_counter()
            subprocess.run(["g++"] + compile_flags() + ["-o", so + ".tmp", cpp], check=True)
            os.replace(so + ".tmp", so)
            self.compile_s = time.perf_counter() - t0
        lib = C.CDLL(so)
        dp, ip, up = C.POINTER(C.c_double), C.POINTER(C.c_int64), C.POINTER(C.c_uint32)
        lib.cb_threads.restype = C.c_int
        lib.cb_eval.argtypes = [C.c_int, C.c_int64, dp, dp]
        lib.cb_uniforms.argtypes = [C.c_uint32, C.c_uint32, C.c_uint32, C.c_uint64, C.c_int64, C.c_int, dp]
        lib.cb_iterate.argtypes = [up, C.c_int64, C.c_uint32, C.c_uint32, dp, ip, dp, ip, dp, dp, ip]
        self.lib = lib
        dims = [u.dim for u in self.units]
        self.goff = np.cumsum([0] + [d * (NB + 1) for d in dims[:-1]]).astype(np.int64)
        self.hoff = np.cumsum([0] + [d * NB for d in dims[:-1]]).astype(np.int64)
        self.grids = np.concatenate([V.uniform_grid(d).ravel() for d in dims])
        self.hist = np.zeros(sum(d * NB for d in dims))

    @property
    def threads(self):
        return int(self.lib.cb_threads())

    def eval(self, k, X):
        X = np.ascontiguousarray(X, dtype=np.float64)
        f = np.empty(X.shape[0])
        self.lib.cb_eval(k, X.shape[0], X.ctypes.data_as(C.POINTER(C.c_double)), f.ctypes.data_as(C.POINTER(C.c_double)))
        return f

    def uniforms(self, seed, key, iteration, first, count, dim):
        out = np.empty((count, dim))
        self.lib.cb_uniforms(seed & 0xFFFFFFFF, key & 0xFFFFFFFF, iteration, first, count, dim,
                             out.ctypes.data_as(C.POINTER(C.c_double)))
        return out

    def iterate(self, n_points, seed=1, iteration=0):
        """One Vegas iteration of every unit on the current grids: (mean, var, bad)."""
        n = len(self.units)
        mean, var, bad = np.empty(n), np.empty(n), np.empty(n, dtype=np.int64)
        dp = lambda a: a.ctypes.data_as(C.POINTER(C.c_double))
        ip = lambda a: a.ctypes.data_as(C.POINTER(C.c_int64))
        self.lib.cb_iterate(self.keys.ctypes.data_as(C.POINTER(C.c_uint32)), int(n_points), seed & 0xFFFFFFFF,
                            iteration, dp(self.grids), ip(self.goff), dp(self.hist), ip(self.hoff), dp(mean),
                            dp(var), ip(bad))
        return mean, var, bad

    def grid(self, k):
        d = self.units[k].dim
        return self.grids[self.goff[k]:self.goff[k] + d * (NB + 1)].reshape(d, NB + 1)

    def histogram(self, k):
        d = self.units[k].dim
        return self.hist[self.hoff[k]:self.hoff[k] + d * NB].reshape(d, NB)

    def refine(self, alpha=V.ALPHA_DEFAULT):
        """Lepage refinement of every unit's grid from the last iteration's histogram."""
        for k in range(len(self.units)):
            self.grids[self.goff[k]:self.goff[k] + self.grid(k).size] = V.refine(self.grid(k), self.histogram(k),
                                                                                  alpha).ravel()
