"""Prefactor series of Eq. 2 (oracle, mpmath).

Eq. 2 of the paper multiplies the parametric integral by
(i pi^{d/2})^l Gamma(A - l d/2) / prod_j Gamma(a_j);  Sec. 4.3 states that the
results are reported with (i pi^{d/2})^l and e^{-l gamma_E eps} pulled out.  The
series that multiplies the eps-expansion of the parametric integral is therefore

    c(eps) = e^{l gamma_E eps} Gamma(A - 2l + l eps) / prod_j Gamma(a_j),   d = 4 - 2 eps.

Its Laurent coefficients are taken here by Cauchy's integral formula on a circle
around eps = 0 (mpmath.taylor with method='quad'), applied to eps^q c(eps) with q
the pole order, so that no evaluation happens at the pole.
"""
from __future__ import annotations

import mpmath as mp


def prefactor_series(indices, loops, kmax, dps=40):
    """Return (q, coeffs): c(eps) = sum_{i>=0} coeffs[i] eps^{i-q}, i = 0..kmax+q.

    q is the order of the pole of c at eps = 0 (0 if regular).  ``kmax`` is the
    highest power of eps wanted.
    """
    A = sum(indices)
    L = loops
    n0 = A - 2 * L
    q = 1 if n0 <= 0 else 0
    with mp.workdps(dps):
        den = mp.mpf(1)
        for a in indices:
            den *= mp.gamma(a)

        def h(e):
            return e ** q * mp.exp(L * mp.euler * e) * mp.gamma(n0 + L * e) / den

        coeffs = mp.taylor(h, 0, kmax + q, method="quad", radius=mp.mpf(1) / (4 * max(L, 1) * (abs(n0) + 1)))
        return q, [mp.mpf(c.real) if isinstance(c, mp.mpc) else mp.mpf(c) for c in coeffs]


def combine(prefactor, integral_orders, integral_values, out_orders):
    """R_n = sum_m c_m I_{n-m} for the requested output orders n.

    ``prefactor`` is (q, coeffs) from prefactor_series; ``integral_values`` maps
    each eps order K of the parametric integral to its value.
    """
    q, coeffs = prefactor
    out = {}
    for n in out_orders:
        s = 0
        for i, c in enumerate(coeffs):
            m = i - q
            K = n - m
            if K in integral_values:
                s += c * integral_values[K]
        out[n] = s
    return out
