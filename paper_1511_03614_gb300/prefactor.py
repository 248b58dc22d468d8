"""Laurent series of the prefactor of Eq. 2 (host, float64).

With (i pi^{d/2})^l and e^{-l gamma_E eps} pulled out (Sec. 4.3) the parametric
integral is multiplied by

    c(eps) = e^{l gamma eps} Gamma(n0 + l eps) / prod_j Gamma(a_j),   n0 = A - 2l,  d = 4 - 2 eps.

Here Gamma(n0 + x) is reduced to Gamma(1 + x) by the recurrence
Gamma(z+1) = z Gamma(z), and e^{gamma x} Gamma(1 + x) = exp(sum_{k>=2} (-1)^k zeta(k) x^k / k)
(the Weierstrass product of Gamma), with zeta(k) summed directly with an
Euler-Maclaurin tail.
"""
from __future__ import annotations

import math


def zeta(k, n=32):
    """Riemann zeta(k) for integer k >= 2 to double precision (Euler-Maclaurin, tail at n)."""
    s = math.fsum(i ** -k for i in range(1, n))
    # tail sum_{i>=n} i^-k = n^{1-k}/(k-1) + n^-k/2 + k n^{-k-1}/12 - k(k+1)(k+2) n^{-k-3}/720 + ...
    t = n ** (1 - k) / (k - 1) + 0.5 * n ** -k + k * n ** (-k - 1) / 12.0 \
        - k * (k + 1) * (k + 2) * n ** (-k - 3) / 720.0 \
        + k * (k + 1) * (k + 2) * (k + 3) * (k + 4) * n ** (-k - 5) / 30240.0
    return s + t


def _mul(a, b, n):
    return [math.fsum(a[i] * b[k - i] for i in range(k + 1) if i < len(a) and k - i < len(b)) for k in range(n)]


def _exp_series(c, n):
    """exp of a power series with c[0] == 0, n terms (recurrence k e_k = sum j c_j e_{k-j})."""
    e = [1.0] + [0.0] * (n - 1)
    for k in range(1, n):
        e[k] = math.fsum(j * c[j] * e[k - j] for j in range(1, k + 1) if j < len(c)) / k
    return e


def series(indices, loops, kmax):
    """(q, coeffs) with c(eps) = sum_i coeffs[i] eps^{i-q}, for powers up to eps^kmax."""
    L = loops
    n0 = sum(indices) - 2 * L
    q = 1 if n0 <= 0 else 0
    nterms = kmax + q + 1
    # e^{gamma x} Gamma(1 + x) with x = L eps
    lg = [0.0, 0.0] + [(-1) ** k * zeta(k) / k * L ** k for k in range(2, nterms + 1)]
    base = _exp_series(lg, nterms + 1)
    # Gamma(n0 + x) = Gamma(1 + x) * prod_{i=1}^{n0-1} (i + x)             (n0 >= 1)
    #              = Gamma(1 + x) / prod_{i=n0}^{0} (i + x)                 (n0 <= 0)
    rat = [1.0]
    if n0 >= 1:
        for i in range(1, n0):
            rat = _mul(rat, [float(i), float(L)], nterms + 1)
    else:
        # 1/(L eps) * prod_{i=n0}^{-1} 1/(i + L eps); the eps^-1 is carried by q
        rat = [1.0 / L]
        for i in range(n0, 0):
            inv = [(1.0 / i) * (-L / i) ** m for m in range(nterms + 1)]
            rat = _mul(rat, inv, nterms + 1)
    out = _mul(base, rat, nterms)
    den = math.prod(math.gamma(a) for a in indices)
    return q, [v / den for v in out]
