"""Sobol low-discrepancy points with a random digital shift (oracle, numpy).

Construction of I. M. Sobol (1967) as organised by Bratley and Fox (1988):
coordinate j uses a primitive polynomial over GF(2) of degree s,
x^s + a_1 x^{s-1} + ... + a_{s-1} x + 1, and odd initial integers m_1..m_s
(m_k < 2^k); further m_k follow the recurrence

    m_k = 2 a_1 m_{k-1} ^ 4 a_2 m_{k-2} ^ ... ^ 2^{s-1} a_{s-1} m_{k-s+1} ^ 2^s m_{k-s} ^ m_{k-s},

and the direction numbers are V_k = m_k 2^{32-k} (32-bit).  Point n (Gray-code
order, Antonov and Saleev 1979) is the XOR of V_k over the set bits k of
g = n ^ (n >> 1).

Fixed choices of this project (no direction-number table is available, and
the quality guarantee of a Sobol sequence, its t-value, does not depend on the
initial m_k): coordinate 1 uses m_k = 1 for all k (van der Corput); coordinates
2, 3, ... use the primitive polynomials of degree >= 1 in increasing order of
degree and, within a degree, of the integer whose bits are the coefficients,
each with all initial m_k = 1.  The primitive polynomials are found here by
brute force (irreducible and of maximal multiplicative order 2^s - 1).

The digital shift of coordinate j for (seed, unit, iteration) is word j mod 4
of Philox4x32-10 with key (seed, unit key) and counter (0, 0, iteration,
0x80000000 + j div 4).  The coordinate is u = (2 (x ^ shift) + 1) 2^-33.
"""
from __future__ import annotations

import numpy as np

from .philox import philox4x32_10

BITS = 32


def _polymulmod(a, b, mod, deg):
    r = 0
    while b:
        if b & 1:
            r ^= a
        b >>= 1
        a <<= 1
        if a >> deg & 1:
            a ^= mod
    return r


def _is_primitive(poly, deg):
    """poly: int with bit i = coefficient of x^i (bit deg and bit 0 set)."""
    order = (1 << deg) - 1
    if deg == 1:
        return poly == 0b11
    # x^order == 1 mod poly and x^(order/p) != 1 for each prime p | order
    def xpow(e):
        result, base = 1, 0b10
        while e:
            if e & 1:
                result = _polymulmod(result, base, poly, deg)
            base = _polymulmod(base, base, poly, deg)
            e >>= 1
        return result
    if xpow(order) != 1:
        return False
    n, p, primes = order, 2, []
    while p * p <= n:
        while n % p == 0:
            primes.append(p)
            n //= p
        p += 1
    if n > 1:
        primes.append(n)
    return all(xpow(order // p) != 1 for p in set(primes))


def primitive_polynomials(count):
    out = []
    deg = 1
    while len(out) < count:
        for poly in range(1 << deg, 1 << (deg + 1)):
            if poly & 1 and _is_primitive(poly, deg):
                out.append((deg, poly))
                if len(out) == count:
                    break
        deg += 1
    return out


def direction_numbers(dim):
    """uint32 array (dim, 32): V[j, k-1] for k = 1..32."""
    V = np.zeros((dim, BITS), dtype=np.uint64)
    for k in range(1, BITS + 1):
        V[0, k - 1] = 1 << (BITS - k)
    for j, (s, poly) in enumerate(primitive_polynomials(dim - 1), start=1):
        a = [(poly >> (s - i)) & 1 for i in range(1, s)]     # a_1..a_{s-1}
        m = [0] * (BITS + 1)
        for k in range(1, s + 1):
            m[k] = 1
        for k in range(s + 1, BITS + 1):
            v = m[k - s] ^ (m[k - s] << s)
            for i in range(1, s):
                if a[i - 1]:
                    v ^= m[k - i] << i
            m[k] = v
        for k in range(1, BITS + 1):
            V[j, k - 1] = m[k] << (BITS - k)
    assert int(V.max()) < (1 << 32)
    return V.astype(np.uint32)


def sobol_ints(first, count, dim):
    """Unshifted 32-bit Sobol integers of points first..first+count-1 (Gray-code order)."""
    V = direction_numbers(dim)
    n = np.arange(first, first + count, dtype=np.uint64)
    g = n ^ (n >> np.uint64(1))
    X = np.zeros((count, dim), dtype=np.uint32)
    for k in range(BITS):
        bit = ((g >> np.uint64(k)) & np.uint64(1)).astype(bool)
        X[bit] ^= V[:, k][None, :]
    return X


def shifts(seed, unit_key, iteration, dim):
    out = np.empty(dim, dtype=np.uint32)
    for q in range((dim + 3) // 4):
        r = philox4x32_10(0, 0, iteration, 0x80000000 + q, seed & 0xFFFFFFFF, unit_key & 0xFFFFFFFF)
        for i in range(4):
            if 4 * q + i < dim:
                out[4 * q + i] = r[i]
    return out


def uniforms(seed, unit_key, iteration, first, count, dim):
    X = sobol_ints(first, count, dim) ^ shifts(seed, unit_key, iteration, dim)[None, :]
    return (2.0 * X.astype(np.float64) + 1.0) * 2.0 ** -33
