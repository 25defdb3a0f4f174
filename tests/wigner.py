"""Exact Wigner 3j symbols (Racah's closed form) and Gaunt integrals for the pins.

Independent of the oracle: integer factorials and exact rationals, converted to
float only at the end.  Used to build the brute-force projection of Phi_L^2
(Eq. 2) onto Y_lm, whose angular prefactor is the I_{l1 l2 l3} of Eq. 22.
"""
from __future__ import annotations

import math
from fractions import Fraction
from functools import lru_cache


@lru_cache(maxsize=None)
def wigner3j(l1: int, l2: int, l3: int, m1: int, m2: int, m3: int) -> float:
    if m1 + m2 + m3 != 0:
        return 0.0
    if l3 < abs(l1 - l2) or l3 > l1 + l2:
        return 0.0
    if abs(m1) > l1 or abs(m2) > l2 or abs(m3) > l3:
        return 0.0
    f = math.factorial
    tri = Fraction(f(l1 + l2 - l3) * f(l1 - l2 + l3) * f(-l1 + l2 + l3), f(l1 + l2 + l3 + 1))
    pre = tri * f(l1 + m1) * f(l1 - m1) * f(l2 + m2) * f(l2 - m2) * f(l3 + m3) * f(l3 - m3)
    kmin = max(0, l2 - l3 - m1, l1 - l3 + m2)
    kmax = min(l1 + l2 - l3, l1 - m1, l2 + m2)
    s = Fraction(0)
    for k in range(kmin, kmax + 1):
        den = (f(k) * f(l3 - l2 + k + m1) * f(l3 - l1 + k - m2) * f(l1 + l2 - l3 - k)
               * f(l1 - k - m1) * f(l2 - k + m2))
        s += Fraction((-1) ** k, den)
    if s == 0:
        return 0.0
    sign = (-1) ** (l1 - l2 - m3) * (1 if s > 0 else -1)
    return sign * math.sqrt(float(pre * s * s))


def gaunt(l1, l2, l3, m1, m2, m3) -> float:
    """int Y_{l1 m1} Y_{l2 m2} Y_{l3 m3} dOmega (orthonormal, Condon-Shortley)."""
    w0 = wigner3j(l1, l2, l3, 0, 0, 0)
    if w0 == 0.0:
        return 0.0
    return math.sqrt((2 * l1 + 1) * (2 * l2 + 1) * (2 * l3 + 1) / (4 * math.pi)) * w0 * \
        wigner3j(l1, l2, l3, m1, m2, m3)
