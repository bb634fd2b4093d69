"""Fourier-harmonic coefficients of the periodic kernel from the paper's own
series, Eq. (taylor), in exact rational arithmetic.

TEST INFRASTRUCTURE ONLY (same import rule as the rest of ``oracle``).

Eq. (taylor) expands exp(-2 sin^2(pi f dt) / sigma^2) (the periodic kernel
without its 1/(sqrt(2 pi) sigma) prefactor) as

    sum_k (-1)^k / (k! sigma^(2k) 2^(k-1)) * sum_{m<=k} C(2k, k-m) (-1)^m g_m cos(2 pi m f dt),

g_0 = 1/2, g_m = 1 otherwise.  Collecting the terms of each harmonic m gives
the coefficient b_m of cos(2 pi m f dt):

    b_m = g_m (-1)^m sum_{k>=m} (-1)^k C(2k, k-m) / (k! sigma^(2k) 2^(k-1)).

The alternating sum cancels catastrophically in floating point for small
sigma, so it is summed here with Python ``fractions`` (exact), truncated
once the remaining terms are provably below 2^-80 of the leading ones.
sigma^2 enters as an exact rational (the decimal string of sigma).
"""
from __future__ import annotations

from fractions import Fraction
from math import comb


def _kappa(sigma) -> Fraction:
    s = Fraction(str(sigma))
    return 1 / (s * s)


def taylor_harmonic_coefficients(sigma, n_max: int, tol_bits: int = 80) -> list:
    """b_0 .. b_{n_max} of Eq. (taylor) regrouped by harmonic, as floats.

    The sum over k is cut when a term falls below 2^-tol_bits and the term
    ratio is already < 1/2 (the terms then decay at least geometrically)."""
    kap = _kappa(sigma)
    out = []
    for m in range(n_max + 1):
        g = Fraction(1, 2) if m == 0 else Fraction(1)
        acc = Fraction(0)
        k = m
        # term_k = (-1)^k C(2k, k-m) kap^k / (k! 2^(k-1))
        fact = Fraction(1)
        for q in range(2, k + 1):
            fact *= q
        prev = None
        while True:
            term = Fraction(comb(2 * k, k - m)) * kap ** k / (fact * Fraction(2) ** (k - 1))
            acc += term if k % 2 == 0 else -term
            if prev is not None and term * 2 < prev and term < Fraction(1, 2 ** tol_bits):
                break
            prev = term
            k += 1
            fact *= k
            if k > m + 20000:
                raise RuntimeError("series did not converge")
        out.append(float(g * (-1) ** m * acc))
    return out
