"""Exact (rational) FD weights derived independently of the oracle.

The weights are obtained by solving the Taylor moment conditions of a
symmetric (second derivative) or antisymmetric (first derivative) stencil of
radius r with exact Fraction arithmetic.  They serve as an independent pin of
the oracle's closed-form weights and as the source of the exact stencil
symbols used by the plane-wave (dispersion) pins.
"""
from fractions import Fraction
import math


def _solve(a, b):
    n = len(b)
    a = [row[:] + [b[i]] for i, row in enumerate(a)]
    for col in range(n):
        piv = next(r for r in range(col, n) if a[r][col] != 0)
        a[col], a[piv] = a[piv], a[col]
        for r in range(n):
            if r != col and a[r][col] != 0:
                f = a[r][col] / a[col][col]
                a[r] = [x - f * y for x, y in zip(a[r], a[col])]
    return [a[i][n] / a[i][i] for i in range(n)]


def second_derivative_weights(r):
    """[w0, w1, ..., wr] with sum_{k=-r..r} w_|k| k^p = 2 delta_{p,2}, p = 0,2,..,2r."""
    rows, rhs = [], []
    for q in range(r + 1):
        p = 2 * q
        row = [Fraction(1) if p == 0 else Fraction(0)]  # k = 0 term: 0^p
        row += [Fraction(2 * k ** p) for k in range(1, r + 1)]
        rows.append(row)
        rhs.append(Fraction(2) if p == 2 else Fraction(0))
    return _solve(rows, rhs)


def first_derivative_weights(r):
    """[0, c1, ..., cr] with sum_k c_k (k^p - (-k)^p) = delta_{p,1}, p = 1,3,..,2r-1."""
    rows, rhs = [], []
    for q in range(r):
        p = 2 * q + 1
        rows.append([Fraction(2 * k ** p) for k in range(1, r + 1)])
        rhs.append(Fraction(1) if p == 1 else Fraction(0))
    return [Fraction(0)] + _solve(rows, rhs)


def second_symbol(r, theta):
    """sigma(theta) >= 0 with  D2 e^{i k x} = -sigma(k h)/h^2 e^{i k x}."""
    w = second_derivative_weights(r)
    return -(float(w[0]) + 2.0 * sum(float(w[k]) * math.cos(k * theta) for k in range(1, r + 1)))


def first_symbol(r, theta):
    """s(theta) with  D1 e^{i k x} = i s(k h)/h e^{i k x}."""
    c = first_derivative_weights(r)
    return 2.0 * sum(float(c[k]) * math.sin(k * theta) for k in range(1, r + 1))


def staggered_weights(r):
    """[0, a1, ..., ar] with sum_k a_k 2 (k - 1/2)^p = delta_{p,1}, p = 1,3,..,2r-1
    (first derivative at a half point from nodes at +-(k - 1/2) h)."""
    rows, rhs = [], []
    half = Fraction(1, 2)
    for q in range(r):
        p = 2 * q + 1
        rows.append([2 * (k - half) ** p for k in range(1, r + 1)])
        rhs.append(Fraction(1) if p == 1 else Fraction(0))
    return [Fraction(0)] + _solve(rows, rhs)


def staggered_symbol(r, theta):
    """s(theta) with  D+ e^{i k x} = e^{i theta/2} i s(theta)/h e^{i k x} and
    D- e^{i k x} = e^{-i theta/2} i s(theta)/h e^{i k x}, theta = k h."""
    a = staggered_weights(r)
    return 2.0 * sum(float(a[k]) * math.sin((k - 0.5) * theta) for k in range(1, r + 1))
