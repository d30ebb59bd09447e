"""The FP64 tanh method of the FP64 kernels, checked on the CPU against
high-precision tanh (mpmath), independently of the device table.

tanh(|x|) on [0, 19.125) is a degree-7 Taylor polynomial around the nearest
multiple of 1/40, with coefficients a_n = P_n(tanh(c)) / n! from the derivative
recursion P_0(T) = T, P_{n+1}(T) = P_n'(T) (1 - T^2); beyond 19.125 it is 1.
"""
import math

import numpy as np
import pytest

mpmath = pytest.importorskip("mpmath")

NCOEF = 8       # a_0 .. a_7
H = 1.0 / 40    # interval width
XMAX = 19.125


def _poly_derivs(n):
    """Coefficient lists (in T, exact integers) of P_0 .. P_{n-1}."""
    P = [0, 1]
    out = []
    for _ in range(n):
        out.append(list(P))
        dP = [d * P[d] for d in range(1, len(P))] or [0]
        Q = [0] * (len(dP) + 2)
        for d, c in enumerate(dP):
            Q[d] += c
            Q[d + 2] -= c
        P = Q
    return out


def _coeffs(c, polys):
    T = mpmath.tanh(mpmath.mpf(c))
    return [float(mpmath.polyval(list(reversed(p)), T) / math.factorial(n)) for n, p in enumerate(polys)]


def test_derivative_recursion_matches_series():
    """P_n(tanh x) are tanh's derivatives: compare with mpmath's differentiation."""
    mpmath.mp.dps = 40
    polys = _poly_derivs(NCOEF)
    for x in (0.0, 0.3, 1.7, 4.0):
        T = mpmath.tanh(x)
        for n, p in enumerate(polys):
            got = mpmath.polyval(list(reversed(p)), T)
            want = mpmath.diff(mpmath.tanh, x, n)
            assert abs(got - want) <= mpmath.mpf(10) ** -30 * (1 + abs(want))


def test_remainder_and_cutoff_bounds():
    mpmath.mp.dps = 40
    Pn = _poly_derivs(NCOEF + 1)[NCOEF]
    ts = [mpmath.mpf(i) / 2000 for i in range(-2000, 2001)]
    mn = max(abs(mpmath.polyval(list(reversed(Pn)), t)) for t in ts)   # max |tanh^(8)| over T in [-1, 1]
    rem = (mpmath.mpf(H) / 2) ** NCOEF * mn / math.factorial(NCOEF)
    assert rem < 3e-17
    # beyond XMAX, +-1 is the correctly rounded tanh: 1 - tanh(XMAX) is below half
    # the spacing (2^-53) of the doubles just under 1
    assert 1 - mpmath.tanh(XMAX) < mpmath.mpf(2) ** -54


def test_piecewise_taylor_accuracy():
    """Float64 Horner on float64 coefficients: within a few units of 2^-53 of tanh."""
    mpmath.mp.dps = 40
    polys = _poly_derivs(NCOEF)
    nint = int(round(XMAX / H)) + 1
    table = [_coeffs(k * H, polys) for k in range(nint)]
    rng = np.random.default_rng(3)
    xs = np.concatenate([rng.uniform(0, XMAX, 4000), np.arange(0, XMAX, H / 2)[:-1], [0.0, 1e-300, 1e-8]])
    worst = 0.0
    for x in xs:
        k = int(round(40.0 * x))
        assert abs(x - k * H) <= H / 2 + 1e-14
        a = table[k]
        t = x - k * H
        p = a[-1]
        for n in range(NCOEF - 2, -1, -1):
            p = p * t + a[n]
        worst = max(worst, abs(p - float(mpmath.tanh(mpmath.mpf(float(x))))))
    assert worst < 6e-16
