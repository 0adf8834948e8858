"""The FP64 kernels' point level (reading R27): the recursion over the order
at a fixed degree reproduces the point stencil of Eqs. (rec2), (rec10),
(rec11) exactly, and stays accurate in FP64.

The stencil x_n^m = -xi x_{n-1}^{m-1} + eta x_{n-1}^{m+1} - z x_{n-1}^m
(x^{-m} = (-1)^m conj x^m, x_0^0 = 1, xi = (x + iy)/2, eta = conj xi) is
run in exact rational arithmetic; the order recursion
(n - m) Q_n^m = -(m + 1) z Q_n^{m+1} - (n + m + 2) |xi|^2 Q_n^{m+2},
Q_n^n = 1, Q_n^{n-1} = -n z, x_n^m = (-xi)^m Q_n^m must agree exactly, and
its FP64 evaluation to a few ulps of each degree's norm."""
from fractions import Fraction as Fr

import numpy as np

P = 20


def _stencil_rows(x, y, z, p):
    xr, xi_ = x / 2, y / 2  # xi = xr + i xi_, eta = xr - i xi_
    rows = [[(Fr(1), Fr(0))]]
    for n in range(1, p + 1):
        prev = rows[-1]

        def get(m):
            if abs(m) > n - 1:
                return (Fr(0), Fr(0))
            if m >= 0:
                return prev[m]
            re, im = prev[-m]
            s = -1 if m % 2 else 1
            return (s * re, -s * im)

        new = []
        for m in range(n + 1):
            ar, ai = get(m - 1)
            br, bi = get(m + 1)
            cr, ci = get(m)
            # -xi a + eta b - z c
            re = -(xr * ar - xi_ * ai) + (xr * br + xi_ * bi) - z * cr
            im = -(xr * ai + xi_ * ar) + (xr * bi - xi_ * br) - z * ci
            new.append((re, im))
        rows.append(new)
    return rows


def _order_rows(x, y, z, p, one, cmul):
    """Rows from the order recursion; arithmetic type given by one/cmul."""
    xi = (x / 2, y / 2)
    x2 = xi[0] * xi[0] + xi[1] * xi[1]
    w = [(one, 0 * one)]
    for m in range(1, p + 1):
        w.append(cmul(w[-1], (-xi[0], -xi[1])))
    rows = []
    for n in range(p + 1):
        Q = [0 * one] * (n + 3)
        Q[n] = one
        if n >= 1:
            Q[n - 1] = -n * z
        for m in range(n - 2, -1, -1):
            Q[m] = (-(m + 1) * z * Q[m + 1] - (n + m + 2) * x2 * Q[m + 2]) / (n - m)
        rows.append([(w[m][0] * Q[m], w[m][1] * Q[m]) for m in range(n + 1)])
    return rows


def _cmul(a, b):
    return (a[0] * b[0] - a[1] * b[1], a[0] * b[1] + a[1] * b[0])


def _points():
    rng = np.random.default_rng(27)
    pts = [tuple(Fr(int(v), 1000) for v in rng.integers(-1000, 1001, 3)) for _ in range(3)]
    pts.append((Fr(0), Fr(0), Fr(7, 10)))          # on the axis
    pts.append((Fr(3, 1000), Fr(-1, 1000), Fr(-9, 10)))  # near the axis
    pts.append((Fr(6, 10), Fr(-7, 10), Fr(0)))     # on the equator
    return pts


def test_order_recursion_is_exact():
    for x, y, z in _points():
        ref = _stencil_rows(x, y, z, P)
        got = _order_rows(x, y, z, P, Fr(1), _cmul)
        assert got == ref


def test_order_recursion_fp64_accuracy():
    for x, y, z in _points():
        ref = _stencil_rows(x, y, z, P)
        got = _order_rows(float(x), float(y), float(z), P, 1.0, _cmul)
        for n in range(P + 1):
            e = np.array([complex(float(r[0]), float(r[1])) for r in ref[n]])
            g = np.array([complex(a, b) for a, b in got[n]])
            scale = np.linalg.norm(e)
            assert scale > 0
            assert np.max(np.abs(g - e)) <= 1e-14 * scale, (x, y, z, n)
