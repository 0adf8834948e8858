"""Brute force on tiny inputs: exact rational integration (sympy) of R_n^m
built from Rodrigues' formula, Eq. (bas2), over elements with rational
vertices, compared with the oracle's quadrature (NORM_MOMENT, p <= 4).

Independent of the oracle's evaluator (three-term recurrence) and of its
quadrature (Gauss rules): here P_n^m comes from differentiating (mu^2-1)^n
and the integrals are the Dirichlet monomial formula a! b! c! / (a+b+c+d)!."""
import math
from fractions import Fraction

import numpy as np
import pytest

sp = pytest.importorskip("sympy")

x, y, z, u, v, w, mu = sp.symbols("x y z u v w mu")


def R_exact(n, m):
    """R_n^m(x,y,z) of Eq. (bas1) as an exact sympy polynomial."""
    am = abs(m)
    Q = sp.diff((mu ** 2 - 1) ** n, mu, n + am) / (2 ** n * sp.factorial(n))
    Q = sp.Poly(sp.expand(Q), mu)
    r2 = x * x + y * y + z * z
    poly = 0
    for (j,), c in Q.terms():  # r^{n-m} Q(z/r) = sum c z^j r^{n-m-j}
        e = n - am - j
        assert e % 2 == 0
        poly += c * z ** j * r2 ** (e // 2)
    xy = (x + sp.I * y) if m >= 0 else (x - sp.I * y)
    T = (-1) ** am * xy ** am * poly  # r^n P_n^|m| e^{i m phi}, Condon-Shortley (-1)^m
    return sp.expand((-1) ** n * sp.I ** am / sp.factorial(n + am) * T)


def simplex_integral(expr, X, kind):
    """exact int over the element of expr(y), y = X0 + u Ru + v Rv + w Rw."""
    X = [[sp.Rational(c) for c in row] for row in X]
    sub = {}
    for d, s in enumerate((x, y, z)):
        e = X[0][d] + u * (X[1][d] - X[0][d])
        if kind >= 1:
            e += v * (X[2][d] - X[0][d])
        if kind >= 2:
            e += w * (X[3][d] - X[0][d])
        sub[s] = e
    P = sp.Poly(sp.expand(expr.subs(sub, simultaneous=True)), u, v, w)
    tot = 0
    dim = kind + 1
    for (a, b, c), coef in P.terms():
        tot += coef * sp.factorial(a) * sp.factorial(b) * sp.factorial(c) / sp.factorial(a + b + c + dim)
    # Jacobian
    M = sp.Matrix([[X[i][d] - X[0][d] for d in range(3)] for i in range(1, kind + 2)])
    if kind == 0:
        J = sp.sqrt(sum(t * t for t in M.row(0)))
    elif kind == 1:
        cr = M.row(0).cross(M.row(1))
        J = sp.sqrt(sum(t * t for t in cr))
    else:
        J = abs(M.det())
    return sp.nsimplify(tot) * J


@pytest.mark.parametrize("kind,name", [(0, "segment"), (1, "triangle"), (2, "tetra")])
def test_exact_rational(orc, kind, name):
    p = 4 if kind < 2 else 3
    Xr = {
        0: [["1/3", "-1/5", "1/7"], ["1/2", "1/4", "-1/3"]],
        1: [["1/3", "-1/5", "1/7"], ["1/2", "1/4", "-1/3"], ["-1/6", "2/5", "1/9"]],
        2: [["1/3", "-1/5", "1/7"], ["1/2", "1/4", "-1/3"], ["-1/6", "2/5", "1/9"], ["1/8", "1/8", "3/5"]],
    }[kind]
    X = np.array([[float(Fraction(c)) for c in row] for row in Xr])
    got = orc.moments(name, X.T.copy(), np.arange(kind + 2, dtype=np.int32)[:, None], np.array([1.0]), p,
                      leaf_c=np.zeros((3, 1)), norm=1)[0]
    for n in range(p + 1):
        for m in range(0, n + 1):
            ex = complex(sp.N(simplex_integral(R_exact(n, m), Xr, kind), 30))
            g = got[n * n + n + m] + (1j * got[n * n + n - m] if m else 0)
            scale = 0.6 ** n / math.sqrt(math.factorial(n + m) * math.factorial(n - m))
            assert abs(g - ex) <= 1e-15 * scale + 1e-17, (n, m, g, ex)
