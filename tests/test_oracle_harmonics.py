"""Pins for the oracle's solid-harmonic evaluator (Eq. (bas1)-(bas3), (bas5)).

Each pin is independent of the evaluator's own code path: hand-derived closed
forms, the textbook Legendre value at the pole, scipy's associated Legendre
routine, symmetry, homogeneity, harmonicity and the derivative rules by finite
differences, and the Green's-function addition theorem."""
import math

import numpy as np
import pytest

rng = np.random.default_rng(1234)


def k(n, m):
    return n * n + n + m


def test_closed_forms_low_degree(orc):
    # Eq. (bas1) with P_1^1 = -sqrt(1-mu^2), P_2^1 = -3 mu sqrt(1-mu^2),
    # P_2^2 = 3 (1-mu^2): R_1^0 = -z, R_1^{+-1} = i xi / i eta,
    # R_2^0 = (3z^2 - r^2)/4, R_2^1 = -i z xi, R_2^2 = -xi^2/2.
    for _ in range(5):
        x, y, z = rng.uniform(-1, 1, 3)
        xi, eta = (x + 1j * y) / 2, (x - 1j * y) / 2
        R = orc.rnm([x, y, z], 2)
        r2 = x * x + y * y + z * z
        exp = {
            (0, 0): 1.0, (1, 0): -z, (1, 1): 1j * xi, (1, -1): 1j * eta,
            (2, 0): (3 * z * z - r2) / 4, (2, 1): -1j * z * xi, (2, 2): -xi * xi / 2,
            (2, -1): -1j * z * eta, (2, -2): -eta * eta / 2,
        }
        for (n, m), v in exp.items():
            assert abs(R[k(n, m)] - v) < 1e-15, (n, m)


def test_pole_value(orc):
    # P_n(1) = 1  =>  R_n^0(0,0,z) = (-1)^n z^n / n!, and R_n^m = 0 for m != 0
    z = 0.7
    p = 12
    R = orc.rnm([0, 0, z], p)
    for n in range(p + 1):
        assert abs(R[k(n, 0)] - (-1) ** n * z ** n / math.factorial(n)) < 1e-15
        for m in range(1, n + 1):
            assert R[k(n, m)] == 0 and R[k(n, -m)] == 0


def test_against_scipy_legendre(orc):
    sp = pytest.importorskip("scipy.special")
    p = 15
    for _ in range(4):
        v = rng.standard_normal(3)
        r = np.linalg.norm(v)
        th = math.acos(v[2] / r)
        ph = math.atan2(v[1], v[0])
        R = orc.rnm(v, p)
        for n in range(p + 1):
            for m in range(-n, n + 1):
                am = abs(m)
                Pnm = sp.lpmv(am, n, math.cos(th))  # includes the Condon-Shortley phase
                exp = (-1) ** n * (1j ** am) / math.factorial(n + am) * r ** n * Pnm * np.exp(1j * m * ph)
                scale = r ** n / math.sqrt(math.factorial(n + am) * math.factorial(n - am))
                assert abs(R[k(n, m)] - exp) <= 1e-12 * scale, (n, m)


def test_conjugate_symmetry_and_homogeneity(orc):
    p = 20
    v = rng.standard_normal(3)
    R = orc.rnm(v, p)
    R2 = orc.rnm(2.5 * v, p)
    for n in range(p + 1):
        for m in range(1, n + 1):
            # Eq. (bas2.1)
            assert abs(R[k(n, -m)] - (-1) ** m * np.conj(R[k(n, m)])) <= 1e-14 * abs(R[k(n, m)]) + 1e-300
        for m in range(-n, n + 1):
            assert abs(R2[k(n, m)] - 2.5 ** n * R[k(n, m)]) <= 1e-12 * abs(R2[k(n, m)]) + 1e-300


def _fd_grad(orc, v, p, h=1e-5):
    g = []
    for d in range(3):
        e = np.zeros(3)
        e[d] = h
        g.append((orc.rnm(v + e, p) - orc.rnm(v - e, p)) / (2 * h))
    return g


def test_derivative_rules_bas5(orc):
    # d/dz R_n^m = -R_{n-1}^m ; (d/dx + i d/dy) R_n^m = i R_{n-1}^{m+1} ;
    # (d/dx - i d/dy) R_n^m = i R_{n-1}^{m-1}   (Eqs. (bas5), (bas7))
    p = 10
    v = rng.uniform(-0.8, 0.8, 3)
    gx, gy, gz = _fd_grad(orc, v, p)
    R = orc.rnm(v, p)

    def Rget(n, m):
        return R[k(n, m)] if abs(m) <= n and n >= 0 else 0.0

    for n in range(1, p + 1):
        for m in range(-n, n + 1):
            tol = 1e-8
            assert abs(gz[k(n, m)] + Rget(n - 1, m)) < tol
            assert abs(gx[k(n, m)] + 1j * gy[k(n, m)] - 1j * Rget(n - 1, m + 1)) < tol
            assert abs(gx[k(n, m)] - 1j * gy[k(n, m)] - 1j * Rget(n - 1, m - 1)) < tol


def test_harmonic(orc):
    p = 12
    v = rng.uniform(-0.7, 0.7, 3)
    h = 1e-3
    lap = -6 * orc.rnm(v, p)
    for d in range(3):
        e = np.zeros(3)
        e[d] = h
        lap = lap + orc.rnm(v + e, p) + orc.rnm(v - e, p)
    lap /= h * h
    assert np.max(np.abs(lap)) < 1e-6


def test_addition_theorem_bas3(orc):
    # G(r, r') = 1/(4 pi |r - r'|) = (1/4pi) sum (-1)^n R_n^{-m}(r') S_n^m(r),
    # truncation error <= (|r'|/|r|)^(p+1) / (|r| - |r'|) (geometric majorant)
    rp = np.array([0.2, -0.1, 0.15])
    r = np.array([0.9, 1.1, -0.6])
    G = 1.0 / (4 * math.pi * np.linalg.norm(r - rp))
    ratio = np.linalg.norm(rp) / np.linalg.norm(r)
    for p in (2, 5, 10, 20, 30):
        R = orc.rnm(rp, p)
        S = orc.snm(r, p)
        acc = 0.0
        for n in range(p + 1):
            for m in range(-n, n + 1):
                acc += (-1) ** n * R[k(n, -m)] * S[k(n, m)]
        acc /= 4 * math.pi
        assert abs(acc.imag) < 1e-15
        bound = ratio ** (p + 1) / (4 * math.pi * (np.linalg.norm(r) - np.linalg.norm(rp)))
        assert abs(acc.real - G) <= bound + 1e-16


def test_singular_against_scipy(orc):
    sp = pytest.importorskip("scipy.special")
    p = 10
    v = rng.standard_normal(3) * 2
    r = np.linalg.norm(v)
    th = math.acos(v[2] / r)
    ph = math.atan2(v[1], v[0])
    S = orc.snm(v, p)
    for n in range(p + 1):
        for m in range(-n, n + 1):
            am = abs(m)
            exp = (1j ** (-am)) * math.factorial(n - am) * r ** (-n - 1) * sp.lpmv(am, n, math.cos(th)) \
                * np.exp(1j * m * ph)
            assert abs(S[k(n, m)] - exp) <= 1e-12 * max(1.0, abs(exp))
