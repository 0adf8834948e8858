"""Pins for the oracle's quadrature moments (Eq. (bas4), (bas9), (bas10)).

Closed forms (rec3 seeds, measure, centroid relations), Gauss exactness,
rotation covariance, the point-charge limit, divergence-theorem identities
linking the tetrahedron and triangle paths, and closed-surface identities."""
import math
import os

import numpy as np
import pytest

import workloads as W

rng = np.random.default_rng(99)
HERE = os.path.dirname(os.path.abspath(__file__))


def k(n, m):
    return n * n + n + m


def unpack(c, p):
    """packed real -> complex F_n^m for m >= 0, as dict."""
    out = {}
    for n in range(p + 1):
        for m in range(0, n + 1):
            out[(n, m)] = c[k(n, m)] + (1j * c[k(n, -m)] if m else 0.0)
    return out


def single(orc, kind, X, sig, c, p, norm=0, density=0, layer=0, nq=0):
    X = np.asarray(X, dtype=np.float64)  # (nv, 3)
    nv = X.shape[0]
    vxyz = X.T.copy()
    idx = np.arange(nv, dtype=np.int32)[:, None]
    sig = np.atleast_1d(np.asarray(sig, dtype=np.float64))
    return orc.moments(kind, vxyz, idx, sig, p, leaf_off=None, leaf_c=np.asarray(c, float).reshape(3, 1),
                       layer=layer, density=density, norm=norm, nq=nq)[0]


def test_gauss_legendre_exact(orc):
    for kq in (1, 2, 3, 5, 8, 13, 20):
        x, w = orc.gauss_legendre(kq)
        for a in range(2 * kq):
            assert abs(np.dot(w, x ** a) - 1.0 / (a + 1)) < 1e-15 * 4


def test_rec3_seeds_golden(orc):
    vals = {}
    with open(os.path.join(HERE, "golden", "rec3_unit_simplex_seeds.txt")) as f:
        for line in f:
            if line.strip() and not line.startswith("#"):
                a, b = line.split()
                vals[a] = float(b)
    # unit simplices: segment (0,0,0)-(1,0,0), triangle T, tetrahedron Q (Jacobian 1)
    e = np.eye(3)
    seg = [np.zeros(3), e[0]]
    tri = [np.zeros(3), e[0], e[1]]
    tet = [np.zeros(3), e[0], e[1], e[2]]
    mom = lambda kind, X: single(orc, kind, X, 1.0, np.zeros(3), 0, norm=1)[0]
    assert abs(mom("segment", seg) - vals["p_0^0"]) < 1e-15
    assert abs(mom("triangle", tri) - vals["i_0^0"]) < 1e-15
    assert abs(mom("tetra", tet) - vals["a_0^0"]) < 1e-15


def test_dirichlet_monomials(orc):
    # NORM_MOMENT of R_1^0 = -z and R_2^0 = (3z^2 - r^2)/4 over unit simplices
    # placed along z: int_T v^a = a! / (a+2)!, int_Q w^a = a!/(a+3)!.
    e = np.eye(3)
    tri = [np.zeros(3), e[0], e[2]]  # v -> z
    m = single(orc, "triangle", tri, 1.0, np.zeros(3), 2, norm=1)
    # R_1^0 = -z : -int v = -1/6 ; R_2^0 = (3z^2 - x^2 - y^2 - z^2)/4 = (2 v^2 - u^2)/4
    assert abs(m[k(1, 0)] + 1.0 / 6) < 1e-15
    exp = (2 * 2 / math.factorial(4) - 2 / math.factorial(4)) / 4
    assert abs(m[k(2, 0)] - exp) < 1e-15
    tet = [np.zeros(3), e[0], e[1], e[2]]
    m = single(orc, "tetra", tet, 1.0, np.zeros(3), 2, norm=1)
    assert abs(m[k(1, 0)] + 1.0 / 24) < 1e-15
    # R_2^0 over Q: (2 w^2 - u^2 - v^2)/4 -> int w^2 = 2/5! each
    assert abs(m[k(2, 0)] - (2 * 2 / 120 - 2 * 2 / 120) / 4) < 1e-15


def random_simplex(kind, scale=0.2, centre=None):
    nv = {"segment": 2, "triangle": 3, "tetra": 4}[kind]
    c0 = rng.uniform(-0.3, 0.3, 3) if centre is None else centre
    X = c0 + scale * rng.standard_normal((nv, 3))
    return X


def measure(kind, X):
    if kind == "segment":
        return np.linalg.norm(X[1] - X[0])
    if kind == "triangle":
        return 0.5 * np.linalg.norm(np.cross(X[1] - X[0], X[2] - X[0]))
    return abs(np.dot(np.cross(X[1] - X[0], X[2] - X[0]), X[3] - X[0])) / 6


@pytest.mark.parametrize("kind", ["segment", "triangle", "tetra"])
def test_zeroth_and_first_order(orc, kind):
    X = random_simplex(kind)
    c = rng.uniform(-0.2, 0.2, 3)
    sig = rng.uniform(-1, 1)
    p = 3
    F = unpack(single(orc, kind, X, sig, c, p), p)
    mu = measure(kind, X)
    xc, yc, zc = X.mean(axis=0) - c  # centroid of a simplex = vertex mean
    assert abs(F[(0, 0)] - sig * mu / (4 * math.pi)) < 1e-15
    # L_1^0 = sig mu z_c / 4pi ; L_1^1 = -i sig mu (x_c - i y_c) / (8 pi)
    assert abs(F[(1, 0)] - sig * mu * zc / (4 * math.pi)) < 1e-15
    assert abs(F[(1, 1)] - (-1j * sig * mu * (xc - 1j * yc) / (8 * math.pi))) < 1e-15


def test_linear_density_mean_and_constant_limit(orc):
    X = random_simplex("triangle")
    c = np.zeros(3)
    s = rng.uniform(-1, 1, 3)
    p = 8
    lin = single(orc, "triangle", X, s, c, p, density=1)
    A = measure("triangle", X)
    assert abs(lin[0] - A * s.mean() / (4 * math.pi)) < 1e-15
    # first moment with linear density: int sig y = A/12 (sum_k s_k x_k + sum_k s_k * sum_j x_j)
    y = X - c
    first = A / 12 * (s @ y + s.sum() * y.sum(axis=0))
    F = unpack(lin, p)
    assert abs(F[(1, 0)] - first[2] / (4 * math.pi)) < 1e-15
    # all-equal vertex densities = constant density
    cst = single(orc, "triangle", X, 0.37, c, p)
    eq = single(orc, "triangle", X, [0.37] * 3, c, p, density=1)
    assert np.max(np.abs(cst - eq)) < 1e-15 * np.max(np.abs(cst)) * 10
    # linearity in the vertex densities
    parts = sum(s[i] * single(orc, "triangle", X, np.eye(3)[i], c, p, density=1) for i in range(3))
    assert np.max(np.abs(parts - lin)) < 1e-14 * np.max(np.abs(lin))


def test_double_layer_low_orders(orc):
    X = random_simplex("triangle")
    c = rng.uniform(-0.2, 0.2, 3)
    sig = 0.8
    p = 2
    D = unpack(single(orc, "triangle", X, sig, c, p, layer=1), p)
    cr = np.cross(X[1] - X[0], X[2] - X[0])
    A = 0.5 * np.linalg.norm(cr)
    nx, ny, nz = cr / np.linalg.norm(cr)
    assert abs(D[(0, 0)]) < 1e-16
    # M_1^0 = sig A n_z / 4pi ; M_1^1 = -(1/4pi) sig A i (n_x - i n_y)/2
    assert abs(D[(1, 0)] - sig * A * nz / (4 * math.pi)) < 1e-15
    assert abs(D[(1, 1)] + sig * A * 1j * (nx - 1j * ny) / (8 * math.pi)) < 1e-15


@pytest.mark.parametrize("kind", ["segment", "triangle", "tetra"])
def test_rotation_about_z(orc, kind):
    # R_n^{-m}(Rot_a y) = e^{-i m a} R_n^{-m}(y)  =>  F_n^m -> e^{-i m a} F_n^m
    p = 9
    X = random_simplex(kind)
    a = 0.73
    Rz = np.array([[math.cos(a), -math.sin(a), 0], [math.sin(a), math.cos(a), 0], [0, 0, 1]])
    F0 = unpack(single(orc, kind, X, 0.6, np.zeros(3), p), p)
    F1 = unpack(single(orc, kind, X @ Rz.T, 0.6, np.zeros(3), p), p)
    for (n, m), v in F0.items():
        assert abs(F1[(n, m)] - np.exp(-1j * m * a) * v) < 1e-15 + 1e-12 * abs(v)


@pytest.mark.parametrize("kind", ["segment", "triangle", "tetra"])
def test_point_limit(orc, kind):
    # shrinking the element to a point y: F / measure -> (1/4pi)(-1)^n R_n^{-m}(y - c)
    p = 6
    y = np.array([0.2, -0.15, 0.1])
    X = y + 1e-6 * rng.standard_normal(({"segment": 2, "triangle": 3, "tetra": 4}[kind], 3))
    F = single(orc, kind, X, 1.0, np.zeros(3), p) / measure(kind, X)
    R = orc.rnm(X.mean(axis=0), p)
    for n in range(p + 1):
        for m in range(0, n + 1):
            exp = (-1) ** n * R[k(n, -m)] / (4 * math.pi)
            got = F[k(n, m)] + (1j * F[k(n, -m)] if m else 0)
            assert abs(got - exp) < 1e-10 * 0.3 ** n + 1e-16


def test_tetra_equals_face_sum(orc):
    # div(y R_n^m) = (n+3) R_n^m  =>  int_V R = 1/(n+3) sum_faces (y . n_f) int_f R
    # (y . n_f constant on a flat face). Links the tetra and triangle paths.
    p = 10
    X = random_simplex("tetra", scale=0.3)
    if np.dot(np.cross(X[1] - X[0], X[2] - X[0]), X[3] - X[0]) < 0:
        X[[2, 3]] = X[[3, 2]]
    c = np.zeros(3)
    vol = single(orc, "tetra", X, 1.0, c, p, norm=1)
    faces = [(1, 2, 3), (0, 3, 2), (0, 1, 3), (0, 2, 1)]  # outward for positive orientation
    acc = np.zeros_like(vol)
    for f in faces:
        F = X[list(f)]
        nrm = np.cross(F[1] - F[0], F[2] - F[0])
        nrm /= np.linalg.norm(nrm)
        hgt = np.dot(F[0] - c, nrm)
        acc += hgt * single(orc, "triangle", F, 1.0, c, p, norm=1)
    for n in range(p + 1):
        sl = slice(n * n, (n + 1) ** 2)
        acc[sl] /= n + 3
    assert np.max(np.abs(acc - vol)) < 1e-15 + 1e-12 * np.max(np.abs(vol))


def test_closed_surface_double_layer_vanishes(orc):
    # sum over a closed outward mesh of int n.grad R dS = int_V lap R = 0;
    # and sum of int (y.n) R dS = (n+3) int_V R, with int_V R_0^0 = volume.
    v, t = W.icosphere(2)
    p = 6
    n_el = t.shape[1]
    centres = np.zeros((3, n_el))
    sig = np.ones(n_el)
    D = orc.moments("triangle", v, t, sig, p, leaf_off=np.array([0, n_el]), leaf_c=np.zeros((3, 1)),
                    layer=1, norm=1)[0]
    assert np.max(np.abs(D)) < 1e-13
    S = orc.moments("triangle", v, t, sig, p, leaf_off=None, leaf_c=centres, norm=1)
    X = v[:, t]
    cr = np.cross((X[:, 1] - X[:, 0]).T, (X[:, 2] - X[:, 0]).T).T
    nrm = cr / np.linalg.norm(cr, axis=0)
    h = np.sum(X[:, 0] * nrm, axis=0)
    vol = np.sum(h * S[:, 0]) / 3
    exact = abs(np.sum(np.einsum("ij,ij->j", np.cross(X[:, 0].T, X[:, 1].T).T, X[:, 2]))) / 6
    assert abs(vol - exact) < 1e-13


def test_leaf_sum_equals_element_sum(orc):
    v, t = W.random_triangles(50, seed=3, spread=0.3, size=0.05)
    p = 7
    off = np.array([0, 10, 10, 31, 50], dtype=np.int64)
    lc = rng.uniform(-0.2, 0.2, (3, 4))
    sig = rng.uniform(-1, 1, 50)
    leaves = orc.moments("triangle", v, t, sig, p, leaf_off=off, leaf_c=lc)
    per = orc.moments("triangle", v, t, sig, p, leaf_off=None,
                      leaf_c=np.repeat(lc, np.diff(off), axis=1))
    for L in range(4):
        exp = per[off[L]:off[L + 1]].sum(axis=0)
        assert np.max(np.abs(leaves[L] - exp)) < 1e-15
    # per-leaf degree: zero above leaf_p
    lp = np.array([7, 3, 0, 5], dtype=np.int32)
    got = orc.moments("triangle", v, t, sig, p, leaf_off=off, leaf_c=lc, leaf_p=lp)
    for L in range(4):
        npl = (lp[L] + 1) ** 2
        assert np.all(got[L, npl:] == 0)
        assert np.max(np.abs(got[L, :npl] - leaves[L, :npl])) < 1e-15


def test_norm_modes_agree(orc):
    # COEFF: F_n^m = (1/4pi)(-1)^n conj-symmetric image of MOMENT (int R_n^{-m} = (-1)^m conj int R_n^m)
    X = random_simplex("triangle")
    p = 6
    Fc = unpack(single(orc, "triangle", X, 0.5, np.zeros(3), p, norm=0), p)
    Fm = unpack(single(orc, "triangle", X, 0.5, np.zeros(3), p, norm=1), p)
    for (n, m), v in Fm.items():
        exp = (-1) ** n * (-1) ** m * np.conj(v) / (4 * math.pi)
        assert abs(Fc[(n, m)] - exp) < 1e-16 + 1e-13 * abs(v)
