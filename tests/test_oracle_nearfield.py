"""Pins of the near-field oracle (oracle.nearfield): the cone-fan quadrature
of (1/4pi) int_e G against closed forms that come from elsewhere --

* a straight line: int ds / sqrt(d^2 + s^2) = asinh(s1/d) - asinh(s0/d);
* a triangle seen from its own vertex A: in polar coordinates about A the
  radial integral is the distance to the opposite edge, which gives
  d (asinh(s_C/d) - asinh(s_B/d)), d the distance from A to the line BC and
  s_B, s_C the coordinates of B and C along BC from the foot of A;
* the solid angle of a triangle (Van Oosterom & Strackee, IEEE TBME 1983):
  tan(Omega/2) = det[R1 R2 R3] / (R1R2R3 + (R1.R2)R3 + (R1.R3)R2 + (R2.R3)R1);
* Gauss's law for a closed polyhedron with outward normals: the double layer
  of unit density, (1/4pi) int n.(r - y)/|r - y|^3, is -1 inside and 0
  outside;
* the potential of the unit cube at its centre: int dV/|y| over
  [-1/2, 1/2]^3 = 3 ln(2 + sqrt 3) - pi/2, and tensor Gauss quadrature of the
  cube at an outside point;
* the multipole path of the oracle (moments of Eq. (bas4) + the far-field
  series of Eq. (bas5)) at targets a few element sizes away.
"""
import itertools

import numpy as np
import pytest

from oracle import nearfield as nf

FOUR_PI = 4.0 * np.pi


def test_segment_asinh(orc):
    rng = np.random.default_rng(1)
    for _ in range(20):
        a, b = rng.normal(size=3), rng.normal(size=3)
        L = np.linalg.norm(b - a)
        l = (b - a) / L
        perp = np.cross(l, rng.normal(size=3))
        perp /= np.linalg.norm(perp)
        d = rng.uniform(0.3, 2.0) * L
        s_foot = rng.uniform(-0.5, 1.5) * L  # foot inside or outside the segment
        r = a + s_foot * l + d * perp
        ref = np.arcsinh((L - s_foot) / d) - np.arcsinh((0.0 - s_foot) / d)
        got = FOUR_PI * nf.element_potential("segment", np.array([a, b]), r)
        assert abs(got - ref) <= 1e-13 * abs(ref)


def test_triangle_from_vertex(orc):
    rng = np.random.default_rng(2)
    for _ in range(20):
        X = rng.normal(size=(3, 3))
        for k in range(3):
            A, B, C = X[k], X[(k + 1) % 3], X[(k + 2) % 3]
            l = (C - B) / np.linalg.norm(C - B)
            F = B + np.dot(A - B, l) * l
            d = np.linalg.norm(A - F)
            sB, sC = np.dot(B - F, l), np.dot(C - F, l)
            ref = d * (np.arcsinh(sC / d) - np.arcsinh(sB / d))
            got = FOUR_PI * nf.element_potential("triangle", X, A, nq=64)
            assert abs(got - ref) <= 1e-12 * abs(ref)


def _vos(X, r):
    R1, R2, R3 = X[0] - r, X[1] - r, X[2] - r
    n1, n2, n3 = np.linalg.norm(R1), np.linalg.norm(R2), np.linalg.norm(R3)
    num = np.dot(R1, np.cross(R2, R3))
    den = n1 * n2 * n3 + np.dot(R1, R2) * n3 + np.dot(R1, R3) * n2 + np.dot(R2, R3) * n1
    return 2.0 * np.arctan2(num, den)


def test_double_layer_solid_angle(orc):
    rng = np.random.default_rng(3)
    for _ in range(30):
        X = rng.normal(size=(3, 3))
        nrm = np.cross(X[1] - X[0], X[2] - X[0])
        nrm /= np.linalg.norm(nrm)
        r = X.mean(axis=0) + rng.normal(size=3) + rng.choice([-1, 1]) * rng.uniform(0.5, 2.0) * nrm
        # n.(r - y)/|r - y|^3 integrates to minus the signed solid angle of
        # (X1, X2, X3) seen from r
        ref = -_vos(X, r)
        got = FOUR_PI * nf.element_potential("triangle", X, r, layer=1, nq=48)
        assert abs(got - ref) <= 1e-10 * max(abs(ref), 1e-2)


def _octahedron(rng):
    V = np.array([[1, 0, 0], [-1, 0, 0], [0, 1, 0], [0, -1, 0], [0, 0, 1], [0, 0, -1]], float)
    V = V * rng.uniform(0.8, 1.2, size=(6, 1))
    faces = []
    for sx, sy, sz in itertools.product((0, 1), (2, 3), (4, 5)):
        f = [sx, sy, sz]
        c = V[f].mean(axis=0)
        if np.dot(np.cross(V[f[1]] - V[f[0]], V[f[2]] - V[f[0]]), c) < 0:  # outward
            f = [sx, sz, sy]
        faces.append(f)
    return V, faces


def test_double_layer_gauss_law(orc):
    rng = np.random.default_rng(4)
    V, faces = _octahedron(rng)
    for r, want in ((np.array([0.1, -0.05, 0.2]), -1.0), (np.array([0.0, 0.0, 0.0]), -1.0),
                    (np.array([1.5, 0.4, -0.3]), 0.0), (np.array([-0.2, 2.0, 1.0]), 0.0)):
        # outward normals: n.(r - y) < 0 seen from inside
        got = sum(nf.element_potential("triangle", V[f], r, layer=1, nq=48) for f in faces)
        assert abs(got - want) <= 1e-10


def _cube_tets():
    tets = []
    for perm in itertools.permutations(range(3)):
        cur = np.zeros(3)
        v = [cur.copy()]
        for ax in perm:
            cur = cur.copy()
            cur[ax] = 1.0
            v.append(cur)
        tets.append(np.array(v) - 0.5)
    return tets


def test_cube_centre_closed_form(orc):
    got = sum(FOUR_PI * nf.element_potential("tetra", T, np.zeros(3)) for T in _cube_tets())
    assert abs(got - (3 * np.log(2 + np.sqrt(3)) - np.pi / 2)) <= 1e-13


def test_cube_outside_tensor_quadrature(orc):
    g, w = orc.gauss_legendre(40)
    x = g - 0.5
    Xg, Yg, Zg = np.meshgrid(x, x, x, indexing="ij")
    Wg = w[:, None, None] * w[None, :, None] * w[None, None, :]
    for r in (np.array([0.9, 0.3, -0.7]), np.array([-1.4, 0.0, 0.2])):
        ref = np.sum(Wg / np.sqrt((Xg - r[0]) ** 2 + (Yg - r[1]) ** 2 + (Zg - r[2]) ** 2))
        got = sum(FOUR_PI * nf.element_potential("tetra", T, r, nq=24) for T in _cube_tets())
        assert abs(got - ref) <= 1e-13 * ref


@pytest.mark.parametrize("kind,layer", [("segment", 0), ("triangle", 0), ("triangle", 1), ("tetra", 0)])
def test_matches_multipole_path(orc, kind, layer):
    rng = np.random.default_rng(5)
    nv = {"segment": 2, "triangle": 3, "tetra": 4}[kind]
    X = 0.3 * rng.normal(size=(nv, 3))
    c = X.mean(axis=0)
    p = 30
    F = orc.moments(kind, X.T.copy(), np.arange(nv, dtype=np.int32)[:, None], np.ones(1), p, leaf_c=c[:, None],
                    layer=layer)
    for _ in range(5):
        u = rng.normal(size=3)
        r = c + 2.0 * u / np.linalg.norm(u)
        ref = orc.farfield(F[0], c, r[None, :], p)[0][0]
        got = nf.element_potential(kind, X, r, layer=layer)
        assert abs(got - ref) <= 1e-12 * abs(ref)
