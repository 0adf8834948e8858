"""Pins of the oracle's direct potential (``oracle.potential``): the
single-layer potential (1/4pi) sum_e int_e sigma / |r - y| of a set of
elements at well-separated targets, by collapsed Gauss product rules.  It is
the reference for the far-field accuracy of the coefficients (the potential
that the expansion of Eq. (bas3) / Eq. (st4) approximates), so it is pinned
to things computed another way:

* a straight line: int ds / sqrt(d^2 + s^2) = asinh(s1/d) - asinh(s0/d);
* the unit cube seen from outside, against a tensor Gauss rule over the
  cube split into six tetrahedra (Kuhn) -- the oracle's tetrahedron rule on
  each, summed, equals the cube integral;
* the near-field oracle (graded fan quadrature, ``oracle.nearfield``, pinned
  to closed forms of its own) for triangles and tetrahedra a few sizes away;
* the multipole path: moments of Eq. (bas4) summed in the series of
  Eq. (bas3) at a distance where the truncation is below rounding, also for
  linear density.
"""
import numpy as np

from oracle import nearfield as nf

FOUR_PI = 4.0 * np.pi


def test_segment_asinh(orc):
    rng = np.random.default_rng(5)
    for _ in range(10):
        a, b = rng.normal(size=3), rng.normal(size=3)
        L = np.linalg.norm(b - a)
        l = (b - a) / L
        perp = np.cross(l, rng.normal(size=3))
        perp /= np.linalg.norm(perp)
        d = rng.uniform(1.5, 4.0) * L
        s_foot = rng.uniform(-0.5, 1.5) * L
        r = a + s_foot * l + d * perp
        exact = (np.arcsinh((L - s_foot) / d) - np.arcsinh(-s_foot / d)) / FOUR_PI
        vxyz = np.stack([a, b], axis=1)
        idx = np.array([[0], [1]], dtype=np.int32)
        got = orc.potential("segment", vxyz, idx, np.array([1.0]), r[None, :], nq=16)[0]
        assert abs(got - exact) <= 1e-14 * abs(exact)


def test_cube_from_six_tetrahedra(orc):
    # unit cube [0,1]^3 as the Kuhn split along the main diagonal
    corners = np.array([[i, j, k] for i in (0, 1) for j in (0, 1) for k in (0, 1)], dtype=float)
    cid = {tuple(c): n for n, c in enumerate(corners.astype(int))}
    tets = []
    import itertools
    for perm in itertools.permutations(range(3)):
        v = np.zeros(3, dtype=int)
        path = [cid[tuple(v)]]
        for ax in perm:
            v = v.copy()
            v[ax] = 1
            path.append(cid[tuple(v)])
        tets.append(path)
    idx = np.array(tets, dtype=np.int32).T.copy()
    vxyz = corners.T.copy()
    tgt = np.array([[2.5, 0.3, 0.4], [-1.7, 1.9, 0.5], [0.5, 0.5, 3.2]])
    got = orc.potential("tetra", vxyz, idx, np.ones(6), tgt, nq=14)
    g, w = orc.gauss_legendre(24)
    X, Y, Z = np.meshgrid(g, g, g, indexing="ij")
    W = w[:, None, None] * w[None, :, None] * w[None, None, :]
    for t, r in enumerate(tgt):
        ref = np.sum(W / np.sqrt((X - r[0]) ** 2 + (Y - r[1]) ** 2 + (Z - r[2]) ** 2)) / FOUR_PI
        assert abs(got[t] - ref) <= 1e-13 * abs(ref)


def test_against_graded_nearfield_oracle(orc):
    rng = np.random.default_rng(7)
    for kind, nv in (("triangle", 3), ("tetra", 4)):
        X = rng.normal(size=(nv, 3)) * 0.3
        if kind == "tetra" and np.linalg.det(X[1:] - X[0]) < 0:
            X[[2, 3]] = X[[3, 2]]
        size = max(np.linalg.norm(X[i] - X[j]) for i in range(nv) for j in range(nv))
        ctr = X.mean(axis=0)
        for dist in (3.0, 5.0, 10.0):
            u = rng.normal(size=3)
            r = ctr + dist * size * u / np.linalg.norm(u)
            ref = nf.element_potential(kind, X, r, nq=24)
            got = orc.potential(kind, X.T.copy(), np.arange(nv, dtype=np.int32)[:, None], np.array([1.0]),
                                r[None, :], nq=14)[0]
            # the graded oracle's cone sum over the four faces of a tetrahedron
            # cancels by about distance / size, so its own rounding grows so
            tol = 1e-13 if kind == "triangle" else 4e-14 * dist
            assert abs(got - ref) <= tol * abs(ref), (kind, dist, got, ref)


def test_against_multipole_series(orc):
    rng = np.random.default_rng(11)
    p = 30
    for kind, nv, density in (("triangle", 3, 0), ("triangle", 3, 1), ("tetra", 4, 0), ("segment", 2, 0)):
        n = 12
        X = [rng.normal(size=(3, n)) * 0.1 for _ in range(nv)]
        vxyz = np.concatenate(X, axis=1)
        idx = np.stack([np.arange(n) + k * n for k in range(nv)]).astype(np.int32)
        sigma = rng.uniform(-1, 1, size=vxyz.shape[1] if density else n)
        c = np.zeros((3, 1))
        rho = np.max(np.linalg.norm(vxyz, axis=0))
        coef = orc.moments(kind, vxyz, idx, sigma, p, leaf_off=np.array([0, n]), leaf_c=c, density=density)[0]
        dirs = rng.normal(size=(6, 3))
        tgt = 4.0 * rho * dirs / np.linalg.norm(dirs, axis=1, keepdims=True)
        ser, _ = orc.farfield(coef, c[:, 0], tgt, p)
        got = orc.potential(kind, vxyz, idx, sigma, tgt, density=density, nq=14)
        scale = np.max(np.abs(got))
        assert np.max(np.abs(got - ser)) <= 1e-13 * scale, (kind, density)
