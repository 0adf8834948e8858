"""Far-field pins for the oracle (Sec. 4.1): the truncated series of Eq. (st4)
built from the oracle's coefficients converges to the layer potential.

References used: the closed-form segment integral of Eq. (num1)-(num3)
(re-derived: int dxi / sqrt(xi^2 - 4 zeta xi cos a + 4 zeta^2) is a log), brute
-force high-order quadrature of G = 1/(4 pi |r - y|) over the element (smooth
for distant r), the divergence-theorem reduction of the tetrahedron potential
to face potentials (Eq. (num7)-(num8)), and the error-bound shapes of
Eq. (num4) / (num6) at the paper's own fixture (Eq. (num0)-(num0.1)).

Reading of "p": the paper's truncation number counts degrees 0..p_paper-1;
this library's p is the maximum degree, so p_paper = p + 1.  The paper draws
its bound curves with C = 0.1 as contours in its (missing) figures; the pins
below check the RATE of Eq. (num4)/(num6) with C = 1, plus the rigorous
geometric majorant |1/|r-y| - sum_{n<=p}| <= (|y|/|r|)^(p+1) / (|r| - |y|)."""
import math
import os

import numpy as np
import pytest

HERE = os.path.dirname(os.path.abspath(__file__))


def fixture(kind, rt=0.1):
    rows = []
    with open(os.path.join(HERE, "golden", "accuracy_fixture.txt")) as f:
        for line in f:
            if line.strip() and not line.startswith("#"):
                parts = line.split()
                if parts[0] == kind:
                    rows.append([float(x) for x in parts[2:5]])
    rc = np.array([math.sqrt(3) / 2, 0.0, 0.0])
    return rc + rt * np.array(rows)


def eval_point(d):
    return d * np.array([math.sqrt(3) / 2, 0.0, 0.5])


def coef(orc, kind, X, p, layer=0, sig=1.0):
    vxyz = X.T.copy()
    idx = np.arange(X.shape[0], dtype=np.int32)[:, None]
    return orc.moments(kind, vxyz, idx, np.array([sig]), p, leaf_off=None,
                       leaf_c=np.zeros((3, 1)), layer=layer)[0]


def series(orc, c, p, r):
    re, im = orc.farfield(c, np.zeros(3), r, p)
    assert abs(im[0]) < 1e-14 * max(1.0, abs(re[0]))
    return re[0]


def K_num1(X, r):
    """Eq. (num1)-(num3): potential of a unit-density segment."""
    r0 = 0.5 * (X[0] + X[1])
    pv = X[1] - X[0]
    J = np.linalg.norm(pv)
    zeta = np.linalg.norm(r - r0) / J
    ca = np.dot(r - r0, pv) / (np.linalg.norm(r - r0) * J)
    num = math.sqrt(4 * zeta ** 2 - 4 * zeta * ca + 1) + 1 - 2 * zeta * ca
    den = math.sqrt(4 * zeta ** 2 + 4 * zeta * ca + 1) - 1 - 2 * zeta * ca
    return math.log(num / den) / (4 * math.pi)


def brute(orc, kind, X, r, layer=0, nq=40):
    """int G(r,y) dmu(y) (or int dG/dn_y) by a high-order collapsed Gauss rule."""
    g, w = orc.gauss_legendre(nq)
    tot = 0.0
    if kind == "segment":
        J = np.linalg.norm(X[1] - X[0])
        for u, wu in zip(g, w):
            y = X[0] + (X[1] - X[0]) * u
            tot += wu / np.linalg.norm(r - y)
        return tot * J / (4 * math.pi)
    if kind == "triangle":
        cr = np.cross(X[1] - X[0], X[2] - X[0])
        J = np.linalg.norm(cr)
        n = cr / J
        for s, ws in zip(g, w):
            for t, wt in zip(g, w):
                y = X[0] + (X[1] - X[0]) * s + (X[2] - X[0]) * (1 - s) * t
                d = r - y
                if layer == 0:
                    f = 1.0 / np.linalg.norm(d)
                else:  # d/dn_y 1/|r-y| = n.(r-y)/|r-y|^3
                    f = np.dot(n, d) / np.linalg.norm(d) ** 3
                tot += ws * wt * (1 - s) * f
        return tot * J / (4 * math.pi)
    raise ValueError(kind)


def test_segment_num1_matches_brute(orc):
    X = fixture("segment")
    r = eval_point(1.5)
    assert abs(K_num1(X, r) - brute(orc, "segment", X, r)) < 1e-15


@pytest.mark.parametrize("d", [1.0, 1.5, 2.5, 4.0])
def test_segment_series_rate_num4(orc, d):
    X = fixture("segment")
    r = eval_point(d)
    Kan = K_num1(X, r)
    q = np.linalg.norm(X.mean(0)) / d  # |r_c - r*| / d
    errs = []
    for p in range(0, 25):
        e = abs(series(orc, coef(orc, "segment", X, p), p, r) - Kan) / abs(Kan)
        errs.append(e)
        # Eq. (num4) with p_paper = p + 1 (floored at round-off)
        assert e <= 1.0 * q ** (p + 1) + 1e-14, (p, e)
        # rigorous majorant with a = max |y| over the segment
        a = np.max(np.linalg.norm(X, axis=1))
        J = np.linalg.norm(X[1] - X[0])
        assert e * abs(Kan) <= J * (a / d) ** (p + 1) / (4 * math.pi * (d - a)) + 1e-14 * abs(Kan)
    assert errs[-1] < 1e-13 or d < 4.0  # round-off level once q^(p+1) is negligible


@pytest.mark.parametrize("layer", [0, 1])
def test_triangle_series_rate(orc, layer):
    X = fixture("triangle")
    d = 1.5
    r = eval_point(d)
    ref = brute(orc, "triangle", X, r, layer=layer)
    q = np.linalg.norm(X.mean(0)) / d
    for p in range(1, 25):
        e = abs(series(orc, coef(orc, "triangle", X, p, layer=layer), p, r) - ref) / abs(ref)
        pp = p + 1
        bound = 1.0 * q ** pp if layer == 0 else 1.0 * pp * q ** (pp - 1)  # (num4) / (num6)
        assert e <= bound + 1e-13, (p, e, bound)


def test_tetra_num8_face_reduction(orc):
    # N(r) = -1/2 sum_j n_j.(r - r_cj) L_j(r), outward faces (Eq. (num8))
    X = fixture("tetra")
    if np.dot(np.cross(X[1] - X[0], X[2] - X[0]), X[3] - X[0]) < 0:
        X[[2, 3]] = X[[3, 2]]
    d = 1.5
    r = eval_point(d)
    faces = [(1, 2, 3), (0, 3, 2), (0, 1, 3), (0, 2, 1)]
    N = 0.0
    for f in faces:
        F = X[list(f)]
        nrm = np.cross(F[1] - F[0], F[2] - F[0])
        nrm /= np.linalg.norm(nrm)
        N += -0.5 * np.dot(nrm, r - F.mean(0)) * brute(orc, "triangle", F, r)
    q = np.linalg.norm(X.mean(0)) / d
    for p in range(0, 25):
        e = abs(series(orc, coef(orc, "tetra", X, p), p, r) - N) / abs(N)
        assert e <= 1.0 * q ** (p + 1) + 1e-13, (p, e)


def test_translation_consistency(orc):
    # expansions about two centres give the same far potential
    X = fixture("triangle")
    r = np.array([3.0, -2.0, 1.5])
    p = 22
    c1 = np.zeros(3)
    c2 = np.array([0.8, 0.1, -0.05])
    vxyz = X.T.copy()
    idx = np.arange(3, dtype=np.int32)[:, None]
    F1 = orc.moments("triangle", vxyz, idx, np.array([0.7]), p, leaf_c=c1.reshape(3, 1))[0]
    F2 = orc.moments("triangle", vxyz, idx, np.array([0.7]), p, leaf_c=c2.reshape(3, 1))[0]
    a = orc.farfield(F1, c1, r, p)[0][0]
    b = orc.farfield(F2, c2, r, p)[0][0]
    assert abs(a - b) < 1e-13 * abs(a)
