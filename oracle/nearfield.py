"""FP64 CPU oracle for near-field element potentials -- TEST INFRASTRUCTURE ONLY.

Only ``tests/``, ``__graft_entry__.smoke()`` and ``bench.py`` may import this
module; the product path never does.

Computes the definition the closed forms of Sec. 4.1 evaluate,

    (1/4pi) int_e G(r, y) dmu(y),   G = 1/|r - y|           (single layer)
                                    G = n.(r - y)/|r - y|^3   (double layer,
                                                               triangles)

by Gauss-Legendre quadrature in coordinates centred on the target, where the
1/|r - y| singularity meets a Jacobian that cancels it:

* segment: the line is split at the foot of the perpendicular from r;
* triangle: the plane is fanned from r0, the projection of r, over the three
  edges, y = r0 + u (a - r0 + v (b - a)), Jacobian u ((a - r0) x (b - a)).n
  (signed: the fan pieces of a projection outside the triangle cancel where
  they overlap);
* tetrahedron: cone coordinates about r over the four outward faces,
  y = r + u (z - r), dV = u^2 ((z - r).n_F) dA_z du (signed likewise), the
  face integrals by the triangle fan.

Panels are graded geometrically toward each near-singular point -- the
target's projection (scale: its height h) and the foot on each edge (scale:
the distance to the edge's line) -- so targets close to an element converge
like distant ones.  A height at the rounding level of the coordinates (16
ulps of |r|_1 + |x1|_1) counts as zero: the target is taken in the plane,
where the double layer has its direct value 0.  None of the
closed forms of Sec. 4.1 is used here.

parity pins: ``tests/test_oracle_nearfield.py`` (textbook closed forms:
asinh antiderivative of a line, the polar integral of a triangle seen from a
vertex, the Van Oosterom-Strackee solid angle, Gauss's 4pi/0 law for closed
polyhedra, the potential of a cube at its centre; and agreement with the
independent multipole path of this oracle at moderate distance).
"""
from __future__ import annotations

import numpy as np

from . import gauss_legendre

INV_4PI = 1.0 / (4.0 * np.pi)


SNAP = 16.0 * np.finfo(np.float64).eps  # heights below 16 ulps of the coordinates count as zero


def _graded(lo, hi, at, delta, nq):
    """Composite Gauss-Legendre rule on [lo, hi] whose panels double in
    length away from the point ``at`` (lo <= at <= hi), the first ones of
    length ``delta``: it resolves an integrand whose nearest complex
    singularity lies about ``delta`` from ``at`` (delta <= 0: one panel per
    side)."""
    g, w = gauss_legendre(nq)
    nodes, weights = [], []
    for sgn, end in ((-1.0, lo), (1.0, hi)):
        span = abs(end - at)
        if span == 0.0:
            continue
        cuts = [0.0]
        step = delta if delta > 0.0 else span
        while cuts[-1] + step < span:
            cuts.append(cuts[-1] + step)
            step = cuts[-1]  # panels [x, 2x] after the first
        cuts.append(span)
        for c0, c1 in zip(cuts[:-1], cuts[1:]):
            nodes.append(at + sgn * (c0 + (c1 - c0) * g))
            weights.append((c1 - c0) * w)
    return np.concatenate(nodes), np.concatenate(weights)


def _segment(X, r, nq):
    a, b = X[0], X[1]
    L = np.linalg.norm(b - a)
    if L == 0.0:
        return 0.0
    l = (b - a) / L
    s0 = float(np.clip(np.dot(r - a, l), 0.0, L))  # foot of the perpendicular, clamped
    dist = np.linalg.norm(r - (a + np.dot(r - a, l) * l))
    s, ws = _graded(0.0, L, s0, dist, nq)
    y = a[None, :] + s[:, None] * l[None, :]
    return float(np.sum(ws / np.linalg.norm(r[None, :] - y, axis=1)))


def _plane_fan(X, r, f, nq):
    """int_T f(r, y, n) dA over the flat triangle X by the fan of three
    sub-triangles from r0, the projection of r onto the plane, each in
    collapsed coordinates y = r0 + u (a - r0 + v (b - a)), Jacobian
    u ((a - r0) x (b - a)).n; graded panels toward u = 0 (scale |h|) and
    toward the foot of r0 on the edge (scale: its distance to the edge's
    line).  Returns (integral, h, n)."""
    nr = np.cross(X[1] - X[0], X[2] - X[0])
    J = np.linalg.norm(nr)
    if J == 0.0:
        return 0.0, 0.0, None
    n = nr / J
    h = float(np.dot(n, r - X[0]))
    if abs(h) <= SNAP * (np.sum(np.abs(r)) + np.sum(np.abs(X[0]))):
        h = 0.0
    tot = 0.0
    for i in range(3):
        a, b = X[i], X[(i + 1) % 3]
        e = b - a
        A = (a - r) + h * n  # a - r0, r0 = r - h n the projection
        jac = float(np.dot(np.cross(A, e), n))
        if jac == 0.0:
            continue
        L = np.linalg.norm(e)
        vstar = float(np.clip(-np.dot(A, e) / (L * L), 0.0, 1.0))
        dline = abs(jac) / L  # distance from r0 to the edge's line
        v, wv = _graded(0.0, 1.0, vstar, dline / L, nq)
        qmax = max(np.linalg.norm(A), np.linalg.norm(A + e))
        u, wu = _graded(0.0, 1.0, 0.0, abs(h) / qmax, nq)
        U, V = np.meshgrid(u, v, indexing="ij")
        # r - y = h n - u (a - r0 + v (b - a)), formed relative to r so that
        # points closer to r than the coordinates' rounding stay distinct
        d = h * n - U[..., None] * (A + V[..., None] * e)
        tot += jac * np.sum(np.outer(wu, wv) * U * f(d, n))
    return tot, h, n


def _single(d, n):
    return 1.0 / np.linalg.norm(d, axis=-1)


def _double(d, n):
    return (d @ n) / np.linalg.norm(d, axis=-1) ** 3


def _cone(d, n):
    return -(d @ n) / np.linalg.norm(d, axis=-1)


def _triangle(X, r, layer, nq):
    v, h, _ = _plane_fan(X, r, _single if layer == 0 else _double, nq)
    if layer == 1 and h == 0.0:
        return 0.0  # n.(r - y) vanishes on the plane: the direct value
    return v


def _tetra(X, r, nq):
    """Cone coordinates about r: y = r + u (z - r), z on an outward face F,
    dV = u^2 ((z - r).n_F) dA du, 1/|y - r| = 1/(u |z - r|); the u integral
    of u is 1/2, the face integral goes to the triangle fan above."""
    c = X.mean(axis=0)
    tot = 0.0
    for f in ((1, 2, 3), (0, 3, 2), (0, 1, 3), (0, 2, 1)):
        F = X[list(f)]
        if np.dot(np.cross(F[1] - F[0], F[2] - F[0]), F[0] - c) < 0.0:  # outward orientation
            F = F[[0, 2, 1]]
        v, h, _ = _plane_fan(F, r, _cone, nq)
        tot += 0.5 * v
    return tot


def element_potential(kind, X, r, layer=0, nq=20):
    """(1/4pi) int_e G(r, y) dmu for one element with vertices X (rows) and
    the target r; kind "segment" | "triangle" | "tetra"; layer 1 (double
    layer) for triangles only."""
    X = np.asarray(X, dtype=np.float64)
    r = np.asarray(r, dtype=np.float64)
    if kind == "segment":
        v = _segment(X, r, nq)
    elif kind == "triangle":
        v = _triangle(X, r, layer, nq)
    elif kind == "tetra":
        v = _tetra(X, r, nq)
    else:
        raise ValueError(kind)
    if layer and kind != "triangle":
        raise ValueError("the double layer is defined for triangles")
    return INV_4PI * v


def potentials(kind, vxyz, idx, sigma, tgt, lists, layer=0, nq=20):
    """sum_e sigma_e element_potential(e, t) over lists[t] for every target
    column of tgt (3, n_tgt); lists: a sequence of element-index sequences."""
    out = np.zeros(tgt.shape[1])
    for t, elems in enumerate(lists):
        for e in elems:
            X = vxyz[:, idx[:, e]].T
            out[t] += sigma[e] * element_potential(kind, X, tgt[:, t], layer, nq)
    return out
