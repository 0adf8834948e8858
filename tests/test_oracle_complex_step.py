"""Pins for the oracle's complex-step moments (``oracle.moments_cs``).

The complex-step function is the derivative authority of the adjoint checks:
Im F(x + i h e_k) / h is the derivative dF/dx_k of the element moments with
respect to one vertex coordinate, exact to rounding for h = 1e-30.  It shares
its evaluator and quadrature with the real oracle only through the same
source text instantiated for complex numbers, so it is pinned here against
things that do not depend on that instantiation:

* its real part equals the real oracle (``oracle.moments``) on the same
  element, both at real vertices and at vertices moved by i h;
* its derivative equals a central difference of the real oracle, for every
  coordinate of every vertex, for segments, triangles with constant and
  linear density, and tetrahedra of both orientations.

The derivative rules behind this are those of Eq. (map4) (the Jacobian of the
element map, |det| for the tetrahedron) and Eqs. (bas5)-(bas7) (derivatives of
R_n^m); a dropped Jacobian term, a wrong sign of the tetrahedron's |det| on
the complex path or a wrong square-root branch changes the derivative by an
amount of the order of the derivative itself, far above the tolerances below.
"""
import numpy as np
import pytest

H_CS = 1e-30
H_FD = 1e-6

NV = {"segment": 2, "triangle": 3, "tetra": 4}


def _element(kind, seed, flip=False):
    rng = np.random.default_rng(seed)
    nv = NV[kind]
    X = 0.3 * rng.standard_normal((3, nv)) + rng.uniform(-0.5, 0.5, size=(3, 1))
    if kind == "tetra":
        d = np.linalg.det(np.stack([X[:, k] - X[:, 0] for k in (1, 2, 3)]))
        if (d < 0) != flip:
            X[:, [2, 3]] = X[:, [3, 2]]
    c = X.mean(axis=1, keepdims=True) + 0.05 * rng.standard_normal((3, 1))
    return np.ascontiguousarray(X), c


def _real(orc, kind, X, sigma, c, p, density, norm):
    idx = np.arange(X.shape[1], dtype=np.int32)[:, None]
    return orc.moments(kind, X, idx, sigma, p, leaf_off=None, leaf_c=c, density=density, norm=norm)[0]


def _cs(orc, kind, X, Xim, sigma, c, p, density, norm):
    idx = np.arange(X.shape[1], dtype=np.int32)[:, None]
    return orc.moments_cs(kind, X, Xim, idx, sigma, c, p, density=density, norm=norm)[0]


CASES = [("segment", 0, False), ("triangle", 0, False), ("triangle", 1, False), ("tetra", 0, False),
         ("tetra", 0, True)]


def _sigma(kind, density, nv, seed):
    rng = np.random.default_rng(seed + 1000)
    return rng.uniform(-1, 1, size=nv if density == 1 else 1)


@pytest.mark.parametrize("kind,density,flip", CASES)
@pytest.mark.parametrize("norm", [0, 1])
def test_real_part_equals_real_oracle(orc, kind, density, flip, norm):
    p = 7
    for seed in range(3):
        X, c = _element(kind, seed, flip)
        sig = _sigma(kind, density, X.shape[1], seed)
        ref = _real(orc, kind, X, sig, c, p, density, norm)
        scale = np.max(np.abs(ref))
        got = _cs(orc, kind, X, np.zeros_like(X), sig, c, p, density, norm)
        assert np.max(np.abs(got.real - ref)) <= 1e-15 * scale
        assert np.max(np.abs(got.imag)) == 0.0
        # a complex step in any coordinate leaves the real part unchanged to O(h^2)
        for v in range(X.shape[1]):
            for d in range(3):
                Xim = np.zeros_like(X)
                Xim[d, v] = H_CS
                got = _cs(orc, kind, X, Xim, sig, c, p, density, norm)
                assert np.max(np.abs(got.real - ref)) <= 1e-15 * scale


@pytest.mark.parametrize("kind,density,flip", CASES)
def test_derivative_equals_central_difference(orc, kind, density, flip):
    p = 8
    norm = 0
    for seed in range(2):
        X, c = _element(kind, seed + 10, flip)
        sig = _sigma(kind, density, X.shape[1], seed)
        for v in range(X.shape[1]):
            for d in range(3):
                Xim = np.zeros_like(X)
                Xim[d, v] = H_CS
                dcs = _cs(orc, kind, X, Xim, sig, c, p, density, norm).imag / H_CS
                Xp = X.copy()
                Xm = X.copy()
                Xp[d, v] += H_FD
                Xm[d, v] -= H_FD
                dfd = (_real(orc, kind, Xp, sig, c, p, density, norm)
                       - _real(orc, kind, Xm, sig, c, p, density, norm)) / (2 * H_FD)
                scale = max(np.max(np.abs(dcs)), 1e-300)
                err = np.max(np.abs(dcs - dfd)) / scale
                assert err < 1e-8, (kind, density, flip, v, d, err)


def test_planted_jacobian_sign_is_caught(orc):
    """The central-difference check separates the true derivative from the
    derivative of a moment whose Jacobian sign is wrong on one side: for a
    negatively oriented tetrahedron the moments use |det| = -det, and the
    derivative of +det differs from the true one by its whole size."""
    p = 4
    X, c = _element("tetra", 3, flip=True)
    sig = np.array([0.7])
    v, d = 1, 0
    Xim = np.zeros_like(X)
    Xim[d, v] = H_CS
    dcs = _cs(orc, "tetra", X, Xim, sig, c, p, 0, 0).imag / H_CS
    # a moment built on +det is the negative of the true one (flip the sign of
    # the whole element's contribution), so its derivative is -dcs
    planted = -dcs
    Xp = X.copy()
    Xm = X.copy()
    Xp[d, v] += H_FD
    Xm[d, v] -= H_FD
    dfd = (_real(orc, "tetra", Xp, sig, c, p, 0, 0) - _real(orc, "tetra", Xm, sig, c, p, 0, 0)) / (2 * H_FD)
    scale = np.max(np.abs(dcs))
    assert np.max(np.abs(dcs - dfd)) / scale < 1e-8
    assert np.max(np.abs(planted - dfd)) / scale > 0.5
