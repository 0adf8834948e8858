"""Pins of the oracle's expansion translation (oracle.translate), the M2M
step that consumes the Q2X leaf coefficients: the translated coefficients
must equal the coefficients computed directly about the new centre by
quadrature of the definition (Eq. (bas4)), for every element kind, both
layers and both norms; translation by zero is the identity; two translations
compose into one."""
import numpy as np
import pytest

from _helpers import norm_err, random_problem


def direct(orc, prob, centre, layer=0, norm=0):
    return orc.moments(prob["kind"], prob["vxyz"], prob["idx"], prob["sigma"], prob["p"],
                       leaf_off=np.array([0, prob["idx"].shape[1]]), leaf_c=centre.reshape(3, 1), layer=layer,
                       density=1 if prob["density"] == "linear" else 0, norm=norm)


@pytest.mark.parametrize("kind,density,layer", [("segment", "const", 0), ("triangle", "const", 0),
                                                ("triangle", "linear", 0), ("triangle", "const", 1),
                                                ("tetra", "const", 0)])
@pytest.mark.parametrize("norm", [0, 1])
def test_translate_equals_direct_quadrature(orc, kind, density, layer, norm):
    p = 10
    prob = random_problem(kind, [12], seed=3, p=p, size=0.05, spread=0.3, density=density)
    c_src = prob["leaf_c"][:, 0]
    c_dst = c_src + np.array([0.07, -0.05, 0.06])
    a = direct(orc, prob, c_src, layer, norm)
    b = direct(orc, prob, c_dst, layer, norm)
    moved = orc.translate(a, c_src.reshape(3, 1), c_dst.reshape(3, 1), p, norm=norm)
    # normalise with the radius about the new centre
    verts = prob["vxyz"][:, np.unique(prob["idx"])]
    rho = np.max(np.linalg.norm(verts - c_dst[:, None], axis=0))
    assert norm_err(moved, b, p, [rho], layer) <= 1e-12


def test_translate_identity_and_composition(orc):
    p = 12
    rng = np.random.default_rng(8)
    coef = rng.standard_normal((4, (p + 1) ** 2))
    c0 = rng.uniform(-1, 1, (3, 4))
    same = orc.translate(coef, c0, c0, p)
    assert np.array_equal(same, orc.pack_complex(orc.unpack_complex(coef, p), p))
    t1 = rng.uniform(-0.2, 0.2, (3, 4))
    t2 = rng.uniform(-0.2, 0.2, (3, 4))
    two = orc.translate(orc.translate(coef, c0, c0 + t1, p), c0 + t1, c0 + t1 + t2, p)
    one = orc.translate(coef, c0, c0 + t1 + t2, p)
    assert np.max(np.abs(two - one)) <= 1e-12 * np.max(np.abs(one))
    for norm in (0, 1):
        back = orc.translate(orc.translate(coef, c0, c0 + t1, p, norm=norm), c0 + t1, c0, p, norm=norm)
        assert np.max(np.abs(back - same)) <= 1e-12 * np.max(np.abs(same))


def test_translate_monopole_and_dipole_closed_form(orc):
    # a point charge q at y: F_n^m about c is q/(4pi) (-1)^n R_n^{-m}(y - c) (Eq. (bas3)),
    # so translating the single-degree-0 expansion about y to c must reproduce it
    p = 8
    y = np.array([0.3, -0.2, 0.45])
    c = np.array([-0.1, 0.25, 0.05])
    q = 1.7
    coef = np.zeros((1, (p + 1) ** 2))
    coef[0, 0] = q / (4 * np.pi)
    moved = orc.translate(coef, y.reshape(3, 1), c.reshape(3, 1), p)
    R = orc.rnm(y - c, p)
    F = np.zeros((p + 1) ** 2, dtype=complex)
    for n in range(p + 1):
        for m in range(-n, n + 1):
            F[n * n + n + m] = q / (4 * np.pi) * (-1) ** n * R[n * n + n - m]
    assert np.max(np.abs(moved[0] - orc.pack_complex(F[None], p)[0])) <= 1e-15 * q
