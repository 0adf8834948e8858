"""GPU tests of q2x_galerkin_triangles (receiver-side integration of local
expansions over triangles): against the oracle's per-element coefficients
contracted with random per-leaf weights (both norms, both layers, several
degree bins), and, with a MOMENT plan, the integral of a point charge's
local expansion over each triangle against direct quadrature of the Green's
function (and of its normal derivative for the double layer)."""
import numpy as np
import pytest

from _helpers import random_problem

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def q2x():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2107_10942_gb300 import build
    build.build()
    import paper_2107_10942_gb300 as q
    return q


def T(a):
    return torch.from_numpy(np.ascontiguousarray(a)).cuda()


@pytest.mark.parametrize("p", [4, 12, 20])
@pytest.mark.parametrize("norm", [0, 1])
@pytest.mark.parametrize("layer", [0, 1])
def test_galerkin_matches_oracle_contraction(q2x, orc, p, norm, layer):
    prob = random_problem("triangle", [5, 0, 40, 33, 1], seed=9 + p, p=p, size=0.05, spread=0.4)
    rng = np.random.default_rng(p)
    nl = prob["leaf_c"].shape[1]
    w = rng.standard_normal((nl, (p + 1) ** 2))
    leaf_of = np.repeat(np.arange(nl), np.diff(prob["leaf_off"]))
    P = orc.moments("triangle", prob["vxyz"], prob["idx"], prob["sigma"], p, leaf_off=None,
                    leaf_c=np.ascontiguousarray(prob["leaf_c"][:, leaf_of]), layer=layer, norm=norm)
    ref = np.sum(P * w[leaf_of], axis=1)
    plan = q2x.Plan(p, norm="coeff" if norm == 0 else "moment", precision="fp64")
    got = plan.galerkin_triangles(T(prob["vxyz"]), T(prob["idx"]), T(w), T(prob["leaf_off"]), T(prob["leaf_c"]),
                                  T(prob["leaf_rho"]), sigma=T(prob["sigma"]), layer=layer).cpu().numpy()
    plan.sync()
    scale = np.sum(np.abs(P * w[leaf_of]), axis=1)
    assert np.max(np.abs(got - ref) / scale) <= 1e-12


@pytest.mark.parametrize("layer", [0, 1])
def test_galerkin_point_charge_local_expansion(q2x, orc, layer):
    p = 16
    prob = random_problem("triangle", [30, 12], seed=4, p=p, size=0.06, spread=0.3)
    nl = prob["leaf_c"].shape[1]
    x0 = np.array([2.5, -1.8, 1.2])
    q = 1.3
    # phi(y) = q / (4 pi |y - x0|) = sum L_n^m R_n^m(y - c),
    # L_n^m = q/(4pi) (-1)^n S_n^{-m}(x0 - c)   (Eq. (bas3))
    L_re = np.zeros((nl, (p + 1) ** 2))
    L_im = np.zeros_like(L_re)
    for Lf in range(nl):
        S = orc.snm(x0 - prob["leaf_c"][:, Lf], p)
        for n in range(p + 1):
            for m in range(n + 1):
                v = q / (4 * np.pi) * (-1) ** n * S[n * n + n - m]
                L_re[Lf, n * n + n + m] = v.real
                L_im[Lf, n * n + n + m] = v.imag
    from paper_2107_10942_gb300.q2x import local_expansion_weights
    w = local_expansion_weights(T(L_re), T(L_im), p)
    plan = q2x.Plan(p, norm="moment", precision="fp64")
    ones = torch.ones(prob["idx"].shape[1], dtype=torch.float64, device="cuda")
    got = plan.galerkin_triangles(T(prob["vxyz"]), T(prob["idx"]), w, T(prob["leaf_off"]), T(prob["leaf_c"]),
                                  T(prob["leaf_rho"]), sigma=ones, layer=layer).cpu().numpy()
    plan.sync()
    # direct quadrature over each triangle (collapsed Gauss, 12 x 12 points)
    xg, wg = orc.gauss_legendre(12)
    ref = np.zeros(prob["idx"].shape[1])
    for e in range(prob["idx"].shape[1]):
        X = prob["vxyz"][:, prob["idx"][:, e]]
        eu, ev = X[:, 1] - X[:, 0], X[:, 2] - X[:, 0]
        nrm = np.cross(eu, ev)
        J = np.linalg.norm(nrm)
        nu = nrm / J
        acc = 0.0
        for i, s in enumerate(xg):
            for j, t in enumerate(xg):
                u, v = s, (1 - s) * t
                y = X[:, 0] + u * eu + v * ev
                dvec = y - x0
                r = np.linalg.norm(dvec)
                f = 1.0 / (4 * np.pi * r) if layer == 0 else -np.dot(nu, dvec) / (4 * np.pi * r ** 3)
                acc += wg[i] * wg[j] * (1 - s) * f
        ref[e] = q * J * acc
    assert np.max(np.abs(got - ref)) <= 1e-9 * np.max(np.abs(ref))
