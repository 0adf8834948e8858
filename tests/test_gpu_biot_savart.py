"""GPU tests of the vector line densities of Eq. (st3): three-component
segment coefficients (Plan.segments_vector) against the oracle, and the
Biot-Savart field H = curl A evaluated from them (q2x_evaluate_curl) against
direct quadrature of (1/4pi) int I x (r - r')/|r - r'|^3 dl over the
segments."""
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


def filament_problem(p):
    prob = random_problem("segment", [60, 7, 33], seed=13, p=p, size=0.05, spread=0.3)
    rng = np.random.default_rng(14)
    current = rng.uniform(-1, 1, (3, prob["idx"].shape[1]))
    return prob, current


def test_vector_coefficients_match_oracle(q2x, orc):
    p = 12
    prob, cur = filament_problem(p)
    plan = q2x.Plan(p, precision="fp64")
    c3 = plan.segments_vector(T(prob["vxyz"]), T(prob["idx"]), T(cur), T(prob["leaf_off"]), T(prob["leaf_c"]),
                              T(prob["leaf_rho"])).cpu().numpy()
    plan.sync()
    for k in range(3):
        ref = orc.moments("segment", prob["vxyz"], prob["idx"], cur[k], p, leaf_off=prob["leaf_off"],
                          leaf_c=prob["leaf_c"])
        assert np.max(np.abs(c3[k] - ref)) <= 1e-12 * np.max(np.abs(ref))


@pytest.mark.parametrize("p", [8, 16])
def test_biot_savart_field_against_quadrature(q2x, orc, p):
    prob, cur = filament_problem(p)
    plan = q2x.Plan(p, precision="fp64")
    c3 = plan.segments_vector(T(prob["vxyz"]), T(prob["idx"]), T(cur), T(prob["leaf_off"]), T(prob["leaf_c"]),
                              T(prob["leaf_rho"]))
    rng = np.random.default_rng(15)
    tgt = rng.normal(size=(3, 25))
    tgt = 2.5 * tgt / np.linalg.norm(tgt, axis=0)
    H = plan.evaluate_curl(c3, T(prob["leaf_c"]), T(tgt)).cpu().numpy()
    plan.sync()
    xg, wg = orc.gauss_legendre(12)
    ref = np.zeros((3, tgt.shape[1]))
    for e in range(prob["idx"].shape[1]):
        a, b = prob["vxyz"][:, prob["idx"][0, e]], prob["vxyz"][:, prob["idx"][1, e]]
        ln = np.linalg.norm(b - a)
        for s, w in zip(xg, wg):
            y = a + s * (b - a)
            d = tgt - y[:, None]
            r3 = np.linalg.norm(d, axis=0) ** 3
            ref += w * ln * np.cross(cur[:, e], d.T).T / (4 * np.pi * r3)
    tol = 1e-9 if p == 16 else 1e-5
    assert np.max(np.abs(H - ref)) <= tol * np.max(np.abs(ref))


def test_curl_needs_coeff_norm(q2x):
    plan = q2x.Plan(4, norm="moment", precision="fp64")
    c3 = torch.zeros((3, 1, 25), dtype=torch.float64, device="cuda")
    with pytest.raises(q2x.Q2XError) as ei:
        plan.evaluate_curl(c3, torch.zeros((3, 1), dtype=torch.float64, device="cuda"),
                           torch.ones((3, 2), dtype=torch.float64, device="cuda"))
    assert ei.value.status == 7
