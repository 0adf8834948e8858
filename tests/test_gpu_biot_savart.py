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


@pytest.mark.parametrize("prec", ["fp64", "fp32"])
def test_vector_chunked_and_per_component_agree(q2x, prec):
    """The fused pass (one recursion, weighted reduce) against one scalar
    segment pass per component; leaf degrees, an empty leaf, no leaf scales
    and accumulation included."""
    p = 10
    prob = random_problem("segment", [23, 0, 9, 40, 1], seed=15, p=p, size=0.05, spread=0.3,
                          leaf_p=[10, 4, 7, 10, 0])
    rng = np.random.default_rng(16)
    cur = rng.uniform(-1, 1, (3, prob["idx"].shape[1]))
    d = {k: T(v) for k, v in prob.items() if hasattr(v, "shape")}
    plan = q2x.Plan(p, precision=prec)
    one = plan.segments_vector(d["vxyz"], d["idx"], T(cur), d["leaf_off"], d["leaf_c"], d["leaf_rho"], d["leaf_p"])
    # without leaf scales (computed internally for FP32, unit scale for FP64) and accumulating
    acc = plan.segments_vector(d["vxyz"], d["idx"], T(cur), d["leaf_off"], d["leaf_c"], None, d["leaf_p"],
                               coef3=one.clone(), accumulate=True)
    ref = torch.stack([plan.segments(d["vxyz"], d["idx"], T(cur[k]), d["leaf_off"], d["leaf_c"], d["leaf_rho"],
                                     d["leaf_p"]) for k in range(3)])
    plan.sync()
    scale = ref.abs().max().item()
    tol = 1e-13 if prec == "fp64" else 1e-6
    assert (one - ref).abs().max().item() <= tol * scale
    assert (acc - 2 * ref).abs().max().item() <= 2 * tol * scale
    assert torch.all(one[:, 1] == 0)  # the empty leaf
    for L, pl in enumerate([10, 4, 7, 10, 0]):  # moments above each leaf's degree are zero
        assert torch.all(one[:, L, (pl + 1) ** 2:] == 0)


def test_leaf_reduce_weighted(q2x):
    rng = np.random.default_rng(17)
    p = 5
    sizes = [0, 5, 1, 300, 0, 17]
    import workloads as W
    off = W.csr_from_leaf_of(np.repeat(np.arange(len(sizes)), sizes), len(sizes))
    n = int(off[-1])
    elem = rng.standard_normal((n, 36))
    w = rng.standard_normal((4, n))
    plan = q2x.Plan(p)
    for nw in (1, 2, 3, 4):
        got = plan.leaf_reduce_weighted(T(elem), p, T(off), T(w[:nw])).cpu().numpy()
        acc0 = torch.full((nw, len(sizes), 36), 2.0, dtype=torch.float64, device="cuda")
        acc = plan.leaf_reduce_weighted(T(elem), p, T(off), T(w[:nw]), coef=acc0, accumulate=True).cpu().numpy()
        plan.sync()
        for j in range(nw):
            for L in range(len(sizes)):
                ref = np.zeros(36)
                for e in range(off[L], off[L + 1]):
                    ref = ref + w[j, e] * elem[e]
                assert np.max(np.abs(got[j, L] - ref)) <= 1e-13 * max(1.0, np.max(np.abs(ref)))
        assert np.array_equal(acc, got + 2.0)
    with pytest.raises(ValueError):  # at most four weight rows
        plan.leaf_reduce_weighted(T(elem), p, T(off), T(np.zeros((5, n))))


def test_vector_nonfinite_component_contributes_zero(q2x):
    """A non-finite current component sets the device error word's
    non-finite bit and its segment contributes zero to all three
    components; the other segments are unaffected."""
    p = 8
    prob, cur = filament_problem(p)
    bad = cur.copy()
    bad[1, 5] = np.nan
    zeroed = cur.copy()
    zeroed[:, 5] = 0.0
    plan = q2x.Plan(p, precision="fp64")
    args = (T(prob["vxyz"]), T(prob["idx"]))
    leaf = (T(prob["leaf_off"]), T(prob["leaf_c"]), T(prob["leaf_rho"]))
    ref = plan.segments_vector(*args, T(zeroed), *leaf)
    plan.sync()
    got = plan.segments_vector(*args, T(bad), *leaf)
    assert plan.device_errors() & 2
    assert torch.equal(got, ref)
