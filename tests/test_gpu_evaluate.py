"""GPU tests of q2x_evaluate (the far-field M2P step): against the oracle's
series sum_{n,m} F_n^m S_n^m (whose convergence to the direct integral of
the Green's function the oracle tests pin), for random expansions, ragged
target lists and every degree bin; the MOMENT norm against the COEFF norm on
the same geometry; Q2X leaf coefficients evaluated at far targets."""
import numpy as np
import pytest

import workloads as W
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


@pytest.mark.parametrize("p", [0, 3, 12, 20])
def test_evaluate_matches_oracle_series(q2x, orc, p):
    rng = np.random.default_rng(31 + p)
    n_exp, n_tgt = 7, 40
    coef = rng.standard_normal((n_exp, (p + 1) ** 2)) * 0.3 ** np.repeat(np.arange(p + 1), 2 * np.arange(p + 1) + 1)
    exp_c = rng.uniform(-0.5, 0.5, (3, n_exp))
    tgt = rng.normal(size=(3, n_tgt))
    tgt = 3.0 * tgt / np.linalg.norm(tgt, axis=0)
    counts = rng.integers(0, 5, n_tgt)
    off = np.concatenate([[0], np.cumsum(counts)]).astype(np.int64)
    idx = rng.integers(0, n_exp, off[-1]).astype(np.int64)
    ref = np.zeros(n_tgt)
    for t in range(n_tgt):
        for e in idx[off[t]:off[t + 1]]:
            re, im = orc.farfield(coef[e], exp_c[:, e], tgt[:, t][None, :], p)
            ref[t] += re[0]
            assert abs(im[0]) <= 1e-12 * (abs(re[0]) + 1e-300) + 1e-300
    plan = q2x.Plan(p, precision="fp64")
    got = plan.evaluate(T(coef), T(exp_c), T(tgt), T(off), T(idx)).cpu().numpy()
    plan.sync()
    assert np.max(np.abs(got - ref)) <= 1e-12 * np.max(np.abs(ref))
    assert np.all(got[counts == 0] == 0)
    # dense default: every target, every expansion
    dense = plan.evaluate(T(coef), T(exp_c), T(tgt)).cpu().numpy()
    ref_d = np.zeros(n_tgt)
    for e in range(n_exp):
        ref_d += orc.farfield(coef[e], exp_c[:, e], tgt.T, p)[0]
    assert np.max(np.abs(dense - ref_d)) <= 1e-12 * np.max(np.abs(ref_d))


@pytest.mark.parametrize("kind,density", [("triangle", "linear"), ("tetra", "const"), ("segment", "const")])
def test_evaluate_q2x_leaves_both_norms(q2x, orc, kind, density):
    p = 10
    prob = random_problem(kind, [20, 3, 40], seed=5, p=p, size=0.05, spread=0.3, density=density)
    d = {k: T(v) for k, v in prob.items() if hasattr(v, "shape")}
    tgt = np.array([[2.5, -1.0, 0.3], [0.1, 3.0, -2.0], [-2.2, -2.2, 2.2]]).T
    vals = {}
    for norm in ("coeff", "moment"):
        plan = q2x.Plan(p, norm=norm, precision="fp64")
        if kind == "triangle":
            c, _ = plan.triangles(d["vxyz"], d["idx"], d["sigma"], d["leaf_off"], d["leaf_c"], d["leaf_rho"], None,
                                  density=density)
        elif kind == "tetra":
            c = plan.tetra(d["vxyz"], d["idx"], d["sigma"], d["leaf_off"], d["leaf_c"], d["leaf_rho"], None)
        else:
            c = plan.segments(d["vxyz"], d["idx"], d["sigma"], d["leaf_off"], d["leaf_c"], d["leaf_rho"], None)
        vals[norm] = plan.evaluate(c, d["leaf_c"], T(tgt)).cpu().numpy()
        plan.sync()
    dens = 1 if density == "linear" else 0
    F = orc.moments(kind, prob["vxyz"], prob["idx"], prob["sigma"], p, leaf_off=prob["leaf_off"],
                    leaf_c=prob["leaf_c"], density=dens)
    ref = sum(orc.farfield(F[L], prob["leaf_c"][:, L], tgt.T, p)[0] for L in range(F.shape[0]))
    assert np.max(np.abs(vals["coeff"] - ref)) <= 1e-12 * np.max(np.abs(ref))
    assert np.max(np.abs(vals["moment"] - ref)) <= 1e-12 * np.max(np.abs(ref))


def test_evaluate_flags_bad_index(q2x):
    plan = q2x.Plan(4, precision="fp64")
    coef = torch.ones((2, 25), dtype=torch.float64, device="cuda")
    c = torch.zeros((3, 2), dtype=torch.float64, device="cuda")
    tgt = torch.full((3, 2), 3.0, dtype=torch.float64, device="cuda")
    off = torch.tensor([0, 1, 2], dtype=torch.int64, device="cuda")
    idx = torch.tensor([1, 7], dtype=torch.int64, device="cuda")
    out = plan.evaluate(coef, c, tgt, off, idx)
    with pytest.raises(q2x.Q2XError):
        plan.sync()
    assert out[1].item() == 0.0 and out[0].item() != 0.0
