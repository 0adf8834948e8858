"""Full-size GPU parity on sampled outputs, in the launch configurations the
benchmark times:

  * the level-9 perturbed sphere (5,242,880 triangles, constant density,
    depth-7 octree, p = 16), FP64 and FP32-mixed, 16 sampled leaves;
  * the mixed ball (2M segments + 4M triangles + 1M tetrahedra, adaptive
    octree, p_leaf in 8..20) as one CUDA-graph batch, 8 sampled leaves;
  * the adjoint on 1M triangles of the level-8 sphere (p = 12): d loss/d sigma
    on sampled elements against the oracle's per-element moments, and
    d loss/d vertex on sampled vertices against complex-step derivatives of
    the oracle.

Every expected value comes from the FP64 oracle, leaf by leaf (or element by
element), on the same seeded inputs."""
import numpy as np
import pytest

import workloads as W
from _helpers import norm_err, oracle_coef

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

TOL = {"fp64": 1e-12, "fp32": 1e-5}


@pytest.fixture(scope="module")
def q2x():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2107_10942_gb300 import build
    build.build()
    import paper_2107_10942_gb300 as q
    return q


def to_dev(prob):
    from paper_2107_10942_gb300.q2x import problem_to_device
    return problem_to_device({k: v for k, v in prob.items() if hasattr(v, "shape")})


def leaf_sub(prob, L):
    off = prob["leaf_off"]
    e0, e1 = off[L], off[L + 1]
    sub = dict(prob)
    sub["idx"] = np.ascontiguousarray(prob["idx"][:, e0:e1])
    sub["sigma"] = prob["sigma"] if prob.get("density") == "linear" else prob["sigma"][e0:e1]
    sub["leaf_off"] = np.array([0, e1 - e0])
    sub["leaf_c"] = np.ascontiguousarray(prob["leaf_c"][:, L:L + 1])
    sub["leaf_p"] = prob["leaf_p"][L:L + 1]
    return sub


@pytest.fixture(scope="module")
def sphere_l9():
    return W.cfg_sphere_const(level=9, depth=7, p=16)


@pytest.mark.parametrize("prec", ["fp64", "fp32"])
def test_sphere_l9_p16_sampled(q2x, orc, sphere_l9, prec):
    prob = sphere_l9
    d = to_dev(prob)
    plan = q2x.Plan(16, precision=prec)
    cs, _ = plan.triangles(d["vxyz"], d["idx"], d["sigma"], d["leaf_off"], d["leaf_c"], d["leaf_rho"], None)
    plan.sync()
    assert plan.device_errors() == 0
    got = cs.cpu().numpy()
    nl = prob["leaf_c"].shape[1]
    sizes = np.diff(prob["leaf_off"])
    rng = np.random.default_rng(11)
    pick = list(rng.choice(np.nonzero(sizes)[0], size=14, replace=False)) + [int(np.argmax(sizes))]
    empty = np.nonzero(sizes == 0)[0]
    if len(empty):
        pick.append(int(empty[0]))
    for L in pick:
        ref = oracle_coef(orc, leaf_sub(prob, L), 0)
        assert norm_err(got[L:L + 1], ref, 16, prob["leaf_rho"][L:L + 1], 0) <= TOL[prec], L
    assert got.shape == (nl, 17 * 17)


@pytest.fixture(scope="module")
def mixed_ball():
    return W.cfg_mixed_ball()


@pytest.mark.parametrize("prec", ["fp32", "fp64"])
def test_mixed_ball_batch_sampled(q2x, orc, mixed_ball, prec):
    m = mixed_ball
    names = {"segment": "segments", "triangle": "triangles", "tetra": "tetra"}
    kinds = {names[k]: {key: torch.from_numpy(v).cuda() for key, v in dd.items()} for k, dd in m["kinds"].items()}
    plan = q2x.Plan(m["p"], precision=prec)
    b = q2x.q2x.Batch(plan, torch.from_numpy(m["leaf_c"]).cuda(), torch.from_numpy(m["leaf_rho"]).cuda(),
                      torch.from_numpy(m["leaf_p"]).cuda(), tile_elems=512, **kinds)
    got = b.run().cpu().numpy()
    plan.sync()
    assert plan.device_errors() == 0
    n_per_leaf = sum(np.diff(dd["leaf_off"]) for dd in m["kinds"].values())
    rng = np.random.default_rng(12)
    cand = np.nonzero((n_per_leaf >= 8) & (n_per_leaf <= 400))[0]
    pick = list(rng.choice(cand, size=6, replace=False))
    pick.append(int(np.argmin(n_per_leaf)))
    for L in pick:
        ref = 0
        for k, dd in m["kinds"].items():
            o = dd["leaf_off"]
            if o[L + 1] > o[L]:
                ref = ref + orc.moments(k, dd["vxyz"], np.ascontiguousarray(dd["idx"][:, o[L]:o[L + 1]]),
                                        dd["sigma"][o[L]:o[L + 1]], m["p"], leaf_off=np.array([0, o[L + 1] - o[L]]),
                                        leaf_c=np.ascontiguousarray(m["leaf_c"][:, L:L + 1]),
                                        leaf_p=m["leaf_p"][L:L + 1])
        assert norm_err(got[L:L + 1], ref, m["p"], m["leaf_rho"][L:L + 1], 0) <= TOL[prec], L
    # coefficients above each leaf's degree stay zero
    for L in rng.choice(len(n_per_leaf), size=200, replace=False):
        assert np.all(got[L, (m["leaf_p"][L] + 1) ** 2:] == 0)


@pytest.fixture(scope="module")
def adjoint_1m():
    return W.cfg_sphere_adjoint(level=8, n_tri=1_000_000, depth=6, p=12)


def test_adjoint_1m_sampled(q2x, orc, adjoint_1m):
    prob = adjoint_1m
    d = to_dev(prob)
    plan = q2x.Plan(12, precision="fp64")
    gv, gs = plan.triangles_single_vjp(d["vxyz"], d["idx"], d["sigma"], d["leaf_off"], d["leaf_c"], d["G"],
                                       d["leaf_rho"], None)
    plan.sync()
    assert plan.device_errors() == 0
    gv, gs = gv.cpu().numpy(), gs.cpu().numpy()
    off = prob["leaf_off"]
    leaf_of = np.repeat(np.arange(off.shape[0] - 1), np.diff(off))
    rng = np.random.default_rng(13)
    # d loss/d sigma_e = sum_c G[leaf(e)]_c F_c(e; sigma = 1)
    el = np.sort(rng.choice(prob["idx"].shape[1], size=300, replace=False))
    F = orc.moments("triangle", prob["vxyz"], np.ascontiguousarray(prob["idx"][:, el]), np.ones(len(el)), 12,
                    leaf_off=None, leaf_c=np.ascontiguousarray(prob["leaf_c"][:, leaf_of[el]]))
    ref = np.sum(F * prob["G"][leaf_of[el]], axis=1)
    assert np.max(np.abs(gs[el] - ref)) <= 1e-11 * np.max(np.abs(ref))
    # d loss/d x_v by complex step of the oracle over the triangles that use v
    scale = np.max(np.abs(gv))
    vim = np.zeros_like(prob["vxyz"])
    h = 1e-30
    for v in rng.choice(prob["vxyz"].shape[1], size=12, replace=False):
        elems = np.nonzero(np.any(prob["idx"] == v, axis=0))[0]
        idx = np.ascontiguousarray(prob["idx"][:, elems])
        ec = np.ascontiguousarray(prob["leaf_c"][:, leaf_of[elems]])
        for k in range(3):
            vim[k, v] = h
            Fc = orc.moments_cs("triangle", prob["vxyz"], vim, idx, prob["sigma"][elems], ec, 12)
            vim[k, v] = 0.0
            cs = np.sum(Fc * prob["G"][leaf_of[elems]]).imag / h
            assert abs(gv[k, v] - cs) <= 1e-10 * scale, (v, k, gv[k, v], cs)
