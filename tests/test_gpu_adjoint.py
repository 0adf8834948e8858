"""GPU tests of the adjoint (q2x_triangles_single_vjp / TrianglesSingle):
d loss/d vertices and d loss/d densities for loss = sum(G * coef), checked
against complex-step derivatives of the FP64 oracle (exact to round-off),
central finite differences (h = 1e-6) of the GPU FP64 forward, and between
the FP32-mixed and FP64 paths."""
import numpy as np
import pytest

import workloads as W

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


@pytest.fixture(scope="module")
def prob():
    # 2,000-triangle subset of the perturbed level-8 sphere, depth-6 leaves, p = 12
    return W.cfg_sphere_adjoint(level=8, n_tri=2000, depth=6, p=12)


def dev(prob):
    from paper_2107_10942_gb300.q2x import problem_to_device
    return problem_to_device({k: v for k, v in prob.items() if k not in ("kind", "density", "layers", "name")})


def gpu_grad(q, prob, prec):
    d = dev(prob)
    plan = q.Plan(prob["p"], precision=prec)
    gv, gs = plan.triangles_single_vjp(d["vxyz"], d["idx"], d["sigma"], d["leaf_off"], d["leaf_c"], d["G"],
                                       d["leaf_rho"], d["leaf_p"])
    plan.sync()
    return gv.cpu().numpy(), gs.cpu().numpy()


def oracle_loss_cs(orc, prob, vre, vim, elems):
    """complex loss sum_e sum_c G[leaf(e)] F_c(e) over the given elements"""
    off = prob["leaf_off"]
    leaf_of = np.repeat(np.arange(off.shape[0] - 1), np.diff(off))
    idx = np.ascontiguousarray(prob["idx"][:, elems])
    ec = np.ascontiguousarray(prob["leaf_c"][:, leaf_of[elems]])
    F = orc.moments_cs("triangle", vre, vim, idx, prob["sigma"][elems], ec, prob["p"])
    return np.sum(F * prob["G"][leaf_of[elems]])


def test_vertex_gradient_vs_complex_step(q2x, orc, prob):
    gv, _ = gpu_grad(q2x, prob, "fp64")
    rng = np.random.default_rng(0)
    vre = prob["vxyz"]
    vim = np.zeros_like(vre)
    h = 1e-30
    scale = np.max(np.abs(gv))
    verts = rng.choice(np.unique(prob["idx"]), size=60, replace=False)
    for v in verts:
        elems = np.where(np.any(prob["idx"] == v, axis=0))[0]
        for d in range(3):
            vim[d, v] = h
            cs = oracle_loss_cs(orc, prob, vre, vim, elems).imag / h
            vim[d, v] = 0.0
            assert abs(gv[d, v] - cs) <= 1e-10 * scale, (v, d, gv[d, v], cs)


def test_sigma_gradient_exact(q2x, orc, prob):
    # loss is linear in each density: d loss/d sigma_e = sum_c G F_c(e) / sigma_e
    _, gs = gpu_grad(q2x, prob, "fp64")
    off = prob["leaf_off"]
    leaf_of = np.repeat(np.arange(off.shape[0] - 1), np.diff(off))
    ones = np.ones(prob["idx"].shape[1])
    F = orc.moments("triangle", prob["vxyz"], prob["idx"], ones, prob["p"], leaf_off=None,
                    leaf_c=np.ascontiguousarray(prob["leaf_c"][:, leaf_of]))
    ref = np.sum(F * prob["G"][leaf_of], axis=1)
    assert np.max(np.abs(gs - ref)) <= 1e-11 * np.max(np.abs(ref))


def test_central_differences_on_gpu_forward(q2x, prob):
    d = dev(prob)
    gv, _ = gpu_grad(q2x, prob, "fp64")
    plan = q2x.Plan(prob["p"], precision="fp64")
    G = d["G"]

    def loss(vx):
        c, _ = plan.triangles(vx, d["idx"], d["sigma"], d["leaf_off"], d["leaf_c"], d["leaf_rho"], d["leaf_p"])
        return float(torch.sum(c * G).item())

    rng = np.random.default_rng(1)
    h = 1e-6
    scale = np.max(np.abs(gv))
    for v in rng.choice(prob["vxyz"].shape[1], size=20, replace=False):
        for dd in range(3):
            xp = d["vxyz"].clone()
            xm = d["vxyz"].clone()
            xp[dd, v] += h
            xm[dd, v] -= h
            fd = (loss(xp) - loss(xm)) / (2 * h)
            assert abs(fd - gv[dd, v]) <= 1e-6 * scale, (v, dd, fd, gv[dd, v])


def test_fp32_adjoint_and_autograd(q2x, prob):
    d = dev(prob)
    gv64, gs64 = gpu_grad(q2x, prob, "fp64")
    plan = q2x.Plan(prob["p"], precision="fp32")
    vx = d["vxyz"].clone().requires_grad_(True)
    sg = d["sigma"].clone().requires_grad_(True)
    coef = q2x.q2x.triangles_single(vx, sg, plan, d["idx"], d["leaf_off"], d["leaf_c"], d["leaf_rho"], d["leaf_p"])
    loss = torch.sum(coef * d["G"])
    gv, gs = torch.autograd.grad(loss, (vx, sg))
    gv, gs = gv.cpu().numpy(), gs.cpu().numpy()
    assert np.max(np.abs(gv - gv64)) <= 2e-5 * np.max(np.abs(gv64))
    assert np.max(np.abs(gs - gs64)) <= 2e-5 * np.max(np.abs(gs64))


def test_high_degree_small_leaves(q2x, orc):
    """p = 20 on depth-8 leaves (leaf scale 2^-7): FP64 adjoint against the
    oracle's complex step, FP32-mixed against FP64."""
    prob = W.cfg_sphere_adjoint(level=8, n_tri=1500, depth=8, p=20)
    gv64, gs64 = gpu_grad(q2x, prob, "fp64")
    gv32, gs32 = gpu_grad(q2x, prob, "fp32")
    scale = np.max(np.abs(gv64))
    assert np.max(np.abs(gv32 - gv64)) <= 2e-5 * scale
    assert np.max(np.abs(gs32 - gs64)) <= 2e-5 * np.max(np.abs(gs64))
    rng = np.random.default_rng(2)
    vim = np.zeros_like(prob["vxyz"])
    h = 1e-30
    for v in rng.choice(np.unique(prob["idx"]), size=15, replace=False):
        elems = np.where(np.any(prob["idx"] == v, axis=0))[0]
        for d in range(3):
            vim[d, v] = h
            cs = oracle_loss_cs(orc, prob, prob["vxyz"], vim, elems).imag / h
            vim[d, v] = 0.0
            assert abs(gv64[d, v] - cs) <= 1e-10 * scale, (v, d, gv64[d, v], cs)
