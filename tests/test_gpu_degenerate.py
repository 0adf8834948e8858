"""Degenerate elements -- zero-length segments, triangles with a repeated
vertex or collinear vertices, flat tetrahedra -- have zero measure, so they
contribute exactly zero: a leaf that holds them next to ordinary elements
gets the coefficients of the ordinary elements alone (both precisions, both
layers), and the near-field potentials of degenerate elements are zero."""
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


def with_degenerates(kind, seed):
    """A two-leaf problem, then the same leaves with degenerate elements
    inserted among the ordinary ones (vertices appended)."""
    prob = random_problem(kind, [9, 14], seed=seed, p=8, size=0.05, spread=0.3)
    vx, idx, off = prob["vxyz"], prob["idx"], prob["leaf_off"]
    nv = idx.shape[0]
    n_vert = vx.shape[1]
    rng = np.random.default_rng(seed + 1)
    new_v, new_e, leaf_of_new = [], [], []
    for L in range(2):
        c = prob["leaf_c"][:, L]
        a = c + 0.03 * rng.standard_normal(3)
        b = c + 0.03 * rng.standard_normal(3)
        d = c + 0.03 * rng.standard_normal(3)
        base = n_vert + len(new_v)
        if kind == "segment":
            new_v += [a]
            new_e += [[base, base]]  # zero length
        elif kind == "triangle":
            new_v += [a, b, a + 0.37 * (b - a)]
            new_e += [[base, base, base + 1], [base, base + 1, base + 2]]  # repeated vertex; collinear
        else:
            mid = (a + b + d) / 3
            new_v += [a, b, d, mid]
            new_e += [[base, base + 1, base + 2, base + 3]]  # flat: the fourth vertex in the face's plane
        leaf_of_new += [L] * (1 if kind != "triangle" else 2)
    vx2 = np.concatenate([vx, np.array(new_v).T], axis=1)
    cols, sig, lof = [], [], []
    for L in range(2):
        ins = [e for e, l in zip(new_e, leaf_of_new) if l == L]
        mid = (off[L] + off[L + 1]) // 2
        block = [idx[:, e] for e in range(off[L], mid)] + [np.array(e) for e in ins] + \
                [idx[:, e] for e in range(mid, off[L + 1])]
        s = list(prob["sigma"][off[L]:mid]) + [1.7] * len(ins) + list(prob["sigma"][mid:off[L + 1]])
        cols += block
        sig += s
        lof += [L] * len(block)
    idx2 = np.stack(cols, axis=1).astype(np.int32)
    off2 = np.concatenate([[0], np.cumsum(np.bincount(lof, minlength=2))]).astype(np.int64)
    deg = dict(prob, vxyz=vx2, idx=np.ascontiguousarray(idx2[:nv]), sigma=np.array(sig), leaf_off=off2)
    return prob, deg


def coefs(q2x, prob, kind, prec):
    d = {k: T(v) for k, v in prob.items() if hasattr(v, "shape")}
    plan = q2x.Plan(8, precision=prec)
    if kind == "segment":
        out = [plan.segments(d["vxyz"], d["idx"], d["sigma"], d["leaf_off"], d["leaf_c"], d["leaf_rho"], None)]
    elif kind == "triangle":
        out = list(plan.triangles(d["vxyz"], d["idx"], d["sigma"], d["leaf_off"], d["leaf_c"], d["leaf_rho"],
                                  None, single=True, double=True))
    else:
        out = [plan.tetra(d["vxyz"], d["idx"], d["sigma"], d["leaf_off"], d["leaf_c"], d["leaf_rho"], None)]
    plan.sync()
    return [o.cpu().numpy() for o in out]


@pytest.mark.parametrize("prec", ["fp64", "fp32"])
@pytest.mark.parametrize("kind", ["segment", "triangle", "tetra"])
def test_degenerate_elements_contribute_zero(q2x, kind, prec):
    prob, deg = with_degenerates(kind, 51)
    ref = coefs(q2x, prob, kind, prec)
    got = coefs(q2x, deg, kind, prec)
    for a, b in zip(got, ref):
        assert np.max(np.abs(a - b)) <= (1e-14 if prec == "fp64" else 1e-6) * np.max(np.abs(b))


def test_degenerate_elements_in_the_near_field(q2x):
    for kind in ("segment", "triangle", "tetra"):
        prob, deg = with_degenerates(kind, 52)
        n0 = prob["idx"].shape[1]
        n1 = deg["idx"].shape[1]
        plan = q2x.Plan(4, precision="fp64")
        tgt = T(np.array([[0.7, -0.2, 0.4], [1.1, 0.9, -0.6]]).T)
        a = plan.nearfield(kind, T(prob["vxyz"]), T(prob["idx"]), T(prob["sigma"]), tgt)
        b = plan.nearfield(kind, T(deg["vxyz"]), T(deg["idx"]), T(deg["sigma"]), tgt)
        plan.sync()
        assert n1 > n0
        assert torch.allclose(a, b, rtol=1e-13, atol=0)
