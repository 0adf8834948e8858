"""GPU tests of q2x_nearfield (exact element potentials, the closed forms of
Sec. 4.1) against the near-field oracle (cone-fan quadrature of the Green's
function): random segments, triangles (single and double layer) and
tetrahedra at targets at moderate distance; collocation targets at the
centroids of the elements of a leaf against every element of that leaf (the
self-element term included); targets at vertices and in the plane of a
triangle; far targets against the expansion path (Q2X leaf coefficients
evaluated by q2x_evaluate); an element index out of range."""
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


def dense_lists(n_tgt, n_elem):
    return [range(n_elem)] * n_tgt


@pytest.mark.parametrize("kind,layer", [("segment", 0), ("triangle", 0), ("triangle", 1), ("tetra", 0)])
def test_nearfield_matches_oracle(q2x, orc, kind, layer):
    from oracle import nearfield as nf
    prob = random_problem(kind, [6], seed=21, p=4, size=0.1, spread=0.2)
    n = prob["idx"].shape[1]
    rng = np.random.default_rng(22)
    tgt = prob["leaf_c"][:, :1] + rng.normal(size=(3, 8)) * 0.8
    plan = q2x.Plan(4, precision="fp64")
    got = plan.nearfield(kind, T(prob["vxyz"]), T(prob["idx"]), T(prob["sigma"]), T(tgt), layer=layer).cpu().numpy()
    plan.sync()
    ref = nf.potentials(kind, prob["vxyz"], prob["idx"], prob["sigma"], tgt, dense_lists(8, n), layer=layer)
    assert np.max(np.abs(got - ref)) <= 1e-12 * np.max(np.abs(ref))


@pytest.mark.parametrize("kind", ["triangle", "tetra"])
def test_nearfield_collocation_self_leaf(q2x, orc, kind):
    """Targets at element centroids, each against every element of its leaf
    (CSR lists, ragged leaves, one empty)."""
    from oracle import nearfield as nf
    sizes = [7, 0, 12, 1, 5]
    prob = random_problem(kind, sizes, seed=25, p=4, size=0.1, spread=0.5)
    vx, idx = prob["vxyz"], prob["idx"]
    n = idx.shape[1]
    tgt = np.stack([vx[:, idx[k]] for k in range(idx.shape[0])]).mean(axis=0)
    off = prob["leaf_off"]
    lists = []
    for L in range(len(sizes)):
        lists += [range(off[L], off[L + 1])] * (off[L + 1] - off[L])
    tgt_off = np.concatenate([[0], np.cumsum([len(l) for l in lists])]).astype(np.int64)
    elem_idx = np.concatenate([np.asarray(l, dtype=np.int64) for l in lists])
    plan = q2x.Plan(4, precision="fp64")
    layers = (0, 1) if kind == "triangle" else (0,)
    for layer in layers:
        got = plan.nearfield(kind, T(vx), T(idx), T(prob["sigma"]), T(tgt), T(tgt_off), T(elem_idx),
                             layer=layer).cpu().numpy()
        plan.sync()
        ref = nf.potentials(kind, vx, idx, prob["sigma"], tgt, lists, layer=layer, nq=48)
        scale = np.max(np.abs(nf.potentials(kind, vx, idx, np.abs(prob["sigma"]), tgt, lists, nq=16)))
        assert got.shape == (n,)
        assert np.max(np.abs(got - ref)) <= 1e-11 * scale


def test_nearfield_targets_on_vertices_and_in_plane(q2x, orc):
    from oracle import nearfield as nf
    prob = random_problem("triangle", [1], seed=24, p=4, size=0.1, spread=0.2)
    vx, idx = prob["vxyz"], prob["idx"]
    X = vx[:, idx[:, 0]].T
    ctr = X.mean(axis=0)
    # the three vertices, and in-plane points outside the triangle (beyond each edge midpoint)
    pts = [X[k] for k in range(3)] + [ctr + 1.7 * ((X[k] + X[(k + 1) % 3]) / 2 - ctr) for k in range(3)]
    tgt = np.array(pts).T
    plan = q2x.Plan(4, precision="fp64")
    for layer in (0, 1):
        got = plan.nearfield("triangle", T(vx), T(idx), T(prob["sigma"]), T(tgt), layer=layer).cpu().numpy()
        plan.sync()
        ref = nf.potentials("triangle", vx, idx, prob["sigma"], tgt, dense_lists(6, 1), layer=layer, nq=64)
        assert np.all(np.isfinite(got))
        if layer == 0:
            assert np.max(np.abs(got - ref)) <= 1e-11 * np.max(np.abs(ref))
        else:  # in the plane, off the element's interior: the double layer vanishes
            assert np.max(np.abs(got)) <= 1e-14


@pytest.mark.parametrize("kind,layer", [("triangle", 0), ("triangle", 1), ("segment", 0), ("tetra", 0)])
def test_nearfield_equals_expansion_far_away(q2x, orc, kind, layer):
    from oracle import nearfield as nf
    p = 20
    prob = random_problem(kind, [25, 9], seed=23, p=p, size=0.05, spread=0.2)
    d = {k: T(v) for k, v in prob.items() if hasattr(v, "shape")}
    # a few leaf sizes away: the series has converged (ratio < 0.2 at p = 20) while the
    # closed forms still hold full accuracy (the tetrahedron's face sum cancels like
    # (distance / size), which is why the closed forms serve the near field only)
    tgt = np.array([[1.2, 0.5, -0.6], [-0.9, 1.0, 0.6]]).T
    plan = q2x.Plan(p, precision="fp64")
    if kind == "triangle":
        cs, cd = plan.triangles(d["vxyz"], d["idx"], d["sigma"], d["leaf_off"], d["leaf_c"], d["leaf_rho"], None,
                                single=True, double=True)
        c = cd if layer else cs
    elif kind == "segment":
        c = plan.segments(d["vxyz"], d["idx"], d["sigma"], d["leaf_off"], d["leaf_c"], d["leaf_rho"], None)
    else:
        c = plan.tetra(d["vxyz"], d["idx"], d["sigma"], d["leaf_off"], d["leaf_c"], d["leaf_rho"], None)
    far = plan.evaluate(c, d["leaf_c"], T(tgt)).cpu().numpy()
    near = plan.nearfield(kind, d["vxyz"], d["idx"], d["sigma"], T(tgt), layer=layer).cpu().numpy()
    plan.sync()
    # The densities carry signs, so the potential is a sum whose terms cancel;
    # both paths make errors of a few ulps of each element's term, so the
    # error is measured against the sum of the terms' magnitudes
    # sum_e |sigma_e phi_e(t)| (the oracle's, per element), not the sum itself.
    scale = 0.0
    for t in range(tgt.shape[1]):
        terms = [abs(prob["sigma"][e]) * abs(nf.element_potential(kind, prob["vxyz"][:, prob["idx"][:, e]].T,
                                                                   tgt[:, t], layer, nq=16))
                 for e in range(prob["idx"].shape[1])]
        scale = max(scale, float(np.sum(terms)))
    assert np.max(np.abs(far - near)) <= 1e-12 * scale


def test_nearfield_accumulate_and_bad_index(q2x):
    prob = random_problem("segment", [3], seed=26, p=4)
    d = {k: T(v) for k, v in prob.items() if hasattr(v, "shape")}
    tgt = T(np.array([[1.0, 1.0], [0.5, -0.5], [2.0, 0.0]]))
    plan = q2x.Plan(4, precision="fp64")
    one = plan.nearfield("segment", d["vxyz"], d["idx"], d["sigma"], tgt)
    two = plan.nearfield("segment", d["vxyz"], d["idx"], d["sigma"], tgt, out=one.clone(), accumulate=True)
    plan.sync()
    assert torch.allclose(two, 2 * one, rtol=1e-15, atol=0)
    off = torch.tensor([0, 2, 3], dtype=torch.int64, device="cuda")
    el = torch.tensor([0, 1, 9], dtype=torch.int64, device="cuda")
    out = plan.nearfield("segment", d["vxyz"], d["idx"], d["sigma"], tgt, off, el)
    with pytest.raises(q2x.Q2XError):
        plan.sync()
    assert out[1].item() == 0.0 and out[0].item() != 0.0
    with pytest.raises(q2x.Q2XError):
        plan.nearfield("segment", d["vxyz"], d["idx"], d["sigma"], tgt, layer=1)


def test_nearfield_empty_lists(q2x):
    """Targets with empty lists get 0 (or keep their value when accumulating);
    no targets and no elements are valid calls."""
    prob = random_problem("triangle", [4], seed=27, p=4)
    d = {k: T(v) for k, v in prob.items() if hasattr(v, "shape")}
    tgt = T(np.array([[1.0, 2.0, 3.0], [0.5, -0.5, 0.0], [2.0, 0.0, 1.0]]))
    plan = q2x.Plan(4, precision="fp64")
    off = torch.tensor([0, 0, 2, 2], dtype=torch.int64, device="cuda")
    el = torch.tensor([1, 3], dtype=torch.int64, device="cuda")
    got = plan.nearfield("triangle", d["vxyz"], d["idx"], d["sigma"], tgt, off, el)
    ref = plan.nearfield("triangle", d["vxyz"], d["idx"], d["sigma"], tgt[:, 1:2].contiguous(),
                         torch.tensor([0, 2], dtype=torch.int64, device="cuda"), el)
    base = torch.full((3,), 7.0, dtype=torch.float64, device="cuda")
    acc = plan.nearfield("triangle", d["vxyz"], d["idx"], d["sigma"], tgt, off, el, out=base.clone(),
                         accumulate=True)
    # every list empty: the index array may be empty (a NULL pointer)
    zero = torch.zeros(4, dtype=torch.int64, device="cuda")
    none = torch.empty(0, dtype=torch.int64, device="cuda")
    empty = plan.nearfield("triangle", d["vxyz"], d["idx"], d["sigma"], tgt, zero, none)
    no_tgt = plan.nearfield("triangle", d["vxyz"], d["idx"], d["sigma"], torch.empty((3, 0), dtype=torch.float64,
                                                                                     device="cuda"))
    plan.sync()
    assert got[0].item() == 0.0 and got[2].item() == 0.0 and got[1].item() == ref[0].item() != 0.0
    assert acc[0].item() == 7.0 and acc[2].item() == 7.0 and acc[1].item() == 7.0 + ref[0].item()
    assert torch.all(empty == 0) and no_tgt.numel() == 0
