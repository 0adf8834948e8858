"""GPU tests of q2x_translate (the M2M step fed by the Q2X leaf coefficients)
and of the octree upward pass built on it: against the oracle's translation
on random expansions (ragged source counts, every degree bin, both norms),
and, end to end, the root and mid-level coefficients of an upward pass
against the oracle's quadrature about those centres."""
import numpy as np
import pytest

import workloads as W
from _helpers import norm_err

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


def oracle_translate_sum(orc, coef, src_c, off, dst_c, p, norm):
    out = np.zeros((len(off) - 1, (p + 1) ** 2))
    for d in range(len(off) - 1):
        s0, s1 = off[d], off[d + 1]
        if s1 > s0:
            moved = orc.translate(coef[s0:s1], src_c[:, s0:s1], np.repeat(dst_c[:, d:d + 1], s1 - s0, axis=1), p,
                                  norm=norm)
            for r in moved:  # in source order, like the kernel
                out[d] += r
    return out


@pytest.mark.parametrize("p", [0, 1, 5, 12, 20])
@pytest.mark.parametrize("norm", ["coeff", "moment"])
def test_translate_matches_oracle(q2x, orc, p, norm):
    rng = np.random.default_rng(p + 7)
    counts = np.array([0, 1, 8, 3, 0, 9, 2, 8, 1, 5, 4, 8, 0, 7, 6, 1, 2, 33])
    off = np.concatenate([[0], np.cumsum(counts)]).astype(np.int64)
    n_src, n_dst = int(off[-1]), len(counts)
    dst_c = rng.uniform(-1, 1, (3, n_dst))
    src_c = np.repeat(dst_c, counts, axis=1) + rng.uniform(-0.2, 0.2, (3, n_src))
    coef = rng.standard_normal((n_src, (p + 1) ** 2))
    nrm = 0 if norm == "coeff" else 1
    ref = oracle_translate_sum(orc, coef, src_c, off, dst_c, p, nrm)
    plan = q2x.Plan(p, norm=norm, precision="fp64")
    T = lambda a: torch.from_numpy(np.ascontiguousarray(a)).cuda()
    got = plan.translate(T(coef), T(src_c), T(off), T(dst_c)).cpu().numpy()
    plan.sync()
    scale = np.max(np.abs(ref), axis=1, keepdims=True)
    scale[scale == 0] = 1.0
    assert np.max(np.abs(got - ref) / scale) <= 1e-13
    assert np.all(got[counts == 0] == 0)
    # accumulate adds in place
    base = rng.standard_normal(ref.shape)
    acc = T(base.copy())
    plan.translate(T(coef), T(src_c), T(off), T(dst_c), dst_coef=acc, accumulate=True)
    plan.sync()
    assert np.max(np.abs(acc.cpu().numpy() - (base + got))) <= 1e-13 * np.max(np.abs(base + got))


def test_translate_bad_offsets_flagged(q2x):
    plan = q2x.Plan(4, precision="fp64")
    coef = torch.ones((3, 25), dtype=torch.float64, device="cuda")
    c = torch.zeros((3, 3), dtype=torch.float64, device="cuda")
    off = torch.tensor([0, 2, 9], dtype=torch.int64, device="cuda")  # beyond n_src
    dc = torch.zeros((3, 2), dtype=torch.float64, device="cuda")
    out = plan.translate(coef, c, off, dc)
    with pytest.raises(q2x.Q2XError):
        plan.sync()
    assert torch.all(out[1] == 0)
    coef5 = torch.ones((3, 36), dtype=torch.float64, device="cuda")
    with pytest.raises(q2x.Q2XError) as ei:
        plan.translate(coef5, c, off, dc, p=5)  # above the plan's p_max
    assert ei.value.status == 2


@pytest.mark.parametrize("prec", ["fp64", "fp32"])
def test_upward_pass_against_quadrature(q2x, orc, prec):
    """Level-4 perturbed sphere, linear density, depth-3 leaves, p = 10: Q2X at
    the leaves then the upward pass; the root (about the cube centre) and two
    level-1 boxes are checked against the oracle's quadrature about those
    centres over all the triangles they contain."""
    from paper_2107_10942_gb300.q2x import problem_to_device
    from paper_2107_10942_gb300.upward import Upward
    p, depth, lo, size = 10, 3, -1.125, 2.25
    prob = W.cfg_sphere_linear(level=4, depth=depth, p=p)
    d = problem_to_device({k: v for k, v in prob.items() if hasattr(v, "shape")})
    plan = q2x.Plan(p, precision=prec)
    leaf, _ = plan.triangles(d["vxyz"], d["idx"], d["sigma"], d["leaf_off"], d["leaf_c"], d["leaf_rho"], None,
                             density="linear")
    plan64 = q2x.Plan(p, precision="fp64")
    up = Upward(plan64, d["leaf_c"], lo, size, depth)
    levels = up.run(leaf)
    plan.sync()
    plan64.sync()
    root = levels[-1].cpu().numpy()
    assert root.shape[0] == 1 and np.allclose(up.levels[-1]["c"][:, 0], 0.0)
    all_idx = prob["idx"]
    ref = orc.moments("triangle", prob["vxyz"], all_idx, prob["sigma"], p, leaf_off=np.array([0, all_idx.shape[1]]),
                      leaf_c=np.zeros((3, 1)), density=1)
    rho = np.max(np.linalg.norm(prob["vxyz"], axis=0))
    tol = 1e-12 if prec == "fp64" else 1e-5
    assert norm_err(root, ref, p, [rho], 0) <= tol
    # level 1 (8 boxes of half size): boxes 0 and 5 against quadrature over their leaves
    lvl1 = levels[-2].cpu().numpy()
    lv = up.levels
    # leaves of each level-1 box via the CSR chain leaves -> depth-1 -> ... -> level 1
    owner = np.arange(prob["leaf_c"].shape[1])
    for lvd in lv[:-1]:
        parent_of = np.repeat(np.arange(len(lvd["dst_off"]) - 1), np.diff(lvd["dst_off"]))
        owner = parent_of[owner]
    leaf_owner = np.repeat(owner, np.diff(prob["leaf_off"]))
    for box in (0, min(5, lvl1.shape[0] - 1)):
        sel = np.nonzero(leaf_owner == box)[0]
        idx = np.ascontiguousarray(all_idx[:, sel])
        c = lv[-2]["c"][:, box]
        r = orc.moments("triangle", prob["vxyz"], idx, prob["sigma"], p, leaf_off=np.array([0, idx.shape[1]]),
                        leaf_c=c.reshape(3, 1), density=1)
        rb = np.max(np.linalg.norm(prob["vxyz"][:, np.unique(idx)] - c[:, None], axis=0))
        assert norm_err(lvl1[box:box + 1], r, p, [rb], 0) <= tol


def test_upward_pass_adaptive_mixed_ball(q2x, orc):
    """Adaptive octree (leaves at depths 2 and 3) over segments, triangles and
    tetrahedra: batch Q2X at the leaves (p = 8 everywhere), then the upward
    pass; the root against the oracle's quadrature of all elements about the
    cube centre, and every depth-1 box against quadrature over its elements."""
    from paper_2107_10942_gb300.upward import Upward
    p = 8
    m = W.cfg_mixed_ball(n_fil=40, n_steps=100, tri_level=4, n_tri=3000, tet_spacing=0.2, n_tet=2500,
                         max_per_leaf=300, max_depth=8, p_lo=p, p_hi=p, seed=11)
    names = {"segment": "segments", "triangle": "triangles", "tetra": "tetra"}
    kinds = {names[k]: {key: torch.from_numpy(v).cuda() for key, v in dd.items()} for k, dd in m["kinds"].items()}
    plan = q2x.Plan(p, precision="fp64")
    b = q2x.q2x.Batch(plan, torch.from_numpy(m["leaf_c"]).cuda(), torch.from_numpy(m["leaf_rho"]).cuda(),
                      torch.from_numpy(m["leaf_p"]).cuda(), **kinds)
    leaf = b.run()
    up = Upward(plan, m["leaf_c"], -1.0, 2.0, m["leaf_depth"])
    outs = up.run(leaf)
    plan.sync()
    assert len(set(m["leaf_depth"].tolist())) > 1

    def quad(centre, leaf_sel):
        ref = 0
        for k, dd in m["kinds"].items():
            o = dd["leaf_off"]
            el = np.concatenate([np.arange(o[L], o[L + 1]) for L in leaf_sel]).astype(np.int64)
            if len(el):
                idx = np.ascontiguousarray(dd["idx"][:, el])
                ref = ref + orc.moments(k, dd["vxyz"], idx, dd["sigma"][el], p, leaf_off=np.array([0, len(el)]),
                                        leaf_c=centre.reshape(3, 1))
        return ref

    def radius(centre, leaf_sel):
        r = 0.0
        for dd in m["kinds"].values():
            o = dd["leaf_off"]
            el = np.concatenate([np.arange(o[L], o[L + 1]) for L in leaf_sel]).astype(np.int64)
            if len(el):
                v = dd["vxyz"][:, np.unique(dd["idx"][:, el])]
                r = max(r, np.max(np.linalg.norm(v - centre[:, None], axis=0)))
        return r

    nl = m["leaf_c"].shape[1]
    root = outs[-1].cpu().numpy()
    c0 = np.zeros(3)
    assert norm_err(root, quad(c0, range(nl)), p, [radius(c0, range(nl))], 0) <= 1e-12
    # depth-1 boxes: the leaves inside each (by position)
    lvl1 = outs[-2].cpu().numpy()
    c1 = up.levels[-2]["c"]
    for box in range(c1.shape[1]):
        inside = np.nonzero(np.all(np.abs(m["leaf_c"] - c1[:, box:box + 1]) < 0.5, axis=0))[0]
        assert norm_err(lvl1[box:box + 1], quad(c1[:, box], inside), p, [radius(c1[:, box], inside)], 0) <= 1e-12


@pytest.mark.parametrize("adaptive", [False, True])
def test_upward_graph_replay_bitwise(q2x, adaptive):
    """The captured pass replays to the same bits as the eager pass, and
    follows new leaf values written into the captured input buffer."""
    from paper_2107_10942_gb300.q2x import problem_to_device
    from paper_2107_10942_gb300.upward import Upward
    p = 8
    if adaptive:
        m = W.cfg_mixed_ball(n_fil=20, n_steps=60, tri_level=3, n_tri=800, tet_spacing=0.25, n_tet=600,
                             max_per_leaf=120, max_depth=8, p_lo=p, p_hi=p, seed=12)
        leaf_c, lo, size, depth = m["leaf_c"], -1.0, 2.0, m["leaf_depth"]
    else:
        prob = W.cfg_sphere_linear(level=4, depth=3, p=p)
        leaf_c, lo, size, depth = prob["leaf_c"], -1.125, 2.25, 3
    nl = leaf_c.shape[1]
    plan = q2x.Plan(p, precision="fp64")
    gen = torch.Generator(device="cuda").manual_seed(5)
    leaf = torch.randn((nl, (p + 1) ** 2), dtype=torch.float64, device="cuda", generator=gen)
    up = Upward(plan, leaf_c, lo, size, depth)
    eager = [t.clone() for t in up.run(leaf)]
    up.capture(leaf)
    got = up.replay()
    torch.cuda.synchronize()
    assert all(torch.equal(a, b) for a, b in zip(eager, got))
    leaf.copy_(torch.randn(leaf.shape, dtype=torch.float64, device="cuda", generator=gen))
    eager2 = [t.clone() for t in up.run(leaf)]
    got2 = [t.clone() for t in up.replay()]
    plan.sync()
    assert all(torch.equal(a, b) for a, b in zip(eager2, got2))
    assert not torch.equal(eager[-1], eager2[-1])


def test_translation_rows_match_oracle_harmonics(q2x, orc):
    """q2x_translation_rows against the oracle's Cartesian R_n^m (Eq. bas1),
    in the coefficients' real packing."""
    p = 14
    rng = np.random.default_rng(41)
    t = rng.normal(size=(3, 9)) * 0.3
    t[:, 0] = 0.0  # the zero shift: R_0^0 = 1, all else 0
    plan = q2x.Plan(p, precision="fp64")
    rows = plan.translation_rows(torch.from_numpy(t).cuda()).cpu().numpy()
    plan.sync()
    for i in range(t.shape[1]):
        R = orc.rnm(t[:, i], p)
        ref = np.zeros((p + 1) ** 2)
        for n in range(p + 1):
            for m in range(n + 1):
                ref[n * n + n + m] = R[n * n + n + m].real
                if m:
                    ref[n * n + n - m] = R[n * n + n + m].imag
        assert np.max(np.abs(rows[i] - ref)) <= 1e-14 * max(1.0, np.max(np.abs(ref)))


@pytest.mark.parametrize("adaptive", [False, True])
def test_upward_precomputed_shifts_agree(q2x, adaptive):
    """The pass with the tree's precomputed shift rows against the pass that
    builds R(t) per translation, and a bad shift index flagged."""
    from paper_2107_10942_gb300.upward import Upward
    p = 10
    if adaptive:
        m = W.cfg_mixed_ball(n_fil=20, n_steps=60, tri_level=3, n_tri=800, tet_spacing=0.25, n_tet=600,
                             max_per_leaf=120, max_depth=8, p_lo=p, p_hi=p, seed=12)
        leaf_c, lo, size, depth = m["leaf_c"], -1.0, 2.0, m["leaf_depth"]
    else:
        prob = W.cfg_sphere_linear(level=4, depth=3, p=p)
        leaf_c, lo, size, depth = prob["leaf_c"], -1.125, 2.25, 3
    nl = leaf_c.shape[1]
    plan = q2x.Plan(p, precision="fp64")
    gen = torch.Generator(device="cuda").manual_seed(6)
    leaf = torch.randn((nl, (p + 1) ** 2), dtype=torch.float64, device="cuda", generator=gen)
    up = Upward(plan, leaf_c, lo, size, depth)
    assert all(rt.shape[0] <= 8 for rt, _ in up.rt[:1]) or adaptive  # an octree level has eight shifts
    fast = [x.clone() for x in up.run(leaf)]
    slow = [x.clone() for x in up.run(leaf, precomputed_shifts=False)]
    plan.sync()
    for a, b in zip(fast, slow):
        assert (a - b).abs().max().item() <= 1e-13 * b.abs().max().item()
    rt, t_idx = up.rt[0]
    bad = t_idx.clone()
    bad[0] = rt.shape[0]
    off, c, out, _, _ = up.dev[0]
    src = leaf if up.identity else leaf.index_select(0, up.deep_idx)
    plan.translate_rt(src, rt, bad, off, dst_coef=out.clone(), p=p)
    with pytest.raises(q2x.Q2XError):
        plan.sync()
