"""GPU parity: the CUDA path (through the C ABI) against the FP64 oracle.

Tolerances, in the normalised coefficient error of _helpers.norm_err:
FP64 path 1e-12, FP32-mixed path 1e-5 (relative to the leaf's largest scaled
coefficient).  Inputs span several warp ranges and a ragged tail, include
empty leaves, single-element leaves and leaves split across ranges."""
import numpy as np
import pytest

import workloads as W
from _helpers import norm_err, oracle_coef, random_problem

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

TOL = {"fp64": 1e-12, "fp32": 1e-5}
SIZES = [1, 0, 37, 5, 64, 100, 3, 0, 250, 31, 33]


@pytest.fixture(scope="module")
def q2x():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2107_10942_gb300 import build
    build.build()
    import paper_2107_10942_gb300 as q
    return q


def dev(prob):
    from paper_2107_10942_gb300.q2x import problem_to_device
    return problem_to_device(prob)


def run(q, prob, prec, norm="coeff", single=True, double=False, per_element=False, use_rho=True,
        use_p=True, plan=None):
    d = dev(prob)
    pl = plan or q.Plan(prob["p"], norm=norm, precision=prec)
    lo = None if per_element else d["leaf_off"]
    if per_element:
        leaf_of = np.repeat(np.arange(prob["leaf_c"].shape[1]), np.diff(prob["leaf_off"]))
        lc = torch.from_numpy(np.ascontiguousarray(prob["leaf_c"][:, leaf_of])).cuda()
        rho = torch.from_numpy(np.ascontiguousarray(prob["leaf_rho"][leaf_of])).cuda() if use_rho else None
        lp = None
    else:
        lc = d["leaf_c"]
        rho = d["leaf_rho"] if use_rho else None
        lp = d["leaf_p"] if use_p else None
    kind = prob["kind"]
    if kind == "segment":
        out = (pl.segments(d["vxyz"], d["idx"], d["sigma"], lo, lc, rho, lp), None)
    elif kind == "tetra":
        out = (pl.tetra(d["vxyz"], d["idx"], d["sigma"], lo, lc, rho, lp), None)
    else:
        out = pl.triangles(d["vxyz"], d["idx"], d["sigma"], lo, lc, rho, lp, density=prob["density"],
                           single=single, double=double)
    pl.sync()
    return [None if o is None else o.cpu().numpy() for o in out]


CASES = [("segment", "const", 0, False), ("triangle", "const", 0, False), ("triangle", "const", 1, False),
         ("triangle", "const", 0, True), ("triangle", "linear", 0, True), ("triangle", "linear", 1, False),
         ("tetra", "const", 0, False)]


@pytest.mark.parametrize("prec", ["fp64", "fp32"])
@pytest.mark.parametrize("p", [0, 1, 3, 8, 12, 16, 20])
@pytest.mark.parametrize("kind,density,layer,both", CASES)
def test_parity(q2x, orc, kind, density, layer, both, prec, p):
    prob = random_problem(kind, SIZES, seed=p * 7 + len(kind), p=p, density=density)
    single = layer == 0 or both
    double = layer == 1 or both
    cs, cd = run(q2x, prob, prec, single=single, double=double)
    if single:
        ref = oracle_coef(orc, prob, layer=0)
        e = norm_err(cs, ref, p, prob["leaf_rho"], 0)
        assert e <= TOL[prec], ("single", e)
    if double:
        ref = oracle_coef(orc, prob, layer=1)
        e = norm_err(cd, ref, p, prob["leaf_rho"], 1)
        assert e <= TOL[prec], ("double", e)
    # empty leaves are exactly zero
    empty = np.where(np.diff(prob["leaf_off"]) == 0)[0]
    for c in (cs, cd):
        if c is not None:
            assert np.all(c[empty] == 0)


@pytest.mark.parametrize("prec", ["fp64", "fp32"])
@pytest.mark.parametrize("kind,density,layer,both", CASES)
def test_point_vertex_on_axis_and_plane(q2x, orc, kind, density, layer, both, prec):
    """The point level's vertex (the element's second) on its leaf centre's
    z-axis, in the centre's z-plane or at the centre itself: x + iy = 0 or
    z = 0 exactly, the cases where the FP64 order recursion over m (reading
    R27) would be ill-conditioned if it divided by |xi|.  p = 20."""
    p = 20
    prob = random_problem(kind, SIZES, seed=2701 + len(kind), p=p, density=density)
    n = prob["idx"].shape[1]
    leaf_of = np.repeat(np.arange(prob["leaf_c"].shape[1]), np.diff(prob["leaf_off"]))
    v2 = prob["idx"][1]
    c = prob["leaf_c"][:, leaf_of]
    sel = np.arange(n) % 4
    prob["vxyz"][0, v2[sel == 0]] = c[0, sel == 0]  # on the axis
    prob["vxyz"][1, v2[sel == 0]] = c[1, sel == 0]
    prob["vxyz"][2, v2[sel == 1]] = c[2, sel == 1]  # in the plane
    prob["vxyz"][:, v2[sel == 2]] = c[:, sel == 2]  # at the centre
    rho = W.leaf_rho(prob["vxyz"], prob["idx"], prob["leaf_off"], prob["leaf_c"])
    prob["leaf_rho"] = np.where(rho > 0, rho, 1.0)
    single = layer == 0 or both
    double = layer == 1 or both
    cs, cd = run(q2x, prob, prec, single=single, double=double)
    for ly, on, got in ((0, single, cs), (1, double, cd)):
        if not on:
            continue
        ref = oracle_coef(orc, prob, layer=ly)
        e = norm_err(got, ref, p, prob["leaf_rho"], ly)
        assert e <= TOL[prec], (ly, e)


@pytest.mark.parametrize("prec", ["fp64", "fp32"])
@pytest.mark.parametrize("kind,density,layer,both", [("segment", "const", 0, False),
                                                     ("triangle", "const", 0, True),
                                                     ("tetra", "const", 0, False)])
def test_runs_of_tiny_and_empty_leaves(q2x, orc, kind, density, layer, both, prec):
    # more than 32 leaves start inside one 32-element round (single-element
    # and empty leaves): the kernel's leaf lookup must leave its 32-leaf
    # window for the search in leaf_off; the rest fit the window
    sizes = [1] * 45 + [0] * 20 + [2, 0] * 25 + [1, 0, 0, 3] * 12 + [70, 0, 0, 0, 1] + [1] * 33
    p = 6
    prob = random_problem(kind, sizes, seed=29, p=p, density=density)
    cs, cd = run(q2x, prob, prec, single=True, double=both)
    assert norm_err(cs, oracle_coef(orc, prob, layer=0), p, prob["leaf_rho"], 0) <= TOL[prec]
    if cd is not None:
        assert norm_err(cd, oracle_coef(orc, prob, layer=1), p, prob["leaf_rho"], 1) <= TOL[prec]
    empty = np.where(np.diff(prob["leaf_off"]) == 0)[0]
    for c in (cs, cd):
        if c is not None:
            assert np.all(c[empty] == 0)


@pytest.mark.parametrize("prec", ["fp64", "fp32"])
def test_moment_norm(q2x, orc, prec):
    for kind, density in (("segment", "const"), ("triangle", "linear"), ("tetra", "const")):
        prob = random_problem(kind, SIZES, seed=5, p=9, density=density)
        cs, cd = run(q2x, prob, prec, norm="moment", single=True, double=(kind == "triangle"))
        assert norm_err(cs, oracle_coef(orc, prob, 0, norm=1), 9, prob["leaf_rho"], 0) <= TOL[prec]
        if cd is not None:
            assert norm_err(cd, oracle_coef(orc, prob, 1, norm=1), 9, prob["leaf_rho"], 1) <= TOL[prec]


@pytest.mark.parametrize("prec", ["fp64", "fp32"])
def test_per_element_mode(q2x, orc, prec):
    prob = random_problem("triangle", [3, 40, 7, 1], seed=11, p=10, density="linear")
    cs, cd = run(q2x, prob, prec, single=True, double=True, per_element=True)
    leaf_of = np.repeat(np.arange(prob["leaf_c"].shape[1]), np.diff(prob["leaf_off"]))
    rho = prob["leaf_rho"][leaf_of]
    assert norm_err(cs, oracle_coef(orc, prob, 0, per_element=True), 10, rho, 0) <= TOL[prec]
    assert norm_err(cd, oracle_coef(orc, prob, 1, per_element=True), 10, rho, 1) <= TOL[prec]


@pytest.mark.parametrize("prec", ["fp64", "fp32"])
def test_leaf_p_and_computed_rho(q2x, orc, prec):
    sizes = [20, 70, 0, 45, 5]
    lp = np.array([12, 3, 7, 0, 9], dtype=np.int32)
    prob = random_problem("tetra", sizes, seed=3, p=12, leaf_p=lp)
    cs, _ = run(q2x, prob, prec, use_rho=False)
    ref = oracle_coef(orc, prob, 0)
    assert norm_err(cs, ref, 12, prob["leaf_rho"], 0) <= TOL[prec]
    for L in range(len(sizes)):
        assert np.all(cs[L, (lp[L] + 1) ** 2:] == 0)


@pytest.mark.parametrize("prec", ["fp64", "fp32"])
def test_accumulate_mixed_kinds(q2x, orc, prec):
    # segments, triangles and tetrahedra into the same leaves
    sizes = [10, 0, 50, 3]
    ps = [random_problem(k, sizes, seed=21, p=8) for k in ("segment", "triangle", "tetra")]
    for pr in ps[1:]:
        pr["leaf_c"] = ps[0]["leaf_c"]
        pr["leaf_rho"] = np.maximum(pr["leaf_rho"], ps[0]["leaf_rho"])
    rho = np.max(np.stack([pr["leaf_rho"] for pr in ps]), axis=0)
    for pr in ps:
        pr["leaf_rho"] = rho
    pl = q2x.Plan(8, precision=prec)
    coef = torch.zeros((len(sizes), 81), dtype=torch.float64, device="cuda")
    for pr in ps:
        d = dev(pr)
        if pr["kind"] == "segment":
            pl.segments(d["vxyz"], d["idx"], d["sigma"], d["leaf_off"], d["leaf_c"], d["leaf_rho"], coef=coef,
                        accumulate=True)
        elif pr["kind"] == "tetra":
            pl.tetra(d["vxyz"], d["idx"], d["sigma"], d["leaf_off"], d["leaf_c"], d["leaf_rho"], coef=coef,
                     accumulate=True)
        else:
            pl.triangles(d["vxyz"], d["idx"], d["sigma"], d["leaf_off"], d["leaf_c"], d["leaf_rho"],
                         coef_single=coef, accumulate=True)
    pl.sync()
    ref = sum(oracle_coef(orc, pr, 0) for pr in ps)
    assert norm_err(coef.cpu().numpy(), ref, 8, rho, 0) <= TOL[prec]


@pytest.mark.parametrize("prec", ["fp64", "fp32"])
def test_leaf_over_many_ranges(q2x, orc, prec):
    # with about 2,200 elements every warp range holds 32 of them, so the
    # 1,500-element leaf spans some 47 ranges (the fix-up's four-chain sums)
    # and the 70-element one three (its single chain); run twice: bit-equal
    prob = random_problem("triangle", [1500, 3, 0, 70, 600], seed=41, p=8, density="const")
    a = run(q2x, prob, prec, single=True, double=True)
    b = run(q2x, prob, prec, single=True, double=True)
    assert np.array_equal(a[0], b[0]) and np.array_equal(a[1], b[1])
    for layer in (0, 1):
        e = norm_err(a[layer], oracle_coef(orc, prob, layer=layer), 8, prob["leaf_rho"], layer)
        assert e <= TOL[prec], (layer, e)


def test_deterministic(q2x):
    prob = random_problem("triangle", SIZES * 3, seed=2, p=12, density="linear")
    for prec in ("fp64", "fp32"):
        a = run(q2x, prob, prec, single=True, double=True)
        b = run(q2x, prob, prec, single=True, double=True)
        assert np.array_equal(a[0], b[0]) and np.array_equal(a[1], b[1])


def test_leaf_reduce_bitexact(q2x):
    rng = np.random.default_rng(0)
    p = 7
    sizes = [0, 5, 1, 300, 0, 17]
    off = W.csr_from_leaf_of(np.repeat(np.arange(len(sizes)), sizes), len(sizes))
    elem = rng.standard_normal((off[-1], 64))
    pl = q2x.Plan(p)
    got = pl.leaf_reduce(torch.from_numpy(elem).cuda(), p, torch.from_numpy(off).cuda()).cpu().numpy()
    pl.sync()
    for L in range(len(sizes)):
        acc = np.zeros(64)
        for e in range(off[L], off[L + 1]):
            acc = acc + elem[e]
        assert np.array_equal(got[L], acc)


def test_device_error_word(q2x):
    prob = random_problem("triangle", [10, 20], seed=1, p=4)
    prob["idx"][1, 3] = prob["vxyz"].shape[1] + 5  # out of range
    with pytest.raises(q2x.Q2XError) as ei:
        run(q2x, prob, "fp64")
    assert ei.value.status == 5
    prob = random_problem("triangle", [10, 20], seed=1, p=4)
    prob["sigma"][4] = np.nan
    pl = q2x.Plan(4)
    with pytest.raises(q2x.Q2XError):
        run(q2x, prob, "fp32", plan=pl)
    # the word is cleared after the report
    pl.sync()


def test_host_argument_errors(q2x):
    pl = q2x.Plan(6)
    with pytest.raises(ValueError):  # idx of the wrong arity, caught by the binding
        pl.segments(torch.zeros((3, 4), dtype=torch.float64, device="cuda"),
                    torch.zeros((3, 4), dtype=torch.int32, device="cuda"), None, None, None)
    with pytest.raises(q2x.Q2XError) as ei:  # NULL sigma, caught by the C ABI
        pl.segments(torch.zeros((3, 4), dtype=torch.float64, device="cuda"),
                    torch.zeros((2, 4), dtype=torch.int32, device="cuda"), None,
                    torch.tensor([0, 4], dtype=torch.int64, device="cuda"),
                    torch.zeros((3, 1), dtype=torch.float64, device="cuda"))
    assert ei.value.status == 1
    with pytest.raises(q2x.Q2XError) as ei:
        q2x.Plan(25)
    assert ei.value.status == 2


def test_fixture_accuracy_on_gpu(q2x, orc):
    """The paper's Sec. 4.1 fixture (r_t = 0.1, d = 1.5) through the GPU path."""
    import math
    rc = np.array([math.sqrt(3) / 2, 0, 0])
    X = rc + 0.1 * np.array([[1, 0, 0], [-0.5, math.sqrt(3) / 2, 0], [-0.5, -math.sqrt(3) / 2, 0]])
    prob = dict(vxyz=X.T.copy(), idx=np.arange(3, dtype=np.int32)[:, None], sigma=np.array([1.0]),
                leaf_off=np.array([0, 1]), leaf_c=np.zeros((3, 1)), leaf_rho=np.array([1.0]),
                leaf_p=np.array([20], dtype=np.int32), p=20, kind="triangle", density="const")
    for prec in ("fp64", "fp32"):
        cs, _ = run(q2x, prob, prec)
        ref = oracle_coef(orc, prob, 0)
        assert norm_err(cs, ref, 20, [1.0], 0) <= TOL[prec]


@pytest.mark.parametrize("prec", ["fp64", "fp32"])
def test_full_size_sphere_sampled(q2x, orc, prec):
    """The level-7 perturbed sphere with linear density, single + double layer,
    depth-5 octree, p = 12, at full size in the bench's launch configuration;
    checked against the oracle on a sample of 12 leaves."""
    prob = W.cfg_sphere_linear(level=7, depth=5, p=12)
    cs, cd = run(q2x, prob, prec, single=True, double=True)
    rng = np.random.default_rng(7)
    nl = prob["leaf_c"].shape[1]
    pick = rng.choice(nl, size=12, replace=False)
    off = prob["leaf_off"]
    for L in pick:
        sub = dict(prob)
        e0, e1 = off[L], off[L + 1]
        sub["idx"] = np.ascontiguousarray(prob["idx"][:, e0:e1])
        sub["leaf_off"] = np.array([0, e1 - e0])
        sub["leaf_c"] = np.ascontiguousarray(prob["leaf_c"][:, L:L + 1])
        sub["leaf_p"] = prob["leaf_p"][L:L + 1]
        for layer, got in ((0, cs), (1, cd)):
            ref = oracle_coef(orc, sub, layer)
            assert norm_err(got[L:L + 1], ref, 12, prob["leaf_rho"][L:L + 1], layer) <= TOL[prec]
