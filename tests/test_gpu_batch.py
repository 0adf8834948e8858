"""GPU tests of the ragged mixed batch (q2x_batch_*): one CUDA-graph replay
(a persistent kernel per kind and degree bin) over segments, triangles and
tetrahedra sharing an adaptive octree with per-leaf degrees, checked against
the oracle (sum over kinds)."""
import json

import numpy as np
import pytest

import workloads as W
from _helpers import norm_err

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

TOL = {"fp64": 1e-12, "fp32": 1e-5}
NAMES = {"segment": "segments", "triangle": "triangles", "tetra": "tetra"}


@pytest.fixture(scope="module")
def q2x():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2107_10942_gb300 import build
    build.build()
    import paper_2107_10942_gb300 as q
    return q


@pytest.fixture(scope="module")
def mixed():
    return W.cfg_mixed_ball(n_fil=40, n_steps=100, tri_level=4, n_tri=3000, tet_spacing=0.2, n_tet=2500,
                            max_per_leaf=300, max_depth=8, p_lo=0, p_hi=20, seed=11)


def device_kinds(m, density="const"):
    out = {}
    for k, d in m["kinds"].items():
        dd = {key: torch.from_numpy(v).cuda() for key, v in d.items() if key != "density"}
        if k == "triangle":
            dd["density"] = density
        out[NAMES[k]] = dd
    return out


def oracle_sum(orc, m, triangle_sigma=None, density=0):
    ref = 0
    for k, d in m["kinds"].items():
        sig = d["sigma"] if (k != "triangle" or triangle_sigma is None) else triangle_sigma
        ref = ref + orc.moments(k, d["vxyz"], d["idx"], sig, m["p"], leaf_off=d["leaf_off"], leaf_c=m["leaf_c"],
                                leaf_p=m["leaf_p"], density=density if k == "triangle" else 0)
    return ref


def make_batch(q, m, prec, tile=0, density="const", kinds=None):
    plan = q.Plan(m["p"], precision=prec)
    kinds = kinds or device_kinds(m, density)
    b = q.q2x.Batch(plan, torch.from_numpy(m["leaf_c"]).cuda(), torch.from_numpy(m["leaf_rho"]).cuda(),
                    torch.from_numpy(m["leaf_p"]).cuda(), tile_elems=tile, **kinds)
    return plan, b, kinds


@pytest.mark.parametrize("prec", ["fp64", "fp32"])
def test_batch_matches_oracle(q2x, orc, mixed, prec):
    plan, b, _ = make_batch(q2x, mixed, prec, tile=128)
    got = b.run().cpu().numpy()
    plan.sync()
    ref = oracle_sum(orc, mixed)
    assert norm_err(got, ref, mixed["p"], mixed["leaf_rho"], 0) <= TOL[prec]
    for L, p in enumerate(mixed["leaf_p"]):
        assert np.all(got[L, (p + 1) ** 2:] == 0)
    info = b.info()
    assert info["tiles"] >= mixed["leaf_c"].shape[1] and info["tile_elems"] == 128


def test_batch_linear_triangles_and_tile_independence(q2x, orc, mixed):
    rng = np.random.default_rng(5)
    m = dict(mixed)
    m["kinds"] = {k: dict(v) for k, v in mixed["kinds"].items()}
    sig_v = rng.uniform(-1, 1, m["kinds"]["triangle"]["vxyz"].shape[1])
    m["kinds"]["triangle"]["sigma"] = sig_v
    outs = []
    for tile in (32, 1000):
        plan, b, _ = make_batch(q2x, m, "fp64", tile=tile, density="linear")
        outs.append(b.run().cpu().numpy())
        plan.sync()
    ref = oracle_sum(orc, m, triangle_sigma=sig_v, density=1)
    for got in outs:
        assert norm_err(got, ref, m["p"], m["leaf_rho"], 0) <= TOL["fp64"]


def test_batch_deterministic_and_live_inputs(q2x, mixed):
    for prec in ("fp64", "fp32"):
        plan, b, kinds = make_batch(q2x, mixed, prec, tile=96)
        a1 = b.run().clone()
        a2 = b.run().clone()
        plan.sync()
        assert torch.equal(a1, a2)
        # the graph reads the inputs at replay time: doubling every density
        # doubles the coefficients (exactly: scaling by 2 is exact)
        for kd in kinds.values():
            kd["sigma"].mul_(2.0)
        a3 = b.run().clone()
        plan.sync()
        assert torch.equal(a3, 2.0 * a1)


def test_batch_tune_and_table(q2x, mixed, tmp_path):
    plan = q2x.Plan(mixed["p"], precision="fp32")
    kinds = device_kinds(mixed)
    args = dict(leaf_c=torch.from_numpy(mixed["leaf_c"]).cuda(), leaf_rho=torch.from_numpy(mixed["leaf_rho"]).cuda(),
                leaf_p=torch.from_numpy(mixed["leaf_p"]).cuda(), **kinds)
    best, times = q2x.q2x.Batch.tune(plan, candidates=(64, 256, 1024), reps=2, **args)
    assert best in (64, 256, 1024) and all(t > 0 for t in times.values())
    path = str(tmp_path / "autotune.json")
    t1 = q2x.q2x.autotuned_tile(plan, "mixed-small", path, candidates=(64, 256), reps=1, **args)
    t2 = q2x.q2x.autotuned_tile(plan, "mixed-small", path, candidates=(64, 256), reps=1, **args)
    assert t1 == t2 and t1 in (64, 256)
    table = json.load(open(path))
    assert len(table) == 1 and list(table.values())[0]["tile_elems"] == t1


def test_batch_rejects_bad_degree(q2x, mixed):
    lp = mixed["leaf_p"].copy()
    lp[3] = 25
    m = dict(mixed)
    m["leaf_p"] = lp
    with pytest.raises(q2x.Q2XError) as ei:
        make_batch(q2x, m, "fp64")
    assert ei.value.status == 2
