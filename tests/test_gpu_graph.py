"""Plan.capture: a captured sequence of q2x calls replays to the same bits
as the eager calls and follows new input values written into the captured
buffers (what bench.py's graph-replay timing relies on)."""
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


@pytest.mark.parametrize("prec", ["fp64", "fp32"])
def test_capture_replays_bitwise(q2x, prec):
    from paper_2107_10942_gb300.q2x import problem_to_device
    prob = random_problem("triangle", [40, 0, 75, 3, 130], seed=31, p=8, density="linear")
    d = problem_to_device({k: v for k, v in prob.items() if hasattr(v, "shape")})
    plan = q2x.Plan(8, precision=prec)
    nl = prob["leaf_c"].shape[1]
    cs = torch.empty((nl, 81), dtype=torch.float64, device="cuda")
    cd = torch.empty_like(cs)

    def step():
        plan.triangles(d["vxyz"], d["idx"], d["sigma"], d["leaf_off"], d["leaf_c"], d["leaf_rho"], None,
                       density="linear", single=True, double=True, coef_single=cs, coef_double=cd)

    step()
    ref_s, ref_d = cs.clone(), cd.clone()
    g = plan.capture(step)
    cs.zero_()
    cd.zero_()
    g.replay()
    torch.cuda.synchronize()
    assert torch.equal(cs, ref_s) and torch.equal(cd, ref_d)
    assert g.kernels >= 2
    d["sigma"].mul_(2.0)
    g.replay()
    plan.sync()
    step()
    plan.sync()
    cs2, cd2 = cs.clone(), cd.clone()
    g.replay()
    torch.cuda.synchronize()
    assert torch.equal(cs, cs2) and torch.equal(cd, cd2)
    assert not torch.equal(cs2, ref_s)


def test_capture_leaf_tiles_fp32(q2x, orc):
    # FP32-mixed single layer runs as leaf tiles built on the device (a leaf
    # of 700 elements takes three tiles and the combine; the empty leaf is
    # zeroed there): the captured call replays bitwise and matches the oracle
    from paper_2107_10942_gb300.q2x import problem_to_device
    from _helpers import norm_err, oracle_coef
    prob = random_problem("triangle", [40, 0, 700, 3, 130], seed=37, p=8, density="const")
    d = problem_to_device({k: v for k, v in prob.items() if hasattr(v, "shape")})
    plan = q2x.Plan(8, precision="fp32")
    nl = prob["leaf_c"].shape[1]
    cs = torch.full((nl, 81), 7.0, dtype=torch.float64, device="cuda")

    def step():
        plan.triangles(d["vxyz"], d["idx"], d["sigma"], d["leaf_off"], d["leaf_c"], d["leaf_rho"], None,
                       single=True, coef_single=cs)

    step()
    plan.sync()
    ref = cs.clone()
    assert norm_err(ref.cpu().numpy(), oracle_coef(orc, prob, layer=0), 8, prob["leaf_rho"], 0) <= 1e-5
    assert torch.all(ref[1] == 0)
    g = plan.capture(step)
    cs.fill_(7.0)
    g.replay()
    torch.cuda.synchronize()
    assert torch.equal(cs, ref)
