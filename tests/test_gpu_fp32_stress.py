"""Adversarial leaves for the FP32-mixed path, against the FP64 oracle.

The FP32-mixed path runs the recursions in FP32 in a scaled local frame; the
steps whose stability needs more are done otherwise: the translation to the
leaf centre keeps FP64 accuracy (exact FP64 -> FP32 pair splits), the seed
J * density is formed in FP64, and the leaf sum over rounds of 32 elements is
compensated (TwoSum).  These cases stress each of those:

* one leaf of 2,000 triangles at p = 20 (63 rounds of 32 elements, the
  largest leaf of the ragged workload and the largest degree);
* densities of equal magnitude and opposite signs, alternating or in two
  blocks (the first 1,000 elements +1, the last 1,000 -1), so the leaf sum is
  far smaller than the sum of the magnitudes of its terms: with the blocked
  signs a plain FP32 running sum carries the rounding of a partial sum about
  1,000 element moments large into a result about 30 times smaller;
* a leaf centre far from the origin, |c| = 1000 rho, so the vertex
  coordinates carry about 10 bits more than the element-to-centre offsets;

through the element kernel (q2x_triangles) and the ragged batch (q2x_batch),
at the FP32-mixed tolerance 1e-5 of the normalised coefficient error."""
import numpy as np
import pytest

from _helpers import norm_err

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

TOL = 1e-5
P = 20
N = 2000


@pytest.fixture(scope="module")
def q2x():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2107_10942_gb300 import build
    build.build()
    import paper_2107_10942_gb300 as q
    return q


def leaf_problem(signs, seed=3):
    """N small random triangles in a ball of radius rho about a centre at
    distance 1000 rho from the origin; one leaf."""
    rng = np.random.default_rng(seed)
    rho = 0.05
    c = 1000.0 * rho * np.array([0.6, -0.64, 0.48])
    u = rng.normal(size=(3, N))
    base = c[:, None] + 0.8 * rho * rng.uniform(0, 1, size=N) ** (1 / 3) * u / np.linalg.norm(u, axis=0)
    verts = [base + 0.08 * rho * rng.normal(size=(3, N)) for _ in range(3)]
    vxyz = np.ascontiguousarray(np.concatenate(verts, axis=1))
    idx = np.ascontiguousarray(np.stack([np.arange(N) + k * N for k in range(3)]).astype(np.int32))
    if signs == "alternating":
        sigma = np.where(np.arange(N) % 2 == 0, 1.0, -1.0)
    else:
        sigma = np.where(np.arange(N) < N // 2, 1.0, -1.0)
    leaf_rho = np.array([np.max(np.linalg.norm(vxyz - c[:, None], axis=0))])
    return dict(vxyz=vxyz, idx=idx, sigma=sigma, leaf_off=np.array([0, N], dtype=np.int64),
                leaf_c=np.ascontiguousarray(c.reshape(3, 1)), leaf_rho=leaf_rho,
                leaf_p=np.array([P], dtype=np.int32))


@pytest.fixture(scope="module", params=["alternating", "blocked"])
def case(request, orc):
    prob = leaf_problem(request.param)
    ref = orc.moments("triangle", prob["vxyz"], prob["idx"], prob["sigma"], P, leaf_off=prob["leaf_off"],
                      leaf_c=prob["leaf_c"])
    # the leaf sum is much smaller than the sum of its terms' magnitudes
    terms = orc.moments("triangle", prob["vxyz"], prob["idx"], np.abs(prob["sigma"]), P,
                        leaf_off=prob["leaf_off"], leaf_c=prob["leaf_c"])
    assert abs(ref[0, 0]) < 0.2 * abs(terms[0, 0])
    return request.param, prob, ref


def test_element_kernel(q2x, case):
    name, prob, ref = case
    from paper_2107_10942_gb300.q2x import problem_to_device
    d = problem_to_device(prob)
    for use_rho in (True, False):
        plan = q2x.Plan(P, precision="fp32")
        cs, _ = plan.triangles(d["vxyz"], d["idx"], d["sigma"], d["leaf_off"], d["leaf_c"],
                               d["leaf_rho"] if use_rho else None, d["leaf_p"])
        plan.sync()
        err = norm_err(cs.cpu().numpy(), ref, P, prob["leaf_rho"], 0)
        assert err <= TOL, (name, use_rho, err)


def test_batch(q2x, case):
    name, prob, ref = case
    dev = {k: torch.from_numpy(v).cuda() for k, v in prob.items()}
    for tile in (64, 512, 2048):
        plan = q2x.Plan(P, precision="fp32")
        b = q2x.q2x.Batch(plan, dev["leaf_c"], dev["leaf_rho"], dev["leaf_p"], tile_elems=tile,
                          triangles=dict(vxyz=dev["vxyz"], idx=dev["idx"], sigma=dev["sigma"],
                                         leaf_off=dev["leaf_off"], density="const"))
        b.run()
        got = b.coef.cpu().numpy()
        plan.sync()
        err = norm_err(got, ref, P, prob["leaf_rho"], 0)
        assert err <= TOL, (name, tile, err)
