"""q2x_triangles_noalloc -- the triangle Q2X call for callers that cannot
allocate device memory (memory handed to their own pool, paths that must not
synchronise the device, no out-of-memory failure allowed at call time).

Called through the C ABI with ctypes and compared with q2x_triangles (the
plan-based entry point) within the parity tolerances of the other tests.  The
scratch array is shared by every call and keeps the last call's contents, so
each check runs after a call on a different, larger problem (other densities,
leaf structure and number of ranges) has left its partial sums there, and
then twice in a row.  Also covered: one output layer only with accumulate = 1,
per-leaf degrees, and the size limit.  This file is collected last on
purpose."""
import ctypes

import numpy as np
import pytest

from _helpers import norm_err, random_problem

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

TOL = {"fp64": 1e-12, "fp32": 1e-5}
P = 12


@pytest.fixture(scope="module")
def q2x():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2107_10942_gb300 import build
    build.build()
    import paper_2107_10942_gb300 as q
    return q


def _p(t):
    return None if t is None else ctypes.c_void_p(t.data_ptr())


def _fn():
    from paper_2107_10942_gb300._lib import lib
    f = lib().q2x_triangles_noalloc
    i64, p_, i = ctypes.c_int64, ctypes.c_void_p, ctypes.c_int
    f.argtypes = [i, i, i, p_, i64, i64, p_, p_, i, p_, i64, p_, p_, p_, p_, p_, p_, i]
    f.restype = ctypes.c_int
    return f


def _call(f, d, prec, density, cs, cd, accumulate=0, leaf_p=True):
    stream = torch.cuda.current_stream()
    n_leaves = d["leaf_c"].shape[1]
    return f(P, 0, 0 if prec == "fp64" else 1, ctypes.c_void_p(stream.cuda_stream), d["idx"].shape[1],
             d["vxyz"].shape[1], _p(d["vxyz"]), _p(d["idx"]), 1 if density == "linear" else 0, _p(d["sigma"]),
             n_leaves, _p(d["leaf_off"]), _p(d["leaf_c"]), _p(d["leaf_rho"]), _p(d["leaf_p"]) if leaf_p else None,
             _p(cs), _p(cd), accumulate)


@pytest.mark.parametrize("prec,density", [("fp64", "linear"), ("fp32", "linear"), ("fp64", "const"),
                                          ("fp32", "const")])
def test_noalloc_matches_plan_entry_point(q2x, prec, density):
    from paper_2107_10942_gb300.q2x import problem_to_device
    f = _fn()
    # the checked problem: leaves straddling 256-element ranges, per-leaf degrees
    sizes = [1, 0, 300, 37, 5, 700, 64, 0, 250, 31, 33, 515]
    leaf_p = np.random.default_rng(5).integers(0, P + 1, size=len(sizes)).astype(np.int32)
    leaf_p[[2, 5, 11]] = P
    prob = random_problem("triangle", sizes, seed=77, p=P, density=density, leaf_p=leaf_p)
    d = problem_to_device(prob)
    # a different, larger problem whose partial sums are left in the scratch
    other = random_problem("triangle", [900, 3, 1200, 0, 410, 2600, 77], seed=78, p=P, density=density)
    do = problem_to_device(other)

    plan = q2x.Plan(P, precision=prec)
    ref_s, ref_d = plan.triangles(d["vxyz"], d["idx"], d["sigma"], d["leaf_off"], d["leaf_c"], d["leaf_rho"],
                                  d["leaf_p"], density=density, single=True, double=True)
    plan.sync()
    ref_s_np, ref_d_np = ref_s.cpu().numpy(), ref_d.cpu().numpy()

    n_leaves = len(sizes)
    nc = (P + 1) ** 2
    for call in range(2):
        ws = torch.empty((other["leaf_c"].shape[1], nc), dtype=torch.float64, device="cuda")
        assert _call(f, do, prec, density, ws, torch.empty_like(ws), leaf_p=False) == 0
        cs = torch.full((n_leaves, nc), float("nan"), dtype=torch.float64, device="cuda")
        cd = torch.full_like(cs, float("nan"))
        assert _call(f, d, prec, density, cs, cd) == 0
        torch.cuda.synchronize()
        got_s, got_d = cs.cpu().numpy(), cd.cpu().numpy()
        assert np.all(np.isfinite(got_s)) and np.all(np.isfinite(got_d))
        assert norm_err(got_s, ref_s_np, P, prob["leaf_rho"], 0) <= TOL[prec], call
        assert norm_err(got_d, ref_d_np, P, prob["leaf_rho"], 1) <= TOL[prec], call
        # entries above each leaf's degree are exactly zero
        for L, pl in enumerate(leaf_p):
            assert np.all(got_s[L, (pl + 1) ** 2:] == 0.0)

    # one layer only, accumulated onto the plan path's result: twice the result
    acc = ref_d.clone()
    assert _call(f, d, prec, density, None, acc, accumulate=1) == 0
    torch.cuda.synchronize()
    assert norm_err(acc.cpu().numpy(), 2.0 * ref_d_np, P, prob["leaf_rho"], 1) <= TOL[prec]
    acc = ref_s.clone()
    assert _call(f, d, prec, density, acc, None, accumulate=1) == 0
    torch.cuda.synchronize()
    assert norm_err(acc.cpu().numpy(), 2.0 * ref_s_np, P, prob["leaf_rho"], 0) <= TOL[prec]


def test_noalloc_rejects_oversize(q2x):
    f = _fn()
    dummy = torch.zeros(8, dtype=torch.float64, device="cuda")
    ptr = ctypes.c_void_p(dummy.data_ptr())
    # p_max = 20 in FP64: at most 256 * floor(16 MiB / (4 * 441 * 8)) = 304,128 elements
    limit = 256 * ((16 << 20) // (4 * 441 * 8))
    for n in (limit + 1, 1 << 62, (1 << 63) - 1):
        st = f(20, 0, 0, None, n, 8, ptr, ptr, 0, ptr, 1, ptr, ptr, ptr, None, ptr, None, 0)
        assert st == 2, n  # Q2X_ERR_RANGE, nothing launched
