"""q2x_triangles_noalloc -- the triangle Q2X call for callers that cannot
allocate device memory (memory handed to their own pool, paths that must not
synchronise the device, no out-of-memory failure allowed at call time).

Called through the C ABI with ctypes and compared with q2x_triangles (the
plan-based entry point) within the parity tolerances of the other tests, on
two calls in a row (the second sees the first call's leftover scratch).  This
file is collected last on purpose."""
import ctypes

import numpy as np
import pytest

from _helpers import norm_err, random_problem

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


def _p(t):
    return None if t is None else ctypes.c_void_p(t.data_ptr())


@pytest.mark.parametrize("prec,density", [("fp64", "linear"), ("fp32", "linear"), ("fp64", "const"),
                                          ("fp32", "const")])
def test_noalloc_matches_plan_entry_point(q2x, prec, density):
    from paper_2107_10942_gb300._lib import lib
    from paper_2107_10942_gb300.q2x import problem_to_device
    L = lib()
    f = L.q2x_triangles_noalloc
    i64, p_, i = ctypes.c_int64, ctypes.c_void_p, ctypes.c_int
    f.argtypes = [i, i, i, p_, i64, i64, p_, p_, i, p_, i64, p_, p_, p_, p_, p_, p_, i]
    f.restype = ctypes.c_int

    p = 12
    sizes = [1, 0, 300, 37, 5, 700, 64, 0, 250, 31, 33, 515]  # leaves straddling 256-element ranges
    prob = random_problem("triangle", sizes, seed=77, p=p, density=density)
    d = problem_to_device(prob)
    plan = q2x.Plan(p, precision=prec)
    ref_s, ref_d = plan.triangles(d["vxyz"], d["idx"], d["sigma"], d["leaf_off"], d["leaf_c"], d["leaf_rho"],
                                  d["leaf_p"], density=density, single=True, double=True)
    plan.sync()
    ref_s, ref_d = ref_s.cpu().numpy(), ref_d.cpu().numpy()

    n_leaves = len(sizes)
    stream = torch.cuda.current_stream()
    dens = 1 if density == "linear" else 0
    for call in range(2):
        cs = torch.full((n_leaves, (p + 1) ** 2), float("nan"), dtype=torch.float64, device="cuda")
        cd = torch.full_like(cs, float("nan"))
        st = f(p, 0, 0 if prec == "fp64" else 1, ctypes.c_void_p(stream.cuda_stream), d["idx"].shape[1],
               d["vxyz"].shape[1], _p(d["vxyz"]), _p(d["idx"]), dens, _p(d["sigma"]), n_leaves, _p(d["leaf_off"]),
               _p(d["leaf_c"]), _p(d["leaf_rho"]), _p(d["leaf_p"]), _p(cs), _p(cd), 0)
        assert st == 0, st
        torch.cuda.synchronize()
        got_s, got_d = cs.cpu().numpy(), cd.cpu().numpy()
        assert np.all(np.isfinite(got_s)) and np.all(np.isfinite(got_d))
        assert norm_err(got_s, ref_s, p, prob["leaf_rho"], 0) <= TOL[prec], call
        assert norm_err(got_d, ref_d, p, prob["leaf_rho"], 1) <= TOL[prec], call


def test_noalloc_rejects_oversize(q2x):
    from paper_2107_10942_gb300._lib import lib
    f = lib().q2x_triangles_noalloc
    f.argtypes = [ctypes.c_int, ctypes.c_int, ctypes.c_int, ctypes.c_void_p, ctypes.c_int64, ctypes.c_int64,
                  ctypes.c_void_p, ctypes.c_void_p, ctypes.c_int, ctypes.c_void_p, ctypes.c_int64,
                  ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p,
                  ctypes.c_void_p, ctypes.c_int]
    f.restype = ctypes.c_int
    dummy = torch.zeros(8, dtype=torch.float64, device="cuda")
    ptr = ctypes.c_void_p(dummy.data_ptr())
    # p_max = 20 in FP64: at most 256 * floor(16 MiB / (4 * 441 * 8)) = 304,128 elements
    n = 256 * ((16 << 20) // (4 * 441 * 8)) + 1
    st = f(20, 0, 0, None, n, 8, ptr, ptr, 0, ptr, 1, ptr, ptr, ptr, None, ptr, None, 0)
    assert st == 2  # Q2X_ERR_RANGE
