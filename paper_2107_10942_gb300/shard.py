"""Leaf sharding for several GPUs (host-side input preparation).

Leaves are independent units of the Q2X step: every coefficient row is a sum
over the elements of one leaf only (Eq. st4), so ranks that own disjoint sets
of whole leaves need no exchange while they compute.  The leaf list (already
in Morton order) is cut into contiguous ranges of nearly equal cost, where a
leaf costs sum over its elements of (p_leaf+1)^2 times the number of
recursion levels of the element kind; each rank receives its leaves' elements
plus the vertices they reference (vertices on a cut are duplicated).  When a
later stage needs every leaf's coefficients, one all_gather of the
per-rank coefficient blocks assembles them (gather_coefficients).

All functions here work on numpy arrays in the layout of the workloads
module: vxyz (3, n_vert), idx (k, n_elem) int32 sorted by leaf, sigma per
element (constant density) or per vertex (linear density), leaf_off (n_leaves
+ 1) int64, leaf_c (3, n_leaves), leaf_rho, leaf_p."""
from __future__ import annotations

import numpy as np

# recursion levels per element kind: segment q,p; triangle q,j,i; linear
# triangle q,j,i,E,Iw; tetrahedron q,j,b,a
LEVELS = {("segment", "const"): 2, ("triangle", "const"): 3, ("triangle", "linear"): 5, ("tetra", "const"): 4}


def leaf_costs(leaf_off, leaf_p, kind="triangle", density="const", layers=1):
    """cost[L] = n_elem(L) * (p_leaf+1)^2 * (levels + layers - 1)."""
    n = np.diff(np.asarray(leaf_off, dtype=np.int64))
    p = np.asarray(leaf_p, dtype=np.int64)
    return n * (p + 1) ** 2 * (LEVELS[(kind, density)] + layers - 1)


def partition_leaves(cost, world):
    """Cut points b[0]=0 <= b[1] <= ... <= b[world]=n_leaves of a contiguous
    partition of the leaves.  Rank r owns leaves b[r]..b[r+1]-1.  Each cut is
    placed where the prefix sum of the cost crosses r/world of the total, so
    every range costs at most total/world + max(cost)."""
    cost = np.asarray(cost, dtype=np.float64)
    if world < 1:
        raise ValueError("world must be >= 1")
    n = cost.shape[0]
    pre = np.concatenate([[0.0], np.cumsum(cost)])
    total = pre[-1]
    b = np.zeros(world + 1, dtype=np.int64)
    b[world] = n
    for r in range(1, world):
        t = total * r / world
        k = int(np.searchsorted(pre, t, side="left"))
        # the nearer of the two prefix boundaries around the target
        if k > 0 and t - pre[k - 1] <= pre[k] - t:
            k -= 1
        b[r] = min(max(k, b[r - 1]), n)
    return b


def shard_problem(prob, lo, hi):
    """The sub-problem of leaves lo..hi-1: their elements, the vertices those
    reference (compacted, idx remapped), their densities, leaf data and a
    rebased leaf_off.  Works for one element kind (keys vxyz, idx, sigma,
    leaf_off, leaf_c, leaf_rho, leaf_p, and optionally density)."""
    off = np.asarray(prob["leaf_off"], dtype=np.int64)
    e0, e1 = int(off[lo]), int(off[hi])
    idx = np.asarray(prob["idx"])[:, e0:e1]
    used, remap = np.unique(idx.reshape(-1), return_inverse=True)
    out = {k: v for k, v in prob.items() if not hasattr(v, "shape")}
    out["vxyz"] = np.ascontiguousarray(np.asarray(prob["vxyz"])[:, used])
    out["idx"] = np.ascontiguousarray(remap.reshape(idx.shape).astype(np.int32))
    sig = np.asarray(prob["sigma"])
    out["sigma"] = np.ascontiguousarray(sig[used] if prob.get("density") == "linear" else sig[e0:e1])
    out["leaf_off"] = np.ascontiguousarray(off[lo:hi + 1] - e0)
    out["leaf_c"] = np.ascontiguousarray(np.asarray(prob["leaf_c"])[:, lo:hi])
    for k in ("leaf_rho", "leaf_p"):
        if k in prob and prob[k] is not None:
            out[k] = np.ascontiguousarray(np.asarray(prob[k])[lo:hi])
    out["leaf_range"] = (int(lo), int(hi))
    return out


def replicate_problem(prob, copies):
    """`copies` independent copies of a one-kind problem, concatenated leaf
    list after leaf list (the weak-scaling workload: N copies over N ranks)."""
    if copies == 1:
        return prob
    nv = prob["vxyz"].shape[1]
    ne = prob["idx"].shape[1]
    out = {k: v for k, v in prob.items() if not hasattr(v, "shape")}
    out["vxyz"] = np.ascontiguousarray(np.tile(prob["vxyz"], (1, copies)))
    out["idx"] = np.ascontiguousarray(np.concatenate([prob["idx"] + c * nv for c in range(copies)], axis=1)
                                      .astype(np.int32))
    out["sigma"] = np.ascontiguousarray(np.tile(prob["sigma"], copies))
    off = np.asarray(prob["leaf_off"], dtype=np.int64)
    out["leaf_off"] = np.ascontiguousarray(np.concatenate([off[:-1] + c * ne for c in range(copies)] +
                                                          [[copies * ne]]).astype(np.int64))
    out["leaf_c"] = np.ascontiguousarray(np.tile(prob["leaf_c"], (1, copies)))
    for k in ("leaf_rho", "leaf_p"):
        if k in prob and prob[k] is not None:
            out[k] = np.ascontiguousarray(np.tile(prob[k], copies))
    return out


def gather_coefficients(coef_local, bounds, group=None):
    """All ranks' coefficient blocks (rows bounds[r]..bounds[r+1]-1 of rank r)
    assembled into the full (n_leaves, n_coef) tensor on every rank, with one
    all_gather (blocks padded to the largest range).  coef_local is a torch
    tensor on the device the process group's backend uses."""
    import torch
    import torch.distributed as dist
    world = dist.get_world_size(group)
    sizes = np.diff(np.asarray(bounds))
    if len(sizes) != world or coef_local.shape[0] != sizes[dist.get_rank(group)]:
        raise ValueError("bounds do not match the process group or the local block")
    rows = int(sizes.max()) if world else 0
    pad = torch.zeros((rows, coef_local.shape[1]), dtype=coef_local.dtype, device=coef_local.device)
    pad[:coef_local.shape[0]] = coef_local
    parts = [torch.empty_like(pad) for _ in range(world)]
    dist.all_gather(parts, pad, group=group)
    return torch.cat([parts[r][:sizes[r]] for r in range(world)], dim=0)
