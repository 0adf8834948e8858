"""Upward pass of a uniform octree fed by the Q2X leaf coefficients: the
coefficients of every box at every level, each level from the one below by
one q2x_translate call (children -> parents).  Box centres and the
child -> parent CSR ranges are host-side preparation, done once."""
from __future__ import annotations

import numpy as np
import torch

from .q2x import Plan


def _morton(ijk: np.ndarray, depth: int) -> np.ndarray:
    code = np.zeros(ijk.shape[1], dtype=np.int64)
    for b in range(depth):
        code |= ((ijk[0] >> b) & 1) << (3 * b + 2)
        code |= ((ijk[1] >> b) & 1) << (3 * b + 1)
        code |= ((ijk[2] >> b) & 1) << (3 * b)
    return code


def octree_levels(leaf_c: np.ndarray, lo: float, size: float, depth: int):
    """Levels of the uniform octree over [lo, lo+size]^3 whose non-empty
    leaves (depth `depth`) have centres leaf_c (3, n_leaves) in Morton order.
    Returns a list, from the leaves upward, of dicts with the destination
    CSR `dst_off` over the boxes of the level below and the centres `c` of the
    boxes of this level (levels depth-1 .. 0)."""
    h = size / (1 << depth)
    ijk = np.rint((np.asarray(leaf_c) - lo) / h - 0.5).astype(np.int64)
    if ijk.size and (ijk.min() < 0 or ijk.max() >= (1 << depth)):
        raise ValueError("leaf centres outside the octree")
    code = _morton(ijk, depth)
    if np.any(np.diff(code) <= 0):
        raise ValueError("leaves must be distinct and in Morton order")
    levels = []
    for d in range(depth, 0, -1):
        pcode = code >> 3
        uniq, first, counts = np.unique(pcode, return_index=True, return_counts=True)
        off = np.zeros(len(uniq) + 1, dtype=np.int64)
        np.cumsum(counts, out=off[1:])
        pijk = ijk[:, first] >> 1
        hp = size / (1 << (d - 1))
        levels.append(dict(dst_off=off, c=lo + (pijk.astype(np.float64) + 0.5) * hp))
        code, ijk = uniq, pijk
    return levels


class Upward:
    """Upward pass over the octree of `octree_levels`: run(leaf_coef) returns
    the coefficient tensors of levels depth-1 .. 0 (the last is the root)."""

    def __init__(self, plan: Plan, leaf_c, lo: float, size: float, depth: int, p: int = None,
                 device="cuda"):
        self.plan = plan
        self.p = plan.p_max if p is None else int(p)
        lc = leaf_c.detach().cpu().numpy() if torch.is_tensor(leaf_c) else np.asarray(leaf_c)
        self.levels = octree_levels(lc, lo, size, depth)
        nc = (self.p + 1) ** 2
        self.leaf_c = torch.as_tensor(np.ascontiguousarray(lc), dtype=torch.float64, device=device)
        self.dev = []
        for lv in self.levels:
            off = torch.from_numpy(lv["dst_off"]).to(device)
            c = torch.from_numpy(np.ascontiguousarray(lv["c"])).to(device)
            out = torch.empty((c.shape[1], nc), dtype=torch.float64, device=device)
            self.dev.append((off, c, out))

    def run(self, leaf_coef):
        src, src_c = leaf_coef, self.leaf_c
        outs = []
        for off, c, out in self.dev:
            self.plan.translate(src, src_c, off, c, dst_coef=out, p=self.p)
            outs.append(out)
            src, src_c = out, c
        return outs
