"""Upward pass of an octree fed by the Q2X leaf coefficients: the
coefficients of every box at every level, each level from the one below by
one q2x_translate call (children -> parents).  Uniform trees (all leaves at
one depth) and adaptive trees (leaves at several depths) are both handled:
at each depth the boxes are the leaves of that depth plus the parents of the
boxes one level down, in Morton order.  Box centres, the child -> parent CSR
ranges and the gathers that merge leaves with internal boxes are host-side
preparation, done once."""
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


def _unmorton(code: np.ndarray, depth: int) -> np.ndarray:
    ijk = np.zeros((3, code.shape[0]), dtype=np.int64)
    for b in range(depth):
        ijk[0] |= ((code >> (3 * b + 2)) & 1) << b
        ijk[1] |= ((code >> (3 * b + 1)) & 1) << b
        ijk[2] |= ((code >> (3 * b)) & 1) << b
    return ijk


def octree_levels(leaf_c: np.ndarray, lo: float, size: float, leaf_depth):
    """Levels of the octree over [lo, lo+size]^3 with leaves centred at leaf_c
    (3, n_leaves) at depths leaf_depth (an int for a uniform tree, or one int
    per leaf).  Returns (max_depth, levels): levels[i] describes depth
    d = max_depth - i - 1 (from just above the deepest leaves up to the root)
    as a dict with
      dst_off   CSR over the boxes of depth d+1 (in Morton order): the children
                of each internal box of depth d
      c         centres (3, n_internal) of the internal boxes of depth d
      nodes     (kind, index) of every box of depth d in Morton order: kind 0
                = internal box (row of this level's output), 1 = leaf (row of
                the leaf coefficients)
    and the boxes of the deepest level are the leaves of that depth."""
    leaf_c = np.asarray(leaf_c, dtype=np.float64)
    nl = leaf_c.shape[1]
    depth = np.broadcast_to(np.asarray(leaf_depth, dtype=np.int64), (nl,)).copy()
    dmax = int(depth.max()) if nl else 0
    codes = np.zeros(nl, dtype=np.int64)
    for d in np.unique(depth):
        sel = depth == d
        h = size / (1 << int(d))
        ijk = np.rint((leaf_c[:, sel] - lo) / h - 0.5).astype(np.int64)
        if ijk.size and (ijk.min() < 0 or ijk.max() >= (1 << int(d))):
            raise ValueError("leaf centres outside the octree")
        codes[sel] = _morton(ijk, int(d))
    # boxes of the deepest level: its leaves, Morton order
    sel = np.nonzero(depth == dmax)[0]
    o = np.argsort(codes[sel], kind="stable")
    cur_codes = codes[sel][o]
    if np.any(np.diff(cur_codes) <= 0):
        raise ValueError("leaves overlap")
    levels = []
    for d in range(dmax - 1, -1, -1):
        pcode = cur_codes >> 3
        if np.any(np.diff(pcode) < 0):
            raise ValueError("boxes are not in Morton order")
        uniq, counts = np.unique(pcode, return_counts=True)
        off = np.zeros(len(uniq) + 1, dtype=np.int64)
        np.cumsum(counts, out=off[1:])
        h = size / (1 << d)
        c = lo + (_unmorton(uniq, d).astype(np.float64) + 0.5) * h
        # boxes of depth d: internal (uniq) and leaves of depth d, merged
        lsel = np.nonzero(depth == d)[0]
        all_codes = np.concatenate([uniq, codes[lsel]])
        kinds = [(0, i) for i in range(len(uniq))] + [(1, int(i)) for i in lsel]
        o = np.argsort(all_codes, kind="stable")
        if np.any(np.diff(all_codes[o]) <= 0):
            raise ValueError("a leaf overlaps an internal box")
        levels.append(dict(dst_off=off, c=c, nodes=[kinds[i] for i in o], codes=all_codes[o]))
        cur_codes = all_codes[o]
    return dmax, levels


class Upward:
    """Upward pass: run(leaf_coef) returns the coefficients of the internal
    boxes of every depth, from just above the deepest leaves to the root (the
    last entry, one row about the cube centre).  For a uniform tree the
    boxes of a level are all internal."""

    def __init__(self, plan: Plan, leaf_c, lo: float, size: float, leaf_depth, p: int = None, device="cuda"):
        self.plan = plan
        self.p = plan.p_max if p is None else int(p)
        lc = leaf_c.detach().cpu().numpy() if torch.is_tensor(leaf_c) else np.asarray(leaf_c)
        ld = leaf_depth.detach().cpu().numpy() if torch.is_tensor(leaf_depth) else leaf_depth
        self.max_depth, self.levels = octree_levels(lc, lo, size, ld)
        nl = lc.shape[1]
        nc = (self.p + 1) ** 2
        self.leaf_c = torch.as_tensor(np.ascontiguousarray(lc), dtype=torch.float64, device=device)
        depth = np.broadcast_to(np.asarray(ld, dtype=np.int64), (nl,))
        # sources of the first translation: the deepest leaves in Morton order
        deep = self._deepest_rows(lc, lo, size, depth)
        self.identity = len(deep) == nl and bool(np.array_equal(deep, np.arange(nl)))
        self.deep_idx = torch.from_numpy(deep).to(device)
        self.dev = []
        # per level: the distinct shifts t = c_src - c_dst of its translations
        # (eight on an octree level) and each source's shift, so that R(t) is
        # computed once for the tree (q2x_translation_rows) instead of once
        # per translation and pass
        self.rt = []
        src_c_h = lc[:, deep]
        for lv in self.levels:
            off = torch.from_numpy(lv["dst_off"]).to(device)
            c = torch.from_numpy(np.ascontiguousarray(lv["c"])).to(device)
            out = torch.empty((c.shape[1], nc), dtype=torch.float64, device=device)
            dest = np.repeat(np.arange(lv["c"].shape[1]), np.diff(lv["dst_off"]))
            t = src_c_h - lv["c"][:, dest]
            t_tab, t_idx = np.unique(t.T, axis=0, return_inverse=True)
            rt = plan.translation_rows(torch.from_numpy(np.ascontiguousarray(t_tab.T)).to(device), self.p)
            self.rt.append((rt, torch.from_numpy(t_idx.reshape(-1).astype(np.int32)).to(device)))
            # the boxes of this depth as the next level's sources, gathered
            # from [internal rows of this level; leaf rows]
            n_int = c.shape[1]
            gidx = np.array([k if kind == 0 else n_int + k for kind, k in lv["nodes"]], dtype=np.int64)
            if len(gidx) == n_int and np.array_equal(gidx, np.arange(n_int)):
                self.dev.append((off, c, out, None, None))
                src_c_h = lv["c"]
            else:
                allc = np.concatenate([lv["c"], lc], axis=1)
                nodes_c = torch.from_numpy(np.ascontiguousarray(allc[:, gidx])).to(device)
                self.dev.append((off, c, out, torch.from_numpy(gidx).to(device), nodes_c))
                src_c_h = allc[:, gidx]

    @staticmethod
    def _deepest_rows(lc, lo, size, depth):
        dmax = int(depth.max())
        sel = np.nonzero(depth == dmax)[0]
        h = size / (1 << dmax)
        codes = _morton(np.rint((lc[:, sel] - lo) / h - 0.5).astype(np.int64), dmax)
        return sel[np.argsort(codes, kind="stable")].astype(np.int64)

    def capture(self, leaf_coef):
        """Record the pass on the buffer `leaf_coef` as one CUDA graph (one
        eager run first sizes the plan's workspace).  `replay()` then re-runs
        the whole pass -- every level's kernels -- with one launch from the
        host, reading whatever `leaf_coef` holds at that time; it returns the
        same list of per-level tensors as `run`."""
        self.run(leaf_coef)
        torch.cuda.synchronize()
        side = torch.cuda.Stream()
        old = self.plan._stream
        self.plan.set_stream(side)
        graph = torch.cuda.CUDAGraph()
        try:
            with torch.cuda.graph(graph, stream=side):
                outs = self.run(leaf_coef)
        finally:
            self.plan.set_stream(old)
        self._graph, self._graph_outs = graph, outs
        return outs

    def replay(self):
        """Replay the captured pass on the current stream."""
        if getattr(self, "_graph", None) is None:
            raise RuntimeError("capture() the pass first")
        self._graph.replay()
        return self._graph_outs

    def run(self, leaf_coef, precomputed_shifts=True):
        """The pass over the leaf rows leaf_coef (one row per leaf, in the
        order of leaf_c); returns one tensor per depth, root last.  With
        precomputed_shifts=False each translation builds its own R(t)
        (q2x_translate) instead of reading the tree's shift rows."""
        src = leaf_coef if self.identity else leaf_coef.index_select(0, self.deep_idx)
        src_c = self.leaf_c if self.identity else self.leaf_c.index_select(1, self.deep_idx)
        outs = []
        for (off, c, out, gidx, nodes_c), (rt, t_idx) in zip(self.dev, self.rt):
            if precomputed_shifts:
                self.plan.translate_rt(src, rt, t_idx, off, dst_coef=out, p=self.p)
            else:
                self.plan.translate(src, src_c, off, c, dst_coef=out, p=self.p)
            outs.append(out)
            if gidx is None:
                src, src_c = out, c
            else:
                src = torch.cat([out, leaf_coef], dim=0).index_select(0, gidx)
                src_c = nodes_c
        return outs
