"""Host-side octree preparation of the upward pass (no GPU): the levels of
uniform and adaptive trees, their child -> parent CSR ranges, box centres,
the merge of leaves with internal boxes, the shifts each level's
translations need (eight per octree level), and the errors on overlapping
or out-of-range leaves."""
import numpy as np
import pytest

from paper_2107_10942_gb300.upward import _morton, _unmorton, octree_levels


def _uniform_leaves(depth, lo, size, frac, seed):
    rng = np.random.default_rng(seed)
    n = 1 << depth
    ijk = np.stack(np.meshgrid(*[np.arange(n)] * 3, indexing="ij")).reshape(3, -1)
    keep = rng.random(ijk.shape[1]) < frac
    h = size / n
    return lo + (ijk[:, keep] + 0.5) * h


def test_morton_roundtrip():
    rng = np.random.default_rng(1)
    for d in (1, 3, 7, 12):
        ijk = rng.integers(0, 1 << d, size=(3, 500))
        assert np.array_equal(_unmorton(_morton(ijk, d), d), ijk)


def _check_tree(leaf_c, lo, size, depth_of_leaf):
    dmax, levels = octree_levels(leaf_c, lo, size, depth_of_leaf)
    nl = leaf_c.shape[1]
    depth = np.broadcast_to(np.asarray(depth_of_leaf), (nl,))
    assert len(levels) == dmax
    seen = np.zeros(nl, dtype=int)
    n_below = int(np.sum(depth == dmax))  # boxes of the deepest level: its leaves
    for i, lv in enumerate(levels):
        d = dmax - i - 1
        h = size / (1 << d)
        off, c = lv["dst_off"], lv["c"]
        assert off[0] == 0 and off[-1] == n_below and np.all(np.diff(off) >= 1) and np.all(np.diff(off) <= 8)
        # box centres on the depth-d grid inside the cube
        g = (c - lo) / h - 0.5
        assert np.allclose(g, np.rint(g)) and g.min() >= 0 and g.max() <= (1 << d) - 1
        # the boxes of this depth: internal boxes, then (merged in Morton order) this depth's leaves
        kinds = [k for k, _ in lv["nodes"]]
        assert kinds.count(0) == c.shape[1]
        for k, j in lv["nodes"]:
            if k == 1:
                assert depth[j] == d
                seen[j] += 1
        assert np.all(np.diff(lv["codes"]) > 0)
        n_below = len(lv["nodes"])
    assert n_below == 1  # the root
    assert np.all(seen[depth < dmax] == 1) and np.all(seen[depth == dmax] == 0)
    return dmax, levels


def test_uniform_tree_levels_and_shifts():
    lo, size, depth = -1.125, 2.25, 4
    lc = _uniform_leaves(depth, lo, size, 0.3, 2)
    dmax, levels = _check_tree(lc, lo, size, depth)
    assert dmax == depth
    # the sources of the first level are the leaves in Morton order; each
    # translation's shift is one of the eight child offsets (+-h/4 per axis)
    h = size / (1 << depth)
    codes = _morton(np.rint((lc - lo) / h - 0.5).astype(np.int64), depth)
    src = lc[:, np.argsort(codes, kind="stable")]
    for i, lv in enumerate(levels):
        dest = np.repeat(np.arange(lv["c"].shape[1]), np.diff(lv["dst_off"]))
        t = src - lv["c"][:, dest]
        hd = size / (1 << (dmax - i - 1))
        assert np.allclose(np.abs(t), hd / 4)
        assert len(np.unique(t.T, axis=0)) <= 8
        src = lv["c"]


def test_adaptive_tree_levels():
    lo, size = -1.0, 2.0
    deep = _uniform_leaves(3, lo, size, 1.0, 3)
    # replace the boxes of one depth-1 octant by a single depth-1 leaf, and one
    # depth-2 box by a depth-2 leaf
    h1, h2 = size / 2, size / 4
    in_oct = np.all(deep < lo + h1, axis=0)
    c1 = np.full((3, 1), lo + 0.5 * h1)
    box2 = np.all((deep >= lo + h1) & (deep < lo + h1 + h2), axis=0)
    c2 = np.full((3, 1), lo + h1 + 0.5 * h2)
    keep = ~(in_oct | box2)
    lc = np.concatenate([deep[:, keep], c1, c2], axis=1)
    depth = np.concatenate([np.full(keep.sum(), 3), [1, 2]])
    dmax, levels = _check_tree(lc, lo, size, depth)
    assert dmax == 3


def test_overlapping_or_outside_leaves_rejected():
    lo, size = -1.0, 2.0
    lc = _uniform_leaves(2, lo, size, 1.0, 4)
    with pytest.raises(ValueError):
        octree_levels(np.concatenate([lc, lc[:, :1]], axis=1), lo, size, 2)  # a leaf twice
    with pytest.raises(ValueError):
        octree_levels(lc + 2.0 * size, lo, size, 2)  # outside the cube
    # a depth-1 leaf over depth-2 leaves of the same octant
    oct1 = np.full((3, 1), lo + size / 4)
    with pytest.raises(ValueError):
        octree_levels(np.concatenate([lc, oct1], axis=1), lo, size, np.concatenate([np.full(lc.shape[1], 2), [1]]))
