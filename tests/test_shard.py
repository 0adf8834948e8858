"""Leaf sharding for several GPUs, on the CPU: the balanced contiguous leaf
partition, shard extraction (vertex compaction, halo vertices duplicated),
the weak-scaling replication, and a world_size-2 gloo run in which each rank
computes its shard with the oracle, the blocks are assembled by
gather_coefficients, and the step time is the max over ranks.  Leaves are
independent (Eq. st4), so the assembled result equals the oracle on the whole
problem bit for bit (the oracle sums each leaf alone, in element order)."""
import os
import socket

import numpy as np
import pytest

import workloads as W
from paper_2107_10942_gb300 import shard as S


def small_sphere(density="linear"):
    if density == "linear":
        prob = W.cfg_sphere_linear(level=3, depth=3, p=4)
    else:
        prob = W.cfg_sphere_const(level=3, depth=3, p=4)
    return prob


def test_partition_is_contiguous_and_balanced():
    rng = np.random.default_rng(0)
    for trial in range(50):
        n = int(rng.integers(0, 200))
        cost = rng.integers(0, 1000, size=n).astype(np.float64)
        if trial % 5 == 0 and n:
            cost[rng.integers(0, n)] = 50000.0  # one dominant leaf
        for world in (1, 2, 3, 8):
            b = S.partition_leaves(cost, world)
            assert b[0] == 0 and b[-1] == n and np.all(np.diff(b) >= 0)
            per = [cost[b[r]:b[r + 1]].sum() for r in range(world)]
            assert abs(sum(per) - cost.sum()) < 1e-6
            bound = cost.sum() / world + (cost.max() if n else 0.0)
            assert max(per) <= bound + 1e-9


def test_partition_equal_costs_splits_evenly():
    b = S.partition_leaves(np.ones(12), 4)
    assert list(b) == [0, 3, 6, 9, 12]
    b = S.partition_leaves(np.ones(10), 3)
    assert np.all(np.abs(np.diff(b) - 10 / 3) < 1)
    with pytest.raises(ValueError):
        S.partition_leaves(np.ones(3), 0)


def test_leaf_costs_levels():
    off = np.array([0, 2, 2, 7])
    lp = np.array([3, 5, 1])
    c = S.leaf_costs(off, lp, "triangle", "linear", layers=2)
    assert list(c) == [2 * 16 * 6, 0, 5 * 4 * 6]
    assert list(S.leaf_costs(off, lp, "segment")) == [2 * 16 * 2, 0, 5 * 4 * 2]
    assert list(S.leaf_costs(off, lp, "tetra")) == [2 * 16 * 4, 0, 5 * 4 * 4]


@pytest.mark.parametrize("density", ["const", "linear"])
def test_shards_reproduce_the_whole_problem(orc, density):
    prob = small_sphere(density)
    dens = 1 if density == "linear" else 0
    full = orc.moments("triangle", prob["vxyz"], prob["idx"], prob["sigma"], prob["p"], leaf_off=prob["leaf_off"],
                       leaf_c=prob["leaf_c"], density=dens)
    cost = S.leaf_costs(prob["leaf_off"], prob["leaf_p"], "triangle", density)
    b = S.partition_leaves(cost, 3)
    parts = []
    shared = 0
    for r in range(3):
        sh = S.shard_problem(prob, b[r], b[r + 1])
        assert sh["leaf_range"] == (b[r], b[r + 1])
        assert sh["idx"].max(initial=-1) < sh["vxyz"].shape[1]
        # every shard vertex is one of the original vertices, at the same place
        e0, e1 = prob["leaf_off"][b[r]], prob["leaf_off"][b[r + 1]]
        assert np.array_equal(sh["vxyz"][:, sh["idx"]], prob["vxyz"][:, prob["idx"][:, e0:e1]])
        shared += sh["vxyz"].shape[1]
        parts.append(orc.moments("triangle", sh["vxyz"], sh["idx"], sh["sigma"], sh["p"],
                                 leaf_off=sh["leaf_off"], leaf_c=sh["leaf_c"], density=dens))
    assert np.array_equal(np.concatenate(parts, axis=0), full)
    # a closed mesh cut into pieces duplicates the vertices on the cuts
    assert shared > prob["vxyz"].shape[1]


def test_replicate_problem(orc):
    prob = small_sphere("const")
    rep = S.replicate_problem(prob, 3)
    nl = prob["leaf_c"].shape[1]
    assert rep["leaf_c"].shape[1] == 3 * nl and rep["idx"].shape[1] == 3 * prob["idx"].shape[1]
    one = orc.moments("triangle", prob["vxyz"], prob["idx"], prob["sigma"], prob["p"], leaf_off=prob["leaf_off"],
                      leaf_c=prob["leaf_c"])
    three = orc.moments("triangle", rep["vxyz"], rep["idx"], rep["sigma"], rep["p"], leaf_off=rep["leaf_off"],
                        leaf_c=rep["leaf_c"])
    assert np.array_equal(three, np.tile(one, (3, 1)))
    b = S.partition_leaves(S.leaf_costs(rep["leaf_off"], rep["leaf_p"]), 3)
    assert list(b) == [0, nl, 2 * nl, 3 * nl]


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank_main(rank, world, port, out_path):
    import time

    import torch
    import torch.distributed as dist
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    import oracle as orc
    prob = small_sphere("linear")
    rep = S.replicate_problem(prob, world)  # weak scaling: one copy per rank
    b = S.partition_leaves(S.leaf_costs(rep["leaf_off"], rep["leaf_p"], "triangle", "linear", 2), world)
    sh = S.shard_problem(rep, b[rank], b[rank + 1])
    dist.barrier()
    t0 = time.perf_counter()
    mine = orc.moments("triangle", sh["vxyz"], sh["idx"], sh["sigma"], sh["p"], leaf_off=sh["leaf_off"],
                       leaf_c=sh["leaf_c"], density=1, nthreads=1)
    dt = time.perf_counter() - t0
    dist.barrier()
    t = torch.tensor([dt], dtype=torch.float64)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    full = S.gather_coefficients(torch.from_numpy(mine), b)
    if rank == 0:
        np.save(out_path, full.numpy())
        with open(out_path + ".txt", "w") as f:
            f.write("%r %r %d\n" % (float(t.item()), dt, sh["leaf_c"].shape[1]))
    dist.barrier()
    dist.destroy_process_group()


def test_two_ranks_gloo(orc, tmp_path):
    import torch.multiprocessing as mp
    out = str(tmp_path / "coef.npy")
    mp.start_processes(_rank_main, args=(2, _free_port(), out), nprocs=2, join=True, start_method="spawn")
    got = np.load(out)
    prob = small_sphere("linear")
    one = orc.moments("triangle", prob["vxyz"], prob["idx"], prob["sigma"], prob["p"], leaf_off=prob["leaf_off"],
                      leaf_c=prob["leaf_c"], density=1)
    assert np.array_equal(got, np.tile(one, (2, 1)))
    tmax, t0, nl0 = open(out + ".txt").read().split()
    assert float(tmax) >= float(t0) and int(nl0) == prob["leaf_c"].shape[1]
