"""Data-parallel sharding of one contraction's block pairs over ranks.

The (A,B) block pairs are independent and write disjoint parts of R, so ranks
need no exchange on the data path; E_L, linear in R, is one scalar all-reduce.
These CPU tests run the host side: the partition (ladder_shard_blocks) and, with
two gloo ranks, the per-rank contraction of the owned pairs (by the oracle) and
the energy all-reduce.  The GPU side (ladder_plan_shard) is in test_gpu_shard.py.
"""
import os
import socket

import numpy as np
import pytest

import oracle
import paper_2603_20912_gb300 as lad
from ladder_inputs import make_inputs

torch = pytest.importorskip("torch")


def test_partition_is_deterministic_longest_first():
    npairs = [10, 40, 40, 5, 25, 25, 3]
    owner = lad.ladder_shard_blocks(npairs, 3)
    assert owner == lad.ladder_shard_blocks(npairs, 3)
    # longest first to the least-loaded rank, ties to the lower rank and by position
    assert owner == [0, 0, 1, 1, 2, 2, 1]
    loads = [sum(n for n, o in zip(npairs, owner) if o == r) for r in range(3)]
    assert max(loads) - min(loads) <= max(npairs)
    assert lad.ladder_shard_blocks(npairs, 1) == [0] * len(npairs)
    assert sorted(lad.ladder_shard_blocks([7, 7], 4)) == [0, 1]   # ranks 2, 3 own nothing
    assert lad.ladder_shard_blocks([], 2) == []
    with pytest.raises(lad.LadderError):
        lad.ladder_shard_blocks([1, 2], 0)


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank_main(rank, world, port, out_dir):
    import torch.distributed as dist
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        no, nv, nchol = 3, 23, 30
        L, t2, _, _ = make_inputs(no, nv, nchol, seed=77)
        plan = lad.ladder_plan_dry(no, nv, nchol, force_n_a=8, force_n_b=6)
        owner = lad.ladder_shard_blocks([b[4] for b in plan["blocks"]], world)
        pairs = [(a, b) for (a0, a1, b0, b1, _), o in zip(plan["blocks"], owner) if o == rank
                 for a in range(a0, a1) for b in range(max(a, b0), b1)]
        Rp = np.zeros_like(t2)
        if pairs:
            out = oracle.ladder_pairs(L, t2, [p[0] for p in pairs], [p[1] for p in pairs])
            for k, (a, b) in enumerate(pairs):
                Rp[:, :, a, b] = out[k]
                if a < b:
                    Rp[:, :, b, a] = out[k].T      # R_ji^ba = R_ij^ab
        E = torch.tensor([oracle.energy(t2, Rp)], dtype=torch.float64)
        dist.all_reduce(E)                          # the only exchange: one scalar
        R = torch.from_numpy(Rp.copy())
        dist.all_reduce(R)                          # test-only assembly, to check disjointness
        counts = [torch.zeros(1, dtype=torch.int64) for _ in range(world)]
        dist.all_gather(counts, torch.tensor([len(pairs)], dtype=torch.int64))
        if rank == 0:
            np.savez(os.path.join(out_dir, "r0.npz"), E=E.numpy(), R=R.numpy(),
                     counts=np.array([int(c) for c in counts]))
    finally:
        dist.destroy_process_group()


def test_two_gloo_ranks_cover_every_pair_once_and_reduce_the_energy(tmp_path):
    import torch.multiprocessing as mp
    world = 2
    mp.spawn(_rank_main, args=(world, _free_port(), str(tmp_path)), nprocs=world, join=True)
    res = np.load(tmp_path / "r0.npz")
    L, t2, _, _ = make_inputs(3, 23, 30, seed=77)
    full = oracle.ladder(L, t2)
    # every a <= b pair owned by exactly one rank, loads balanced within one block
    assert int(res["counts"].sum()) == 23 * 24 // 2
    assert abs(int(res["counts"][0]) - int(res["counts"][1])) <= 8 * 6
    # disjoint parts: their sum is the full R (mirrors agree with the direct sums to rounding)
    assert np.max(np.abs(res["R"] - full)) <= 1e-13 * np.max(np.abs(full))
    assert float(res["E"][0]) == pytest.approx(oracle.energy(t2, full), rel=1e-12)


def _shard_rank_main(rank, world, port, out_dir, precision):
    """One gloo rank: its block pairs from the library's own shard selection (ladder_plan_shard's
    host logic, run without a GPU), the oracle's contraction of those pairs, E_L all-reduced."""
    import torch.distributed as dist
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        no, nv, nchol = 3, 29, 40
        L, t2, _, _ = make_inputs(no, nv, nchol, seed=78)
        # the default plan of this shape is one block pair: the shard selection re-blocks
        mine = lad.ladder_plan_shard_dry(no, nv, nchol, rank, world, precision=precision)
        pairs = [(a, b) for (a0, a1, b0, b1, _) in mine["blocks"]
                 for a in range(a0, a1) for b in range(max(a, b0), b1)]
        Rp = np.zeros_like(t2)
        if pairs:
            out = oracle.ladder_pairs(L, t2, [p[0] for p in pairs], [p[1] for p in pairs])
            for k, (a, b) in enumerate(pairs):
                Rp[:, :, a, b] = out[k]
                if a < b:
                    Rp[:, :, b, a] = out[k].T
        E = torch.tensor([oracle.energy(t2, Rp)], dtype=torch.float64)
        dist.all_reduce(E)
        owned = torch.zeros(nv, nv, dtype=torch.int64)
        for a, b in pairs:
            owned[a, b] += 1
        dist.all_reduce(owned)
        blocks = [torch.zeros(1, dtype=torch.int64) for _ in range(world)]
        dist.all_gather(blocks, torch.tensor([mine["n_block_pairs"]], dtype=torch.int64))
        if rank == 0:
            np.savez(os.path.join(out_dir, f"shard{precision}.npz"), E=E.numpy(), owned=owned.numpy(),
                     blocks=np.array([int(b) for b in blocks]), na=mine["n_a"], nb=mine["n_b"])
    finally:
        dist.destroy_process_group()


@pytest.mark.parametrize("precision", [lad.LADDER_FP64, lad.LADDER_EMU_BF16])
def test_two_gloo_ranks_shard_through_the_library_planner(tmp_path, precision):
    import torch.multiprocessing as mp
    world = 2
    no, nv, nchol = 3, 29, 40
    assert lad.ladder_plan_dry(no, nv, nchol, precision)["n_block_pairs"] == 1
    mp.spawn(_shard_rank_main, args=(world, _free_port(), str(tmp_path), precision), nprocs=world, join=True)
    res = np.load(tmp_path / f"shard{precision}.npz")
    owned = res["owned"]
    # every a <= b pair exactly once over the ranks, nothing below the diagonal
    iu = np.triu_indices(nv)
    assert np.all(owned[iu] == 1)
    assert int(owned.sum()) == nv * (nv + 1) // 2
    # re-blocked to at least two block pairs per rank, each rank holding some
    assert int(res["blocks"].sum()) >= 2 * world and np.all(res["blocks"] >= 1)
    L, t2, _, _ = make_inputs(no, nv, nchol, seed=78)
    assert float(res["E"][0]) == pytest.approx(oracle.energy(t2, oracle.ladder(L, t2)), rel=1e-12)
    # the library's shard of rank r equals its partition of the re-selected blocking
    both = [lad.ladder_plan_shard_dry(no, nv, nchol, r, world, precision=precision) for r in range(world)]
    whole = lad.ladder_plan_dry(no, nv, nchol, precision, force_n_a=both[0]["n_a"], force_n_b=both[0]["n_b"])
    owner = lad.ladder_shard_blocks([b[4] for b in whole["blocks"]], world)
    for r in range(world):
        assert both[r]["blocks"] == [blk for blk, o in zip(whole["blocks"], owner) if o == r]
    with pytest.raises(lad.LadderError):
        lad.ladder_plan_shard_dry(no, nv, nchol, 2, 2)
