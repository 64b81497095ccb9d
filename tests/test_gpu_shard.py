"""Sharded plans (ladder_plan_shard) run one after another on one GPU: the shards'
R parts are disjoint and add up to the unsharded result, and their energies add
up to its E_L (the multi-GPU data path without the GPUs)."""
import numpy as np
import pytest

import oracle
import paper_2603_20912_gb300 as lad
from ladder_inputs import make_inputs
from conftest import rel_fro

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")


@pytest.fixture(scope="module", autouse=True)
def _built():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2603_20912_gb300 import build
    build.build()


def _run(plan, Ld, td):
    R = torch.zeros_like(td)
    lad.ladder_apply(plan, Ld, td, R)
    E = lad.ladder_energy(plan, td, R)
    torch.cuda.synchronize()
    assert plan.last_status() == lad.LADDER_OK
    return R, E


@pytest.mark.parametrize("precision", [lad.LADDER_FP64, lad.LADDER_EMU_BF16])
@pytest.mark.parametrize("world", [2, 3, 5])
def test_shards_add_up_to_the_whole(precision, world):
    no, nv, nchol = 4, 45, 60
    L, t2, _, _ = make_inputs(no, nv, nchol, seed=31)
    Ld, td = torch.from_numpy(L).cuda(), torch.from_numpy(t2).cuda()
    budget = 1 << 34
    full = lad.ladder_plan(no, nv, nchol, precision, ws_budget_bytes=budget)
    if precision == lad.LADDER_FP64:
        full.set_path(lad.LADDER_PATH_ERI)   # the shards run the rebuild order
    R_full, E_full = _run(full, Ld, td)
    R_sum = torch.zeros_like(td)
    E_sum = 0.0
    covered = 0
    for rank in range(world):
        plan = lad.ladder_plan(no, nv, nchol, precision, ws_budget_bytes=budget)
        plan.shard(rank, world)
        d = plan.describe()
        covered += d["n_block_pairs"]
        R, E = _run(plan, Ld, td)
        assert not torch.any((R != 0) & (R_sum != 0))   # disjoint entries
        R_sum += R
        E_sum += E
    assert covered >= 2 * world
    if precision == lad.LADDER_EMU_BF16:
        assert torch.equal(R_sum, R_full)   # exact integer sums: independent of the blocking
    else:
        assert rel_fro(R_sum.cpu().numpy(), R_full.cpu().numpy()) <= 1e-14
    assert E_sum == pytest.approx(E_full, rel=1e-12)
    assert rel_fro(R_sum.cpu().numpy(), oracle.ladder(L, t2)) <= (1e-12 if precision == lad.LADDER_FP64 else 1e-10)


def test_shard_rejections():
    plan = lad.ladder_plan(3, 20, 30, lad.LADDER_FP64, ws_budget_bytes=1 << 30)
    for rank, world in [(-1, 2), (2, 2), (0, 0)]:
        with pytest.raises(lad.LadderError):
            plan.shard(rank, world)
    plan.shard(1, 2)
    with pytest.raises(lad.LadderError):
        plan.shard(0, 2)
    with pytest.raises(lad.LadderError):
        plan.set_blocks(5, 5)
