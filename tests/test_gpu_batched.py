"""Batched uneven instances (one call, worker streams, CUDA-graph capture) against the oracle."""
import numpy as np
import pytest

import oracle
import paper_2603_20912_gb300 as lad
from ladder_inputs import batched_shapes, make_inputs
from conftest import rel_fro
from test_gpu_fp64 import check_sampled

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")
EMU = lad.LADDER_EMU_BF16


@pytest.fixture(scope="module", autouse=True)
def _built():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2603_20912_gb300 import build
    build.build()


SMALL = [(5, 19, 72), (3, 37, 45), (7, 24, 93), (2, 61, 40), (6, 9, 30), (4, 50, 120)]


def _make(shapes, seed0=500):
    host = [make_inputs(o, v, x, seed=seed0 + k)[:2] for k, (o, v, x) in enumerate(shapes)]
    Ls = [torch.from_numpy(L).cuda() for L, _ in host]
    ts = [torch.from_numpy(t).cuda() for _, t in host]
    return host, Ls, ts


@pytest.mark.parametrize("precision,tol", [(lad.LADDER_FP64, 1e-12), (EMU, 1e-10)])
def test_small_batch_matches_oracle_per_instance(precision, tol):
    host, Ls, ts = _make(SMALL)
    plan = lad.ladder_plan_batched([s[0] for s in SMALL], [s[1] for s in SMALL], [s[2] for s in SMALL], precision)
    Rs = [torch.zeros_like(t) for t in ts]
    lad.ladder_apply_batched(plan, Ls, ts, Rs)
    torch.cuda.synchronize()
    assert plan.last_status() == lad.LADDER_OK
    for (L, t), R in zip(host, Rs):
        assert rel_fro(R.cpu().numpy(), oracle.ladder(L, t)) <= tol


def test_batched_equals_single_plans_bitwise():
    host, Ls, ts = _make(SMALL)
    plan = lad.ladder_plan_batched([s[0] for s in SMALL], [s[1] for s in SMALL], [s[2] for s in SMALL], EMU)
    Rs = [torch.zeros_like(t) for t in ts]
    lad.ladder_apply_batched(plan, Ls, ts, Rs)
    for (o, v, x), L, t, R in zip(SMALL, Ls, ts, Rs):
        single = lad.ladder_plan(o, v, x, EMU)
        R1 = torch.zeros_like(t)
        lad.ladder_apply(single, L, t, R1)
        torch.cuda.synchronize()
        assert torch.equal(R, R1)


def test_tuner_picks_a_schedule_and_results_stay_exact():
    host, Ls, ts = _make(SMALL)
    plan = lad.ladder_plan_batched([s[0] for s in SMALL], [s[1] for s in SMALL], [s[2] for s in SMALL], EMU)
    ws = plan.workspace()
    scratch = [torch.zeros_like(t) for t in ts]
    k = lad.ladder_tune_batched(plan, Ls, ts, scratch, ws)
    assert k in (1, 2, 4, 6) or k < 0   # streams, or minus the number of groups
    assert plan.batched_choice()["ladder_tile"] in (96, 64)
    Rs = [torch.zeros_like(t) for t in ts]
    lad.ladder_apply_batched(plan, Ls, ts, Rs, ws)
    torch.cuda.synchronize()
    for (L, t), R in zip(host, Rs):
        assert rel_fro(R.cpu().numpy(), oracle.ladder(L, t)) <= 1e-10


def test_graph_capture_and_replay_is_deterministic():
    host, Ls, ts = _make(SMALL)
    plan = lad.ladder_plan_batched([s[0] for s in SMALL], [s[1] for s in SMALL], [s[2] for s in SMALL], EMU)
    ws = plan.workspace()
    Rs = [torch.zeros_like(t) for t in ts]
    s = torch.cuda.Stream()
    s.wait_stream(torch.cuda.current_stream())
    with torch.cuda.stream(s):
        lad.ladder_apply_batched(plan, Ls, ts, Rs, ws, stream=s)   # warm-up outside capture
    torch.cuda.synchronize()
    g = torch.cuda.CUDAGraph()
    with torch.cuda.graph(g, stream=s):
        for R in Rs:
            R.zero_()
        lad.ladder_apply_batched(plan, Ls, ts, Rs, ws, stream=s)
    outs = []
    for _ in range(2):
        g.replay()
        torch.cuda.synchronize()
        outs.append([R.clone() for R in Rs])
    for a, b in zip(*outs):
        assert torch.equal(a, b)
    for (L, t), R in zip(host, outs[0]):
        assert rel_fro(R.cpu().numpy(), oracle.ladder(L, t)) <= 1e-10


@pytest.fixture(autouse=True)
def _release_cached_memory():
    yield
    torch.cuda.empty_cache()   # batched workspaces are large; later tests plan from free memory


def test_uneven_24_instance_batch_sampled_parity():
    shapes = batched_shapes()
    assert len(shapes) == 24
    host = [make_inputs(s.no, s.nv, s.nchol, s.seed)[:2] for s in shapes]
    Ls = [torch.from_numpy(L).cuda() for L, _ in host]
    ts = [torch.from_numpy(t).cuda() for _, t in host]
    plan = lad.ladder_plan_batched([s.no for s in shapes], [s.nv for s in shapes], [s.nchol for s in shapes], EMU)
    Rs = [torch.zeros_like(t) for t in ts]
    lad.ladder_apply_batched(plan, Ls, ts, Rs)
    torch.cuda.synchronize()
    assert plan.last_status() == lad.LADDER_OK
    for k, ((L, t), R) in enumerate(zip(host, Rs)):
        check_sampled(R.cpu().numpy(), L, t, 1e-10, nsample=8, seed=k)


@pytest.mark.parametrize("schedule", [-1, -2, -4, 1, 3])
def test_every_schedule_gives_the_same_bits(schedule):
    # grouped (one ERI and one ladder launch per shape over all instances of a group) and
    # worker-stream schedules: exact integer sums make every schedule bit-identical
    shapes = SMALL + [(12, 40, 60), (2, 88, 50)]   # both ladder shapes (o^2 > 128 and <= 128)
    host, Ls, ts = _make(shapes, seed0=900)
    plan = lad.ladder_plan_batched([s[0] for s in shapes], [s[1] for s in shapes], [s[2] for s in shapes], EMU)
    ws = plan.workspace()
    ref = []
    for (o, v, x), L, t in zip(shapes, Ls, ts):
        single = lad.ladder_plan(o, v, x, EMU)
        R1 = torch.zeros_like(t)
        lad.ladder_apply(single, L, t, R1)
        ref.append(R1)
    got = lad.ladder_batched_schedule(plan, schedule)
    if schedule < 0:
        assert got < 0
        if schedule == -1:
            assert got == -1                   # all instances in one group
    Rs = [torch.zeros_like(t) for t in ts]
    lad.ladder_apply_batched(plan, Ls, ts, Rs, ws)
    torch.cuda.synchronize()
    assert plan.last_status() == lad.LADDER_OK
    for R, R1 in zip(Rs, ref):
        assert torch.equal(R, R1)


@pytest.mark.parametrize("bn", [16, 48, 64, 80])
def test_ladder_tile_width_does_not_change_a_bit(bn):
    # one-SM ladder (no^2 <= 128) in both forms: exact integer sums, any column tile width
    for (o, v, x), form in (((7, 61, 90), 0), ((10, 47, 70), 1)):
        L, t2, _, _ = make_inputs(o, v, x, seed=bn + v)
        Ld, td = torch.from_numpy(L).cuda(), torch.from_numpy(t2).cuda()
        out = []
        for width in (96, bn):
            plan = lad.ladder_plan(o, v, x, EMU)
            plan.set_form(form)
            plan.set_ladder_tile(width)
            assert plan.ladder_tile() == width
            R = torch.zeros_like(td)
            lad.ladder_apply(plan, Ld, td, R)
            torch.cuda.synchronize()
            assert plan.last_status() == lad.LADDER_OK
            out.append(R)
        assert torch.equal(out[0], out[1])
        assert rel_fro(out[1].cpu().numpy(), oracle.ladder(L, t2)) <= 1e-10
    plan = lad.ladder_plan(3, 20, 30, EMU)
    for bad in (0, 8, 40, 112):
        with pytest.raises(lad.LadderError):
            plan.set_ladder_tile(bad)


def test_tuned_choice_is_bit_identical_to_single_plans():
    # the tuner varies schedule, batch split and ladder tile width; whatever it keeps, every
    # instance's R equals its single-plan R bit for bit
    shapes = SMALL + [(12, 40, 60), (2, 88, 50)]
    host, Ls, ts = _make(shapes, seed0=950)
    plan = lad.ladder_plan_batched([s[0] for s in shapes], [s[1] for s in shapes], [s[2] for s in shapes], EMU)
    ws = plan.workspace()
    scratch = [torch.zeros_like(t) for t in ts]
    lad.ladder_tune_batched(plan, Ls, ts, scratch, ws)
    assert plan.batched_choice()["ladder_tile"] in (96, 64)
    Rs = [torch.zeros_like(t) for t in ts]
    lad.ladder_apply_batched(plan, Ls, ts, Rs, ws)
    torch.cuda.synchronize()
    assert plan.last_status() == lad.LADDER_OK
    for (o, v, x), L, t, R in zip(shapes, Ls, ts, Rs):
        single = lad.ladder_plan(o, v, x, EMU)
        R1 = torch.zeros_like(t)
        lad.ladder_apply(single, L, t, R1)
        torch.cuda.synchronize()
        assert torch.equal(R, R1)


def test_split_form_instances_share_a_group_bit_for_bit():
    # instances that take the symmetric/antisymmetric form (no = 20, 24 at these sizes) join the
    # group: one ERI launch, their combine passes, one ladder launch with their X and Y items
    # beside the plain instances' items; exact integer sums, so the bits of single plans
    pm = [(20, 12, 8), (20, 16, 12), (24, 28, 40)]
    for o, v, x in pm:
        assert lad.ladder_form_model(o, v, x, 0) == 1
    shapes = SMALL + pm
    host, Ls, ts = _make(shapes, seed0=1300)
    plan = lad.ladder_plan_batched([s[0] for s in shapes], [s[1] for s in shapes], [s[2] for s in shapes], EMU)
    ws = plan.workspace()
    assert lad.ladder_batched_schedule(plan, -1) == -1   # one group of all nine instances
    Rs = [torch.zeros_like(t) for t in ts]
    lad.ladder_apply_batched(plan, Ls, ts, Rs, ws)
    torch.cuda.synchronize()
    assert plan.last_status() == lad.LADDER_OK
    for (o, v, x), (L, t), Ld, td, R in zip(shapes, host, Ls, ts, Rs):
        single = lad.ladder_plan(o, v, x, EMU)
        R1 = torch.zeros_like(td)
        lad.ladder_apply(single, Ld, td, R1)
        torch.cuda.synchronize()
        assert torch.equal(R, R1)
        assert rel_fro(R.cpu().numpy(), oracle.ladder(L, t)) <= 1e-10
