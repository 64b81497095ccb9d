"""C-ABI library checks that need no GPU: it loads, exports every symbol the
headers declare, and the host-side planner obeys its contract."""
import ctypes
import glob
import os
import re

import numpy as np
import pytest

import paper_2603_20912_gb300 as lad
from ladder_inputs import CONFIGS

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _declared_functions():
    names = set()
    for h in glob.glob(os.path.join(ROOT, "include", "*.h")):
        text = open(h).read()
        text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
        for m in re.finditer(r"^\s*[A-Za-z_][\w\s\*]*?\b([a-z_][a-z0-9_]*)\s*\(", text, flags=re.M):
            if m.group(1) not in ("if", "while", "for", "return", "sizeof"):
                names.add(m.group(1))
    return sorted(names)


@pytest.fixture(scope="module")
def lib():
    from paper_2603_20912_gb300 import build
    build.build()
    return lad.lib()


def test_library_exports_every_declared_symbol(lib):
    decl = _declared_functions()
    assert "ladder_apply" in decl and "ladder_plan" in decl and "ladder_energy" in decl
    for name in decl:
        assert hasattr(lib, name), f"{name} declared in include/ but not exported"
    for name in lad.EXPORTED_SYMBOLS:
        assert name in decl, f"binding exposes {name} which no header declares"


def test_strerror_and_flops(lib):
    for code in range(7):
        assert lad.ladder_strerror(code)
    assert "unknown" in lad.ladder_strerror(99)
    for no, nv, X in [(5, 19, 72), (10, 200, 630), (20, 400, 1260)]:
        p = nv * (nv + 1) / 2
        assert lad.ladder_flops(no, nv, X) == pytest.approx(2 * X * nv * nv * p + 2 * no * no * nv * nv * p, rel=1e-15)
    assert lad.ladder_flops(10, 200, 630) == pytest.approx(1.174e12, rel=2e-3)


def test_null_arguments_are_rejected_without_a_gpu(lib):
    vp = ctypes.c_void_p
    assert lib.ladder_plan(None, 5, 19, 72, 0, 0, 0, 0) == lad.LADDER_ERR_ARG
    h = vp()
    assert lib.ladder_plan(ctypes.byref(h), 0, 19, 72, 0, 0, 0, 0) == lad.LADDER_ERR_ARG
    assert lib.ladder_plan(ctypes.byref(h), 5, 19, 72, lad.LADDER_EMU_INT8, 0, 0, 0) == lad.LADDER_ERR_UNSUPPORTED
    assert lib.ladder_apply(None, None, None, None, None, None) == lad.LADDER_ERR_ARG
    assert lib.ladder_energy(None, None, None, None, None, None) == lad.LADDER_ERR_ARG
    assert lib.ladder_workspace_bytes(None) == 0
    assert lib.ladder_apply_host(None, None, None, None, None, None, None) == lad.LADDER_ERR_ARG
    assert lib.ladder_host_staging_bytes(None) == 0
    lib.ladder_plan_destroy(None)


def _coverage(nv, blocks):
    seen = np.zeros((nv, nv), dtype=np.int64)
    for a0, a1, b0, b1, n in blocks:
        cnt = 0
        for a in range(a0, a1):
            for b in range(max(a, b0), b1):
                seen[a, b] += 1
                cnt += 1
        assert cnt == n and n > 0
    return seen


@pytest.mark.parametrize("precision", [lad.LADDER_FP64, lad.LADDER_EMU_BF16])
@pytest.mark.parametrize("no,nv,nchol", [(5, 19, 72), (10, 200, 630), (20, 400, 1260), (3, 1, 2)])
def test_planner_default_budget_covers_every_pair_once(lib, precision, no, nv, nchol):
    r = lad.ladder_plan_dry(no, nv, nchol, precision, ws_budget_bytes=180 << 30)
    assert r["ws_bytes"] <= 180 << 30
    seen = _coverage(nv, r["blocks"])
    iu = np.triu_indices(nv)
    assert np.all(seen[iu] == 1)
    assert seen.sum() == nv * (nv + 1) // 2


@pytest.mark.parametrize("precision", [lad.LADDER_FP64, lad.LADDER_EMU_BF16])
def test_planner_honours_small_budgets(lib, precision):
    no, nv, nchol = 20, 400, 1260
    full = lad.ladder_plan_dry(no, nv, nchol, precision, ws_budget_bytes=1 << 42)
    last_ws = full["ws_bytes"]
    for frac in (0.5, 0.2, 0.05, 0.01):
        budget = int(full["ws_bytes"] * frac)
        try:
            r = lad.ladder_plan_dry(no, nv, nchol, precision, ws_budget_bytes=budget)
        except lad.LadderError as e:
            assert e.status == lad.LADDER_ERR_BUDGET
            continue
        assert r["ws_bytes"] <= budget
        assert r["n_block_pairs"] > 1
        seen = _coverage(nv, r["blocks"])
        assert np.all(seen[np.triu_indices(nv)] == 1) and seen.sum() == nv * (nv + 1) // 2
        last_ws = r["ws_bytes"]
    assert last_ws < full["ws_bytes"]


def test_planner_allows_and_chooses_asymmetric_blocks(lib):
    # A forced asymmetric blocking is valid and covers the triangle once.
    r = lad.ladder_plan_dry(4, 37, 20, lad.LADDER_FP64, ws_budget_bytes=1 << 40, force_n_a=5, force_n_b=11)
    assert (r["n_a"], r["n_b"]) == (5, 11)
    seen = _coverage(37, r["blocks"])
    assert np.all(seen[np.triu_indices(37)] == 1) and seen.sum() == 37 * 38 // 2
    # Execution order is b-blocks outer, a-blocks inner (the C-split loop nest).
    bs = [b[2] for b in r["blocks"]]
    assert bs == sorted(bs)
    # Over a sweep of budgets the cost model picks n_a != n_b somewhere.
    asym = False
    for budget_mb in (40, 80, 160, 320, 640, 1280, 2560):
        try:
            q = lad.ladder_plan_dry(20, 400, 1260, lad.LADDER_FP64, ws_budget_bytes=budget_mb << 20)
        except lad.LadderError:
            continue
        asym |= q["n_a"] != q["n_b"]
    assert asym


def test_planner_rejects_impossible_budget(lib):
    with pytest.raises(lad.LadderError) as e:
        lad.ladder_plan_dry(10, 200, 630, lad.LADDER_FP64, ws_budget_bytes=1024)
    assert e.value.status == lad.LADDER_ERR_BUDGET
    with pytest.raises(lad.LadderError) as e:
        lad.ladder_plan_dry(10, 200, 630, lad.LADDER_FP64, ws_budget_bytes=1 << 40, force_n_a=201, force_n_b=3)
    assert e.value.status == lad.LADDER_ERR_ARG


def test_planner_workspace_formula_fp64(lib):
    # FP64: the workspace is the packed V block of the largest block pair, v^2 doubles per pair.
    r = lad.ladder_plan_dry(10, 200, 630, lad.LADDER_FP64, ws_budget_bytes=1 << 40)
    maxp = max(b[4] for b in r["blocks"])
    assert r["ws_bytes"] >= maxp * 200 * 200 * 8
    assert r["ws_bytes"] < maxp * 200 * 200 * 8 + 4096
    # One batch at c2 when the budget allows the whole packed triangle (6.43 GB).
    assert r["n_block_pairs"] == 1 and maxp == 200 * 201 // 2


def test_form_model_decisions():
    # The split (symmetric/antisymmetric) form pays where the ladder is a large share of the call:
    # not at c1/c2 (100 (i,j) rows fill one 128-row tile; the combine pass costs more than it
    # saves), yes at c3 and at the paper-scale shapes (nocc = 100).
    assert lad.ladder_form_model(5, 19, 72) == 0
    assert lad.ladder_form_model(10, 200, 630) == 0
    assert lad.ladder_form_model(20, 400, 1260) == 1
    assert lad.ladder_form_model(100, 700, 4000) == 1
    assert lad.ladder_form_model(100, 800, 4500) == 1
    for bad in [(0, 5, 5, 0), (5, 0, 5, 0), (5, 5, 0, 0), (5, 5, 5, 4), (5, 5, 5, 9)]:
        with pytest.raises(lad.LadderError):
            lad.ladder_form_model(*bad)


def test_header_enum_values_match_the_binding():
    # every LADDER_* enumerator declared in include/ladder.h has the same value in the binding
    text = open(os.path.join(ROOT, "include", "ladder.h")).read()
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    found = {}
    for body in re.findall(r"enum\s*\{(.*?)\}", text, flags=re.S):
        for name, val in re.findall(r"(LADDER_[A-Z0-9_]+)\s*=\s*(\d+)", body):
            found[name] = int(val)
    assert {"LADDER_PATH_FUSED", "LADDER_KERNEL_FUSED", "LADDER_KERNEL_CLASSES"} <= set(found)
    for name, val in found.items():
        if name == "LADDER_KERNEL_CLASSES":
            continue
        assert getattr(lad, name) == val, name


def test_path_model_decisions(lib):
    # the factorised order R_ij = sum_P L_P T_ij L_P^T is taken for FP64 plans when it needs
    # 1.25x fewer flops than rebuilding (ac|bd): 4 X o(o+1)/2 v^3 against 2 X v^2 p + 2 o^2 v^2 p;
    # otherwise the rebuild fused on the chip when its accumulators hold no^2 <= 1024 rows
    def rule(no, nv, nchol):
        p = nv * (nv + 1) / 2
        eri = 2.0 * nchol * nv * nv * p + 2.0 * no * no * nv * nv * p
        fact = 4.0 * nchol * no * (no + 1) / 2 * nv ** 3
        return 1 if 1.25 * fact < eri else (2 if no * no <= 1024 else 0)
    for name, want in (("c1", 2), ("c2", 2), ("c3", 2)):
        s = CONFIGS[name]
        assert lad.ladder_path_model(s.no, s.nv, s.nchol, lad.LADDER_FP64) == want
    assert lad.ladder_path_model(12, 64, 8, lad.LADDER_FP64) == 1
    assert lad.ladder_path_model(33, 400, 1260, lad.LADDER_FP64) == 0
    for no in (1, 3, 10, 30, 33):
        for nv in (5, 40, 300):
            for nchol in (1, 8, 100, 1000):
                assert lad.ladder_path_model(no, nv, nchol, lad.LADDER_FP64) == rule(no, nv, nchol)
                assert lad.ladder_path_model(no, nv, nchol, lad.LADDER_EMU_BF16) == 0
    with pytest.raises(lad.LadderError):
        lad.ladder_path_model(0, 5, 5)


def test_dry_planner_batches_cholesky_vectors_when_their_planes_do_not_fit(lib):
    # L^T digit planes of all 20000 vectors: 12 x 64 x 64 x 20000 bytes = 983 MB > the budget;
    # sliced in batches they fit, and the workspace respects the budget
    no, nv, nchol = 2, 64, 20000
    budget = 700 * 10 ** 6
    d = lad.ladder_plan_dry(no, nv, nchol, lad.LADDER_EMU_BF16, ws_budget_bytes=budget)
    assert d["ws_bytes"] <= budget
    covered = sum(b[4] for b in d["blocks"])
    assert covered == nv * (nv + 1) // 2
    # at the default workload the planes fit with room to spare: no batches, the same blocking
    s = CONFIGS["c3"]
    d3 = lad.ladder_plan_dry(s.no, s.nv, s.nchol, lad.LADDER_EMU_BF16, ws_budget_bytes=int(0.88 * 280e9))
    assert (d3["n_a"], d3["n_b"]) == (400, 200)
