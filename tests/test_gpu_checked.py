"""The index-checked build (-DLADDER_CHECK): every store of the emulated kernels into the
workspace and into R tests its index and, on failure, records LADDER_ERR_BOUNDS and skips
the store (no trap, no fault).  Small shapes covering the kernels' index paths - ragged tiles,
padded layouts, whole-sector V stores, both ladder shapes, forced blockings, the
symmetric/antisymmetric form (int64 V, combine pass, T' and T'' slices, two ladder items, four-way
finalisation) and the grouped batched schedule - must run with a clean status and the usual
parity."""
import json
import os
import subprocess
import sys

import pytest

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")
ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))

WORKLOAD = r"""
import json, numpy as np, torch
import oracle, paper_2603_20912_gb300 as lad
from ladder_inputs import make_inputs
assert lad.LIB_PATH.endswith("libladder_check.so"), lad.LIB_PATH
EMU = lad.LADDER_EMU_BF16
out = []

def rel(a, b):
    return float(np.linalg.norm((a - b).ravel()) / max(np.linalg.norm(b.ravel()), 1e-300))

cases = [(5, 19, 72, None), (1, 1, 1, None), (2, 1, 5, None), (4, 9, 1, None), (6, 65, 17, None),
         (3, 32, 50, None), (2, 47, 40, (5, 3)), (12, 40, 60, None), (3, 37, 45, (3, 7)), (3, 23, 1500, None)]
for no, nv, x, blocks in cases:
    L, t2, _, _ = make_inputs(no, nv, x, seed=no * 100 + nv)
    plan = lad.ladder_plan(no, nv, x, EMU)
    if blocks:
        plan.set_blocks(*blocks)
    R = torch.zeros(t2.shape, dtype=torch.float64, device="cuda")
    lad.ladder_apply(plan, torch.from_numpy(L).cuda(), torch.from_numpy(t2).cuda(), R)
    torch.cuda.synchronize()
    out.append({"shape": [no, nv, x], "status": plan.last_status(),
                "rel": rel(R.cpu().numpy(), oracle.ladder(L, t2))})

# the symmetric/antisymmetric form: odd and even nv, one tile and several, both ladder shapes
for no, nv, x, blocks in [(5, 19, 72, None), (1, 7, 9, None), (2, 1, 5, None), (4, 45, 60, (7, 3)),
                          (18, 30, 40, None), (3, 64, 70, None)]:
    L, t2, _, _ = make_inputs(no, nv, x, seed=no * 100 + nv + 1)
    plan = lad.ladder_plan(no, nv, x, EMU)
    plan.set_form(1)
    if blocks:
        plan.set_blocks(*blocks)
    R = torch.zeros(t2.shape, dtype=torch.float64, device="cuda")
    lad.ladder_apply(plan, torch.from_numpy(L).cuda(), torch.from_numpy(t2).cuda(), R)
    torch.cuda.synchronize()
    out.append({"shape": [no, nv, x, "pm"], "status": plan.last_status(),
                "rel": rel(R.cpu().numpy(), oracle.ladder(L, t2))})

shapes = [(5, 19, 72), (3, 37, 45), (12, 40, 60), (2, 88, 50)]
host = [make_inputs(o, v, x, seed=700 + k)[:2] for k, (o, v, x) in enumerate(shapes)]
plan = lad.ladder_plan_batched([s[0] for s in shapes], [s[1] for s in shapes], [s[2] for s in shapes], EMU)
lad.ladder_batched_schedule(plan, -1)
Rs = [torch.zeros(t.shape, dtype=torch.float64, device="cuda") for _, t in host]
lad.ladder_apply_batched(plan, [torch.from_numpy(L).cuda() for L, _ in host],
                         [torch.from_numpy(t).cuda() for _, t in host], Rs)
torch.cuda.synchronize()
out.append({"shape": "batch", "status": plan.last_status(),
            "rel": max(rel(R.cpu().numpy(), oracle.ladder(L, t)) for (L, t), R in zip(host, Rs))})
print(json.dumps(out))
"""


def test_checked_build_runs_clean():
    from paper_2603_20912_gb300 import build
    build.build(check=True)
    env = dict(os.environ, LADDER_CHECKED_LIBRARY="1")
    r = subprocess.run([sys.executable, "-c", WORKLOAD], env=env, cwd=ROOT, capture_output=True, text=True,
                       timeout=900)
    assert r.returncode == 0, r.stdout[-3000:] + r.stderr[-3000:]
    results = json.loads(r.stdout.strip().splitlines()[-1])
    assert len(results) == 17
    for res in results:
        assert res["status"] == 0, res
        assert res["rel"] <= 1e-10, res
