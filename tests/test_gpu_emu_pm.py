"""The symmetric/antisymmetric form of the emulated ladder (ladder_plan_set_form(plan, 1)):
the same contraction over c <= d and i <= j in two halves X (symmetric) and Y (antisymmetric),
against the oracle at the emulated tolerances, exact and blocking-independent like the plain form."""
import numpy as np
import pytest

import oracle
import paper_2603_20912_gb300 as lad
from ladder_inputs import CONFIGS, make_inputs
from conftest import rel_fro
from test_gpu_fp64 import check_sampled, dev, _golden, _golden_energy

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")
EMU = lad.LADDER_EMU_BF16
TOL_R = 1e-10
TOL_E = 1e-8


@pytest.fixture(scope="module", autouse=True)
def _built():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2603_20912_gb300 import build
    build.build()


def pm_ladder(L, t2, blocks=None, budget=0):
    nchol, nv, _ = L.shape
    no = t2.shape[0]
    torch.cuda.empty_cache()
    plan = lad.ladder_plan(no, nv, nchol, EMU, ws_budget_bytes=budget)
    plan.set_form(1)
    if blocks is not None:
        plan.set_blocks(*blocks)
    R = torch.zeros(t2.shape, dtype=torch.float64, device="cuda")
    lad.ladder_apply(plan, dev(L), dev(t2), R)
    torch.cuda.synchronize()
    assert plan.last_status() == lad.LADDER_OK
    return R.cpu().numpy(), plan


# X and Y on CTA pairs in one ladder launch (no = 18, 20), both on single CTAs (no = 12), and
# X on CTA pairs with Y on single CTAs in two launches (no = 16: 136 and 120 rows).
@pytest.mark.parametrize("no,nv,nchol", [(5, 19, 72), (1, 7, 9), (2, 1, 5), (3, 32, 50), (4, 45, 60),
                                         (18, 30, 40), (12, 47, 33), (3, 23, 1500), (16, 29, 35),
                                         (20, 33, 21)])
def test_parity_with_the_oracle(no, nv, nchol):
    L, t2, _, _ = make_inputs(no, nv, nchol, seed=no * 1000 + nv)
    R, plan = pm_ladder(L, t2)
    ref = oracle.ladder(L, t2)
    assert rel_fro(R, ref) <= TOL_R
    E = lad.ladder_energy(plan, dev(t2), dev(R))
    assert abs(E - oracle.energy(t2, ref)) <= TOL_E


@pytest.mark.parametrize("blocks", [(3, 7), (7, 3), (19, 2)])
def test_blocking_does_not_change_a_single_bit(blocks):
    s = CONFIGS["c1"]
    L, t2, _, _ = make_inputs(s.no, s.nv, s.nchol, s.seed)
    R1, _ = pm_ladder(L, t2)
    Rb, plan = pm_ladder(L, t2, blocks=blocks)
    assert (plan.describe()["n_a"], plan.describe()["n_b"]) == blocks
    assert np.array_equal(Rb, R1)


def test_form_rejections():
    plan = lad.ladder_plan(3, 20, 30, lad.LADDER_FP64)
    with pytest.raises(lad.LadderError) as e:
        plan.set_form(1)
    assert e.value.status == lad.LADDER_ERR_UNSUPPORTED
    plan = lad.ladder_plan(3, 20, 30, EMU)
    with pytest.raises(lad.LadderError) as e:
        plan.set_form(2)
    assert e.value.status == lad.LADDER_ERR_ARG


@pytest.mark.parametrize("name", ["c2", "c3"])
def test_full_size_sampled_parity(name):
    s = CONFIGS[name]
    L, t2, _, _ = make_inputs(s.no, s.nv, s.nchol, s.seed)
    R, plan = pm_ladder(L, t2)
    check_sampled(R, L, t2, TOL_R)
    E = lad.ladder_energy(plan, dev(t2), dev(R))
    Eg, Fg = _golden_energy(name), _golden(name, "R_fro")
    assert abs(E - Eg) <= TOL_E
    assert abs(float(np.linalg.norm(R.ravel())) - Fg) <= TOL_R * Fg
