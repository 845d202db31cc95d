"""GPU execution of plans with the permutation lowering under both victim
rules (§IV-D demand model): the state matches the FP64 oracle decoded through
the retained layout, and the permutations made equal the host replay."""
import numpy as np
import pytest

import oracle
import workloads as W
from gpu_helpers import GState, check_close

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def q():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_2608_16940_gb300 as q
    return q


@pytest.mark.parametrize("victim", [0, 1], ids=["first_free", "farthest"])
@pytest.mark.parametrize("name", ["fusion", "qaoa"])
def test_permute_lowering_victim_rules(q, victim, name):
    n = 16
    if name == "fusion":
        ops, _ = W.fusion_circuit(n=n, layers=6, seed=2, with_inverse=False)
        opts = q.make_opts(planner=q.QSA_PLAN_DP, kmax=4, kmax_diag=4, lowering=q.QSA_LOWER_PERMUTE,
                           victim=victim, timing=1)
    else:
        ops, _ = W.qaoa_circuit(n=n, p=3, seed=4)
        opts = q.make_opts(planner=q.QSA_PLAN_DP, kmax=3, kmax_diag=10, lowering=q.QSA_LOWER_PERMUTE,
                           victim=victim, timing=1)
    plan = q.qsa_plan_create(ops, n, opts)
    st = GState(q, torch, n)
    try:
        pr, ps, lay = q.qsa_plan_promotions(plan, n, victim)
        stats = q.qsa_plan_execute(st.h, plan)
        assert stats["permutes"] == ps
        assert q.qsa_get_layout(st.h) == lay
        check_close(oracle.run_circuit(n, ops), st.logical())
    finally:
        st.close()
        q.qsa_plan_destroy(plan)
