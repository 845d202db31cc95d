"""Error paths and cleanup on the GPU, with failures injected on the host
(qsa_debug_fail_alloc: an allocation reports out-of-memory before any device
call is made; no device fault is involved), and the per-state cost model.

- state creation whose second allocation fails releases the first;
- a plan whose upload fails on its first or second buffer holds nothing
  afterwards, leaves the state usable, and uploads on the next execution;
- a scratch allocation that fails leaves the state usable;
- a cost model attached to one state drives the DP-MLP plans of
  qsa_apply_circuit on that state only, and detaching it restores the
  process-wide model.
"""
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
    yield q
    q.qsa_debug_fail_alloc(-1)
    q.qsa_costmodel_set(None)


def test_state_create_second_allocation_failure_frees_the_first(q):
    live = q.qsa_debug_live_allocations()
    q.qsa_debug_fail_alloc(1)   # the amplitudes are allocated, the error word is not
    try:
        with pytest.raises(q.QsaError) as e:
            q.qsa_state_create(14)
        assert e.value.code == q.QSA_E_NOMEM
    finally:
        q.qsa_debug_fail_alloc(-1)
    assert q.qsa_debug_live_allocations() == live
    s = q.qsa_state_create(14)
    assert q.qsa_debug_live_allocations() == live + 2
    q.qsa_state_destroy(s)
    assert q.qsa_debug_live_allocations() == live


@pytest.mark.parametrize("nth", [0, 1])
def test_plan_upload_failure_holds_nothing_and_retries(q, nth):
    """A layer plan with a dense block: both upload buffers are needed."""
    n = 14
    ops, _ = W.qaoa_circuit(n=n, p=1, seed=4)
    ops = ops + [W.Op((2, 9), W.haar_unitary(4, np.random.default_rng(1)), False)]
    plan = q.qsa_plan_create(ops, n, q.make_opts(planner=q.QSA_PLAN_DP, kmax=2, kmax_diag=12, layer=1))
    st = GState(q, torch, n)
    try:
        live = q.qsa_debug_live_allocations()
        q.qsa_debug_fail_alloc(nth)
        try:
            with pytest.raises(q.QsaError) as e:
                q.qsa_plan_execute(st.h, plan)
            assert e.value.code == q.QSA_E_NOMEM
        finally:
            q.qsa_debug_fail_alloc(-1)
        assert q.qsa_debug_live_allocations() == live
        q.qsa_state_reset(st.h)
        q.qsa_plan_execute(st.h, plan)   # uploads now
        check_close(oracle.run_circuit(n, ops), st.logical())
    finally:
        q.qsa_plan_destroy(plan)
        st.close()


def test_scratch_failure_keeps_the_state_usable(q):
    n = 12
    st = GState(q, torch, n)
    try:
        q.qsa_apply_fused(st.h, [3], W.H)
        live = q.qsa_debug_live_allocations()
        q.qsa_debug_fail_alloc(0)
        try:
            with pytest.raises(q.QsaError) as e:
                q.qsa_probabilities(st.h)   # its output buffer is a fresh allocation
            assert e.value.code == q.QSA_E_NOMEM
        finally:
            q.qsa_debug_fail_alloc(-1)
        assert q.qsa_debug_live_allocations() == live
        probs, norm = q.qsa_probabilities(st.h)
        assert abs(norm - 1) < 1e-6 and abs(probs[0] - 0.5) < 1e-6 and abs(probs[8] - 0.5) < 1e-6
    finally:
        st.close()


def _steep_model(q):
    """f(x) = 30 relu(relu(k / 6)) = 5 k: a block of k qubits costs e^(5k)
    (merging qubits never pays); the flat model (all zeros) costs 1 per block."""
    p = np.zeros(q.MLP_PARAMS, dtype=np.float32)
    p[0] = 1.0                    # W1[0][0] on k / 6
    p[64 * 37 + 64] = 1.0         # W2[0][0]
    p[64 * 37 + 64 + 64 * 64 + 64] = 30.0   # W3[0]
    return p


def test_attached_cost_model_drives_only_its_state(q, tmp_path):
    n = 12
    ops = W.brick_circuit(n=n, layers=6, seed=2)
    opts = q.make_opts(planner=q.QSA_PLAN_DP_MLP, kmax=4, kmax_diag=4)
    path = str(tmp_path / "steep.qsacm")
    q.qsa_costmodel_set(_steep_model(q))
    q.qsa_costmodel_save(path)
    q.qsa_costmodel_set(np.zeros(q.MLP_PARAMS, dtype=np.float32))   # process-wide: flat
    a, b = GState(q, torch, n), GState(q, torch, n)
    try:
        q.qsa_costmodel_load(a.h, path)
        sa = q.qsa_apply_circuit(a.h, ops, opts)
        sb = q.qsa_apply_circuit(b.h, ops, opts)
        ref = oracle.run_circuit(n, ops)
        check_close(ref, a.logical())
        check_close(ref, b.logical())
        assert sa["blocks"] > sb["blocks"], (sa["blocks"], sb["blocks"])
        q.qsa_costmodel_load(a.h, None)   # detach: the process-wide model again
        q.qsa_state_reset(a.h)
        assert q.qsa_apply_circuit(a.h, ops, opts)["blocks"] == sb["blocks"]
    finally:
        q.qsa_costmodel_set(None)
        a.close()
        b.close()
