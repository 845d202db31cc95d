"""GPU parity of the product lowering (one-qubit factors on distinct qubits,
one pass of the tile engine; several when more than 6 targets lie above the
tile's contiguous low bits) against the FP64 oracle, and of plans with
product units."""
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


@pytest.mark.parametrize("k", list(range(1, 12)))
def test_apply_product_matches_oracle(q, k):
    n = 14
    rng = np.random.default_rng(200 + k)
    psi = W.random_state(n, seed=k)
    st = GState(q, torch, n, init=psi)
    try:
        ref = psi.copy()
        for trial in range(3):
            t = [int(v) for v in rng.choice(n, size=k, replace=False)]
            fac = [W.haar_unitary(2, rng) for _ in range(k)]
            q.qsa_apply_product(st.h, t, fac)
            oracle.apply_product(ref, t, fac)
        check_close(ref, st.logical())
    finally:
        st.close()


def test_apply_product_high_targets_split_into_passes(q):
    """Eleven targets all above the tile's low bits need two passes."""
    n = 20
    rng = np.random.default_rng(3)
    psi = W.random_state(n, seed=3)
    st = GState(q, torch, n, init=psi)
    try:
        t = list(range(9, 20))
        fac = [W.haar_unitary(2, rng) for _ in t]
        q.qsa_apply_product(st.h, t, fac)
        ref = psi.copy()
        oracle.apply_product(ref, t, fac)
        check_close(ref, st.logical())
    finally:
        st.close()


@pytest.mark.parametrize("kprod,planner", [(11, 2), (4, 2), (6, 1), (8, 3)])
def test_plans_with_product_units_match_oracle(q, kprod, planner):
    n = 16
    for ops in (W.qaoa_circuit(n=n, p=3, seed=kprod)[0], W.brick_circuit(n, 8, seed=kprod)):
        st = GState(q, torch, n)
        try:
            stats = q.qsa_apply_circuit(st.h, ops, q.make_opts(planner=planner, kmax=4, kmax_diag=8,
                                                               kmax_prod=kprod, timing=1))
            check_close(oracle.run_circuit(n, ops), st.logical())
            if ops and planner in (1, 2):
                assert stats["prod_blocks"] > 0
        finally:
            st.close()


def test_apply_product_argument_errors(q):
    st = GState(q, torch, 13)
    try:
        with pytest.raises(q.QsaError):
            q.qsa_apply_product(st.h, list(range(12)), [np.eye(2)] * 12)
        with pytest.raises(q.QsaError):
            q.qsa_apply_product(st.h, [2, 2], [np.eye(2)] * 2)
    finally:
        st.close()


@pytest.mark.parametrize("n", [1, 3, 4, 5])
def test_apply_product_tiny_states(q, n):
    """States below 32 amplitudes take the per-factor path; 5 qubits is the
    smallest tile the lane-mapped rounds cover."""
    rng = np.random.default_rng(n)
    psi = W.random_state(n, seed=n)
    st = GState(q, torch, n, init=psi)
    try:
        t = [int(v) for v in rng.permutation(n)]
        fac = [W.haar_unitary(2, rng) for _ in t]
        q.qsa_apply_product(st.h, t, fac)
        ref = psi.copy()
        oracle.apply_product(ref, t, fac)
        check_close(ref, st.logical())
    finally:
        st.close()
