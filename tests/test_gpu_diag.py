"""GPU parity of the diagonal streaming path (Alg. 2 diagonal branch) against
the FP64 oracle: single diagonal operators of width 1..12 at any physical
positions and under a non-identity layout, circuits whose diagonal blocks are
wider than the dense cap, and the argument errors."""
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


def _rand_diag(k, rng, unit):
    d = rng.standard_normal(1 << k) + 1j * rng.standard_normal(1 << k)
    return d / np.abs(d) if unit else 0.5 * d


@pytest.mark.parametrize("k", list(range(1, 13)))
def test_apply_diag_matches_oracle(q, k):
    """Random complex tables (non-unitary included) at random positions that
    cover bit 0, the table boundaries 11/12 and the top bit; N = 14."""
    n = 14
    rng = np.random.default_rng(100 + k)
    psi = W.random_state(n, seed=k)
    st = GState(q, torch, n, init=psi)
    try:
        ref = psi.copy()
        for trial in range(3):
            forced = [0, 11, 12, n - 1][: min(k, 4)]
            rest = [int(v) for v in rng.permutation([x for x in range(n) if x not in forced])[: k - len(forced)]]
            t = [int(v) for v in rng.permutation(forced + rest)]
            d = _rand_diag(k, rng, unit=trial != 1)
            q.qsa_apply_diag(st.h, t, d)
            oracle.apply_diag(ref, t, d)
        got = st.logical()
        scale = max(1.0, float(np.max(np.abs(ref))))
        assert np.max(np.abs(got - ref)) <= 1e-5 * scale
    finally:
        st.close()


def test_apply_diag_under_layout(q):
    """Logical targets resolve through L: with a permuted layout the update
    matches the oracle on the decoded logical state."""
    n = 13
    rng = np.random.default_rng(7)
    psi = W.random_state(n, seed=7)
    st = GState(q, torch, n, init=psi)
    try:
        lay = [int(v) for v in rng.permutation(n)]
        q.qsa_set_layout(st.h, lay)
        ref = psi.copy()
        for k in (2, 5, 9):
            t = [int(v) for v in rng.choice(n, size=k, replace=False)]
            d = _rand_diag(k, rng, unit=True)
            q.qsa_apply_diag(st.h, t, d)
            oracle.apply_diag(ref, t, d)
        check_close(ref, st.logical())
        assert q.qsa_get_layout(st.h) == lay
    finally:
        st.close()


@pytest.mark.parametrize("kmax,kdiag,planner", [(2, 8, 2), (4, 12, 2), (6, 6, 1), (3, 10, 0)])
def test_circuits_with_diagonal_blocks_match_oracle(q, kmax, kdiag, planner):
    """QAOA (ZZ layers are diagonal) and a diagonal-heavy QFT through the
    planner with diagonal blocks up to kdiag wide, against the oracle."""
    n = 14
    for ops in (W.qaoa_circuit(n=n, p=3, seed=kdiag)[0], W.basis_prep(n, 0x2b5d) + W.qft_ops(n)):
        st = GState(q, torch, n)
        try:
            stats = q.qsa_apply_circuit(st.h, ops, q.make_opts(planner=planner, kmax=kmax, kmax_diag=kdiag,
                                                               timing=1))
            ref = oracle.run_circuit(n, ops)
            check_close(ref, st.logical())
            if planner:
                assert stats["diag_blocks"] > 0
        finally:
            st.close()


def test_plan_blocks_report_wide_diagonal_widths(q):
    """A compiled plan with kmax 3 and kmax_diag 10 holds diagonal blocks wider
    than 3; executing it twice equals the oracle's circuit applied twice."""
    n = 12
    ops, _ = W.qaoa_circuit(n=n, p=2, seed=3)
    plan = q.qsa_plan_create(ops, n, q.make_opts(planner=q.QSA_PLAN_DP, kmax=3, kmax_diag=10))
    try:
        _, widths = q.qsa_plan_blocks(plan)
        assert max(widths) > 3 and max(widths) <= 10
        st = GState(q, torch, n)
        try:
            q.qsa_plan_execute(st.h, plan)
            q.qsa_plan_execute(st.h, plan)
            ref = oracle.run_circuit(n, ops + ops)
            check_close(ref, st.logical())
        finally:
            st.close()
    finally:
        q.qsa_plan_destroy(plan)


def test_apply_diag_argument_errors(q):
    st = GState(q, torch, 12)
    try:
        with pytest.raises(q.QsaError):
            q.qsa_apply_diag(st.h, list(range(12)) + [0], np.ones(1 << 13))
        with pytest.raises(q.QsaError):
            q.qsa_apply_diag(st.h, [3, 3], np.ones(4))
        with pytest.raises(q.QsaError):
            q.qsa_apply_diag(st.h, [12], np.ones(2))
    finally:
        st.close()
