"""Split-TF32 tensor-core path (k = 5, 6) against the FP64 oracle and the FP32
CUDA-core path.  Tolerance: the same 1e-5 fidelity / amplitude bounds as the
FP32 path; 3xTF32 keeps FP32-level error, which the last test quantifies."""
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


@pytest.mark.parametrize("k,n", [(5, 11), (6, 11), (5, 12), (6, 12), (5, 13), (6, 13), (6, 14), (5, 17), (6, 17)])
def test_tc_single_op_matches_oracle(q, k, n):
    rng = np.random.default_rng(7 * k + n)
    psi = W.random_state(n, seed=n + k)
    st = GState(q, torch, n, init=psi.astype(np.complex64))
    ref = psi.astype(np.complex64).astype(np.complex128)
    try:
        for trial in range(3):
            t = tuple(int(v) for v in rng.choice(n, size=k, replace=False))
            G = W.haar_unitary(1 << k, rng)
            q.qsa_apply_fused_ex(st.h, t, G, q.QSA_LOWER_STRIDED, q.QSA_PREC_TF32X3)
            oracle.apply(ref, t, G)
        check_close(ref, st.logical())
    finally:
        st.close()


@pytest.mark.parametrize("targets", [(0, 1, 2, 3, 4), (0, 1, 2, 3, 4, 5), (13, 12, 11, 10, 9, 8),
                                     (0, 7, 15, 3, 11), (15, 0, 14, 1, 13, 2), (15, 14, 13, 12, 11, 10),
                                     (1, 2, 3, 4, 5, 6), (5, 4, 3, 2, 1), (15, 14, 13, 12, 0), (2, 9, 4, 15, 6)])
def test_tc_target_orders_and_positions(q, targets):
    """Target sets at the lowest positions, at the highest, with and without
    position 0 (two layouts of a chunk's row reads), in and out of order."""
    n = 16
    k = len(targets)
    rng = np.random.default_rng(sum(targets))
    G = W.haar_unitary(1 << k, rng)
    psi = W.random_state(n, 3)
    st = GState(q, torch, n, init=psi.astype(np.complex64))
    ref = psi.astype(np.complex64).astype(np.complex128)
    try:
        q.qsa_apply_fused_ex(st.h, targets, G, q.QSA_LOWER_STRIDED, q.QSA_PREC_TF32X3)
        oracle.apply(ref, targets, G)
        check_close(ref, st.logical())
    finally:
        st.close()


def test_tc_many_chunks_per_cta(q):
    """N = 23: about 28 chunks of 2^11 amplitudes per CTA, so every ring of the
    kernel (raw stages, operand buffers, accumulators) wraps several times;
    k = 5 and 6, with and without a target at position 0."""
    n = 23
    rng = np.random.default_rng(23)
    psi = W.random_state(n, seed=5)
    st = GState(q, torch, n, init=psi.astype(np.complex64))
    ref = psi.astype(np.complex64).astype(np.complex128)
    try:
        for t in [(0, 7, 22, 3, 15, 9), (4, 21, 13, 1, 18), (0, 11, 5, 20, 2), (22, 6, 1, 14, 3, 19)]:
            G = W.haar_unitary(1 << len(t), rng)
            q.qsa_apply_fused_ex(st.h, t, G, q.QSA_LOWER_STRIDED, q.QSA_PREC_TF32X3)
            oracle.apply(ref, t, G)
        check_close(ref, st.logical())
    finally:
        st.close()


def test_tc_wide_circuit_uses_tensor_cores(q):
    """Alternating k = 5 / 6 Haar operators on random target sets (the wide
    workload's structure at N = 18): every block runs on the tensor cores."""
    n = 18
    ops = W.wide_circuit(n, n_ops=16, widths=(5, 6), seed=2)
    st = GState(q, torch, n)
    try:
        stats = q.qsa_apply_circuit(st.h, ops, q.make_opts(planner=q.QSA_PLAN_PER_GATE, kmax=6, kmax_diag=6,
                                                           precision=q.QSA_PREC_TF32X3))
        assert stats["tc_blocks"] == len(ops)
        ref = oracle.run_circuit(n, ops)
        check_close(ref, st.logical())
    finally:
        st.close()


def test_tc_deep_circuit_keeps_fidelity(q, capsys):
    """100 alternating k = 6 / 5 Haar operators at N = 20: the tensor-core
    accumulation bias must not build up with depth (1 - F <= 1e-5)."""
    n = 20
    ops = W.wide_circuit(n, n_ops=100, widths=(6, 5), seed=9)
    ref = oracle.run_circuit(n, ops)
    res = {}
    for prec in (q.QSA_PREC_FP32, q.QSA_PREC_TF32X3):
        st = GState(q, torch, n)
        try:
            q.qsa_apply_circuit(st.h, ops, q.make_opts(planner=0, kmax=6, kmax_diag=6, precision=prec))
            got = st.logical()
            res[prec] = (1 - oracle.fidelity(ref, got), oracle.max_abs_diff(ref, got),
                         float(np.vdot(got, got).real) - 1)
        finally:
            st.close()
    with capsys.disabled():
        print(f"\n100 ops k=5/6 N=20: FP32 (1-F, max|d|, norm-1) = {res[0]}; 3xTF32 = {res[1]}")
    for prec in res:
        assert abs(res[prec][0]) <= 1e-5 and res[prec][1] <= 1e-5


def test_tc_agrees_with_fp32_path_and_reports_error(q):
    n = 16
    ops = W.wide_circuit(n, n_ops=12, widths=(6, 5), seed=5)
    ref = oracle.run_circuit(n, ops)
    out = {}
    for prec in (q.QSA_PREC_FP32, q.QSA_PREC_TF32X3):
        st = GState(q, torch, n)
        try:
            q.qsa_apply_circuit(st.h, ops, q.make_opts(planner=0, kmax=6, kmax_diag=6, precision=prec))
            out[prec] = st.logical()
        finally:
            st.close()
    e32 = oracle.max_abs_diff(ref, out[0])
    etc = oracle.max_abs_diff(ref, out[1])
    # 3xTF32 keeps FP32-level accuracy: within a small factor of the FP32 path
    assert etc <= max(4 * e32, 2e-6), (etc, e32)
    check_close(out[0], out[1])
