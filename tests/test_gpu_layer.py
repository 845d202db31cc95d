"""GPU parity of layer blocks (diagonal gates on one or two qubits anywhere,
then one-qubit factors, one tile pass) against the FP64 oracle: every class
of diagonal gate relative to a tile (all qubits in it, one in it, none),
factors only, diagonal gates only, more factor positions than one tile holds
(several passes), small states (other kernels), permuted layouts; plans with
layer units (QAOA, brickwork, mixed circuits), a plan run under a layout
other than its own, and the statistics."""
import numpy as np
import pytest

import oracle
import workloads as W
from gpu_helpers import GState, check_close  # noqa: F401

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def q():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_2608_16940_gb300 as q
    return q


def _diag_ops(n, count, rng, unit=True):
    out = []
    for _ in range(count):
        k = 1 if rng.random() < 0.3 else 2
        t = tuple(int(v) for v in rng.choice(n, size=k, replace=False))
        d = np.exp(1j * rng.uniform(0, 2 * np.pi, 1 << k))
        if not unit:
            d = d * rng.uniform(0.8, 1.2, 1 << k)
        out.append(W.Op(t, np.diag(d), True))
    return out


def _run(q, n, diag, targets, factors, layout=None, seed=0):
    psi = W.random_state(n, seed=seed)
    st = GState(q, torch, n, init=psi)
    try:
        if layout is not None:
            q.qsa_set_layout(st.h, layout, 1)
        q.qsa_apply_layer(st.h, diag, targets, factors)
        ref = psi.copy()
        oracle.apply_layer(ref, diag, targets, factors)
        got = st.logical()
        # non-unit diagonal entries leave the state unnormalised: compare in norm
        assert np.linalg.norm(got - ref) <= 1e-5 * np.linalg.norm(ref)
        assert oracle.max_abs_diff(ref, got) <= 1e-5
    finally:
        st.close()


@pytest.mark.parametrize("n,k,n_diag,seed,permuted", [(12, 6, 20, 0, False), (13, 8, 30, 1, True),
                                                      (16, 9, 40, 2, False), (16, 12, 60, 3, True),
                                                      (20, 7, 80, 4, False), (22, 10, 100, 5, True)])
def test_layer_matches_oracle(q, n, k, n_diag, seed, permuted):
    rng = np.random.default_rng(seed)
    layout = [int(v) for v in rng.permutation(n)] if permuted else list(range(n))
    # factor qubits that fit one tile: at most 9 at positions >= 3
    low = [qb for qb in range(n) if layout[qb] < 3]
    high = [qb for qb in range(n) if layout[qb] >= 3]
    nl = min(len(low), int(rng.integers(0, 4)), k)
    t = [int(v) for v in rng.choice(low, size=nl, replace=False)] + \
        [int(v) for v in rng.choice(high, size=min(9, k - nl), replace=False)]
    fac = [W.haar_unitary(2, rng) for _ in t]
    _run(q, n, _diag_ops(n, n_diag, rng, unit=seed % 2 == 0), t, fac, layout if permuted else None, seed)


_X = np.array([[0, 1], [1, 0]], dtype=complex)
_Y = np.array([[0, -1j], [1j, 0]], dtype=complex)
_S = np.diag([1, 1j])
_RX = np.array([[1, -1j], [-1j, 1]], dtype=complex) / np.sqrt(2)   # |F00| = |F01|
_SXY = _X @ np.diag([np.exp(0.3j), np.exp(-1.1j)])                 # F00 = 0, F01 = phase


@pytest.mark.parametrize("n,targets", [(12, [0, 1, 2, 3]), (14, [0, 1, 2, 3]), (14, [0, 4, 5, 7]),
                                       (16, [1, 3, 6, 9, 10, 11]), (18, [0, 1, 2, 12, 13, 14, 15, 16, 17]),
                                       (20, [2, 4, 8, 11, 15, 19])],
                         ids=["n12-round0", "n14-round0", "n14-rounds01", "n16-rounds012", "n18-high",
                              "n20-spread"])
def test_layer_rotation_forms(q, n, targets):
    """Factors at the boundaries of the rotation forms on every round: cotangent
    form with u = 0 (X, Y, X times phases: halves exchanged, stored back through
    the exchanged index, including round 0 as the last round where a 16-byte
    chunk's two halves trade places), |c| = |s| (tangent form, t = 1), s = 0
    (phases only, t = 0) and Haar factors; with and without diagonal gates."""
    rng = np.random.default_rng(n + len(targets))
    kinds = [_X, _Y, _SXY, _RX, _S, W.H]
    fac = [kinds[j % len(kinds)] if j < len(kinds) else W.haar_unitary(2, rng) for j in range(len(targets))]
    fac = fac[len(targets) % 3:] + fac[:len(targets) % 3]
    _run(q, n, [], targets, fac, seed=n)
    _run(q, n, _diag_ops(n, 3 * n, rng), targets, fac, seed=n + 1)
    # every factor in the cotangent form with u = 0
    _run(q, n, _diag_ops(n, n, rng), targets, [_X for _ in targets], seed=n + 2)


def test_layer_diagonal_only_and_factors_only(q):
    rng = np.random.default_rng(10)
    _run(q, 14, _diag_ops(14, 50, rng), [], [])
    _run(q, 14, [], [0, 1, 2, 3], [W.haar_unitary(2, rng) for _ in range(4)])
    _run(q, 14, [], [13, 12, 5], [W.haar_unitary(2, rng) for _ in range(3)])
    _run(q, 16, [], [15], [W.H])


def test_layer_gate_classes(q):
    """n = 18, factors on qubits 0..2 and 10..18: ZZ inside the tile, across
    its boundary (either qubit order) and outside it, one-qubit phases in and
    out."""
    n = 18
    rng = np.random.default_rng(11)
    t = [0, 1, 2] + list(range(9, 18))
    fac = [W.haar_unitary(2, rng) for _ in t]
    diag = [W.Op((0, 12), np.diag(np.exp(1j * rng.uniform(0, 6, 4))), True),
            W.Op((5, 12), np.diag(np.exp(1j * rng.uniform(0, 6, 4))), True),
            W.Op((12, 6), np.diag(np.exp(1j * rng.uniform(0, 6, 4))), True),
            W.Op((4, 7), np.diag(np.exp(1j * rng.uniform(0, 6, 4))), True),
            W.Op((8,), np.diag(np.exp(1j * rng.uniform(0, 6, 2))), True),
            W.Op((17,), np.diag(np.exp(1j * rng.uniform(0, 6, 2))), True)]
    _run(q, n, diag, t, fac)


@pytest.mark.parametrize("n,seed", [(16, 20), (13, 21)])
def test_layer_non_unitary_factors(q, n, seed):
    """Factors that are not unitary take the general complex butterflies (no
    rotation split); mixed with unitary ones and with every gate class."""
    rng = np.random.default_rng(seed)
    t = [0, 2] + [int(v) for v in rng.choice(range(3, n), size=7, replace=False)]
    fac = [W.haar_unitary(2, rng) for _ in t]
    fac[3] = rng.standard_normal((2, 2)) + 1j * rng.standard_normal((2, 2))
    _run(q, n, _diag_ops(n, 30, rng), t, fac)


def test_layer_diagonal_and_antidiagonal_factors(q):
    """Factors with a zero off-diagonal or a zero diagonal (the rotation split's
    edge cases)."""
    rng = np.random.default_rng(22)
    t = [1, 5, 9, 14]
    fac = [np.diag(np.exp(1j * rng.uniform(0, 6, 2))), W.X, np.array([[0, 1j], [1j, 0]]), W.H]
    _run(q, 16, _diag_ops(16, 20, rng), t, fac)


def test_layer_more_factors_than_a_tile_holds(q):
    """Twelve factors all at positions >= 3: two passes (diagonal ops in the first)."""
    n = 20
    rng = np.random.default_rng(12)
    t = list(range(5, 17))
    _run(q, n, _diag_ops(n, 30, rng), t, [W.haar_unitary(2, rng) for _ in t])


@pytest.mark.parametrize("n", [3, 8, 11])
def test_layer_small_states(q, n):
    rng = np.random.default_rng(13 + n)
    t = [int(v) for v in rng.choice(n, size=min(n, 5), replace=False)]
    _run(q, n, _diag_ops(n, 10, rng), t, [W.haar_unitary(2, rng) for _ in t])


@pytest.mark.parametrize("kind,n,planner,kmax,prec", [("qaoa", 16, 2, 6, 1), ("qaoa", 20, 3, 6, 1),
                                                     ("brick", 14, 2, 4, 0), ("mixed", 14, 2, 4, 0),
                                                     ("mixed", 13, 1, 4, 0)])
def test_plans_with_layer_units_match_oracle(q, kind, n, planner, kmax, prec):
    rng = np.random.default_rng(n + planner)
    if kind == "qaoa":
        ops, _ = W.qaoa_circuit(n, 3, seed=1)
    elif kind == "brick":
        ops = W.brick_circuit(n, 8, seed=2)
        ops = [W.Op(o.targets, o.matrix, o.name == "cz" or o.diag, o.name) for o in ops]
    else:
        from test_oracle_layer import _mixed_circuit
        ops = _mixed_circuit(n, 200, rng)
    st = GState(q, torch, n)
    try:
        stats = q.qsa_apply_circuit(st.h, ops, q.make_opts(planner=planner, kmax=kmax, kmax_diag=kmax, layer=1,
                                                           precision=prec))
        assert stats["layer_blocks"] > 0
        check_close(oracle.run_circuit(n, ops), st.logical())
    finally:
        st.close()


def test_plan_under_another_layout(q):
    """A plan built for the identity layout, executed on a state whose layout
    was permuted: layer blocks are prepared again for that layout."""
    n = 16
    ops, _ = W.qaoa_circuit(n, 2, seed=3)
    p = q.qsa_plan_create(ops, n, q.make_opts(planner=2, kmax=6, kmax_diag=6, layer=1, timing=1))
    st = GState(q, torch, n)
    try:
        q.qsa_set_layout(st.h, [int(v) for v in np.random.default_rng(4).permutation(n)], 1)
        stats = q.qsa_plan_execute(st.h, p)
        assert stats["layer_blocks"] > 0 and stats["layer_seconds"] > 0
        check_close(oracle.run_circuit(n, ops), st.logical())
    finally:
        st.close()
        q.qsa_plan_destroy(p)


def test_layer_argument_errors(q):
    st = GState(q, torch, 12)
    try:
        bad = [([W.Op((0, 1, 2), np.eye(8), True)], [], []),          # three-qubit diagonal op
               ([W.Op((0, 1), W.CNOT, True)], [], []),                 # not diagonal
               ([], [0, 0], [np.eye(2), np.eye(2)]),                   # repeated factor qubit
               ([], [12], [np.eye(2)]),                                # qubit out of range
               ([], list(range(12)) + [0], [np.eye(2)] * 13)]          # more than 12 factors
        for dg, t, f in bad:
            with pytest.raises(q.QsaError) as e:
                q.qsa_apply_layer(st.h, dg, t, f)
            assert e.value.code == q.QSA_E_ARG
    finally:
        st.close()


@pytest.mark.parametrize("kind,n,layer,permuted", [("qaoa", 16, 1, False), ("qaoa", 16, 1, True),
                                                   ("brick", 14, 0, False), ("mixed", 13, 1, True),
                                                   ("qaoa", 12, 1, False), ("qaoa", 8, 1, True)])
def test_zero_init_plans_match_oracle(q, kind, n, layer, permuted):
    """Plans with the zero-state prefix (a write-only pass; N < 12: all ones
    then the diagonal kernels) against the oracle, on identity and relabelled
    layouts."""
    rng = np.random.default_rng(n + layer)
    if kind == "qaoa":
        ops, _ = W.qaoa_circuit(n, 2, seed=4)
    elif kind == "brick":
        ops = W.brick_circuit(n, 5, seed=4)
    else:
        from test_oracle_layer import _mixed_circuit
        ops = [W.Op((qb,), W.haar_unitary(2, rng), False) for qb in range(n)] + _mixed_circuit(n, 80, rng)
    st = GState(q, torch, n)
    try:
        if permuted:
            q.qsa_set_layout(st.h, [int(v) for v in rng.permutation(n)], 0)
        stats = q.qsa_apply_circuit(st.h, ops, q.make_opts(planner=2, kmax=4, kmax_diag=4, layer=layer,
                                                           zero_init=1))
        assert stats["layer_blocks"] + stats["diag_blocks"] >= 1   # N < 12: diagonal kernels
        check_close(oracle.run_circuit(n, ops), st.logical())
    finally:
        st.close()


def test_zero_init_plan_needs_the_zero_state_and_other_layouts(q):
    n = 14
    ops, _ = W.qaoa_circuit(n, 2, seed=5)
    p = q.qsa_plan_create(ops, n, q.make_opts(planner=2, kmax=4, kmax_diag=4, layer=1, zero_init=1))
    st = GState(q, torch, n)
    try:
        q.qsa_apply_fused(st.h, [0], W.H)
        with pytest.raises(q.QsaError) as e:
            q.qsa_plan_execute(st.h, p)
        assert e.value.code == q.QSA_E_STATE
        # built for the identity layout, run on a relabelled zero state
        q.qsa_state_reset(st.h)
        q.qsa_set_layout(st.h, [int(v) for v in np.random.default_rng(6).permutation(n)], 0)
        q.qsa_plan_execute(st.h, p)
        check_close(oracle.run_circuit(n, ops), st.logical())
    finally:
        st.close()
        q.qsa_plan_destroy(p)


@pytest.mark.parametrize("zero_init,n", [(1, 16), (0, 14), (1, 9)])
def test_execute_from_zero_discards_the_state(q, zero_init, n):
    """qsa_plan_execute_from_zero on a state holding arbitrary data: the result
    is the circuit applied to |0...0> (without clearing when the plan starts
    with the zero-state preparation), in the plan's layout."""
    ops, _ = W.qaoa_circuit(n if n % 2 == 0 else n + 1, 2, seed=7)
    if n % 2:
        ops = [o for o in ops if max(o.targets) < n]
    layout = [int(v) for v in np.random.default_rng(n).permutation(n)]
    p = q.qsa_plan_create(ops, n, q.make_opts(planner=2, kmax=4, kmax_diag=4, layer=1, zero_init=zero_init),
                          layout=layout)
    st = GState(q, torch, n, init=W.random_state(n, seed=3))
    try:
        for _ in range(2):
            q.qsa_plan_execute_from_zero(st.h, p)
            assert q.qsa_get_layout(st.h) == layout
            check_close(oracle.run_circuit(n, ops), st.logical())
    finally:
        st.close()
        q.qsa_plan_destroy(p)
