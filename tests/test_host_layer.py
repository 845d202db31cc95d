"""Host-only checks of the layer grouping (no GPU): the library's execution
order equals the oracle's layer_units order, its layer blocks are the
oracle's layer units (same ops, same diagonal part) and every other block is
a run of consecutive oracle units; options and argument errors."""
import numpy as np
import pytest

import oracle
import workloads as W
from test_oracle_layer import _mixed_circuit


@pytest.fixture(scope="module")
def q():
    import __graft_entry__
    __graft_entry__._build_module().build()
    import paper_2608_16940_gb300 as q
    return q


def _check_plan(q, ops, n, opts, layout):
    p = q.qsa_plan_create(ops, n, opts, layout=layout)
    try:
        order = q.qsa_plan_order(p)
        first, _ = q.qsa_plan_blocks(p)
        kinds, nd = q.qsa_plan_block_kinds(p)
    finally:
        q.qsa_plan_destroy(p)
    ref_order, ref_units = oracle.layer_units(ops, n, layout)
    assert order == ref_order
    bounds = {u[0] for u in ref_units} | {len(ops)}
    ref_layer = {u[0]: (u[1], u[3]) for u in ref_units if u[2]}
    ends = first[1:] + [len(ops)]
    for s, e, k, d in zip(first, ends, kinds, nd):
        assert s in bounds and e in bounds
        if k == 3:
            assert ref_layer.get(s) == (e, d)
    return kinds


@pytest.mark.parametrize("n,n_ops,seed,planner,permuted", [(12, 150, 0, 2, False), (14, 200, 1, 2, True),
                                                           (16, 300, 2, 1, True), (20, 250, 3, 3, False),
                                                           (13, 120, 4, 2, True), (8, 100, 5, 2, False)])
def test_layer_grouping_matches_oracle(q, n, n_ops, seed, planner, permuted):
    rng = np.random.default_rng(seed)
    ops = _mixed_circuit(n, n_ops, rng)
    layout = [int(v) for v in rng.permutation(n)] if permuted else None
    kinds = _check_plan(q, ops, n, q.make_opts(planner=planner, kmax=4, kmax_diag=4, layer=1), layout)
    assert 3 in kinds


@pytest.mark.parametrize("n,p,seed", [(16, 3, 0), (30, 8, 0)])
def test_qaoa_layers_match_oracle(q, n, p, seed):
    ops, _ = W.qaoa_circuit(n, p, seed)
    kinds = _check_plan(q, ops, n, q.make_opts(planner=2, kmax=6, kmax_diag=12, layer=1), None)
    assert all(k == 3 for k in kinds)
    if n == 30:
        assert len(kinds) == 27


def test_bench_plan_has_24_passes(q):
    """The bench's plan (N = 30 QAOA, p = 8, interleaved layout, layer units,
    zero-state prefix): one preparation block that also takes the first layer
    block, then 23 layer blocks; each fits one tile in the plan's layout (so
    24 passes, the floor for 216 factors on positions >= 3 at 9 per pass)."""
    import bench
    n = 30
    ops, _ = W.qaoa_circuit(n, 8, seed=0)
    layout = bench.interleaved_layout(n)
    p = q.qsa_plan_create(ops, n, q.make_opts(planner=2, kmax=6, kmax_diag=12, layer=1, zero_init=1), layout=layout)
    try:
        kinds, _ = q.qsa_plan_block_kinds(p)
        first, _ = q.qsa_plan_blocks(p)
        order = q.qsa_plan_order(p)
    finally:
        q.qsa_plan_destroy(p)
    assert kinds == [4] + [3] * 23
    run = [ops[i] for i in order]                  # execution order; block j is run[first[j]:first[j + 1]]
    P = oracle.zero_init_prefix(ops)               # the prefix's one-qubit ops are generated, not factors
    for j, (s, e) in enumerate(zip(first, first[1:] + [len(ops)])):
        qubits = {qb for o in run[max(s, P):e] if len(o.targets) == 1 and not o.diag for qb in o.targets}
        assert len(qubits) <= 12 and sum(1 for qb in qubits if layout[qb] >= 3) <= 9


def test_layer_off_keeps_the_input_order(q):
    ops = W.brick_circuit(12, 6, seed=1)
    p = q.qsa_plan_create(ops, 12, q.make_opts(planner=2, kmax=4))
    try:
        assert q.qsa_plan_order(p) == list(range(len(ops)))
        assert 3 not in q.qsa_plan_block_kinds(p)[0]
    finally:
        q.qsa_plan_destroy(p)


def test_layer_options_validated(q):
    ops = W.brick_circuit(12, 2, seed=1)
    with pytest.raises(q.QsaError) as e:
        q.qsa_plan_create(ops, 12, q.make_opts(layer=2))
    assert e.value.code == q.QSA_E_ARG


@pytest.mark.parametrize("kind,n", [("qaoa", 30), ("qaoa", 16), ("brick", 12), ("mixed", 14)])
def test_zero_init_prefix_matches_oracle(q, kind, n):
    """The zero_init plan's first block covers exactly the oracle's prefix, in
    input order, together with the first unit after it when that is a layer
    unit (both share the write-only pass); the rest is grouped as without it."""
    rng = np.random.default_rng(n)
    if kind == "qaoa":
        ops, _ = W.qaoa_circuit(n, 3, seed=0)
    elif kind == "brick":
        ops = W.brick_circuit(n, 4, seed=0)
    else:
        ops = [W.Op((qb,), W.haar_unitary(2, rng), False) for qb in range(n)] + _mixed_circuit(n, 60, rng)
    P = oracle.zero_init_prefix(ops)
    p = q.qsa_plan_create(ops, n, q.make_opts(planner=2, kmax=4, kmax_diag=4, layer=1, zero_init=1))
    try:
        order = q.qsa_plan_order(p)
        first, _ = q.qsa_plan_blocks(p)
        kinds, _ = q.qsa_plan_block_kinds(p)
    finally:
        q.qsa_plan_destroy(p)
    assert P > 0 and kinds[0] == 4 and 4 not in kinds[1:]
    assert order[:P] == list(range(P))
    ref_order, ref_units = oracle.layer_units(ops[P:], n)
    assert order[P:] == [x + P for x in ref_order]
    end0 = P + ref_units[0][1] if ref_units and ref_units[0][2] else P
    assert first[0] == 0 and (len(first) == 1 or first[1] == end0)
