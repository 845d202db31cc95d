"""Pins for the oracle's layer blocks (no GPU): the grouping reorders a
circuit only across ops that commute, so the reordered stream and the blocks
(diagonal gates then per-qubit factor products) give the input circuit's state
at small N for random mixes of one-qubit, diagonal and dense ops; a
hand-worked grouping (tests/golden/layer_units_hand_example.json); the
grouping's defining invariants; the tile-fit rule at its boundary."""
import json
import os

import numpy as np
import pytest

import oracle
import workloads as W

GOLDEN = os.path.join(os.path.dirname(__file__), "golden", "layer_units_hand_example.json")


def _diag_gate(k, rng):
    return np.diag(np.exp(1j * rng.uniform(0, 2 * np.pi, 1 << k)))


def _mixed_circuit(n, n_ops, rng):
    """One-qubit Haar gates, flagged diagonal gates on 1..3 qubits, dense
    two-qubit Haar gates and unflagged diagonal two-qubit gates."""
    ops = []
    for _ in range(n_ops):
        r = rng.random()
        if r < 0.35:
            ops.append(W.Op((int(rng.integers(0, n)),), W.haar_unitary(2, rng), False))
        elif r < 0.75:
            k = 1 if r < 0.45 else (2 if r < 0.7 else 3)
            t = tuple(int(v) for v in rng.choice(n, size=k, replace=False))
            ops.append(W.Op(t, _diag_gate(k, rng), True))
        elif r < 0.9:
            t = tuple(int(v) for v in rng.choice(n, size=2, replace=False))
            ops.append(W.Op(t, W.haar_unitary(4, rng), False))
        else:
            t = tuple(int(v) for v in rng.choice(n, size=2, replace=False))
            ops.append(W.Op(t, _diag_gate(2, rng), False))
    return ops


@pytest.mark.parametrize("n,n_ops,seed,lookahead,permuted", [(4, 60, 0, 256, False), (5, 80, 1, 2, False),
                                                             (6, 120, 2, 256, True), (7, 90, 3, 5, True),
                                                             (8, 100, 4, 256, False), (13, 60, 5, 256, True)])
def test_grouped_circuit_equals_input_circuit(n, n_ops, seed, lookahead, permuted):
    rng = np.random.default_rng(seed)
    ops = _mixed_circuit(n, n_ops, rng)
    layout = [int(v) for v in rng.permutation(n)] if permuted else None
    order, units = oracle.layer_units(ops, n, layout, lookahead)
    ref = oracle.run_circuit(n, ops)
    re = oracle.run_circuit(n, [ops[i] for i in order])
    assert np.max(np.abs(ref - re)) < 1e-12
    psi = oracle.zero_state(n)
    for s, e, is_layer, nd in units:
        if is_layer:
            dg, qs, fs = oracle.layer_block(ops, order[s:e], nd)
            oracle.apply_layer(psi, dg, qs, fs)
        else:
            oracle.apply(psi, ops[order[s]].targets, ops[order[s]].matrix)
    assert np.max(np.abs(ref - psi)) < 1e-12
    assert sum(u[2] for u in units) >= 1


@pytest.mark.parametrize("seed", range(6))
def test_grouping_invariants(seed):
    rng = np.random.default_rng(100 + seed)
    n = int(rng.integers(12, 17))
    ops = _mixed_circuit(n, 200, rng)
    layout = [int(v) for v in rng.permutation(n)]
    order, units = oracle.layer_units(ops, n, layout)
    assert sorted(order) == list(range(len(ops)))
    pos = 0
    for s, e, is_layer, nd in units:
        assert s == pos and e > s
        pos = e
        idx = order[s:e]
        if not is_layer:
            op = ops[idx[0]]
            assert e - s == 1 and not (len(op.targets) == 1 or (op.diag and len(op.targets) <= 2))
            continue
        dpart, fpart = idx[:nd], idx[nd:]
        assert all(ops[i].diag and len(ops[i].targets) <= 2 for i in dpart)
        assert all(len(ops[i].targets) == 1 for i in fpart)
        fq = {ops[i].targets[0] for i in fpart}
        assert oracle.layer_fits([layout[q] for q in fq], n)
        # a diagonal gate sharing a qubit with a factor precedes that factor's ops in the circuit
        for i in dpart:
            for f in fpart:
                if set(ops[i].targets) & set(ops[f].targets):
                    assert i < f
        assert dpart == sorted(dpart) and fpart == sorted(fpart)
    assert pos == len(order)


def test_hand_worked_grouping():
    data = json.load(open(GOLDEN))
    for case in data["cases"]:
        ops = [W.Op(tuple(t), np.eye(1 << len(t), dtype=np.complex128), d, name) for name, t, d in case["ops"]]
        order, units = oracle.layer_units(ops, case["n"], case["layout"])
        assert order == case["order"], case["why"]
        assert [list(u) for u in units] == case["units"], case["why"]


def test_tile_fit_boundary():
    assert oracle.layer_fits(range(12), 30)
    assert oracle.layer_fits([0, 1, 2] + list(range(20, 29)), 30)
    assert not oracle.layer_fits(list(range(20, 30)), 30)
    assert oracle.layer_fits(list(range(3, 12)), 12)
    assert not oracle.layer_fits(list(range(2, 12)) + [0, 1, 12], 13)
    assert oracle.layer_fits(range(8), 8)


def test_qaoa_layers_cover_each_round_in_three_passes():
    """The QAOA bench circuit (N = 30, p = 8): 30 H, then per round 45 ZZ and
    30 RX; each block holds at most 12 factor qubits, so a round needs at
    least three passes, and the grouping reaches that."""
    ops, _ = W.qaoa_circuit(30, 8, 0)
    order, units = oracle.layer_units(ops, 30)
    assert all(u[2] for u in units)
    assert len(units) == 3 + 8 * 3
