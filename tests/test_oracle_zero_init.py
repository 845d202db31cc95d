"""Pins for the oracle's zero-state prefix (no GPU): the closed form
prod_q a_q[x_q] * prod_g d_g(x) equals running the prefix gate by gate from
|0...0> on random circuits (a one-qubit op taken after a diagonal gate on its
qubit, or a reversed bit order, breaks it); the prefix stops where the rule
says on hand cases (a dense op, a three-qubit diagonal, a one-qubit op after
a diagonal gate on its qubit)."""
import numpy as np
import pytest

import oracle
import workloads as W
from test_oracle_layer import _mixed_circuit


@pytest.mark.parametrize("n,seed", [(4, 0), (5, 1), (6, 2), (8, 3), (7, 4)])
def test_closed_form_equals_gate_by_gate(n, seed):
    rng = np.random.default_rng(seed)
    ops = [W.Op((q,), W.haar_unitary(2, rng), False) for q in range(n)] + _mixed_circuit(n, 40, rng)
    P = oracle.zero_init_prefix(ops)
    assert P >= n
    ref = oracle.run_circuit(n, ops[:P])
    assert np.max(np.abs(oracle.zero_init_state(n, ops[:P]) - ref)) < 1e-12


def test_qaoa_prefix_is_h_layer_and_first_cost_layer():
    ops, edges = W.qaoa_circuit(16, 3, seed=0)
    P = oracle.zero_init_prefix(ops)
    assert P == 16 + len(edges)
    ref = oracle.run_circuit(16, ops[:P])
    assert np.max(np.abs(oracle.zero_init_state(16, ops[:P]) - ref)) < 1e-12


def test_prefix_hand_cases():
    h, x = W.H, W.X
    zz = np.diag(np.exp(1j * np.array([0.1, 0.2, 0.3, 0.4])))
    ops = [W.Op((0,), h), W.Op((0,), x), W.Op((0, 1), zz, True), W.Op((2,), h), W.Op((1,), h)]
    assert oracle.zero_init_prefix(ops) == 4          # H(1) after the ZZ on 1 stops it
    ops = [W.Op((0, 1), W.CNOT), W.Op((0,), h)]
    assert oracle.zero_init_prefix(ops) == 0          # a dense two-qubit op first
    ops = [W.Op((0, 1, 2), np.eye(8), True), W.Op((0,), h)]
    assert oracle.zero_init_prefix(ops) == 0          # diagonal on three qubits is not taken
