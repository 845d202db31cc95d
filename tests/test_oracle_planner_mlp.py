"""Pins for the oracle's fusion partitions (§IV-C) and cost-model network."""
import itertools

import numpy as np
import pytest

import oracle
import workloads as W


def _gate(t, diag=False):
    return W.Op(tuple(t), np.eye(1 << len(t), dtype=np.complex128), diag)


def _partitions(h):
    for cuts in itertools.product([0, 1], repeat=h - 1):
        blocks, s = [], 0
        for i, c in enumerate(cuts):
            if c:
                blocks.append((s, i + 1))
                s = i + 1
        blocks.append((s, h))
        yield blocks


def _score(gates, blocks, kmax, kmax_diag):
    tot = 0.0
    for j, i in blocks:
        w = len({q for g in gates[j:i] for q in g.targets})
        diag = all(g.diag for g in gates[j:i])
        if w > (kmax_diag if diag else kmax) and i - j > 1:
            return None
        tot += oracle.gamma_score(w, diag)
    return tot


@pytest.mark.parametrize("seed", range(8))
def test_dp_partition_is_optimal_by_brute_force(seed):
    """Eq. dp-recurrence reaches the minimum of sum Gamma over every feasible
    partition of the window (exhaustive enumeration, h <= 10)."""
    rng = np.random.default_rng(seed)
    h = int(rng.integers(4, 11))
    gates = []
    for _ in range(h):
        k = int(rng.integers(1, 4))
        t = rng.choice(6, size=k, replace=False)
        gates.append(_gate(t, diag=bool(rng.random() < 0.4)))
    kmax, kmax_diag = 3, 3
    blocks = oracle.dp_window(gates, kmax, kmax_diag)
    got = _score(gates, blocks, kmax, kmax_diag)
    best = min(s for s in (_score(gates, b, kmax, kmax_diag) for b in _partitions(h)) if s is not None)
    assert got is not None and got == best
    assert blocks[0][0] == 0 and blocks[-1][1] == h
    assert all(a[1] == b[0] for a, b in zip(blocks, blocks[1:]))


def test_dp_over_cap_gate_stays_singleton():
    gates = [_gate([0]), _gate([0, 1, 2, 3]), _gate([1])]
    blocks = oracle.dp_window(gates, 2, 2)
    assert (1, 2) in blocks


def test_dp_tie_break_takes_smallest_start():
    """With a constant score, the final block [1,1,2] (j=1) wins over j=2,3."""
    gates = [_gate([0]), _gate([1]), _gate([1]), _gate([2])]
    blocks = oracle.dp_window(gates, 2, 2, score=lambda w, d, b: 1.0)
    assert blocks == [(0, 1), (1, 4)]


def test_greedy_partition_invariants():
    rng = np.random.default_rng(0)
    gates = [_gate(rng.choice(10, size=int(rng.integers(1, 3)), replace=False)) for _ in range(200)]
    for kmax in (2, 3, 4, 6):
        blocks = oracle.greedy_partition(gates, kmax)
        assert blocks[0][0] == 0 and blocks[-1][1] == len(gates)
        for (j, i), nxt in zip(blocks, blocks[1:] + [None]):
            w = len({q for g in gates[j:i] for q in g.targets})
            assert w <= kmax
            if nxt is not None:  # maximal: adding the next gate would overflow
                w2 = len({q for g in gates[j:i + 1] for q in g.targets})
                assert w2 > kmax


def _rand_params(rng, scale=0.3, nonneg=False):
    ps = [rng.standard_normal(s) * scale for s in oracle.MLP_SHAPES]
    if nonneg:
        ps = [np.abs(p) for p in ps]
    return ps


def test_mlp_forward_reduces_to_linear_map_when_relu_inactive():
    """With non-negative weights and inputs every ReLU passes its input, so
    the network is the affine map W3 W2 W1 x + W3 W2 b1 + W3 b2 + b3."""
    rng = np.random.default_rng(1)
    P = _rand_params(rng, nonneg=True)
    X = np.abs(rng.standard_normal((16, 37)))
    y, _ = oracle.mlp_forward(P, X)
    W1, b1, W2, b2, W3, b3 = P
    ref = (W3 @ W2 @ W1 @ X.T)[0] + (W3 @ W2 @ b1)[0] + (W3 @ b2)[0] + b3[0]
    assert np.max(np.abs(y - ref)) < 1e-10


def test_mlp_gradients_match_central_differences():
    rng = np.random.default_rng(2)
    P = _rand_params(rng)
    X = rng.standard_normal((32, 37))
    t = rng.standard_normal(32)
    _, grads = oracle.mlp_loss_grad(P, X, t)
    h = 1e-6
    for pi in range(len(P)):
        flat = P[pi].reshape(-1)
        for idx in rng.choice(flat.size, size=min(6, flat.size), replace=False):
            old = flat[idx]
            flat[idx] = old + h
            lp, _ = oracle.mlp_loss_grad(P, X, t)
            flat[idx] = old - h
            lm, _ = oracle.mlp_loss_grad(P, X, t)
            flat[idx] = old
            num = (lp - lm) / (2 * h)
            ana = grads[pi].reshape(-1)[idx]
            assert abs(num - ana) <= 1e-6 * max(1.0, abs(num))


def test_adam_first_step_is_lr_times_sign():
    """At t = 1 the bias-corrected moments are g and g^2, so the update is
    lr * g / (|g| + eps)."""
    rng = np.random.default_rng(3)
    P = _rand_params(rng)
    G = [rng.standard_normal(p.shape) for p in P]
    Z = [np.zeros_like(p) for p in P]
    newP, m, v = oracle.adam_step(P, G, Z, Z, 1, lr=1e-3)
    for p, q, g in zip(P, newP, G):
        assert np.max(np.abs((p - q) - 1e-3 * g / (np.abs(g) + 1e-8))) < 1e-15
