"""Pins for the oracle's product lowering and product-unit grouping (no GPU):
the Kronecker product of the factors, a Hadamard-layer closed form, and the
grouping's defining properties checked by brute force."""
import numpy as np
import pytest

import oracle
import workloads as W


@pytest.mark.parametrize("n,k,seed", [(3, 2, 0), (6, 4, 1), (8, 8, 2), (7, 3, 3)])
def test_apply_product_equals_kronecker_of_factors(n, k, seed):
    """Equals the Kronecker operator of U_{k-1} (x) ... (x) U_0 (N <= 8)."""
    rng = np.random.default_rng(seed)
    t = [int(v) for v in rng.choice(n, size=k, replace=False)]
    fac = [W.haar_unitary(2, rng) for _ in range(k)]
    G = np.array([[1.0 + 0j]])
    for u in fac:                     # factor j acts on bit j of the block index
        G = np.kron(u, G)
    psi = W.random_state(n, seed=seed)
    ref = oracle.full_operator(n, t, G) @ psi
    out = psi.copy()
    oracle.apply_product(out, t, fac)
    assert np.max(np.abs(out - ref)) < 1e-13


def test_apply_product_hadamard_layer_closed_form():
    """H on every qubit of |0...0> gives the uniform superposition."""
    n = 9
    psi = oracle.zero_state(n)
    oracle.apply_product(psi, list(range(n)), [W.H] * n)
    assert np.max(np.abs(psi - 2 ** (-n / 2))) < 1e-14


@pytest.mark.parametrize("seed,kp", [(0, 4), (1, 11), (2, 2), (3, 1)])
def test_product_units_properties(seed, kp):
    """Units partition the ops in order; a multi-op unit holds only
    non-diagonal one-qubit ops on at most kp qubits and cannot be extended by
    the next op; runs never start in the middle of an extendable run."""
    rng = np.random.default_rng(seed)
    ops = []
    for _ in range(300):
        r = rng.random()
        if r < 0.6:
            ops.append(W.Op((int(rng.integers(0, 14)),), W.H.copy(), False))
        elif r < 0.8:
            ops.append(W.Op((int(rng.integers(0, 14)),), np.diag([1, 1j]), True))
        else:
            t = tuple(int(v) for v in rng.choice(14, size=2, replace=False))
            ops.append(W.Op(t, W.CZ.copy(), True))
    units = oracle.product_units(ops, kp)
    assert units[0][0] == 0 and units[-1][1] == len(ops)
    assert all(a[1] == b[0] for a, b in zip(units[:-1], units[1:]))
    single = lambda o: len(o.targets) == 1 and not o.diag
    for a, b in units:
        blk = ops[a:b]
        if b - a > 1:
            assert kp >= 2 and all(single(o) for o in blk)
            assert len({o.targets[0] for o in blk}) <= kp
        if kp >= 2 and all(single(o) for o in blk) and b < len(ops) and single(ops[b]):
            # the run stopped because the next op would exceed kp qubits
            assert ops[b].targets[0] not in {o.targets[0] for o in blk}
            assert len({o.targets[0] for o in blk}) == kp


@pytest.mark.parametrize("seed", [0, 1])
def test_fuse_product_equals_sequential_application(seed):
    """Per-qubit products in circuit order (repeated qubits included) applied
    as one product operator equal the ops applied one by one."""
    rng = np.random.default_rng(seed)
    n = 8
    ops = [W.Op((int(rng.integers(0, n)),), W.haar_unitary(2, rng), False) for _ in range(40)]
    t, fac = oracle.fuse_product(ops)
    psi = W.random_state(n, seed=seed)
    seq = psi.copy()
    for o in ops:
        oracle.apply(seq, o.targets, o.matrix)
    out = psi.copy()
    oracle.apply_product(out, t, fac)
    assert np.max(np.abs(out - seq)) < 1e-12
    # a transposed product order (earlier op on the left) is detected
    bad = {}
    for o in ops:
        q = o.targets[0]
        bad[q] = bad.get(q, np.eye(2)) @ o.matrix
    out2 = psi.copy()
    oracle.apply_product(out2, sorted(bad), [bad[q] for q in sorted(bad)])
    assert np.max(np.abs(out2 - seq)) > 1e-3
