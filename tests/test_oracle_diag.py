"""Pins for the oracle's diagonal branch (Alg. 2, diag mode) and the fused
diagonal of a block of diagonal gates (no GPU).

Each test checks the oracle against something other than itself: the
independently built Kronecker operator of diag(d), the tensor-axis
(broadcast) form of the same product, closed forms of Z and ZZ rotations, the
dense block product, sequential application, and commutativity.
"""
import numpy as np
import pytest

import oracle
import workloads as W


def _random_diag(k, rng, unit=False):
    d = rng.standard_normal(1 << k) + 1j * rng.standard_normal(1 << k)
    return d / np.abs(d) if unit else d


@pytest.mark.parametrize("n,k,seed", [(1, 1, 0), (3, 2, 1), (5, 3, 2), (7, 5, 3), (8, 6, 4), (8, 8, 5)])
def test_apply_diag_equals_kronecker_operator(n, k, seed):
    """psi <- d[c(x)] equals P^T (I ⊗ diag(d)) P psi, for any target order and
    non-unitary d (N <= 8)."""
    rng = np.random.default_rng(seed)
    for trial in range(3):
        t = tuple(int(v) for v in rng.choice(n, size=k, replace=False))
        d = _random_diag(k, rng)
        psi = W.random_state(n, seed=seed * 7 + trial)
        ref = oracle.full_operator(n, t, np.diag(d)) @ psi
        out = psi.copy()
        oracle.apply_diag(out, t, d)
        assert np.max(np.abs(out - ref)) < 1e-13


@pytest.mark.parametrize("n,k,seed", [(10, 10, 0), (13, 12, 1), (12, 7, 2)])
def test_apply_diag_equals_tensor_axis_broadcast(n, k, seed):
    """Wide operators: the same product written as a broadcast over the state
    tensor's axes (axis n-1-q holds qubit q), beyond Kronecker sizes."""
    rng = np.random.default_rng(seed)
    t = [int(v) for v in rng.choice(n, size=k, replace=False)]
    d = _random_diag(k, rng)
    psi = W.random_state(n, seed=seed)
    # d as a k-axis tensor: axis k-1-j holds bit j (target t[j])
    dt = d.reshape([2] * k)
    # move d's axes to the state's axes n-1-t[j], size-1 elsewhere
    src = [k - 1 - j for j in range(k)]
    dst = [n - 1 - t[j] for j in range(k)]
    order = np.argsort(dst)
    dfull = np.transpose(dt, [src[i] for i in order])
    shape = [1] * n
    for ax in dst:
        shape[ax] = 2
    ref = (psi.reshape([2] * n) * dfull.reshape(shape)).reshape(-1)
    out = psi.copy()
    oracle.apply_diag(out, t, d)
    assert np.max(np.abs(out - ref)) < 1e-13


def test_apply_diag_closed_forms():
    """Z on qubit q flips the sign of the amplitudes with bit q set; the ZZ
    rotation exp(-i g/2 Z_a Z_b) = cos(g/2) I - i sin(g/2) Z_a Z_b."""
    n = 6
    psi = W.random_state(n, seed=3)
    x = np.arange(1 << n)
    out = psi.copy()
    oracle.apply_diag(out, (4,), np.array([1.0, -1.0]))
    assert np.max(np.abs(out - psi * (1 - 2 * ((x >> 4) & 1)))) < 1e-15
    g = 0.7
    zz = np.array([1, -1, -1, 1], dtype=float)
    out = psi.copy()
    oracle.apply_diag(out, (1, 5), np.exp(-0.5j * g * zz))
    s = (1 - 2 * ((x >> 1) & 1)) * (1 - 2 * ((x >> 5) & 1))
    ref = np.cos(g / 2) * psi - 1j * np.sin(g / 2) * s * psi
    assert np.max(np.abs(out - ref)) < 1e-14


def test_apply_diag_target_order_matters():
    """Bit j of the index is target j: swapping targets needs the entries
    permuted to match, and an asymmetric table detects a transposed order."""
    n = 4
    psi = W.random_state(n, seed=1)
    d = np.array([1.0, 2.0, 3.0, 4.0])
    a = psi.copy()
    oracle.apply_diag(a, (0, 2), d)
    b = psi.copy()
    oracle.apply_diag(b, (2, 0), d[[0, 2, 1, 3]])
    c = psi.copy()
    oracle.apply_diag(c, (2, 0), d)
    assert np.max(np.abs(a - b)) < 1e-15
    assert np.max(np.abs(a - c)) > 0.1


@pytest.mark.parametrize("seed", [0, 1, 2])
def test_fuse_diag_equals_dense_block_product(seed):
    """The fused diagonal equals the diagonal of the dense block product
    (§IV-C), whose off-diagonal part is zero."""
    rng = np.random.default_rng(seed)
    n = 8
    gates = []
    for _ in range(12):
        k = int(rng.integers(1, 4))
        t = tuple(int(v) for v in rng.choice(n, size=k, replace=False))
        gates.append(W.Op(t, np.diag(_random_diag(k, rng)), True))
    bt = sorted({q for g in gates for q in g.targets})[:6]
    gates = [g for g in gates if set(g.targets) <= set(bt)]
    M = oracle.block_product(gates, bt)
    d = oracle.fuse_diag(gates, bt)
    assert np.max(np.abs(M - np.diag(d))) < 1e-12


@pytest.mark.parametrize("seed,width", [(0, 8), (1, 12)])
def test_fuse_diag_equals_sequential_and_commutes(seed, width):
    """Applying the fused diagonal once equals applying the gates one by one;
    diagonal gates commute, so the reversed order gives the same diagonal."""
    rng = np.random.default_rng(seed)
    n = width + 1
    gates = []
    for _ in range(30):
        k = int(rng.integers(1, 3))
        t = tuple(int(v) for v in rng.choice(width, size=k, replace=False))
        gates.append(W.Op(t, np.diag(_random_diag(k, rng, unit=True)), True))
    bt = sorted({q for g in gates for q in g.targets})
    d = oracle.fuse_diag(gates, bt)
    psi = W.random_state(n, seed=seed)
    seq = psi.copy()
    for g in gates:
        oracle.apply(seq, g.targets, g.matrix)
    fused = psi.copy()
    oracle.apply_diag(fused, bt, d)
    assert np.max(np.abs(seq - fused)) < 1e-12
    assert np.max(np.abs(oracle.fuse_diag(gates[::-1], bt) - d)) < 1e-12
