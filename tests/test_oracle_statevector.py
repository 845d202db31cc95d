"""Pins for the FP64 oracle's state-vector arithmetic (no GPU).

Each test checks the oracle against something other than itself: an
independently built Kronecker matrix, a closed form, an invariant, or the
paper's worked example (Fig. axis-shift-tensor, §IV-B).
"""
import json
import os

import numpy as np
import pytest

import oracle
import workloads as W

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


@pytest.mark.parametrize("n,k,seed", [(3, 1, 0), (4, 2, 1), (5, 3, 2), (6, 4, 3), (7, 5, 4), (8, 6, 5), (8, 2, 6),
                                      (6, 6, 7), (1, 1, 8)])
def test_apply_matches_full_kronecker_operator(n, k, seed):
    """orc_apply on any ordered target tuple equals P^T (I ⊗ G) P (N <= 8)."""
    rng = np.random.default_rng(seed)
    for trial in range(3):
        targets = tuple(int(v) for v in rng.choice(n, size=k, replace=False))
        G = W.haar_unitary(1 << k, rng)
        psi = W.random_state(n, seed=seed * 10 + trial)
        ref = oracle.full_operator(n, targets, G) @ psi
        out = psi.copy()
        oracle.apply(out, targets, G)
        assert np.max(np.abs(out - ref)) < 1e-13


def test_apply_target_order_matters():
    """A dropped or swapped target order would map CNOT(0->1) to CNOT(1->0)."""
    psi = oracle.zero_state(2)
    oracle.apply(psi, (0,), W.X)           # |01> (qubit 0 set): index 1
    oracle.apply(psi, (0, 1), W.CNOT)      # control 0 -> target 1: index 3
    assert abs(psi[3] - 1) < 1e-15
    psi = oracle.zero_state(2)
    oracle.apply(psi, (0,), W.X)
    oracle.apply(psi, (1, 0), W.CNOT)      # control 1 (clear): unchanged
    assert abs(psi[1] - 1) < 1e-15


@pytest.mark.parametrize("n", [2, 5, 10, 14])
def test_ghz_closed_form(n):
    psi = oracle.run_circuit(n, W.ghz_ops(n))
    ref = np.zeros(1 << n, dtype=np.complex128)
    ref[0] = ref[-1] = 1 / np.sqrt(2)
    assert np.max(np.abs(psi - ref)) < 1e-14


@pytest.mark.parametrize("n,seed", [(3, 0), (6, 1), (10, 2), (12, 3)])
def test_qft_of_basis_state_closed_form(n, seed):
    """QFT|x> = 2^{-n/2} sum_y exp(2 pi i x y / 2^n) |y>."""
    x = int(np.random.default_rng(seed).integers(0, 1 << n))
    psi = oracle.run_circuit(n, W.basis_prep(n, x) + W.qft_ops(n))
    y = np.arange(1 << n)
    ref = np.exp(2j * np.pi * ((x * y) % (1 << n)) / (1 << n)) / np.sqrt(1 << n)
    assert np.max(np.abs(psi - ref)) < 1e-12


def test_norm_preserved_and_inverse_returns_to_zero():
    n = 10
    ops, x0 = W.fusion_circuit(n=n, layers=4, seed=3, with_inverse=False)
    psi = oracle.run_circuit(n, ops)
    assert abs(np.vdot(psi, psi).real - 1) < 1e-12
    psi = oracle.run_circuit(n, W.inverse(ops), psi)
    ref = oracle.zero_state(n)
    assert np.max(np.abs(psi - ref)) < 1e-12


@pytest.mark.parametrize("seed", [0, 1, 2, 3])
def test_clifford_probabilities_are_dyadic(seed):
    """Stabiliser states: every probability is 0 or 2^-r, with 2^r nonzero."""
    n = 8
    psi = oracle.run_circuit(n, W.random_clifford(n, 60, seed))
    p = oracle.probabilities(psi)
    nz = p[p > 1e-12]
    r = int(round(-np.log2(nz[0])))
    assert len(nz) == 1 << r
    assert np.max(np.abs(nz - 2.0 ** -r)) < 1e-12
    assert np.all((p < 1e-12) | (np.abs(p - 2.0 ** -r) < 1e-12))


def test_expect_z_special_cases():
    n = 6
    # basis state |x>: <Z_mask> = (-1)^{popcount(x & mask)}
    x = 0b101101
    psi = oracle.run_circuit(n, W.basis_prep(n, x))
    for mask in [0, 1, 2, 4, 0b111111, 0b100001]:
        assert oracle.expect_z(psi, mask) == (-1) ** bin(x & mask).count("1")
    # GHZ: <Z_a> = 0, <Z_a Z_b> = 1, empty mask = norm
    psi = oracle.run_circuit(n, W.ghz_ops(n))
    assert abs(oracle.expect_z(psi, 1 << 3)) < 1e-15
    assert abs(oracle.expect_z(psi, (1 << 1) | (1 << 4)) - 1) < 1e-15
    assert abs(oracle.expect_z(psi, 0) - 1) < 1e-15


@pytest.mark.parametrize("seed", [0, 1])
def test_block_product_equals_sequential_application(seed):
    """§IV-C: a block's product (later gates on the left) applied once equals
    its gates applied one by one."""
    rng = np.random.default_rng(seed)
    n = 7
    gates = []
    for _ in range(6):
        k = int(rng.integers(1, 3))
        t = tuple(int(v) for v in rng.choice([1, 3, 4, 6], size=k, replace=False))
        gates.append(W.Op(t, W.haar_unitary(1 << k, rng)))
    block_targets = sorted({q for g in gates for q in g.targets})
    M = oracle.block_product(gates, block_targets)
    psi = W.random_state(n, seed)
    a = psi.copy()
    for g in gates:
        oracle.apply(a, g.targets, g.matrix)
    b = psi.copy()
    oracle.apply(b, block_targets, M)
    assert np.max(np.abs(a - b)) < 1e-13
    # and a reversed multiplication order is detectably wrong
    M_bad = np.eye(1 << len(block_targets), dtype=np.complex128)
    for g in gates:
        M_bad = M_bad @ oracle.kron_embed(g.matrix, g.targets, block_targets)
    c = psi.copy()
    oracle.apply(c, block_targets, M_bad)
    assert np.max(np.abs(a - c)) > 1e-3


def test_fig2_axis_shift_worked_example():
    """§IV-B, Fig. axis-shift-tensor: identity layout, V = (2, 4); after lazy
    TTGT the stored row-major axis order is (4, 2, N-1, ..., 5, 3, 1, 0)."""
    with open(os.path.join(GOLDEN, "fig2_axis_shift.json")) as f:
        g = json.load(f)
    n = g["N"]
    rng = np.random.default_rng(0)
    G = W.haar_unitary(4, rng)
    psi = W.random_state(n, 1)
    Lp, stored = oracle.lazy_ttgt(psi.copy(), list(range(n)), tuple(g["V"]), G)
    # row-major axis order: logical qubit at physical position N-1, N-2, ..., 0
    order = [Lp.index(pos) for pos in range(n - 1, -1, -1)]
    assert order == g["row_major_axis_order"]
    # Theorem 1: decoding the stored state through L' gives the canonical result
    ref = psi.copy()
    oracle.apply(ref, tuple(g["V"]), G)
    assert np.max(np.abs(oracle.decode_state(stored, Lp) - ref)) < 1e-13


def test_decode_encode_roundtrip_and_theorem1_random_layouts():
    """Theorem 1 (component form): with stored = Pi_L psi, applying G on the
    physical targets L(V) and decoding equals applying G on V canonically."""
    n = 7
    rng = np.random.default_rng(5)
    for _ in range(4):
        L = [int(v) for v in rng.permutation(n)]
        psi = W.random_state(n, int(rng.integers(1 << 30)))
        stored = oracle.encode_state(psi, L)
        assert np.array_equal(oracle.decode_state(stored, L), psi)
        V = tuple(int(v) for v in rng.choice(n, size=3, replace=False))
        G = W.haar_unitary(8, rng)
        oracle.apply(stored, tuple(L[q] for q in V), G)
        ref = psi.copy()
        oracle.apply(ref, V, G)
        assert np.max(np.abs(oracle.decode_state(stored, L) - ref)) < 1e-13
