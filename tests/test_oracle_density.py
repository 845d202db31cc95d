"""Pins for the oracle's density-matrix functions (no GPU): pure-state
evolution against the state-vector oracle, the depolarising closed form,
trace, Hermiticity and positivity of random channels, and the vectorised
superoperator convention (row bits low, column bits high) against both."""
import numpy as np
import pytest

import oracle
import workloads as W


def _random_channel(k, r, rng):
    return W.random_kraus(k, r, rng)


def test_pure_state_evolution_matches_state_vector_oracle():
    n = 5
    ops = W.brick_circuit(n, 3, seed=1)
    rho = oracle.dm_zero(n)
    for o in ops:
        rho = oracle.dm_apply_channel(rho, o.targets, [o.matrix])
    psi = oracle.run_circuit(n, ops)
    assert np.max(np.abs(rho - np.outer(psi, psi.conj()))) < 1e-12


def test_depolarising_closed_form():
    """(1-p) rho + p/3 (X rho X + Y rho Y + Z rho Z) on one qubit of a product
    state equals (1 - 4p/3) rho + 4p/3 (Tr_q rho) (x) I/2 there."""
    rng = np.random.default_rng(2)
    p = 0.3
    a = W.random_state(1, seed=4)
    b = W.random_state(2, seed=5)
    psi = np.kron(b, a)                 # qubit 0 = a, qubits 1..2 = b
    rho = np.outer(psi, psi.conj())
    X = np.array([[0, 1], [1, 0]]); Y = np.array([[0, -1j], [1j, 0]]); Z = np.diag([1, -1])
    kr = [np.sqrt(1 - p) * np.eye(2), np.sqrt(p / 3) * X, np.sqrt(p / 3) * Y, np.sqrt(p / 3) * Z]
    out = oracle.dm_apply_channel(rho, (0,), kr)
    ra = np.outer(a, a.conj())
    rb = np.outer(b, b.conj())
    ref = np.kron(rb, (1 - 4 * p / 3) * ra + (4 * p / 3) * np.eye(2) / 2)
    assert np.max(np.abs(out - ref)) < 1e-13


@pytest.mark.parametrize("k,r,seed", [(1, 3, 0), (2, 4, 1), (3, 2, 2)])
def test_random_channels_preserve_trace_hermiticity_positivity(k, r, seed):
    rng = np.random.default_rng(seed)
    n = 5
    psi = W.random_state(n, seed=seed)
    rho = np.outer(psi, psi.conj())
    t = [int(v) for v in rng.choice(n, size=k, replace=False)]
    out = oracle.dm_apply_channel(rho, t, _random_channel(k, r, rng))
    assert abs(np.trace(out) - 1) < 1e-12
    assert np.max(np.abs(out - out.conj().T)) < 1e-13
    assert np.min(np.linalg.eigvalsh(out)) > -1e-12


@pytest.mark.parametrize("k,seed", [(1, 0), (2, 1), (3, 2)])
def test_superoperator_on_the_vectorised_matrix(k, seed):
    """vec(sum E rho E^dagger) = (sum conj(E) (x) E) vec(rho) applied to the
    2n-axis vector at targets (t, t + n): row copies first (low bits), column
    copies second (high bits); the transposed convention is detected."""
    rng = np.random.default_rng(seed)
    n = 4
    kr = _random_channel(k, 2, rng)
    t = [int(v) for v in rng.choice(n, size=k, replace=False)]
    A = W.random_state(2 * n, seed=seed).reshape(1 << n, 1 << n)
    rho = A @ A.conj().T
    rho /= np.trace(rho)
    ref = oracle.dm_apply_channel(rho, t, kr)
    v = oracle.dm_vec(rho)
    oracle.apply(v, list(t) + [q + n for q in t], oracle.dm_superoperator(kr))
    assert np.max(np.abs(oracle.dm_unvec(v) - ref)) < 1e-12
    w = oracle.dm_vec(rho)
    oracle.apply(w, [q + n for q in t] + list(t), oracle.dm_superoperator(kr))
    assert np.max(np.abs(oracle.dm_unvec(w) - ref)) > 1e-6
