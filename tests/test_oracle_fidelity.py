"""Closed-form pins of the oracle's parity metrics (no GPU): the fidelity
F = |<psi_ref|psi>|^2 without renormalisation, so a norm change counts
against it, and the largest amplitude difference max_i |psi_ref_i - psi_i|.

Every GPU parity verdict goes through these two functions, so each is held
to values fixed by the mathematics: a dropped square, a renormalisation, a
real part taken instead of the modulus, or a sum or 2-norm in place of the
maximum fails one of them.
"""
import numpy as np

import oracle
import workloads as W


def test_fidelity_of_zero_and_plus_is_one_half():
    zero = np.array([1, 0], dtype=np.complex128)
    plus = W.H @ zero
    assert abs(oracle.fidelity(zero, plus) - 0.5) < 1e-15


def test_fidelity_ignores_a_global_phase():
    psi = W.random_state(6, seed=3).astype(np.complex128)
    psi /= np.linalg.norm(psi)
    for th in (0.3, np.pi / 2, np.pi, 4.0):
        assert abs(oracle.fidelity(psi, np.exp(1j * th) * psi) - 1) < 1e-13


def test_fidelity_counts_a_norm_change():
    psi = W.random_state(5, seed=4).astype(np.complex128)
    psi /= np.linalg.norm(psi)
    assert abs(oracle.fidelity(psi, 0.999 * psi) - 0.998001) < 1e-13


def test_fidelity_of_a_rotated_pair():
    """|00> against cos a |00> + sin a |11>: F = cos^2 a; orthogonal states give 0."""
    ref = np.zeros(4, dtype=np.complex128)
    ref[0] = 1
    for a in (0.0, 0.4, 1.1, np.pi / 2):
        psi = np.zeros(4, dtype=np.complex128)
        psi[0], psi[3] = np.cos(a), 1j * np.sin(a)
        assert abs(oracle.fidelity(ref, psi) - np.cos(a) ** 2) < 1e-15
    assert oracle.fidelity(ref, np.array([0, 1, 0, 0], dtype=np.complex128)) == 0.0


def test_max_abs_diff_is_the_largest_modulus():
    a = np.array([0.1, 0.3j, 0, 0], dtype=np.complex128)
    assert abs(oracle.max_abs_diff(a, np.zeros(4)) - 0.3) < 1e-15      # not the sum 0.4 nor the 2-norm
    basis = np.zeros(8, dtype=np.complex128)
    basis[5] = 1
    th = 0.7
    assert abs(oracle.max_abs_diff(basis, np.exp(1j * th) * basis) - 2 * np.sin(th / 2)) < 1e-15
    psi = W.random_state(4, seed=1).astype(np.complex128)
    assert abs(oracle.max_abs_diff(psi, -psi) - 2 * np.max(np.abs(psi))) < 1e-15
