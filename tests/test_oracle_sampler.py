"""Pins for the oracle's counter-based generator and CDF sampler (no GPU)."""
import math
from fractions import Fraction

import numpy as np
import pytest
from scipy import stats

import oracle
import workloads as W


@pytest.mark.parametrize("key,ctr", [((0, 0), (0, 0, 0, 0)), ((0x1234, 0x5678), (7, 0, 0, 0)),
                                      ((2**64 - 1, 3), (2**64 - 1, 5, 9, 11)), ((42, 0), (123456789, 17, 0, 0))])
def test_philox4x64_10_matches_numpy(key, ctr):
    """numpy.random.Philox is Philox4x64-10; it increments the 256-bit counter
    (with carry) before each block, so its first block is our block at ctr+1."""
    c = np.array(ctr, dtype=np.uint64)
    bg = np.random.Philox(key=np.array(key, dtype=np.uint64), counter=c)
    ref = [int(v) for v in bg.random_raw(4)]
    nxt = list(ctr)
    for i in range(4):  # counter + 1 with carry
        nxt[i] = (nxt[i] + 1) % 2**64
        if nxt[i] != 0:
            break
    assert oracle.philox4x64_10(nxt, key) == ref


def _brute_force_sample(psi_logical, L, shots, seed, stream):
    """Same reading written with exact rationals and numpy's Philox: weights
    floor(re^2 2^60) + floor(im^2 2^60) in physical order, linear scan for the
    first cumulative value above u."""
    n = int(psi_logical.size).bit_length() - 1
    w = []
    for y in range(1 << n):
        x = sum(((y >> L[q]) & 1) << q for q in range(n))
        a = psi_logical[x]
        w.append(math.floor(Fraction(float(a.real)) ** 2 * 2 ** 60) +
                 math.floor(Fraction(float(a.imag)) ** 2 * 2 ** 60))
    total = sum(w)
    out = []
    for s in range(shots):
        # numpy's block at counter c is Philox(c + 1): start from (s - 1, stream)
        if s == 0:
            c = np.array([2**64 - 1, stream - 1, 0, 0], dtype=np.uint64)  # stream >= 1
        else:
            c = np.array([s - 1, stream, 0, 0], dtype=np.uint64)
        r = int(np.random.Philox(key=np.array([seed, 0], dtype=np.uint64), counter=c).random_raw(1)[0])
        u = (r * total) >> 64
        acc = 0
        for y in range(1 << n):
            acc += w[y]
            if acc > u:
                break
        out.append(sum(((y >> L[q]) & 1) << q for q in range(n)))
    return np.array(out, dtype=np.uint64)


@pytest.mark.parametrize("n,seed,perm", [(3, 0, False), (5, 1, True), (6, 2, True)])
def test_sampler_matches_brute_force(n, seed, perm):
    psi = W.random_state(n, seed, zero_frac=0.3)
    L = list(np.random.default_rng(seed).permutation(n)) if perm else list(range(n))
    out, _ = oracle.sample(psi, L, 64, seed=seed + 100, stream=3)
    ref = _brute_force_sample(psi, [int(v) for v in L], 64, seed + 100, 3)
    assert np.array_equal(out, ref)


def test_basis_state_gives_single_outcome():
    n = 9
    x = 0b101100111
    psi = oracle.run_circuit(n, W.basis_prep(n, x))
    L = [int(v) for v in np.random.default_rng(0).permutation(n)]
    out, _ = oracle.sample(psi, L, 500, seed=7)
    assert np.all(out == x)


def test_zero_probability_bins_never_drawn():
    """Strict upper bound (§IV-E): an empty bin is never selected."""
    n = 8
    psi = W.random_state(n, 3, zero_frac=0.7)
    out, _ = oracle.sample(psi, list(range(n)), 20000, seed=11)
    assert np.all(np.abs(psi[out.astype(np.int64)]) > 0)


def test_chi_square_goodness_of_fit_with_layout():
    n = 4
    psi = W.random_state(n, 9)
    L = [2, 0, 3, 1]
    shots = 40000
    out, _ = oracle.sample(psi, L, shots, seed=5)
    obs = np.bincount(out.astype(np.int64), minlength=1 << n)
    exp = np.abs(psi) ** 2 * shots
    chi2, pval = stats.chisquare(obs, exp)
    assert pval > 1e-4


def test_near_boundary_flags():
    n = 6
    psi = W.random_state(n, 2)
    _, f0 = oracle.sample(psi, list(range(n)), 1000, seed=1, near_frac=0.0)
    _, f1 = oracle.sample(psi, list(range(n)), 1000, seed=1, near_frac=1.0)
    assert f0.sum() == 0 and f1.all()
