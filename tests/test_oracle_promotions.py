"""Pins for the oracle's replay of on-demand promotions (§IV-D, Corollary
"ideal minimal demand-promotion count"; first-free rule beside it), no GPU.

- a hand-worked example (tests/golden/promotions_hand_example.json);
- the Corollary itself: on tiny streams, farthest-next-use reaches the minimum
  total promotion count found by exhaustive search over all victim choices;
- invariants on larger streams: every target is local when its tuple runs,
  the layout stays a bijection, first-free never beats farthest-next-use.
"""
import json
import os

import numpy as np
import pytest

import oracle

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


def test_hand_worked_example():
    g = json.load(open(os.path.join(GOLDEN, "promotions_hand_example.json")))
    for pol in ("first_free", "farthest"):
        counts, lay = oracle.promotion_replay(g["tuples"], g["n"], g["frames"], pol, g["layout"])
        assert counts == g[pol]["counts"] and lay == g[pol]["layout"], pol


def _brute_min(tuples, n, frames, L):
    """Minimum total promotions over every sequence of eligible victims."""
    best = [float("inf")]

    def rec(i, L, acc):
        if acc >= best[0]:
            return
        if i == len(tuples):
            best[0] = acc
            return
        tup = tuples[i]
        missing = [q for q in tup if L[q] >= frames]

        def place(mi, L, pinned, acc):
            if mi == len(missing):
                rec(i + 1, L, acc)
                return
            q = missing[mi]
            inv = {p: qq for qq, p in enumerate(L)}
            for v in range(frames):
                if v in pinned:
                    continue
                L2 = list(L)
                qv = inv[v]
                L2[q], L2[qv] = v, L[q]
                place(mi + 1, L2, pinned | {v}, acc + 1)

        place(0, L, {L[q] for q in tup if L[q] < frames}, acc)

    rec(0, list(L), 0)
    return best[0]


@pytest.mark.parametrize("seed", range(12))
def test_farthest_next_use_is_minimal_on_tiny_streams(seed):
    rng = np.random.default_rng(seed)
    n = int(rng.integers(4, 7))
    frames = int(rng.integers(2, 4))
    tuples = []
    for _ in range(int(rng.integers(4, 8))):
        k = int(rng.integers(1, min(2, frames) + 1))
        tuples.append([int(v) for v in rng.choice(n, size=k, replace=False)])
    L = [int(v) for v in rng.permutation(n)]
    far, _ = oracle.promotion_replay(tuples, n, frames, "farthest", L)
    ff, _ = oracle.promotion_replay(tuples, n, frames, "first_free", L)
    m = _brute_min(tuples, n, frames, L)
    assert sum(far) == m
    assert sum(ff) >= m


@pytest.mark.parametrize("policy", ["first_free", "farthest"])
def test_invariants_on_long_streams(policy):
    """Every target is local when its tuple runs, the layout stays a
    bijection, and (Corollary) farthest-next-use never needs more promotions
    than first-free."""
    rng = np.random.default_rng(5)
    n, frames = 20, 11
    tuples = [[int(v) for v in rng.choice(n, size=int(rng.integers(1, 7)), replace=False)] for _ in range(300)]
    counts, L, hist = oracle.promotion_replay(tuples, n, frames, policy, None, history=True)
    for t, lay in zip(tuples, hist):
        assert sorted(lay) == list(range(n))
        assert all(lay[q] < frames for q in t)
    assert hist[-1] == L
    far, _ = oracle.promotion_replay(tuples, n, frames, "farthest")
    ff, _ = oracle.promotion_replay(tuples, n, frames, "first_free")
    assert sum(far) <= sum(ff)
