"""Pins for the oracle's fusion pipeline as a whole (no GPU): Eq. dp-recurrence
per window, the cross-window merge and its repeats (§IV-C).  Its parts are
pinned elsewhere (the DP by exhaustive enumeration); here the composition is
held to what must hold whatever the windows and repeats do:
  * the blocks partition the ops into contiguous runs, in order;
  * every block respects the width cap of its mode (dense kmax, all-diagonal
    kmax_diag);
  * applying the fused blocks (each the product of its ops) gives the
    circuit's state;
  * the total Gamma never exceeds that of the per-gate partition or of one
    pass of the DP over the whole stream in windows (a merge is taken only
    when it does not raise Gamma, and a repeat starts from the previous
    blocks);
  * repeats stop once the block count no longer falls: more allowed repeats
    than needed change nothing.
A merge that ignores the cap, joins across a gap, or raises Gamma, and a
block product in the wrong order, each fail one of these."""
import numpy as np
import pytest

import oracle
import workloads as W


def _circuit(rng, n, n_ops, kin=3, diag_frac=0.35):
    ops = []
    for _ in range(n_ops):
        k = int(rng.integers(1, kin + 1))
        t = tuple(int(v) for v in rng.choice(n, size=k, replace=False))
        if rng.random() < diag_frac:
            ops.append(W.Op(t, np.diag(np.exp(1j * rng.uniform(0, 2 * np.pi, 1 << k))), True))
        else:
            ops.append(W.Op(t, W.haar_unitary(1 << k, rng), False))
    return ops


def _blocks(ops, starts):
    ends = starts[1:] + [len(ops)]
    return [(s, e) for s, e in zip(starts, ends)]


def _gamma(ops, blocks):
    tot = 0.0
    for s, e in blocks:
        t = set()
        for o in ops[s:e]:
            t |= set(o.targets)
        tot += oracle.gamma_score(len(t), all(o.diag for o in ops[s:e]))
    return tot


@pytest.mark.parametrize("seed,n,n_ops,kmax,kdiag,window,rounds",
                         [(0, 6, 40, 3, 3, 8, 4), (1, 7, 60, 4, 6, 5, 4), (2, 8, 80, 2, 4, 16, 2),
                          (3, 6, 50, 3, 5, 64, 4), (4, 5, 45, 4, 4, 3, 4)])
def test_pipeline_invariants(seed, n, n_ops, kmax, kdiag, window, rounds):
    rng = np.random.default_rng(seed)
    ops = _circuit(rng, n, n_ops, kin=min(3, kmax))
    starts = oracle.fuse_pipeline(ops, kmax, kdiag, window, rounds)
    assert starts[0] == 0 and all(a < b for a, b in zip(starts, starts[1:])) and starts[-1] < len(ops)
    blocks = _blocks(ops, starts)
    psi = oracle.zero_state(n)
    psi[:] = W.random_state(n, seed=seed).astype(np.complex128)
    ref = oracle.run_circuit(n, ops, psi.copy())
    got = psi.copy()
    for s, e in blocks:
        t = sorted({q for o in ops[s:e] for q in o.targets})
        cap = kdiag if all(o.diag for o in ops[s:e]) else kmax
        assert len(t) <= cap
        oracle.apply(got, t, oracle.block_product(ops[s:e], t))
    assert np.max(np.abs(got - ref)) < 1e-10
    per_gate = [(i, i + 1) for i in range(len(ops))]
    one_pass = _blocks(ops, oracle.fuse_pipeline(ops, kmax, kdiag, window, 1))
    assert _gamma(ops, blocks) <= _gamma(ops, one_pass) + 1e-9 <= _gamma(ops, per_gate) + 2e-9
    # more repeats than the pipeline takes change nothing
    assert oracle.fuse_pipeline(ops, kmax, kdiag, window, 50) == oracle.fuse_pipeline(ops, kmax, kdiag, window,
                                                                                      rounds + 50)


def test_reversed_block_product_is_caught():
    """The state check above is sensitive to the order of a block's product:
    a block of two non-commuting gates applied in reverse differs."""
    rng = np.random.default_rng(9)
    ops = [W.Op((0, 1), W.haar_unitary(4, rng), False), W.Op((1, 2), W.haar_unitary(4, rng), False)]
    psi = W.random_state(3, seed=1).astype(np.complex128)
    ref = oracle.run_circuit(3, ops, psi.copy())
    bad = psi.copy()
    oracle.apply(bad, [0, 1, 2], oracle.block_product(ops[::-1], [0, 1, 2]))
    assert np.max(np.abs(bad - ref)) > 1e-3
