"""Host-only checks of the density-matrix lowering (no GPU): the library's
superoperator of a channel equals the oracle's sum of conj(E) (x) E with the
row copies first (§IV-B density-matrix wrapper), lowered channels fuse through
the host block product into operators that act on vec(rho) like the channels
themselves, and bad arguments are rejected."""
import numpy as np
import pytest

import oracle
import workloads as W


@pytest.fixture(scope="module")
def q():
    import __graft_entry__
    __graft_entry__._build_module().build()
    import paper_2608_16940_gb300 as q
    return q


@pytest.mark.parametrize("k,r,n,seed", [(1, 1, 2, 0), (1, 4, 5, 1), (2, 3, 4, 2), (2, 16, 9, 3), (3, 2, 17, 4),
                                        (3, 1, 6, 5)])
def test_superoperator_matches_oracle(q, k, r, n, seed):
    rng = np.random.default_rng(seed)
    t = [int(v) for v in rng.choice(n, size=k, replace=False)]
    kr = W.random_kraus(k, r, rng)
    op = q.qsa_dm_superoperator(n, t, kr)
    assert list(op.targets) == t + [v + n for v in t]
    ref = oracle.dm_superoperator(kr)
    assert np.max(np.abs(op.matrix - ref)) < 1e-14


def test_lowered_channels_fuse_into_the_channel_sequence(q):
    """A CNOT then two-qubit depolarising noise, lowered and fused into one
    4-axis operator, acts on vec(rho) as the two channels do on rho."""
    n = 3
    rng = np.random.default_rng(7)
    psi = W.random_state(n, seed=7)
    rho = np.outer(psi, psi.conj())
    chans = [W.Channel((2, 0), [W.CNOT]), W.Channel((2, 0), W.depolarising_kraus(2, 0.2)),
             W.Channel((1,), W.random_kraus(1, 3, rng))]
    ops = [q.qsa_dm_superoperator(n, c.targets, c.kraus) for c in chans]
    t, M = q.qsa_fuse_ops(ops)
    v = oracle.dm_vec(rho).copy()
    oracle.apply(v, t, M)
    ref = rho
    for c in chans:
        ref = oracle.dm_apply_channel(ref, c.targets, c.kraus)
    assert np.max(np.abs(oracle.dm_unvec(v) - ref)) < 1e-13


def test_superoperator_argument_errors(q):
    e1 = [np.eye(2)]
    for args in [(1, [0], e1), (18, [0], e1), (4, [4], e1), (4, [-1], e1), (4, [1, 1], [np.eye(4)]),
                 (4, [0, 1, 2, 3], [np.eye(16)]), (4, [0], np.zeros((0, 2, 2)))]:
        with pytest.raises(q.QsaError) as e:
            q.qsa_dm_superoperator(*args)
        assert e.value.code == q.QSA_E_ARG
