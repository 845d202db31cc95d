"""Batched noisy trajectories: one persistent launch (captured in a CUDA
graph) evolves many states of uneven depth; every state and its sampled
counts are checked against the FP64 oracle.

Counts: the oracle samples its own FP64 state with the same Philox stream
(trajectory index) and seed.  Every cumulative weight of the two states
differs by at most delta = sum_y |p_gpu(y) - p_ref(y)|, and the multiply-high
draw moves by at most |total_gpu - total_ref| <= delta, so a draw can differ
only when the oracle's u lies within 2 delta of a CDF boundary: the multiset
difference is bounded by twice the oracle's near-boundary flags at that
distance."""
import numpy as np
import pytest

import oracle
import workloads as W
from gpu_helpers import check_close

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def q():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_2608_16940_gb300 as q
    return q


def _check_counts(vals, cnts, psi_ref, psi_gpu, n, shots, seed, stream):
    delta = float(np.sum(np.abs(np.abs(psi_gpu) ** 2 - np.abs(psi_ref) ** 2)))
    out, flg = oracle.sample(psi_ref, list(range(n)), shots, seed, stream, near_frac=2 * delta + 1e-15)
    rv, rc = np.unique(out, return_counts=True)
    got = dict(zip(vals.astype(np.int64).tolist(), cnts.astype(np.int64).tolist()))
    ref = dict(zip(rv.astype(np.int64).tolist(), rc.astype(np.int64).tolist()))
    diff = sum(abs(got.get(k, 0) - ref.get(k, 0)) for k in set(got) | set(ref))
    assert diff <= 2 * int(flg.sum()), (diff, int(flg.sum()))
    assert int(cnts.sum()) == shots


@pytest.mark.parametrize("use_graph", [0, 1])
def test_batch_matches_oracle(q, use_graph):
    n, n_traj, shots, seed = 10, 12, 3000, 5
    trajs, depths = W.trajectory_batch(n_traj=n_traj, n=n, dmin=2, dmax=9, seed=3, p=0.05)
    b = q.qsa_batch_create(n, trajs, q.make_opts(planner=q.QSA_PLAN_DP, kmax=4, kmax_diag=4))
    states = torch.zeros(n_traj << n, dtype=torch.complex64, device="cuda:0")
    try:
        for rep in range(2):   # a replay gives the same results
            q.qsa_batch_run(b, states.data_ptr(), states.numel() * 8, shots, seed, 0, use_graph)
            res = q.qsa_batch_counts(b, n_traj, shots)
            got = states.cpu().numpy().reshape(n_traj, 1 << n).astype(np.complex128)
            for t in range(n_traj):
                ref = oracle.run_circuit(n, trajs[t])
                check_close(ref, got[t])
                _check_counts(res[t][0], res[t][1], ref, got[t], n, shots, seed, t)
    finally:
        q.qsa_batch_destroy(b)


@pytest.mark.parametrize("n", [6, 11, 13, 15])
def test_cluster_edge_cases(q, n):
    """A trajectory runs on a cluster of CTAs that split each pass's tiles:
    states of one tile (all but one CTA idle), of a few tiles, and of more
    tiles than CTAs; empty trajectories (the clear and nothing else), a single
    trajectory, and more trajectories than clusters in flight."""
    deep, _ = W.trajectory_batch(n_traj=3, n=n, dmin=4, dmax=9, seed=n, p=0.05)
    cases = [[deep[0]], [[], deep[1], [], deep[2], []]]
    for trajs in cases:
        b = q.qsa_batch_create(n, trajs, q.make_opts(planner=q.QSA_PLAN_DP, kmax=4, kmax_diag=4))
        states = torch.full((len(trajs) << n,), 7.0 + 1j, dtype=torch.complex64, device="cuda:0")
        try:
            q.qsa_batch_run(b, states.data_ptr(), states.numel() * 8, 100, 3, 0, 1)
            got = states.cpu().numpy().reshape(len(trajs), 1 << n).astype(np.complex128)
            for t, ops in enumerate(trajs):
                check_close(oracle.run_circuit(n, ops), got[t])
        finally:
            q.qsa_batch_destroy(b)


def test_graph_and_direct_paths_agree(q):
    n, n_traj, shots = 12, 20, 1000
    trajs, _ = W.trajectory_batch(n_traj=n_traj, n=n, dmin=3, dmax=12, seed=8, p=0.02)
    b = q.qsa_batch_create(n, trajs, q.make_opts(planner=q.QSA_PLAN_GREEDY, kmax=3, kmax_diag=3))
    s1 = torch.zeros(n_traj << n, dtype=torch.complex64, device="cuda:0")
    s2 = torch.zeros_like(s1)
    try:
        q.qsa_batch_run(b, s1.data_ptr(), s1.numel() * 8, shots, 9, 0, 0)
        r1 = q.qsa_batch_counts(b, n_traj, shots)
        q.qsa_batch_run(b, s2.data_ptr(), s2.numel() * 8, shots, 9, 0, 1)
        r2 = q.qsa_batch_counts(b, n_traj, shots)
        assert torch.equal(s1, s2)
        for a, c in zip(r1, r2):
            assert np.array_equal(a[0], c[0]) and np.array_equal(a[1], c[1])
    finally:
        q.qsa_batch_destroy(b)


def test_watchdog_budget_reports_timeout(q):
    """A cycle budget too small to finish makes every CTA stop between blocks
    and the call report QSA_E_TIMEOUT; the batch then runs normally again."""
    n, n_traj = 14, 8
    trajs, _ = W.trajectory_batch(n_traj=n_traj, n=n, dmin=20, dmax=30, seed=1)
    b = q.qsa_batch_create(n, trajs, q.make_opts(planner=q.QSA_PLAN_GREEDY, kmax=2, kmax_diag=2))
    states = torch.zeros(n_traj << n, dtype=torch.complex64, device="cuda:0")
    try:
        with pytest.raises(q.QsaError) as e:
            q.qsa_batch_run(b, states.data_ptr(), states.numel() * 8, 100, 1, 1000, 0)
        assert e.value.code == q.QSA_E_TIMEOUT
        q.qsa_batch_run(b, states.data_ptr(), states.numel() * 8, 100, 1, 0, 1)
        got = states.cpu().numpy().reshape(n_traj, 1 << n).astype(np.complex128)
        check_close(oracle.run_circuit(n, trajs[0]), got[0])
    finally:
        q.qsa_batch_destroy(b)


def test_batch_argument_errors(q):
    trajs, _ = W.trajectory_batch(n_traj=2, n=6, dmin=1, dmax=2, seed=0)
    with pytest.raises(q.QsaError):
        q.qsa_batch_create(6, trajs, q.make_opts(kmax=5, kmax_diag=5))
    with pytest.raises(q.QsaError):
        q.qsa_batch_create(23, trajs)
    b = q.qsa_batch_create(6, trajs, q.make_opts(kmax=4, kmax_diag=4))
    small = torch.zeros(64, dtype=torch.complex64, device="cuda:0")
    try:
        with pytest.raises(q.QsaError):
            q.qsa_batch_run(b, small.data_ptr(), small.numel() * 8, 10, 1)
        big = torch.zeros(2 << 6, dtype=torch.complex64, device="cuda:0")
        with pytest.raises(q.QsaError):
            q.qsa_batch_run(b, big.data_ptr(), big.numel() * 8, 20000, 1)
    finally:
        q.qsa_batch_destroy(b)


def test_full_size_batch_sampled_trajectories(q):
    """256 trajectories at N = 20, depths uniform in 10..60, p = 1e-3,
    10k shots each: the two shallowest trajectories are checked in full
    against the oracle; every trajectory's counts sum to the shot count."""
    n, n_traj, shots, seed = 20, 256, 10000, 0
    trajs, depths = W.trajectory_batch(n_traj=n_traj, n=n, dmin=10, dmax=60, seed=seed, p=1e-3)
    b = q.qsa_batch_create(n, trajs, q.make_opts(planner=q.QSA_PLAN_DP, kmax=4, kmax_diag=4))
    states = torch.zeros(n_traj << n, dtype=torch.complex64, device="cuda:0")
    try:
        st = q.qsa_batch_run(b, states.data_ptr(), states.numel() * 8, shots, seed, 0, 1)
        res = q.qsa_batch_counts(b, n_traj, shots)
        assert all(int(c.sum()) == shots for _, c in res)
        got = states.cpu().numpy().reshape(n_traj, 1 << n)
        for t in np.argsort(depths, kind="stable")[:2]:
            ref = oracle.run_circuit(n, trajs[t])
            check_close(ref, got[t].astype(np.complex128))
            _check_counts(res[t][0], res[t][1], ref, got[t].astype(np.complex128), n, shots, seed, int(t))
        assert st["seconds"] > 0
    finally:
        q.qsa_batch_destroy(b)
