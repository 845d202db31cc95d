"""The exchange plan of a sharded state (§IV-D, Alg. lazy-mpi), no GPU.

qsa_plan_exchanges lists, for a plan run on 2^r ranks, the rank-bit / local-
bit swaps that make each block's targets local, each one pairwise exchange of
half a slab between XOR partners.  Checked here:

- a hand-worked case (first-free victims; the layout the swaps leave);
- on random circuits: after a block's exchanges its targets are local, every
  exchange pairs a rank position with a local position that holds no target
  of the block, diagonal blocks need none, and the final layout is the
  replay of the swaps;
- end to end with two gloo ranks on CPU: each rank holds half of an N = 8
  state, swaps halves with its partner for every listed exchange, applies
  each block on its local positions (diagonal blocks with its own rank bit
  fixed), and the gathered state decoded through the final layout equals the
  oracle's single-node result.  The per-rank updates use the oracle's
  routines (this checks the plan and the exchange rule, not a device path).
"""
import os
import socket

import numpy as np
import pytest

import oracle
import workloads as W

torch = pytest.importorskip("torch")
import torch.distributed as dist  # noqa: E402
import torch.multiprocessing as mp  # noqa: E402


@pytest.fixture(scope="module")
def q():
    import __graft_entry__
    __graft_entry__._build_module().build()
    import paper_2608_16940_gb300 as q
    return q


def _random_ops(rng, n, n_ops, kin=3, diag_frac=0.3):
    ops = []
    for _ in range(n_ops):
        k = int(rng.integers(1, kin + 1))
        t = tuple(int(v) for v in rng.choice(n, size=k, replace=False))
        if rng.random() < diag_frac:
            ops.append(W.Op(t, np.diag(np.exp(1j * rng.uniform(0, 2 * np.pi, 1 << k))), True))
        else:
            ops.append(W.Op(t, W.haar_unitary(1 << k, rng), False))
    return ops


def test_hand_worked_exchanges(q):
    """N = 4 on 2 ranks (position 3 is the rank bit), identity layout, first-
    free victims: the gate on qubit 3 swaps position 3 with local position 0
    (qubit 0 moves to the rank bit); the gate on qubit 0 then swaps position 3
    with the first local position holding none of its targets, position 0
    again, which restores the identity layout; the diagonal gate needs no
    exchange."""
    ops = [W.Op((3,), W.H, False), W.Op((0,), W.H, False), W.Op((1, 2), W.CZ, True)]
    plan = q.qsa_plan_create(ops, 4, q.make_opts(planner=q.QSA_PLAN_PER_GATE))
    try:
        ex, lay = q.qsa_plan_exchanges(plan, 4, 1)
    finally:
        q.qsa_plan_destroy(plan)
    assert ex == [(0, 3, 0), (1, 3, 0)]
    assert lay == [0, 1, 2, 3]


@pytest.mark.parametrize("seed,n,r,victim", [(0, 8, 1, 0), (1, 10, 2, 1), (2, 12, 3, 0), (3, 9, 1, 1)])
def test_exchange_invariants(q, seed, n, r, victim):
    rng = np.random.default_rng(seed)
    ops = _random_ops(rng, n, 120)
    plan = q.qsa_plan_create(ops, n, q.make_opts(planner=q.QSA_PLAN_DP, kmax=3, kmax_diag=3))
    try:
        first, widths = q.qsa_plan_blocks(plan)
        kinds, _ = q.qsa_plan_block_kinds(plan)
        start = [int(v) for v in rng.permutation(n)]
        ex, lay = q.qsa_plan_exchanges(plan, n, r, layout=start, victim=victim)
    finally:
        q.qsa_plan_destroy(plan)
    local = n - r
    L = list(start)
    bounds = first + [len(ops)]
    e = 0
    for b in range(len(first)):
        targets = sorted({t for o in ops[bounds[b]:bounds[b + 1]] for t in o.targets})
        while e < len(ex) and ex[e][0] == b:
            _, pr, pl = ex[e]
            assert pr >= local and pl < local
            assert pl not in [L[t] for t in targets]
            qa, qb = L.index(pr), L.index(pl)
            L[qa], L[qb] = pl, pr
            e += 1
        if kinds[b] == 1:   # diagonal
            assert not any(x[0] == b for x in ex)
        else:
            assert all(L[t] < local for t in targets)
    assert e == len(ex) and L == lay


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _sharded_rank(rank, ws, port, out):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank), WORLD_SIZE=str(ws))
    dist.init_process_group("gloo", rank=rank, world_size=ws)
    import paper_2608_16940_gb300 as q
    n, r = 8, 1
    local = n - r
    ops = _random_ops(np.random.default_rng(42), n, 60)
    plan = q.qsa_plan_create(ops, n, q.make_opts(planner=q.QSA_PLAN_DP, kmax=3, kmax_diag=3))
    try:
        first, _ = q.qsa_plan_blocks(plan)
        kinds, _ = q.qsa_plan_block_kinds(plan)
        ex, final = q.qsa_plan_exchanges(plan, n, r, victim=1)
    finally:
        q.qsa_plan_destroy(plan)
    slab = np.zeros(1 << local, dtype=np.complex128)
    if rank == 0:
        slab[0] = 1.0
    L = list(range(n))
    bounds = first + [len(ops)]
    idx = np.arange(1 << local)
    e = 0
    for b in range(len(first)):
        while e < len(ex) and ex[e][0] == b:
            _, pr, pl = ex[e]
            j = pr - local
            partner = rank ^ (1 << j)
            mine = (rank >> j) & 1
            sel = ((idx >> pl) & 1) != mine        # the half whose bit pl differs from my rank bit j
            send = torch.from_numpy(np.ascontiguousarray(slab[sel]).view(np.float64))   # gloo: real pairs
            recv = torch.empty_like(send)
            reqs = [dist.isend(send, partner), dist.irecv(recv, partner)]
            for rq in reqs:
                rq.wait()
            slab[sel] = recv.numpy().view(np.complex128)
            qa, qb = L.index(pr), L.index(pl)
            L[qa], L[qb] = pl, pr
            e += 1
        blk = ops[bounds[b]:bounds[b + 1]]
        targets = sorted({t for o in blk for t in o.targets})
        M = oracle.block_product(blk, targets)
        phys = [L[t] for t in targets]
        if kinds[b] == 1:
            # diagonal: entry index from the physical bits, rank bits fixed by this rank
            d = np.diag(M)
            y = (rank << local) | idx
            c = np.zeros_like(idx)
            for jj, p in enumerate(phys):
                c |= ((y >> p) & 1) << jj
            slab *= d[c]
        else:
            assert all(p < local for p in phys)
            oracle.apply(slab, phys, M)
    gathered = [torch.empty(2 << local, dtype=torch.float64) for _ in range(ws)] if rank == 0 else None
    dist.gather(torch.from_numpy(slab.view(np.float64)), gathered, dst=0)
    if rank == 0:
        stored = np.concatenate([g.numpy().view(np.complex128) for g in gathered])
        got = oracle.decode_state(stored, L)
        ref = oracle.run_circuit(n, ops)
        out["err"] = float(np.max(np.abs(got - ref)))
        out["layout_match"] = L == final
        out["exchanges"] = len(ex)
    dist.destroy_process_group()


def test_two_gloo_ranks_run_a_sharded_state():
    ws = 2
    port = _free_port()
    with mp.Manager() as m:
        out = m.dict()
        mp.start_processes(_sharded_rank, args=(ws, port, out), nprocs=ws, start_method="spawn")
        res = dict(out)
    assert res["layout_match"] and res["exchanges"] > 0
    assert res["err"] < 1e-12, res
