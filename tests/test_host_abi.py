"""Host-only checks of libqsa (no GPU): the library loads and exports every
entry point declared in include/*.h; the host planner and block product agree
with the oracle; argument validation rejects bad input before any launch."""
import glob
import os
import re

import numpy as np
import pytest

import oracle
import workloads as W

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def q():
    import __graft_entry__
    __graft_entry__._build_module().build()
    import paper_2608_16940_gb300 as q
    return q


def _declared():
    names = set()
    for h in glob.glob(os.path.join(ROOT, "include", "*.h")):
        src = open(h).read()
        src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
        for m in re.finditer(r"\b(qsa_[a-z0-9_]+)\s*\(", src):
            names.add(m.group(1))
    return names


def test_every_declared_symbol_is_exported(q):
    import ctypes
    lib = ctypes.CDLL(q.LIB_PATH)
    declared = _declared()
    assert len(declared) >= 20
    missing = [n for n in sorted(declared) if not hasattr(lib, n)]
    assert not missing, missing


def _random_circuit(rng, n, n_ops, kmax_in=2, diag_frac=0.3):
    ops = []
    for _ in range(n_ops):
        k = int(rng.integers(1, kmax_in + 1))
        t = tuple(int(v) for v in rng.choice(n, size=k, replace=False))
        d = bool(rng.random() < diag_frac)
        ops.append(W.Op(t, np.eye(1 << k, dtype=np.complex128), d))
    return ops


@pytest.mark.parametrize("seed,n,n_ops,kmax,kdiag,window,rounds",
                         [(0, 6, 40, 3, 3, 64, 4), (1, 10, 300, 4, 4, 64, 4), (2, 8, 200, 4, 2, 16, 4),
                          (3, 12, 500, 5, 5, 64, 1), (4, 5, 130, 2, 2, 7, 3), (5, 14, 700, 6, 6, 64, 4)])
def test_dp_planner_matches_oracle_pipeline(q, seed, n, n_ops, kmax, kdiag, window, rounds):
    rng = np.random.default_rng(seed)
    ops = _random_circuit(rng, n, n_ops, kmax_in=min(3, kmax))
    got = q.qsa_plan_circuit(ops, n, q.make_opts(planner=q.QSA_PLAN_DP, kmax=kmax, kmax_diag=kdiag,
                                                  window=window, rounds=rounds))
    ref = oracle.fuse_pipeline(ops, kmax, kdiag, window, rounds)
    assert got == ref


@pytest.mark.parametrize("seed,n,n_ops,kmax,kdiag", [(10, 12, 300, 2, 8), (11, 14, 400, 4, 12), (12, 10, 250, 3, 6),
                                                    (13, 16, 500, 6, 10)])
def test_dp_planner_with_wide_diagonal_cap_matches_oracle(q, seed, n, n_ops, kmax, kdiag):
    """Diagonal blocks wider than the dense cap (kmax_diag > kmax): the DP and
    merge pipeline agree with the oracle's."""
    rng = np.random.default_rng(seed)
    ops = _random_circuit(rng, n, n_ops, kmax_in=min(3, kmax), diag_frac=0.6)
    for o in ops:
        if o.diag:
            o.matrix = np.diag(np.exp(1j * rng.uniform(0, 6.3, size=1 << len(o.targets))))
    got = q.qsa_plan_circuit(ops, n, q.make_opts(planner=q.QSA_PLAN_DP, kmax=kmax, kmax_diag=kdiag))
    ref = oracle.fuse_pipeline(ops, kmax, kdiag, 64, 4)
    assert got == ref


@pytest.mark.parametrize("seed,n,kmax,kdiag,kprod", [(20, 14, 4, 4, 6), (21, 20, 6, 12, 11), (22, 10, 3, 8, 2),
                                                      (23, 16, 2, 2, 11)])
def test_dp_planner_with_product_units_matches_oracle(q, seed, n, kmax, kdiag, kprod):
    """Runs of one-qubit ops become product units: the DP pipeline over them
    agrees with the oracle's (fuse_pipeline_products)."""
    rng = np.random.default_rng(seed)
    ops = []
    for _ in range(500):
        r = rng.random()
        if r < 0.55:
            ops.append(W.Op((int(rng.integers(0, n)),), W.haar_unitary(2, rng), False))
        elif r < 0.8:
            t = tuple(int(v) for v in rng.choice(n, size=2, replace=False))
            ops.append(W.Op(t, W.zz(float(rng.uniform(0, 6))), True))
        else:
            t = tuple(int(v) for v in rng.choice(n, size=int(rng.integers(2, 4)), replace=False))
            ops.append(W.Op(t, np.eye(1 << len(t), dtype=np.complex128), False))
    for planner in (q.QSA_PLAN_DP,):
        got = q.qsa_plan_circuit(ops, n, q.make_opts(planner=planner, kmax=kmax, kmax_diag=kdiag, kmax_prod=kprod))
        assert got == oracle.fuse_pipeline_products(ops, kmax, kdiag, kprod)
    with pytest.raises(q.QsaError):
        q.qsa_plan_circuit(ops, n, q.make_opts(kmax_prod=12))


def test_diagonal_options_and_flags_are_validated(q):
    ops = [W.Op((0, 1), W.CZ.copy(), True)]
    with pytest.raises(q.QsaError):
        q.qsa_plan_circuit(ops, 4, q.make_opts(kmax=4, kmax_diag=13))
    assert q.qsa_plan_circuit(ops, 4, q.make_opts(kmax=2, kmax_diag=12)) == [0]
    bad = [W.Op((0, 1), W.CNOT.copy(), True)]   # flagged diagonal but not diagonal
    with pytest.raises(q.QsaError):
        q.qsa_plan_circuit(bad, 4, q.make_opts())


def _dense_tuples(q, plan, ops):
    """The plan's dense blocks as target tuples in the order the library
    promotes them: a single op keeps its own order, a fused block its
    ascending union; all-diagonal blocks need no promotion."""
    first, _ = q.qsa_plan_blocks(plan)
    bounds = first + [len(ops)]
    out = []
    for a, b in zip(bounds[:-1], bounds[1:]):
        blk = ops[a:b]
        if all(o.diag for o in blk):
            continue
        out.append(list(blk[0].targets) if len(blk) == 1 else sorted({t for o in blk for t in o.targets}))
    return out


@pytest.mark.parametrize("seed,n,kmax,kdiag", [(0, 14, 3, 3), (1, 16, 4, 10), (2, 20, 6, 6), (3, 12, 2, 12)])
def test_promotion_replay_matches_oracle(q, seed, n, kmax, kdiag):
    """qsa_plan_promotions (host) equals the oracle's replay of the demand
    model for both victim rules, from a random initial layout."""
    rng = np.random.default_rng(seed)
    ops = _random_circuit(rng, n, 400, kmax_in=min(3, kmax), diag_frac=0.3)
    plan = q.qsa_plan_create(ops, n, q.make_opts(planner=q.QSA_PLAN_DP, kmax=kmax, kmax_diag=kdiag))
    try:
        tuples = _dense_tuples(q, plan, ops)
        lay = [int(v) for v in rng.permutation(n)]
        for rule, name in ((q.QSA_VICTIM_FIRST_FREE, "first_free"), (q.QSA_VICTIM_FARTHEST, "farthest")):
            pr, ps, out = q.qsa_plan_promotions(plan, n, rule, lay)
            counts, ref = oracle.promotion_replay(tuples, n, min(11, n), name, lay)
            assert pr == sum(counts) and ps == sum(c > 0 for c in counts) and out == ref, name
        with pytest.raises(q.QsaError):
            q.qsa_plan_promotions(plan, n, 2)
    finally:
        q.qsa_plan_destroy(plan)


@pytest.mark.parametrize("kmax", [1, 2, 3, 4, 6])
def test_greedy_and_per_gate_planners_match_oracle(q, kmax):
    rng = np.random.default_rng(kmax)
    ops = _random_circuit(rng, 9, 250)
    got = q.qsa_plan_circuit(ops, 9, q.make_opts(planner=q.QSA_PLAN_GREEDY, kmax=kmax, kmax_diag=kmax))
    ref = [s for s, _ in oracle.greedy_partition(ops, kmax)]
    assert got == ref
    got = q.qsa_plan_circuit(ops, 9, q.make_opts(planner=q.QSA_PLAN_PER_GATE))
    assert got == list(range(len(ops)))


def test_dp_mlp_without_model_falls_back_to_greedy(q):
    q.qsa_costmodel_set(None)
    rng = np.random.default_rng(3)
    ops = _random_circuit(rng, 8, 120)
    got = q.qsa_plan_circuit(ops, 8, q.make_opts(planner=q.QSA_PLAN_DP_MLP, kmax=4))
    ref = [s for s, _ in oracle.greedy_partition(ops, 4)]
    assert got == ref


@pytest.mark.parametrize("seed", range(4))
def test_fuse_ops_matches_oracle_block_product(q, seed):
    rng = np.random.default_rng(seed)
    pool = [int(v) for v in rng.choice(20, size=5, replace=False)]
    gates = []
    for _ in range(7):
        k = int(rng.integers(1, 4))
        t = tuple(int(v) for v in rng.choice(pool, size=k, replace=False))
        gates.append(W.Op(t, W.haar_unitary(1 << k, rng)))
    tg, M = q.qsa_fuse_ops(gates)
    assert tg == sorted({x for g in gates for x in g.targets})
    ref = oracle.block_product(gates, tg)
    assert np.max(np.abs(M - ref)) < 1e-13


def test_fuse_ops_rejects_blocks_wider_than_six(q):
    gates = [W.Op((i, i + 1), np.eye(4, dtype=np.complex128)) for i in range(0, 8, 2)]
    with pytest.raises(q.QsaError) as e:
        q.qsa_fuse_ops(gates)
    assert e.value.code == q.QSA_E_ARG


def test_plan_rejects_bad_ops(q):
    bad = [W.Op((0, 0), np.eye(4, dtype=np.complex128))]
    with pytest.raises(q.QsaError):
        q.qsa_plan_circuit(bad, 4)
    bad = [W.Op((5,), np.eye(2, dtype=np.complex128))]
    with pytest.raises(q.QsaError):
        q.qsa_plan_circuit(bad, 4)
    with pytest.raises(q.QsaError):
        q.qsa_plan_circuit([W.Op((0,), np.eye(2))], 4, q.make_opts(kmax=7))


def test_state_create_argument_errors(q):
    with pytest.raises(q.QsaError) as e:
        q.qsa_state_create(0)
    assert e.value.code == q.QSA_E_ARG
    with pytest.raises(q.QsaError) as e:
        q.qsa_state_create(35)
    assert e.value.code == q.QSA_E_ARG
    with pytest.raises(q.QsaError) as e:
        q.qsa_state_create(4, q.QSA_C128)
    assert e.value.code == q.QSA_E_UNSUPPORTED


def test_costmodel_features_layout(q):
    x = q.qsa_costmodel_features(3, (1 << 0) | (1 << 17) | (1 << 33), 30, 4)
    assert x.shape == (37,)
    assert abs(x[0] - 0.5) < 1e-7 and x[1] == 1 and x[18] == 1 and x[34] == 1 and x[2] == 0
    assert abs(x[35] - 30 / 34) < 1e-7 and abs(x[36] - 2 / 8) < 1e-7
