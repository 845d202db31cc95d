"""The binding's op marshalling (OpArray) writes the C records the ABI reads:
width, targets, a pointer to the row-major interleaved matrix and the diagonal
flag, for mixed widths, numpy or nested-list matrices and an empty list.  No
GPU: the records are read back through ctypes."""
import ctypes

import numpy as np
import pytest

import workloads as W


@pytest.fixture(scope="module")
def q():
    import __graft_entry__
    __graft_entry__._build_module().build()
    import paper_2608_16940_gb300 as q
    return q


class _Op:
    def __init__(self, targets, matrix, diag=False):
        self.targets, self.matrix, self.diag = tuple(targets), matrix, diag


def _read(rec):
    k = rec.k
    m = np.ctypeslib.as_array(rec.matrix, shape=(2 << (2 * k),)).view(np.complex128).reshape(1 << k, 1 << k)
    return k, list(rec.targets)[:k], m, rec.flags


def test_records_match_the_ops(q):
    rng = np.random.default_rng(3)
    ops = []
    for i in range(60):
        k = int(rng.integers(1, 7))
        t = [int(v) for v in rng.choice(20, size=k, replace=False)]
        if i % 3 == 0:
            ops.append(_Op(t, np.diag(np.exp(1j * rng.uniform(0, 6.3, 1 << k))), diag=True))
        elif i % 3 == 1:
            ops.append(_Op(t, W.haar_unitary(1 << k, rng)))
        else:   # nested lists, real entries
            ops.append(_Op(t, rng.normal(size=(1 << k, 1 << k)).tolist()))
    oa = q.OpArray(ops)
    assert oa.n == len(ops)
    for i, o in enumerate(ops):
        k, t, m, flags = _read(oa.arr[i])
        assert k == len(o.targets) and t == list(o.targets)
        assert np.array_equal(m, np.asarray(o.matrix, dtype=np.complex128))
        assert flags == (q.QSA_OP_DIAG if o.diag else 0)
    # the matrices live in one buffer owned by the array
    base = oa.mats.ctypes.data
    addrs = [ctypes.cast(oa.arr[i].matrix, ctypes.c_void_p).value for i in range(len(ops))]
    assert addrs[0] == base and all(b > a for a, b in zip(addrs, addrs[1:]))


def test_empty_list(q):
    oa = q.OpArray([])
    assert oa.n == 0 and len(oa.arr) == 1


def test_plan_from_records_equals_plan_from_ops(q):
    """The planner sees the same circuit through either path (op lists are
    marshalled on every call)."""
    ops, _ = W.qaoa_circuit(n=10, p=2, seed=1)
    opts = q.make_opts(planner=q.QSA_PLAN_DP, kmax=4, kmax_diag=4)
    p1 = q.qsa_plan_create(ops, 10, opts)
    p2 = q.qsa_plan_create(q.OpArray(ops), 10, opts)
    try:
        assert q.qsa_plan_blocks(p1) == q.qsa_plan_blocks(p2)
    finally:
        q.qsa_plan_destroy(p1)
        q.qsa_plan_destroy(p2)


def test_matrix_size_must_match_the_targets(q):
    """A matrix that is not 2^k x 2^k for its k targets is refused before any
    record is written (the records index one shared buffer by the widths)."""
    good = _Op([0, 1], np.eye(4))
    with pytest.raises(ValueError):
        q.OpArray([good, _Op([2], np.eye(4))])
    with pytest.raises(ValueError):
        q.OpArray([_Op([3, 4, 5], np.eye(4)), good])
    oa = q.OpArray([good, _Op([2], [[0, 1], [1, 0]])])
    assert oa.n == 2 and _read(oa.arr[1])[1] == [2]
