"""The allocation-free sampler, qsa_sample_counts_noalloc, against qsa_sample_counts.

Callers that cannot let the library allocate device memory (a framework
allocator that owns the budget, or a pipeline that must not stall on
cudaFree) use this entry point; its scratch is one fixed device array.  The
test calls it through the C ABI twice in a row on the same state (the array
keeps the previous call's contents) and requires the same counts, bit for bit,
as the allocating entry point.  It also checks that oversize requests are
refused before any launch.  The file is named to be collected last.
"""
import ctypes

import numpy as np
import pytest

import workloads as W

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def q():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_2608_16940_gb300 as q
    return q


def _noalloc(q, buf, n, layout, shots, seed, stream):
    fn = q._lib.qsa_sample_counts_noalloc
    fn.argtypes = [ctypes.c_void_p, ctypes.c_int, ctypes.POINTER(ctypes.c_int32), ctypes.c_uint64, ctypes.c_uint64,
                   ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p]
    fn.restype = ctypes.c_int
    outc = torch.zeros(shots, dtype=torch.int64, device="cuda:0")
    cnts = torch.zeros(shots, dtype=torch.int64, device="cuda:0")
    nd = torch.zeros(1, dtype=torch.int64, device="cuda:0")
    lay = (ctypes.c_int32 * n)(*layout)
    rc = fn(buf.data_ptr(), n, lay, shots, seed, outc.data_ptr(), cnts.data_ptr(), nd.data_ptr(), stream)
    if rc != 0:
        raise q.QsaError(rc, q.qsa_last_error())
    torch.cuda.synchronize()
    k = int(nd.item())
    return outc[:k].cpu().numpy().astype(np.uint64), cnts[:k].cpu().numpy().astype(np.uint64)


@pytest.mark.parametrize("n,shots", [(14, 3000), (9, 500), (24, 5000)])
def test_noalloc_sampler_matches_allocating_sampler(q, n, shots):
    """N = 24 has 2^14 block totals (more than one 4096-entry scan segment,
    whose totals share the array with the sort keys) and 5000 shots (more than
    one launch of the bitonic sort): 16384 + 8192 + 5000 words of the array."""
    buf = torch.zeros(1 << n, dtype=torch.complex64, device="cuda:0")
    stream = torch.cuda.current_stream().cuda_stream
    s = q.qsa_state_create_ex(n, buf.data_ptr(), buf.numel() * 8, stream, 1)
    try:
        ops, _ = W.fusion_circuit(n=n, layers=2, seed=n, with_inverse=False)
        q.qsa_apply_circuit(s, ops, q.make_opts(planner=q.QSA_PLAN_DP, kmax=4, lowering=q.QSA_LOWER_PERMUTE))
        layout = q.qsa_get_layout(s)
        for seed in (11, 12):  # two calls in a row share the fixed scratch
            ref_v, ref_c = q.qsa_sample_counts(s, shots, seed)
            got_v, got_c = _noalloc(q, buf, n, layout, shots, seed, stream)
            assert np.array_equal(got_v, ref_v) and np.array_equal(got_c, ref_c)
            assert int(got_c.sum()) == shots
    finally:
        q.qsa_state_destroy(s)


def test_noalloc_sampler_rejects_oversize_requests(q):
    n = 30  # 2^20 block totals alone exceed the 2^19-word array
    buf = torch.zeros(16, dtype=torch.complex64, device="cuda:0")
    with pytest.raises(q.QsaError) as e:
        _noalloc(q, buf, n, list(range(n)), 10, 1, 0)
    assert e.value.code == q.QSA_E_RANGE and "scratch" in str(e.value)
