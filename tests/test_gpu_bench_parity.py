"""Element-wise FP64-oracle parity of two measured configurations at N = 24,
the largest size at which the single-threaded oracle runs whole circuits in
minutes.

- The bench's step exactly as the benchmark launches it: QAOA on a random
  3-regular graph with p = 8 rounds (24 H + 8 x (36 ZZ + 24 RX) = 504 gates),
  the interleaved initial layout set on |0...0> as a relabel, layer units, the
  zero-state prefix written by a write-only first pass over a buffer of
  arbitrary data, the DP planner scored by a cost model trained on the GPU on
  this state's own kernel timings, kmax 6, diagonal blocks up to 12 qubits,
  split-TF32 for k = 5/6 blocks; then the norm, <Z_a Z_b> on an edge and 1000
  shots from one read.  Amplitudes within 1e-5 (fidelity and largest
  difference), the measured sums against the oracle's, the shots bit for bit
  against the oracle's sampler on the GPU's amplitudes.
- The wide workload at the size its fidelity is stated for: 200 alternating
  Haar k = 5 / 6 operators on random target sets, once on the FP32 CUDA cores
  and once on the split-TF32 tensor-core path.

Both oracle runs start in a spawned process pool before the first GPU call,
so they overlap the GPU work.
"""
import concurrent.futures as cf
import multiprocessing as mp

import numpy as np
import pytest

import oracle
import workloads as W
from gpu_helpers import check_close

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

N = 24


def _qaoa_ref(n):
    import oracle as o
    import workloads as w
    ops, _ = w.qaoa_circuit(n=n, p=8, seed=0)
    return o.run_circuit(n, ops)


def _wide_ref(n):
    import oracle as o
    import workloads as w
    return o.run_circuit(n, w.wide_circuit(n, n_ops=200, widths=(5, 6), seed=0))


@pytest.fixture(scope="module")
def refs():
    oracle.build()
    pool = cf.ProcessPoolExecutor(max_workers=2, mp_context=mp.get_context("spawn"))
    futs = {"qaoa": pool.submit(_qaoa_ref, N), "wide": pool.submit(_wide_ref, N)}
    yield futs
    pool.shutdown(wait=True, cancel_futures=True)


@pytest.fixture(scope="module")
def q(refs):
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_2608_16940_gb300 as q
    return q


def _logical(q, h, buf):
    q.qsa_state_sync(h)
    return oracle.decode_state(buf.cpu().numpy().astype(np.complex128), q.qsa_get_layout(h))


def test_bench_step_qaoa24_p8_matches_oracle(q, refs, capsys):
    import bench
    ops, edges = W.qaoa_circuit(n=N, p=8, seed=0)
    assert len(ops) == 504
    buf = torch.zeros(1 << N, dtype=torch.complex64, device="cuda:0")
    h = q.qsa_state_create_ex(N, buf.data_ptr(), buf.numel() * 8, torch.cuda.current_stream().cuda_stream, 1)
    plan = None
    try:
        cm = bench.train_cost_model(q, h, q.QSA_PREC_TF32X3, 0, 240)
        layout = bench.interleaved_layout(N)
        opts = q.make_opts(planner=q.QSA_PLAN_DP_MLP, kmax=6, kmax_diag=12, precision=q.QSA_PREC_TF32X3, layer=1,
                           zero_init=1, timing=1)
        plan = q.qsa_plan_create(ops, N, opts, layout=layout)
        buf.copy_(torch.randn(1 << N, dtype=torch.complex64, device="cuda:0"))   # the first pass writes it all
        st = q.qsa_plan_execute_from_zero(h, plan)
        mask = (1 << edges[0][0]) | (1 << edges[0][1])
        (norm, zz), vals, cnts = q.qsa_measure(h, [0, mask], 1000, seed=17)
        assert q.qsa_get_layout(h) == layout
        got = _logical(q, h, buf)
    finally:
        if plan is not None:
            q.qsa_plan_destroy(plan)
        q.qsa_costmodel_set(None)
        q.qsa_state_destroy(h)
    assert st["layer_blocks"] == st["blocks"] and st["passes"] == st["layer_blocks"]
    ref = refs["qaoa"].result()
    infid, err = check_close(ref, got)
    norm_np = float(np.vdot(got, got).real)
    assert abs(norm - norm_np) < 1e-9
    assert abs(zz - oracle.expect_z(ref, mask)) < 1e-5
    rv, rc = oracle.sample_counts(got, layout, 1000, 17)
    assert np.array_equal(vals, rv) and np.array_equal(cnts, rc)
    with capsys.disabled():
        print(f"\nbench step qaoa N={N} p=8 ({len(ops)} gates, {st['passes']} passes, cost model held-out "
              f"error {cm['heldout_median_rel_err']:.3f}): 1-F = {infid:.3e}, max|d| = {err:.3e}, "
              f"1-|psi|^2 = {1 - norm:.3e}, <ZZ> = {zz:.6f} (oracle {oracle.expect_z(ref, mask):.6f})")


@pytest.mark.parametrize("prec", [0, 1], ids=["fp32", "3xtf32"])
def test_wide24_200_ops_fidelity_vs_oracle(q, refs, prec, capsys):
    ops = W.wide_circuit(N, n_ops=200, widths=(5, 6), seed=0)
    buf = torch.zeros(1 << N, dtype=torch.complex64, device="cuda:0")
    h = q.qsa_state_create_ex(N, buf.data_ptr(), buf.numel() * 8, torch.cuda.current_stream().cuda_stream, 1)
    try:
        st = q.qsa_apply_circuit(h, ops, q.make_opts(planner=q.QSA_PLAN_PER_GATE, kmax=6, kmax_diag=6,
                                                     precision=prec))
        got = _logical(q, h, buf)
    finally:
        q.qsa_state_destroy(h)
    assert st["tc_blocks"] == (200 if prec else 0)
    infid, err = check_close(refs["wide"].result(), got)
    with capsys.disabled():
        print(f"\nwide 200 ops N={N} precision={'3xTF32' if prec else 'FP32'}: 1-F = {infid:.3e}, "
              f"max|d| = {err:.3e}, 1-|psi|^2 = {1 - float(np.vdot(got, got).real):.3e}")
