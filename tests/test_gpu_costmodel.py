"""Cost-model kernels against the FP64 oracle, and what the trained model
gains the fusion planner.

Tolerances: FP32 kernels vs the FP64 restatement, relative 1e-4 (forward),
gradients within 1e-4 of max |g|, Adam parameters within 1e-6.
"""
import time

import numpy as np
import pytest

import oracle
import workloads as W
from gpu_helpers import GState

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def q():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_2608_16940_gb300 as q
    return q


def _split(p):
    out, o = [], 0
    for shp in oracle.MLP_SHAPES:
        c = int(np.prod(shp))
        out.append(p[o:o + c].reshape(shp).astype(np.float64))
        o += c
    return out


def _flat(ps):
    return np.concatenate([np.asarray(x).reshape(-1) for x in ps])


def _dev(a):
    return torch.from_numpy(np.ascontiguousarray(a, dtype=np.float32)).cuda()


def test_mlp_forward_matches_oracle(q):
    rng = np.random.default_rng(0)
    P = q.qsa_costmodel_init(3)
    P[6400:6656] += 0.05 * rng.standard_normal(256).astype(np.float32)   # non-zero biases too
    X = rng.random((300, 37)).astype(np.float32)
    dP, dX = _dev(P), _dev(X)
    y = torch.zeros(300, device="cuda")
    ws = torch.zeros(q.qsa_mlp_workspace_bytes(300) // 4, device="cuda")
    q.qsa_mlp_forward(dP.data_ptr(), dX.data_ptr(), 300, y.data_ptr(), ws.data_ptr())
    torch.cuda.synchronize()
    ref, _ = oracle.mlp_forward(_split(P.astype(np.float64)), X.astype(np.float64))
    got = y.cpu().numpy().astype(np.float64)
    assert np.max(np.abs(got - ref)) <= 1e-4 * max(1.0, np.max(np.abs(ref)))


def test_mlp_gradients_match_oracle_backprop(q):
    rng = np.random.default_rng(1)
    P = q.qsa_costmodel_init(4)
    n = 257
    X = rng.random((n, 37)).astype(np.float32)
    t = rng.standard_normal(n).astype(np.float32)
    dP, dX, dt = _dev(P), _dev(X), _dev(t)
    G = torch.zeros(q.MLP_PARAMS, device="cuda")
    L = torch.zeros(1, device="cuda")
    ws = torch.zeros(q.qsa_mlp_workspace_bytes(n) // 4, device="cuda")
    q.qsa_mlp_loss_grad(dP.data_ptr(), dX.data_ptr(), dt.data_ptr(), n, G.data_ptr(), L.data_ptr(), ws.data_ptr())
    torch.cuda.synchronize()
    Lr, gr = oracle.mlp_loss_grad(_split(P.astype(np.float64)), X.astype(np.float64), t.astype(np.float64))
    g = G.cpu().numpy().astype(np.float64)
    ref = _flat(gr)
    assert abs(float(L.item()) - Lr) <= 1e-5 * max(1.0, Lr)
    assert np.max(np.abs(g - ref)) <= 1e-4 * np.max(np.abs(ref))


def test_adam_step_matches_oracle(q):
    rng = np.random.default_rng(2)
    P = q.qsa_costmodel_init(5)
    G = rng.standard_normal(q.MLP_PARAMS).astype(np.float32)
    M = (0.1 * rng.standard_normal(q.MLP_PARAMS)).astype(np.float32)
    V = np.abs(0.01 * rng.standard_normal(q.MLP_PARAMS)).astype(np.float32)
    dP, dG, dM, dV = _dev(P), _dev(G), _dev(M), _dev(V)
    q.qsa_mlp_adam_step(dP.data_ptr(), dG.data_ptr(), dM.data_ptr(), dV.data_ptr(), q.MLP_PARAMS, 3, 1e-3)
    torch.cuda.synchronize()
    newp, newm, newv = oracle.adam_step([P.astype(np.float64)], [G.astype(np.float64)], [M.astype(np.float64)],
                                        [V.astype(np.float64)], 3, lr=1e-3)
    assert np.max(np.abs(dP.cpu().numpy() - newp[0])) < 1e-6
    assert np.max(np.abs(dM.cpu().numpy() - newm[0])) < 1e-6


def test_training_decreases_loss(q):
    rng = np.random.default_rng(3)
    X = rng.random((512, 37)).astype(np.float32)
    w = rng.standard_normal(37)
    y = (np.tanh(X @ w) + 0.1 * X[:, 0]).astype(np.float32)
    _, losses = q.qsa_costmodel_train(X, y, epochs=40, batch=64, lr=3e-3, seed=7)
    assert losses[-1] < 0.2 * losses[0]


def _time_plan(q, st, plan, reps=3):
    ts = []
    for _ in range(reps):
        q.qsa_state_reset(st.h)
        q.qsa_state_sync(st.h)
        t0 = time.perf_counter()
        q.qsa_plan_execute(st.h, plan)
        q.qsa_state_sync(st.h)
        ts.append(time.perf_counter() - t0)
    return float(np.median(ts))


def test_learned_planner_gain_over_heuristics(q, capsys):
    """Collect timings from the library's own kernels at N = 26, train the
    model on the GPU, then plan the QAOA workload (3-regular graph, p = 8) with
    the width-limit greedy heuristic, the 4^k DP and the model-scored DP; the
    measured time of each plan is what the model is scored against.  FP32 with
    kmax 6 is a setting where both heuristics mispredict: a 5- or 6-qubit
    block on the CUDA cores costs several memory passes (greedy takes them
    whenever they fit), and 4^k overprices the 2- to 4-qubit blocks that all
    cost about one pass; the learned DP must beat both by 5 %."""
    n = 26
    st = GState(q, torch, n)
    try:
        X, y = q.qsa_costmodel_collect(st.h, 600, reps=3, precision=q.QSA_PREC_FP32, seed=11)
        perm = np.random.default_rng(0).permutation(len(y))
        tr, te = perm[:500], perm[500:]
        params, losses = q.qsa_costmodel_train(X[tr], y[tr], epochs=200, batch=32, lr=2e-3, seed=1,
                                               weight_decay=1e-2)
        assert losses[-1] < losses[0]
        q.qsa_costmodel_set(params)
        pred = q.qsa_costmodel_predict(X[te])
        rel = np.abs(pred - np.exp(y[te])) / np.exp(y[te])
        ops, _ = W.qaoa_circuit(n=n, p=8, seed=0)
        times, blocks = {}, {}
        for name, planner in [("greedy", q.QSA_PLAN_GREEDY), ("dp_4k", q.QSA_PLAN_DP), ("dp_mlp", q.QSA_PLAN_DP_MLP)]:
            plan = q.qsa_plan_create(ops, n, q.make_opts(planner=planner, kmax=6, kmax_diag=6))
            blocks[name] = q.qsa_plan_info(plan)["blocks"]
            _time_plan(q, st, plan, reps=1)
            times[name] = _time_plan(q, st, plan)
            q.qsa_plan_destroy(plan)
        with capsys.disabled():
            print(f"\ncost model: held-out median |t_hat - t| / t = {np.median(rel):.3f}; "
                  f"blocks {blocks}; seconds {times}; "
                  f"gain vs greedy {times['greedy'] / times['dp_mlp']:.2f}x, vs 4^k DP "
                  f"{times['dp_4k'] / times['dp_mlp']:.2f}x")
        assert np.median(rel) < 0.10
        assert times["dp_mlp"] <= 0.95 * min(times["greedy"], times["dp_4k"])
    finally:
        q.qsa_costmodel_set(None)
        st.close()


@pytest.mark.parametrize("precision", ["tf32x3", "fp32"])
def test_learned_planner_on_the_fusion_workload(q, capsys, precision):
    """The fusion workload at N = 28 (QFT of a seeded basis state, 40 layers of
    Haar U(2) on every qubit and U(4) on random matchings, then the inverse;
    4.2k gates), kmax 6, diagonal blocks up to 12 qubits: the width-limit
    heuristic, the 4^k DP and the DP scored by a cost model trained on this
    state's own kernel timings (1000 samples), each plan timed with CUDA
    events.  Every plan returns the state to |0...0>.  With split-TF32 for
    k = 5, 6 every width costs about one pass, so the learned DP can at best
    match the greedy plan (within 5 %); in FP32 the wide blocks cost several
    passes and the learned DP must beat greedy by 10 % and the 4^k DP by 5 %."""
    import bench
    buf = torch.empty(1 << 28, dtype=torch.complex64, device="cuda:0")
    try:
        rec = bench.planner_record(q, torch, buf, torch.cuda.current_stream().cuda_stream, 0, precision=precision)
    finally:
        del buf
        torch.cuda.empty_cache()
    with capsys.disabled():
        print(f"\nfusion28 {precision} planners: greedy {rec['greedy']['seconds']:.4f} s "
              f"({rec['greedy']['blocks']} blocks), dp_4k {rec['dp_4k']['seconds']:.4f} s ({rec['dp_4k']['blocks']}), "
              f"dp_mlp {rec['dp_mlp']['seconds']:.4f} s ({rec['dp_mlp']['blocks']}); gain vs greedy "
              f"{rec['gain_vs_greedy']:.2f}x, vs 4^k DP {rec['gain_vs_dp_4k']:.2f}x; held-out median error "
              f"{rec['cost_model']['heldout_median_rel_err']:.3f}")
    for name in ("greedy", "dp_4k", "dp_mlp"):
        assert rec[name]["return_probability"] > 1 - 1e-4, (name, rec[name]["return_probability"])
    assert rec["cost_model"]["heldout_median_rel_err"] < 0.10
    if precision == "fp32":
        assert rec["gain_vs_greedy"] >= 1.10 and rec["gain_vs_dp_4k"] >= 1.05
    else:
        assert rec["gain_vs_greedy"] >= 0.95
