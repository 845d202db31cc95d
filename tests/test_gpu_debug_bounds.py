"""The bounds-checked build (libqsa_debug.so) on the GPU: the paths whose
state accesses it checks (FP32 fused updates in every stage form, the
permutation lowering, the product and layer kernels through a QAOA plan, the
split-TF32 kernel, batched trajectories) run against the FP64 oracle in a
subprocess that loads that build, and no check may fail."""
import json
import os
import subprocess
import sys

import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))

SCRIPT = r"""
import json, numpy as np, torch
import paper_2608_16940_gb300 as q, oracle, workloads as W
assert q.qsa_debug_bounds_enabled()
out = {"worst": 0.0}
def check(ref, got):
    out["worst"] = max(out["worst"], float(np.max(np.abs(ref - got))))
rng = np.random.default_rng(7)
for n, sets in ((12, [(11,), (10, 11), (2, 3), (0, 1), (1, 2, 3), (3, 0, 2, 1), (8, 9, 10, 11), (1, 3, 5, 7)]),
                (14, [(0, 5, 13), (13, 2), (6, 7, 8, 9, 10), (0, 1, 2, 3, 4, 5), (12, 3, 7, 1, 9, 0)])):
    psi = W.random_state(n, 3)
    buf = torch.from_numpy(psi.astype(np.complex64)).cuda()
    h = q.qsa_state_create_ex(n, buf.data_ptr(), buf.numel() * 8, torch.cuda.current_stream().cuda_stream, 0)
    ref = psi.astype(np.complex64).astype(np.complex128)
    for t in sets:
        for prec, low in ((q.QSA_PREC_FP32, q.QSA_LOWER_STRIDED), (q.QSA_PREC_TF32X3, q.QSA_LOWER_STRIDED),
                          (q.QSA_PREC_FP32, q.QSA_LOWER_PERMUTE)):
            G = W.haar_unitary(1 << len(t), rng)
            q.qsa_apply_fused_ex(h, t, G, low, prec)
            oracle.apply(ref, t, G)
    torch.cuda.synchronize()
    got = oracle.decode_state(buf.cpu().numpy().astype(np.complex128), q.qsa_get_layout(h))
    check(ref, got)
    q.qsa_state_destroy(h)
# a QAOA plan: layer units, zero-state prefix, product and diagonal blocks
ops, _ = W.qaoa_circuit(n=14, p=3, seed=2)
buf = torch.zeros(1 << 14, dtype=torch.complex64, device="cuda:0")
h = q.qsa_state_create_ex(14, buf.data_ptr(), buf.numel() * 8, torch.cuda.current_stream().cuda_stream, 1)
for layer, kprod in ((1, 0), (0, 4)):
    q.qsa_state_reset(h)
    q.qsa_apply_circuit(h, ops, q.make_opts(planner=q.QSA_PLAN_DP, kmax=6, kmax_diag=12, layer=layer,
                                            zero_init=layer, kmax_prod=kprod, precision=q.QSA_PREC_TF32X3))
    torch.cuda.synchronize()
    got = oracle.decode_state(buf.cpu().numpy().astype(np.complex128), q.qsa_get_layout(h))
    check(oracle.run_circuit(14, ops), got)
q.qsa_state_destroy(h)
# batched trajectories on clusters
trajs, _ = W.trajectory_batch(n_traj=6, n=12, dmin=3, dmax=8, seed=4, p=0.05)
b = q.qsa_batch_create(12, trajs, q.make_opts(planner=q.QSA_PLAN_DP, kmax=4, kmax_diag=4))
states = torch.zeros(6 << 12, dtype=torch.complex64, device="cuda:0")
q.qsa_batch_run(b, states.data_ptr(), states.numel() * 8, 100, 1, 0, 0)
got = states.cpu().numpy().reshape(6, 1 << 12).astype(np.complex128)
for t in range(6):
    check(oracle.run_circuit(12, trajs[t]), got[t])
q.qsa_batch_destroy(b)
torch.cuda.synchronize()
out["bounds"] = list(q.qsa_debug_bounds_status())
print(json.dumps(out))
"""


def test_debug_build_paths_stay_in_bounds():
    import __graft_entry__
    __graft_entry__._build_module().build(debug_bounds=True)
    env = dict(os.environ, QSA_LIB_VARIANT="debug")
    r = subprocess.run([sys.executable, "-c", SCRIPT], cwd=ROOT, env=env, capture_output=True, text=True, timeout=900)
    assert r.returncode == 0, r.stderr[-3000:]
    res = json.loads(r.stdout.strip().splitlines()[-1])
    print(res)
    assert res["bounds"] == [0, 0], res
    assert res["worst"] < 1e-5, res
