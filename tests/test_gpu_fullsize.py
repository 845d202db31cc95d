"""Full-size runs in the bench's launch configuration, checked where the FP64
oracle cannot run the whole circuit: closed forms at sampled indices and
invariants that hold at any size.

- N = 28 fusion workload: the QFT of a random basis state matches its closed
  form at sampled indices, and the whole circuit followed by its inverse
  returns to |0...0>;
- N = 30 QAOA workload (kmax 4 FP32, kmax 6 with split-TF32 for k = 5, 6,
  product units, and the bench's layer units): norm 1, global bit-flip symmetry of the state
  (p(x) = p(~x), <Z_q> = 0), and the fused path agrees with the plain
  per-gate path at sampled amplitudes;
- N = 32 / 33 wide workload (k = 5, 6 on the tensor cores): ops then their
  inverse return to |0...0>; N = 33 exercises indices beyond 2^32.
- the N = 20, 200-op instance of the wide workload against the FP64 oracle;
- N = 33 diagonal streaming update across the 2^32 index boundary: closed
  form at the populated amplitudes and return under the conjugate table.
"""
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


class Big:
    def __init__(self, q, n):
        self.q, self.n = q, n
        self.buf = torch.empty(1 << n, dtype=torch.complex64, device="cuda:0")
        self.h = q.qsa_state_create_ex(n, self.buf.data_ptr(), self.buf.numel() * 8,
                                       torch.cuda.current_stream().cuda_stream, 1)

    def amps(self, logical_idx):
        """Logical amplitudes at the given indices, decoded through the layout."""
        L = self.q.qsa_get_layout(self.h)
        x = np.asarray(logical_idx, dtype=np.int64)
        y = np.zeros_like(x)
        for qb in range(self.n):
            y |= ((x >> qb) & 1) << L[qb]
        self.q.qsa_state_sync(self.h)
        return self.buf[torch.from_numpy(y).cuda()].cpu().numpy().astype(np.complex128)

    def close(self):
        self.q.qsa_state_destroy(self.h)
        del self.buf
        torch.cuda.empty_cache()


def test_fusion28_qft_closed_form_and_inverse_return(q):
    n = 28
    ops, x0 = W.fusion_circuit(n=n, layers=40, seed=0, with_inverse=True)
    prefix = W.basis_prep(n, x0) + W.qft_ops(n)
    st = Big(q, n)
    try:
        opts = q.make_opts(planner=q.QSA_PLAN_DP, kmax=4, kmax_diag=4, lowering=q.QSA_LOWER_PERMUTE)
        q.qsa_apply_circuit(st.h, prefix, opts)
        ys = np.random.default_rng(1).integers(0, 1 << n, size=256)
        got = st.amps(ys)
        ref = np.exp(2j * np.pi * ((x0 * ys) % (1 << n)) / (1 << n)) / np.sqrt(1 << n)
        assert np.max(np.abs(got - ref)) < 1e-6
        q.qsa_state_reset(st.h)
        stats = q.qsa_apply_circuit(st.h, ops, opts)
        assert stats["blocks"] < len(ops)
        a0 = st.amps([0])[0]
        assert abs(a0) ** 2 >= 1 - 1e-5
    finally:
        st.close()


@pytest.mark.parametrize("kmax,kdiag,kprod,prec,layer,interleave",
                         [(4, 4, 0, 0, 0, False), (6, 6, 0, 1, 0, False), (6, 12, 6, 1, 0, False),
                          (6, 12, 0, 1, 1, False), (6, 12, 0, 1, 1, True)],
                         ids=["kmax4-fp32", "kmax6-3xtf32", "kdiag12-kprod6-3xtf32", "layer-kdiag12-3xtf32",
                              "bench-interleaved-layer-kdiag12-3xtf32"])
def test_qaoa30_symmetries_and_fused_equals_per_gate(q, kmax, kdiag, kprod, prec, layer, interleave):
    """The bench's workload and launch configuration (interleaved initial
    layout set on |0...0>, zero-state prefix, layer units, kmax 6, diagonal
    blocks up to 12 qubits, split-TF32 for k = 5, 6), layer units on the
    identity layout, the product-unit configuration and two dense-only ones."""
    n = 30
    ops, edges = W.qaoa_circuit(n=n, p=8, seed=0)
    st = Big(q, n)
    try:
        if interleave:
            import bench
            q.qsa_set_layout(st.h, bench.interleaved_layout(n), 0)
        stats = q.qsa_apply_circuit(st.h, ops, q.make_opts(planner=q.QSA_PLAN_DP, kmax=kmax, kmax_diag=kdiag,
                                                           kmax_prod=kprod, precision=prec, layer=layer,
                                                           zero_init=1 if interleave else 0))
        if layer:
            assert stats["layer_blocks"] == (24 if interleave else 27) and stats["passes"] == stats["layer_blocks"]
        assert abs(q.qsa_expectation_z(st.h, 0) - 1) < 1e-5
        for qb in (0, 7, 29):
            assert abs(q.qsa_expectation_z(st.h, 1 << qb)) < 1e-5
        xs = np.random.default_rng(2).integers(0, 1 << n, size=128)
        a = st.amps(xs)
        b = st.amps(xs ^ ((1 << n) - 1))
        pa, pb = np.abs(a) ** 2, np.abs(b) ** 2
        assert np.all(np.abs(pa - pb) <= 1e-3 * (pa + pb) + 1e-15)
        q.qsa_state_reset(st.h)
        q.qsa_apply_circuit(st.h, ops, q.make_opts(planner=q.QSA_PLAN_PER_GATE))
        c = st.amps(xs)
        assert np.linalg.norm(a - c) <= 1e-4 * np.linalg.norm(a)
    finally:
        st.close()


@pytest.mark.parametrize("n,n_ops", [(32, 20), (33, 8), (34, 4)])
def test_wide_tensor_core_ops_then_inverse_return(q, n, n_ops):
    ops = W.wide_circuit(n, n_ops=n_ops, widths=(5, 6), seed=n)
    st = Big(q, n)
    try:
        stats = q.qsa_apply_circuit(st.h, ops + W.inverse(ops),
                                    q.make_opts(planner=0, kmax=6, kmax_diag=6, precision=q.QSA_PREC_TF32X3))
        assert stats["tc_blocks"] == 2 * n_ops
        a0 = st.amps([0])[0]
        assert abs(a0) ** 2 >= 1 - 1e-5
        assert abs(q.qsa_expectation_z(st.h, 0) - 1) < 1e-5
    finally:
        st.close()


@pytest.mark.parametrize("prec", [0, 1])
def test_wide_200_ops_fidelity_vs_oracle(q, prec, capsys):
    n = 20
    ops = W.wide_circuit(n, n_ops=200, widths=(5, 6), seed=0)
    st = Big(q, n)
    try:
        q.qsa_apply_circuit(st.h, ops, q.make_opts(planner=0, kmax=6, kmax_diag=6, precision=prec))
        got = st.amps(np.arange(1 << n))
        ref = oracle.run_circuit(n, ops)
        infid, err = check_close(ref, got)
        with capsys.disabled():
            print(f"\nwide 200 ops N=20 precision={'3xTF32' if prec else 'FP32'}: 1-F = {infid:.3e}, "
                  f"max|d| = {err:.3e}")
    finally:
        st.close()


@pytest.mark.parametrize("n", [33, 34])
def test_diag33_beyond_2_32_closed_form_and_inverse(q, n):
    """N = 33 and 34 (the largest state, 128 GiB): H on qubits 0 and N - 1,
    then a 12-qubit diagonal that includes qubit N - 1 (index bit beyond 2^32)
    and bits 0, 11, 12, 23, 24: the four populated amplitudes are d[c] / 2 at
    their target bits; the conjugate table returns the state."""
    top = n - 1
    st = Big(q, n)
    rng = np.random.default_rng(33)
    try:
        for qb in (0, top):
            q.qsa_apply_fused(st.h, [qb], W.H)
        t = [top, 0, 11, 12, 23, 24, 5, 17, 29, 30, 2, 8]
        d = np.exp(1j * rng.uniform(0, 2 * np.pi, size=1 << len(t)))
        q.qsa_apply_diag(st.h, t, d)
        idx = np.array([0, 1, 1 << top, (1 << top) | 1], dtype=np.int64)
        c = np.array([sum(((int(x) >> tq) & 1) << j for j, tq in enumerate(t)) for x in idx])
        got = st.amps(idx)
        assert np.max(np.abs(got - 0.5 * d[c])) < 1e-6
        q.qsa_apply_diag(st.h, t, np.conj(d))
        got = st.amps(idx)
        assert np.max(np.abs(got - 0.5)) < 1e-6
        assert abs(q.qsa_expectation_z(st.h, 0) - 1) < 1e-5
    finally:
        st.close()


@pytest.mark.parametrize("n", [33, 34])
def test_layer33_beyond_2_32_closed_form_and_inverse(q, n):
    """N = 33 and 34 layer blocks whose factors and phase gates reach qubit
    N - 1 (indices beyond 2^32): after H on qubits 0, 17, N - 1 with
    ZZ(N - 1, 5), ZZ(17, N - 1) and a phase on N - 1 the populated amplitudes
    match their closed form; the inverse blocks (factors first, then the
    conjugate phases) return to |0...0>."""
    top = n - 1
    zz = lambda g: np.diag(np.exp(-0.5j * g * np.array([1, -1, -1, 1])))
    diag = [W.Op((top, 5), zz(0.7), True), W.Op((17, top), zz(1.9), True),
            W.Op((top,), np.diag([1, np.exp(0.3j)]), True)]
    t = [0, 17, top]
    st = Big(q, n)
    try:
        q.qsa_apply_layer(st.h, [], t, [W.H] * 3)
        q.qsa_apply_layer(st.h, diag, [], [])
        xs = np.array([0, 1, 1 << 17, 1 << top, (1 << top) | 1, (1 << top) | (1 << 17) | 1, 1 << 5], dtype=np.int64)
        got = st.amps(xs)
        ref = []
        for x in xs:
            populated = (int(x) & ~((1 << 0) | (1 << 17) | (1 << top))) == 0
            b = [(int(x) >> k) & 1 for k in (top, 5, 17)]
            ph = np.exp(-0.5j * 0.7 * (1 - 2 * (b[0] ^ b[1]))) * np.exp(-0.5j * 1.9 * (1 - 2 * (b[2] ^ b[0])))
            ph *= np.exp(0.3j) if b[0] else 1.0
            ref.append(ph / np.sqrt(8) if populated else 0.0)
        assert np.max(np.abs(got - np.array(ref))) < 1e-6
        inv = [W.Op(o.targets, o.matrix.conj().T, True) for o in diag]
        q.qsa_apply_layer(st.h, inv, [], [])
        q.qsa_apply_layer(st.h, [], t, [W.H] * 3)
        assert abs(st.amps([0])[0] - 1) < 1e-5
    finally:
        st.close()
