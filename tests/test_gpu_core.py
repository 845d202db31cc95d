"""GPU parity tests: the CUDA path through the C ABI against the FP64 oracle.

Tolerances (floating point): 1 - |<psi_gpu|psi_ref>|^2 <= 1e-5 and
max |psi_gpu - psi_ref| <= 1e-5; permutation, probabilities-from-identical-
amplitudes and sampling are compared bit for bit.
"""
import numpy as np
import pytest

import oracle
import workloads as W

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

FID_TOL = 1e-5
AMP_TOL = 1e-5


@pytest.fixture(scope="module")
def q():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_2608_16940_gb300 as q
    return q


class GState:
    """A libqsa state over a torch-owned complex64 buffer on cuda:0."""

    def __init__(self, q, n, init=None):
        self.q, self.n = q, n
        self.buf = torch.zeros(1 << n, dtype=torch.complex64, device="cuda:0")
        if init is not None:
            self.buf.copy_(torch.from_numpy(np.ascontiguousarray(init, dtype=np.complex64)))
            torch.cuda.synchronize()
        self.stream = torch.cuda.current_stream().cuda_stream
        self.h = q.qsa_state_create_ex(n, self.buf.data_ptr(), self.buf.numel() * 8, self.stream,
                                       0 if init is not None else 1)

    def stored(self):
        torch.cuda.synchronize()
        return self.buf.cpu().numpy().astype(np.complex128)

    def logical(self):
        return oracle.decode_state(self.stored(), self.q.qsa_get_layout(self.h))

    def close(self):
        self.q.qsa_state_destroy(self.h)


def _check_close(ref, got):
    f = oracle.fidelity(ref, got)
    e = oracle.max_abs_diff(ref, got)
    assert abs(1 - f) <= FID_TOL and e <= AMP_TOL, (1 - f, e)


@pytest.mark.parametrize("k", [1, 2, 3, 4, 5, 6])
@pytest.mark.parametrize("n", [6, 9, 14, 17])
@pytest.mark.parametrize("lowering", [0, 2])
def test_single_fused_op_matches_oracle(q, k, n, lowering):
    if k > n:
        pytest.skip("k > n")
    rng = np.random.default_rng(100 * k + n + lowering)
    psi = W.random_state(n, seed=k * 31 + n)
    st = GState(q, n, init=psi.astype(np.complex64))
    ref = psi.astype(np.complex64).astype(np.complex128)
    try:
        for trial in range(3):
            t = tuple(int(v) for v in rng.choice(n, size=k, replace=False))
            G = W.haar_unitary(1 << k, rng)
            q.qsa_apply_fused_ex(st.h, t, G, lowering, q.QSA_PREC_FP32)
            oracle.apply(ref, t, G)
        _check_close(ref, st.logical())
    finally:
        st.close()


@pytest.mark.parametrize("targets", [(0,), (1, 0), (0, 1, 2, 3, 4, 5), (13, 0), (5, 12, 13), (10, 11, 12, 13)])
def test_low_and_high_target_mixes(q, targets):
    n = 14
    rng = np.random.default_rng(len(targets))
    k = len(targets)
    G = W.haar_unitary(1 << k, rng)
    psi = W.random_state(n, 7)
    st = GState(q, n, init=psi.astype(np.complex64))
    ref = psi.astype(np.complex64).astype(np.complex128)
    try:
        q.qsa_apply_fused(st.h, targets, G)
        oracle.apply(ref, targets, G)
        _check_close(ref, st.logical())
    finally:
        st.close()


# Target sets that select each stage form of the FP32 k <= 4 kernels (from the
# five lowest non-target positions, the bits that vary across a warp): plain
# layout (no target among the low positions), swizzled gathers (two or more of
# positions 0..3 are targets, not both 0 and 1), and swizzled gathers with the
# in-place write-back (positions 0 and 1 are both targets).
FORM_TARGETS = {
    "plain": {1: (11,), 2: (10, 11), 3: (9, 10, 11), 4: (8, 9, 10, 11)},
    "swizzled": {2: (2, 3), 3: (1, 2, 3), 4: (1, 3, 5, 7)},
    "write_back": {2: (0, 1), 3: (1, 0, 7), 4: (3, 0, 2, 1)},
}


@pytest.mark.parametrize("form,k", [(f, k) for f, d in FORM_TARGETS.items() for k in d])
@pytest.mark.parametrize("n", [12, 15])
def test_fp32_stage_forms_match_oracle(q, form, k, n):
    targets = FORM_TARGETS[form][k]
    rng = np.random.default_rng(7 * k + n)
    psi = W.random_state(n, 11 + k)
    st = GState(q, n, init=psi.astype(np.complex64))
    ref = psi.astype(np.complex64).astype(np.complex128)
    try:
        for _ in range(2):
            G = W.haar_unitary(1 << k, rng)
            q.qsa_apply_fused_ex(st.h, targets, G, 0, q.QSA_PREC_FP32)
            oracle.apply(ref, targets, G)
        _check_close(ref, st.logical())
    finally:
        st.close()


def test_brick_circuit_per_gate_matches_oracle(q):
    """Plain per-gate path at N=12 (20 brick layers of Haar U(2) + CZ)."""
    n = 12
    ops = W.brick_circuit(n, 20, seed=0)
    st = GState(q, n)
    try:
        stats = q.qsa_apply_circuit(st.h, ops, q.make_opts(planner=q.QSA_PLAN_PER_GATE))
        assert stats["blocks"] == len(ops)
        ref = oracle.run_circuit(n, ops)
        _check_close(ref, st.logical())
        probs, norm = q.qsa_probabilities(st.h)
        assert abs(norm - 1) < 1e-5
        assert np.max(np.abs(probs - np.abs(ref) ** 2)) < 1e-5
    finally:
        st.close()


@pytest.mark.parametrize("planner,kmax,lowering", [(1, 2, 0), (1, 4, 0), (2, 4, 0), (2, 4, 2), (2, 6, 0),
                                                   (2, 5, 2)])
def test_fused_circuit_matches_oracle(q, planner, kmax, lowering):
    n = 16
    ops, x0 = W.fusion_circuit(n=n, layers=3, seed=planner * 10 + kmax, with_inverse=False)
    st = GState(q, n)
    try:
        stats = q.qsa_apply_circuit(st.h, ops, q.make_opts(planner=planner, kmax=kmax, kmax_diag=kmax,
                                                           lowering=lowering))
        assert stats["blocks"] < len(ops)
        ref = oracle.run_circuit(n, ops)
        _check_close(ref, st.logical())
    finally:
        st.close()


def test_fusion_workload_returns_to_zero(q):
    """QFT on a random basis state + layers + the inverse returns to |0...0>."""
    n = 18
    ops, _ = W.fusion_circuit(n=n, layers=6, seed=1, with_inverse=True)
    st = GState(q, n)
    try:
        q.qsa_apply_circuit(st.h, ops, q.make_opts(planner=q.QSA_PLAN_DP, kmax=4, lowering=q.QSA_LOWER_PERMUTE))
        got = st.logical()
        assert abs(got[0]) ** 2 >= 1 - FID_TOL
    finally:
        st.close()


@pytest.mark.parametrize("n", [3, 11, 15, 20])
def test_permutation_is_bit_exact(q, n):
    rng = np.random.default_rng(n)
    psi = W.random_state(n, n).astype(np.complex64)
    st = GState(q, n, init=psi)
    ref = psi.copy()
    try:
        for _ in range(4):
            npairs = int(rng.integers(1, min(6, n // 2) + 1))
            pos = [int(v) for v in rng.choice(n, size=2 * npairs, replace=False)]
            a, b = pos[:npairs], pos[npairs:]
            q.qsa_permute_bits(st.h, a, b)
            idx = np.arange(1 << n, dtype=np.int64)
            src = idx.copy()
            for x, y in zip(a, b):
                bx, by = (src >> x) & 1, (src >> y) & 1
                src = src ^ ((bx ^ by) << x) ^ ((bx ^ by) << y)
            ref = ref[src]
        got = st.stored().astype(np.complex64)
        assert np.array_equal(got.view(np.uint64), ref.view(np.uint64))
        # the layout map records the same transpositions: decoding gives the input
        assert np.array_equal(st.logical().astype(np.complex64).view(np.uint64), psi.view(np.uint64))
    finally:
        st.close()


def test_set_layout_materialise_and_metadata(q):
    n = 13
    rng = np.random.default_rng(2)
    psi = W.random_state(n, 3).astype(np.complex64)
    st = GState(q, n, init=psi)
    try:
        L = [int(v) for v in rng.permutation(n)]
        q.qsa_set_layout(st.h, L, 1)
        assert q.qsa_get_layout(st.h) == L
        assert np.array_equal(st.stored().astype(np.complex64), oracle.encode_state(psi, L))
        with pytest.raises(q.QsaError) as e:
            q.qsa_set_layout(st.h, list(range(n)), 0)
        assert e.value.code == q.QSA_E_STATE
    finally:
        st.close()
    st = GState(q, n)
    try:
        L = [int(v) for v in rng.permutation(n)]
        q.qsa_set_layout(st.h, L, 0)        # |0..0> is permutation invariant
        G = W.haar_unitary(8, rng)
        q.qsa_apply_fused(st.h, (0, 5, 9), G)
        ref = oracle.zero_state(n)
        oracle.apply(ref, (0, 5, 9), G)
        _check_close(ref, st.logical())
    finally:
        st.close()


def test_probabilities_bit_exact_on_identical_amplitudes(q):
    n = 15
    psi = W.random_state(n, 4).astype(np.complex64)
    st = GState(q, n, init=psi)
    try:
        L = [int(v) for v in np.random.default_rng(4).permutation(n)]
        q.qsa_set_layout(st.h, L, 1)
        probs, norm = q.qsa_probabilities(st.h)
        ref = oracle.probabilities(psi.astype(np.complex128))
        assert np.array_equal(probs, ref)
        assert abs(norm - ref.sum()) < 1e-12
    finally:
        st.close()


def test_expectation_z_matches_oracle(q):
    n = 14
    psi = W.random_state(n, 5).astype(np.complex64)
    st = GState(q, n, init=psi)
    p64 = psi.astype(np.complex128)
    try:
        q.qsa_set_layout(st.h, [int(v) for v in np.random.default_rng(5).permutation(n)], 1)
        for mask in [0, 1, 1 << 13, 0b101, (1 << 7) | (1 << 2), (1 << n) - 1]:
            got = q.qsa_expectation_z(st.h, mask)
            assert abs(got - oracle.expect_z(p64, mask)) < 1e-12
    finally:
        st.close()
    st = GState(q, n)
    try:
        q.qsa_apply_circuit(st.h, W.ghz_ops(n))
        assert abs(q.qsa_expectation_z(st.h, 1 << 3)) < 1e-6
        assert abs(q.qsa_expectation_z(st.h, (1 << 2) | (1 << 9)) - 1) < 1e-6
    finally:
        st.close()


def test_expectation_z_batch_equals_single_masks(q):
    """Several masks in one pass: each result bit-identical to the one-mask
    reduction (same per-thread accumulation order) and to the oracle."""
    n = 15
    psi = W.random_state(n, 6).astype(np.complex64)
    st = GState(q, n, init=psi)
    p64 = psi.astype(np.complex128)
    try:
        q.qsa_set_layout(st.h, [int(v) for v in np.random.default_rng(6).permutation(n)], 1)
        for masks in ([0], [0, 1 << 14], [3, 0b1010, (1 << n) - 1, 1 << 7]):
            got = q.qsa_expectation_z_batch(st.h, masks)
            for m, g in zip(masks, got):
                assert g == q.qsa_expectation_z(st.h, m)
                assert abs(g - oracle.expect_z(p64, m)) < 1e-12
        for bad in ([], [0] * 5, [1 << n]):
            with pytest.raises(q.QsaError):
                q.qsa_expectation_z_batch(st.h, bad)
    finally:
        st.close()


@pytest.mark.parametrize("n,shots,perm,zero_frac", [(4, 100, False, 0.0), (10, 1000, True, 0.5),
                                                    (13, 5000, True, 0.0), (16, 9000, False, 0.9),
                                                    (23, 3000, True, 0.0), (24, 1000, False, 0.3),
                                                    (24, 1, False, 0.0)])
def test_sampler_bit_exact_vs_oracle(q, n, shots, perm, zero_frac):
    """N >= 23 has more than one 4096-entry segment of block weights (the
    multi-CTA scan; with one shot the one-CTA scan)."""
    psi = W.random_state(n, 6 + n, zero_frac=zero_frac).astype(np.complex64)
    st = GState(q, n, init=psi)
    L = [int(v) for v in np.random.default_rng(n).permutation(n)] if perm else list(range(n))
    try:
        q.qsa_set_layout(st.h, L, 1)
        vals, cnts = q.qsa_sample_counts(st.h, shots, seed=1234)
        rv, rc = oracle.sample_counts(psi.astype(np.complex128), L, shots, 1234)
        assert np.array_equal(vals, rv) and np.array_equal(cnts, rc)
        assert int(cnts.sum()) == shots
    finally:
        st.close()


@pytest.mark.parametrize("n", [12, 16])
def test_sampler_components_at_two(q, n):
    """Blocks holding a component of magnitude 2 (the largest the weights are
    defined for: floor(2^2 2^60) = 2^62) beside blocks without one: the
    weights pass takes its general per-component path for those blocks only,
    and the draws, counts and <Z> sums still match the oracle."""
    psi = W.random_state(n, 90 + n)
    rng = np.random.default_rng(n)
    for y in rng.choice(1 << n, size=2, replace=False):
        if rng.random() < 0.5:
            psi[y] = complex(-2.0 if rng.random() < 0.5 else 2.0, psi[y].imag)
        else:
            psi[y] = complex(psi[y].real, -2.0 if rng.random() < 0.5 else 2.0)
    psi = psi.astype(np.complex64)
    st = GState(q, n, init=psi)
    p64 = psi.astype(np.complex128)
    L = list(range(n))
    try:
        masks = [0, 1 << (n - 1), 0b1011]
        z, vals, cnts = q.qsa_measure(st.h, masks, 4000, seed=5)
        rv, rc = oracle.sample_counts(p64, L, 4000, 5)
        assert np.array_equal(vals, rv) and np.array_equal(cnts, rc)
        for m, g in zip(masks, z):
            ref = oracle.expect_z(p64, m)
            assert abs(g - ref) < 1e-12 * max(1.0, abs(ref))
    finally:
        st.close()


@pytest.mark.parametrize("n,perm", [(12, True), (23, False)])
def test_measure_equals_expectations_and_sampling(q, n, perm):
    """qsa_measure: the same counts as qsa_sample_counts (bit for bit) and the
    same sums as qsa_expectation_z to FP64 rounding, from one pass."""
    psi = W.random_state(n, 40 + n).astype(np.complex64)
    st = GState(q, n, init=psi)
    p64 = psi.astype(np.complex128)
    try:
        if perm:
            q.qsa_set_layout(st.h, [int(v) for v in np.random.default_rng(n).permutation(n)], 1)
        masks = [0, 1 << (n - 1), 0b1011, (1 << n) - 1]
        z, vals, cnts = q.qsa_measure(st.h, masks, 2000, seed=77)
        v2, c2 = q.qsa_sample_counts(st.h, 2000, seed=77)
        assert np.array_equal(vals, v2) and np.array_equal(cnts, c2)
        for m, g in zip(masks, z):
            assert abs(g - q.qsa_expectation_z(st.h, m)) < 1e-13
            assert abs(g - oracle.expect_z(p64, m)) < 1e-12
        z0, v0, c0 = q.qsa_measure(st.h, [], 500, seed=1)
        assert z0 == [] and int(c0.sum()) == 500
        with pytest.raises(q.QsaError):
            q.qsa_measure(st.h, [0] * 5, 10, seed=1)
    finally:
        st.close()


def test_sampler_capacity_and_basis_state(q):
    n = 12
    st = GState(q, n)
    try:
        x = 0b101100101101
        q.qsa_apply_circuit(st.h, W.basis_prep(n, x))
        vals, cnts = q.qsa_sample_counts(st.h, 777, seed=3)
        assert list(vals) == [x] and list(cnts) == [777]
        q.qsa_apply_circuit(st.h, [W.Op((0,), W.H), W.Op((1,), W.H)])
        with pytest.raises(q.QsaError) as e:
            q.qsa_sample_counts(st.h, 1000, seed=3, capacity=2)
        assert e.value.code == q.QSA_E_RANGE
    finally:
        st.close()


def test_invalid_arguments_rejected_before_launch(q):
    st = GState(q, 8)
    try:
        for t in [(8,), (1, 1), (-1,)]:
            with pytest.raises(q.QsaError) as e:
                q.qsa_apply_fused(st.h, t, np.eye(1 << len(t)))
            assert e.value.code == q.QSA_E_ARG
        with pytest.raises(q.QsaError):
            q.qsa_set_layout(st.h, [0, 0, 1, 2, 3, 4, 5, 6], 1)
        with pytest.raises(q.QsaError):
            q.qsa_permute_bits(st.h, [1, 2], [2, 3])
        with pytest.raises(q.QsaError):
            q.qsa_sample_counts(st.h, 0, 1)
    finally:
        st.close()
