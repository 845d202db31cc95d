"""GPU parity of the density-matrix path (§IV-B density-matrix wrapper; n =
2..17 qubits held as a 2n-qubit vec(rho)) against the FP64 oracle's
sum_i E_i rho E_i^dagger: sequences of random channels applied one at a time
(FP32 and split-TF32 for the 6-axis superoperators of 3-qubit channels), under
a permuted layout, and lowered channels fused by the planner; the diagonal
readout (probabilities, trace, Tr(rho Z)); and the largest size, n = 17 (2^34
amplitudes, 128 GiB), against per-cluster oracle results on sampled
elements."""
import numpy as np
import pytest

import oracle
import workloads as W
from gpu_helpers import GState

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

TOL = 1e-5   # max |vec(rho)_gpu - vec(rho)_ref|, FP32 data


@pytest.fixture(scope="module")
def q():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_2608_16940_gb300 as q
    return q


def _oracle_rho(n, chans):
    rho = oracle.dm_zero(n)
    for c in chans:
        rho = oracle.dm_apply_channel(rho, c.targets, c.kraus)
    return rho


def _z_expect(rho, mask):
    d = np.real(np.diag(rho))
    x = np.arange(d.size)
    sign = np.array([1 - 2 * (bin(int(v) & mask).count("1") & 1) for v in x])
    return float(np.sum(d * sign))


def _check_readout(q, h, n, rho):
    probs, tr = q.qsa_dm_probabilities(h, n)
    ref = np.real(np.diag(rho))
    assert abs(tr - np.trace(rho).real) < TOL
    assert np.max(np.abs(probs - ref)) < TOL
    _, tr2 = q.qsa_dm_probabilities(h, n, want_probs=False)
    assert tr2 == pytest.approx(tr, abs=1e-12)
    for mask in (0, 1, (1 << n) - 1, 0b101 & ((1 << n) - 1)):
        assert abs(q.qsa_dm_expectation_z(h, n, mask) - _z_expect(rho, mask)) < TOL


@pytest.mark.parametrize("n,n_ch,seed,prec,permuted", [(2, 12, 0, 0, False), (3, 20, 1, 0, True),
                                                       (5, 30, 2, 0, False), (7, 24, 3, 1, True),
                                                       (8, 16, 4, 1, False)])
def test_channel_sequence_matches_oracle(q, n, n_ch, seed, prec, permuted):
    rng = np.random.default_rng(seed)
    chans = W.random_channel_circuit(n, n_ch, rng, kmax=min(3, n))
    st = GState(q, torch, 2 * n)
    try:
        if permuted:
            q.qsa_set_layout(st.h, [int(v) for v in rng.permutation(2 * n)], 1)
        for c in chans:
            q.qsa_dm_apply_channel(st.h, n, c.targets, c.kraus, prec)
        rho = _oracle_rho(n, chans)
        got = st.logical()
        assert np.max(np.abs(got - oracle.dm_vec(rho))) < TOL
        _check_readout(q, st.h, n, rho)
    finally:
        st.close()


def test_unitary_circuit_gives_pure_state_projector(q):
    """A unitary brick circuit as one-operator channels: rho = |psi><psi| with
    psi from the state-vector oracle."""
    n = 6
    ops = W.brick_circuit(n, 4, seed=9)
    st = GState(q, torch, 2 * n)
    try:
        for o in ops:
            q.qsa_dm_apply_channel(st.h, n, o.targets, [o.matrix])
        psi = oracle.run_circuit(n, ops)
        rho = np.outer(psi, psi.conj())
        assert np.max(np.abs(st.logical() - oracle.dm_vec(rho))) < TOL
        _check_readout(q, st.h, n, rho)
    finally:
        st.close()


@pytest.mark.parametrize("n,planner,kmax,prec", [(7, 2, 6, 1), (7, 1, 4, 0), (6, 2, 6, 0)])
def test_lowered_channels_through_fused_plans(q, n, planner, kmax, prec):
    """Noisy GHZ plus random channels, lowered to 2k-axis operators and
    planned like any circuit: the fused blocks act as the channel sequence."""
    rng = np.random.default_rng(n + planner)
    chans = W.noisy_ghz_channels(n, 0.05) + W.random_channel_circuit(n, 10, rng, kmax=3)
    ops = [q.qsa_dm_superoperator(n, c.targets, c.kraus) for c in chans]
    st = GState(q, torch, 2 * n)
    try:
        stats = q.qsa_apply_circuit(st.h, ops, q.make_opts(planner=planner, kmax=kmax, precision=prec))
        assert stats["blocks"] < len(ops)
        rho = _oracle_rho(n, chans)
        assert np.max(np.abs(st.logical() - oracle.dm_vec(rho))) < TOL
        _check_readout(q, st.h, n, rho)
    finally:
        st.close()


def test_depolarised_to_maximally_mixed(q):
    """Depolarising noise with p = 3/4 on every qubit maps any state to I/2^n."""
    n = 9
    rng = np.random.default_rng(5)
    st = GState(q, torch, 2 * n)
    try:
        for c in W.random_channel_circuit(n, 12, rng, kmax=3):
            q.qsa_dm_apply_channel(st.h, n, c.targets, c.kraus)
        for t in range(n):
            q.qsa_dm_apply_channel(st.h, n, [t], W.depolarising_kraus(1, 0.75))
        probs, tr = q.qsa_dm_probabilities(st.h, n)
        assert abs(tr - 1) < TOL
        assert np.max(np.abs(probs - 1.0 / (1 << n))) < 1e-7
        got = st.logical()
        ref = oracle.dm_vec(np.eye(1 << n) / (1 << n))
        assert np.max(np.abs(got - ref)) < 1e-7
    finally:
        st.close()


def test_density_argument_errors(q):
    st = GState(q, torch, 8)
    try:
        for args in [(3, [0], [np.eye(2)]), (4, [4], [np.eye(2)]), (4, [0, 0], [np.eye(4)]),
                     (4, [0, 1, 2, 3], [np.eye(16)])]:
            with pytest.raises(q.QsaError) as e:
                q.qsa_dm_apply_channel(st.h, *args)
            assert e.value.code == q.QSA_E_ARG
        with pytest.raises(q.QsaError):
            q.qsa_dm_probabilities(st.h, 3)
        with pytest.raises(q.QsaError):
            q.qsa_dm_expectation_z(st.h, 4, 1 << 4)
    finally:
        st.close()


def _cluster_rho(n_c, chans):
    rho = oracle.dm_zero(n_c)
    for t, kr in chans:
        rho = oracle.dm_apply_channel(rho, t, kr)
    return rho


def test_n17_largest_density_matrix(q):
    """n = 17 (2^34 complex64 amplitudes): channels on disjoint qubit clusters
    keep rho a tensor product, so every element is a product of small
    oracle results; the full diagonal, the trace, Tr(rho Z) and 4096 sampled
    off-diagonal elements are checked."""
    n = 17
    rng = np.random.default_rng(17)
    clusters = [  # (qubits, [(local targets, kraus)])
        ((0, 16), [((0,), [W.H]), ((0, 1), [W.CNOT]), ((1,), W.amplitude_damping_kraus(0.3)),
                   ((1, 0), W.depolarising_kraus(2, 0.1))]),
        ((3, 8, 12), [((2, 0, 1), [W.haar_unitary(8, rng)]), ((0, 1, 2), W.random_kraus(3, 2, rng))]),
        ((9,), [((0,), [W.H]), ((0,), W.depolarising_kraus(1, 0.3))]),
        ((15,), [((0,), W.random_kraus(1, 3, rng))]),
    ]
    torch.cuda.empty_cache()
    st = GState(q, torch, 2 * n)
    try:
        for qs, chans in clusters:
            for t, kr in chans:
                q.qsa_dm_apply_channel(st.h, n, [qs[j] for j in t], kr, 1)
        rhos = [_cluster_rho(len(qs), chans) for qs, chans in clusters]
        used = 0
        for qs, _ in clusters:
            for v in qs:
                used |= 1 << v

        def expected(rows, cols):
            val = np.ones(rows.size, dtype=np.complex128)
            val[((rows | cols) & ~used & ((1 << n) - 1)) != 0] = 0
            for (qs, _), r in zip(clusters, rhos):
                ri = np.zeros(rows.size, dtype=np.int64)
                ci = np.zeros(rows.size, dtype=np.int64)
                for j, v in enumerate(qs):
                    ri |= ((rows >> v) & 1) << j
                    ci |= ((cols >> v) & 1) << j
                val *= r[ri, ci]
            return val

        x = np.arange(1 << n, dtype=np.int64)
        probs, tr = q.qsa_dm_probabilities(st.h, n)
        ref_diag = expected(x, x).real
        assert abs(tr - 1) < TOL
        assert np.max(np.abs(probs - ref_diag)) < 1e-6
        for mask in (1 << 16, (1 << 3) | (1 << 12), (1 << 9) | (1 << 15) | 1):
            ref = float(np.sum(ref_diag * (1 - 2 * (np.array([bin(int(v) & mask).count("1") for v in x]) & 1))))
            assert abs(q.qsa_dm_expectation_z(st.h, n, mask) - ref) < TOL

        # sampled elements: rows and columns over the clusters' qubits (others 0)
        bits = [v for qs, _ in clusters for v in qs]
        m = 4096
        rows = np.zeros(m, dtype=np.int64)
        cols = np.zeros(m, dtype=np.int64)
        for v in bits:
            rows |= rng.integers(0, 2, m) << v
            cols |= rng.integers(0, 2, m) << v
        lay = q.qsa_get_layout(st.h)
        logical = rows | (cols << n)
        phys = np.zeros(m, dtype=np.int64)
        for lq in range(2 * n):
            phys |= ((logical >> lq) & 1) << lay[lq]
        q.qsa_state_sync(st.h)
        got = st.buf[torch.from_numpy(phys).to("cuda:0")].cpu().numpy().astype(np.complex128)
        assert np.max(np.abs(got - expected(rows, cols))) < 1e-6
    finally:
        st.close()
        del st
        torch.cuda.empty_cache()
