// Density matrices through the state-vector path (§IV-B density-matrix
// wrapper): vec(rho) column-major on 2n qubits, a k-qubit channel as the
// 2k-qubit superoperator sum_i conj(E_i) (x) E_i applied by the fused dense
// path at (targets, targets + n), and the diagonal read out on the GPU.
#include <cuda_runtime.h>

#include <complex>
#include <vector>

#include "qsa.h"
#include "qsa_internal.h"
#include "qsa_runtime.h"

using namespace qsa;

namespace {

qsa_status check_dm(qsa_state s, int n) {
    qsa_status st = check_state(s);
    if (st != QSA_OK) return st;
    if (n < 2 || n > 17) return fail(QSA_E_ARG, "density matrices have 2..17 qubits");
    if (s->n != 2 * n) return fail(QSA_E_ARG, "the state must have 2n qubits for an n-qubit density matrix");
    return QSA_OK;
}

qsa_status dm_diag(qsa_state s, int n, uint64_t mask, bool want_probs, double* out_host, double* sum_out) {
    qsa_status st = ensure_dev(s, reinterpret_cast<void**>(&s->d_red), &s->red_cap,
                               sizeof(double) * (reduce_partials() + 8));
    if (st != QSA_OK) return st;
    double* d_sum = s->d_red + reduce_partials();
    double* d_out = nullptr;
    const size_t dim = size_t(1) << n;
    if (want_probs) {
        st = ensure_dev(s, reinterpret_cast<void**>(&s->d_dm), &s->dm_cap, sizeof(double) * dim);
        if (st != QSA_OK) return st;
        d_out = s->d_dm;
    }
    cudaError_t e = launch_dm_diag(s->psi, n, s->L, mask, d_out, s->d_red, d_sum, s->stream, &s->launches);
    if (e != cudaSuccess) return cuda_fail(s, e, "density-matrix diagonal kernel");
    if (want_probs && out_host) {
        e = cudaMemcpyAsync(out_host, d_out, sizeof(double) * dim, cudaMemcpyDeviceToHost, s->stream);
        if (e != cudaSuccess) return cuda_fail(s, e, "density-matrix diagonal copy");
    }
    double sum = 0.0;
    e = cudaMemcpyAsync(&sum, d_sum, sizeof(double), cudaMemcpyDeviceToHost, s->stream);
    if (e != cudaSuccess) return cuda_fail(s, e, "density-matrix reduction copy");
    st = sync_and_check(s, "density-matrix readout");
    if (st != QSA_OK) return st;
    if (sum_out) *sum_out = sum;
    return QSA_OK;
}

}  // namespace

extern "C" {

qsa_status qsa_dm_superoperator(int n, const int32_t* targets, int k, const double* kraus, int n_kraus,
                                int32_t* targets_out, double* matrix_out) {
    if (n < 2 || n > 17) return fail(QSA_E_ARG, "density matrices have 2..17 qubits");
    if (k < 1 || k > 3) return fail(QSA_E_ARG, "density-matrix channels act on 1..3 qubits");
    if (!targets || !targets_out || !matrix_out) return fail(QSA_E_ARG, "NULL argument");
    qsa_status st = validate_targets(n, targets, k);
    if (st != QSA_OK) return st;
    if (n_kraus < 1 || !kraus) return fail(QSA_E_ARG, "a channel needs at least one Kraus operator");
    const size_t d = size_t(1) << k, D = d * d;
    // S[c1 * d + r1][c0 * d + r0] = sum_i conj(E_i[c1][c0]) E_i[r1][r0]
    std::vector<std::complex<double>> S(D * D, 0.0);
    for (int i = 0; i < n_kraus; ++i) {
        const double* E = kraus + static_cast<size_t>(i) * 2 * d * d;
        auto e = [&](size_t r, size_t c) { return std::complex<double>(E[2 * (r * d + c)], E[2 * (r * d + c) + 1]); };
        for (size_t c1 = 0; c1 < d; ++c1)
            for (size_t c0 = 0; c0 < d; ++c0) {
                const std::complex<double> a = std::conj(e(c1, c0));
                if (a == 0.0) continue;
                for (size_t r1 = 0; r1 < d; ++r1)
                    for (size_t r0 = 0; r0 < d; ++r0) S[(c1 * d + r1) * D + (c0 * d + r0)] += a * e(r1, r0);
            }
    }
    for (size_t i = 0; i < D * D; ++i) {
        matrix_out[2 * i] = S[i].real();
        matrix_out[2 * i + 1] = S[i].imag();
    }
    for (int j = 0; j < k; ++j) {
        targets_out[j] = targets[j];
        targets_out[j + k] = targets[j] + n;
    }
    return QSA_OK;
}

qsa_status qsa_dm_apply_channel(qsa_state s, int n, const int32_t* targets, int k, const double* kraus,
                                int n_kraus, int precision) {
    qsa_status st = check_dm(s, n);
    if (st != QSA_OK) return st;
    int32_t tg[6];
    std::vector<double> S;
    if (k >= 1 && k <= 3) S.resize(2 * (size_t(1) << (4 * k)));
    st = qsa_dm_superoperator(n, targets, k, kraus, n_kraus, tg, S.data());
    if (st != QSA_OK) return st;
    return qsa_apply_fused_ex(s, tg, 2 * k, S.data(), QSA_LOWER_AUTO, precision);
}

qsa_status qsa_dm_probabilities(qsa_state s, int n, double* out_host, double* trace_out) {
    qsa_status st = check_dm(s, n);
    if (st != QSA_OK) return st;
    return dm_diag(s, n, 0, out_host != nullptr, out_host, trace_out);
}

qsa_status qsa_dm_expectation_z(qsa_state s, int n, uint64_t mask, double* out) {
    qsa_status st = check_dm(s, n);
    if (st != QSA_OK) return st;
    if (!out) return fail(QSA_E_ARG, "out is NULL");
    if (mask >> n) return fail(QSA_E_ARG, "mask has bits beyond n");
    return dm_diag(s, n, mask, false, nullptr, out);
}

}  // extern "C"
