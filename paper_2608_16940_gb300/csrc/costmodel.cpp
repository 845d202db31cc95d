// Cost model, host side: feature encoding, the process-wide loaded network
// and its evaluation for the DP-MLP planner.  Training runs on the GPU
// (mlp.cu); the planner's queries are host evaluations of the same network.
#include <cmath>
#include <cstring>
#include <mutex>
#include <vector>

#include "qsa.h"
#include "qsa_costmodel.h"
#include "qsa_runtime.h"

namespace qsa {

namespace {
std::mutex g_mu;
std::vector<double> g_params;  // kMlpParams values, layout W1 b1 W2 b2 W3 b3
bool g_loaded = false;
}  // namespace

void costmodel_features(int k, uint64_t phys_mask, int n, int batch, float* x) {
    x[0] = static_cast<float>(k) / 6.0f;
    for (int i = 0; i < 34; ++i) x[1 + i] = static_cast<float>((phys_mask >> i) & 1ull);
    x[35] = static_cast<float>(n) / 34.0f;
    x[36] = static_cast<float>(std::log2(static_cast<double>(batch < 1 ? 1 : batch)) / 8.0);
}

bool costmodel_loaded() {
    std::lock_guard<std::mutex> g(g_mu);
    return g_loaded;
}

static double forward(const std::vector<double>& P, const float* x) {
    const double* W1 = P.data();
    const double* b1 = W1 + kMlpH * kMlpIn;
    const double* W2 = b1 + kMlpH;
    const double* b2 = W2 + kMlpH * kMlpH;
    const double* W3 = b2 + kMlpH;
    const double* b3 = W3 + kMlpH;
    double a1[kMlpH], a2[kMlpH];
    for (int i = 0; i < kMlpH; ++i) {
        double z = b1[i];
        for (int j = 0; j < kMlpIn; ++j) z += W1[i * kMlpIn + j] * x[j];
        a1[i] = z > 0 ? z : 0;
    }
    for (int i = 0; i < kMlpH; ++i) {
        double z = b2[i];
        for (int j = 0; j < kMlpH; ++j) z += W2[i * kMlpH + j] * a1[j];
        a2[i] = z > 0 ? z : 0;
    }
    double y = b3[0];
    for (int j = 0; j < kMlpH; ++j) y += W3[j] * a2[j];
    return y;
}

double costmodel_predict_seconds(int k, uint64_t phys_mask, int n, int batch) {
    float x[kMlpIn];
    costmodel_features(k, phys_mask, n, batch, x);
    std::lock_guard<std::mutex> g(g_mu);
    if (!g_loaded) return NAN;
    return std::exp(forward(g_params, x));
}

}  // namespace qsa

using namespace qsa;

extern "C" {

qsa_status qsa_costmodel_features(int k, uint64_t phys_mask, int n_qubits, int batch, float* out37) {
    if (!out37 || k < 1 || k > QSA_MAX_K || n_qubits < 1 || n_qubits > QSA_MAX_QUBITS)
        return fail(QSA_E_ARG, "bad feature arguments");
    costmodel_features(k, phys_mask, n_qubits, batch, out37);
    return QSA_OK;
}

qsa_status qsa_costmodel_set(const float* params) {
    std::lock_guard<std::mutex> g(g_mu);
    if (!params) {
        g_loaded = false;
        g_params.clear();
        return QSA_OK;
    }
    g_params.assign(params, params + kMlpParams);
    g_loaded = true;
    return QSA_OK;
}

qsa_status qsa_costmodel_predict(const float* features, size_t n, double* seconds_out) {
    if (!features || !seconds_out) return fail(QSA_E_ARG, "NULL argument");
    std::lock_guard<std::mutex> g(g_mu);
    if (!g_loaded) return fail(QSA_E_STATE, "no cost model is loaded");
    for (size_t i = 0; i < n; ++i) seconds_out[i] = std::exp(forward(g_params, features + i * kMlpIn));
    return QSA_OK;
}

}  // extern "C"
