// Cost model, host side: feature encoding, the process-wide loaded network
// and its evaluation for the DP-MLP planner.  Training runs on the GPU
// (mlp.cu); the planner's queries are host evaluations of the same network.
#include <cmath>
#include <cstdio>
#include <cstring>
#include <memory>
#include <mutex>
#include <string>
#include <vector>

#include "qsa.h"
#include "qsa_costmodel.h"
#include "qsa_runtime.h"

namespace qsa {

namespace {
std::mutex g_mu;
CostModel g_model;   // the process-wide network, or null

// Model files: the 8 bytes "QSACM001", the parameter count (uint32), then
// the parameters as float32, all little-endian (the byte order of every host
// this library builds for).
constexpr char kMagic[8] = {'Q', 'S', 'A', 'C', 'M', '0', '0', '1'};

bool write_model(const char* path, const CostParams& P, std::string* why) {
    FILE* f = std::fopen(path, "wb");
    if (!f) {
        *why = std::string("cannot open ") + path + " for writing";
        return false;
    }
    std::vector<float> v(P.begin(), P.end());
    const uint32_t cnt = static_cast<uint32_t>(v.size());
    bool ok = std::fwrite(kMagic, 1, 8, f) == 8 && std::fwrite(&cnt, sizeof(cnt), 1, f) == 1 &&
              std::fwrite(v.data(), sizeof(float), v.size(), f) == v.size();
    ok = (std::fclose(f) == 0) && ok;
    if (!ok) *why = std::string("short write to ") + path;
    return ok;
}

bool read_model(const char* path, CostModel* out, std::string* why) {
    FILE* f = std::fopen(path, "rb");
    if (!f) {
        *why = std::string("cannot open ") + path;
        return false;
    }
    char magic[8];
    uint32_t cnt = 0;
    std::vector<float> v(kMlpParams);
    bool ok = std::fread(magic, 1, 8, f) == 8 && std::memcmp(magic, kMagic, 8) == 0 &&
              std::fread(&cnt, sizeof(cnt), 1, f) == 1 && cnt == static_cast<uint32_t>(kMlpParams) &&
              std::fread(v.data(), sizeof(float), v.size(), f) == v.size();
    char extra;
    ok = ok && std::fread(&extra, 1, 1, f) == 0;   // nothing after the parameters
    std::fclose(f);
    if (!ok) {
        *why = std::string(path) + " is not a cost-model file of " + std::to_string(kMlpParams) + " parameters";
        return false;
    }
    for (float x : v)
        if (!std::isfinite(x)) {
            *why = std::string(path) + " holds a non-finite parameter";
            return false;
        }
    *out = std::make_shared<const CostParams>(v.begin(), v.end());
    return true;
}
}  // namespace

void costmodel_features(int k, uint64_t phys_mask, int n, int batch, float* x) {
    x[0] = static_cast<float>(k) / 6.0f;
    for (int i = 0; i < 34; ++i) x[1 + i] = static_cast<float>((phys_mask >> i) & 1ull);
    x[35] = static_cast<float>(n) / 34.0f;
    x[36] = static_cast<float>(std::log2(static_cast<double>(batch < 1 ? 1 : batch)) / 8.0);
}

CostModel costmodel_global() {
    std::lock_guard<std::mutex> g(g_mu);
    return g_model;
}

bool costmodel_loaded() { return costmodel_global() != nullptr; }

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

double costmodel_eval(const CostParams& P, int k, uint64_t phys_mask, int n, int batch) {
    float x[kMlpIn];
    costmodel_features(k, phys_mask, n, batch, x);
    return std::exp(forward(P, x));
}

double costmodel_predict_seconds(int k, uint64_t phys_mask, int n, int batch) {
    const CostModel m = costmodel_global();
    return m ? costmodel_eval(*m, k, phys_mask, n, batch) : NAN;
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
    CostModel m = params ? std::make_shared<const CostParams>(params, params + kMlpParams) : nullptr;
    std::lock_guard<std::mutex> g(g_mu);
    g_model = std::move(m);
    return QSA_OK;
}

qsa_status qsa_costmodel_predict(const float* features, size_t n, double* seconds_out) {
    if (!features || !seconds_out) return fail(QSA_E_ARG, "NULL argument");
    const CostModel m = costmodel_global();
    if (!m) return fail(QSA_E_STATE, "no cost model is loaded");
    for (size_t i = 0; i < n; ++i) seconds_out[i] = std::exp(forward(*m, features + i * kMlpIn));
    return QSA_OK;
}

qsa_status qsa_costmodel_save(const char* path) {
    if (!path) return fail(QSA_E_ARG, "path is NULL");
    const CostModel m = costmodel_global();
    if (!m) return fail(QSA_E_STATE, "no cost model is loaded");
    std::string why;
    if (!write_model(path, *m, &why)) return fail(QSA_E_ARG, why);
    return QSA_OK;
}

qsa_status qsa_costmodel_load(qsa_state s, const char* path) {
    CostModel m;
    if (path) {
        std::string why;
        if (!read_model(path, &m, &why)) return fail(QSA_E_ARG, why);
    }
    if (s) {
        s->cm = std::move(m);
        return QSA_OK;
    }
    std::lock_guard<std::mutex> g(g_mu);
    g_model = std::move(m);
    return QSA_OK;
}

}  // extern "C"
