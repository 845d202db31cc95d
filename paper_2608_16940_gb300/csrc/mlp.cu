// Cost model: a 37 -> 64 -> 64 -> 1 ReLU network that predicts log(seconds)
// of one fused-operator pass from (k, physical target mask, N, batch), trained
// on timings the library collects from its own kernels.  Forward, backward
// and Adam (Kingma & Ba 2015, Algorithm 1) run as CUDA kernels in FP32;
// batch reductions use a fixed order, so results are deterministic.
//
// Parameter layout (6657 floats): W1[64][37], b1[64], W2[64][64], b2[64],
// W3[1][64], b3[1].
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <cstring>
#include <numeric>
#include <string>
#include <vector>

#include "qsa.h"
#include "qsa_costmodel.h"
#include "qsa_internal.h"
#include "qsa_runtime.h"

namespace qsa {

namespace {

constexpr int IN = kMlpIn, H = kMlpH;
constexpr int OFF_W1 = 0, OFF_B1 = H * IN, OFF_W2 = OFF_B1 + H, OFF_B2 = OFF_W2 + H * H, OFF_W3 = OFF_B2 + H,
              OFF_B3 = OFF_W3 + H;

// Z = X W^T + b, A = relu(Z) (A may be null); one thread per (sample, unit).
__global__ void k_dense(const float* __restrict__ X, int in, const float* __restrict__ W, const float* __restrict__ b,
                        int out, size_t n, float* __restrict__ Z, float* __restrict__ A) {
    const size_t idx = static_cast<size_t>(blockIdx.x) * blockDim.x + threadIdx.x;
    if (idx >= n * out) return;
    const size_t s = idx / out;
    const int o = static_cast<int>(idx % out);
    float z = b[o];
    const float* x = X + s * in;
    const float* w = W + static_cast<size_t>(o) * in;
    for (int i = 0; i < in; ++i) z = fmaf(w[i], x[i], z);
    Z[idx] = z;
    if (A) A[idx] = z > 0.f ? z : 0.f;
}

// dy = 2 (y - t) / n and the per-sample squared error.
__global__ void k_loss_delta(const float* __restrict__ y, const float* __restrict__ t, size_t n,
                             float* __restrict__ dy, float* __restrict__ sq) {
    const size_t s = static_cast<size_t>(blockIdx.x) * blockDim.x + threadIdx.x;
    if (s >= n) return;
    const float e = y[s] - t[s];
    dy[s] = 2.f * e / static_cast<float>(n);
    sq[s] = e * e;
}

// out[0] = mean of v[0..n-1] (one CTA, fixed order).
__global__ void k_mean(const float* __restrict__ v, size_t n, float* __restrict__ out) {
    __shared__ double sh[256];
    double a = 0.0;
    for (size_t i = threadIdx.x; i < n; i += blockDim.x) a += v[i];
    sh[threadIdx.x] = a;
    __syncthreads();
    for (int st = blockDim.x >> 1; st > 0; st >>= 1) {
        if (static_cast<int>(threadIdx.x) < st) sh[threadIdx.x] += sh[threadIdx.x + st];
        __syncthreads();
    }
    if (threadIdx.x == 0) *out = static_cast<float>(sh[0] / static_cast<double>(n));
}

// dprev[s][i] = (sum_o dnext[s][o] W[o][i]) * (zprev[s][i] > 0)
__global__ void k_backprop(const float* __restrict__ dnext, int out, const float* __restrict__ W, int in,
                           const float* __restrict__ zprev, size_t n, float* __restrict__ dprev) {
    const size_t idx = static_cast<size_t>(blockIdx.x) * blockDim.x + threadIdx.x;
    if (idx >= n * in) return;
    const size_t s = idx / in;
    const int i = static_cast<int>(idx % in);
    float a = 0.f;
    for (int o = 0; o < out; ++o) a = fmaf(dnext[s * out + o], W[static_cast<size_t>(o) * in + i], a);
    dprev[idx] = zprev[idx] > 0.f ? a : 0.f;
}

// dW[o][i] = sum_s delta[s][o] act[s][i];  db[o] = sum_s delta[s][o]
// (one thread per (o, i) plus one per o for the bias; fixed summation order).
__global__ void k_weight_grad(const float* __restrict__ delta, int out, const float* __restrict__ act, int in,
                              size_t n, float* __restrict__ dW, float* __restrict__ db) {
    const int idx = blockIdx.x * blockDim.x + threadIdx.x;
    if (idx >= out * (in + 1)) return;
    const int o = idx / (in + 1), i = idx % (in + 1);
    float a = 0.f;
    if (i < in) {
        for (size_t s = 0; s < n; ++s) a = fmaf(delta[s * out + o], act[s * in + i], a);
        dW[static_cast<size_t>(o) * in + i] = a;
    } else {
        for (size_t s = 0; s < n; ++s) a += delta[s * out + o];
        db[o] = a;
    }
}

// Adam: m = b1 m + (1-b1) g; v = b2 v + (1-b2) g^2;
// p -= lr * (m / c1) / (sqrt(v / c2) + eps), with c1 = 1 - b1^t, c2 = 1 - b2^t.
// With wd > 0 the gradient of the L2 penalty (wd / 2) |p|^2 is added first.
__global__ void k_adam(float* __restrict__ p, const float* __restrict__ g, float* __restrict__ m,
                       float* __restrict__ v, size_t count, float lr, float b1, float b2, float eps, float c1,
                       float c2, float wd) {
    const size_t i = static_cast<size_t>(blockIdx.x) * blockDim.x + threadIdx.x;
    if (i >= count) return;
    const float gi = g[i] + wd * p[i];
    const float mi = b1 * m[i] + (1.f - b1) * gi;
    const float vi = b2 * v[i] + (1.f - b2) * gi * gi;
    m[i] = mi;
    v[i] = vi;
    p[i] -= lr * (mi / c1) / (sqrtf(vi / c2) + eps);
}

inline unsigned blocks_for(size_t work, int threads) {
    return static_cast<unsigned>((work + threads - 1) / threads);
}

// Workspace per sample: z1, a1, z2, a2 (4 x 64), y, dy, sq (3), d2, d1 (2 x 64)
constexpr size_t kWsPerSample = 6 * H + 3;

struct Ws {
    float *z1, *a1, *z2, *a2, *y, *dy, *sq, *d2, *d1;
};
Ws carve(float* base, size_t n) {
    Ws w;
    w.z1 = base;
    w.a1 = w.z1 + n * H;
    w.z2 = w.a1 + n * H;
    w.a2 = w.z2 + n * H;
    w.y = w.a2 + n * H;
    w.dy = w.y + n;
    w.sq = w.dy + n;
    w.d2 = w.sq + n;
    w.d1 = w.d2 + n * H;
    return w;
}

cudaError_t forward(const float* P, const float* X, size_t n, const Ws& w, float* y, cudaStream_t st) {
    const int T = 256;
    k_dense<<<blocks_for(n * H, T), T, 0, st>>>(X, IN, P + OFF_W1, P + OFF_B1, H, n, w.z1, w.a1);
    k_dense<<<blocks_for(n * H, T), T, 0, st>>>(w.a1, H, P + OFF_W2, P + OFF_B2, H, n, w.z2, w.a2);
    k_dense<<<blocks_for(n, T), T, 0, st>>>(w.a2, H, P + OFF_W3, P + OFF_B3, 1, n, y, nullptr);
    return cudaGetLastError();
}

cudaError_t loss_grad(const float* P, const float* X, const float* t, size_t n, const Ws& w, float* G, float* loss,
                      cudaStream_t st) {
    const int T = 256;
    cudaError_t e = forward(P, X, n, w, w.y, st);
    if (e != cudaSuccess) return e;
    k_loss_delta<<<blocks_for(n, T), T, 0, st>>>(w.y, t, n, w.dy, w.sq);
    if (loss) k_mean<<<1, 256, 0, st>>>(w.sq, n, loss);
    // layer 3: dW3 = dy^T a2, db3 = sum dy
    k_weight_grad<<<blocks_for(1 * (H + 1), T), T, 0, st>>>(w.dy, 1, w.a2, H, n, G + OFF_W3, G + OFF_B3);
    // d2 = (dy W3) * (z2 > 0)
    k_backprop<<<blocks_for(n * H, T), T, 0, st>>>(w.dy, 1, P + OFF_W3, H, w.z2, n, w.d2);
    k_weight_grad<<<blocks_for(H * (H + 1), T), T, 0, st>>>(w.d2, H, w.a1, H, n, G + OFF_W2, G + OFF_B2);
    // d1 = (d2 W2) * (z1 > 0)
    k_backprop<<<blocks_for(n * H, T), T, 0, st>>>(w.d2, H, P + OFF_W2, H, w.z1, n, w.d1);
    k_weight_grad<<<blocks_for(H * (IN + 1), T), T, 0, st>>>(w.d1, H, X, IN, n, G + OFF_W1, G + OFF_B1);
    return cudaGetLastError();
}

// splitmix64 (Steele, Lea & Flood 2014) for initialisation and shuffling.
uint64_t splitmix(uint64_t& s) {
    uint64_t z = (s += 0x9E3779B97F4A7C15ull);
    z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
    z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
    return z ^ (z >> 31);
}
double uniform01(uint64_t& s) { return static_cast<double>(splitmix(s) >> 11) * (1.0 / 9007199254740992.0); }

}  // namespace

}  // namespace qsa

using namespace qsa;

extern "C" {

size_t qsa_mlp_workspace_bytes(size_t n) { return sizeof(float) * kWsPerSample * n; }

qsa_status qsa_mlp_forward(const float* params_dev, const float* X_dev, size_t n, float* y_dev, float* workspace_dev,
                           void* stream) {
    if (!params_dev || !X_dev || !y_dev || !workspace_dev || n == 0) return fail(QSA_E_ARG, "NULL argument or n = 0");
    Ws w = carve(workspace_dev, n);
    cudaError_t e = forward(params_dev, X_dev, n, w, y_dev, static_cast<cudaStream_t>(stream));
    if (e != cudaSuccess) return fail(QSA_E_CUDA, std::string("mlp forward: ") + cudaGetErrorString(e));
    return QSA_OK;
}

qsa_status qsa_mlp_loss_grad(const float* params_dev, const float* X_dev, const float* t_dev, size_t n,
                             float* grads_dev, float* loss_dev, float* workspace_dev, void* stream) {
    if (!params_dev || !X_dev || !t_dev || !grads_dev || !workspace_dev || n == 0)
        return fail(QSA_E_ARG, "NULL argument or n = 0");
    Ws w = carve(workspace_dev, n);
    cudaError_t e = loss_grad(params_dev, X_dev, t_dev, n, w, grads_dev, loss_dev, static_cast<cudaStream_t>(stream));
    if (e != cudaSuccess) return fail(QSA_E_CUDA, std::string("mlp backward: ") + cudaGetErrorString(e));
    return QSA_OK;
}

qsa_status qsa_mlp_adam_step(float* params_dev, const float* grads_dev, float* m_dev, float* v_dev, size_t count,
                             int step, float lr, float beta1, float beta2, float eps, void* stream) {
    if (!params_dev || !grads_dev || !m_dev || !v_dev || step < 1) return fail(QSA_E_ARG, "bad Adam arguments");
    const float c1 = static_cast<float>(1.0 - std::pow(static_cast<double>(beta1), step));
    const float c2 = static_cast<float>(1.0 - std::pow(static_cast<double>(beta2), step));
    k_adam<<<blocks_for(count, 256), 256, 0, static_cast<cudaStream_t>(stream)>>>(params_dev, grads_dev, m_dev, v_dev,
                                                                                  count, lr, beta1, beta2, eps, c1, c2,
                                                                                  0.f);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return fail(QSA_E_CUDA, std::string("adam: ") + cudaGetErrorString(e));
    return QSA_OK;
}

qsa_status qsa_costmodel_init(uint64_t seed, float* params_host) {
    if (!params_host) return fail(QSA_E_ARG, "NULL argument");
    // He-uniform weights: U(-sqrt(6/fan_in), +sqrt(6/fan_in)); zero biases.
    uint64_t s = seed ^ 0x5DEECE66Dull;
    std::memset(params_host, 0, sizeof(float) * kMlpParams);
    auto fill = [&](int off, int count, int fan_in) {
        const double a = std::sqrt(6.0 / fan_in);
        for (int i = 0; i < count; ++i) params_host[off + i] = static_cast<float>((2.0 * uniform01(s) - 1.0) * a);
    };
    fill(OFF_W1, H * IN, IN);
    fill(OFF_W2, H * H, H);
    fill(OFF_W3, H, H);
    return QSA_OK;
}

qsa_status qsa_costmodel_train(const float* X_host, const float* y_host, size_t n, int epochs, int batch, float lr,
                               float weight_decay, uint64_t seed, float* params_inout_host, float* epoch_loss_host) {
    if (!X_host || !y_host || !params_inout_host || n == 0 || epochs < 1 || batch < 1 || weight_decay < 0.f)
        return fail(QSA_E_ARG, "bad training arguments");
    // Standardise the targets (log-seconds sit far from the network's initial
    // output): train on (y - mu) / sigma with the output layer rescaled to
    // match, then fold mu and sigma back into W3 and b3.
    double mu = 0.0, var = 0.0;
    for (size_t i = 0; i < n; ++i) mu += y_host[i];
    mu /= static_cast<double>(n);
    for (size_t i = 0; i < n; ++i) var += (y_host[i] - mu) * (y_host[i] - mu);
    const double sigma = std::max(1e-6, std::sqrt(var / static_cast<double>(n)));
    std::vector<float> yn(n);
    for (size_t i = 0; i < n; ++i) yn[i] = static_cast<float>((y_host[i] - mu) / sigma);
    for (int j = 0; j < H; ++j) params_inout_host[OFF_W3 + j] = static_cast<float>(params_inout_host[OFF_W3 + j] / sigma);
    params_inout_host[OFF_B3] = static_cast<float>((params_inout_host[OFF_B3] - mu) / sigma);
    y_host = yn.data();
    const size_t bsz = std::min<size_t>(static_cast<size_t>(batch), n);
    float *dX = nullptr, *dY = nullptr, *dP = nullptr, *dG = nullptr, *dM = nullptr, *dV = nullptr, *dWs = nullptr,
          *dLoss = nullptr, *dXb = nullptr, *dYb = nullptr, *dOut = nullptr;
    const size_t np = kMlpParams;
    cudaStream_t st = nullptr;
    cudaError_t e = cudaStreamCreateWithFlags(&st, cudaStreamNonBlocking);
    auto A = [&](float** p, size_t cnt) {
        if (e == cudaSuccess) e = dev_malloc(p, sizeof(float) * cnt);
    };
    A(&dX, n * IN);
    A(&dY, n);
    A(&dP, np);
    A(&dG, np);
    A(&dM, np);
    A(&dV, np);
    A(&dWs, kWsPerSample * n);
    A(&dLoss, 1);
    A(&dXb, bsz * IN);
    A(&dYb, bsz);
    A(&dOut, n);
    if (e == cudaSuccess) e = cudaMemcpyAsync(dX, X_host, sizeof(float) * n * IN, cudaMemcpyHostToDevice, st);
    if (e == cudaSuccess) e = cudaMemcpyAsync(dY, y_host, sizeof(float) * n, cudaMemcpyHostToDevice, st);
    if (e == cudaSuccess) e = cudaMemcpyAsync(dP, params_inout_host, sizeof(float) * np, cudaMemcpyHostToDevice, st);
    if (e == cudaSuccess) e = cudaMemsetAsync(dM, 0, sizeof(float) * np, st);
    if (e == cudaSuccess) e = cudaMemsetAsync(dV, 0, sizeof(float) * np, st);
    std::vector<size_t> order(n);
    std::iota(order.begin(), order.end(), size_t(0));
    std::vector<float> xb(bsz * IN), yb(bsz);
    uint64_t rs = seed;
    int step = 0;
    for (int ep = 0; ep < epochs && e == cudaSuccess; ++ep) {
        for (size_t i = n; i > 1; --i) std::swap(order[i - 1], order[splitmix(rs) % i]);  // Fisher-Yates
        for (size_t b0 = 0; b0 + bsz <= n && e == cudaSuccess; b0 += bsz) {
            for (size_t r = 0; r < bsz; ++r) {
                std::memcpy(&xb[r * IN], X_host + order[b0 + r] * IN, sizeof(float) * IN);
                yb[r] = y_host[order[b0 + r]];
            }
            e = cudaMemcpyAsync(dXb, xb.data(), sizeof(float) * bsz * IN, cudaMemcpyHostToDevice, st);
            if (e == cudaSuccess) e = cudaMemcpyAsync(dYb, yb.data(), sizeof(float) * bsz, cudaMemcpyHostToDevice, st);
            if (e == cudaSuccess) e = loss_grad(dP, dXb, dYb, bsz, carve(dWs, bsz), dG, nullptr, st);
            ++step;
            if (e == cudaSuccess) {
                const float c1 = static_cast<float>(1.0 - std::pow(0.9, step));
                const float c2 = static_cast<float>(1.0 - std::pow(0.999, step));
                k_adam<<<blocks_for(np, 256), 256, 0, st>>>(dP, dG, dM, dV, np, lr, 0.9f, 0.999f, 1e-8f, c1, c2,
                                                            weight_decay);
                e = cudaGetLastError();
            }
            // the pageable staging vectors are reused: wait for the copies
            if (e == cudaSuccess) e = cudaStreamSynchronize(st);
        }
        if (epoch_loss_host && e == cudaSuccess) {
            Ws w = carve(dWs, n);
            e = forward(dP, dX, n, w, dOut, st);
            if (e == cudaSuccess) {
                k_loss_delta<<<blocks_for(n, 256), 256, 0, st>>>(dOut, dY, n, w.dy, w.sq);
                k_mean<<<1, 256, 0, st>>>(w.sq, n, dLoss);
                e = cudaMemcpyAsync(&epoch_loss_host[ep], dLoss, sizeof(float), cudaMemcpyDeviceToHost, st);
            }
        }
    }
    if (e == cudaSuccess) e = cudaMemcpyAsync(params_inout_host, dP, sizeof(float) * np, cudaMemcpyDeviceToHost, st);
    if (e == cudaSuccess) e = cudaStreamSynchronize(st);
    for (float* p : {dX, dY, dP, dG, dM, dV, dWs, dLoss, dXb, dYb, dOut})
        if (p) dev_free(p);
    if (st) cudaStreamDestroy(st);
    // fold the standardisation back into the output layer (also on failure,
    // so the caller's parameters keep their meaning)
    for (int j = 0; j < H; ++j) params_inout_host[OFF_W3 + j] = static_cast<float>(params_inout_host[OFF_W3 + j] * sigma);
    params_inout_host[OFF_B3] = static_cast<float>(params_inout_host[OFF_B3] * sigma + mu);
    if (epoch_loss_host)
        for (int ep = 0; ep < epochs; ++ep) epoch_loss_host[ep] = static_cast<float>(epoch_loss_host[ep] * sigma * sigma);
    if (e != cudaSuccess) return fail(QSA_E_CUDA, std::string("cost-model training: ") + cudaGetErrorString(e));
    return QSA_OK;
}

// Time one fused-operator pass for n_samples random (k, physical targets)
// on the state (identity matrices, so the amplitudes are unchanged) and
// return the features and log(median seconds over reps launches).
qsa_status qsa_costmodel_collect(qsa_state s, size_t n_samples, int reps, int precision, uint64_t seed,
                                 float* X_host, float* y_host) {
    qsa_status stt = check_state(s);
    if (stt != QSA_OK) return stt;
    if (!X_host || !y_host || reps < 1 || precision < 0 || precision > 1) return fail(QSA_E_ARG, "bad arguments");
    const int n = s->n;
    const int kmax = std::min(QSA_MAX_K, n);
    // identity matrices for k = 1..kmax, uploaded once
    std::vector<float> hm;
    std::vector<size_t> off(kmax + 1, 0);
    for (int k = 1; k <= kmax; ++k) {
        off[k] = hm.size();
        const size_t D = size_t(1) << k;
        hm.resize(hm.size() + 2 * D * D, 0.f);
        for (size_t i = 0; i < D; ++i) hm[off[k] + 2 * (i * D + i)] = 1.f;
        while (hm.size() % 4) hm.push_back(0.f);
    }
    stt = ensure_dev(s, reinterpret_cast<void**>(&s->d_mat), &s->mat_cap, hm.size() * sizeof(float));
    if (stt != QSA_OK) return stt;
    cudaError_t e = cudaMemcpyAsync(s->d_mat, hm.data(), hm.size() * sizeof(float), cudaMemcpyHostToDevice, s->stream);
    if (e != cudaSuccess) return cuda_fail(s, e, "collect upload");
    cudaEvent_t a, b;
    cudaEventCreate(&a);
    cudaEventCreate(&b);
    uint64_t rs = seed;
    std::vector<float> t(reps);
    for (size_t i = 0; i < n_samples; ++i) {
        const int k = 1 + static_cast<int>(splitmix(rs) % static_cast<uint64_t>(kmax));
        int perm[QSA_MAX_QUBITS];
        for (int q = 0; q < n; ++q) perm[q] = q;
        for (int q = n; q > 1; --q) std::swap(perm[q - 1], perm[splitmix(rs) % static_cast<uint64_t>(q)]);
        int phys[QSA_MAX_K];
        uint64_t mask = 0;
        for (int j = 0; j < k; ++j) {
            phys[j] = perm[j];
            mask |= 1ull << perm[j];
        }
        for (int r = 0; r < reps && e == cudaSuccess; ++r) {
            cudaEventRecord(a, s->stream);
            stt = apply_physical(s, phys, k, s->d_mat + off[k], precision, nullptr);
            if (stt != QSA_OK) break;
            cudaEventRecord(b, s->stream);
            e = cudaEventSynchronize(b);
            float ms = 0.f;
            if (e == cudaSuccess) e = cudaEventElapsedTime(&ms, a, b);
            t[r] = ms;
        }
        if (stt != QSA_OK || e != cudaSuccess) break;
        std::sort(t.begin(), t.end());
        costmodel_features(k, mask, n, 1, X_host + i * kMlpIn);
        y_host[i] = static_cast<float>(std::log(std::max(1e-9, t[reps / 2] * 1e-3)));
    }
    cudaEventDestroy(a);
    cudaEventDestroy(b);
    if (stt != QSA_OK) return stt;
    if (e != cudaSuccess) return cuda_fail(s, e, "collect timing");
    return sync_and_check(s, "collect");
}

}  // extern "C"
