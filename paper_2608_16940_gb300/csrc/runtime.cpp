// Host runtime behind the C ABI in include/qsa.h: state objects, the layout
// map, lowering dispatch, circuit execution and output reductions.
//
// Layout map (§II, Theorem 1): L[q] = physical position of logical qubit q.
// The stored amplitude at y equals the logical amplitude at x with
// x_q = y_{L(q)}.  Every physical permutation composes L with the same
// transpositions (Lemma "distributed promotion swap"), so consumers decode
// through L instead of restoring canonical order (§IV-D).
#include <cuda_runtime.h>

#include <algorithm>
#include <atomic>
#include <cstdio>
#include <cstdlib>
#include <cstring>
#include <string>
#include <vector>

#include "qsa.h"
#include "qsa_internal.h"
#include "qsa_runtime.h"

namespace {
thread_local std::string g_err;

// Allocations to go before an injected failure (-1: none) and the number of
// device allocations the library holds.
std::atomic<int64_t> g_alloc_fail_in{-1};
std::atomic<int64_t> g_live_allocs{0};
// QSA_FAULT_ALLOC=<n> at load time: the n-th device allocation (0 = the
// first) fails.
struct FaultEnv {
    FaultEnv() {
        if (const char* v = std::getenv("QSA_FAULT_ALLOC")) g_alloc_fail_in.store(std::atoll(v));
    }
} g_fault_env;
}  // namespace

namespace qsa {

cudaError_t dev_malloc_raw(void** p, size_t bytes) {
    int64_t left = g_alloc_fail_in.load();
    while (left >= 0 && !g_alloc_fail_in.compare_exchange_weak(left, left - 1)) {
    }
    if (left == 0) {   // the injected failure: nothing is allocated
        *p = nullptr;
        return cudaErrorMemoryAllocation;
    }
    cudaError_t e = cudaMalloc(p, bytes);
    if (e == cudaSuccess) g_live_allocs.fetch_add(1);
    return e;
}

void dev_free(void* p) {
    if (!p) return;
    cudaFree(p);
    g_live_allocs.fetch_sub(1);
}

qsa_status fail(qsa_status st, const std::string& msg) {
    g_err = msg;
    return st;
}

qsa_status cuda_fail(qsa_state s, cudaError_t e, const char* where) {
    if (s) s->failed = true;
    return fail(QSA_E_CUDA, std::string(where) + ": " + cudaGetErrorString(e));
}

// Synchronise the state's stream and report a device-side give-up recorded
// in the error word by a bounded wait (QSA_E_TIMEOUT; the state is then failed).
qsa_status sync_and_check(qsa_state s, const char* where) {
    int h[4] = {0, 0, 0, 0};
    cudaError_t e = cudaMemcpyAsync(h, s->d_err, sizeof(h), cudaMemcpyDeviceToHost, s->stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(s->stream);
    if (e != cudaSuccess) return cuda_fail(s, e, where);
    if (h[0] != 0) {
        s->failed = true;
        return fail(QSA_E_TIMEOUT, std::string(where) + ": a kernel gave up a bounded wait (code " +
                                       std::to_string(h[0]) + ", work item " + std::to_string(h[1]) + ", block " +
                                       std::to_string(h[2]) + "); the amplitudes are invalid");
    }
    return QSA_OK;
}

qsa_status check_state(qsa_state s) {
    if (!s) return fail(QSA_E_ARG, "state is NULL");
    if (s->failed) return fail(QSA_E_STATE, "state is marked failed after a CUDA error");
    return QSA_OK;
}

qsa_status ensure_dev(qsa_state s, void** ptr, size_t* cap, size_t bytes) {
    if (*cap >= bytes && *ptr) return QSA_OK;
    if (*ptr) {
        cudaStreamSynchronize(s->stream);
        dev_free(*ptr);
        *ptr = nullptr;
        *cap = 0;
    }
    size_t want = std::max<size_t>(bytes, 4096);
    cudaError_t e = dev_malloc(ptr, want);
    if (e != cudaSuccess) {
        cudaGetLastError();
        *ptr = nullptr;
        return fail(QSA_E_NOMEM, std::string("cudaMalloc of scratch failed: ") + cudaGetErrorString(e));
    }
    *cap = want;
    return QSA_OK;
}

void to_float_matrix(const double* m, int k, float* out) {
    const size_t cnt = 2ull << (2 * k);
    for (size_t i = 0; i < cnt; ++i) out[i] = static_cast<float>(m[i]);
}

qsa_status validate_targets(int n, const int32_t* targets, int k, int kmax) {
    if (!targets) return fail(QSA_E_ARG, "targets is NULL");
    if (k < 1 || k > kmax) return fail(QSA_E_ARG, "k must be in 1.." + std::to_string(kmax));
    if (k > n) return fail(QSA_E_ARG, "k exceeds the number of qubits");
    uint64_t seen = 0;
    for (int j = 0; j < k; ++j) {
        if (targets[j] < 0 || targets[j] >= n) return fail(QSA_E_ARG, "target out of range");
        if (seen & (1ull << targets[j])) return fail(QSA_E_ARG, "repeated target");
        seen |= 1ull << targets[j];
    }
    return QSA_OK;
}

// Swap physical positions pairs (pa[i], pb[i]) in data and layout.
qsa_status permute_positions(qsa_state s, const int* pa, const int* pb, int np, qsa_run_stats* rs) {
    if (np == 0) return QSA_OK;
    Timer tm(s, rs ? &rs->permute_seconds : nullptr);
    cudaError_t e = launch_permute(s->psi, s->n, pa, pb, np, s->stream, &s->launches);
    tm.stop();
    if (e != cudaSuccess) return cuda_fail(s, e, "permute kernel");
    int inv[64];
    for (int q = 0; q < s->n; ++q) inv[s->L[q]] = q;
    for (int i = 0; i < np; ++i) {
        int qa = inv[pa[i]], qb = inv[pb[i]];
        s->L[qa] = pb[i];
        s->L[qb] = pa[i];
        inv[pa[i]] = qb;
        inv[pb[i]] = qa;
    }
    if (rs) {
        rs->permutes += 1;
        rs->passes += 1;
        rs->hbm_bytes += 16.0 * static_cast<double>(1ull << s->n);
    }
    return QSA_OK;
}

// Promote targets outside the in-block bits (positions >= inblock) to the
// lowest free in-block positions (first-free victim choice, §IV-D), updating
// phys[] to the new positions.
int choose_promotions(const int32_t* L, int n, int* phys, int k, int frames, int victim, const int32_t* next_use,
                      int* pa, int* pb) {
    int inv[QSA_MAX_QUBITS];
    for (int q = 0; q < n; ++q) inv[L[q]] = q;
    uint64_t pinned = 0;
    for (int j = 0; j < k; ++j)
        if (phys[j] < frames) pinned |= 1ull << phys[j];
    int np = 0;
    for (int j = 0; j < k; ++j) {
        if (phys[j] < frames) continue;
        int v = -1;
        int64_t best = -1;
        for (int f = 0; f < frames; ++f) {
            if ((pinned >> f) & 1) continue;
            if (victim != QSA_VICTIM_FARTHEST) {
                v = f;
                break;
            }
            const int64_t key = next_use[inv[f]];
            if (key > best) {   // strict: ties keep the lowest frame
                best = key;
                v = f;
            }
        }
        if (v < 0) return -1;
        const int hp = phys[j], qv = inv[v], qt = inv[hp];
        pa[np] = hp;
        pb[np] = v;
        ++np;
        inv[v] = qt;
        inv[hp] = qv;
        pinned |= 1ull << v;
        phys[j] = v;
    }
    return np;
}

qsa_status promote_targets(qsa_state s, int* phys, int k, int inblock, qsa_run_stats* rs) {
    int pa[QSA_MAX_K], pb[QSA_MAX_K];
    const int np = choose_promotions(s->L, s->n, phys, k, std::min(inblock, s->n), QSA_VICTIM_FIRST_FREE, nullptr,
                                     pa, pb);
    if (np < 0) return fail(QSA_E_ARG, "not enough free in-block positions");
    return permute_positions(s, pa, pb, np, rs);
}

qsa_status apply_physical(qsa_state s, const int* phys, int k, const float* d_mat, int precision,
                          qsa_run_stats* rs) {
    cudaError_t e;
    bool tc = precision == QSA_PREC_TF32X3 && (k == 5 || k == 6) && tc_available(s, k);
    {
        Timer tm(s, rs ? (tc ? &rs->tc_seconds : &rs->apply_seconds) : nullptr);
        if (tc)
            e = launch_apply_tc(s->psi, s->n, phys, k, d_mat, s->d_err, s->stream, &s->launches);
        else
            e = launch_apply_fp32(s->psi, s->n, phys, k, d_mat, s->stream, &s->launches);
        tm.stop();
    }
    if (e != cudaSuccess) return cuda_fail(s, e, tc ? "tensor-core apply kernel" : "apply kernel");
    s->known_zero = false;
    if (rs) {
        rs->blocks += 1;
        rs->passes += 1;
        rs->tc_blocks += tc ? 1 : 0;
        rs->hbm_bytes += 16.0 * static_cast<double>(1ull << s->n);
    }
    return QSA_OK;
}

qsa_status apply_logical(qsa_state s, const int32_t* targets, int k, const float* d_mat, int lowering,
                         int precision, qsa_run_stats* rs) {
    int phys[6];
    for (int j = 0; j < k; ++j) phys[j] = s->L[targets[j]];
    if (lowering == QSA_LOWER_PERMUTE) {
        qsa_status st = promote_targets(s, phys, k, kInBlockBits, rs);
        if (st != QSA_OK) return st;
    }
    return apply_physical(s, phys, k, d_mat, precision, rs);
}

qsa_status apply_diag_logical(qsa_state s, const int32_t* targets, int k, const float* d_tab, qsa_run_stats* rs) {
    int phys[QSA_MAX_DIAG];
    for (int j = 0; j < k; ++j) phys[j] = s->L[targets[j]];
    cudaError_t e;
    {
        Timer tm(s, rs ? &rs->diag_seconds : nullptr);
        e = launch_apply_diag(s->psi, s->n, phys, k, d_tab, s->stream, &s->launches);
        tm.stop();
    }
    if (e != cudaSuccess) return cuda_fail(s, e, "diagonal kernel");
    s->known_zero = false;
    if (rs) {
        rs->blocks += 1;
        rs->passes += 1;
        rs->diag_blocks += 1;
        rs->hbm_bytes += 16.0 * static_cast<double>(1ull << s->n);
    }
    return QSA_OK;
}

qsa_status apply_prod_logical(qsa_state s, const int32_t* targets, int k, const float* d_fac, qsa_run_stats* rs) {
    int phys[QSA_MAX_PROD];
    for (int j = 0; j < k; ++j) phys[j] = s->L[targets[j]];
    const uint64_t l0 = s->launches;
    cudaError_t e;
    {
        Timer tm(s, rs ? &rs->prod_seconds : nullptr);
        e = launch_apply_prod(s->psi, s->n, phys, k, d_fac, s->stream, &s->launches);
        tm.stop();
    }
    if (e != cudaSuccess) return cuda_fail(s, e, "product kernel");
    s->known_zero = false;
    if (rs) {
        const uint64_t passes = s->launches - l0;
        rs->blocks += 1;
        rs->passes += passes;
        rs->prod_blocks += 1;
        rs->hbm_bytes += 16.0 * static_cast<double>(1ull << s->n) * static_cast<double>(passes);
    }
    return QSA_OK;
}

// ---- timers ------------------------------------------------------------------
Timer::Timer(qsa_state s, double* acc) : s_(s), acc_(s->timing ? acc : nullptr) {
    if (!acc_) return;
    if (s_->ev_free.empty()) {
        cudaEvent_t a, b;
        cudaEventCreate(&a);
        cudaEventCreate(&b);
        ev_[0] = a;
        ev_[1] = b;
    } else {
        auto p = s_->ev_free.back();
        s_->ev_free.pop_back();
        ev_[0] = p.first;
        ev_[1] = p.second;
    }
    cudaEventRecord(ev_[0], s_->stream);
}

void Timer::stop() {
    if (!acc_ || stopped_) return;
    stopped_ = true;
    cudaEventRecord(ev_[1], s_->stream);
    s_->ev_pending.push_back({ev_[0], ev_[1], acc_});
}

Timer::~Timer() { stop(); }

void collect_timers(qsa_state s, double* total) {
    if (s->ev_pending.empty()) return;
    cudaStreamSynchronize(s->stream);
    for (auto& p : s->ev_pending) {
        float ms = 0.f;
        cudaEventElapsedTime(&ms, p.a, p.b);
        *p.acc += ms * 1e-3;
        if (total) *total += ms * 1e-3;
        s->ev_free.push_back({p.a, p.b});
    }
    s->ev_pending.clear();
}

}  // namespace qsa

using namespace qsa;

extern "C" {

qsa_status qsa_debug_fail_alloc(int64_t nth) {
    g_alloc_fail_in.store(nth < 0 ? -1 : nth);
    return QSA_OK;
}

uint64_t qsa_debug_live_allocations(void) {
    const int64_t v = g_live_allocs.load();
    return v < 0 ? 0 : static_cast<uint64_t>(v);
}

uint64_t qsa_debug_bounds_status(void) {
    for (uint64_t w : {bounds_word_apply(), bounds_word_layer(), bounds_word_tc()})
        if (w) return w;
    return 0;
}

int qsa_debug_bounds_enabled(void) {
#ifdef QSA_DEBUG_BOUNDS
    return 1;
#else
    return 0;
#endif
}

const char* qsa_last_error(void) { return g_err.c_str(); }

qsa_status qsa_state_create_ex(int n_qubits, qsa_dtype dtype, void* dev_buf, size_t bytes, void* cuda_stream,
                               int init_zero, qsa_state* out) {
    if (!out) return fail(QSA_E_ARG, "out is NULL");
    *out = nullptr;
    if (dtype == QSA_C128) return fail(QSA_E_UNSUPPORTED, "complex128 states are not implemented");
    if (dtype != QSA_C64) return fail(QSA_E_ARG, "unknown dtype");
    if (n_qubits < 1 || n_qubits > QSA_MAX_QUBITS) return fail(QSA_E_ARG, "n_qubits must be in 1..34");
    const size_t need = sizeof(float2) << n_qubits;
    auto* s = new qsa_state_s();
    s->n = n_qubits;
    s->stream = static_cast<cudaStream_t>(cuda_stream);
    for (int q = 0; q < n_qubits; ++q) s->L[q] = q;
    if (dev_buf) {
        if (bytes < need) {
            delete s;
            return fail(QSA_E_ARG, "device buffer smaller than 8 * 2^N bytes");
        }
        if (reinterpret_cast<uintptr_t>(dev_buf) % 16) {
            delete s;
            return fail(QSA_E_ARG, "device buffer must be 16-byte aligned");
        }
        s->psi = static_cast<float2*>(dev_buf);
        s->owned = false;
    } else {
        void* p = nullptr;
        cudaError_t e = dev_malloc(&p, need);
        if (e != cudaSuccess) {
            cudaGetLastError();
            delete s;
            return fail(QSA_E_NOMEM, std::string("cudaMalloc of the state failed: ") + cudaGetErrorString(e));
        }
        s->psi = static_cast<float2*>(p);
        s->owned = true;
        init_zero = 1;
    }
    auto discard = [&]() {
        if (s->owned) dev_free(s->psi);
        dev_free(s->d_err);
        delete s;
    };
    cudaError_t e = dev_malloc(&s->d_err, sizeof(int) * 4);
    if (e != cudaSuccess) {
        cudaGetLastError();
        discard();
        return fail(QSA_E_NOMEM, std::string("cudaMalloc of the error word failed: ") + cudaGetErrorString(e));
    }
    e = cudaMemsetAsync(s->d_err, 0, sizeof(int) * 4, s->stream);
    if (e != cudaSuccess) {
        qsa_status st = cuda_fail(s, e, "error word");
        discard();
        return st;
    }
    if (init_zero) {
        e = launch_init_zero(s->psi, s->n, s->stream, &s->launches);
        if (e != cudaSuccess) {
            qsa_status st = cuda_fail(s, e, "init");
            discard();
            return st;
        }
        s->known_zero = true;
    }
    *out = s;
    return QSA_OK;
}

qsa_status qsa_state_create(int n_qubits, qsa_dtype dtype, qsa_state* out) {
    return qsa_state_create_ex(n_qubits, dtype, nullptr, 0, nullptr, 1, out);
}

qsa_status qsa_state_destroy(qsa_state s) {
    if (!s) return fail(QSA_E_ARG, "state is NULL");
    cudaStreamSynchronize(s->stream);
    cudaGetLastError();
    if (s->owned && s->psi) dev_free(s->psi);
    if (s->d_mat) dev_free(s->d_mat);
    if (s->d_red) dev_free(s->d_red);
    if (s->d_dm) dev_free(s->d_dm);
    if (s->d_lrec) dev_free(s->d_lrec);
    if (s->d_samp) dev_free(s->d_samp);
    if (s->d_err) dev_free(s->d_err);
    if (s->d_mlp) dev_free(s->d_mlp);
    for (auto& p : s->ev_free) {
        cudaEventDestroy(p.first);
        cudaEventDestroy(p.second);
    }
    for (auto& p : s->ev_pending) {
        cudaEventDestroy(p.a);
        cudaEventDestroy(p.b);
    }
    delete s;
    return QSA_OK;
}

qsa_status qsa_set_stream(qsa_state s, void* cuda_stream) {
    if (!s) return fail(QSA_E_ARG, "state is NULL");
    s->stream = static_cast<cudaStream_t>(cuda_stream);
    return QSA_OK;
}

qsa_status qsa_state_reset(qsa_state s) {
    if (!s) return fail(QSA_E_ARG, "state is NULL");
    if (s->failed) {
        cudaError_t e = cudaDeviceSynchronize();
        if (e != cudaSuccess) return fail(QSA_E_STATE, "device is not healthy");
        s->failed = false;
    }
    for (int q = 0; q < s->n; ++q) s->L[q] = q;
    cudaError_t e = launch_init_zero(s->psi, s->n, s->stream, &s->launches);
    if (e != cudaSuccess) return cuda_fail(s, e, "reset");
    s->known_zero = true;
    return QSA_OK;
}

qsa_status qsa_state_info(qsa_state s, int* n_qubits, void** dev_amplitudes) {
    if (!s) return fail(QSA_E_ARG, "state is NULL");
    if (n_qubits) *n_qubits = s->n;
    if (dev_amplitudes) *dev_amplitudes = s->psi;
    return QSA_OK;
}

qsa_status qsa_get_layout(qsa_state s, int32_t* phys_of_logical) {
    if (!s || !phys_of_logical) return fail(QSA_E_ARG, "NULL argument");
    for (int q = 0; q < s->n; ++q) phys_of_logical[q] = s->L[q];
    return QSA_OK;
}

qsa_status qsa_set_layout(qsa_state s, const int32_t* phys_of_logical, int materialise) {
    qsa_status st = check_state(s);
    if (st != QSA_OK) return st;
    if (!phys_of_logical) return fail(QSA_E_ARG, "layout is NULL");
    uint64_t seen = 0;
    for (int q = 0; q < s->n; ++q) {
        int p = phys_of_logical[q];
        if (p < 0 || p >= s->n || ((seen >> p) & 1)) return fail(QSA_E_ARG, "layout is not a bijection on 0..N-1");
        seen |= 1ull << p;
    }
    if (!materialise) {
        if (!s->known_zero) return fail(QSA_E_STATE, "metadata-only relabel needs the state |0..0>");
        for (int q = 0; q < s->n; ++q) s->L[q] = phys_of_logical[q];
        return QSA_OK;
    }
    // Passes of disjoint transpositions; each swap puts one logical qubit in
    // its final position.
    for (int guard = 0; guard < 2 * QSA_MAX_QUBITS; ++guard) {
        int pa[QSA_MAX_QUBITS], pb[QSA_MAX_QUBITS], np = 0;
        uint64_t used = 0;
        for (int q = 0; q < s->n; ++q) {
            int a = s->L[q], b = phys_of_logical[q];
            if (a == b || ((used >> a) & 1) || ((used >> b) & 1)) continue;
            used |= (1ull << a) | (1ull << b);
            pa[np] = a;
            pb[np] = b;
            ++np;
        }
        if (np == 0) break;
        for (int i = 0; i < np; i += 6) {
            st = permute_positions(s, pa + i, pb + i, std::min(6, np - i), nullptr);
            if (st != QSA_OK) return st;
        }
    }
    for (int q = 0; q < s->n; ++q)
        if (s->L[q] != phys_of_logical[q]) return fail(QSA_E_STATE, "layout materialisation did not converge");
    return QSA_OK;
}

qsa_status qsa_permute_bits(qsa_state s, const int32_t* phys_a, const int32_t* phys_b, int n_pairs) {
    qsa_status st = check_state(s);
    if (st != QSA_OK) return st;
    if (n_pairs < 0 || (n_pairs > 0 && (!phys_a || !phys_b))) return fail(QSA_E_ARG, "bad pair list");
    uint64_t seen = 0;
    std::vector<int> a(n_pairs), b(n_pairs);
    for (int i = 0; i < n_pairs; ++i) {
        int x = phys_a[i], y = phys_b[i];
        if (x < 0 || x >= s->n || y < 0 || y >= s->n || x == y) return fail(QSA_E_ARG, "bad position");
        if (((seen >> x) & 1) || ((seen >> y) & 1)) return fail(QSA_E_ARG, "positions must be distinct");
        seen |= (1ull << x) | (1ull << y);
        a[i] = x;
        b[i] = y;
    }
    for (int i = 0; i < n_pairs; i += 6) {
        st = permute_positions(s, a.data() + i, b.data() + i, std::min(6, n_pairs - i), nullptr);
        if (st != QSA_OK) return st;
    }
    return QSA_OK;
}

qsa_status qsa_apply_fused_ex(qsa_state s, const int32_t* targets, int k, const double* matrix, int lowering,
                              int precision) {
    qsa_status st = check_state(s);
    if (st != QSA_OK) return st;
    st = validate_targets(s->n, targets, k);
    if (st != QSA_OK) return st;
    if (!matrix) return fail(QSA_E_ARG, "matrix is NULL");
    if (lowering < 0 || lowering > 2) return fail(QSA_E_ARG, "unknown lowering");
    if (precision < 0 || precision > 1) return fail(QSA_E_ARG, "unknown precision");
    const size_t cnt = 2ull << (2 * k);
    std::vector<float> hm(cnt);
    to_float_matrix(matrix, k, hm.data());
    st = ensure_dev(s, reinterpret_cast<void**>(&s->d_mat), &s->mat_cap, cnt * sizeof(float));
    if (st != QSA_OK) return st;
    // pageable source: the copy is staged before the call returns
    cudaError_t e = cudaMemcpyAsync(s->d_mat, hm.data(), cnt * sizeof(float), cudaMemcpyHostToDevice, s->stream);
    if (e != cudaSuccess) return cuda_fail(s, e, "matrix upload");
    return apply_logical(s, targets, k, s->d_mat, lowering, precision, nullptr);
}

qsa_status qsa_apply_fused(qsa_state s, const int32_t* targets, int k, const double* matrix) {
    return qsa_apply_fused_ex(s, targets, k, matrix, QSA_LOWER_AUTO, QSA_PREC_FP32);
}

qsa_status qsa_apply_product(qsa_state s, const int32_t* targets, int k, const double* factors) {
    qsa_status st = check_state(s);
    if (st != QSA_OK) return st;
    st = validate_targets(s->n, targets, k, QSA_MAX_PROD);
    if (st != QSA_OK) return st;
    if (!factors) return fail(QSA_E_ARG, "factors is NULL");
    const size_t cnt = 8ull * k;
    std::vector<float> hf(cnt);
    for (size_t i = 0; i < cnt; ++i) hf[i] = static_cast<float>(factors[i]);
    st = ensure_dev(s, reinterpret_cast<void**>(&s->d_mat), &s->mat_cap, cnt * sizeof(float));
    if (st != QSA_OK) return st;
    // pageable source: the copy is staged before the call returns
    cudaError_t e = cudaMemcpyAsync(s->d_mat, hf.data(), cnt * sizeof(float), cudaMemcpyHostToDevice, s->stream);
    if (e != cudaSuccess) return cuda_fail(s, e, "factor upload");
    return apply_prod_logical(s, targets, k, s->d_mat, nullptr);
}

qsa_status qsa_apply_diag(qsa_state s, const int32_t* targets, int k, const double* diag) {
    qsa_status st = check_state(s);
    if (st != QSA_OK) return st;
    st = validate_targets(s->n, targets, k, QSA_MAX_DIAG);
    if (st != QSA_OK) return st;
    if (!diag) return fail(QSA_E_ARG, "diag is NULL");
    const size_t cnt = 2ull << k;
    std::vector<float> hd(cnt);
    ModulusCarry carry;
    to_float_moduli(diag, cnt / 2, hd.data(), 1.0 / static_cast<double>(cnt / 2), &carry);
    st = ensure_dev(s, reinterpret_cast<void**>(&s->d_mat), &s->mat_cap, cnt * sizeof(float));
    if (st != QSA_OK) return st;
    // pageable source: the copy is staged before the call returns
    cudaError_t e = cudaMemcpyAsync(s->d_mat, hd.data(), cnt * sizeof(float), cudaMemcpyHostToDevice, s->stream);
    if (e != cudaSuccess) return cuda_fail(s, e, "diagonal upload");
    return apply_diag_logical(s, targets, k, s->d_mat, nullptr);
}

qsa_status qsa_expectation_z(qsa_state s, uint64_t logical_mask, double* out) {
    qsa_status st = check_state(s);
    if (st != QSA_OK) return st;
    if (!out) return fail(QSA_E_ARG, "out is NULL");
    if (s->n < 64 && (logical_mask >> s->n)) return fail(QSA_E_ARG, "mask has bits beyond N");
    uint64_t pm = 0;
    for (int q = 0; q < s->n; ++q)
        if ((logical_mask >> q) & 1) pm |= 1ull << s->L[q];
    st = ensure_dev(s, reinterpret_cast<void**>(&s->d_red), &s->red_cap, sizeof(double) * (reduce_partials() + 8));
    if (st != QSA_OK) return st;
    double* d_out = s->d_red + reduce_partials();
    cudaError_t e = launch_reduce_z(s->psi, s->n, pm, s->d_red, d_out, s->stream, &s->launches);
    if (e != cudaSuccess) return cuda_fail(s, e, "reduction kernel");
    e = cudaMemcpyAsync(out, d_out, sizeof(double), cudaMemcpyDeviceToHost, s->stream);
    if (e != cudaSuccess) return cuda_fail(s, e, "reduction result");
    return sync_and_check(s, "reduction result");
}

qsa_status qsa_expectation_z_batch(qsa_state s, const uint64_t* logical_masks, int n_masks, double* out) {
    qsa_status st = check_state(s);
    if (st != QSA_OK) return st;
    if (!logical_masks || !out) return fail(QSA_E_ARG, "NULL argument");
    if (n_masks < 1 || n_masks > QSA_MAX_ZMASKS) return fail(QSA_E_ARG, "n_masks must be in 1..4");
    uint64_t pm[QSA_MAX_ZMASKS];
    for (int m = 0; m < n_masks; ++m) {
        if (s->n < 64 && (logical_masks[m] >> s->n)) return fail(QSA_E_ARG, "mask has bits beyond N");
        pm[m] = 0;
        for (int q = 0; q < s->n; ++q)
            if ((logical_masks[m] >> q) & 1) pm[m] |= 1ull << s->L[q];
    }
    const size_t nb = static_cast<size_t>(reduce_partials());
    st = ensure_dev(s, reinterpret_cast<void**>(&s->d_red), &s->red_cap,
                    sizeof(double) * (QSA_MAX_ZMASKS * nb + 8));
    if (st != QSA_OK) return st;
    double* d_out = s->d_red + QSA_MAX_ZMASKS * nb;
    cudaError_t e = launch_reduce_z_multi(s->psi, s->n, pm, n_masks, s->d_red, d_out, s->stream, &s->launches);
    if (e != cudaSuccess) return cuda_fail(s, e, "reduction kernel");
    e = cudaMemcpyAsync(out, d_out, sizeof(double) * n_masks, cudaMemcpyDeviceToHost, s->stream);
    if (e != cudaSuccess) return cuda_fail(s, e, "reduction results");
    return sync_and_check(s, "reduction results");
}

qsa_status qsa_state_sync(qsa_state s) {
    qsa_status st = check_state(s);
    if (st != QSA_OK) return st;
    return sync_and_check(s, "synchronise");
}

qsa_status qsa_probabilities_device(qsa_state s, double* out_dev, double* norm_out) {
    qsa_status st = check_state(s);
    if (st != QSA_OK) return st;
    if (out_dev) {
        cudaError_t e = launch_probs_logical(s->psi, s->n, s->L, out_dev, s->stream, &s->launches);
        if (e != cudaSuccess) return cuda_fail(s, e, "probability kernel");
    }
    if (norm_out) return qsa_expectation_z(s, 0, norm_out);
    cudaError_t e = cudaStreamSynchronize(s->stream);
    if (e != cudaSuccess) return cuda_fail(s, e, "probabilities");
    return QSA_OK;
}

qsa_status qsa_probabilities(qsa_state s, double* out_host, double* norm_out) {
    qsa_status st = check_state(s);
    if (st != QSA_OK) return st;
    if (out_host) {
        const size_t bytes = sizeof(double) << s->n;
        double* tmp = nullptr;
        cudaError_t e = dev_malloc(&tmp, bytes);
        if (e != cudaSuccess) {
            cudaGetLastError();
            return fail(QSA_E_NOMEM, "cudaMalloc of the probability buffer failed");
        }
        e = launch_probs_logical(s->psi, s->n, s->L, tmp, s->stream, &s->launches);
        if (e == cudaSuccess) e = cudaMemcpyAsync(out_host, tmp, bytes, cudaMemcpyDeviceToHost, s->stream);
        if (e != cudaSuccess) {
            dev_free(tmp);
            return cuda_fail(s, e, "probabilities");
        }
        st = sync_and_check(s, "probabilities");
        dev_free(tmp);
        if (st != QSA_OK) return st;
    }
    if (norm_out) return qsa_expectation_z(s, 0, norm_out);
    return QSA_OK;
}

qsa_status qsa_sample_counts(qsa_state s, uint64_t shots, uint64_t seed, uint64_t* outcomes, uint64_t* counts,
                             size_t capacity, size_t* n_distinct) {
    return qsa_measure(s, nullptr, 0, nullptr, shots, seed, outcomes, counts, capacity, n_distinct);
}

qsa_status qsa_measure(qsa_state s, const uint64_t* z_masks, int n_masks, double* z_out, uint64_t shots,
                       uint64_t seed, uint64_t* outcomes, uint64_t* counts, size_t capacity, size_t* n_distinct) {
    qsa_status st = check_state(s);
    if (st != QSA_OK) return st;
    if (!n_distinct) return fail(QSA_E_ARG, "n_distinct is NULL");
    if (shots < 1 || shots > (1ull << 26)) return fail(QSA_E_ARG, "shots must be in 1..2^26");
    if (capacity > 0 && (!outcomes || !counts)) return fail(QSA_E_ARG, "output arrays are NULL");
    if (n_masks < 0 || n_masks > QSA_MAX_ZMASKS) return fail(QSA_E_ARG, "n_masks must be in 0..4");
    if (n_masks > 0 && (!z_masks || !z_out)) return fail(QSA_E_ARG, "z_masks or z_out is NULL");
    uint64_t pm[QSA_MAX_ZMASKS] = {};
    for (int m = 0; m < n_masks; ++m) {
        if (s->n < 64 && (z_masks[m] >> s->n)) return fail(QSA_E_ARG, "mask has bits beyond N");
        for (int q = 0; q < s->n; ++q)
            if ((z_masks[m] >> q) & 1) pm[m] |= 1ull << s->L[q];
    }
    const size_t nbp = static_cast<size_t>(reduce_partials());
    if (n_masks > 0) {
        st = ensure_dev(s, reinterpret_cast<void**>(&s->d_red), &s->red_cap,
                        sizeof(double) * (QSA_MAX_ZMASKS * nbp + 8));
        if (st != QSA_OK) return st;
    }
    const size_t scratch = sample_scratch_bytes(s->n, shots);
    const size_t outb = sizeof(uint64_t) * (2 * shots + 4);
    st = ensure_dev(s, &s->d_samp, &s->samp_cap, scratch + outb);
    if (st != QSA_OK) return st;
    uint64_t* d_keys = reinterpret_cast<uint64_t*>(static_cast<char*>(s->d_samp) + scratch);
    uint64_t* d_cnts = d_keys + shots;
    uint64_t* d_nd = d_cnts + shots;
    double* d_zout = n_masks > 0 ? s->d_red + QSA_MAX_ZMASKS * nbp : nullptr;
    cudaError_t e = launch_sample_z(s->psi, s->n, s->L, shots, seed, 0, s->d_samp, d_keys, d_cnts, d_nd, pm, n_masks,
                                    n_masks > 0 ? s->d_red : nullptr, d_zout, s->stream, &s->launches);
    if (e != cudaSuccess) return cuda_fail(s, e, "sampler kernels");
    if (n_masks > 0) {
        e = cudaMemcpyAsync(z_out, d_zout, sizeof(double) * n_masks, cudaMemcpyDeviceToHost, s->stream);
        if (e != cudaSuccess) return cuda_fail(s, e, "expectation results");
    }
    uint64_t hdr[2] = {0, 0};
    const int bsz = s->n >= 10 ? 1024 : (1 << s->n);
    const uint64_t nblocks = (1ull << s->n) / bsz;
    e = cudaMemcpyAsync(&hdr[0], d_nd, sizeof(uint64_t), cudaMemcpyDeviceToHost, s->stream);
    if (e == cudaSuccess)
        e = cudaMemcpyAsync(&hdr[1], static_cast<uint64_t*>(s->d_samp) + (nblocks - 1), sizeof(uint64_t),
                            cudaMemcpyDeviceToHost, s->stream);
    if (e != cudaSuccess) return cuda_fail(s, e, "sampler result");
    st = sync_and_check(s, "sampler result");
    if (st != QSA_OK) return st;
    if (hdr[1] == 0) return fail(QSA_E_STATE, "every amplitude weight is zero");
    *n_distinct = static_cast<size_t>(hdr[0]);
    if (capacity < hdr[0]) return fail(QSA_E_RANGE, "capacity smaller than the number of distinct outcomes");
    e = cudaMemcpyAsync(outcomes, d_keys, sizeof(uint64_t) * hdr[0], cudaMemcpyDeviceToHost, s->stream);
    if (e == cudaSuccess)
        e = cudaMemcpyAsync(counts, d_cnts, sizeof(uint64_t) * hdr[0], cudaMemcpyDeviceToHost, s->stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(s->stream);
    if (e != cudaSuccess) return cuda_fail(s, e, "sampler copy");
    return QSA_OK;
}

}  // extern "C"
