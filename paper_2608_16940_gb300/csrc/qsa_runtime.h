// Host-side state object and helpers shared by runtime.cpp and planner.cpp.
#pragma once

#include <cuda_runtime.h>

#include <array>
#include <complex>
#include <string>
#include <utility>
#include <vector>

#include "qsa.h"
#include "qsa_costmodel.h"
#include "qsa_internal.h"

struct qsa_state_s {
    int n = 0;
    float2* psi = nullptr;
    bool owned = false;
    cudaStream_t stream = nullptr;
    int32_t L[QSA_MAX_QUBITS] = {};   // layout map: logical -> physical
    bool known_zero = false;          // state is |0..0> (metadata-only relabel allowed)
    bool failed = false;              // sticky after a CUDA error
    uint64_t launches = 0;            // kernels issued on this state
    bool timing = false;              // record CUDA events around launches
    // device scratch (grown on demand)
    float* d_mat = nullptr;
    size_t mat_cap = 0;
    double* d_red = nullptr;
    size_t red_cap = 0;
    void* d_samp = nullptr;
    size_t samp_cap = 0;
    float* d_mlp = nullptr;
    size_t mlp_cap = 0;
    double* d_dm = nullptr;           // density-matrix diagonal readout
    size_t dm_cap = 0;
    void* d_lrec = nullptr;           // per-tile records of layer passes
    size_t lrec_cap = 0;
    int* d_err = nullptr;             // device error word written by bounded waits
    qsa::CostModel cm;                // cost model attached to this state (qsa_costmodel_load), or null
    // CUDA-event timers
    struct Pending {
        cudaEvent_t a, b;
        double* acc;
    };
    std::vector<std::pair<cudaEvent_t, cudaEvent_t>> ev_free;
    std::vector<Pending> ev_pending;
};

// A layer block on logical qubits: diagonal ops (k = 1, 2; entries d[c], bit
// j of c <-> q[j]) applied first, then one-qubit factors on distinct qubits.
struct LayerDiagOp {
    int k = 1;
    int32_t q[2] = {0, 0};
    std::complex<double> d[4];
};
struct LayerSpec {
    bool generate = false;                                  // write-only on a state taken as all ones
    std::vector<LayerDiagOp> diag;
    std::vector<int32_t> t;                                 // factor qubits
    std::vector<std::array<std::complex<double>, 4>> f;     // factor j on t[j], row-major
};
// One prepared pass: geometry, offsets relative to the payload at dev_off.
struct LayerLaunch {
    qsa::LayerGeom g;
    qsa::LayerPayload p;
    size_t dev_off = 0;
};

struct PlanBlock {
    int32_t t[QSA_MAX_DIAG];   // ordered logical targets of the fused block (QSA_MAX_DIAG >= QSA_MAX_LAYER);
                               // a layer block lists its factor qubits
    int k = 0;
    bool diag = false;         // diagonal mode: 2^k entries, streaming kernel
    bool prod = false;         // product of one-qubit factors: 8 floats per factor, product kernel
    int layer = -1;            // layer block: index into qsa_plan_s::layers
    bool init = false;         // zero-state preparation (a write-only layer block)
    int n_diag = 0;            // layer block: ops of its diagonal part
    size_t off = 0;            // float offset of its matrix / diagonal in host_mat / d_mat
    size_t first_op = 0;       // in execution order
};

struct PlanLayer {
    LayerSpec spec;
    std::vector<LayerLaunch> launches;   // for the plan's layout (empty when N < 12)
};

struct qsa_plan_s {
    int n = 0;
    qsa_plan_opts opts{};
    size_t n_ops = 0;
    int max_width = 0;
    std::vector<PlanBlock> blocks;
    std::vector<float> host_mat;   // all fused matrices, FP32, 16-byte aligned
    float* d_mat = nullptr;        // device copy (uploaded on first execution)
    std::vector<int32_t> next_use; // per block, per logical qubit: next dense block targeting it
    int dev = -1;
    std::vector<size_t> order;     // execution order of the input ops
    std::vector<int32_t> L0;       // the layout the plan was built for
    std::vector<PlanLayer> layers;
    std::vector<unsigned char> host_layer;   // layer payloads (16-byte aligned)
    unsigned char* d_layer = nullptr;
};

namespace qsa {

// In-block bits: the low positions a tile of the FP32 kernels covers as one
// contiguous run (2^11 amplitudes = 16 KiB).
constexpr int kInBlockBits = 11;

qsa_status fail(qsa_status st, const std::string& msg);
qsa_status cuda_fail(qsa_state s, cudaError_t e, const char* where);
qsa_status check_state(qsa_state s);
qsa_status sync_and_check(qsa_state s, const char* where);
qsa_status ensure_dev(qsa_state s, void** ptr, size_t* cap, size_t bytes);
void to_float_matrix(const double* m, int k, float* out);
// Running sum of the modulus errors left by the FP32 constants of one plan,
// each weighted by the share of the state it multiplies (see f2_modulus).
struct ModulusCarry {
    double acc = 0.0;
};
// FP32 complex number within a few ulps of z whose squared modulus, weighted
// by `weight` and added to the carry, leaves the carry nearest zero (with no
// carry: whose squared modulus is nearest m2); the carry is updated.  See
// layer_host.cpp.
float2 f2_modulus(std::complex<double> z, double m2, double weight = 1.0, ModulusCarry* carry = nullptr);
// A table of `count` interleaved complex numbers rounded that way, each with
// its own modulus as the target and the given weight.
void to_float_moduli(const double* z, size_t count, float* out, double weight, ModulusCarry* carry);
qsa_status validate_targets(int n, const int32_t* targets, int k, int kmax = QSA_MAX_K);
qsa_status apply_logical(qsa_state s, const int32_t* targets, int k, const float* d_mat, int lowering,
                         int precision, qsa_run_stats* rs);
qsa_status apply_physical(qsa_state s, const int* phys, int k, const float* d_mat, int precision,
                          qsa_run_stats* rs);
qsa_status permute_positions(qsa_state s, const int* pa, const int* pb, int np, qsa_run_stats* rs);
// Victims for the targets of one dense block under the demand model (§IV-D):
// phys[j] (positions of the block's targets) are updated in place and the
// position pairs to swap written to (pa[i], pb[i]); returns their count, or -1
// if the frames (positions 0..frames-1) cannot hold the block.  next_use[q]
// (per logical qubit; QSA_VICTIM_FARTHEST only) is the index of the next dense
// block targeting q, INT32_MAX for never.  L is not modified.
int choose_promotions(const int32_t* L, int n, int* phys, int k, int frames, int victim, const int32_t* next_use,
                      int* pa, int* pb);
qsa_status promote_targets(qsa_state s, int* phys, int k, int inblock, qsa_run_stats* rs);
// Diagonal block on logical targets (the layout resolves them; it is not changed).
qsa_status apply_diag_logical(qsa_state s, const int32_t* targets, int k, const float* d_tab, qsa_run_stats* rs);
// Product block on logical targets (factor j on targets[j]; layout unchanged).
qsa_status apply_prod_logical(qsa_state s, const int32_t* targets, int k, const float* d_fac, qsa_run_stats* rs);
bool tc_available(qsa_state s, int k);

// Layer blocks (layer.cu kernel; host preparation in layer_host.cpp).
// True if factor positions pos[0..k) fit one tile (at most 9 at 3 or above).
bool layer_fits(int n, const int* pos, int k);
// The passes of a layer block for layout L (N >= 12): factors split into
// groups that fit a tile (in target order), the diagonal ops in the first;
// payloads appended to *bytes (16-byte aligned), dev_off relative to its start.
std::vector<LayerLaunch> prepare_layer(int n, const int32_t* L, const LayerSpec& spec,
                                       std::vector<unsigned char>* bytes, ModulusCarry* carry = nullptr);
qsa_status run_layer_launches(qsa_state s, const std::vector<LayerLaunch>& ls, const unsigned char* d_base,
                              qsa_run_stats* rs);
// Prepare for the state's current layout, upload to scratch and run (N < 12:
// the diagonal and product kernels, op by op).
qsa_status apply_layer_logical(qsa_state s, const LayerSpec& spec, qsa_run_stats* rs);
// Plan-time hand-over between consecutive layer blocks: each unitary factor
// F = diag(p) R diag(q) of *from becomes R diag(q), and diag(p) (a one-qubit
// diagonal gate, which precedes every op of *to) joins the front of *to's
// diagonal part, where it costs nothing extra.
void layer_move_exit_phases(LayerSpec* from, LayerSpec* to);
// Diagonal entries of a k = 1, 2 op (QSA_E_ARG if an off-diagonal entry is non-zero).
qsa_status layer_diag_from_op(const qsa_op& op, LayerDiagOp* out);

// Records a pair of CUDA events around the launches issued during its
// lifetime; the elapsed time is added to *acc by collect_timers().
class Timer {
  public:
    Timer(qsa_state s, double* acc);
    ~Timer();
    void stop();

  private:
    qsa_state s_;
    double* acc_;
    cudaEvent_t ev_[2] = {nullptr, nullptr};
    bool stopped_ = false;
};
void collect_timers(qsa_state s, double* total);
// qsa_plan_create with an explicit cost model for QSA_PLAN_DP_MLP (null: the
// width-limit heuristic).
qsa_status plan_create(const qsa_op* ops, size_t n_ops, int n_qubits, const qsa_plan_opts* opts,
                       const int32_t* layout, const CostModel& model, qsa_plan* out);

}  // namespace qsa
