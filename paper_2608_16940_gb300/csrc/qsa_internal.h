// Internal declarations shared by the runtime (.cpp) and the kernels (.cu).
#pragma once

#include <cuda_runtime.h>
#include <cstddef>
#include <cstdint>

#include "qsa.h"

namespace qsa {

// Tile geometry of one full-state pass (§IV-B: the 2^k x 2^(N-k) view is
// walked tile by tile).  A tile is every amplitude whose index agrees with the
// tile's base on all "outer" bit positions; its T tile bits are the m lowest
// positions (contiguous runs of 2^m amplitudes) plus nx extra positions
// xpos[] >= m.  Tiles partition the state, so a pass can run in place.
struct TileGeom {
    int n;          // qubits
    int T;          // tile bits
    int m;          // run bits (positions 0..m-1)
    int nx;         // extra tile bits
    int xpos[6];    // extra positions, ascending
    uint64_t ntiles;
};

// Chooses m so that every position in `special` is a tile bit and
// m + #(special >= m) <= T (T = min(T_want, n)).  Returns false if more than
// six special positions would be extra bits.
bool make_geom(int n, const int* special, int ns, int T_want, TileGeom* g);

// Every device allocation of the library goes through these: a host-side
// test hook can make the n-th allocation fail as if the device were out of
// memory (qsa_debug_fail_alloc, QSA_FAULT_ALLOC), and the live allocations
// are counted (qsa_debug_live_allocations), so the error paths and their
// cleanup are tested without any device fault.
cudaError_t dev_malloc_raw(void** p, size_t bytes);
template <typename T>
cudaError_t dev_malloc(T** p, size_t bytes) {
    return dev_malloc_raw(reinterpret_cast<void**>(p), bytes);
}
void dev_free(void* p);

// First bounds-check record of each checked translation unit ((code << 48) |
// index, 0 if none; always 0 unless built with -DQSA_DEBUG_BOUNDS).
uint64_t bounds_word_apply();
uint64_t bounds_word_layer();
uint64_t bounds_word_tc();

// Number of SMs of the current device (cached per device).
int num_sms();
// cudaFuncSetAttribute(kernel, MaxDynamicSharedMemorySize, bytes) on the
// current device unless a size at least as large was set there before (the
// attribute belongs to the device's context; cached per device and kernel).
cudaError_t set_smem_attr(const void* kernel, int bytes);

// One fused block of a trajectory in the batched kernel (k <= 4, tile bits 11).
struct BatchBlock {
    int32_t k, T, m, nx;
    int32_t xpos[6], tl[6], tls[6];
    uint32_t mat_off;   // float offset of G in the matrix table
    int32_t form;       // 0 plain stage, 1 swizzled gathers, 2 swizzled with in-place write-back
    uint8_t fv[16];     // slot vectors of the swizzled stage
};

struct BatchArgs {
    float2* states;            // n_traj consecutive states of 2^n amplitudes
    int n, n_traj;
    const BatchBlock* blocks;
    const uint32_t* bstart;    // n_traj + 1 block offsets
    const int32_t* order;      // trajectories in queue order (longest first)
    const float* mats;
    unsigned int* queue;       // work counter, zero before the launch
    int* err;                  // set to 7 when the cycle budget runs out
    unsigned long long budget; // clock64 cycles per CTA, 0 = unlimited
};

bool make_batch_block(int n, const int* phys, int k, uint32_t mat_off, BatchBlock* b);
cudaError_t launch_batch_evolve(const BatchArgs& a, cudaStream_t st, uint64_t* launches);

// One CTA per trajectory: sample `shots` outcomes of every state (identity
// layout) with Philox stream id = trajectory index, sort, run-length encode.
// Outputs per trajectory t at t * shots: outcomes, counts; n_distinct[t].
cudaError_t launch_batch_sample(const float2* states, int n, int n_traj, uint32_t shots, uint64_t seed,
                                uint32_t* out_keys, uint32_t* out_counts, uint32_t* n_distinct, cudaStream_t st,
                                uint64_t* launches);

// ---- launchers (return the first CUDA error; *launches incremented) --------
cudaError_t launch_init_zero(float2* psi, int n, cudaStream_t st, uint64_t* launches);
// Every amplitude set to 1 (the start of a write-only preparation on small states).
cudaError_t launch_fill_one(float2* psi, int n, cudaStream_t st, uint64_t* launches);

// FP32 fused dense update: phys[j] = physical position of target j (V order),
// d_mat = 2*4^k floats (row-major, interleaved) in device memory.
cudaError_t launch_apply_fp32(float2* psi, int n, const int* phys, int k, const float* d_mat,
                              cudaStream_t st, uint64_t* launches);

// Split-TF32 tensor-core update for k = 5, 6.  d_mat as above.  d_err: one
// int in device memory; the kernel writes a non-zero code when a bounded wait
// gives up.  Returns cudaErrorNotSupported for other k.
cudaError_t launch_apply_tc(float2* psi, int n, const int* phys, int k, const float* d_mat, int* d_err,
                            cudaStream_t st, uint64_t* launches);
// Diagonal streaming update (k <= QSA_MAX_DIAG): psi[y] *= d_tab[c(y)], bit j
// of c = bit phys[j] of y; d_tab is 2^k interleaved FP32 complex numbers.
cudaError_t launch_apply_diag(float2* psi, int n, const int* phys, int k, const float* d_tab, cudaStream_t st,
                              uint64_t* launches);
// Product of one-qubit factors (k <= QSA_MAX_PROD): factor j (2x2 complex,
// row-major, 8 floats at d_fac + 8 j) on physical position phys[j].
cudaError_t launch_apply_prod(float2* psi, int n, const int* phys, int k, const float* d_fac, cudaStream_t st,
                              uint64_t* launches);
// Diagonal of a vectorised n-qubit density matrix held as a 2n-qubit state:
// rho_xx to d_out (device, 2^n doubles, nullable) and
// sum_x rho_xx (-1)^popc(x & mask) to *d_sum (device), via d_partials
// (reduce_partials() doubles).
cudaError_t launch_dm_diag(const float2* psi, int n, const int32_t* layout_host, uint64_t mask, double* d_out,
                           double* d_partials, double* d_sum, cudaStream_t st, uint64_t* launches);

// Layer block launch (one pass; see layer.cu).  Tile of 12 bits: positions
// 0..m-1 plus xpos[0..nx-1] (ascending, >= m), m + nx = 12, m >= 3.
struct LayerGeom {
    int m = 12, nx = 0;
    int xpos[12] = {};
};
// A diagonal gate relative to a tile: cross (a = tile bit, b = outside
// position, d[2 * o + v] for outside bit o and tile bit v) or out (a, b =
// positions, b < 0 for one qubit, d[v_a + 2 v_b]).
struct LayerGate {
    int32_t a, b;
    float2 d[4];
};
// Byte offsets of one launch's data in its device payload.
struct LayerPayload {
    uint32_t active = 0;      // tile bits with a factor
    uint32_t pmask = 0;       // tile bits whose per-tile phases are multiplied in
    int ncross = 0, nout = 0;
    int cstart[13] = {};
    bool has_din = false;     // 2^12-entry table of the gates with every qubit in the tile
    bool rotation = false;    // factors as real rotations (their phases as per-bit and per-round tables)
    uint32_t rpmask = 0;      // rotation mode: rounds whose exit phases are not all 1
    uint32_t rswap = 0;       // rotation mode: tile bits whose halves the pass leaves exchanged
    bool generate = false;    // write-only: the input is taken as 1 for every amplitude (not read)
    size_t off_fac = 0, off_cross = 0, off_out = 0, off_din = 0, off_qph = 0, off_rp = 0, off_sph = 0, bytes = 0;
    // rotation mode: host copies of the payload's FP32 rotation coefficients (t or u per tile bit)
    // and per-round exit phases (3 x 16 complex, interleaved), passed with the launch
    float rot[12] = {};
    float rp[96] = {};
};
size_t layer_smem_bytes(bool with_din);
// Rotation-mode passes with per-tile phases first write one record per tile
// to d_rec (device, layer_record_bytes(n) bytes; the call fails without it).
size_t layer_record_bytes(int n);
cudaError_t launch_layer_records(float2* psi, int n, const LayerGeom& g, const unsigned char* d_payload,
                                 const LayerPayload& p, void* d_rec, cudaStream_t st, uint64_t* launches);
cudaError_t launch_apply_layer(float2* psi, int n, const LayerGeom& g, const unsigned char* d_payload,
                               const LayerPayload& p, void* d_rec, cudaStream_t st, uint64_t* launches);

// In-place swap of physical bit pairs (pa[i] <-> pb[i]), all positions distinct.
cudaError_t launch_permute(float2* psi, int n, const int* pa, const int* pb, int npairs, cudaStream_t st,
                           uint64_t* launches);

// FP64 sum of (-1)^{popcount(y & physmask)} |psi_y|^2 into *d_out (device).
// d_partials must hold reduce_partials() doubles.
int reduce_partials();
constexpr int kMaxZMasks = 4;
struct ZMasks {
    int n;
    uint64_t m[kMaxZMasks];
};
// Several <Z_mask> sums in one pass: d_partials holds nmasks * reduce_partials()
// doubles, d_out nmasks doubles (device).  nmasks in 1..kMaxZMasks.
cudaError_t launch_reduce_z_multi(const float2* psi, int n, const uint64_t* physmasks, int nmasks,
                                  double* d_partials, double* d_out, cudaStream_t st, uint64_t* launches);
cudaError_t launch_reduce_z(const float2* psi, int n, uint64_t physmask, double* d_partials, double* d_out,
                            cudaStream_t st, uint64_t* launches);

// out[x] = |psi_{encode(x)}|^2 for logical x; d_layout = int32 L[0..n-1] on device.
cudaError_t launch_probs_logical(const float2* psi, int n, const int32_t* d_layout, double* out,
                                 cudaStream_t st, uint64_t* launches);

// Sampler scratch sizes and launch (see qsa_sample_counts).
uint64_t next_pow2_u64(uint64_t v);
size_t sample_scratch_bytes(int n, uint64_t shots);
cudaError_t launch_sample(const float2* psi, int n, const int32_t* d_layout, uint64_t shots, uint64_t seed,
                          uint64_t stream_id, void* d_scratch, uint64_t* d_out_keys, uint64_t* d_out_counts,
                          uint64_t* d_n_distinct, cudaStream_t st, uint64_t* launches);
// The same with <Z_mask> sums for nmasks (0..kMaxZMasks) physical masks taken in
// the weights pass: d_zpartials holds nmasks * reduce_partials() doubles, the
// sums go to d_zout[0..nmasks) (device).
cudaError_t launch_sample_z(const float2* psi, int n, const int32_t* layout_host, uint64_t shots, uint64_t seed,
                            uint64_t stream_id, void* d_scratch, uint64_t* d_out_keys, uint64_t* d_out_counts,
                            uint64_t* d_n_distinct, const uint64_t* physmasks, int nmasks, double* d_zpartials,
                            double* d_zout, cudaStream_t st, uint64_t* launches);

}  // namespace qsa
