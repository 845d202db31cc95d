// Split-TF32 (3xTF32) fused dense update on tcgen05 tensor cores, k = 5, 6.
//
// The update of one group of 2^k amplitudes (§IV-B: M' = G M on the
// 2^k x 2^(N-k) view) is a real matrix-vector product after embedding complex
// numbers as 2x2 real blocks: u[2c+t] = (Re, Im)(psi_c) and
// R[2r+s][2c+t] = [[Re G, -Im G], [Im G, Re G]][s][t], u' = R u.
//
// Work unit: a chunk of 2^11 amplitudes, the state restricted to 11 bit
// positions (the targets and the lowest non-target positions) with every
// other bit fixed.  A chunk is 32 rows of 64 amplitudes: a row fixes the five
// lowest non-target positions ("row bits"), and its 64 amplitudes run over
// six "K bits" (k = 6: the targets in ascending position; k = 5: the targets
// and the sixth non-target position, so a row holds two groups).  One chunk
// is the GEMM
//     D (128 x 32) = A (128 x 128) . B (32 x 128)^T,
// A = R (k = 6) or blockdiag(R, R) (k = 5) in the K-bit numbering, B = the
// chunk's rows as real vectors of 128 floats: D[2 nu + s][row] is part s of
// output amplitude nu of the row.  Both operands are split into hi and lo
// parts and D = A_hi B_hi + (A_hi B_lo + A_lo B_hi), the three-product
// split-TF32 scheme of Ootomo & Yokota 2022 ("Recovering single precision
// accuracy from Tensor Cores while surpassing the FP32 theoretical peak
// performance").
//
// Tensor cores round their FP32 accumulation toward zero, which biases every
// rounded sum towards zero; over a deep circuit that shrinks the norm
// linearly with depth.  The dominant product is therefore made exact: hi
// parts are block-quantised per row and K half (64 values) to integer
// multiples c q of a power-of-two quantum q (|c| <= 2048 for the matrix,
// <= 128 for the state), so every partial sum of a 64-term half of
// A_hi B_hi is an integer multiple of q_A q_B of magnitude at most 2^24:
// exact in FP32, nothing for the tensor core to round.
// Each half accumulates into its own tensor-memory columns and the epilogue
// adds the two and the correction accumulator in FP32 with round-to-nearest.
// lo = x - hi (exact) is rounded to TF32 to nearest; the correction products
// (about 2^-9 of the result) accumulate in tensor memory, where their
// rounding is far below FP32 resolution of the output.
//
// CTA roles (one persistent CTA per SM, 736 threads).  Chunks go through the
// tensor core in pairs (chunks 2p and 2p + 1 of the CTA's list): each MMA has
// N = 64, the B rows of both chunks, which halves the MMA instructions per
// chunk against N = 32.
//   warps 16-19 producers: copy each chunk from HBM into a 4-stage ring with
//               16-byte cp.async (mbarrier-tracked; each warp a quarter of
//               the chunk's copies), in an XOR layout chosen per launch so
//               that the converters' reads are free of bank conflicts for any
//               target positions;
//   warps 0-7   converters in two teams of four; team t converts chunk
//               2p + t of every pair into rows 32 t .. 32 t + 31 of B buffer
//               p mod 2 (two buffers, so the conversion of a pair overlaps
//               the MMAs of the previous one).  A lane holds one K quarter
//               (16 amplitudes) of one row: the values into registers (the
//               raw stage is released right away), the K half's quantum
//               (maximum shared with the lane holding the other quarter), the
//               hi / lo split and the B operand (K-major, 128-byte swizzle);
//   warps 20-22 one thread each issues one of the pair's three products
//               (16 MMAs, N = 64) into its own accumulator columns: a single
//               issuing thread left the tensor pipe idle most of the time.
//               Warp 20 allocates tensor memory; A (hi and lo) stays there for
//               the whole launch;
//   warps 8-15  epilogue in two groups of four; group g takes chunk 2p + g of
//               every pair (accumulator columns 32 g .. 32 g + 31), warp w on
//               tensor-memory lanes 32 (w % 4) ...: sums the accumulators into
//               the group's staging area in a second XOR layout (chunk-local
//               order), then stores the chunk back in 16-byte units exactly as
//               the producers read it, so every warp store covers 512
//               consecutive bytes whatever the target positions.  At the
//               start group g builds K half g of A in tensor memory, from G
//               staged in B buffer 0 (the converters start writing B once A
//               is ready).
// Tensor memory (512 columns): A_hi 128, A_lo 128, and one accumulator set of
// 256 columns (two exact main halves and the two correction products, 64
// columns each for the pair).
// Every mbarrier wait is bounded; on timeout the CTA records an error code,
// drains its copies and MMAs, frees tensor memory and returns.
#include <cuda_runtime.h>

#include <algorithm>
#include <cstdint>
#include <type_traits>

#include "qsa_bounds.cuh"
#include "qsa_internal.h"
#include "qsa_runtime.h"

namespace qsa {

namespace {

constexpr int kThreads = 736;
constexpr int kConvWarps = 8;                // warps 0-7: converters, two teams of four
constexpr int kEpiWarp = 8;                  // warps 8-15: epilogue, two groups of four
constexpr int kProdWarp = 16;                // warps 16-19: producers
constexpr int kProducers = 4;
static_assert(kProducers == 4, "the producers' unit loops are specialised for four warps");
constexpr int kMmaWarp = 20;                 // warps 20-22: MMA issuers (warp 20 owns tensor memory)
constexpr int kIssuers = 3;
constexpr int kChunkBits = 11;               // amplitudes per chunk: 2^11
constexpr int kNR = 4;                       // raw chunk stages
// chunks go through the MMA in pairs: a B operand holds 64 rows, two chunks
// of 32 (one per converter team), and each MMA has N = 64; two B buffers
// (pair p in buffer p mod 2) let the conversion of a pair overlap the MMAs
// of the one before
constexpr int kNB = 2;
constexpr uint64_t kWaitNs = 1000000000ull;   // a wait gives up after one second
constexpr uint32_t kSuspendNs = 100000;        // a try_wait may sleep this long before it returns

constexpr uint32_t kRawBytes = (1u << kChunkBits) * 8;   // 16 KiB
constexpr uint32_t kKBlock = 64 * 128;                   // one K block of B: 64 rows x 32 floats (128 B)
constexpr uint32_t kHalfB = 4 * kKBlock;                 // one split part of B: 64 rows x 128 floats
constexpr uint32_t kBBytes = 2 * kHalfB;                 // hi + lo
// epilogue staging: one chunk per epilogue group, in the output layout
constexpr uint32_t kOutBytes = kRawBytes;
// shared memory carve-up (from a 1024-byte aligned base)
constexpr uint32_t OFF_B = 0;
constexpr uint32_t OFF_RAW = OFF_B + kNB * kBBytes;
constexpr uint32_t OFF_STG = OFF_RAW + kNR * kRawBytes;
constexpr uint32_t OFF_BARS = OFF_STG + 2 * kOutBytes;
constexpr int BAR_RFULL = 0, BAR_REMPTY = kNR, BAR_BFULL = 2 * kNR, BAR_BEMPTY = BAR_BFULL + kNB,
              BAR_DFULL = BAR_BEMPTY + kNB, BAR_DEMPTY = BAR_DFULL + 1, BAR_AREADY = BAR_DEMPTY + 1,
              BAR_FIN = BAR_AREADY + 1, NBARS = BAR_FIN + 1;
constexpr uint32_t OFF_MISC = OFF_BARS + NBARS * 8;        // tensor-memory address, abort word
constexpr size_t kSmem = 1024 + OFF_MISC + 16;
static_assert(kSmem <= 232448, "shared memory per CTA");
// tensor memory columns
// accumulators of a pair: main K half 0, main K half 1, A_hi B_lo, A_lo B_hi
// (64 columns each: chunk 2p in the first 32, chunk 2p + 1 in the next 32)
constexpr uint32_t COL_AHI = 0, COL_ALO = 128, COL_D = 256, D_COLS = 256;
constexpr uint32_t kTmemCols = 512;
static_assert(COL_D + D_COLS <= kTmemCols, "tensor memory");
// instruction descriptor: D FP32, A and B TF32, both K-major, N = 64, M = 128
constexpr uint32_t kIdesc = (1u << 4) | (2u << 7) | (2u << 10) | ((64u >> 3) << 17) | ((128u >> 4) << 24);

__device__ __forceinline__ uint32_t smem_u32(const void* p) {
    return static_cast<uint32_t>(__cvta_generic_to_shared(p));
}

__device__ __forceinline__ void mbar_init(uint32_t a, uint32_t count) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;\n" ::"r"(a), "r"(count) : "memory");
}
__device__ __forceinline__ void mbar_arrive(uint32_t a) {
    asm volatile("{\n .reg .b64 st;\n mbarrier.arrive.shared::cta.b64 st, [%0];\n}\n" ::"r"(a) : "memory");
}
__device__ __forceinline__ bool mbar_try(uint32_t a, uint32_t parity) {
    uint32_t ok;
    asm volatile(
        "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2, %3;\n selp.b32 %0, 1, 0, p;\n}\n"
        : "=r"(ok)
        : "r"(a), "r"(parity), "r"(kSuspendNs)
        : "memory");
    return ok != 0;
}
__device__ __forceinline__ uint64_t global_ns() {
    uint64_t t;
    asm volatile("mov.u64 %0, %%globaltimer;\n" : "=l"(t));
    return t;
}
// Bounded wait; gives up (and raises the CTA abort word) after kWaitNs or as
// soon as another role has aborted.  The thread sleeps inside try_wait until
// the phase completes (or kSuspendNs passes), so waiting warps take few issue
// slots from the working ones.  The first give-up on the device records its
// code, the chunk it waited for and the CTA in gerr[0..2].
__device__ bool mbar_wait(uint32_t a, uint32_t parity, volatile int* abort_flag, int* gerr, int code,
                          uint64_t item = 0) {
    if (mbar_try(a, parity)) return true;
    const uint64_t t0 = global_ns();
    for (;;) {
        if (mbar_try(a, parity)) return true;
        if (*abort_flag) return false;
        if (global_ns() - t0 > kWaitNs) break;
    }
    *abort_flag = 1;
    if (atomicCAS(gerr, 0, code) == 0) {
        gerr[1] = static_cast<int>(item);
        gerr[2] = static_cast<int>(blockIdx.x);
    }
    return false;
}

// Named barrier over nthreads threads; group_all also returns the AND of v
// over them.  Every thread of the group reaches each call the same number of
// times (the group's exits are decided by group_all).
__device__ __forceinline__ void group_sync(uint32_t id, uint32_t nthreads) {
    asm volatile("bar.sync %0, %1;\n" ::"r"(id), "r"(nthreads) : "memory");
}
__device__ __forceinline__ bool group_all(uint32_t id, uint32_t nthreads, bool v) {
    uint32_t r;
    asm volatile(
        "{\n .reg .pred p, q;\n setp.ne.u32 p, %1, 0;\n bar.red.and.pred q, %2, %3, p;\n selp.u32 %0, 1, 0, q;\n}\n"
        : "=r"(r)
        : "r"(static_cast<uint32_t>(v)), "r"(id), "r"(nthreads)
        : "memory");
    return r != 0;
}
__device__ __forceinline__ void fence_async_smem() { asm volatile("fence.proxy.async.shared::cta;\n" ::: "memory"); }
__device__ __forceinline__ void fence_mbar_init() { asm volatile("fence.mbarrier_init.release.cluster;\n" ::: "memory"); }
__device__ __forceinline__ void tc_fence_before() { asm volatile("tcgen05.fence::before_thread_sync;\n" ::: "memory"); }
__device__ __forceinline__ void tc_fence_after() { asm volatile("tcgen05.fence::after_thread_sync;\n" ::: "memory"); }

__device__ __forceinline__ void tmem_alloc(uint32_t dst, uint32_t ncols) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;\n" ::"r"(dst), "r"(ncols)
                 : "memory");
}
__device__ __forceinline__ void tmem_relinquish() {
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;\n" ::: "memory");
}
__device__ __forceinline__ void tmem_dealloc(uint32_t taddr, uint32_t ncols) {
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;\n" ::"r"(taddr), "r"(ncols) : "memory");
}

// A operand in tensor memory (M = 128 lanes, K-step of 8 columns), B in shared memory.
__device__ __forceinline__ void mma_tf32_ts(uint32_t d_tmem, uint32_t a_tmem, uint64_t bdesc, uint32_t idesc,
                                            uint32_t accumulate) {
    asm volatile(
        "{\n .reg .pred p;\n setp.ne.b32 p, %4, 0;\n"
        " tcgen05.mma.cta_group::1.kind::tf32 [%0], [%1], %2, %3, p;\n}\n" ::"r"(d_tmem),
        "r"(a_tmem), "l"(bdesc), "r"(idesc), "r"(accumulate)
        : "memory");
}
__device__ __forceinline__ void mma_commit(uint32_t mbar) {
    asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];\n" ::"r"(mbar)
                 : "memory");
}

// 32 lanes x 8 consecutive 32-bit columns (one row per thread).
__device__ __forceinline__ void tmem_ld8(uint32_t taddr, uint32_t* r) {
    asm volatile("tcgen05.ld.sync.aligned.32x32b.x8.b32 {%0, %1, %2, %3, %4, %5, %6, %7}, [%8];\n"
                 : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7])
                 : "r"(taddr));
}
__device__ __forceinline__ void tmem_ld_wait() { asm volatile("tcgen05.wait::ld.sync.aligned;\n" ::: "memory"); }
// 32 lanes x 16 consecutive 32-bit columns (one row per thread).
__device__ __forceinline__ void tmem_st16(uint32_t taddr, const float* v) {
    asm volatile(
        "tcgen05.st.sync.aligned.32x32b.x16.b32 [%0], "
        "{%1, %2, %3, %4, %5, %6, %7, %8, %9, %10, %11, %12, %13, %14, %15, %16};\n" ::"r"(taddr),
        "r"(__float_as_uint(v[0])), "r"(__float_as_uint(v[1])), "r"(__float_as_uint(v[2])), "r"(__float_as_uint(v[3])),
        "r"(__float_as_uint(v[4])), "r"(__float_as_uint(v[5])), "r"(__float_as_uint(v[6])), "r"(__float_as_uint(v[7])),
        "r"(__float_as_uint(v[8])), "r"(__float_as_uint(v[9])), "r"(__float_as_uint(v[10])), "r"(__float_as_uint(v[11])),
        "r"(__float_as_uint(v[12])), "r"(__float_as_uint(v[13])), "r"(__float_as_uint(v[14])), "r"(__float_as_uint(v[15]))
        : "memory");
}
__device__ __forceinline__ void tmem_st_wait() { asm volatile("tcgen05.wait::st.sync.aligned;\n" ::: "memory"); }

__device__ __forceinline__ void cp_async16(uint32_t dst, const void* src) {
    asm volatile("cp.async.cg.shared.global [%0], [%1], 16;\n" ::"r"(dst), "l"(src) : "memory");
}
// The mbarrier counts one arrival for this thread once all its earlier
// cp.async copies have landed.
__device__ __forceinline__ void cp_async_arrive_noinc(uint32_t mbar) {
    asm volatile("cp.async.mbarrier.arrive.noinc.shared::cta.b64 [%0];\n" ::"r"(mbar) : "memory");
}
__device__ __forceinline__ void cp_async_wait_all() { asm volatile("cp.async.wait_all;\n" ::: "memory"); }

__device__ __forceinline__ float tf32_rna(float x) {
    uint32_t r;
    asm("cvt.rna.tf32.f32 %0, %1;\n" : "=r"(r) : "f"(x));
    return __uint_as_float(r);
}

// Block split of a 64-value segment (one row, one K half): hi = c q with the
// shared power-of-two quantum q = 2^(E+1-S), E = exponent of the segment's
// largest magnitude, and the integer c = round(x / q), |c| <= 2^S.  The
// matrix A takes S = 11 (c is then an exact TF32 integer) and the state B
// S = 7: every partial sum of a 64-term dot product of the two is an integer
// multiple of q_A q_B of magnitude at most 64 * 2^11 * 2^7 = 2^24, exactly
// representable in FP32, so the tensor core adds the segment's products
// without rounding.  The split is asymmetric because the matrix's rounding
// error (lo rounded to TF32) is the same for every group of the state and so
// changes the norm coherently, while the state's is independent from
// amplitude to amplitude.  The rounding to a multiple of q is (x + M) - M
// with M = 1.5 * 2^(E+24-S), whose ulp is q (round to nearest even, valid for
// |x| < 2^(E+1)).  lo = x - hi is exact in FP32 (|lo| <= q / 2) and is rounded
// to TF32 to nearest.  Segments below 2^-95 keep everything in lo.
constexpr int kSplitA = 11, kSplitB = 7;
template <int S>
__device__ __forceinline__ float seg_magic(float mx) {
    int e = static_cast<int>((__float_as_uint(mx) >> 23) & 0xFFu);
    e = e < 32 ? 32 : (e > 254 - (24 - S) ? 254 - (24 - S) : e);
    return __uint_as_float((static_cast<uint32_t>(e + 24 - S) << 23) | 0x400000u);
}
__device__ __forceinline__ void split_one(float x, float magic, float& hi, float& lo) {
    hi = __fsub_rn(__fadd_rn(x, magic), magic);
    lo = tf32_rna(__fsub_rn(x, hi));
}

// Shared-memory matrix descriptor: K-major, 128-byte swizzle, 8-row atoms
// 1024 bytes apart (stride byte offset), descriptor version 1.
__device__ __forceinline__ uint64_t sw128_desc(uint32_t saddr) {
    return static_cast<uint64_t>((saddr >> 4) & 0x3FFFu) | (static_cast<uint64_t>(1) << 16) |
           (static_cast<uint64_t>(1024 >> 4) << 32) | (static_cast<uint64_t>(1) << 46) |
           (static_cast<uint64_t>(2) << 61);
}

__device__ __forceinline__ uint64_t insert_zero(uint64_t v, int p) {
    uint64_t lo = v & ((1ull << p) - 1ull);
    return ((v >> p) << (p + 1)) | lo;
}

struct TcArgs {
    float2* psi;
    const float* mat;     // G, 2 * 4^k floats (row-major, interleaved), operator order
    int* err;
    uint64_t nchunks;
    uint64_t gbit[kChunkBits];   // global amplitude offset of chunk-local position p
    uint32_t sbit[kChunkBits];   // stage byte address (XOR) contribution of chunk-local position p
    uint32_t obit[kChunkBits];   // the same for the output staging
    int m, nx;                   // chunk-local positions: 0..m-1 and xpos[0..nx-1]
    int xpos[6];
    int kp[6];                   // chunk-local position of K bit b
    int rp[5];                   // chunk-local position of row bit b
    int vbit[6];                 // operator bit of K bit b (b < k; for k = 5, K bit 5 is the group bit)
    int k;
    // Copy unit U = lane + 32 u (16 bytes: elements 2U, 2U+1): the parts of its global offset, stage
    // address and output staging address given by u's bits (chunk-local positions 6..10), read at
    // compile-time u, so they enter the instructions from the parameter bank
    uint64_t gi[32];
    uint32_t si[32];
    uint32_t oi[32];
};

__device__ __forceinline__ uint64_t chunk_base(const TcArgs& a, uint64_t t) {
    uint64_t b = t << a.m;
#pragma unroll
    for (int e = 0; e < 6; ++e)
        if (e < a.nx) b = insert_zero(b, a.xpos[e]);
    return b;
}

// Entry [2 nu + s][2 kap + t] of A: the real embedding of G in the K-bit
// numbering (k = 5: blockdiag(R, R), the block given by bit 5).  perm maps a
// K-bit index to the operator index (bit b to bit vbit[b]); gs is G in shared
// memory.
__device__ __forceinline__ float a_entry(const TcArgs& a, const float2* gs, const int* perm, int nu, int kap, int s,
                                         int t) {
    if (a.k == 5 && (nu >> 5) != (kap >> 5)) return 0.f;
    const int m = a.k == 5 ? 31 : 63;
    const float2 g = gs[(perm[nu & m] << a.k) + perm[kap & m]];
    return s == 0 ? (t == 0 ? g.x : -g.y) : (t == 0 ? g.y : g.x);
}

// PAIR: chunk-local position 0 is a K bit (a target at position 0), so the
// two amplitudes of a K pair are one 16-byte unit of the stage.
template <bool PAIR>
__global__ void __launch_bounds__(kThreads, 1) k_apply_tc(TcArgs a) {
    extern __shared__ unsigned char smem_raw[];
    const uint32_t raw_addr = smem_u32(smem_raw);
    unsigned char* sm = smem_raw + ((1024u - (raw_addr & 1023u)) & 1023u);
    unsigned char* Bsm = sm + OFF_B;
    unsigned char* Raw = sm + OFF_RAW;
    const uint32_t bar0 = smem_u32(sm + OFF_BARS);
    auto bar = [&](int i) { return bar0 + 8u * static_cast<uint32_t>(i); };
    uint32_t* tmem_slot = reinterpret_cast<uint32_t*>(sm + OFF_MISC);
    volatile int* abort_flag = reinterpret_cast<volatile int*>(sm + OFF_MISC + 4);

    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;

    if (tid == 0) {
        for (int i = 0; i < kNR; ++i) {
            mbar_init(bar(BAR_RFULL + i), 32 * kProducers);   // every producer lane
            mbar_init(bar(BAR_REMPTY + i), 128);   // the converting team
        }
        for (int i = 0; i < kNB; ++i) {
            mbar_init(bar(BAR_BFULL + i), 256);         // both converter teams
            mbar_init(bar(BAR_BEMPTY + i), kIssuers);   // one commit per issuer
        }
        mbar_init(bar(BAR_DFULL), kIssuers);
        mbar_init(bar(BAR_DEMPTY), 256);        // both epilogue groups
        mbar_init(bar(BAR_AREADY), 256);   // both epilogue groups build A
        mbar_init(bar(BAR_FIN), kIssuers);
        *abort_flag = 0;
        fence_mbar_init();
    }
    if (warp == kMmaWarp) {
        tmem_alloc(smem_u32(tmem_slot), kTmemCols);
        tmem_relinquish();
    }
    // G into B buffer 0 with coalesced loads; the epilogue builds A from
    // there (scattered reads of G from global memory took about 0.17 ms per
    // launch), and the converters write B only once A is ready
    const float2* g_sm = reinterpret_cast<const float2*>(Bsm);
    int* perm = reinterpret_cast<int*>(Bsm + 32768);   // after G (at most 32 KiB)
    for (int i = tid; i < (1 << (2 * a.k)); i += kThreads)
        reinterpret_cast<float2*>(Bsm)[i] = reinterpret_cast<const float2*>(a.mat)[i];
    if (tid < 64) {
        int o = 0;
#pragma unroll
        for (int b = 0; b < 6; ++b)
            if (b < a.k && ((tid >> b) & 1)) o |= 1 << a.vbit[b];
        perm[tid] = o;
    }
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    const uint32_t tmem = *tmem_slot;

    const uint64_t nch = a.nchunks;
    const uint64_t my = nch > blockIdx.x ? (nch - blockIdx.x + gridDim.x - 1) / gridDim.x : 0;

    if (warp >= kProdWarp && warp < kProdWarp + kProducers) {
        // ---------------- producers ----------------
        constexpr int kU = 32 / kProducers;
        const int u0 = kU * (warp - kProdWarp);   // this warp's copies: units lane + 32 u, u0 <= u < u0 + kU
        uint64_t gl = 0;   // this lane's part of its units (unit bits 0..4 = positions 1..5)
        uint32_t sl = 0;
#pragma unroll
        for (int b = 0; b < 5; ++b)
            if ((lane >> b) & 1) {
                gl |= a.gbit[1 + b];
                sl ^= a.sbit[1 + b];
            }
        const uint32_t raw0 = smem_u32(Raw);
        for (uint64_t i = 0; i < my; ++i) {
            const int s = static_cast<int>(i % kNR);
            if (i >= kNR) {
                const bool ok = mbar_wait(bar(BAR_REMPTY + s), static_cast<uint32_t>(i / kNR - 1) & 1u, abort_flag,
                                          a.err, 21, i);
                if (!__all_sync(0xffffffffu, ok)) break;
            }
            const uint64_t base = chunk_base(a, blockIdx.x + i * gridDim.x) | gl;
            const uint32_t d0 = raw0 + static_cast<uint32_t>(s) * kRawBytes;
            // this warp's units at compile-time indices (one copy of the loop per producer warp)
            auto copy_units = [&](auto pw) {
                constexpr int v0 = kU * decltype(pw)::value;
#pragma unroll
                for (int u = v0; u < v0 + kU; ++u)
                    if (dbg::in_bounds(base | a.gi[u], 2, a.nchunks << kChunkBits, 21))
                        cp_async16(d0 + (sl ^ a.si[u]), a.psi + (base | a.gi[u]));
            };
            switch (u0 / kU) {
                case 0: copy_units(std::integral_constant<int, 0>{}); break;
                case 1: copy_units(std::integral_constant<int, 1>{}); break;
                case 2: copy_units(std::integral_constant<int, 2>{}); break;
                default: copy_units(std::integral_constant<int, 3>{}); break;
            }
            cp_async_arrive_noinc(bar(BAR_RFULL + s));
        }
        cp_async_wait_all();   // no copy may land after the CTA has left
    } else if (warp < kConvWarps) {
        // ---------------- converters ----------------
        const int team = warp >> 2, wt = warp & 3;
        // this lane: row rho, K quarter 2 h + sub (16 amplitudes); the two
        // quarters of a K half sit in lanes l and l ^ 16 of one warp
        const int rho = 16 * (wt & 1) + (lane & 15), h = wt >> 1, sub = lane >> 4;
        uint32_t srow = 0;
#pragma unroll
        for (int b = 0; b < 5; ++b)
            if ((rho >> b) & 1) srow ^= a.sbit[a.rp[b]];
        if (h) srow ^= a.sbit[a.kp[5]];
        if (sub) srow ^= a.sbit[a.kp[4]];
        uint32_t ks[4];
#pragma unroll
        for (int b = 0; b < 4; ++b) ks[b] = a.sbit[a.kp[b]];
        auto kaddr = [&](int c) {   // c < 16 is a compile-time constant in the unrolled loops
            uint32_t o = 0;
#pragma unroll
            for (int b = 0; b < 4; ++b)
                if ((c >> b) & 1) o ^= ks[b];
            return o;
        };
        const uint32_t brow = static_cast<uint32_t>(rho >> 3) * 1024u + static_cast<uint32_t>(rho & 7) * 128u;
        const uint32_t bsw = static_cast<uint32_t>(rho & 7);
        const uint64_t npairs = (my + 1) / 2;
        unsigned char* Bteam = Bsm + 4096u * static_cast<uint32_t>(team);   // rows 32 team .. 32 team + 31
        for (uint64_t pr = 0; pr < npairs; ++pr) {
            const int bb = static_cast<int>(pr & 1);
            const uint64_t i = 2 * pr + static_cast<uint64_t>(team);   // this team's chunk of the pair
            float x[32];
            const bool have = i < my;   // the last pair of an odd count has one chunk
            if (have) {
                const int s = static_cast<int>(i % kNR);
                const bool ok =
                    mbar_wait(bar(BAR_RFULL + s), static_cast<uint32_t>(i / kNR) & 1u, abort_flag, a.err, 22, i);
                if (!__all_sync(0xffffffffu, ok)) break;
                // x[2 c + t] = part t of amplitude 32 h + 16 sub + c of the row
                const unsigned char* stg = Raw + static_cast<uint32_t>(s) * kRawBytes;   // element at srow ^ kaddr
                if (PAIR) {
#pragma unroll
                    for (int c2 = 0; c2 < 8; ++c2) {
                        const float4 v = *reinterpret_cast<const float4*>(stg + (srow ^ kaddr(2 * c2)));
                        x[4 * c2] = v.x;
                        x[4 * c2 + 1] = v.y;
                        x[4 * c2 + 2] = v.z;
                        x[4 * c2 + 3] = v.w;
                    }
                } else {
#pragma unroll
                    for (int c = 0; c < 16; ++c) {
                        const float2 v = *reinterpret_cast<const float2*>(stg + (srow ^ kaddr(c)));
                        x[2 * c] = v.x;
                        x[2 * c + 1] = v.y;
                    }
                }
                mbar_arrive(bar(BAR_REMPTY + s));   // the values are in registers: the stage may refill
            }
            if (pr == 0) {   // B buffer 0 holds G until A is built
                const bool ok = mbar_wait(bar(BAR_AREADY), 0, abort_flag, a.err, 28, i);
                if (!__all_sync(0xffffffffu, ok)) break;
            }
            if (pr >= kNB) {   // the MMAs of pair pr - 2 have read this buffer
                const bool ok = mbar_wait(bar(BAR_BEMPTY + bb), static_cast<uint32_t>(pr / kNB - 1) & 1u, abort_flag,
                                          a.err, 23, i);
                if (!__all_sync(0xffffffffu, ok)) break;
            }
            unsigned char* Bhi = Bteam + static_cast<uint32_t>(bb) * kBBytes;
            unsigned char* Blo = Bhi + kHalfB;
            // the segment maximum spans the K half: both quarters (uniform across the warp)
            float mx = 0.f;
            if (have) {
                float m4[4] = {0.f, 0.f, 0.f, 0.f};
#pragma unroll
                for (int j = 0; j < 32; ++j) m4[j & 3] = fmaxf(m4[j & 3], fabsf(x[j]));
                mx = fmaxf(fmaxf(m4[0], m4[1]), fmaxf(m4[2], m4[3]));
            }
            mx = fmaxf(mx, __shfl_xor_sync(0xffffffffu, mx, 16));
            if (have) {
                const float magic = seg_magic<kSplitB>(mx);
                // K = 64 h + 32 sub + 4 u + (0..3): K block 2 h + sub, 16-byte unit u
#pragma unroll
                for (int u = 0; u < 8; ++u) {
                    float4 hv, lv;
                    split_one(x[4 * u], magic, hv.x, lv.x);
                    split_one(x[4 * u + 1], magic, hv.y, lv.y);
                    split_one(x[4 * u + 2], magic, hv.z, lv.z);
                    split_one(x[4 * u + 3], magic, hv.w, lv.w);
                    const uint32_t off = static_cast<uint32_t>(2 * h + sub) * kKBlock + brow +
                                         ((static_cast<uint32_t>(u) ^ bsw) << 4);
                    *reinterpret_cast<float4*>(Bhi + off) = hv;
                    *reinterpret_cast<float4*>(Blo + off) = lv;
                }
                fence_async_smem();   // the operand, visible to the tensor core
            }
            mbar_arrive(bar(BAR_BFULL + bb));
        }
    } else if (warp >= kMmaWarp && warp < kMmaWarp + kIssuers) {
        // ---------------- MMA issuers: product mi of every pair ----------------
        if (lane == 0) {
            const int mi = warp - kMmaWarp;   // 0: A_hi B_hi (two exact halves), 1: A_hi B_lo, 2: A_lo B_hi
            bool ok = mbar_wait(bar(BAR_AREADY), 0, abort_flag, a.err, 24);
            tc_fence_after();
            const uint32_t b0 = smem_u32(Bsm);
            const uint32_t acol = tmem + (mi == 2 ? COL_ALO : COL_AHI);
            const uint64_t npairs = (my + 1) / 2;
            const uint32_t dcol = tmem + COL_D + (mi == 0 ? 0u : 64u + 64u * mi);
            // B: hi for the main product and A_lo B_hi, lo for A_hi B_lo; the descriptor's
            // address field is addr / 16 below 2^14, so a K-step adds a constant to it
            const uint64_t bdesc0 = sw128_desc(b0 + (mi == 1 ? kHalfB : 0u));
            for (uint64_t pr = 0; pr < npairs && ok; ++pr) {
                const int bb = static_cast<int>(pr & 1);
                if (!mbar_wait(bar(BAR_BFULL + bb), static_cast<uint32_t>(pr / kNB) & 1u, abort_flag, a.err, 25, 2 * pr))
                    break;
                if (pr >= 1 &&
                    !mbar_wait(bar(BAR_DEMPTY), static_cast<uint32_t>(pr - 1) & 1u, abort_flag, a.err, 26, 2 * pr))
                    break;
                tc_fence_after();
                const uint64_t bdesc = bdesc0 + ((static_cast<uint64_t>(bb) * kBBytes) >> 4);
#pragma unroll
                for (int kk = 0; kk < 16; ++kk) {   // K-steps of 8
                    const uint64_t boff = (static_cast<uint64_t>(kk >> 2) * kKBlock + 32u * static_cast<uint64_t>(kk & 3)) >> 4;
                    const uint32_t dk = mi == 0 ? dcol + 64u * static_cast<uint32_t>(kk >> 3) : dcol;
                    const uint32_t acc = mi == 0 ? static_cast<uint32_t>((kk & 7) != 0) : static_cast<uint32_t>(kk != 0);
                    mma_tf32_ts(dk, acol + 8u * kk, bdesc + boff, kIdesc, acc);
                }
                mma_commit(bar(BAR_BEMPTY + bb));
                mma_commit(bar(BAR_DFULL));
            }
            // drain: no MMA may be in flight when the CTA tears down
            mma_commit(bar(BAR_FIN));
            const uint64_t t0 = global_ns();
            while (!mbar_try(bar(BAR_FIN), 0) && global_ns() - t0 < kWaitNs) {
            }
        }
        __syncwarp();
    } else {
        // ---------------- epilogue (warps 8-15) ----------------
        const int q = warp & 3;                  // tensor-memory lane quarter
        const int grp = (warp - kEpiWarp) >> 2;  // accumulator set / chunk parity of this group
        const uint32_t lane_t = tmem + (static_cast<uint32_t>(q * 32) << 16);
        {
            // A: row n = 32 q + lane of the embedding, hi and lo of K half grp
            const int n = 32 * q + lane, nu = n >> 1, s = n & 1, h = grp;
            float mx = 0.f;   // entry 2 kap + t of the half: kap = 32 h + (j >> 1), t = j & 1
#pragma unroll 8
            for (int j = 0; j < 64; ++j) mx = fmaxf(mx, fabsf(a_entry(a, g_sm, perm, nu, 32 * h + (j >> 1), s, j & 1)));
            const float magic = seg_magic<kSplitA>(mx);
#pragma unroll 1
            for (int c = 0; c < 4; ++c) {
                float hi[16], lo[16];
#pragma unroll
                for (int j = 0; j < 16; ++j)
                    split_one(a_entry(a, g_sm, perm, nu, 32 * h + 8 * c + (j >> 1), s, j & 1), magic, hi[j], lo[j]);
                tmem_st16(lane_t + COL_AHI + 64u * h + 16u * c, hi);
                tmem_st16(lane_t + COL_ALO + 64u * h + 16u * c, lo);
            }
            tmem_st_wait();
            tc_fence_before();
            mbar_arrive(bar(BAR_AREADY));
        }
        // The group writes its chunk into its staging area in the output
        // layout (lane: output part lane & 1 of amplitude nu, register: row),
        // then each warp stores a quarter of the chunk's 16-byte units in
        // chunk-local order, mirroring the producers' copies.
        unsigned char* ost = sm + OFF_STG + static_cast<uint32_t>(grp) * kOutBytes;
        const int nu = 16 * q + (lane >> 1);
        uint32_t onu = 4u * static_cast<uint32_t>(lane & 1);
#pragma unroll
        for (int b = 0; b < 6; ++b)
            if ((nu >> b) & 1) onu ^= a.obit[a.kp[b]];
        uint32_t orow[5];
#pragma unroll
        for (int b = 0; b < 5; ++b) orow[b] = a.obit[a.rp[b]];
        uint64_t gl = 0;   // this lane's part of its units (positions 1..5)
        uint32_t ol = 0;
#pragma unroll
        for (int b = 0; b < 5; ++b)
            if ((lane >> b) & 1) {
                gl |= a.gbit[1 + b];
                ol ^= a.obit[1 + b];
            }
        const uint32_t gbar = 1u + static_cast<uint32_t>(grp);   // named barrier of the group (128 threads)
        const uint32_t dcol = lane_t + COL_D + 32u * static_cast<uint32_t>(grp);   // this group's chunk of a pair
        const uint64_t npairs = (my + 1) / 2;
        for (uint64_t pr = 0; pr < npairs; ++pr) {
            const uint64_t i = 2 * pr + static_cast<uint64_t>(grp);
            bool ok = mbar_wait(bar(BAR_DFULL), static_cast<uint32_t>(pr) & 1u, abort_flag, a.err, 27, i);
            // one decision for the whole group (its warps meet at a named barrier
            // below); as a barrier it also means that the group's stores of its
            // previous chunk have read the staging area
            if (!group_all(gbar, 128, ok)) break;
            if (i >= my) {   // the last pair of an odd count has one chunk
                mbar_arrive(bar(BAR_DEMPTY));
                continue;
            }
            tc_fence_after();
            // output part (lane & 1) of amplitude nu, rows 8 hh .. 8 hh + 7
#pragma unroll
            for (int hh = 0; hh < 4; ++hh) {
                uint32_t m0[8], m1[8], ca[8], cb[8];
                tmem_ld8(dcol + 8u * hh, m0);
                tmem_ld8(dcol + 64u + 8u * hh, m1);
                tmem_ld8(dcol + 128u + 8u * hh, ca);
                tmem_ld8(dcol + 192u + 8u * hh, cb);
                tmem_ld_wait();
#pragma unroll
                for (int r = 0; r < 8; ++r) {
                    const int row = 8 * hh + r;
                    uint32_t ad = onu;
#pragma unroll
                    for (int b = 0; b < 5; ++b)
                        if ((row >> b) & 1) ad ^= orow[b];
                    *reinterpret_cast<float*>(ost + ad) =
                        __fadd_rn(__fadd_rn(__uint_as_float(m0[r]), __uint_as_float(m1[r])),
                                  __fadd_rn(__uint_as_float(ca[r]), __uint_as_float(cb[r])));
                }
            }
            tc_fence_before();
            mbar_arrive(bar(BAR_DEMPTY));
            group_sync(gbar, 128);   // the chunk is staged
            const uint64_t base = chunk_base(a, blockIdx.x + i * gridDim.x) | gl;
            // this warp's quarter of the units at compile-time indices
            auto store_units = [&](auto qq) {
                constexpr int v0 = 8 * decltype(qq)::value;
#pragma unroll
                for (int u = v0; u < v0 + 8; ++u)
                    if (dbg::in_bounds(base | a.gi[u], 2, a.nchunks << kChunkBits, 22))
                        __stcs(reinterpret_cast<float4*>(a.psi + (base | a.gi[u])),
                               *reinterpret_cast<const float4*>(ost + (ol ^ a.oi[u])));
            };
            switch (q) {
                case 0: store_units(std::integral_constant<int, 0>{}); break;
                case 1: store_units(std::integral_constant<int, 1>{}); break;
                case 2: store_units(std::integral_constant<int, 2>{}); break;
                default: store_units(std::integral_constant<int, 3>{}); break;
            }
        }
    }
    tc_fence_before();
    __syncthreads();
    if (warp == kMmaWarp) {
        tc_fence_after();
        tmem_dealloc(tmem, kTmemCols);
    }
}

// Stage byte address contributions of the 11 chunk-local positions: element
// l sits at 16-byte unit U = l >> 1 (byte 8 (l & 1) within it), in 128-byte
// line U >> 3 at slot (U & 7) ^ f(U >> 3), f linear.  Lanes of a converter
// warp differ in the row bits; f is chosen so that the row bits read
// together (16 lanes of 8-byte reads, or 8 lanes of 16-byte reads when
// position 0 is a K bit) land on distinct slots.
void stage_layout(const int* rp, bool pair, uint32_t* sbit) {
    uint32_t fvec[kChunkBits] = {};   // slot vector of line bit p - 4
    const int first = pair ? 0 : 1;
    uint32_t used = 0;
    for (int b = first; b < first + 3; ++b)
        if (rp[b] >= 1 && rp[b] <= 3) used |= 1u << (rp[b] - 1);
    for (int b = first; b < first + 3; ++b)
        if (rp[b] >= 4) {
            int j = 0;
            while ((used >> j) & 1u) ++j;
            used |= 1u << j;
            fvec[rp[b]] = 1u << j;
        }
    for (int p = 0; p < kChunkBits; ++p) {
        if (p == 0)
            sbit[p] = 8u;
        else if (p <= 3)
            sbit[p] = 16u << (p - 1);
        else
            sbit[p] = (128u << (p - 4)) ^ (fvec[p] << 4);
    }
}

// Output staging: the same element-in-unit and slot bits for positions 0..3
// (16-byte units read back in chunk-local order, 8 lanes on distinct slots),
// and slot vectors for the K positions at 4 and above among K bits 0..3 (the
// bits that vary across an epilogue warp's lanes), so that a warp's staging
// writes meet at most two to a bank.
void out_layout(const int* kp, uint32_t* obit) {
    uint32_t fvec[kChunkBits] = {};
    uint32_t used = 0;
    for (int b = 0; b < 4; ++b)
        if (kp[b] >= 1 && kp[b] <= 3) used |= 1u << (kp[b] - 1);
    for (int b = 0; b < 4; ++b)
        if (kp[b] >= 4) {
            int j = 0;
            while (j < 3 && ((used >> j) & 1u)) ++j;
            if (j < 3) {
                used |= 1u << j;
                fvec[kp[b]] = 1u << j;
            }
        }
    for (int p = 0; p < kChunkBits; ++p) {
        if (p == 0)
            obit[p] = 8u;
        else if (p <= 3)
            obit[p] = 16u << (p - 1);
        else
            obit[p] = (128u << (p - 4)) ^ (fvec[p] << 4);
    }
}

template <bool PAIR>
cudaError_t launch_pair(const TcArgs& a, uint64_t nchunks, cudaStream_t st, uint64_t* launches) {
    auto kern = k_apply_tc<PAIR>;
    cudaError_t e = set_smem_attr(reinterpret_cast<const void*>(kern), static_cast<int>(kSmem));
    if (e != cudaSuccess) return e;
    uint64_t grid = static_cast<uint64_t>(num_sms());   // one CTA per SM (all tensor memory)
    if (grid > nchunks) grid = nchunks;
    kern<<<static_cast<unsigned>(grid), kThreads, kSmem, st>>>(a);
    ++*launches;
    return cudaGetLastError();
}

}  // namespace

QSA_BOUNDS_READER(bounds_word_tc)

bool tc_available(qsa_state s, int k) { return (k == 5 || k == 6) && s->n >= kChunkBits; }

cudaError_t launch_apply_tc(float2* psi, int n, const int* phys, int k, const float* d_mat, int* d_err,
                            cudaStream_t st, uint64_t* launches) {
    if (k != 5 && k != 6) return cudaErrorNotSupported;
    if (n < kChunkBits) return cudaErrorInvalidValue;
    TileGeom g;
    if (!make_geom(n, phys, k, kChunkBits, &g) || g.T != kChunkBits || g.m < 5) return cudaErrorInvalidValue;
    TcArgs a{};
    a.psi = psi;
    a.mat = d_mat;
    a.err = d_err;
    a.nchunks = g.ntiles;
    a.m = g.m;
    a.nx = g.nx;
    a.k = k;
    for (int e = 0; e < 6; ++e) a.xpos[e] = g.xpos[e];
    for (int p = 0; p < kChunkBits; ++p) a.gbit[p] = p < g.m ? (1ull << p) : (1ull << g.xpos[p - g.m]);
    auto local_of = [&](int p) {
        if (p < g.m) return p;
        for (int e = 0; e < g.nx; ++e)
            if (g.xpos[e] == p) return g.m + e;
        return -1;
    };
    int tl[6], tls[6];
    bool is_t[kChunkBits] = {};
    for (int j = 0; j < k; ++j) {
        tl[j] = local_of(phys[j]);
        if (tl[j] < 0) return cudaErrorInvalidValue;
        tls[j] = tl[j];
        is_t[tl[j]] = true;
    }
    std::sort(tls, tls + k);
    int np[kChunkBits], nn = 0;
    for (int p = 0; p < kChunkBits; ++p)
        if (!is_t[p]) np[nn++] = p;
    for (int b = 0; b < k; ++b) {
        a.kp[b] = tls[b];
        for (int j = 0; j < k; ++j)
            if (tl[j] == tls[b]) a.vbit[b] = j;
    }
    if (k == 5) {
        a.kp[5] = np[5];
        a.vbit[5] = 0;
    }
    for (int b = 0; b < 5; ++b) a.rp[b] = np[b];
    const bool pair = tls[0] == 0;
    stage_layout(a.rp, pair, a.sbit);
    out_layout(a.kp, a.obit);
    for (int u = 0; u < 32; ++u) {
        a.gi[u] = 0;
        a.si[u] = a.oi[u] = 0;
        for (int b = 0; b < 5; ++b)
            if ((u >> b) & 1) {
                a.gi[u] |= a.gbit[6 + b];
                a.si[u] ^= a.sbit[6 + b];
                a.oi[u] ^= a.obit[6 + b];
            }
    }
    return pair ? launch_pair<true>(a, g.ntiles, st, launches) : launch_pair<false>(a, g.ntiles, st, launches);
}

}  // namespace qsa
