// Split-TF32 (3xTF32) fused dense update on tcgen05 tensor cores, k = 5, 6.
//
// The update of one group of 2^k amplitudes (§IV-B: M' = G M on the
// 2^k x 2^(N-k) view) is a real matrix-vector product after embedding
// complex numbers as 2x2 real blocks:  u[2c+t] = (Re, Im)(psi_c),
// R[2r+s][2c+t] = [[Re G, -Im G], [Im G, Re G]][s][t],  u' = R u.
// A tile of 128 groups is one GEMM  D (128 x 2^(k+1)) = U (128 x K) R^T with
// K = 2^(k+1):  the state tile is the MMA's A operand (M = 128 rows, one
// group per row, K-major), R is the B operand (N = K rows, K-major).  Both
// are split into hi/lo parts and D = U_hi R_hi^T + (U_lo R_hi^T + U_hi R_lo^T)
// (the three-product split-TF32 scheme of Ootomo & Yokota 2022, "Recovering
// single precision accuracy from Tensor Cores while surpassing the FP32
// theoretical peak performance").
//
// Tensor cores round their FP32 accumulation toward zero, which biases every
// rounded sum towards zero; over a deep circuit that shrinks the norm
// linearly with depth.  Two measures remove the bias from the dominant term:
//   - as the split-TF32 method prescribes, U_hi R_hi^T is accumulated outside
//     the tensor core: every segment of two K-steps (16 values of K) writes a
//     fresh partial product into one of NMAIN tensor-memory buffers and the
//     epilogue warps add the partials in FP32 with round-to-nearest;
//   - hi parts are block-quantised per 16-value segment (a shared
//     power-of-two quantum, integer multiples of magnitude <= 1024, as in
//     Ozaki-type splittings), so each 16-term partial and its 8-term half
//     are exactly representable FP32 numbers and the tensor core has
//     nothing to round.
// lo = x - hi (exact) is rounded to TF32 to nearest; the two small
// correction products (about 2^-10 of the result) accumulate in tensor
// memory, where their rounding is far below FP32 resolution of the output.
// Combinations are numbered by ascending tile-local target position, so a
// K-chunk (16 combinations) fixes the highest target bits and its 2048
// amplitudes run in address order.
//
// CTA roles (one persistent CTA per SM, 416 threads):
//   warps 0-3   loaders: copy each K-chunk in address order (16-byte
//               cp.async, mbarrier-tracked NR-stage ring), then thread g
//               gathers row g, splits it hi/lo and stores both into its
//               tensor-memory lane: the MMA's A operand (two chunk buffers);
//   warps 4-11  epilogue: warp w reads tensor-memory lanes 32*(w%4).. and
//               half (w-4)/4 of the columns, sums the partials, adds the
//               correction accumulator and writes the outputs back through
//               a small shared staging area, one coalesced run per store;
//   warp 12     allocates tensor memory and issues the MMAs (one thread);
//               B (the split R) stays in shared memory for the whole launch.
// Tensor memory (512 columns): NMAIN main partials + NCORR corrections of NK
// columns, and 128 columns of A (k = 6: 2 + 1, k = 5: 4 + 2).
// Every mbarrier wait is bounded; on timeout the CTA records an error code,
// drains its MMAs, frees tensor memory and returns.
#include <cuda_runtime.h>

#include <algorithm>
#include <cstdint>

#include "qsa_internal.h"
#include "qsa_runtime.h"

namespace qsa {

namespace {

constexpr int kTcThreads = 416;
constexpr int kEpiThreads = 256;
constexpr int kGroups = 128;                 // MMA M
constexpr uint32_t kWaitLimit = 1u << 22;    // try_wait rounds before giving up

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
        "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n selp.b32 %0, 1, 0, p;\n}\n"
        : "=r"(ok)
        : "r"(a), "r"(parity)
        : "memory");
    return ok != 0;
}
// Bounded wait; gives up (and raises the CTA abort word) after kWaitLimit
// rounds or as soon as another role has aborted.
__device__ bool mbar_wait(uint32_t a, uint32_t parity, volatile int* abort_flag, int* gerr, int code) {
    for (uint32_t i = 0; i < kWaitLimit; ++i) {
        if (mbar_try(a, parity)) return true;
        if (*abort_flag) return false;
    }
    *abort_flag = 1;
    atomicExch(gerr, code);
    return false;
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

// 32 lanes x 32 consecutive 32-bit columns (one row per thread).
__device__ __forceinline__ void tmem_ld32(uint32_t taddr, uint32_t* r) {
    asm volatile(
        "tcgen05.ld.sync.aligned.32x32b.x32.b32 "
        "{%0, %1, %2, %3, %4, %5, %6, %7, %8, %9, %10, %11, %12, %13, %14, %15, "
        "%16, %17, %18, %19, %20, %21, %22, %23, %24, %25, %26, %27, %28, %29, %30, %31}, [%32];\n"
        : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]),
          "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]), "=r"(r[15]),
          "=r"(r[16]), "=r"(r[17]), "=r"(r[18]), "=r"(r[19]), "=r"(r[20]), "=r"(r[21]), "=r"(r[22]), "=r"(r[23]),
          "=r"(r[24]), "=r"(r[25]), "=r"(r[26]), "=r"(r[27]), "=r"(r[28]), "=r"(r[29]), "=r"(r[30]), "=r"(r[31])
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

// Block split of S values (S <= 16: two MMA K-steps): hi = c * q with the
// shared quantum q = 2^(E-9), E = exponent of max |x|, and the integer
// c = round(x / q), |c| <= 1024.  Every dot product of two such segments, and
// every partial sum of it, is an integer multiple of q_a q_b of magnitude at
// most 16 * 2^20 = 2^24: exactly representable in FP32, so the tensor core
// adds the two K-steps of a segment without rounding and its round-toward-
// zero never engages on the main product.  The rounding to a multiple of q is
// (x + M) - M with M = 1.5 * 2^(E+14), whose ulp is q (round to nearest even,
// valid for |x| < 2^(E+1)).  lo = x - hi is exact in FP32 (|lo| <= q / 2) and
// is rounded to TF32 to nearest.  Segments below 2^-95 keep everything in lo.
struct SegQuant {
    float m;   // 1.5 * 2^(E+14)
};
__device__ __forceinline__ SegQuant seg_quant(float mx) {
    int e = static_cast<int>((__float_as_uint(mx) >> 23) & 0xFFu);
    e = e < 32 ? 32 : (e > 240 ? 240 : e);
    SegQuant sq;
    sq.m = __uint_as_float((static_cast<uint32_t>(e + 14) << 23) | 0x400000u);
    return sq;
}
__device__ __forceinline__ void split_one(float x, const SegQuant& sq, float& hi, float& lo) {
    hi = __fsub_rn(__fadd_rn(x, sq.m), sq.m);
    lo = tf32_rna(__fsub_rn(x, hi));
}
template <int S>
__device__ __forceinline__ void block_split(const float* x, float* hi, float* lo) {
    static_assert(S <= 16, "segment too long for an exact FP32 partial");
    float mx = 0.f;
#pragma unroll
    for (int i = 0; i < S; ++i) mx = fmaxf(mx, fabsf(x[i]));
    const SegQuant sq = seg_quant(mx);
#pragma unroll
    for (int i = 0; i < S; ++i) split_one(x[i], sq, hi[i], lo[i]);
}

// Shared-memory matrix descriptor: K-major, 128-byte swizzle, 8-row atoms
// 1024 bytes apart (stride byte offset), descriptor version 1.
__device__ __forceinline__ uint64_t sw128_desc(uint32_t saddr) {
    return static_cast<uint64_t>((saddr >> 4) & 0x3FFFu) | (static_cast<uint64_t>(1) << 16) |
           (static_cast<uint64_t>(1024 >> 4) << 32) | (static_cast<uint64_t>(1) << 46) |
           (static_cast<uint64_t>(2) << 61);
}
// Byte offset of 32-bit element kin (< 32) of row `row` in a K-major region
// of 128-byte rows with the 128-byte swizzle (16-byte chunk index XOR row%8).
__device__ __forceinline__ uint32_t sw128_off(uint32_t row, uint32_t kin) {
    return (row >> 3) * 1024u + (row & 7u) * 128u + ((((kin >> 2) ^ (row & 7u))) << 4) + ((kin & 3u) << 2);
}

__device__ __forceinline__ uint64_t insert_zero(uint64_t v, int p) {
    uint64_t lo = v & ((1ull << p) - 1ull);
    return ((v >> p) << (p + 1)) | lo;
}

struct TcArgs {
    float2* psi;
    const float* mat;   // G, 2 * 4^k floats (row-major, interleaved)
    int* err;
    uint64_t ntiles;
    int m, nx;
    int xpos[6];
    int tl[6];          // tile-local position of target j (V order)
    int tls[6];         // ascending
};

__device__ __forceinline__ uint64_t tc_tile_base(const TcArgs& a, uint64_t t) {
    uint64_t b = t << a.m;
#pragma unroll
    for (int e = 0; e < 6; ++e)
        if (e < a.nx) b = insert_zero(b, a.xpos[e]);
    return b;
}

template <int K>
struct TcCfg {
    static constexpr int D = 1 << K;                 // amplitudes per group
    static constexpr int NK = 2 * D;                 // GEMM N and K
    static constexpr int KC = NK / 32;               // K-chunks of 32 floats (16 combinations)
    static constexpr int KSEGS = NK / 16;            // exact main partials per tile
    static constexpr int NR = K == 6 ? 5 : 8;        // raw chunk stages
    static constexpr int NMAIN = K == 6 ? 2 : 4;     // main partial buffers
    static constexpr int NCORR = K == 6 ? 1 : 2;     // correction accumulators
    static constexpr uint32_t B_REGION = NK * 128;   // one K-block of B
    static constexpr uint32_t B_BYTES = KC * B_REGION;
    static constexpr uint32_t RAW_BYTES = kGroups * 128;   // one chunk: 2048 complex64 in address order
    // tensor memory: main partials, correction accumulators, and the A operand
    // (two chunk buffers of 32 hi + 32 lo columns)
    static constexpr uint32_t COL_MAIN = 0, COL_CORR = NMAIN * NK, COL_A = COL_CORR + NCORR * NK;
    static constexpr uint32_t TMEM_COLS = COL_A + 128;
    static_assert(TMEM_COLS == 512, "one CTA owns all tensor memory of its SM");
    static constexpr uint32_t IDESC = (1u << 4)      // D: FP32
                                      | (2u << 7)    // A: TF32
                                      | (2u << 10)   // B: TF32
                                      | (static_cast<uint32_t>(NK >> 3) << 17) |
                                      (static_cast<uint32_t>(kGroups >> 4) << 24);
    // per epilogue warp: 256 staged outputs, one padding slot per 32
    static constexpr uint32_t STAGE_ELEMS = 256 + 8;
    // shared memory carve-up (from a 1024-byte aligned base)
    static constexpr uint32_t OFF_BLO = B_BYTES, OFF_RAW = 2 * B_BYTES;
    static constexpr uint32_t OFF_RUNOFF = OFF_RAW + NR * RAW_BYTES;
    static constexpr uint32_t OFF_LOFF = OFF_RUNOFF + 64 * 8;
    static constexpr uint32_t OFF_CPY = OFF_LOFF + 64 * 4;   // copy offsets (8), row read slots (16)
    static constexpr uint32_t OFF_BARS = OFF_CPY + 8 * 8 + 16 * 4;
    // barriers: A chunk full/empty (2+2), main full/empty (NMAIN+NMAIN),
    // correction full/empty (NCORR+NCORR), raw stage full/empty (NR+NR), drain (1)
    static constexpr int BAR_FULL = 0, BAR_EMPTY = 2, BAR_MFULL = 4, BAR_MEMPTY = 4 + NMAIN,
                         BAR_CFULL = 4 + 2 * NMAIN, BAR_CEMPTY = BAR_CFULL + NCORR, BAR_RFULL = BAR_CEMPTY + NCORR,
                         BAR_REMPTY = BAR_RFULL + NR, BAR_FIN = BAR_REMPTY + NR, NBARS = BAR_FIN + 1;
    static constexpr uint32_t OFF_MISC = OFF_BARS + NBARS * 8;   // tensor-memory address, abort word
    static constexpr uint32_t OFF_STAGE = OFF_MISC + 16;
    static constexpr size_t SMEM = 1024 + OFF_STAGE + kEpiThreads / 32 * STAGE_ELEMS * 8;
};

template <int K>
__global__ void __launch_bounds__(kTcThreads, 1) k_apply_tc(TcArgs a) {
    using C = TcCfg<K>;
    constexpr int D = C::D, NK = C::NK, KC = C::KC, NR = C::NR, NMAIN = C::NMAIN, NCORR = C::NCORR,
                  HALF = NK / 2;
    extern __shared__ unsigned char smem_raw[];
    const uint32_t raw = smem_u32(smem_raw);
    unsigned char* sm = smem_raw + ((1024u - (raw & 1023u)) & 1023u);
    unsigned char* Bhi = sm;
    unsigned char* Blo = sm + C::OFF_BLO;
    unsigned char* Raw = sm + C::OFF_RAW;   // [stage][row g][16 complex64]
    uint64_t* runoff = reinterpret_cast<uint64_t*>(sm + C::OFF_RUNOFF);
    int* loff = reinterpret_cast<int*>(sm + C::OFF_LOFF);
    uint64_t* cpy_goff = reinterpret_cast<uint64_t*>(sm + C::OFF_CPY);
    uint32_t* rd_slot = reinterpret_cast<uint32_t*>(sm + C::OFF_CPY + 8 * 8);
    const uint32_t bar0 = smem_u32(sm + C::OFF_BARS);
    auto bar = [&](int i) { return bar0 + 8u * static_cast<uint32_t>(i); };
    uint32_t* tmem_slot = reinterpret_cast<uint32_t*>(sm + C::OFF_MISC);
    volatile int* abort_flag = reinterpret_cast<volatile int*>(sm + C::OFF_MISC + 4);
    float2* stage = reinterpret_cast<float2*>(sm + C::OFF_STAGE);

    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;

    // Combinations are numbered in ascending tile-local target position
    // (bit i of c <-> position tls[i]); vpos[i] is the operator's own index of
    // that target, so combination c is the operator's basis index vo(c).
    int vpos[6];
#pragma unroll
    for (int i = 0; i < 6; ++i) {
        vpos[i] = 0;
#pragma unroll
        for (int j = 0; j < K; ++j)
            if (i < K && a.tl[j] == a.tls[i]) vpos[i] = j;
    }
    auto vo = [&](int c) {
        int r = 0;
#pragma unroll
        for (int i = 0; i < K; ++i) r |= ((c >> i) & 1) << vpos[i];
        return r;
    };

    for (int r = tid; r < (1 << a.nx); r += blockDim.x) {
        uint64_t off = 0;
#pragma unroll
        for (int e = 0; e < 6; ++e)
            if (e < a.nx && ((r >> e) & 1)) off |= 1ull << a.xpos[e];
        runoff[r] = off;
    }
    for (int c = tid; c < D; c += blockDim.x) {
        int o = 0;
#pragma unroll
        for (int i = 0; i < K; ++i)
            if ((c >> i) & 1) o |= 1 << a.tls[i];
        loff[c] = o;
    }
    // Chunk copies: a K-chunk holds the 2048 amplitudes whose tile-local index
    // l has the chunk's combination bits tls[4..k-1] fixed; element e is l
    // with those bits squeezed out, so e runs in address order.  The raw stage
    // keeps e in address order, 16-byte units XOR-swizzled within 128-byte
    // rows (unit ^= row % 8); thread t copies units t + 128 i, i < 8.  Global
    // offsets and stage slots are bitwise linear in e, so each splits into a
    // per-thread part and a shared table.
    auto gbit = [&](int p) -> uint64_t { return p < a.m ? (1ull << p) : (1ull << a.xpos[p - a.m]); };
    auto goff_of = [&](uint32_t l) {
        uint64_t o = 0;
        for (int p = 0; p < 7 + K; ++p)
            if ((l >> p) & 1u) o |= gbit(p);
        return o;
    };
    auto spread = [&](uint32_t e) {   // element index -> tile-local index
#pragma unroll
        for (int q = 4; q < K; ++q) e = static_cast<uint32_t>(insert_zero(e, a.tls[q]));
        return e;
    };
    auto squeeze = [&](uint32_t l) {   // tile-local index (fixed bits 0) -> element index
        uint32_t e = 0;
        int kb = 0;
        for (int p = 0; p < 7 + K; ++p) {
            bool fixed = false;
#pragma unroll
            for (int q = 4; q < K; ++q) fixed |= (p == a.tls[q]);
            if (!fixed) e |= ((l >> p) & 1u) << kb++;
        }
        return e;
    };
    auto slot_of = [](uint32_t e) { return ((((e >> 1) ^ ((e >> 4) & 7u)) << 4) | ((e & 1u) << 3)); };
    if (tid < 8) cpy_goff[tid] = goff_of(spread(static_cast<uint32_t>(tid) << 8));
    if (tid >= 32 && tid < 48) {   // combination c4 of a row: its element part and stage slot
        const int c4 = tid - 32;
        uint32_t l = 0;
#pragma unroll
        for (int q = 0; q < 4; ++q) l |= ((static_cast<uint32_t>(c4) >> q) & 1u) << a.tls[q];
        rd_slot[c4] = slot_of(squeeze(l));
    }
    // B operand: the real embedding R of G in the sorted numbering, split hi / lo.
    const float2* G = reinterpret_cast<const float2*>(a.mat);
    for (int e = tid; e < NK * (NK / 16); e += blockDim.x) {
        const int n = e / (NK / 16), s16 = e - n * (NK / 16);   // row n, segment s16 (two K-steps)
        const int row = vo(n >> 1) * D;
        float x[16], hi[16], lo[16];
#pragma unroll
        for (int i = 0; i < 16; ++i) {
            const int kk = 16 * s16 + i;
            const float2 g = G[row + vo(kk >> 1)];
            x[i] = (n & 1) ? ((kk & 1) ? g.x : g.y) : ((kk & 1) ? -g.y : g.x);
        }
        block_split<16>(x, hi, lo);
#pragma unroll
        for (int i = 0; i < 16; ++i) {
            const int kk = 16 * s16 + i;
            const uint32_t off = static_cast<uint32_t>(kk >> 5) * C::B_REGION + sw128_off(n, kk & 31);
            *reinterpret_cast<float*>(Bhi + off) = hi[i];
            *reinterpret_cast<float*>(Blo + off) = lo[i];
        }
    }
    if (tid == 0) {
        for (int i = 0; i < 2; ++i) {
            mbar_init(bar(C::BAR_FULL + i), 128);
            mbar_init(bar(C::BAR_EMPTY + i), 1);
        }
        for (int i = 0; i < NMAIN; ++i) {
            mbar_init(bar(C::BAR_MFULL + i), 1);
            mbar_init(bar(C::BAR_MEMPTY + i), kEpiThreads);
        }
        for (int i = 0; i < NCORR; ++i) {
            mbar_init(bar(C::BAR_CFULL + i), 1);
            mbar_init(bar(C::BAR_CEMPTY + i), kEpiThreads);
        }
        for (int i = 0; i < NR; ++i) {
            mbar_init(bar(C::BAR_RFULL + i), 128);
            mbar_init(bar(C::BAR_REMPTY + i), 128);
        }
        mbar_init(bar(C::BAR_FIN), 1);
        *abort_flag = 0;
        fence_mbar_init();
    }
    fence_async_smem();
    if (warp == 12) {
        tmem_alloc(smem_u32(tmem_slot), C::TMEM_COLS);
        tmem_relinquish();
    }
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    const uint32_t tmem = *tmem_slot;

    const uint64_t ntiles = a.ntiles;
    const uint64_t my_tiles = ntiles > blockIdx.x ? (ntiles - blockIdx.x + gridDim.x - 1) / gridDim.x : 0;
    const uint32_t mmask = (1u << a.m) - 1u;

    if (warp < 4) {
        // ---------------- loaders ----------------
        // The loaders copy every K-chunk in address order (8-byte cp.async,
        // consecutive threads on consecutive amplitudes) into an NR-stage raw
        // ring, NR - 1 chunks ahead; thread g then reads row g, splits it into
        // hi / lo and writes both into its tensor-memory lane (the MMA's A
        // operand, two chunk buffers).
        const int g = tid;
        const uint64_t goffT = goff_of(spread(static_cast<uint32_t>(tid) << 1));
        const uint32_t sdstT = slot_of(static_cast<uint32_t>(tid) << 1);
        uint32_t lbg = static_cast<uint32_t>(g);   // row g's own tile-local bits (targets zero)
#pragma unroll
        for (int j = 0; j < K; ++j) lbg = static_cast<uint32_t>(insert_zero(lbg, a.tls[j]));
        const uint32_t rslot = slot_of(squeeze(lbg));
        const uint64_t gq4 = gbit(a.tls[4]), gq5 = K == 6 ? gbit(a.tls[K - 1]) : 0ull;
        const uint32_t raw0 = smem_u32(Raw);
        uint64_t base_t = ~0ull, base_v = 0;   // the tile base, formed once per tile
        auto issue = [&](uint64_t idx, int slot) {
            const uint64_t t = blockIdx.x + (idx / KC) * gridDim.x;
            const int j = static_cast<int>(idx % KC);
            if (t != base_t) {
                base_t = t;
                base_v = tc_tile_base(a, t);
            }
            const uint64_t o0 = base_v | ((j & 1) ? gq4 : 0ull) | ((j & 2) ? gq5 : 0ull) | goffT;
            const uint32_t d0 = raw0 + static_cast<uint32_t>(slot) * C::RAW_BYTES;
#pragma unroll
            for (int i = 0; i < 8; ++i)   // unit t + 128 i: element 2t + 256 i, slot part 2048 i
                cp_async16(d0 + (sdstT ^ (static_cast<uint32_t>(i) << 11)), a.psi + (o0 | cpy_goff[i]));
            cp_async_arrive_noinc(bar(C::BAR_RFULL + slot));
        };
        const uint64_t total = my_tiles * KC;
#pragma unroll
        for (int s0 = 0; s0 < NR; ++s0)
            if (static_cast<uint64_t>(s0) < total) issue(s0, s0);
        const uint32_t lane_a = tmem + (static_cast<uint32_t>(warp * 32) << 16) + C::COL_A;
        for (uint64_t idx = 0; idx < total; ++idx) {
            const int slot = static_cast<int>(idx % NR);
            const bool wr = mbar_wait(bar(C::BAR_RFULL + slot), static_cast<uint32_t>(idx / NR) & 1u, abort_flag,
                                      a.err, 7);
            if (!__all_sync(0xffffffffu, wr)) break;
            float2 v[16];
            const unsigned char* stg0 = Raw + static_cast<uint32_t>(slot) * C::RAW_BYTES;
#pragma unroll
            for (int c4 = 0; c4 < 16; ++c4) v[c4] = *reinterpret_cast<const float2*>(stg0 + (rslot ^ rd_slot[c4]));
            mbar_arrive(bar(C::BAR_REMPTY + slot));
            // refill the previous chunk's stage (every loader has read it by now)
            if (idx >= 1 && idx - 1 + NR < total) {
                const int ps = static_cast<int>((idx - 1) % NR);
                const bool we = mbar_wait(bar(C::BAR_REMPTY + ps), static_cast<uint32_t>((idx - 1) / NR) & 1u,
                                          abort_flag, a.err, 8);
                if (!__all_sync(0xffffffffu, we)) break;
                issue(idx - 1 + NR, ps);
            }
            const uint32_t b = static_cast<uint32_t>(idx & 1), f = static_cast<uint32_t>(idx >> 1);
            // tcgen05.st is warp-collective: leave together if any lane gave up
            const bool w = f < 1 || mbar_wait(bar(C::BAR_EMPTY + b), (f - 1) & 1, abort_flag, a.err, 1);
            if (!__all_sync(0xffffffffu, w)) break;
            tc_fence_after();
#pragma unroll
            for (int s16 = 0; s16 < 2; ++s16) {   // the chunk's 2 segments of 16 floats
                const float2* x = v + 8 * s16;
                float mx = 0.f;
#pragma unroll
                for (int i = 0; i < 8; ++i) mx = fmaxf(mx, fmaxf(fabsf(x[i].x), fabsf(x[i].y)));
                const SegQuant sq = seg_quant(mx);
                float h[16], l[16];
#pragma unroll
                for (int i = 0; i < 8; ++i) {
                    split_one(x[i].x, sq, h[2 * i], l[2 * i]);
                    split_one(x[i].y, sq, h[2 * i + 1], l[2 * i + 1]);
                }
                tmem_st16(lane_a + b * 64 + 16 * s16, h);
                tmem_st16(lane_a + b * 64 + 32 + 16 * s16, l);
            }
            tmem_st_wait();
            tc_fence_before();
            mbar_arrive(bar(C::BAR_FULL + b));
        }
        cp_async_wait_all();   // no copy may land after the CTA has left
    } else if (warp < 12) {
        // ---------------- epilogue ----------------
        const int qw = warp & 3;              // tensor-memory lane quarter
        const int half = (warp - 4) >> 2;     // column half
        const uint32_t lane_base = tmem + (static_cast<uint32_t>(qw * 32) << 16) + half * HALF;
        // Store rounds: the outputs (g = 32 qw + lane, 8 combinations) of one
        // round vary in the 5 lowest non-target local bits and in positions
        // tls[0..2]; rank r numbers them in ascending local position.
        float2* stg = stage + (warp - 4) * C::STAGE_ELEMS;
        uint32_t tmask = 0;
#pragma unroll
        for (int j = 0; j < K; ++j) tmask |= 1u << a.tls[j];
        uint32_t vmask = (1u << a.tls[0]) | (1u << a.tls[1]) | (1u << a.tls[2]);
        uint32_t rank_g = 0;
        {
            int kb = 0;
            for (int b = 0; b < 7 + K && kb < 5; ++b)
                if (!((tmask >> b) & 1u)) {
                    vmask |= 1u << b;
                    ++kb;
                }
            kb = 0;
            for (int b = 0; b < 7 + K && kb < 5; ++b)
                if (!((tmask >> b) & 1u)) {
                    rank_g |= ((static_cast<uint32_t>(lane) >> kb) & 1u) << __popc(vmask & ((1u << b) - 1u));
                    ++kb;
                }
        }
        const uint32_t rc0 = 1u << __popc(vmask & ((1u << a.tls[0]) - 1u));
        const uint32_t rc1 = 1u << __popc(vmask & ((1u << a.tls[1]) - 1u));
        const uint32_t rc2 = 1u << __popc(vmask & ((1u << a.tls[2]) - 1u));
        // local position of rank bit q, and the global offset of each rank bit
        auto goff1 = [&](uint32_t l) -> uint64_t { return (l & mmask) | runoff[l >> a.m]; };
        uint64_t goL = 0, gb5 = 0, gb6 = 0, gb7 = 0;
        {
            int q = 0;
            for (int b = 0; b < 7 + K; ++b)
                if ((vmask >> b) & 1u) {
                    const uint64_t gq = goff1(1u << b);
                    if (q < 5 && ((lane >> q) & 1)) goL |= gq;
                    if (q == 5) gb5 = gq;
                    if (q == 6) gb6 = gq;
                    if (q == 7) gb7 = gq;
                    ++q;
                }
        }
        // group bits above the lowest five (the lane-quarter index qw)
        uint32_t lfix = static_cast<uint32_t>(qw) << 5;
#pragma unroll
        for (int j = 0; j < K; ++j) lfix = static_cast<uint32_t>(insert_zero(lfix, a.tls[j]));
        uint64_t sc = 0;   // global segment counter (main buffers)
        bool ok = true;
        for (uint64_t i = 0; i < my_tiles && ok; ++i) {
            float acc[HALF];
#pragma unroll
            for (int c = 0; c < HALF; ++c) acc[c] = 0.f;
#pragma unroll 1
            for (int s = 0; s < C::KSEGS; ++s, ++sc) {
                const uint32_t mb = static_cast<uint32_t>(sc % NMAIN), mu = static_cast<uint32_t>(sc / NMAIN);
                const bool w = mbar_wait(bar(C::BAR_MFULL + mb), mu & 1, abort_flag, a.err, 2);
                // tcgen05.ld is warp-collective: leave together if any lane gave up
                if (!__all_sync(0xffffffffu, w)) {
                    ok = false;
                    break;
                }
                tc_fence_after();
                uint32_t r[HALF];
#pragma unroll
                for (int h = 0; h < HALF / 32; ++h) tmem_ld32(lane_base + C::COL_MAIN + mb * NK + 32 * h, r + 32 * h);
                tmem_ld_wait();
                tc_fence_before();
                mbar_arrive(bar(C::BAR_MEMPTY + mb));
#pragma unroll
                for (int c = 0; c < HALF; ++c) acc[c] += __uint_as_float(r[c]);
            }
            if (!ok) break;
            const uint32_t d = static_cast<uint32_t>(i % NCORR), u = static_cast<uint32_t>(i / NCORR);
            const bool w = mbar_wait(bar(C::BAR_CFULL + d), u & 1, abort_flag, a.err, 3);
            if (!__all_sync(0xffffffffu, w)) break;
            tc_fence_after();
            {
                uint32_t r[HALF];
#pragma unroll
                for (int h = 0; h < HALF / 32; ++h) tmem_ld32(lane_base + C::COL_CORR + d * NK + 32 * h, r + 32 * h);
                tmem_ld_wait();
                tc_fence_before();
                mbar_arrive(bar(C::BAR_CEMPTY + d));
#pragma unroll
                for (int c = 0; c < HALF; ++c) acc[c] += __uint_as_float(r[c]);
            }
            // Write-out in rounds of 8 combinations: the warp's 256 outputs of a
            // round go through its shared staging area in tile-local index
            // order, so each warp store covers consecutive addresses.
            const uint64_t t = blockIdx.x + i * gridDim.x;
            const uint64_t base = tc_tile_base(a, t);
#pragma unroll
            for (int rd = 0; rd < HALF / 16; ++rd) {
#pragma unroll
                for (int c3 = 0; c3 < 8; ++c3) {
                    const int o = 8 * rd + c3;
                    const uint32_t r = rank_g | ((c3 & 1) ? rc0 : 0u) | ((c3 & 2) ? rc1 : 0u) | ((c3 & 4) ? rc2 : 0u);
                    stg[r + (r >> 5)] = make_float2(acc[2 * o], acc[2 * o + 1]);
                }
                __syncwarp();
                const uint32_t lf = lfix | static_cast<uint32_t>(loff[half * (HALF / 2) + 8 * rd]);
                float2* dst = a.psi + (base | (lf & mmask) | runoff[lf >> a.m]) + goL;
#pragma unroll
                for (int j = 0; j < 8; ++j) {
                    const uint64_t off = ((j & 1) ? gb5 : 0ull) | ((j & 2) ? gb6 : 0ull) | ((j & 4) ? gb7 : 0ull);
                    __stcs(dst + off, stg[33 * j + lane]);
                }
                __syncwarp();
            }
        }
    } else if (lane == 0) {
        // ---------------- MMA issuer ----------------
        const uint32_t bhi = smem_u32(Bhi), blo = smem_u32(Blo);
        uint64_t cc = 0, sc = 0;
        bool ok = true;
        for (uint64_t i = 0; i < my_tiles && ok; ++i) {
            const uint32_t d = static_cast<uint32_t>(i % NCORR), u = static_cast<uint32_t>(i / NCORR);
            const uint32_t corr = tmem + C::COL_CORR + d * NK;
            for (int j = 0; j < KC && ok; ++j, ++cc) {
                const uint32_t b = static_cast<uint32_t>(cc & 1), f = static_cast<uint32_t>(cc >> 1);
                if (!mbar_wait(bar(C::BAR_FULL + b), f & 1, abort_flag, a.err, 5)) {
                    ok = false;
                    break;
                }
                tc_fence_after();
                const uint32_t ahi = tmem + C::COL_A + b * 64, alo = ahi + 32;
#pragma unroll
                for (int s2 = 0; s2 < 2; ++s2, ++sc) {   // the chunk's two 16-value segments
                    const uint32_t mb = static_cast<uint32_t>(sc % NMAIN), mu = static_cast<uint32_t>(sc / NMAIN);
                    if (mu >= 1 && !mbar_wait(bar(C::BAR_MEMPTY + mb), (mu - 1) & 1, abort_flag, a.err, 6)) {
                        ok = false;
                        break;
                    }
                    tc_fence_after();
                    // the segment's main partial first (exact in FP32), committed
                    // before its correction products so the epilogue starts early
#pragma unroll
                    for (int h = 0; h < 2; ++h) {
                        const int kk = 2 * s2 + h;
                        const uint32_t boff = static_cast<uint32_t>(j) * C::B_REGION + 32 * kk;
                        mma_tf32_ts(tmem + C::COL_MAIN + mb * NK, ahi + 8 * kk, sw128_desc(bhi + boff), C::IDESC, h);
                    }
                    mma_commit(bar(C::BAR_MFULL + mb));
                    // the tile's first correction product overwrites the accumulator:
                    // the epilogue must have read it for tile i - NCORR
                    if (j == 0 && s2 == 0 && u >= 1) {
                        if (!mbar_wait(bar(C::BAR_CEMPTY + d), (u - 1) & 1, abort_flag, a.err, 4)) {
                            ok = false;
                            break;
                        }
                        tc_fence_after();
                    }
#pragma unroll
                    for (int h = 0; h < 2; ++h) {
                        const int kk = 2 * s2 + h;
                        const uint32_t boff = static_cast<uint32_t>(j) * C::B_REGION + 32 * kk;
                        mma_tf32_ts(corr, alo + 8 * kk, sw128_desc(bhi + boff), C::IDESC, (j | kk) != 0);
                        mma_tf32_ts(corr, ahi + 8 * kk, sw128_desc(blo + boff), C::IDESC, 1);
                    }
                }
                if (!ok) break;
                mma_commit(bar(C::BAR_EMPTY + b));
            }
            if (ok) mma_commit(bar(C::BAR_CFULL + d));
        }
        // drain: no MMA may be in flight when the CTA tears down
        mma_commit(bar(C::BAR_FIN));
        for (uint32_t it = 0; it < kWaitLimit; ++it)
            if (mbar_try(bar(C::BAR_FIN), 0)) break;
    }
    tc_fence_before();
    __syncthreads();
    if (warp == 12) {
        tc_fence_after();
        tmem_dealloc(tmem, C::TMEM_COLS);
    }
}

template <int K>
cudaError_t launch_tc_k(float2* psi, int n, const int* phys, const float* d_mat, int* d_err, cudaStream_t st,
                        uint64_t* launches) {
    using C = TcCfg<K>;
    const int T = 7 + K;
    TileGeom g;
    if (n < T || !make_geom(n, phys, K, T, &g) || g.T != T) return cudaErrorInvalidValue;
    TcArgs a{};
    a.psi = psi;
    a.mat = d_mat;
    a.err = d_err;
    a.ntiles = g.ntiles;
    a.m = g.m;
    a.nx = g.nx;
    for (int e = 0; e < 6; ++e) a.xpos[e] = g.xpos[e];
    for (int j = 0; j < K; ++j) {
        int p = phys[j], loc = p;
        if (p >= g.m) {
            int e = 0;
            while (g.xpos[e] != p) ++e;
            loc = g.m + e;
        }
        a.tl[j] = loc;
        a.tls[j] = loc;
    }
    std::sort(a.tls, a.tls + K);
    auto kern = k_apply_tc<K>;
    static bool attr = false;
    if (!attr) {
        cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                             static_cast<int>(C::SMEM));
        if (e != cudaSuccess) return e;
        attr = true;
    }
    int occ = 0;
    cudaError_t e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, kern, kTcThreads, C::SMEM);
    if (e != cudaSuccess) return e;
    if (occ < 1) return cudaErrorInvalidConfiguration;
    // tensor memory: at most 512 columns per SM across resident CTAs
    const int per_sm = std::min(occ, static_cast<int>(512 / C::TMEM_COLS));
    uint64_t grid = static_cast<uint64_t>(num_sms()) * per_sm;
    if (grid > g.ntiles) grid = g.ntiles;
    kern<<<static_cast<unsigned>(grid), kTcThreads, C::SMEM, st>>>(a);
    ++*launches;
    return cudaGetLastError();
}

}  // namespace

bool tc_available(qsa_state s, int k) { return (k == 5 && s->n >= 12) || (k == 6 && s->n >= 13); }

cudaError_t launch_apply_tc(float2* psi, int n, const int* phys, int k, const float* d_mat, int* d_err,
                            cudaStream_t st, uint64_t* launches) {
    if (k == 5) return launch_tc_k<5>(psi, n, phys, d_mat, d_err, st, launches);
    if (k == 6) return launch_tc_k<6>(psi, n, phys, d_mat, d_err, st, launches);
    return cudaErrorNotSupported;
}

}  // namespace qsa
