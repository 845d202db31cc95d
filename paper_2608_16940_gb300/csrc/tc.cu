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
//     the tensor core: every K-step (K = 8) writes a fresh partial product
//     into one of two ping-pong tensor-memory buffers and the epilogue warps
//     add the partials in FP32 with round-to-nearest;
//   - hi parts are block-quantised per K-step segment of 8 values (a shared
//     power-of-two quantum, 10-bit integer multiples, as in Ozaki-type
//     splittings), so each 8-term partial is an exactly representable FP32
//     number and the tensor core has nothing to round.
// lo = x - hi (exact) is rounded to TF32 to nearest; the two small
// correction products (about 2^-10 of the result) accumulate in tensor
// memory, where their rounding is far below FP32 resolution of the output.
//
// CTA roles (one persistent CTA per SM, 416 threads):
//   warps 0-3   loaders: thread g owns group g, reads its amplitudes of one
//               K-chunk (16 amplitudes = 32 floats) from HBM, splits hi/lo and
//               writes both into 128-byte-swizzled K-major chunk buffers
//               (double buffered);
//   warps 4-11  epilogue: warp w reads tensor-memory lanes 32*(w%4).. and
//               half (w-4)/4 of the columns, sums the partials, adds the
//               correction accumulator and writes the outputs in place;
//   warp 12     allocates tensor memory and issues the MMAs (one thread).
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

__device__ __forceinline__ void mma_tf32(uint32_t d_tmem, uint64_t adesc, uint64_t bdesc, uint32_t idesc,
                                         uint32_t accumulate) {
    asm volatile(
        "{\n .reg .pred p;\n setp.ne.b32 p, %4, 0;\n"
        " tcgen05.mma.cta_group::1.kind::tf32 [%0], %1, %2, %3, p;\n}\n" ::"r"(d_tmem),
        "l"(adesc), "l"(bdesc), "r"(idesc), "r"(accumulate)
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

__device__ __forceinline__ float tf32_rna(float x) {
    uint32_t r;
    asm("cvt.rna.tf32.f32 %0, %1;\n" : "=r"(r) : "f"(x));
    return __uint_as_float(r);
}

// Block split of 8 values that form one MMA K-step: hi = round(x / q) * q with
// the shared quantum q = 2^(E-9), E = exponent of max |x|, so every |hi| / q
// is an integer <= 2^10 and the 8-term dot product of two such segments is an
// integer multiple of q_a q_b below 2^23 in magnitude: exactly representable
// in FP32, so the tensor core's round-toward-zero never engages on the main
// product.  lo = x - hi is exact in FP32 and is rounded to TF32 to nearest.
__device__ __forceinline__ void block_split8(const float* x, float* hi, float* lo) {
    float mx = 0.f;
#pragma unroll
    for (int i = 0; i < 8; ++i) mx = fmaxf(mx, fabsf(x[i]));
    const int e8 = static_cast<int>((__float_as_uint(mx) >> 23) & 0xFFu);
    if (e8 < 32) {   // segment is (numerically) zero: keep everything in lo
#pragma unroll
        for (int i = 0; i < 8; ++i) {
            hi[i] = 0.f;
            lo[i] = tf32_rna(x[i]);
        }
        return;
    }
    const float q = __uint_as_float(static_cast<uint32_t>(e8 - 9) << 23);      // 2^(E-9)
    const float qi = __uint_as_float(static_cast<uint32_t>(254 - e8 + 9) << 23);  // 2^(9-E)
#pragma unroll
    for (int i = 0; i < 8; ++i) {
        const float h = __fmul_rn(rintf(__fmul_rn(x[i], qi)), q);
        hi[i] = h;
        lo[i] = tf32_rna(__fsub_rn(x[i], h));
    }
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
    static constexpr int KC = NK / 32;               // K-chunks of 32 floats
    static constexpr int KSTEPS = NK / 8;            // MMA K-steps per tile
    static constexpr uint32_t B_REGION = NK * 128;   // one K-block of B
    static constexpr uint32_t B_BYTES = KC * B_REGION;
    static constexpr uint32_t A_BYTES = kGroups * 128;
    // tensor memory: two main partial buffers, two correction accumulators
    static constexpr uint32_t COL_MAIN = 0, COL_CORR = 2 * NK;
    static constexpr uint32_t TMEM_COLS = 4 * NK;
    static constexpr uint32_t IDESC = (1u << 4)      // D: FP32
                                      | (2u << 7)    // A: TF32
                                      | (2u << 10)   // B: TF32
                                      | (static_cast<uint32_t>(NK >> 3) << 17) |
                                      (static_cast<uint32_t>(kGroups >> 4) << 24);
    static constexpr size_t SMEM = 1024 + 2 * B_BYTES + 4 * A_BYTES + 64 * 8 + 64 * 4 + 16 * 8;
};

template <int K>
__global__ void __launch_bounds__(kTcThreads, 1) k_apply_tc(TcArgs a) {
    using C = TcCfg<K>;
    constexpr int D = C::D, NK = C::NK, KC = C::KC, HALF = NK / 2;
    extern __shared__ unsigned char smem_raw[];
    const uint32_t raw = smem_u32(smem_raw);
    unsigned char* sm = smem_raw + ((1024u - (raw & 1023u)) & 1023u);
    unsigned char* Bhi = sm;
    unsigned char* Blo = sm + C::B_BYTES;
    unsigned char* Abuf = sm + 2 * C::B_BYTES;   // [buffer b][hi | lo]
    uint64_t* runoff = reinterpret_cast<uint64_t*>(Abuf + 4 * C::A_BYTES);
    int* loff = reinterpret_cast<int*>(runoff + 64);
    uint64_t* bars = reinterpret_cast<uint64_t*>(loff + 64);
    uint32_t* tmem_slot = reinterpret_cast<uint32_t*>(bars + 14);
    volatile int* abort_flag = reinterpret_cast<volatile int*>(tmem_slot + 1);
    // barriers: A chunk full/empty, main partial full/empty, correction full/empty, drain
    const uint32_t full0 = smem_u32(bars + 0), empty0 = smem_u32(bars + 2), mfull0 = smem_u32(bars + 4),
                   mempty0 = smem_u32(bars + 6), cfull0 = smem_u32(bars + 8), cempty0 = smem_u32(bars + 10),
                   fin = smem_u32(bars + 12);

    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;

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
        for (int j = 0; j < K; ++j)
            if ((c >> j) & 1) o |= 1 << a.tl[j];
        loff[c] = o;
    }
    // B operand: the real embedding R of G, split hi / lo.
    const float2* G = reinterpret_cast<const float2*>(a.mat);
    for (int e = tid; e < NK * (NK / 8); e += blockDim.x) {
        const int n = e / (NK / 8), s8 = e - n * (NK / 8);   // row n, K-step segment s8
        float x[8], hi[8], lo[8];
#pragma unroll
        for (int i = 0; i < 8; ++i) {
            const int kk = 8 * s8 + i;
            const float2 g = G[(n >> 1) * D + (kk >> 1)];
            x[i] = (n & 1) ? ((kk & 1) ? g.x : g.y) : ((kk & 1) ? -g.y : g.x);
        }
        block_split8(x, hi, lo);
#pragma unroll
        for (int i = 0; i < 8; ++i) {
            const int kk = 8 * s8 + i;
            const uint32_t off = static_cast<uint32_t>(kk >> 5) * C::B_REGION + sw128_off(n, kk & 31);
            *reinterpret_cast<float*>(Bhi + off) = hi[i];
            *reinterpret_cast<float*>(Blo + off) = lo[i];
        }
    }
    if (tid == 0) {
        for (int i = 0; i < 2; ++i) {
            mbar_init(full0 + 8 * i, 128);
            mbar_init(empty0 + 8 * i, 1);
            mbar_init(mfull0 + 8 * i, 1);
            mbar_init(mempty0 + 8 * i, kEpiThreads);
            mbar_init(cfull0 + 8 * i, 1);
            mbar_init(cempty0 + 8 * i, kEpiThreads);
        }
        mbar_init(fin, 1);
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
        const int g = tid;
        uint32_t lbg = static_cast<uint32_t>(g);
#pragma unroll
        for (int j = 0; j < K; ++j) lbg = static_cast<uint32_t>(insert_zero(lbg, a.tls[j]));
        const uint64_t total = my_tiles * KC;
        float2 cur[16], nxt[16];
        auto load = [&](uint64_t idx, float2* v) {
            const uint64_t t = blockIdx.x + (idx / KC) * gridDim.x;
            const int j = static_cast<int>(idx % KC);
            const uint64_t base = tc_tile_base(a, t);
#pragma unroll
            for (int cl = 0; cl < 16; ++cl) {
                const uint32_t lj = lbg | static_cast<uint32_t>(loff[16 * j + cl]);
                v[cl] = a.psi[base | (lj & mmask) | runoff[lj >> a.m]];
            }
        };
        if (total) load(0, cur);
        for (uint64_t idx = 0; idx < total; ++idx) {
            if (idx + 1 < total) load(idx + 1, nxt);
            const uint32_t b = static_cast<uint32_t>(idx & 1), f = static_cast<uint32_t>(idx >> 1);
            if (f >= 1 && !mbar_wait(empty0 + 8 * b, (f - 1) & 1, abort_flag, a.err, 1)) break;
            unsigned char* Ahi = Abuf + b * 2 * C::A_BYTES;
            unsigned char* Alo = Ahi + C::A_BYTES;
#pragma unroll
            for (int s8 = 0; s8 < 4; ++s8) {   // the chunk's 4 K-steps of 8 floats
                float x[8], h[8], l[8];
#pragma unroll
                for (int i = 0; i < 4; ++i) {
                    x[2 * i] = cur[4 * s8 + i].x;
                    x[2 * i + 1] = cur[4 * s8 + i].y;
                }
                block_split8(x, h, l);
#pragma unroll
                for (int c4 = 0; c4 < 2; ++c4) {
                    const uint32_t off = sw128_off(static_cast<uint32_t>(g), static_cast<uint32_t>(8 * s8 + 4 * c4));
                    *reinterpret_cast<float4*>(Ahi + off) =
                        make_float4(h[4 * c4], h[4 * c4 + 1], h[4 * c4 + 2], h[4 * c4 + 3]);
                    *reinterpret_cast<float4*>(Alo + off) =
                        make_float4(l[4 * c4], l[4 * c4 + 1], l[4 * c4 + 2], l[4 * c4 + 3]);
                }
            }
            fence_async_smem();
            mbar_arrive(full0 + 8 * b);
#pragma unroll
            for (int cl = 0; cl < 16; ++cl) cur[cl] = nxt[cl];
        }
    } else if (warp < 12) {
        // ---------------- epilogue ----------------
        const int qw = warp & 3;              // tensor-memory lane quarter
        const int half = (warp - 4) >> 2;     // column half
        const int g = qw * 32 + lane;
        uint32_t lbg = static_cast<uint32_t>(g);
#pragma unroll
        for (int j = 0; j < K; ++j) lbg = static_cast<uint32_t>(insert_zero(lbg, a.tls[j]));
        const uint32_t lane_base = tmem + (static_cast<uint32_t>(qw * 32) << 16) + half * HALF;
        uint64_t sc = 0;   // global K-step counter (main buffers)
        bool ok = true;
        for (uint64_t i = 0; i < my_tiles && ok; ++i) {
            float acc[HALF];
#pragma unroll
            for (int c = 0; c < HALF; ++c) acc[c] = 0.f;
            for (int s = 0; s < C::KSTEPS; ++s, ++sc) {
                const uint32_t mb = static_cast<uint32_t>(sc & 1), mu = static_cast<uint32_t>(sc >> 1);
                const bool w = mbar_wait(mfull0 + 8 * mb, mu & 1, abort_flag, a.err, 2);
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
                mbar_arrive(mempty0 + 8 * mb);
#pragma unroll
                for (int c = 0; c < HALF; ++c) acc[c] += __uint_as_float(r[c]);
            }
            if (!ok) break;
            const uint32_t d = static_cast<uint32_t>(i & 1), u = static_cast<uint32_t>(i >> 1);
            const bool w = mbar_wait(cfull0 + 8 * d, u & 1, abort_flag, a.err, 3);
            if (!__all_sync(0xffffffffu, w)) break;
            tc_fence_after();
            {
                uint32_t r[HALF];
#pragma unroll
                for (int h = 0; h < HALF / 32; ++h) tmem_ld32(lane_base + C::COL_CORR + d * NK + 32 * h, r + 32 * h);
                tmem_ld_wait();
                tc_fence_before();
                mbar_arrive(cempty0 + 8 * d);
#pragma unroll
                for (int c = 0; c < HALF; ++c) acc[c] += __uint_as_float(r[c]);
            }
            const uint64_t t = blockIdx.x + i * gridDim.x;
            const uint64_t base = tc_tile_base(a, t);
#pragma unroll
            for (int o = 0; o < HALF / 2; ++o) {
                const uint32_t lj = lbg | static_cast<uint32_t>(loff[half * (HALF / 2) + o]);
                a.psi[base | (lj & mmask) | runoff[lj >> a.m]] = make_float2(acc[2 * o], acc[2 * o + 1]);
            }
        }
    } else if (lane == 0) {
        // ---------------- MMA issuer ----------------
        const uint32_t bhi = smem_u32(Bhi), blo = smem_u32(Blo);
        uint64_t cc = 0, sc = 0;
        bool ok = true;
        for (uint64_t i = 0; i < my_tiles && ok; ++i) {
            const uint32_t d = static_cast<uint32_t>(i & 1), u = static_cast<uint32_t>(i >> 1);
            if (u >= 1 && !mbar_wait(cempty0 + 8 * d, (u - 1) & 1, abort_flag, a.err, 4)) break;
            const uint32_t corr = tmem + C::COL_CORR + d * NK;
            for (int j = 0; j < KC && ok; ++j, ++cc) {
                const uint32_t b = static_cast<uint32_t>(cc & 1), f = static_cast<uint32_t>(cc >> 1);
                if (!mbar_wait(full0 + 8 * b, f & 1, abort_flag, a.err, 5)) {
                    ok = false;
                    break;
                }
                const uint32_t ahi = smem_u32(Abuf + b * 2 * C::A_BYTES), alo = ahi + C::A_BYTES;
#pragma unroll
                for (int kk = 0; kk < 4; ++kk, ++sc) {
                    const uint32_t mb = static_cast<uint32_t>(sc & 1), mu = static_cast<uint32_t>(sc >> 1);
                    if (mu >= 1 && !mbar_wait(mempty0 + 8 * mb, (mu - 1) & 1, abort_flag, a.err, 6)) {
                        ok = false;
                        break;
                    }
                    tc_fence_after();
                    const uint64_t dah = sw128_desc(ahi + 32 * kk), dal = sw128_desc(alo + 32 * kk);
                    const uint32_t boff = static_cast<uint32_t>(j) * C::B_REGION + 32 * kk;
                    const uint64_t dbh = sw128_desc(bhi + boff), dbl = sw128_desc(blo + boff);
                    mma_tf32(tmem + C::COL_MAIN + mb * NK, dah, dbh, C::IDESC, 0);   // fresh partial
                    mma_tf32(corr, dal, dbh, C::IDESC, (j | kk) != 0);
                    mma_tf32(corr, dah, dbl, C::IDESC, 1);
                    mma_commit(mfull0 + 8 * mb);
                }
                if (!ok) break;
                mma_commit(empty0 + 8 * b);
            }
            if (ok) mma_commit(cfull0 + 8 * d);
        }
        // drain: no MMA may be in flight when the CTA tears down
        mma_commit(fin);
        for (uint32_t it = 0; it < kWaitLimit; ++it)
            if (mbar_try(fin, 0)) break;
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
