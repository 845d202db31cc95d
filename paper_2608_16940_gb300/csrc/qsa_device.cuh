// Device helpers shared by the kernels: bit insertion, 16-byte cp.async,
// the sampler's integer weights, warp scans, Philox4x64-10 and layout decode.
#pragma once

#include <cuda_runtime.h>

#include <cstdint>

#include "qsa.h"

namespace qsa {
namespace dev {

// Insert a zero bit at position p (positions handled in ascending order).
__device__ __forceinline__ uint64_t insert_zero(uint64_t v, int p) {
    uint64_t lo = v & ((1ull << p) - 1ull);
    return ((v >> p) << (p + 1)) | lo;
}

__device__ __forceinline__ void cp_async16(void* smem, const void* gmem) {
    unsigned s = static_cast<unsigned>(__cvta_generic_to_shared(smem));
    asm volatile("cp.async.cg.shared.global [%0], [%1], 16;\n" ::"r"(s), "l"(gmem) : "memory");
}
__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;\n" ::: "memory"); }
template <int N>
__device__ __forceinline__ void cp_async_wait() {
    asm volatile("cp.async.wait_group %0;\n" ::"n"(N) : "memory");
}

// Two FP32 values in one 64-bit register pair, and the paired FMA
// (fma.rn.f32x2: both lanes rounded to nearest like fmaf).
__device__ __forceinline__ uint64_t pack2(float lo, float hi) {
    uint64_t r;
    asm("mov.b64 %0, {%1, %2};" : "=l"(r) : "f"(lo), "f"(hi));
    return r;
}
__device__ __forceinline__ float2 unpack2(uint64_t v) {
    float2 f;
    asm("mov.b64 {%0, %1}, %2;" : "=f"(f.x), "=f"(f.y) : "l"(v));
    return f;
}
__device__ __forceinline__ uint64_t fma2(uint64_t a, uint64_t b, uint64_t c) {
    uint64_t d;
    asm("fma.rn.f32x2 %0, %1, %2, %3;" : "=l"(d) : "l"(a), "l"(b), "l"(c));
    return d;
}

// floor(v^2 * 2^60) exactly, in integers: v = M * 2^(E - 150) with a 24-bit M
// (E = max(biased exponent, 1)), so v^2 2^60 = M^2 2^(2E - 240).  One 32 x 32
// -> 64-bit product forms M^2 2^15 = (M 2^8)(M 2^7) < 2^63, and one right
// shift by 255 - 2E (>= 1 for |v| < 2; from 63 on it leaves 0, like any
// larger shift) takes it to the scale; |v| >= 2 saturates at 2^62.
__device__ __forceinline__ uint64_t sq_fixed60(float v) {
    const uint32_t b = __float_as_uint(v) & 0x7fffffffu;
    const uint32_t e8 = b >> 23;
    const uint32_t M = (b & 0x7fffffu) | (e8 ? 0x800000u : 0u);
    const int E = e8 ? static_cast<int>(e8) : 1;
    const uint64_t sq15 = static_cast<uint64_t>(M << 8) * (M << 7);
    const uint64_t r = sq15 >> min(max(255 - 2 * E, 0), 63);
    return E >= 128 ? (1ull << 62) : r;
}

// Sampling weight of one amplitude: floor(re^2 2^60) + floor(im^2 2^60).
__device__ __forceinline__ uint64_t weight(float2 a) { return sq_fixed60(a.x) + sq_fixed60(a.y); }

__device__ __forceinline__ uint64_t warp_incl_scan_u64(uint64_t v) {
    const int lane = threadIdx.x & 31;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        uint64_t t = __shfl_up_sync(0xffffffffu, v, o);
        if (lane >= o) v += t;
    }
    return v;
}

__device__ __forceinline__ uint64_t warp_sum_u64(uint64_t v) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    return v;
}

// Philox4x64-10 (Salmon et al., SC'11), word 0 of the block at (ctr, key).
__device__ __forceinline__ uint64_t philox4x64_10_w0(uint64_t c0, uint64_t c1, uint64_t c2, uint64_t c3,
                                                     uint64_t k0, uint64_t k1) {
    const uint64_t M0 = 0xD2E7470EE14C6C93ull, M1 = 0xCA5A826395121157ull;
    const uint64_t W0 = 0x9E3779B97F4A7C15ull, W1 = 0xBB67AE8584CAA73Bull;
#pragma unroll
    for (int r = 0; r < 10; ++r) {
        if (r) {
            k0 += W0;
            k1 += W1;
        }
        const uint64_t hi0 = __umul64hi(M0, c0), lo0 = M0 * c0;
        const uint64_t hi1 = __umul64hi(M1, c2), lo1 = M1 * c2;
        const uint64_t n0 = hi1 ^ c1 ^ k0, n2 = hi0 ^ c3 ^ k1;
        c0 = n0;
        c1 = lo1;
        c2 = n2;
        c3 = lo0;
    }
    return c0;
}

struct Layout {
    int n;
    int L[QSA_MAX_QUBITS];
};

__device__ __forceinline__ uint64_t encode_logical(uint64_t x, const Layout& lay) {
    uint64_t y = 0;
#pragma unroll
    for (int q = 0; q < QSA_MAX_QUBITS; ++q)
        if (q < lay.n) y |= ((x >> q) & 1ull) << lay.L[q];
    return y;
}

__device__ __forceinline__ uint64_t decode_physical(uint64_t y, const Layout& lay) {
    uint64_t x = 0;
#pragma unroll
    for (int q = 0; q < QSA_MAX_QUBITS; ++q)
        if (q < lay.n) x |= ((y >> lay.L[q]) & 1ull) << q;
    return x;
}

}  // namespace dev
}  // namespace qsa
