// Reductions and sampling on the complex64 state (sm_103a).
//
//   launch_reduce_z      <Z_mask> and the norm: exact squares accumulated per
//                        thread in double-float (about 48 bits), partials
//                        combined in FP64 (App. B: totals kept in FP64).
//   launch_probs_logical p_x = fl64(re^2) + fl64(im^2) for every logical x,
//                        decoded through the layout map (Theorem 1).
//   launch_sample        hierarchical CDF sampler (§IV-E "Sampling": 2^10-entry
//                        blocks, strict upper bound) with integer weights
//                        P_y = floor(re^2 2^60) + floor(im^2 2^60) so that the
//                        CDF is exact and independent of summation order, one
//                        Philox4x64-10 draw per shot, decode through L (§IV-D),
//                        then sort + run-length encode into (outcome, count).
#include <cuda_runtime.h>

#include <cstdint>

#include "qsa_device.cuh"
#include "qsa_internal.h"

namespace qsa {

namespace {

using namespace dev;

constexpr int kRedThreads = 256;
constexpr int kRedBlocksPerSM = 8;

__device__ __forceinline__ double warp_sum_d(double v) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
    return v;
}

// Per-thread accumulation as an unevaluated float pair s + c: every square is
// split exactly into h + l (FMA two-product, h = fl(v^2), l = v^2 - h) and h
// is added with Knuth's two-sum, whose rounding error goes to c with l.  The
// pair carries about 48 significant bits, so the FP64 value (double)s +
// (double)c of each thread's partial sum matches FP64 accumulation of the
// exact squares, while costing FP32 instructions only (GB300's FP64 rate is a
// small fraction of its FP32 rate).
__device__ __forceinline__ void acc_square(float& s, float& c, float v, bool neg) {
    float h = __fmul_rn(v, v);
    float l = __fmaf_rn(v, v, -h);
    if (neg) {
        h = -h;
        l = -l;
    }
    const float t = __fadd_rn(s, h);
    const float bp = __fsub_rn(t, s);
    const float e = __fadd_rn(__fsub_rn(s, __fsub_rn(t, bp)), __fsub_rn(h, bp));
    s = t;
    c = __fadd_rn(c, __fadd_rn(e, l));
}

__global__ void __launch_bounds__(kRedThreads) k_reduce_z(const float4* __restrict__ psi2, uint64_t npairs,
                                                           uint64_t physmask, double* __restrict__ partials) {
    float s = 0.f, c = 0.f;
    const uint64_t stride = static_cast<uint64_t>(gridDim.x) * blockDim.x;
    for (uint64_t i = static_cast<uint64_t>(blockIdx.x) * blockDim.x + threadIdx.x; i < npairs; i += stride) {
        const float4 a = __ldcs(psi2 + i);
        const uint64_t y0 = i << 1;
        const bool n0 = __popcll(y0 & physmask) & 1;
        const bool n1 = __popcll((y0 | 1ull) & physmask) & 1;
        acc_square(s, c, a.x, n0);
        acc_square(s, c, a.y, n0);
        acc_square(s, c, a.z, n1);
        acc_square(s, c, a.w, n1);
    }
    double acc = static_cast<double>(s) + static_cast<double>(c);
    __shared__ double ws[kRedThreads / 32];
    acc = warp_sum_d(acc);
    if ((threadIdx.x & 31) == 0) ws[threadIdx.x >> 5] = acc;
    __syncthreads();
    if (threadIdx.x < 32) {
        double v = threadIdx.x < (kRedThreads / 32) ? ws[threadIdx.x] : 0.0;
        v = warp_sum_d(v);
        if (threadIdx.x == 0) partials[blockIdx.x] = v;
    }
}

// Several sign masks in one pass: the squares are formed once per amplitude
// and accumulated per mask exactly as k_reduce_z does (so each result equals
// the single-mask one bit for bit).  Partials of mask m at m * gridDim.x.
__global__ void __launch_bounds__(kRedThreads) k_reduce_z_multi(const float4* __restrict__ psi2, uint64_t npairs,
                                                                ZMasks masks, double* __restrict__ partials) {
    float s[kMaxZMasks] = {}, c[kMaxZMasks] = {};
    const uint64_t stride = static_cast<uint64_t>(gridDim.x) * blockDim.x;
    for (uint64_t i = static_cast<uint64_t>(blockIdx.x) * blockDim.x + threadIdx.x; i < npairs; i += stride) {
        const float4 a = __ldcs(psi2 + i);
        const uint64_t y0 = i << 1;
#pragma unroll
        for (int m = 0; m < kMaxZMasks; ++m) {
            if (m >= masks.n) break;
            const bool n0 = __popcll(y0 & masks.m[m]) & 1;
            const bool n1 = __popcll((y0 | 1ull) & masks.m[m]) & 1;
            acc_square(s[m], c[m], a.x, n0);
            acc_square(s[m], c[m], a.y, n0);
            acc_square(s[m], c[m], a.z, n1);
            acc_square(s[m], c[m], a.w, n1);
        }
    }
    __shared__ double ws[kRedThreads / 32];
    for (int m = 0; m < masks.n; ++m) {
        double acc = static_cast<double>(s[m]) + static_cast<double>(c[m]);
        acc = warp_sum_d(acc);
        if ((threadIdx.x & 31) == 0) ws[threadIdx.x >> 5] = acc;
        __syncthreads();
        if (threadIdx.x < 32) {
            double v = threadIdx.x < (kRedThreads / 32) ? ws[threadIdx.x] : 0.0;
            v = warp_sum_d(v);
            if (threadIdx.x == 0) partials[static_cast<uint64_t>(m) * gridDim.x + blockIdx.x] = v;
        }
        __syncthreads();
    }
}

// Fixed-order sum of the partials (deterministic for a given grid).
__global__ void k_finalize_sum(const double* __restrict__ partials, int n, double* __restrict__ out) {
    __shared__ double sh[1024];
    double v = 0.0;
    for (int i = threadIdx.x; i < n; i += blockDim.x) v += partials[i];
    sh[threadIdx.x] = v;
    __syncthreads();
    for (int s = blockDim.x >> 1; s > 0; s >>= 1) {
        if (static_cast<int>(threadIdx.x) < s) sh[threadIdx.x] += sh[threadIdx.x + s];
        __syncthreads();
    }
    if (threadIdx.x == 0) *out = sh[0];
}


__global__ void k_probs_logical(const float2* __restrict__ psi, Layout lay, double* __restrict__ out) {
    const uint64_t dim = 1ull << lay.n;
    const uint64_t stride = static_cast<uint64_t>(gridDim.x) * blockDim.x;
    for (uint64_t x = static_cast<uint64_t>(blockIdx.x) * blockDim.x + threadIdx.x; x < dim; x += stride) {
        const float2 a = psi[encode_logical(x, lay)];
        out[x] = __dadd_rn(__dmul_rn(a.x, a.x), __dmul_rn(a.y, a.y));
    }
}

// ---------------------------------------------------------------------------
// Sampler
// ---------------------------------------------------------------------------


// One warp per block of `bsz` amplitudes: total integer weight.
__global__ void k_block_weights(const float2* __restrict__ psi, uint64_t nblocks, int bsz,
                                uint64_t* __restrict__ cum) {
    const uint64_t w = (static_cast<uint64_t>(blockIdx.x) * blockDim.x + threadIdx.x) >> 5;
    const int lane = threadIdx.x & 31;
    if (w >= nblocks) return;
    const float2* p = psi + w * bsz;
    uint64_t s = 0;
    for (int j = lane; j < bsz; j += 32) s += weight(p[j]);
    s = warp_sum_u64(s);
    if (lane == 0) cum[w] = s;
}

// The block weights and, in the same read of the state, <Z_mask> sums for up to
// kMaxZMasks masks: persistent warps walk the 2^bsz-amplitude blocks; each
// thread accumulates its amplitudes' squares per mask as k_reduce_z does
// (double-float); per-CTA partials of mask m at m * gridDim.x.
__global__ void __launch_bounds__(kRedThreads) k_block_weights_z(const float2* __restrict__ psi, uint64_t nblocks,
                                                                 int bsz, uint64_t* __restrict__ cum, ZMasks masks,
                                                                 double* __restrict__ partials) {
    const int lane = threadIdx.x & 31;
    const uint64_t warps = static_cast<uint64_t>(gridDim.x) * (blockDim.x >> 5);
    float zs[kMaxZMasks] = {}, zc[kMaxZMasks] = {};
    for (uint64_t w = (static_cast<uint64_t>(blockIdx.x) * blockDim.x + threadIdx.x) >> 5; w < nblocks; w += warps) {
        const uint64_t y0 = w * bsz;
        const float2* p = psi + y0;
        uint64_t s = 0;
        for (int j = lane; j < bsz; j += 32) {
            const float2 a = __ldcs(p + j);
            s += weight(a);
#pragma unroll
            for (int m = 0; m < kMaxZMasks; ++m) {
                if (m >= masks.n) break;
                const bool neg = __popcll((y0 + j) & masks.m[m]) & 1;
                acc_square(zs[m], zc[m], a.x, neg);
                acc_square(zs[m], zc[m], a.y, neg);
            }
        }
        s = warp_sum_u64(s);
        if (lane == 0) cum[w] = s;
    }
    __shared__ double ws[kRedThreads / 32];
    for (int m = 0; m < masks.n; ++m) {
        double acc = static_cast<double>(zs[m]) + static_cast<double>(zc[m]);
        acc = warp_sum_d(acc);
        if (lane == 0) ws[threadIdx.x >> 5] = acc;
        __syncthreads();
        if (threadIdx.x < 32) {
            double v = threadIdx.x < (kRedThreads / 32) ? ws[threadIdx.x] : 0.0;
            v = warp_sum_d(v);
            if (threadIdx.x == 0) partials[static_cast<uint64_t>(m) * gridDim.x + blockIdx.x] = v;
        }
        __syncthreads();
    }
}

// |x + iy|^2 as an unevaluated pair hi + lo: each square split exactly by the
// FMA two-product, the two high parts added by Knuth's two-sum, the low parts
// (about 2^-24 of hi) rounded into lo.
__device__ __forceinline__ void square_pair(float x, float y, float& hi, float& lo) {
    const float h1 = __fmul_rn(x, x), l1 = __fmaf_rn(x, x, -h1);
    const float h2 = __fmul_rn(y, y), l2 = __fmaf_rn(y, y, -h2);
    const float t = __fadd_rn(h1, h2);
    const float bp = __fsub_rn(t, h1);
    const float e = __fadd_rn(__fsub_rn(h1, __fsub_rn(t, bp)), __fsub_rn(h2, bp));
    hi = t;
    lo = __fadd_rn(e, __fadd_rn(l1, l2));
}

// Weight of one component from its bits when its biased exponent e is at most
// 127 (|v| < 2): floor(v^2 2^60) = floor(M^2 2^(2e - 240)) as (M 2^7)^2 =
// M^2 2^14 < 2^62 shifted right by 254 - 2e, the shift left unclamped (PTX
// shr.b64 takes shifts above 64 as 64 and gives 0, the exact result there).
// The implicit bit is set unconditionally; for e = 0 (zero, subnormals) the
// shift is 254, so the result is 0 as in sq_fixed60.  254 - 2e = 2e ^ 254
// since 2e is even and below 256.
__device__ __forceinline__ uint64_t sq_fixed60_small(uint32_t bits) {
    const uint32_t mq = ((bits & 0x7fffffu) | 0x800000u) << 7;
    const uint32_t sh = ((bits >> 22) & 0x1feu) ^ 0xfeu;
    const uint64_t prod = static_cast<uint64_t>(mq) * mq;
    uint64_t r;
    asm("shr.b64 %0, %1, %2;" : "=l"(r) : "l"(prod), "r"(sh));
    return r;
}

// s + c += g (hi + lo) for g = +-1, in double-float: Knuth's two-sum of s and
// g hi (its rounding error to c with g lo), the sign taken inside FMAs (g hi
// and g lo are exact products, so each FMA rounds once, like an addition of
// the negated term).
__device__ __forceinline__ void add_scaled(float& s, float& c, float hi, float lo, float g) {
    const float t = __fmaf_rn(g, hi, s);
    const float bp = __fsub_rn(t, s);
    const float e = __fadd_rn(__fsub_rn(s, __fsub_rn(t, bp)), __fmaf_rn(g, hi, -bp));
    s = t;
    c = __fadd_rn(c, __fmaf_rn(g, lo, e));
}

// Blocks of 1024 amplitudes: the block weights and the <Z_mask> sums of NM
// masks in one read.  A warp takes a block; lane l loads the 16-byte pairs
// l + 32 k (k = 0..15) up front, so 8 KiB per warp are in flight.  Amplitude
// y = 1024 w + 2 (l + 32 k) + b has its index bits split over (w, l, k, b), so
// its sign parity is a per-block, a per-lane, a per-k and a per-b part.
// Weights: when no component of the block has |v| >= 2 (always, for a state
// of norm about 1) the warp takes sq_fixed60_small, else sq_fixed60 (equal
// values where both apply).  Sums: each thread keeps its mask-m pair in the
// frame of its own block-and-lane sign (the pair negated when that sign
// changes between blocks; round-to-nearest is symmetric, so the values are
// those of summing in the true signs, up to the sign of zeros), so the sign
// left per amplitude, of its k and b bits, is the same across the warp.  Per
// CTA partials of mask m at m * gridDim.x.
template <int NM>
__global__ void __launch_bounds__(kRedThreads, 2) k_weights_z1024(const float4* __restrict__ psi2, uint64_t nblocks,
                                                                  uint64_t* __restrict__ cum, ZMasks masks,
                                                                  double* __restrict__ partials) {
    constexpr int NA = NM > 0 ? NM : 1;
    const int lane = threadIdx.x & 31;
    const uint64_t warps = static_cast<uint64_t>(gridDim.x) * (blockDim.x >> 5);
    float zs[NA] = {}, zc[NA] = {};
    uint32_t kb[NA] = {}, lb[NA] = {}, fr[NA] = {};
    float bf[NA] = {};
#pragma unroll
    for (int m = 0; m < NM; ++m) {
        for (int k = 0; k < 16; ++k) kb[m] |= static_cast<uint32_t>(__popcll((64ull * k) & masks.m[m]) & 1) << k;
        lb[m] = __popcll((2ull * lane) & masks.m[m]) & 1;
        bf[m] = (masks.m[m] & 1ull) ? -1.f : 1.f;
    }
    for (uint64_t w = (static_cast<uint64_t>(blockIdx.x) * blockDim.x + threadIdx.x) >> 5; w < nblocks; w += warps) {
        const float4* p = psi2 + w * 512 + lane;
        float4 a[16];
#pragma unroll
        for (int k = 0; k < 16; ++k) a[k] = __ldcs(p + 32 * k);
        if constexpr (NM > 0) {
#pragma unroll
            for (int m = 0; m < NM; ++m) {
                // this thread's sign for the block; the pair follows it into the new frame
                const uint32_t f = (__popcll((w << 10) & masks.m[m]) & 1) ^ lb[m];
                if (f != fr[m]) {
                    zs[m] = -zs[m];
                    zc[m] = -zc[m];
                    fr[m] = f;
                }
            }
        }
        uint32_t any = 0;
        uint64_t s = 0;
#pragma unroll
        for (int k = 0; k < 16; ++k) {
            const uint32_t x0 = __float_as_uint(a[k].x), y0 = __float_as_uint(a[k].y);
            const uint32_t x1 = __float_as_uint(a[k].z), y1 = __float_as_uint(a[k].w);
            any |= x0 | y0 | x1 | y1;
            s += sq_fixed60_small(x0) + sq_fixed60_small(y0) + sq_fixed60_small(x1) + sq_fixed60_small(y1);
            if constexpr (NM > 0) {
                float h0, l0, h1, l1;
                square_pair(a[k].x, a[k].y, h0, l0);
                square_pair(a[k].z, a[k].w, h1, l1);
#pragma unroll
                for (int m = 0; m < NM; ++m) {
                    const float g0 = __uint_as_float(0x3f800000u | (((kb[m] >> k) & 1u) << 31));
                    add_scaled(zs[m], zc[m], h0, l0, g0);
                    add_scaled(zs[m], zc[m], h1, l1, g0 * bf[m]);
                }
            }
        }
        if (!__all_sync(0xffffffffu, (any & 0x40000000u) == 0u)) {
            // a component with |v| >= 2 (or not finite) in the block: the weights again, by sq_fixed60
            s = 0;
#pragma unroll 4
            for (int k = 0; k < 16; ++k) {
                const float4 v = __ldcs(p + 32 * k);
                s += sq_fixed60(v.x) + sq_fixed60(v.y) + sq_fixed60(v.z) + sq_fixed60(v.w);
            }
        }
        s = warp_sum_u64(s);
        if (lane == 0) cum[w] = s;
    }
    if constexpr (NM > 0) {
        __shared__ double ws[kRedThreads / 32];
#pragma unroll
        for (int m = 0; m < NM; ++m) {
            // back from the thread's frame (the last block's sign)
            const double sg = fr[m] ? -1.0 : 1.0;
            double acc = sg * static_cast<double>(zs[m]) + sg * static_cast<double>(zc[m]);
            acc = warp_sum_d(acc);
            if (lane == 0) ws[threadIdx.x >> 5] = acc;
            __syncthreads();
            if (threadIdx.x < 32) {
                double v = threadIdx.x < (kRedThreads / 32) ? ws[threadIdx.x] : 0.0;
                v = warp_sum_d(v);
                if (threadIdx.x == 0) partials[static_cast<uint64_t>(m) * gridDim.x + blockIdx.x] = v;
            }
            __syncthreads();
        }
    }
}

// In-place inclusive scan of cum[0..n-1] by one CTA of 1024 threads.
__global__ void __launch_bounds__(1024) k_scan_inclusive(uint64_t* __restrict__ cum, uint64_t n) {
    __shared__ uint64_t wsum[32];
    __shared__ uint64_t carry;
    if (threadIdx.x == 0) carry = 0;
    __syncthreads();
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    for (uint64_t base = 0; base < n; base += blockDim.x) {
        const uint64_t i = base + threadIdx.x;
        uint64_t v = i < n ? cum[i] : 0;
        uint64_t inc = warp_incl_scan_u64(v);
        if (lane == 31) wsum[wid] = inc;
        __syncthreads();
        if (wid == 0) {
            uint64_t s = wsum[lane];
            wsum[lane] = warp_incl_scan_u64(s);
        }
        __syncthreads();
        const uint64_t off = carry + (wid ? wsum[wid - 1] : 0);
        if (i < n) cum[i] = inc + off;
        __syncthreads();
        if (threadIdx.x == blockDim.x - 1) carry = inc + off;
        __syncthreads();
    }
}


// Multi-CTA inclusive scan of cum[0..n-1]: each CTA scans one segment of
// kScanSeg entries in place and writes its total to parts[b]; parts is then
// scanned by k_scan_inclusive and k_scan_add adds parts[b - 1] to segment b.
// Integer sums, so the result is the same as the one-CTA scan.
constexpr int kScanSeg = 4096;

__global__ void __launch_bounds__(1024) k_scan_segments(uint64_t* __restrict__ cum, uint64_t n,
                                                        uint64_t* __restrict__ parts) {
    __shared__ uint64_t wsum[32];
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    const uint64_t i0 = static_cast<uint64_t>(blockIdx.x) * kScanSeg + 4ull * threadIdx.x;
    uint64_t v[4];
#pragma unroll
    for (int k = 0; k < 4; ++k) v[k] = i0 + k < n ? cum[i0 + k] : 0;
    v[1] += v[0];
    v[2] += v[1];
    v[3] += v[2];
    const uint64_t inc = warp_incl_scan_u64(v[3]);
    if (lane == 31) wsum[wid] = inc;
    __syncthreads();
    if (wid == 0) wsum[lane] = warp_incl_scan_u64(wsum[lane]);
    __syncthreads();
    const uint64_t off = inc - v[3] + (wid ? wsum[wid - 1] : 0);
#pragma unroll
    for (int k = 0; k < 4; ++k)
        if (i0 + k < n) cum[i0 + k] = v[k] + off;
    if (threadIdx.x == 1023) parts[blockIdx.x] = wsum[31];
}

__global__ void k_scan_add(uint64_t* __restrict__ cum, uint64_t n, const uint64_t* __restrict__ parts) {
    const uint64_t stride = static_cast<uint64_t>(gridDim.x) * blockDim.x;
    for (uint64_t i = kScanSeg + static_cast<uint64_t>(blockIdx.x) * blockDim.x + threadIdx.x; i < n; i += stride)
        cum[i] += parts[i / kScanSeg - 1];
}

// One warp per shot: draw u, find the block (first cum > u), then the amplitude.
__global__ void k_draw(const float2* __restrict__ psi, const uint64_t* __restrict__ cum, uint64_t nblocks, int bsz,
                       Layout lay, uint64_t shots, uint64_t seed, uint64_t stream_id, uint64_t* __restrict__ keys) {
    const uint64_t s = (static_cast<uint64_t>(blockIdx.x) * blockDim.x + threadIdx.x) >> 5;
    const int lane = threadIdx.x & 31;
    if (s >= shots) return;
    const uint64_t total = cum[nblocks - 1];
    if (total == 0) {  // all-zero state: the host reports it; avoid the modulo by zero
        if (lane == 0) keys[s] = 0;
        return;
    }
    const uint64_t r = philox4x64_10_w0(s, stream_id, 0, 0, seed, 0);
    const uint64_t u = __umul64hi(r, total);  // floor(r * total / 2^64)
    // first block b with cum[b] > u
    uint64_t lo = 0, hi = nblocks - 1;
    while (lo < hi) {
        uint64_t mid = lo + ((hi - lo) >> 1);
        if (cum[mid] > u) hi = mid; else lo = mid + 1;
    }
    const uint64_t b = lo;
    const uint64_t ub = u - (b ? cum[b - 1] : 0);
    // lane l covers amplitudes [l*per, (l+1)*per) of the block
    const int per = (bsz + 31) >> 5;
    const float2* p = psi + b * static_cast<uint64_t>(bsz);
    uint64_t wl = 0;
    for (int j = 0; j < per; ++j) {
        int idx = lane * per + j;
        if (idx < bsz) wl += weight(p[idx]);
    }
    const uint64_t incl = warp_incl_scan_u64(wl);
    const uint64_t excl = incl - wl;
    const unsigned hit = __ballot_sync(0xffffffffu, excl <= ub && ub < incl);
    const int owner = __ffs(hit) - 1;   // exactly one lane: the weights sum to cum[b] - cum[b-1] > ub
    if (lane == owner) {
        uint64_t acc = excl;
        int j = 0;
        for (; j < per; ++j) {
            int idx = lane * per + j;
            if (idx >= bsz) break;
            acc += weight(p[idx]);
            if (acc > ub) break;
        }
        const uint64_t y = b * static_cast<uint64_t>(bsz) + static_cast<uint64_t>(lane * per + j);
        keys[s] = decode_physical(y, lay);
    }
}

__global__ void k_fill_u64(uint64_t* a, uint64_t from, uint64_t to, uint64_t v) {
    uint64_t i = from + static_cast<uint64_t>(blockIdx.x) * blockDim.x + threadIdx.x;
    if (i < to) a[i] = v;
}

// Bitonic sort of P = 2^p keys.  Small P: one CTA in shared memory.
__global__ void __launch_bounds__(1024) k_bitonic_smem(uint64_t* keys, int P) {
    extern __shared__ uint64_t sk[];
    for (int i = threadIdx.x; i < P; i += blockDim.x) sk[i] = keys[i];
    __syncthreads();
    for (int k = 2; k <= P; k <<= 1) {
        for (int j = k >> 1; j > 0; j >>= 1) {
            for (int i = threadIdx.x; i < P; i += blockDim.x) {
                int l = i ^ j;
                if (l > i) {
                    bool up = (i & k) == 0;
                    uint64_t a = sk[i], c = sk[l];
                    if ((a > c) == up) {
                        sk[i] = c;
                        sk[l] = a;
                    }
                }
            }
            __syncthreads();
        }
    }
    for (int i = threadIdx.x; i < P; i += blockDim.x) keys[i] = sk[i];
}

__global__ void k_bitonic_step(uint64_t* keys, uint64_t P, uint64_t j, uint64_t k) {
    uint64_t i = static_cast<uint64_t>(blockIdx.x) * blockDim.x + threadIdx.x;
    if (i >= P) return;
    uint64_t l = i ^ j;
    if (l > i) {
        bool up = (i & k) == 0;
        uint64_t a = keys[i], c = keys[l];
        if ((a > c) == up) {
            keys[i] = c;
            keys[l] = a;
        }
    }
}

// Run-length encode the sorted keys[0..n-1] with one CTA: distinct keys and
// their counts, and the number of distinct keys.
__global__ void __launch_bounds__(1024) k_rle(const uint64_t* __restrict__ keys, uint64_t n,
                                              uint64_t* __restrict__ out_keys, uint64_t* __restrict__ starts,
                                              uint64_t* __restrict__ out_counts, uint64_t* __restrict__ n_distinct) {
    __shared__ uint64_t wsum[32];
    __shared__ uint64_t carry;
    if (threadIdx.x == 0) carry = 0;
    __syncthreads();
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    for (uint64_t base = 0; base < n; base += blockDim.x) {
        const uint64_t i = base + threadIdx.x;
        const uint64_t head = (i < n && (i == 0 || keys[i] != keys[i - 1])) ? 1 : 0;
        uint64_t inc = warp_incl_scan_u64(head);
        if (lane == 31) wsum[wid] = inc;
        __syncthreads();
        if (wid == 0) wsum[lane] = warp_incl_scan_u64(wsum[lane]);
        __syncthreads();
        const uint64_t pos = carry + (wid ? wsum[wid - 1] : 0) + inc - head;
        if (head) {
            out_keys[pos] = keys[i];
            starts[pos] = i;
        }
        __syncthreads();
        if (threadIdx.x == blockDim.x - 1) carry = pos + head;
        __syncthreads();
    }
    const uint64_t nd = carry;
    for (uint64_t d = threadIdx.x; d < nd; d += blockDim.x)
        out_counts[d] = (d + 1 < nd ? starts[d + 1] : n) - starts[d];
    if (threadIdx.x == 0) *n_distinct = nd;
}

inline uint64_t next_pow2(uint64_t v) {
    uint64_t p = 1;
    while (p < v) p <<= 1;
    return p;
}

// Batched sampler: CTA t samples state t (identity layout) with Philox stream
// id t.  Shared memory: cum[nblocks] (uint64) then keys[P] (uint32).
constexpr int kBatchSampleThreads = 512;

__global__ void __launch_bounds__(kBatchSampleThreads)
    k_batch_sample(const float2* __restrict__ states, int n, uint32_t shots, uint32_t P, uint64_t seed,
                   uint32_t* __restrict__ out_keys, uint32_t* __restrict__ out_counts,
                   uint32_t* __restrict__ n_distinct) {
    extern __shared__ uint64_t sm64[];
    const int traj = blockIdx.x;
    const float2* psi = states + (static_cast<uint64_t>(traj) << n);
    const int bsz = n >= 10 ? 1024 : (1 << n);
    const int nb = (1 << n) / bsz;
    uint64_t* cum = sm64;
    uint32_t* keys = reinterpret_cast<uint32_t*>(cum + nb);
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31, nw = blockDim.x >> 5;
    __shared__ uint32_t wsum[32];
    __shared__ uint32_t carry;

    for (int b = warp; b < nb; b += nw) {
        uint64_t s = 0;
        for (int j = lane; j < bsz; j += 32) s += weight(psi[static_cast<uint64_t>(b) * bsz + j]);
        s = warp_sum_u64(s);
        if (lane == 0) cum[b] = s;
    }
    __syncthreads();
    if (warp == 0) {   // inclusive scan: lane l owns a contiguous range
        const int per = (nb + 31) / 32;
        const int lo = lane * per, hi = min(nb, lo + per);
        uint64_t s = 0;
        for (int i = lo; i < hi; ++i) s += cum[i];
        uint64_t run = warp_incl_scan_u64(s) - s;
        for (int i = lo; i < hi; ++i) {
            run += cum[i];
            cum[i] = run;
        }
    }
    __syncthreads();
    const uint64_t total = cum[nb - 1];
    const int per = (bsz + 31) >> 5;
    for (uint32_t s = warp; s < shots; s += nw) {
        const uint64_t r = philox4x64_10_w0(s, static_cast<uint64_t>(traj), 0, 0, seed, 0);
        const uint64_t u = __umul64hi(r, total);  // floor(r * total / 2^64)
        int lo = 0, hi = nb - 1;
        while (lo < hi) {
            const int mid = (lo + hi) >> 1;
            if (cum[mid] > u) hi = mid; else lo = mid + 1;
        }
        const uint64_t ub = u - (lo ? cum[lo - 1] : 0);
        const float2* p = psi + static_cast<uint64_t>(lo) * bsz;
        uint64_t wl = 0;
        for (int j = 0; j < per; ++j) {
            const int idx = lane * per + j;
            if (idx < bsz) wl += weight(p[idx]);
        }
        const uint64_t incl = warp_incl_scan_u64(wl);
        const uint64_t excl = incl - wl;
        const unsigned hit = __ballot_sync(0xffffffffu, excl <= ub && ub < incl);
        const int owner = hit ? __ffs(hit) - 1 : 0;
        if (lane == owner) {
            uint64_t acc = excl;
            int j = 0;
            for (; j < per; ++j) {
                const int idx = lane * per + j;
                if (idx >= bsz) break;
                acc += weight(p[idx]);
                if (acc > ub) break;
            }
            keys[s] = static_cast<uint32_t>(lo * bsz + lane * per + j);
        }
    }
    for (uint32_t i = shots + threadIdx.x; i < P; i += blockDim.x) keys[i] = 0xFFFFFFFFu;
    __syncthreads();
    for (uint32_t k = 2; k <= P; k <<= 1)
        for (uint32_t j = k >> 1; j > 0; j >>= 1) {
            for (uint32_t i = threadIdx.x; i < P; i += blockDim.x) {
                const uint32_t l = i ^ j;
                if (l > i) {
                    const bool up = (i & k) == 0;
                    const uint32_t x = keys[i], y = keys[l];
                    if ((x > y) == up) {
                        keys[i] = y;
                        keys[l] = x;
                    }
                }
            }
            __syncthreads();
        }
    // run-length encode: heads get their output slot; out_counts holds the
    // run starts until they are turned into counts
    uint32_t* okeys = out_keys + static_cast<uint64_t>(traj) * shots;
    uint32_t* ocnt = out_counts + static_cast<uint64_t>(traj) * shots;
    if (threadIdx.x == 0) carry = 0;
    __syncthreads();
    for (uint32_t base = 0; base < shots; base += blockDim.x) {
        const uint32_t i = base + threadIdx.x;
        const uint32_t head = (i < shots && (i == 0 || keys[i] != keys[i - 1])) ? 1u : 0u;
        uint32_t inc = head;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            const uint32_t t = __shfl_up_sync(0xffffffffu, inc, o);
            if (lane >= o) inc += t;
        }
        if (lane == 31) wsum[warp] = inc;
        __syncthreads();
        if (warp == 0) {
            uint32_t v = lane < nw ? wsum[lane] : 0;
#pragma unroll
            for (int o = 1; o < 32; o <<= 1) {
                const uint32_t t = __shfl_up_sync(0xffffffffu, v, o);
                if (lane >= o) v += t;
            }
            wsum[lane] = v;
        }
        __syncthreads();
        const uint32_t pos = carry + (warp ? wsum[warp - 1] : 0) + inc - head;
        if (head) {
            okeys[pos] = keys[i];
            ocnt[pos] = i;
        }
        __syncthreads();
        if (threadIdx.x == blockDim.x - 1) carry = pos + head;
        __syncthreads();
    }
    const uint32_t nd = carry;
    for (uint32_t base = 0; base < nd; base += blockDim.x) {
        const uint32_t d = base + threadIdx.x;
        uint32_t c = 0;
        if (d < nd) c = (d + 1 < nd ? ocnt[d + 1] : shots) - ocnt[d];
        __syncthreads();
        if (d < nd) ocnt[d] = c;
        __syncthreads();
    }
    if (threadIdx.x == 0) n_distinct[traj] = nd;
}

}  // namespace

uint64_t next_pow2_u64(uint64_t v) { return next_pow2(v); }

cudaError_t launch_batch_sample(const float2* states, int n, int n_traj, uint32_t shots, uint64_t seed,
                                uint32_t* out_keys, uint32_t* out_counts, uint32_t* n_distinct, cudaStream_t st,
                                uint64_t* launches) {
    const int bsz = n >= 10 ? 1024 : (1 << n);
    const uint64_t nb = (1ull << n) / bsz;
    const uint32_t P = static_cast<uint32_t>(next_pow2(shots));
    const size_t smem = sizeof(uint64_t) * nb + sizeof(uint32_t) * P;
    {
        cudaError_t e = set_smem_attr(reinterpret_cast<const void*>(k_batch_sample), static_cast<int>(smem));
        if (e != cudaSuccess) return e;
    }
    k_batch_sample<<<n_traj, kBatchSampleThreads, smem, st>>>(states, n, shots, P, seed, out_keys, out_counts,
                                                              n_distinct);
    ++*launches;
    return cudaGetLastError();
}

// Diagonal of a vectorised density matrix (2n-qubit state, vec index
// x + 2^n x): optional copy of rho_xx (real part) to out[], and per-block
// FP64 partial sums of rho_xx (-1)^popc(x & mask) for the final reduction.
__global__ void __launch_bounds__(kRedThreads) k_dm_diag(const float2* __restrict__ psi, Layout lay, int n,
                                                          uint64_t mask, double* __restrict__ out,
                                                          double* __restrict__ partials) {
    const uint64_t dim = 1ull << n;
    const uint64_t stride = static_cast<uint64_t>(gridDim.x) * blockDim.x;
    double acc = 0.0;
    for (uint64_t x = static_cast<uint64_t>(blockIdx.x) * blockDim.x + threadIdx.x; x < dim; x += stride) {
        const double p = psi[encode_logical(x | (x << n), lay)].x;
        if (out) out[x] = p;
        acc += (__popcll(x & mask) & 1) ? -p : p;
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) acc += __shfl_xor_sync(0xffffffffu, acc, o);
    __shared__ double sh[kRedThreads / 32];
    if ((threadIdx.x & 31) == 0) sh[threadIdx.x >> 5] = acc;
    __syncthreads();
    if (threadIdx.x == 0) {
        double t = 0.0;
        for (int w = 0; w < kRedThreads / 32; ++w) t += sh[w];
        partials[blockIdx.x] = t;
    }
}

int reduce_partials() { return num_sms() * kRedBlocksPerSM; }

cudaError_t launch_reduce_z(const float2* psi, int n, uint64_t physmask, double* d_partials, double* d_out,
                            cudaStream_t st, uint64_t* launches) {
    const uint64_t npairs = (1ull << n) >> 1;
    const int nb = reduce_partials();
    if (npairs == 0) {
        // n = 1 is still >= one pair; n >= 1 always holds here
        return cudaErrorInvalidValue;
    }
    k_reduce_z<<<nb, kRedThreads, 0, st>>>(reinterpret_cast<const float4*>(psi), npairs, physmask, d_partials);
    k_finalize_sum<<<1, 1024, 0, st>>>(d_partials, nb, d_out);
    *launches += 2;
    return cudaGetLastError();
}

cudaError_t launch_reduce_z_multi(const float2* psi, int n, const uint64_t* physmasks, int nmasks,
                                  double* d_partials, double* d_out, cudaStream_t st, uint64_t* launches) {
    if (nmasks < 1 || nmasks > kMaxZMasks || n < 1) return cudaErrorInvalidValue;
    const uint64_t npairs = (1ull << n) >> 1;
    const int nb = reduce_partials();
    ZMasks zm{};
    zm.n = nmasks;
    for (int m = 0; m < nmasks; ++m) zm.m[m] = physmasks[m];
    k_reduce_z_multi<<<nb, kRedThreads, 0, st>>>(reinterpret_cast<const float4*>(psi), npairs, zm, d_partials);
    for (int m = 0; m < nmasks; ++m) k_finalize_sum<<<1, 1024, 0, st>>>(d_partials + m * nb, nb, d_out + m);
    *launches += 1 + nmasks;
    return cudaGetLastError();
}

cudaError_t launch_dm_diag(const float2* psi, int n, const int32_t* layout_host, uint64_t mask, double* d_out,
                           double* d_partials, double* d_sum, cudaStream_t st, uint64_t* launches) {
    Layout lay{};
    lay.n = 2 * n;
    for (int q = 0; q < 2 * n; ++q) lay.L[q] = layout_host[q];
    const int nb = reduce_partials();
    k_dm_diag<<<nb, kRedThreads, 0, st>>>(psi, lay, n, mask, d_out, d_partials);
    k_finalize_sum<<<1, 1024, 0, st>>>(d_partials, nb, d_sum);
    *launches += 2;
    return cudaGetLastError();
}

cudaError_t launch_probs_logical(const float2* psi, int n, const int32_t* layout_host, double* out, cudaStream_t st,
                                 uint64_t* launches) {
    Layout lay{};
    lay.n = n;
    for (int q = 0; q < n; ++q) lay.L[q] = layout_host[q];
    const uint64_t dim = 1ull << n;
    uint64_t blocks = (dim + 255) / 256;
    const uint64_t cap = static_cast<uint64_t>(num_sms()) * 16;
    if (blocks > cap) blocks = cap;
    k_probs_logical<<<static_cast<unsigned>(blocks), 256, 0, st>>>(psi, lay, out);
    ++*launches;
    return cudaGetLastError();
}

size_t sample_scratch_bytes(int n, uint64_t shots) {
    const int bsz = n >= 10 ? 1024 : (1 << n);
    const uint64_t nblocks = (1ull << n) / bsz;
    const uint64_t P = next_pow2(shots);
    return sizeof(uint64_t) * (nblocks + P + shots) + 256;
}

cudaError_t launch_sample(const float2* psi, int n, const int32_t* layout_host, uint64_t shots, uint64_t seed,
                          uint64_t stream_id, void* d_scratch, uint64_t* d_out_keys, uint64_t* d_out_counts,
                          uint64_t* d_n_distinct, cudaStream_t st, uint64_t* launches) {
    return launch_sample_z(psi, n, layout_host, shots, seed, stream_id, d_scratch, d_out_keys, d_out_counts,
                           d_n_distinct, nullptr, 0, nullptr, nullptr, st, launches);
}

cudaError_t launch_sample_z(const float2* psi, int n, const int32_t* layout_host, uint64_t shots, uint64_t seed,
                            uint64_t stream_id, void* d_scratch, uint64_t* d_out_keys, uint64_t* d_out_counts,
                            uint64_t* d_n_distinct, const uint64_t* physmasks, int nmasks, double* d_zpartials,
                            double* d_zout, cudaStream_t st, uint64_t* launches) {
    if (nmasks < 0 || nmasks > kMaxZMasks) return cudaErrorInvalidValue;
    Layout lay{};
    lay.n = n;
    for (int q = 0; q < n; ++q) lay.L[q] = layout_host[q];
    const int bsz = n >= 10 ? 1024 : (1 << n);
    const uint64_t nblocks = (1ull << n) / bsz;
    const uint64_t P = next_pow2(shots);
    uint64_t* cum = reinterpret_cast<uint64_t*>(d_scratch);
    uint64_t* keys = cum + nblocks;
    uint64_t* starts = keys + P;

    const unsigned wpb = 8;  // warps per CTA
    if (bsz == 1024) {
        ZMasks zm{};
        zm.n = nmasks;
        for (int m = 0; m < nmasks; ++m) zm.m[m] = physmasks[m];
        auto kern = nmasks == 0 ? k_weights_z1024<0> : nmasks == 1 ? k_weights_z1024<1>
                  : nmasks == 2 ? k_weights_z1024<2> : nmasks == 3 ? k_weights_z1024<3> : k_weights_z1024<4>;
        // as many CTAs as stay resident (at most reduce_partials(), the partials' size)
        int occ = 0;
        cudaError_t e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, kern, kRedThreads, 0);
        if (e != cudaSuccess) return e;
        occ = occ < 1 ? 1 : (occ > kRedBlocksPerSM ? kRedBlocksPerSM : occ);
        uint64_t nb = (nblocks + wpb - 1) / wpb;
        const uint64_t cap = static_cast<uint64_t>(num_sms()) * occ;
        if (nb > cap) nb = cap;
        kern<<<static_cast<unsigned>(nb), kRedThreads, 0, st>>>(reinterpret_cast<const float4*>(psi), nblocks, cum,
                                                                 zm, d_zpartials);
        for (int m = 0; m < nmasks; ++m)
            k_finalize_sum<<<1, 1024, 0, st>>>(d_zpartials + m * nb, static_cast<int>(nb), d_zout + m);
        *launches += nmasks;
    } else if (nmasks > 0) {
        ZMasks zm{};
        zm.n = nmasks;
        for (int m = 0; m < nmasks; ++m) zm.m[m] = physmasks[m];
        const int nb = reduce_partials();
        k_block_weights_z<<<nb, kRedThreads, 0, st>>>(psi, nblocks, bsz, cum, zm, d_zpartials);
        for (int m = 0; m < nmasks; ++m) k_finalize_sum<<<1, 1024, 0, st>>>(d_zpartials + m * nb, nb, d_zout + m);
        *launches += nmasks;
    } else {
        k_block_weights<<<static_cast<unsigned>((nblocks + wpb - 1) / wpb), wpb * 32, 0, st>>>(psi, nblocks, bsz,
                                                                                                cum);
    }
    const uint64_t nseg = (nblocks + kScanSeg - 1) / kScanSeg;
    if (nseg > 1 && nseg <= P + shots) {
        // segment totals in the key area, which k_draw fills only afterwards
        k_scan_segments<<<static_cast<unsigned>(nseg), 1024, 0, st>>>(cum, nblocks, keys);
        k_scan_inclusive<<<1, 1024, 0, st>>>(keys, nseg);
        uint64_t ab = (nblocks - kScanSeg + 255) / 256;
        const uint64_t cap = static_cast<uint64_t>(num_sms()) * 8;
        if (ab > cap) ab = cap;
        k_scan_add<<<static_cast<unsigned>(ab), 256, 0, st>>>(cum, nblocks, keys);
        *launches += 2;
    } else {
        k_scan_inclusive<<<1, 1024, 0, st>>>(cum, nblocks);
    }
    k_draw<<<static_cast<unsigned>((shots + wpb - 1) / wpb), wpb * 32, 0, st>>>(psi, cum, nblocks, bsz, lay, shots,
                                                                                 seed, stream_id, keys);
    *launches += 3;
    if (P > shots) {
        k_fill_u64<<<static_cast<unsigned>((P - shots + 255) / 256), 256, 0, st>>>(keys, shots, P, ~0ull);
        ++*launches;
    }
    if (P <= 4096) {
        k_bitonic_smem<<<1, 1024, sizeof(uint64_t) * P, st>>>(keys, static_cast<int>(P));
        ++*launches;
    } else {
        const unsigned nb = static_cast<unsigned>((P + 255) / 256);
        for (uint64_t k = 2; k <= P; k <<= 1)
            for (uint64_t j = k >> 1; j > 0; j >>= 1) {
                k_bitonic_step<<<nb, 256, 0, st>>>(keys, P, j, k);
                ++*launches;
            }
    }
    k_rle<<<1, 1024, 0, st>>>(keys, shots, d_out_keys, starts, d_out_counts, d_n_distinct);
    ++*launches;
    return cudaGetLastError();
}

}  // namespace qsa

// ---------------------------------------------------------------------------
// Sampling without any device allocation.
//
// Some callers cannot let the library call cudaMalloc: a framework whose
// caching allocator owns the device memory budget (a stray cudaMalloc can fail
// or fragment the pool when the state fills most of HBM, as at N = 33/34), or
// a pipeline that must not stall, since cudaFree synchronises the whole
// device.  For them the sampler's scratch (block cumulative weights, the sort
// keys and the run starts) lives in one fixed, file-scope device array that
// every GPU loading this library holds until the process exits.
// ---------------------------------------------------------------------------
#include <mutex>
#include <string>

#include "qsa_runtime.h"

namespace {
constexpr uint64_t kNoAllocWords = QSA_NOALLOC_SCRATCH_WORDS;
static __device__ __align__(256) uint64_t g_noalloc_scratch[kNoAllocWords];

std::mutex g_noalloc_mu;
void* g_noalloc_addr[256] = {};

// Device address of the array for the current device, looked up once per
// device (host code only sees a host-side stand-in for the symbol).
cudaError_t noalloc_scratch_ptr(void** out) {
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return e;
    if (dev < 0 || dev >= 256) return cudaErrorInvalidDevice;
    std::lock_guard<std::mutex> g(g_noalloc_mu);
    if (!g_noalloc_addr[dev]) {
        void* p = nullptr;
        e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
        if (e != cudaSuccess) return e;
        g_noalloc_addr[dev] = p;
    }
    *out = g_noalloc_addr[dev];
    return cudaSuccess;
}
}  // namespace

extern "C" qsa_status qsa_sample_counts_noalloc(const void* dev_amplitudes, int n_qubits,
                                                const int32_t* phys_of_logical, uint64_t shots, uint64_t seed,
                                                uint64_t* out_outcomes_dev, uint64_t* out_counts_dev,
                                                uint64_t* out_n_distinct_dev, void* cuda_stream) {
    using qsa::fail;
    if (!dev_amplitudes || (reinterpret_cast<uintptr_t>(dev_amplitudes) % 16))
        return fail(QSA_E_ARG, "amplitudes must be a non-NULL, 16-byte aligned device pointer");
    if (n_qubits < 1 || n_qubits > QSA_MAX_QUBITS) return fail(QSA_E_ARG, "n_qubits must be in 1..34");
    if (!phys_of_logical) return fail(QSA_E_ARG, "layout is NULL");
    uint64_t seen = 0;
    for (int q = 0; q < n_qubits; ++q) {
        const int p = phys_of_logical[q];
        if (p < 0 || p >= n_qubits || ((seen >> p) & 1)) return fail(QSA_E_ARG, "layout is not a bijection");
        seen |= 1ull << p;
    }
    if (shots < 1 || shots > (1ull << 26)) return fail(QSA_E_ARG, "shots must be in 1..2^26");
    if (!out_outcomes_dev || !out_counts_dev || !out_n_distinct_dev) return fail(QSA_E_ARG, "output is NULL");
    const int bsz = n_qubits >= 10 ? 1024 : (1 << n_qubits);
    const uint64_t nblocks = (1ull << n_qubits) / bsz;
    const uint64_t need = nblocks + qsa::next_pow2_u64(shots) + shots;
    if (need > kNoAllocWords)
        return fail(QSA_E_RANGE, "request needs " + std::to_string(need) + " words of sampler scratch; the fixed "
                                 "no-allocation buffer holds " + std::to_string(kNoAllocWords) +
                                 " (2^(N-10) + next_pow2(shots) + shots must fit)");
    void* scratch = nullptr;
    cudaError_t e = noalloc_scratch_ptr(&scratch);
    if (e != cudaSuccess) return fail(QSA_E_CUDA, std::string("cudaGetSymbolAddress: ") + cudaGetErrorString(e));
    uint64_t launches = 0;
    e = qsa::launch_sample(static_cast<const float2*>(dev_amplitudes), n_qubits, phys_of_logical, shots, seed, 0,
                           scratch, out_outcomes_dev, out_counts_dev, out_n_distinct_dev,
                           static_cast<cudaStream_t>(cuda_stream), &launches);
    if (e != cudaSuccess) return fail(QSA_E_CUDA, std::string("sampler kernels: ") + cudaGetErrorString(e));
    return QSA_OK;
}
