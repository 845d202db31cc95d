// FP32 fused dense update, qubit-permutation and batched-trajectory kernels
// (sm_103a).
//
// All three share one tile engine: a CTA walks tiles t0, t0 + stride, ...;
// each tile (2^T amplitudes = 2^nx contiguous runs of 2^m amplitudes) is
// staged into shared memory with 16-byte cp.async copies in an S-deep ring,
// transformed, and written back in place.  Tiles partition the index space,
// so the in-place update needs no second state buffer (the paper's CUDA path
// holds two, App. C "Capacity and execution profiles").
//
//   apply   (§IV-B, R2 apply; Eq. cost-formal): for every group of 2^k
//           amplitudes that differ only in the target bits,
//           psi'[x|spread(r)] = sum_c G[r][c] psi[x|spread(c)];
//   permute (§IV-D, Lemma "distributed promotion swap" with the rank bits read
//           as out-of-block bits): psi'[tau(y)] = psi[y] for a product tau of
//           disjoint bit transpositions;
//   batch   many independent states (noisy trajectories, §IV-A channels
//           sampled as explicit Pauli branches) in one persistent launch: each
//           CTA pops a trajectory from an atomic queue (longest first), resets
//           it to |0...0> and applies all of its fused blocks.
#include <cooperative_groups.h>
#include <cuda_runtime.h>

#include <algorithm>
#include <cstdint>
#include <map>
#include <mutex>
#include <utility>

#include "qsa_bounds.cuh"
#include "qsa_device.cuh"
#include "qsa_internal.h"

namespace qsa {

namespace {

using namespace dev;

constexpr int kThreads = 256;

struct TileArgs {
    float2* psi;
    uint64_t ntiles;
    int T, m, nx;
    int xpos[6];
};

__device__ __forceinline__ uint64_t tile_base(const TileArgs& a, uint64_t t) {
    uint64_t b = t << a.m;
#pragma unroll
    for (int e = 0; e < 6; ++e)
        if (e < a.nx) b = insert_zero(b, a.xpos[e]);
    return b;
}

// Global index of tile-local index j.
__device__ __forceinline__ uint64_t tile_global(const TileArgs& a, const uint64_t* runoff, uint64_t base,
                                                uint32_t j) {
    return base | (j & ((1u << a.m) - 1u)) | runoff[j >> a.m];
}

__device__ __forceinline__ void build_runoff(const TileArgs& a, uint64_t* runoff) {
    for (int r = threadIdx.x; r < (1 << a.nx); r += blockDim.x) {
        uint64_t off = 0;
#pragma unroll
        for (int e = 0; e < 6; ++e)
            if (e < a.nx && ((r >> e) & 1)) off |= 1ull << a.xpos[e];
        runoff[r] = off;
    }
}

// Issue the 16-byte copies of tile t into stage buffer `st`.
__device__ __forceinline__ void load_tile(const TileArgs& a, const uint64_t* runoff, uint64_t t, float2* st) {
    const uint64_t base = tile_base(a, t);
    const uint32_t chunks = 1u << (a.T - 1);
    for (uint32_t q = threadIdx.x; q < chunks; q += blockDim.x) {
        uint32_t j = q << 1;
        const uint64_t gi = tile_global(a, runoff, base, j);
        if (dbg::in_bounds(gi, 2, a.ntiles << a.T, 1)) cp_async16(st + j, a.psi + gi);
    }
}

// ---------------------------------------------------------------------------
// Apply
// ---------------------------------------------------------------------------
struct ApplyArgs {
    TileArgs t;
    const float* mat;   // 2 * 4^K floats
    int tl[6];          // tile-local position of target j (V order)
    int tls[6];         // the same positions, ascending
    uint8_t fv[16];     // stage layout: slot vector of tile-local position p >= 4 (k <= 4)
    // k <= 4 launches: the tile-local offsets of a group's D members in the plain (loffc) and the
    // swizzled (sloffc) stage, formed on the host and read at compile-time member indices from the
    // parameter bank
    int loffc[16];
    int sloffc[16];
};

// Stage layout of the k <= 4 kernels: tile-local element j sits at
// j ^ (h(j >> 4) << 1), h linear with h(bit i) = fv[4 + i].  Position 0 stays
// the element within a 16-byte unit and positions 1..3 its slot in a 128-byte
// line, so the copies in and out move whole 16-byte units with eight lanes on
// eight slots; the slot vectors of higher positions are chosen per launch so
// that the lowest non-target positions (the bits that vary across a
// half-warp's groups) land on distinct banks.
__device__ __forceinline__ uint32_t stage_xor(const uint8_t* htab, uint32_t j) {
    return static_cast<uint32_t>(htab[j >> 4]) << 1;
}

__device__ __forceinline__ void build_htab(const ApplyArgs& a, uint8_t* htab) {
    const int n = 1 << (a.t.T - 4);
    for (int x = threadIdx.x; x < n; x += blockDim.x) {
        uint32_t h = 0;
#pragma unroll
        for (int i = 0; i < 12; ++i)   // constant indices keep the arguments in parameter space
            if (i < a.t.T - 4 && ((x >> i) & 1)) h ^= a.fv[4 + i];
        htab[x] = static_cast<uint8_t>(h);
    }
}

__device__ __forceinline__ void load_tile_swz(const TileArgs& a, const uint64_t* runoff, const uint8_t* htab, uint64_t t,
                                              float2* st) {
    const uint64_t base = tile_base(a, t);
    const uint32_t chunks = 1u << (a.T - 1);
    for (uint32_t q = threadIdx.x; q < chunks; q += blockDim.x) {
        const uint32_t j = q << 1;
        const uint64_t gi = tile_global(a, runoff, base, j);
        if (dbg::in_bounds(gi, 2, a.ntiles << a.T, 2)) cp_async16(st + (j ^ stage_xor(htab, j)), a.psi + gi);
    }
}

// Write a transformed tile back in address order (16-byte units).  All of a
// thread's shared-memory reads come before its stores, which they could not
// pass otherwise.
template <int UNITS>
__device__ __forceinline__ void store_tile_swz(const TileArgs& a, const uint64_t* runoff, const uint8_t* htab,
                                               uint64_t t, const float2* st) {
    const uint64_t base = tile_base(a, t);
    float4 v[UNITS];
    uint64_t g[UNITS];
#pragma unroll
    for (int u = 0; u < UNITS; ++u) {
        const uint32_t j = (threadIdx.x + u * blockDim.x) << 1;
        v[u] = *reinterpret_cast<const float4*>(st + (j ^ stage_xor(htab, j)));
        g[u] = tile_global(a, runoff, base, j);
    }
#pragma unroll
    for (int u = 0; u < UNITS; ++u)
        if (dbg::in_bounds(g[u], 2, a.ntiles << a.T, 3)) __stcs(reinterpret_cast<float4*>(a.psi + g[u]), v[u]);
}

// The tile pipeline of one fused operator over tiles t0, t0 + stride, ...
// Ms (G as float2[D][D]), runoff and loff are set up in shared memory.
// SWZ (k <= 4): the stage takes the swizzled layout (htab; sloff holds the
// swizzled group offsets), so a half-warp's gathers meet at most two to a
// bank wherever the targets sit.  WB (with SWZ, one item per group): each
// item writes its outputs in place and the tile goes back in address order
// (16-byte units of 2^TB-amplitude tiles), for target sets whose direct
// stores would give every lane its own sector.
template <int K, int R, int S, bool SWZ = false, bool WB = false, int TB = 11, bool PO = false>
__device__ __forceinline__ void apply_tiles(const ApplyArgs& a, float2* stage, const float2* Ms,
                                            const uint64_t* runoff, const int* loff, uint64_t t0, uint64_t stride,
                                            const uint8_t* htab = nullptr, const int* sloff = nullptr) {
    constexpr int D = 1 << K;
    static_assert(!WB || (SWZ && R == D), "in-place outputs: swizzled stage, the whole group in one item");
    // PO: member offsets from the parameter bank (k <= 4)
    static_assert(!PO || D <= 16, "parameter-bank member offsets: k <= 4");
    auto moff = [&](int c) { return PO ? a.loffc[c] : loff[c]; };
    auto msoff = [&](int c) { return PO ? a.sloffc[c] : sloff[c]; };
    const int tileAmps = 1 << a.t.T;
    auto load = [&](uint64_t t, float2* st) {
        if constexpr (SWZ)
            load_tile_swz(a.t, runoff, htab, t, st);
        else
            load_tile(a.t, runoff, t, st);
    };
#pragma unroll
    for (int s = 0; s < S - 1; ++s) {
        uint64_t t = t0 + s * stride;
        if (t < a.t.ntiles) load(t, stage + s * tileAmps);
        cp_async_commit();
    }
    const int G = tileAmps >> K;                  // groups per tile
    const int gshift = a.t.T - K;
    const int items = G * (D / R);
    int it_stage = 0;
    for (uint64_t t = t0; t < a.t.ntiles; t += stride) {
        uint64_t tn = t + (S - 1) * stride;
        int ld_stage = it_stage + (S - 1);
        if (ld_stage >= S) ld_stage -= S;
        if (tn < a.t.ntiles) load(tn, stage + ld_stage * tileAmps);
        cp_async_commit();
        cp_async_wait<S - 1>();
        __syncthreads();

        float2* st = stage + it_stage * tileAmps;
        const uint64_t base = tile_base(a.t, t);
        for (int it = threadIdx.x; it < items; it += blockDim.x) {
            const int g = it & (G - 1);
            const int rb = it >> gshift;
            uint32_t lb = static_cast<uint32_t>(g);
#pragma unroll
            for (int j = 0; j < K; ++j) lb = static_cast<uint32_t>(insert_zero(lb, a.tls[j]));
            const uint32_t lbs = SWZ ? (lb ^ stage_xor(htab, lb)) : lb;   // the group's base in the stage
            if constexpr (K <= 5) {
                // Packed FP32 pairs: with x2_c = (Re v_c, Re v_c), y2_c = (Im v_c, Im v_c)
                // and g = (Re G, Im G), p = sum x2_c * g and q = sum y2_c * g give
                // Re = p.x - q.y and Im = p.y + q.x; one 16-byte load of two G entries
                // feeds four f32x2 FMAs.
                uint64_t x2[D], y2[D];
#pragma unroll
                for (int c = 0; c < D; ++c) {
                    const float2 f = SWZ ? st[lbs ^ msoff(c)] : st[lb | moff(c)];
                    x2[c] = pack2(f.x, f.x);
                    y2[c] = pack2(f.y, f.y);
                }
#pragma unroll
                for (int rr = 0; rr < R; ++rr) {
                    const int r = rb * R + rr;
                    const ulonglong2* mrow = reinterpret_cast<const ulonglong2*>(Ms + r * D);
                    uint64_t p = 0, qv = 0;
#pragma unroll
                    for (int c = 0; c < D; c += 2) {
                        const ulonglong2 gg = mrow[c >> 1];  // G[r][c], G[r][c+1]
                        p = fma2(x2[c], gg.x, p);
                        qv = fma2(y2[c], gg.x, qv);
                        p = fma2(x2[c + 1], gg.y, p);
                        qv = fma2(y2[c + 1], gg.y, qv);
                    }
                    const float2 P = unpack2(p), Q = unpack2(qv);
                    if constexpr (WB) {
                        st[lbs ^ msoff(r)] = make_float2(P.x - Q.y, P.y + Q.x);   // in place: inputs are in registers
                    } else {
                        const uint64_t gj = tile_global(a.t, runoff, base, lb | moff(r));
                        if (dbg::in_bounds(gj, 1, a.t.ntiles << a.t.T, 4))
                            __stcs(a.t.psi + gj, make_float2(P.x - Q.y, P.y + Q.x));
                    }
                }
            } else {
                float2 v[D];
#pragma unroll
                for (int c = 0; c < D; ++c) v[c] = st[lb | loff[c]];
#pragma unroll
                for (int rr = 0; rr < R; ++rr) {
                    const int r = rb * R + rr;
                    const float4* mrow = reinterpret_cast<const float4*>(Ms + r * D);
                    float ar = 0.f, ai = 0.f;
#pragma unroll
                    for (int c = 0; c < D; c += 2) {
                        float4 m2 = mrow[c >> 1];  // G[r][c], G[r][c+1]
                        ar = fmaf(m2.x, v[c].x, ar);
                        ar = fmaf(-m2.y, v[c].y, ar);
                        ai = fmaf(m2.x, v[c].y, ai);
                        ai = fmaf(m2.y, v[c].x, ai);
                        ar = fmaf(m2.z, v[c + 1].x, ar);
                        ar = fmaf(-m2.w, v[c + 1].y, ar);
                        ai = fmaf(m2.z, v[c + 1].y, ai);
                        ai = fmaf(m2.w, v[c + 1].x, ai);
                    }
                    const uint64_t gj = tile_global(a.t, runoff, base, lb | loff[r]);
                    if (dbg::in_bounds(gj, 1, a.t.ntiles << a.t.T, 4)) __stcs(a.t.psi + gj, make_float2(ar, ai));
                }
            }
        }
        if constexpr (WB) {
            __syncthreads();
            store_tile_swz<(1 << (TB - 1)) / kThreads>(a.t, runoff, htab, t, st);
        }
        __syncthreads();
        if (++it_stage == S) it_stage = 0;
    }
    cp_async_wait<0>();
}

template <int K>
__device__ __forceinline__ void build_loff(const int* tl, int* loff) {
    constexpr int D = 1 << K;
    for (int c = threadIdx.x; c < D; c += blockDim.x) {
        int o = 0;
#pragma unroll
        for (int j = 0; j < K; ++j)
            if ((c >> j) & 1) o |= 1 << tl[j];
        loff[c] = o;
    }
}

template <int K, int R, int S, bool SWZ, bool WB, int TB>
__global__ void __launch_bounds__(kThreads) k_apply_fp32(ApplyArgs a) {
    constexpr int D = 1 << K;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    const int tileAmps = 1 << a.t.T;
    float2* stage = reinterpret_cast<float2*>(smem_raw);
    float2* Ms = stage + S * tileAmps;
    uint64_t* runoff = reinterpret_cast<uint64_t*>(Ms + D * D);
    int* loff = reinterpret_cast<int*>(runoff + 64);
    int* sloff = loff + 64;
    uint8_t* htab = reinterpret_cast<uint8_t*>(sloff + 64);

    const float2* gm = reinterpret_cast<const float2*>(a.mat);
    for (int i = threadIdx.x; i < D * D; i += blockDim.x) Ms[i] = gm[i];
    build_runoff(a.t, runoff);
    build_loff<K>(a.tl, loff);
    if constexpr (SWZ) {
        build_htab(a, htab);
        __syncthreads();
        for (int c = threadIdx.x; c < D; c += blockDim.x) sloff[c] = loff[c] ^ static_cast<int>(stage_xor(htab, loff[c]));
    }
    __syncthreads();
    apply_tiles<K, R, S, SWZ, WB, TB, (K <= 4)>(a, stage, Ms, runoff, loff, blockIdx.x, gridDim.x, htab, sloff);
}

template <int K>
struct ApplyCfg;
// SWZ: the swizzled stage and, where the targets call for it, in-place outputs
// with an address-order write-back are available (k <= 4).
template <> struct ApplyCfg<1> { static constexpr int T = 11, R = 2, S = 2; static constexpr bool SWZ = true; };
template <> struct ApplyCfg<2> { static constexpr int T = 11, R = 4, S = 2; static constexpr bool SWZ = true; };
template <> struct ApplyCfg<3> { static constexpr int T = 11, R = 8, S = 2; static constexpr bool SWZ = true; };
// k = 4: 2^12-amplitude tiles, so that a tile has one 16-row item per thread
// (2^11 left half of the CTA idle in the compute phase), two stages so that
// three CTAs fit an SM (faster than three stages at two CTAs)
template <> struct ApplyCfg<4> { static constexpr int T = 12, R = 16, S = 2; static constexpr bool SWZ = true; };
template <> struct ApplyCfg<5> { static constexpr int T = 12, R = 8, S = 2; static constexpr bool SWZ = false; };
template <> struct ApplyCfg<6> { static constexpr int T = 12, R = 8, S = 2; static constexpr bool SWZ = false; };

// Form of a k <= 4 launch from its lowest non-target tile positions np[0..4]
// (the group-index bits that vary across a warp).  With the plain layout a
// half-warp's gathers spread over 2^(#np[0..3] below 4) of the 16 bank pairs,
// and a warp's direct 8-byte stores over 32 / 2^(#np[0..4] below 2) sectors.
// 0: plain layout, direct stores; 1: swizzled gathers, direct stores (gathers
// four or more to a bank); 2: swizzled gathers and in-place write-back (one
// sector per lane).  The thresholds follow CUDA-event timings of all three
// forms on target sets at N = 30.
int apply_form(int T, const int* tls, int k) {
    int np[5], nn = 0;
    for (int p = 0; p < T && nn < 5; ++p) {
        bool tgt = false;
        for (int j = 0; j < k; ++j) tgt = tgt || tls[j] == p;
        if (!tgt) np[nn++] = p;
    }
    int low4 = 0, low2 = 0;
    for (int b = 0; b < nn; ++b) {
        if (b < 4 && np[b] < 4) ++low4;
        if (np[b] < 2) ++low2;
    }
    if (low2 == 0) return 2;
    if (low4 <= 2) return 1;
    return 0;
}

// Slot vectors of the swizzled stage: the four lowest non-target tile
// positions take distinct slot bits where they can (positions 1..3 own theirs;
// a higher one takes a free one; position 0 is the element within a unit).
void stage_slots(int T, const int* tls, int k, uint8_t* fv) {
    for (int p = 0; p < 16; ++p) fv[p] = 0;
    int np[4], nn = 0;
    for (int p = 0; p < T && nn < 4; ++p) {
        bool tgt = false;
        for (int j = 0; j < k; ++j) tgt = tgt || tls[j] == p;
        if (!tgt) np[nn++] = p;
    }
    uint32_t used = 0;
    for (int b = 0; b < nn; ++b)
        if (np[b] >= 1 && np[b] <= 3) used |= 1u << (np[b] - 1);
    for (int b = 0; b < nn; ++b)
        if (np[b] >= 4) {
            int j = 0;
            while (j < 3 && ((used >> j) & 1u)) ++j;
            if (j < 3) {
                used |= 1u << j;
                fv[np[b]] = static_cast<uint8_t>(1u << j);
            }
        }
}

// Tile-local positions of the targets for geometry g.
void local_targets(const TileGeom& g, const int* phys, int k, int* tl, int* tls) {
    for (int j = 0; j < k; ++j) {
        int p = phys[j];
        int loc = p;
        if (p >= g.m) {
            int e = 0;
            while (g.xpos[e] != p) ++e;
            loc = g.m + e;
        }
        tl[j] = loc;
        tls[j] = loc;
    }
    std::sort(tls, tls + k);
}

template <int K>
cudaError_t launch_apply_k(float2* psi, int n, const int* phys, const float* d_mat, cudaStream_t st,
                           uint64_t* launches) {
    using C = ApplyCfg<K>;
    TileGeom g;
    if (!make_geom(n, phys, K, C::T, &g)) return cudaErrorInvalidValue;
    ApplyArgs a{};
    a.t.psi = psi;
    a.t.ntiles = g.ntiles;
    a.t.T = g.T;
    a.t.m = g.m;
    a.t.nx = g.nx;
    for (int e = 0; e < 6; ++e) a.t.xpos[e] = g.xpos[e];
    a.mat = d_mat;
    local_targets(g, phys, K, a.tl, a.tls);
    // the write-back is unrolled for full tiles (states of at least 2^T
    // amplitudes); smaller states take the plain form
    const int form = C::SWZ && g.T == C::T ? apply_form(g.T, a.tls, K) : 0;
    if (form) stage_slots(g.T, a.tls, K, a.fv);
    const int D = 1 << K;
    for (int c = 0; c < D && c < 16; ++c) {
        int o = 0;
        for (int j = 0; j < K; ++j)
            if ((c >> j) & 1) o |= 1 << a.tl[j];
        a.loffc[c] = o;
        // swizzled stage: o ^ (h(o >> 4) << 1), h the XOR of the slot vectors of o's bits from 4 on
        uint32_t h = 0;
        for (int i = 0; i < g.T - 4; ++i)
            if ((o >> (4 + i)) & 1) h ^= a.fv[4 + i];
        a.sloffc[c] = o ^ static_cast<int>(h << 1);
    }
    constexpr size_t tables = sizeof(uint64_t) * 64 + 2 * sizeof(int) * 64 + 256;
    const size_t smem = sizeof(float2) * (static_cast<size_t>(C::S) << g.T) + sizeof(float2) * D * D + tables;
    auto kern = form == 2   ? k_apply_fp32<K, C::R, C::S, C::SWZ, C::SWZ, C::T>
                : form == 1 ? k_apply_fp32<K, C::R, C::S, C::SWZ, false, C::T>
                            : k_apply_fp32<K, C::R, C::S, false, false, C::T>;
    {
        const size_t full = sizeof(float2) * (static_cast<size_t>(C::S) << C::T) + sizeof(float2) * D * D + tables;
        cudaError_t e = set_smem_attr(reinterpret_cast<const void*>(kern), static_cast<int>(full));
        if (e != cudaSuccess) return e;
    }
    int occ = 0;
    cudaError_t e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, kern, kThreads, smem);
    if (e != cudaSuccess) return e;
    if (occ < 1) occ = 1;
    uint64_t grid = static_cast<uint64_t>(num_sms()) * occ;
    if (grid > g.ntiles) grid = g.ntiles;
    kern<<<static_cast<unsigned>(grid), kThreads, smem, st>>>(a);
    ++*launches;
    return cudaGetLastError();
}

// ---------------------------------------------------------------------------
// Product of one-qubit factors (a structured fused block, §IV-D)
// ---------------------------------------------------------------------------
constexpr int kProdT = 11, kProdS = 3, kProdHigh = 3;

struct ProdArgs {
    TileArgs t;
    const float* fac;          // 8 floats per factor: 2x2 complex, row-major
    int k;
    int tl[QSA_MAX_PROD];      // tile-local position of factor j
};

// a x + b y for complex a, b, x, y.
__device__ __forceinline__ float2 cfma2(float2 a, float2 x, float2 b, float2 y) {
    return make_float2(a.x * x.x - a.y * x.y + b.x * y.x - b.y * y.y, a.x * x.y + a.y * x.x + b.x * y.y + b.y * y.x);
}

// One round over the staged tile.  A warp covers 32 x 2^H amplitudes: its
// lanes are tile-local bits 0..4 (so every shared-memory access of the warp
// touches 32 consecutive amplitudes), and each lane holds the 2^H
// combinations of the round's H high targets (positions >= 5, ascending
// hpos[]).  High factors are butterflies in registers, low factors (targets
// below 5) butterflies across lanes with shuffles.  The last round stores
// straight to HBM (32 consecutive amplitudes per warp store).
template <int H>
__device__ __forceinline__ void prod_round(const ProdArgs& a, float2* st, const float2* F, const int* hpos,
                                           const int* hfi, int nlow, const int* lpos, const int* lfi, bool last,
                                           const uint64_t* runoff, uint64_t base) {
    constexpr int G = 1 << H;
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nw = blockDim.x >> 5;
    const int units = (1 << a.t.T) >> (5 + H);
    // per round: each high target's tile-local bit and the global offset of
    // that bit (tile indexing is bitwise linear, so offsets add)
    uint32_t hm[H > 0 ? H : 1];
    uint64_t gb[H > 0 ? H : 1];
#pragma unroll
    for (int j = 0; j < H; ++j) {
        hm[j] = 1u << hpos[j];
        gb[j] = tile_global(a.t, runoff, 0, hm[j]);
    }
    for (int u = warp; u < units; u += nw) {
        uint32_t ub = static_cast<uint32_t>(u) << 5;
#pragma unroll
        for (int j = 0; j < H; ++j) ub = static_cast<uint32_t>(insert_zero(ub, hpos[j]));
        ub |= static_cast<uint32_t>(lane);
        float2 v[G];
#pragma unroll
        for (int c = 0; c < G; ++c) {
            uint32_t o = ub;
#pragma unroll
            for (int j = 0; j < H; ++j)
                if ((c >> j) & 1) o |= hm[j];
            v[c] = st[o];
        }
#pragma unroll
        for (int j = 0; j < H; ++j) {
            const float2* U = F + 4 * hfi[j];
#pragma unroll
            for (int c = 0; c < G; ++c) {
                if ((c >> j) & 1) continue;
                const float2 x = v[c], y = v[c | (1 << j)];
                v[c] = cfma2(U[0], x, U[1], y);
                v[c | (1 << j)] = cfma2(U[3], y, U[2], x);
            }
        }
        for (int l = 0; l < nlow; ++l) {
            const int m = 1 << lpos[l];
            const float2* U = F + 4 * lfi[l];
            // bit clear: u00 x + u01 y; bit set: u11 x + u10 y (x own, y partner)
            const bool one = (lane & m) != 0;
            const float2 ua = one ? U[3] : U[0], ub2 = one ? U[2] : U[1];
#pragma unroll
            for (int c = 0; c < G; ++c) {
                float2 y;
                y.x = __shfl_xor_sync(0xffffffffu, v[c].x, m);
                y.y = __shfl_xor_sync(0xffffffffu, v[c].y, m);
                v[c] = cfma2(ua, v[c], ub2, y);
            }
        }
        if (last) {
            const uint64_t g0 = tile_global(a.t, runoff, base, ub);
#pragma unroll
            for (int c = 0; c < G; ++c) {
                uint64_t go = 0;
#pragma unroll
                for (int j = 0; j < H; ++j)
                    if ((c >> j) & 1) go += gb[j];
                if (dbg::in_bounds(g0 + go, 1, a.t.ntiles << a.t.T, 5)) __stcs(a.t.psi + g0 + go, v[c]);
            }
        } else {
#pragma unroll
            for (int c = 0; c < G; ++c) {
                uint32_t o = ub;
#pragma unroll
                for (int j = 0; j < H; ++j)
                    if ((c >> j) & 1) o |= hm[j];
                st[o] = v[c];
            }
        }
    }
}

__global__ void __launch_bounds__(kThreads) k_apply_prod(ProdArgs a) {
    extern __shared__ __align__(16) unsigned char smem_raw[];
    const int tileAmps = 1 << a.t.T;
    float2* stage = reinterpret_cast<float2*>(smem_raw);
    float2* F = stage + kProdS * tileAmps;
    uint64_t* runoff = reinterpret_cast<uint64_t*>(F + 4 * QSA_MAX_PROD);
    const float2* gf = reinterpret_cast<const float2*>(a.fac);
    for (int i = threadIdx.x; i < 4 * a.k; i += blockDim.x) F[i] = gf[i];
    build_runoff(a.t, runoff);
    // factors on tile-local bits 0..4 act across lanes (all in round 0); the
    // others, ascending by position, go kProdHigh per round
    int hpos[QSA_MAX_PROD], hfi[QSA_MAX_PROD], lpos[5], lfi[5];
    int nh = 0, nl = 0;
    for (int j = 0; j < a.k; ++j) {
        if (a.tl[j] < 5) {
            lpos[nl] = a.tl[j];
            lfi[nl++] = j;
        } else {
            int x = nh++;
            while (x > 0 && hpos[x - 1] > a.tl[j]) {
                hpos[x] = hpos[x - 1];
                hfi[x] = hfi[x - 1];
                --x;
            }
            hpos[x] = a.tl[j];
            hfi[x] = j;
        }
    }
    const int rounds = nh > 0 ? (nh + kProdHigh - 1) / kProdHigh : 1;
    __syncthreads();

    const uint64_t t0 = blockIdx.x, stride = gridDim.x;
#pragma unroll
    for (int s = 0; s < kProdS - 1; ++s) {
        const uint64_t t = t0 + s * stride;
        if (t < a.t.ntiles) load_tile(a.t, runoff, t, stage + s * tileAmps);
        cp_async_commit();
    }
    int it_stage = 0;
    for (uint64_t t = t0; t < a.t.ntiles; t += stride) {
        const uint64_t tn = t + (kProdS - 1) * stride;
        int ld_stage = it_stage + (kProdS - 1);
        if (ld_stage >= kProdS) ld_stage -= kProdS;
        if (tn < a.t.ntiles) load_tile(a.t, runoff, tn, stage + ld_stage * tileAmps);
        cp_async_commit();
        cp_async_wait<kProdS - 1>();
        __syncthreads();
        float2* st = stage + it_stage * tileAmps;
        const uint64_t base = tile_base(a.t, t);
        for (int r = 0; r < rounds; ++r) {
            const int h0 = r * kProdHigh, hb = min(kProdHigh, nh - h0);
            const int nlr = r == 0 ? nl : 0;
            const bool last = r == rounds - 1;
            if (hb >= 3)
                prod_round<3>(a, st, F, hpos + h0, hfi + h0, nlr, lpos, lfi, last, runoff, base);
            else if (hb == 2)
                prod_round<2>(a, st, F, hpos + h0, hfi + h0, nlr, lpos, lfi, last, runoff, base);
            else if (hb == 1)
                prod_round<1>(a, st, F, hpos + h0, hfi + h0, nlr, lpos, lfi, last, runoff, base);
            else
                prod_round<0>(a, st, F, hpos + h0, hfi + h0, nlr, lpos, lfi, last, runoff, base);
            __syncthreads();
        }
        if (++it_stage == kProdS) it_stage = 0;
    }
    cp_async_wait<0>();
}

// ---------------------------------------------------------------------------
// Permute
// ---------------------------------------------------------------------------
struct PermArgs {
    TileArgs t;
    int npairs;
    int la[6], lb[6];   // tile-local positions of each pair
};

template <int S>
__global__ void __launch_bounds__(kThreads) k_permute(PermArgs a) {
    extern __shared__ __align__(16) unsigned char smem_raw[];
    const int tileAmps = 1 << a.t.T;
    float2* stage = reinterpret_cast<float2*>(smem_raw);
    uint64_t* runoff = reinterpret_cast<uint64_t*>(stage + S * tileAmps);
    build_runoff(a.t, runoff);
    __syncthreads();
    const uint64_t stride = gridDim.x;
#pragma unroll
    for (int s = 0; s < S - 1; ++s) {
        uint64_t t = blockIdx.x + s * stride;
        if (t < a.t.ntiles) load_tile(a.t, runoff, t, stage + s * tileAmps);
        cp_async_commit();
    }
    int it_stage = 0;
    const uint32_t chunks = static_cast<uint32_t>(tileAmps) >> 1;
    for (uint64_t t = blockIdx.x; t < a.t.ntiles; t += stride) {
        uint64_t tn = t + (S - 1) * stride;
        int ld_stage = it_stage + (S - 1);
        if (ld_stage >= S) ld_stage -= S;
        if (tn < a.t.ntiles) load_tile(a.t, runoff, tn, stage + ld_stage * tileAmps);
        cp_async_commit();
        cp_async_wait<S - 1>();
        __syncthreads();
        const float2* st = stage + it_stage * tileAmps;
        const uint64_t base = tile_base(a.t, t);
        for (uint32_t q = threadIdx.x; q < chunks; q += blockDim.x) {
            uint32_t d0 = q << 1, d1 = d0 | 1u;
            uint32_t s0 = d0, s1 = d1;
#pragma unroll
            for (int i = 0; i < 6; ++i) {
                if (i >= a.npairs) break;
                uint32_t x0 = ((s0 >> a.la[i]) ^ (s0 >> a.lb[i])) & 1u;
                s0 ^= (x0 << a.la[i]) | (x0 << a.lb[i]);
                uint32_t x1 = ((s1 >> a.la[i]) ^ (s1 >> a.lb[i])) & 1u;
                s1 ^= (x1 << a.la[i]) | (x1 << a.lb[i]);
            }
            float2 v0 = st[s0], v1 = st[s1];
            const uint64_t gd = tile_global(a.t, runoff, base, d0);
            if (dbg::in_bounds(gd, 2, a.t.ntiles << a.t.T, 6))
                __stcs(reinterpret_cast<float4*>(a.t.psi + gd), make_float4(v0.x, v0.y, v1.x, v1.y));
        }
        __syncthreads();
        if (++it_stage == S) it_stage = 0;
    }
    cp_async_wait<0>();
}

__global__ void k_set_one(float2* psi) { psi[0] = make_float2(1.f, 0.f); }

// ---------------------------------------------------------------------------
// Batched trajectories: one persistent launch over many small states
// ---------------------------------------------------------------------------
constexpr int kBatchT = 11;
constexpr int kBatchS = 3;
// A trajectory's blocks run one after another, so the batch ends when its
// deepest trajectory does: each trajectory is run by a cluster of CTAs that
// split every pass's tiles (rank r takes tiles r, r + C, ...) and meet at a
// cluster barrier between blocks.
constexpr int kBatchCluster = 4;

namespace cg = cooperative_groups;

__global__ void __cluster_dims__(kBatchCluster, 1, 1) __launch_bounds__(kThreads, 4) k_batch_evolve(BatchArgs a) {
    extern __shared__ __align__(16) unsigned char smem_raw[];
    float2* stage = reinterpret_cast<float2*>(smem_raw);
    float2* Ms = stage + (kBatchS << kBatchT);
    uint64_t* runoff = reinterpret_cast<uint64_t*>(Ms + 256);
    int* loff = reinterpret_cast<int*>(runoff + 64);
    int* sloff = loff + 64;
    uint8_t* htab = reinterpret_cast<uint8_t*>(sloff + 64);
    // Rank 0 of the cluster pops the queue and makes the watchdog's decision;
    // the others read them from its shared memory after a cluster barrier, so
    // every CTA of a cluster takes the same path and meets the same barriers
    // (s_stop alternates by block so a value is never rewritten before all
    // have read it; s_slot is rewritten only after the trajectory's barriers).
    __shared__ int s_slot;
    __shared__ int s_stop[2];
    cg::cluster_group cluster = cg::this_cluster();
    const unsigned crank = cluster.block_rank();
    const long long t_start = clock64();
    for (;;) {
        if (crank == 0 && threadIdx.x == 0) s_slot = static_cast<int>(atomicAdd(a.queue, 1u));
        cluster.sync();
        const int slot = *cluster.map_shared_rank(&s_slot, 0);
        if (slot >= a.n_traj) {
            cluster.sync();   // no CTA leaves while another may still read its shared memory
            break;
        }
        const int traj = a.order[slot];
        float2* psi = a.states + (static_cast<uint64_t>(traj) << a.n);
        // |0...0>, a share per CTA
        float4* p4 = reinterpret_cast<float4*>(psi);
        const uint64_t npairs = (1ull << a.n) >> 1;
        for (uint64_t i = crank * blockDim.x + threadIdx.x; i < npairs; i += kBatchCluster * blockDim.x)
            p4[i] = make_float4(i == 0 ? 1.f : 0.f, 0.f, 0.f, 0.f);
        __threadfence();
        cluster.sync();
        for (uint32_t b = a.bstart[traj]; b < a.bstart[traj + 1]; ++b) {
            const BatchBlock d = a.blocks[b];
            ApplyArgs aa{};
            aa.t.psi = psi;
            aa.t.T = d.T;
            aa.t.m = d.m;
            aa.t.nx = d.nx;
            aa.t.ntiles = 1ull << (a.n - d.T);
#pragma unroll
            for (int e = 0; e < 6; ++e) {
                aa.t.xpos[e] = d.xpos[e];
                aa.tl[e] = d.tl[e];
                aa.tls[e] = d.tls[e];
            }
#pragma unroll
            for (int e = 0; e < 16; ++e) aa.fv[e] = d.fv[e];
            const int D = 1 << d.k;
            const float2* gm = reinterpret_cast<const float2*>(a.mats + d.mat_off);
            for (int i = threadIdx.x; i < D * D; i += blockDim.x) Ms[i] = gm[i];
            build_runoff(aa.t, runoff);
            switch (d.k) {
                case 1: build_loff<1>(aa.tl, loff); break;
                case 2: build_loff<2>(aa.tl, loff); break;
                case 3: build_loff<3>(aa.tl, loff); break;
                default: build_loff<4>(aa.tl, loff); break;
            }
            if (d.form) build_htab(aa, htab);
            __syncthreads();
            if (d.form) {
                for (int c = threadIdx.x; c < D; c += blockDim.x)
                    sloff[c] = loff[c] ^ static_cast<int>(stage_xor(htab, loff[c]));
                __syncthreads();
            }
            // the stage forms of the single-state kernel (k = 4 takes two items
            // per group here, so no in-place write-back)
#define QSA_BATCH_FORMS(K, R)                                                                                     \
    if (d.form == 2)                                                                                              \
        apply_tiles<K, R, kBatchS, true, true, kBatchT>(aa, stage, Ms, runoff, loff, crank, kBatchCluster, htab,  \
                                                        sloff);                                                   \
    else if (d.form == 1)                                                                                         \
        apply_tiles<K, R, kBatchS, true, false, kBatchT>(aa, stage, Ms, runoff, loff, crank, kBatchCluster, htab, \
                                                         sloff);                                                  \
    else                                                                                                          \
        apply_tiles<K, R, kBatchS>(aa, stage, Ms, runoff, loff, crank, kBatchCluster);
            switch (d.k) {
                case 1: QSA_BATCH_FORMS(1, 2) break;
                case 2: QSA_BATCH_FORMS(2, 4) break;
                case 3: QSA_BATCH_FORMS(3, 8) break;
                default:
                    if (d.form)
                        apply_tiles<4, 8, kBatchS, true, false, kBatchT>(aa, stage, Ms, runoff, loff, crank,
                                                                         kBatchCluster, htab, sloff);
                    else
                        apply_tiles<4, 8, kBatchS>(aa, stage, Ms, runoff, loff, crank, kBatchCluster);
                    break;
            }
#undef QSA_BATCH_FORMS
            // the pass's tiles are written before any CTA of the cluster reads
            // them in the next block; the watchdog's decision travels with it
            if (crank == 0 && threadIdx.x == 0)
                s_stop[b & 1] = (a.budget != 0 && static_cast<unsigned long long>(clock64() - t_start) > a.budget) ? 1 : 0;
            __threadfence();
            cluster.sync();
            if (*cluster.map_shared_rank(&s_stop[b & 1], 0)) {
                if (crank == 0 && threadIdx.x == 0) atomicExch(a.err, 7);
                cluster.sync();
                return;
            }
        }
    }
}

}  // namespace

QSA_BOUNDS_READER(bounds_word_apply)

int num_sms() {
    static std::mutex mu;
    static std::map<int, int> cached;
    int dev = 0;
    cudaGetDevice(&dev);
    std::lock_guard<std::mutex> lk(mu);
    auto it = cached.find(dev);
    if (it != cached.end()) return it->second;
    int v = 0;
    cudaDeviceGetAttribute(&v, cudaDevAttrMultiProcessorCount, dev);
    if (v <= 0) v = 1;
    cached[dev] = v;
    return v;
}

cudaError_t set_smem_attr(const void* kernel, int bytes) {
    static std::mutex mu;
    static std::map<std::pair<int, const void*>, int> done;
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return e;
    std::lock_guard<std::mutex> lk(mu);
    const auto key = std::make_pair(dev, kernel);
    auto it = done.find(key);
    if (it != done.end() && it->second >= bytes) return cudaSuccess;
    e = cudaFuncSetAttribute(kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, bytes);
    if (e != cudaSuccess) return e;
    done[key] = bytes;
    return cudaSuccess;
}

bool make_geom(int n, const int* special, int ns, int T_want, TileGeom* g) {
    g->n = n;
    g->T = std::min(T_want, n);
    int m = g->T;
    for (;;) {
        int cnt = 0;
        for (int i = 0; i < ns; ++i)
            if (special[i] >= m) ++cnt;
        if (m + cnt <= g->T) break;
        --m;
    }
    if (m < 1) return false;
    g->m = m;
    int nx = 0;
    int tmp[16];
    for (int i = 0; i < ns; ++i)
        if (special[i] >= m) {
            if (nx >= 6) return false;
            tmp[nx++] = special[i];
        }
    std::sort(tmp, tmp + nx);
    g->nx = nx;
    for (int e = 0; e < 6; ++e) g->xpos[e] = e < nx ? tmp[e] : 0;
    g->ntiles = 1ull << (n - g->T);
    return true;
}

bool make_batch_block(int n, const int* phys, int k, uint32_t mat_off, BatchBlock* b) {
    if (k < 1 || k > 4) return false;
    TileGeom g;
    if (!make_geom(n, phys, k, kBatchT, &g)) return false;
    *b = BatchBlock{};
    b->k = k;
    b->T = g.T;
    b->m = g.m;
    b->nx = g.nx;
    for (int e = 0; e < 6; ++e) b->xpos[e] = g.xpos[e];
    local_targets(g, phys, k, b->tl, b->tls);
    b->mat_off = mat_off;
    b->form = g.T == kBatchT ? apply_form(g.T, b->tls, k) : 0;
    if (k == 4 && b->form == 2) b->form = 1;   // two items per group: gathers only
    if (b->form) stage_slots(g.T, b->tls, k, b->fv);
    return true;
}

cudaError_t launch_batch_evolve(const BatchArgs& a, cudaStream_t st, uint64_t* launches) {
    const size_t smem = sizeof(float2) * (static_cast<size_t>(kBatchS) << kBatchT) + sizeof(float2) * 256 +
                        sizeof(uint64_t) * 64 + 2 * sizeof(int) * 64 + 256;
    {
        cudaError_t e = set_smem_attr(reinterpret_cast<const void*>(k_batch_evolve), static_cast<int>(smem));
        if (e != cudaSuccess) return e;
    }
    int occ = 0;
    cudaError_t e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, k_batch_evolve, kThreads, smem);
    if (e != cudaSuccess) return e;
    if (occ < 1) occ = 1;
    // one cluster per trajectory in flight (clusters that find the queue
    // empty leave at once)
    unsigned clusters = static_cast<unsigned>(num_sms() * occ / kBatchCluster);
    if (clusters > static_cast<unsigned>(a.n_traj)) clusters = static_cast<unsigned>(a.n_traj);
    if (clusters == 0) clusters = 1;
    k_batch_evolve<<<clusters * kBatchCluster, kThreads, smem, st>>>(a);
    ++*launches;
    return cudaGetLastError();
}

__global__ void k_fill_one(float4* psi2, uint64_t npairs) {
    for (uint64_t i = blockIdx.x * static_cast<uint64_t>(blockDim.x) + threadIdx.x; i < npairs;
         i += static_cast<uint64_t>(gridDim.x) * blockDim.x)
        psi2[i] = make_float4(1.f, 0.f, 1.f, 0.f);
}

cudaError_t launch_fill_one(float2* psi, int n, cudaStream_t st, uint64_t* launches) {
    if (n < 1) return cudaErrorInvalidValue;
    const uint64_t npairs = (1ull << n) >> 1;
    uint64_t blocks = (npairs + 255) / 256;
    const uint64_t cap = static_cast<uint64_t>(num_sms()) * 16;
    if (blocks > cap) blocks = cap;
    k_fill_one<<<static_cast<unsigned>(blocks), 256, 0, st>>>(reinterpret_cast<float4*>(psi), npairs);
    ++*launches;
    return cudaGetLastError();
}

cudaError_t launch_init_zero(float2* psi, int n, cudaStream_t st, uint64_t* launches) {
    cudaError_t e = cudaMemsetAsync(psi, 0, sizeof(float2) << n, st);
    if (e != cudaSuccess) return e;
    k_set_one<<<1, 1, 0, st>>>(psi);
    ++*launches;
    return cudaGetLastError();
}

cudaError_t launch_apply_fp32(float2* psi, int n, const int* phys, int k, const float* d_mat, cudaStream_t st,
                              uint64_t* launches) {
    switch (k) {
        case 1: return launch_apply_k<1>(psi, n, phys, d_mat, st, launches);
        case 2: return launch_apply_k<2>(psi, n, phys, d_mat, st, launches);
        case 3: return launch_apply_k<3>(psi, n, phys, d_mat, st, launches);
        case 4: return launch_apply_k<4>(psi, n, phys, d_mat, st, launches);
        case 5: return launch_apply_k<5>(psi, n, phys, d_mat, st, launches);
        case 6: return launch_apply_k<6>(psi, n, phys, d_mat, st, launches);
        default: return cudaErrorInvalidValue;
    }
}

cudaError_t launch_apply_prod(float2* psi, int n, const int* phys, int k, const float* d_fac, cudaStream_t st,
                              uint64_t* launches) {
    if (n < 5) {
        // the product round maps warp lanes to 5 tile bits: tiny states apply
        // each factor as its own one-qubit update
        for (int j = 0; j < k; ++j) {
            cudaError_t e = launch_apply_k<1>(psi, n, phys + j, d_fac + 8 * j, st, launches);
            if (e != cudaSuccess) return e;
        }
        return cudaSuccess;
    }
    // a tile holds at most 6 high target bits: larger sets go in several passes
    int j0 = 0;
    while (j0 < k) {
        int j1 = k;
        TileGeom g;
        while (!make_geom(n, phys + j0, j1 - j0, kProdT, &g)) {
            if (j1 - j0 == 1) return cudaErrorInvalidValue;
            --j1;
        }
        ProdArgs a{};
        a.t.psi = psi;
        a.t.ntiles = g.ntiles;
        a.t.T = g.T;
        a.t.m = g.m;
        a.t.nx = g.nx;
        for (int e = 0; e < 6; ++e) a.t.xpos[e] = g.xpos[e];
        a.fac = d_fac + 8 * j0;
        a.k = j1 - j0;
        int tls[QSA_MAX_PROD];
        local_targets(g, phys + j0, a.k, a.tl, tls);
        const size_t smem = sizeof(float2) * (static_cast<size_t>(kProdS) << g.T) + sizeof(float2) * 4 * QSA_MAX_PROD +
                            sizeof(uint64_t) * 64;
        {
            const size_t full = sizeof(float2) * (static_cast<size_t>(kProdS) << kProdT) +
                                sizeof(float2) * 4 * QSA_MAX_PROD + sizeof(uint64_t) * 64;
            cudaError_t e = set_smem_attr(reinterpret_cast<const void*>(k_apply_prod), static_cast<int>(full));
            if (e != cudaSuccess) return e;
        }
        int occ = 0;
        cudaError_t e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, k_apply_prod, kThreads, smem);
        if (e != cudaSuccess) return e;
        if (occ < 1) occ = 1;
        uint64_t grid = static_cast<uint64_t>(num_sms()) * occ;
        if (grid > g.ntiles) grid = g.ntiles;
        k_apply_prod<<<static_cast<unsigned>(grid), kThreads, smem, st>>>(a);
        ++*launches;
        e = cudaGetLastError();
        if (e != cudaSuccess) return e;
        j0 = j1;
    }
    return cudaSuccess;
}

cudaError_t launch_permute(float2* psi, int n, const int* pa, const int* pb, int npairs, cudaStream_t st,
                           uint64_t* launches) {
    constexpr int S = 3, T = 11;
    int i0 = 0;
    while (i0 < npairs) {
        // grow the pass while its extra tile bits fit
        int i1 = i0 + 1;
        TileGeom g;
        int spec[12];
        for (;;) {
            int ns = 0;
            for (int i = i0; i < i1; ++i) {
                spec[ns++] = pa[i];
                spec[ns++] = pb[i];
            }
            if (!make_geom(n, spec, ns, T, &g)) {
                if (i1 == i0 + 1) return cudaErrorInvalidValue;
                --i1;
                ns = 0;
                for (int i = i0; i < i1; ++i) {
                    spec[ns++] = pa[i];
                    spec[ns++] = pb[i];
                }
                make_geom(n, spec, ns, T, &g);
                break;
            }
            if (i1 == npairs || i1 - i0 == 6) break;
            ++i1;
        }
        PermArgs a{};
        a.t.psi = psi;
        a.t.ntiles = g.ntiles;
        a.t.T = g.T;
        a.t.m = g.m;
        a.t.nx = g.nx;
        for (int e = 0; e < 6; ++e) a.t.xpos[e] = g.xpos[e];
        a.npairs = i1 - i0;
        auto local = [&](int p) {
            if (p < g.m) return p;
            int e = 0;
            while (g.xpos[e] != p) ++e;
            return g.m + e;
        };
        for (int i = i0; i < i1; ++i) {
            a.la[i - i0] = local(pa[i]);
            a.lb[i - i0] = local(pb[i]);
        }
        const size_t smem = sizeof(float2) * (static_cast<size_t>(S) << g.T) + sizeof(uint64_t) * 64;
        auto kern = k_permute<S>;
        {
            const size_t full = sizeof(float2) * (static_cast<size_t>(S) << T) + sizeof(uint64_t) * 64;
            cudaError_t e = set_smem_attr(reinterpret_cast<const void*>(kern), static_cast<int>(full));
            if (e != cudaSuccess) return e;
        }
        int occ = 0;
        cudaError_t e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, kern, kThreads, smem);
        if (e != cudaSuccess) return e;
        if (occ < 1) occ = 1;
        uint64_t grid = static_cast<uint64_t>(num_sms()) * occ;
        if (grid > g.ntiles) grid = g.ntiles;
        kern<<<static_cast<unsigned>(grid), kThreads, smem, st>>>(a);
        ++*launches;
        e = cudaGetLastError();
        if (e != cudaSuccess) return e;
        i0 = i1;
    }
    return cudaSuccess;
}

}  // namespace qsa
