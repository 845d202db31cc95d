// Layer blocks (a structured fused block, §IV-D "structured blocks may use
// cheaper lowerings"): one- and two-qubit diagonal gates on any qubits, then a
// layer of one-qubit factors, in one pass over the state.
//
// A tile is 2^12 amplitudes: the m lowest positions (m >= 3, one run of 2^m
// contiguous amplitudes) and nx = 12 - m higher positions holding the
// factors' remaining qubits.  Relative to a tile, every diagonal gate falls
// into one of three classes, precomputed on the host:
//   all-in  (its qubits are tile bits): multiplied into one 2^12-entry table
//           over the tile-local index, applied elementwise;
//   cross   (one qubit in the tile, one outside): with the outside bit fixed
//           by the tile, a one-qubit phase on its tile bit, folded into that
//           bit's factor (F' = F diag(d0, d1)), or multiplied in where the bit
//           has no factor;
//   out     (no qubit in the tile): a scalar per tile, multiplied in.
// Unitary factors run in rotation mode: each factor is split on the host as
// F = diag(p) R diag(q) with R = [[c, -s], [s, c]] real, and R in turn as
// kappa * M with one coefficient of each row of M equal to 1 (tangent form
// M = [[1, -t], [t, 1]], t = s / c, when c >= s; else the cotangent form
// M = [[u, -1], [1, u]], u = c / s, whose first row is negated into p), so a
// factor costs one packed multiply-add per amplitude.  The cotangent form runs
// as the tangent form with t = -u, which yields row 1 and -row 0 in exchanged
// places; the pass leaves them exchanged and takes every later table entry
// and store offset at the exchanged index, so no round branches per factor.
// kappa and the q phases join the per-bit phases (with the cross phases,
// applied in round 0 before any rotation) and the p phases a 16-entry table
// of its round (applied after the round's rotations).  Other factors run in
// general mode (complex 2x2 butterflies, cross phases folded into them).
// Per tile: 16-byte cp.async copies into a 2-stage ring (XOR-swizzled 16-byte
// chunks), with the tile's per-tile phase record (rotation mode: written by
// k_layer_records before the pass; general mode: formed by warp 0); then
// three register rounds over tile bits 0-3, 4-7 and 8-11 (each thread holds
// the 16 amplitudes that differ in the round's bits); the last active round
// stores to HBM.  Whether the pass has a diagonal table, per-tile phases,
// exit phases or a generated input is a template argument, so the rounds are
// straight-line code.
#include <cuda_runtime.h>

#include <cstddef>
#include <cstdint>

#include "qsa_device.cuh"
#include "qsa_bounds.cuh"
#include "qsa_internal.h"

namespace qsa {

namespace {

using namespace dev;

constexpr int kLT = 12;                 // tile bits
constexpr int kLAmps = 1 << kLT;        // amplitudes per tile
constexpr int kLThreads = 256;
constexpr int kLStages = 2;

// Per-tile phases of rotation mode, written by k_layer_records before the
// pass: the product of the pmask bits' phases (d0, d1) split over tile bits
// 0..3 (times the scalar of the out gates), 4..7 and 8..11, 16 entries each.
struct LayerRec {
    float2 pl[16];            // bits 0..3 of round 0's local index, times the scalar
    float2 pa[16], pb[16];    // products over tile bits 4..7 and 8..11 (fixed per thread in round 0)
};
static_assert(sizeof(LayerRec) == 48 * sizeof(float2) && offsetof(LayerRec, pa) == 16 * sizeof(float2),
              "the records kernel writes pl and pa as one 32-entry array");

struct LayerArgs {
    float2* psi;
    uint64_t ntiles;
    int m, nx;
    int xpos[kLT];            // positions of tile bits m..11, ascending
    uint32_t fmask;           // tile bits with a factor
    uint32_t pmask;           // tile bits with a per-tile phase applied as a multiply
    uint32_t rpmask;          // rotation mode: rounds with exit phases
    uint32_t rswap;           // rotation mode: tile bits left exchanged (place j of the tile holds
                              // the amplitude of tile-local index j ^ rswap after their rotations)
    int generate;             // write-only: every amplitude enters as 1 (nothing is read)
    int ncross, nout;
    int cstart[kLT + 1];      // cross gates of tile bit b: [cstart[b], cstart[b + 1])
    const float2* fac;        // general mode: kLT x 4 complex (2x2 row-major); rotation mode:
                              // (t or u, 0) of each factor's rotation
    const LayerGate* cross;   // a = tile bit, b = outside position, d[2 * o + v]
    const LayerGate* outg;    // a, b = positions (b < 0: one qubit), d[v_a + 2 v_b]
    const float2* din;        // table of the gates with every qubit in the tile: 2^12 entries in
                              // tile-local order (copied to shared memory), or nullptr
    const float2* qph;        // rotation mode: each tile bit's entry phases q (kLT x 2)
    const float2* sph;        // rotation mode without per-tile phases: per round, the product of
                              // its bits' entry phases q (3 x 16, the LayerRec layout), formed on
                              // the host
    const LayerRec* rec;      // rotation mode with per-tile phases: one record per tile, or nullptr
    // Read with compile-time indices, so they enter the instructions from the parameter bank
    // (no shared-memory loads):
    uint64_t goff[56];        // offsets of a round's local bits (goff[16 R + i] for tile-local
                              // (i ^ exchanged round bits) << 4R) and of the load loop's chunk
                              // strides (goff[48 + k] for tile-local 512 k)
    float rot[kLT];           // rotation mode: each tile bit's coefficient (t or u; 0 without a factor)
    float rpe[96];            // rotation mode: per round, the exit phases of its 16 places (interleaved)
    // Tile bases: base(t) deposits t's bits into the positions outside the tile (omask, ascending);
    // base(t + s) = ((base(t) | ~omask) + dstride) & omask with dstride = base(s) (the carries run
    // through the tile's positions), s the launch's grid size.
    uint64_t omask, dstride;
};

struct LayerShared {
    float2 tf[kLT][4];        // general mode: this tile's factors (cross phases folded in)
    LayerRec ph;              // per-tile phases (general mode and static rotation mode)
};
// round 0 reads the phase tables two entries at a time (16-byte loads): every
// array of the shared layout in k_apply_layer starts on a 16-byte boundary
static_assert(sizeof(LayerShared) % 16 == 0 && offsetof(LayerShared, ph) % 16 == 0 && sizeof(LayerRec) % 16 == 0,
              "16-byte aligned shared tables");

// Slot of tile-local amplitude j: 16-byte chunk c = j / 2 is stored at
// c ^ ((c >> 3) & 7), which spreads each round's warp accesses over all banks.
// The map is linear over XOR, so for j and x with disjoint bits
// lsw(j | x) = lsw(j) ^ lsw(x): a thread forms lsw of its own bits once and
// combines it with compile-time constants.
__host__ __device__ constexpr int lsw(int j) { return (((j >> 1) ^ ((j >> 4) & 7)) << 1) | (j & 1); }

__device__ __forceinline__ float2 cmulf(float2 a, float2 b) {
    return make_float2(fmaf(a.x, b.x, -a.y * b.y), fmaf(a.x, b.y, a.y * b.x));
}

__device__ __forceinline__ uint64_t layer_base(const LayerArgs& a, uint64_t t) {
    uint64_t b = t << a.m;
#pragma unroll
    for (int e = 0; e < kLT; ++e)
        if (e < a.nx) b = insert_zero(b, a.xpos[e]);
    return b;
}

// Global offset of tile-local index j within the tile (OR-linear over disjoint bits).
__device__ __forceinline__ uint64_t layer_global(const LayerArgs& a, const uint64_t* runoff, uint64_t base, int j) {
    return base | static_cast<uint64_t>(j & ((1 << a.m) - 1)) | runoff[j >> a.m];
}

// General factor: v[i], v[i | 2^LB] <- F (v[i], v[i | 2^LB]) for the 8 pairs.
template <int LB>
__device__ __forceinline__ void butterfly(float2 (&v)[16], const float2* F) {
    const float2 f00 = F[0], f01 = F[1], f10 = F[2], f11 = F[3];
#pragma unroll
    for (int i = 0; i < 16; ++i) {
        if ((i >> LB) & 1) continue;
        const float2 x0 = v[i], x1 = v[i | (1 << LB)];
        v[i] = make_float2(f00.x * x0.x - f00.y * x0.y + f01.x * x1.x - f01.y * x1.y,
                           f00.x * x0.y + f00.y * x0.x + f01.x * x1.y + f01.y * x1.x);
        v[i | (1 << LB)] = make_float2(f10.x * x0.x - f10.y * x0.y + f11.x * x1.x - f11.y * x1.y,
                                       f10.x * x0.y + f10.y * x0.x + f11.x * x1.y + f11.y * x1.x);
    }
}

// Scaled real rotation in the tangent form on local bit LB, both components
// of an amplitude in one packed pair, one fma.rn.f32x2 per output:
// (x0, x1) <- (x0 - t x1, x1 + t x0); t = 0 is the identity.
template <int LB>
__device__ __forceinline__ void rotation(float2 (&v)[16], float coef) {
    const uint64_t t2 = pack2(coef, coef), nt2 = pack2(-coef, -coef);
#pragma unroll
    for (int i = 0; i < 16; ++i) {
        if ((i >> LB) & 1) continue;
        const uint64_t x0 = pack2(v[i].x, v[i].y), x1 = pack2(v[i | (1 << LB)].x, v[i | (1 << LB)].y);
        v[i] = unpack2(fma2(nt2, x1, x0));
        v[i | (1 << LB)] = unpack2(fma2(t2, x0, x1));
    }
}

// This thread's part of the global offsets of round R's stores: tile-local
// jb at the exchanged index, jb its amplitudes' common bits outside the round.
template <int R>
__device__ __forceinline__ uint64_t store_offset(const LayerArgs& a, const uint64_t* runoff) {
    const int t = threadIdx.x;
    const int jb = (t & ((1 << (4 * R)) - 1)) | ((t >> (4 * R)) << (4 * R + 4));
    return layer_global(a, runoff, 0, jb ^ static_cast<int>(a.rswap & ~(15u << (4 * R)) & 0xfffu));
}

// Whether a pass has a diagonal table (DIN), per-tile phases (PH) and exit
// phases (RP), and whether it generates its input (GEN): known at compile
// time (1 present, 0 absent) or read at run time (2); LAST: the round stores
// to HBM (soff: this thread's store_offset for the round).
// One round over tile bits 4R..4R+3: read the stage; (R = 0) multiply by the
// entry table and the per-tile phases; apply the round's factors; (last
// round, rotation mode) multiply by the exit table; write back to the stage
// or (last round) to HBM.
template <bool ROT, int R, int DIN, int PH, int RP, int GEN, bool LAST>
__device__ __forceinline__ void layer_round(const LayerArgs& a, float2* stage, const float2* din_s,
                                            const LayerShared& sh, const LayerRec& pr, uint64_t soff,
                                            uint64_t base, bool phase) {
    const int t = threadIdx.x;
    const int jb = (t & ((1 << (4 * R)) - 1)) | ((t >> (4 * R)) << (4 * R + 4));
    const int sb = lsw(jb);   // slot of (jb | x) = sb ^ lsw(x)
    float2 v[16];
    if constexpr (R == 0) {
        if (GEN == 1 || (GEN == 2 && a.generate)) {
#pragma unroll
            for (int i = 0; i < 16; ++i) v[i] = make_float2(1.f, 0.f);
        } else {
#pragma unroll
            for (int i = 0; i < 16; i += 2) {
                const float4 p = *reinterpret_cast<const float4*>(stage + (sb ^ lsw(i)));
                v[i] = make_float2(p.x, p.y);
                v[i + 1] = make_float2(p.z, p.w);
            }
        }
        if (DIN == 1 || (DIN == 2 && din_s)) {
#pragma unroll
            for (int i = 0; i < 16; i += 2) {
                const float4 d = *reinterpret_cast<const float4*>(din_s + (sb ^ lsw(i)));
                v[i] = cmulf(v[i], make_float2(d.x, d.y));
                v[i + 1] = cmulf(v[i + 1], make_float2(d.z, d.w));
            }
        }
        if (PH == 1 || (PH == 2 && phase)) {
            // phases of tile bits 4..11 (fixed for this thread) times those of the 16 local amplitudes
            const float2 ph = cmulf(pr.pa[(jb >> 4) & 15], pr.pb[(jb >> 8) & 15]);
#pragma unroll
            for (int i = 0; i < 16; i += 2) {
                const float4 q = reinterpret_cast<const float4*>(pr.pl)[i >> 1];   // two entries per load
                v[i] = cmulf(v[i], cmulf(ph, make_float2(q.x, q.y)));
                v[i + 1] = cmulf(v[i + 1], cmulf(ph, make_float2(q.z, q.w)));
            }
        }
    } else {
#pragma unroll
        for (int i = 0; i < 16; ++i) v[i] = stage[sb ^ lsw(i << (4 * R))];
    }
    const uint32_t act = (a.fmask >> (4 * R)) & 15u;
    if constexpr (ROT) {
        // rounds 1 and 2 (and a full round 0) run all four without branches
        // (t = 0 on bits without a factor); round 0 often carries one factor
        // only, on tile bit 3 (the lowest position above the run), and
        // otherwise branches per bit
        if (R > 0 || act == 15u) {
            rotation<0>(v, a.rot[4 * R + 0]);
            rotation<1>(v, a.rot[4 * R + 1]);
            rotation<2>(v, a.rot[4 * R + 2]);
            rotation<3>(v, a.rot[4 * R + 3]);
        } else if (act == 8u) {
            rotation<3>(v, a.rot[3]);
        } else {
            if (act & 1u) rotation<0>(v, a.rot[0]);
            if (act & 2u) rotation<1>(v, a.rot[1]);
            if (act & 4u) rotation<2>(v, a.rot[2]);
            if (act & 8u) rotation<3>(v, a.rot[3]);
        }
        if (RP != 0 && act && ((a.rpmask >> R) & 1u)) {
            // exit phases of the round's factor bits (they follow only their own rotations)
#pragma unroll
            for (int i = 0; i < 16; ++i) v[i] = cmulf(v[i], make_float2(a.rpe[32 * R + 2 * i], a.rpe[32 * R + 2 * i + 1]));
        }
    } else {
        if (act & 1u) butterfly<0>(v, sh.tf[4 * R + 0]);
        if (act & 2u) butterfly<1>(v, sh.tf[4 * R + 1]);
        if (act & 4u) butterfly<2>(v, sh.tf[4 * R + 2]);
        if (act & 8u) butterfly<3>(v, sh.tf[4 * R + 3]);
    }
    if constexpr (LAST) {
        // global offset of (jb | x) = offset(jb) | offset(x) at the exchanged index:
        // soff = offset(jb ^ exchanged bits outside the round), formed once per thread
        // (store_offset); goff[16 R + i] holds offset((i ^ exchanged round bits) << 4R)
        const uint64_t gb = base | soff;
        // (round 0 never stores: as the last round it goes through the stage)
        static_assert(R > 0, "round 0 writes to the stage");
#pragma unroll
        for (int i = 0; i < 16; ++i)
            if (dbg::in_bounds(gb | a.goff[16 * R + i], 1, a.ntiles << 12, 11)) __stcs(a.psi + (gb | a.goff[16 * R + i]), v[i]);
    } else {
        if constexpr (R == 0) {
#pragma unroll
            for (int i = 0; i < 16; i += 2)
                *reinterpret_cast<float4*>(stage + (sb ^ lsw(i))) = make_float4(v[i].x, v[i].y, v[i + 1].x, v[i + 1].y);
        } else {
#pragma unroll
            for (int i = 0; i < 16; ++i) stage[sb ^ lsw(i << (4 * R))] = v[i];
        }
    }
}

// Lane l < 16 of a warp forms entry l of the three phase tables from lane b's
// phases (d0, d1) of tile bit b (all lanes take part in the shuffles).
__device__ __forceinline__ void phase_tables(uint32_t pmask, float2 d0, float2 d1, float2 sc, LayerRec* out) {
    const int lane = threadIdx.x & 31;
    float2 pl = sc, pa = make_float2(1.f, 0.f), pb = make_float2(1.f, 0.f);
#pragma unroll
    for (int b = 0; b < kLT; ++b) {
        float2 e0, e1;
        e0.x = __shfl_sync(0xffffffffu, d0.x, b);
        e0.y = __shfl_sync(0xffffffffu, d0.y, b);
        e1.x = __shfl_sync(0xffffffffu, d1.x, b);
        e1.y = __shfl_sync(0xffffffffu, d1.y, b);
        if (!((pmask >> b) & 1u)) continue;
        const float2 e = ((lane >> (b & 3)) & 1) ? e1 : e0;
        if (b < 4)
            pl = cmulf(pl, e);
        else if (b < 8)
            pa = cmulf(pa, e);
        else
            pb = cmulf(pb, e);
    }
    if (lane < 16) {
        out->pl[lane] = pl;
        out->pa[lane] = pa;
        out->pb[lane] = pb;
    }
}

// The tile's factors and phases (warp 0): the scalar of the out gates (lanes
// over gates, product across lanes); each tile bit's cross phases (lane b),
// folded into the bit's factor (general mode, factor bits) or kept as a
// phase; then the phases of round 0's 16 local amplitudes times the scalar.
template <bool ROT>
__device__ __forceinline__ void tile_phases(const LayerArgs& a, uint64_t base, LayerShared& sh) {
    const int lane = threadIdx.x & 31;
    float2 sc = make_float2(1.f, 0.f);
    for (int g = lane; g < a.nout; g += 32) {
        const LayerGate& G = a.outg[g];
        int v = static_cast<int>((base >> G.a) & 1ull);
        if (G.b >= 0) v |= static_cast<int>((base >> G.b) & 1ull) << 1;
        sc = cmulf(sc, G.d[v]);
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
        float2 other;
        other.x = __shfl_xor_sync(0xffffffffu, sc.x, o);
        other.y = __shfl_xor_sync(0xffffffffu, sc.y, o);
        sc = cmulf(sc, other);
    }
    const bool fold = !ROT && ((a.fmask >> lane) & 1u);
    float2 d0 = make_float2(1.f, 0.f), d1 = make_float2(1.f, 0.f);
    if (lane < kLT && (fold || ((a.pmask >> lane) & 1u))) {
        for (int g = a.cstart[lane]; g < a.cstart[lane + 1]; ++g) {
            const LayerGate& G = a.cross[g];
            const int o = static_cast<int>((base >> G.b) & 1ull);
            d0 = cmulf(d0, G.d[2 * o]);
            d1 = cmulf(d1, G.d[2 * o + 1]);
        }
        if (fold) {
            const float2* F = a.fac + 4 * lane;
            sh.tf[lane][0] = cmulf(F[0], d0);
            sh.tf[lane][1] = cmulf(F[1], d1);
            sh.tf[lane][2] = cmulf(F[2], d0);
            sh.tf[lane][3] = cmulf(F[3], d1);
        }
    }
    phase_tables(a.pmask, d0, d1, sc, &sh.ph);
}

// Rotation mode, one warp per 32 consecutive tiles: lane j forms tile t0 + j's
// scalar of the out gates and each pmask bit's cross phases times its
// rotation's entry phases (every tile reads the same gates, so their loads
// are broadcasts and the lanes do not diverge), into shared memory; then,
// tile by tile, lane l forms entry l of the record's pl and pa tables and
// lanes 0..15 entry l of pb, so each record is written by consecutive lanes.
constexpr int kRecThreads = 128;
__global__ void __launch_bounds__(kRecThreads) k_layer_records(LayerArgs a, LayerRec* recs) {
    __shared__ float2 ph[kRecThreads / 32][2 * kLT + 1][32];   // [bit phase (2 b + v) | scalar][tile]
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    const uint64_t warps = static_cast<uint64_t>(gridDim.x) * (blockDim.x >> 5);
    for (uint64_t t0 = (static_cast<uint64_t>(blockIdx.x) * (blockDim.x >> 5) + w) * 32; t0 < a.ntiles;
         t0 += warps * 32) {
        const uint64_t t = t0 + lane;
        if (t < a.ntiles) {
            const uint64_t base = layer_base(a, t);
            float2 sc = make_float2(1.f, 0.f);
            for (int g = 0; g < a.nout; ++g) {
                const LayerGate& G = a.outg[g];
                int v = static_cast<int>((base >> G.a) & 1ull);
                if (G.b >= 0) v |= static_cast<int>((base >> G.b) & 1ull) << 1;
                sc = cmulf(sc, G.d[v]);
            }
            ph[w][2 * kLT][lane] = sc;
#pragma unroll
            for (int b = 0; b < kLT; ++b) {
                float2 d0 = make_float2(1.f, 0.f), d1 = make_float2(1.f, 0.f);
                if ((a.pmask >> b) & 1u) {
                    for (int g = a.cstart[b]; g < a.cstart[b + 1]; ++g) {
                        const LayerGate& G = a.cross[g];
                        const int o = static_cast<int>((base >> G.b) & 1ull);
                        d0 = cmulf(d0, G.d[2 * o]);
                        d1 = cmulf(d1, G.d[2 * o + 1]);
                    }
                    d0 = cmulf(d0, a.qph[2 * b]);
                    d1 = cmulf(d1, a.qph[2 * b + 1]);
                }
                ph[w][2 * b][lane] = d0;
                ph[w][2 * b + 1][lane] = d1;
            }
        }
        __syncwarp();
        const uint64_t left = a.ntiles - t0;
        const int nt = left < 32 ? static_cast<int>(left) : 32;
        const int i = lane & 15, r = lane >> 4;   // lanes 0..15: pl[i], lanes 16..31: pa[i]
        for (int j = 0; j < nt; ++j) {
            float2 x = r == 0 ? ph[w][2 * kLT][j] : make_float2(1.f, 0.f);
            float2 y = make_float2(1.f, 0.f);
#pragma unroll
            for (int lb = 0; lb < 4; ++lb) {
                x = cmulf(x, ph[w][2 * (4 * r + lb) + ((i >> lb) & 1)][j]);
                y = cmulf(y, ph[w][2 * (8 + lb) + ((i >> lb) & 1)][j]);
            }
            LayerRec* out = recs + t0 + j;
            reinterpret_cast<float2*>(out->pl)[lane] = x;   // pl[0..15], then pa[0..15]
            if (lane < 16) out->pb[i] = y;
        }
        __syncwarp();
    }
}

template <bool ROT, int DIN, int PH, int RP, int GEN>
__global__ void __launch_bounds__(kLThreads, 2) k_apply_layer(LayerArgs a) {
    extern __shared__ __align__(16) unsigned char smem_raw[];
    float2* stage = reinterpret_cast<float2*>(smem_raw);                        // kLStages x 4096
    uint64_t* runoff = reinterpret_cast<uint64_t*>(stage + kLStages * kLAmps);  // 512
    LayerShared& sh = *reinterpret_cast<LayerShared*>(runoff + 512);
    LayerRec* recs = reinterpret_cast<LayerRec*>(&sh + 1);                      // kLStages
    float2* din_s = a.din ? reinterpret_cast<float2*>(recs + kLStages) : nullptr;   // 4096, swizzled

    for (int r = threadIdx.x; r < (1 << a.nx); r += blockDim.x) {
        uint64_t off = 0;
        for (int e = 0; e < a.nx; ++e)
            if ((r >> e) & 1) off |= 1ull << a.xpos[e];
        runoff[r] = off;
    }
    const bool dynamic = a.ncross > 0 || a.nout > 0;
    const bool phase = a.pmask != 0 || a.nout > 0;
    if (ROT) {
        if (!dynamic)   // static phases: the rotations' entry phases only, tables from the host
            for (int i = threadIdx.x; i < 48; i += blockDim.x) reinterpret_cast<float2*>(&sh.ph)[i] = a.sph[i];
    } else if (!dynamic) {
        for (int i = threadIdx.x; i < 4 * kLT; i += blockDim.x) sh.tf[i >> 2][i & 3] = a.fac[i];
    }
    if (din_s)
        for (int j = threadIdx.x; j < kLAmps; j += blockDim.x) din_s[lsw(j)] = a.din[j];
    __syncthreads();

    // rounds that do work; the last of them writes to HBM
    int first = -1, last = -1;
    for (int r = 0; r < 3; ++r)
        if (((a.fmask >> (4 * r)) & 15u) || (r == 0 && (a.din || phase || a.generate))) {
            if (first < 0) first = r;
            last = r;
        }

    const uint64_t stride = gridDim.x;
    // rotation mode takes the per-tile phases from the records (fetched with
    // the tile), general mode forms them in warp 0
    const bool use_rec = ROT && a.rec;
    // this thread's chunks are 2 * threadIdx.x + 512 k, k = 0..7
    const uint64_t gld = layer_global(a, runoff, 0, 2 * threadIdx.x);
    // this thread's store offsets for a last round 1 or 2
    const uint64_t soff1 = store_offset<1>(a, runoff), soff2 = store_offset<2>(a, runoff);
    const int sld = lsw(2 * threadIdx.x);
    auto load = [&](uint64_t t, uint64_t tbase, int sidx) {
        const uint64_t base = tbase | gld;
        float2* st = stage + sidx * kLAmps;
        if (GEN == 0 || (GEN == 2 && !a.generate))
#pragma unroll
            for (int k = 0; k < kLAmps / 2 / kLThreads; ++k)
                if (dbg::in_bounds(base | a.goff[48 + k], 2, a.ntiles << 12, 12))
                    cp_async16(st + (sld ^ lsw(512 * k)), a.psi + (base | a.goff[48 + k]));
        if (use_rec && threadIdx.x < static_cast<int>(sizeof(LayerRec) / 16))
            cp_async16(reinterpret_cast<float4*>(recs + sidx) + threadIdx.x,
                       reinterpret_cast<const float4*>(a.rec + t) + threadIdx.x);
    };
    // Barriers per tile: one after the tile lands (it also frees the other
    // buffer, whose tile every thread has finished, for the next copies) and
    // one before round 2.  Round 0 hands data to round 1 inside a warp: round-1
    // thread u reads what round-0 threads 16 (u >> 4) .. 16 (u >> 4) + 15 wrote,
    // so a warp barrier suffices there.  General mode with per-tile factors
    // rewrites the shared factors each tile and keeps an end-of-tile barrier.
    const bool r1 = ((a.fmask >> 4) & 15u) != 0;
    const bool end_sync = dynamic && !use_rec;
    uint64_t nbase = layer_base(a, blockIdx.x);   // base of the next tile to load
    if (blockIdx.x < a.ntiles) load(blockIdx.x, nbase, 0);
    cp_async_commit();
    int cur = 0;
    for (uint64_t t = blockIdx.x; t < a.ntiles; t += stride) {
        const uint64_t base = nbase;
        nbase = ((nbase | ~a.omask) + a.dstride) & a.omask;
        if (end_sync && threadIdx.x < 32) tile_phases<ROT>(a, base, sh);
        cp_async_wait<0>();
        __syncthreads();
        const uint64_t tn = t + stride;
        if (tn < a.ntiles) load(tn, nbase, cur ^ 1);
        cp_async_commit();
        float2* st = stage + cur * kLAmps;
        const LayerRec& pr = use_rec ? recs[cur] : sh.ph;
        if (first == 0) {
            // round 0 always writes to the stage: its threads hold 16 consecutive
            // amplitudes, so when it is the last round the tile is copied out in
            // 16-byte chunks by consecutive threads instead (coalesced stores)
            layer_round<ROT, 0, DIN, PH, RP, GEN, false>(a, st, din_s, sh, pr, 0, base, phase);
            if (last == 0) {
                // the amplitudes of tile-local j, j + 1 are in place (j ^ rswap),
                // (j + 1) ^ rswap: chunk (j ^ rswap) / 2, halves exchanged if bit 0 is
                __syncthreads();
                const int sx = lsw((2 * threadIdx.x) ^ static_cast<int>(a.rswap & 14u));
                const bool hx = a.rswap & 1u;
#pragma unroll
                for (int k = 0; k < kLAmps / 2 / kLThreads; ++k) {
                    float4 c = *reinterpret_cast<const float4*>(st + (sx ^ lsw(512 * k)));
                    if (hx) c = make_float4(c.z, c.w, c.x, c.y);
                    if (dbg::in_bounds(base | gld | a.goff[48 + k], 2, a.ntiles << 12, 13))
                        __stcs(reinterpret_cast<float4*>(a.psi + (base | gld | a.goff[48 + k])), c);
                }
            } else if (r1) {
                __syncwarp();
            } else {
                __syncthreads();
            }
        }
        if (first <= 1 && last >= 1 && r1) {
            if (last == 1)
                layer_round<ROT, 1, DIN, PH, RP, GEN, true>(a, st, din_s, sh, pr, soff1, base, phase);
            else
                layer_round<ROT, 1, DIN, PH, RP, GEN, false>(a, st, din_s, sh, pr, 0, base, phase);
            if (last > 1) __syncthreads();
        }
        if (last == 2) layer_round<ROT, 2, DIN, PH, RP, GEN, true>(a, st, din_s, sh, pr, soff2, base, phase);
        if (end_sync) __syncthreads();
        cur ^= 1;
    }
    cp_async_wait<0>();
}

}  // namespace

size_t layer_smem_bytes(bool with_din) {
    return sizeof(float2) * kLStages * kLAmps + sizeof(uint64_t) * 512 + sizeof(LayerShared) +
           sizeof(LayerRec) * kLStages + (with_din ? sizeof(float2) * kLAmps : 0);
}

size_t layer_record_bytes(int n) { return n < kLT ? 0 : sizeof(LayerRec) << (n - kLT); }

namespace {

// The launch's arguments: geometry, payload pointers and the tables read from
// the parameter bank (N - 12 <= 24 tile-index bits: states of up to 2^36
// amplitudes, beyond QSA_MAX_QUBITS)
bool layer_args(float2* psi, int n, const LayerGeom& g, const unsigned char* d_payload, const LayerPayload& p,
                LayerArgs* out) {
    if (n < kLT || n - kLT > 24 || g.m + g.nx != kLT || g.m < 3) return false;
    LayerArgs& a = *out;
    a = LayerArgs{};
    a.psi = psi;
    a.ntiles = 1ull << (n - kLT);
    a.m = g.m;
    a.nx = g.nx;
    for (int e = 0; e < kLT; ++e) a.xpos[e] = e < g.nx ? g.xpos[e] : 0;
    a.fmask = p.active;
    a.pmask = p.pmask;
    a.rpmask = p.rpmask;
    a.rswap = p.rswap;
    a.generate = p.generate ? 1 : 0;
    a.ncross = p.ncross;
    a.nout = p.nout;
    for (int b = 0; b <= kLT; ++b) a.cstart[b] = p.cstart[b];
    a.fac = reinterpret_cast<const float2*>(d_payload + p.off_fac);
    a.cross = reinterpret_cast<const LayerGate*>(d_payload + p.off_cross);
    a.outg = reinterpret_cast<const LayerGate*>(d_payload + p.off_out);
    a.din = p.has_din ? reinterpret_cast<const float2*>(d_payload + p.off_din) : nullptr;
    a.qph = reinterpret_cast<const float2*>(d_payload + p.off_qph);
    a.sph = reinterpret_cast<const float2*>(d_payload + p.off_sph);
    // global offsets of tile-local indices: the low m bits in place, bit m + e at xpos[e]
    auto offset = [&](int j) {
        uint64_t off = static_cast<uint64_t>(j & ((1 << g.m) - 1));
        for (int e = 0; e < g.nx; ++e)
            if ((j >> (g.m + e)) & 1) off |= 1ull << g.xpos[e];
        return off;
    };
    for (int t = 0; t < 56; ++t) {
        const int R = t >> 4;
        a.goff[t] = offset(t < 48 ? ((t & 15) ^ static_cast<int>((p.rswap >> (4 * R)) & 15u)) << (4 * R)
                                  : (t - 48) << 9);
    }
    uint64_t tmask = (1ull << g.m) - 1;
    for (int e = 0; e < g.nx; ++e) tmask |= 1ull << g.xpos[e];
    a.omask = ((1ull << n) - 1) & ~tmask;
    a.dstride = 0;   // set with the grid size
    for (int b = 0; b < kLT; ++b) a.rot[b] = p.rot[b];
    for (int i = 0; i < 96; ++i) a.rpe[i] = p.rp[i];
    return true;
}

bool needs_records(const LayerPayload& p) { return p.rotation && (p.ncross > 0 || p.nout > 0); }

}  // namespace

cudaError_t launch_layer_records(float2* psi, int n, const LayerGeom& g, const unsigned char* d_payload,
                                 const LayerPayload& p, void* d_rec, cudaStream_t st, uint64_t* launches) {
    if (!needs_records(p)) return cudaSuccess;
    LayerArgs a;
    if (!layer_args(psi, n, g, d_payload, p, &a) || !d_rec) return cudaErrorInvalidValue;
    // 32 tiles per warp
    uint64_t nb = (a.ntiles + kRecThreads - 1) / kRecThreads;
    const uint64_t cap = static_cast<uint64_t>(num_sms()) * 16;
    if (nb > cap) nb = cap;
    k_layer_records<<<static_cast<unsigned>(nb), kRecThreads, 0, st>>>(a, static_cast<LayerRec*>(d_rec));
    ++*launches;
    return cudaGetLastError();
}

cudaError_t launch_apply_layer(float2* psi, int n, const LayerGeom& g, const unsigned char* d_payload,
                               const LayerPayload& p, void* d_rec, cudaStream_t st, uint64_t* launches) {
    LayerArgs a;
    if (!layer_args(psi, n, g, d_payload, p, &a)) return cudaErrorInvalidValue;
    const size_t smem = layer_smem_bytes(p.has_din);
    {
        for (auto kern : {k_apply_layer<true, 0, 0, 0, 0>, k_apply_layer<true, 0, 1, 0, 0>, k_apply_layer<true, 1, 0, 0, 0>,
                          k_apply_layer<true, 1, 1, 0, 0>, k_apply_layer<true, 0, 0, 2, 0>, k_apply_layer<true, 0, 1, 2, 0>,
                          k_apply_layer<true, 1, 0, 2, 0>, k_apply_layer<true, 1, 1, 2, 0>, k_apply_layer<true, 2, 2, 2, 1>,
                          k_apply_layer<true, 1, 1, 0, 1>, k_apply_layer<false, 2, 2, 2, 2>}) {
            cudaError_t e = set_smem_attr(reinterpret_cast<const void*>(kern), static_cast<int>(layer_smem_bytes(true)));
            if (e != cudaSuccess) return e;
        }
    }
    if (needs_records(p)) {
        if (!d_rec) return cudaErrorInvalidValue;
        a.rec = static_cast<const LayerRec*>(d_rec);   // written by launch_layer_records before
    }
    // rotation mode: the diagonal table and the per-tile phases fixed at compile time (the write-only
    // pass too in its usual form: a diagonal table, per-tile phases, exit phases handed on)
    const bool ph = p.pmask != 0 || p.nout > 0;
    auto kern = !p.rotation ? k_apply_layer<false, 2, 2, 2, 2>
                : p.generate ? (p.has_din && ph && p.rpmask == 0 ? k_apply_layer<true, 1, 1, 0, 1>
                                                                 : k_apply_layer<true, 2, 2, 2, 1>)
                : p.rpmask == 0
                    ? (p.has_din ? (ph ? k_apply_layer<true, 1, 1, 0, 0> : k_apply_layer<true, 1, 0, 0, 0>)
                                 : (ph ? k_apply_layer<true, 0, 1, 0, 0> : k_apply_layer<true, 0, 0, 0, 0>))
                    : (p.has_din ? (ph ? k_apply_layer<true, 1, 1, 2, 0> : k_apply_layer<true, 1, 0, 2, 0>)
                                 : (ph ? k_apply_layer<true, 0, 1, 2, 0> : k_apply_layer<true, 0, 0, 2, 0>));
    int occ = 0;
    cudaError_t e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, kern, kLThreads, smem);
    if (e != cudaSuccess) return e;
    if (occ < 1) occ = 1;
    uint64_t grid = static_cast<uint64_t>(num_sms()) * occ;
    if (grid > a.ntiles) grid = a.ntiles;
    // the grid size deposited into the positions outside the tile
    for (uint64_t v = grid, pos = 0; v && pos < 64; ++pos)
        if ((a.omask >> pos) & 1) {
            if (v & 1) a.dstride |= 1ull << pos;
            v >>= 1;
        }
    kern<<<static_cast<unsigned>(grid), kLThreads, smem, st>>>(a);
    ++*launches;
    return cudaGetLastError();
}

QSA_BOUNDS_READER(bounds_word_layer)

}  // namespace qsa
