// Diagonal streaming update: the diagonal branch of the axis-shifted lowering
// (Alg. 2: multiply each amplitude by the diagonal entry indexed by the
// target bits; Eq. cost-diag-formal: one streaming pass, no permutation, the
// layout unchanged).
//
// Each thread updates pairs of amplitudes (one 16-byte float4, physical
// indices y and y + 1) and keeps six pairs in flight; four 256-thread CTAs per
// SM fit both the registers and the widest (2^12-entry) table.  The entry index c(y)
// (bit j = bit p_j of y) is assembled from three shared tables over bits
// 0..11, 12..23 and 24..33 of y; the 2^k-entry FP32 table itself sits in
// shared memory.  Loads and stores stream (evict-first): 16 B per amplitude.
#include <cuda_runtime.h>

#include <algorithm>
#include <cstdint>

#include "qsa_internal.h"

namespace qsa {

namespace {

constexpr int kDiagThreads = 256;
constexpr int kDiagUnroll = 6;

struct DiagArgs {
    float4* psi;
    uint64_t npairs;
    const float2* d;
    int k;
    int p[QSA_MAX_DIAG];
};

__device__ __forceinline__ float4 cmul2(float4 v, float2 a, float2 b) {
    float4 w;
    w.x = v.x * a.x - v.y * a.y;
    w.y = v.x * a.y + v.y * a.x;
    w.z = v.z * b.x - v.w * b.y;
    w.w = v.z * b.y + v.w * b.x;
    return w;
}

__global__ void __launch_bounds__(kDiagThreads, 4) k_apply_diag(DiagArgs a) {
    extern __shared__ __align__(16) unsigned char smem[];
    float2* d = reinterpret_cast<float2*>(smem);
    uint16_t* t0 = reinterpret_cast<uint16_t*>(d + (1 << a.k));   // bits 0..11 of y
    uint16_t* t1 = t0 + 4096;                                       // bits 12..23
    uint16_t* t2 = t1 + 4096;                                       // bits 24..33
    for (int i = threadIdx.x; i < (1 << a.k); i += blockDim.x) d[i] = a.d[i];
    for (int i = threadIdx.x; i < 4096; i += blockDim.x) {
        uint32_t c0 = 0, c1 = 0, c2 = 0;
        for (int j = 0; j < a.k; ++j) {
            const int p = a.p[j];
            if (p < 12)
                c0 |= ((static_cast<uint32_t>(i) >> p) & 1u) << j;
            else if (p < 24)
                c1 |= ((static_cast<uint32_t>(i) >> (p - 12)) & 1u) << j;
            else
                c2 |= ((static_cast<uint32_t>(i) >> (p - 24)) & 1u) << j;
        }
        t0[i] = static_cast<uint16_t>(c0);
        t1[i] = static_cast<uint16_t>(c1);
        if (i < 1024) t2[i] = static_cast<uint16_t>(c2);
    }
    __syncthreads();

    const uint64_t stride = static_cast<uint64_t>(gridDim.x) * blockDim.x;
    for (uint64_t q0 = static_cast<uint64_t>(blockIdx.x) * blockDim.x + threadIdx.x; q0 < a.npairs;
         q0 += kDiagUnroll * stride) {
        float4 v[kDiagUnroll];
#pragma unroll
        for (int u = 0; u < kDiagUnroll; ++u) {
            const uint64_t q = q0 + u * stride;
            if (q < a.npairs) v[u] = __ldcs(a.psi + q);
        }
#pragma unroll
        for (int u = 0; u < kDiagUnroll; ++u) {
            const uint64_t q = q0 + u * stride;
            if (q < a.npairs) {
                const uint64_t y = q << 1;
                const uint32_t hi = static_cast<uint32_t>(t1[(y >> 12) & 4095u]) | t2[(y >> 24) & 1023u];
                const uint32_t lo = static_cast<uint32_t>(y) & 4095u;
                __stcs(a.psi + q, cmul2(v[u], d[t0[lo] | hi], d[t0[lo | 1u] | hi]));
            }
        }
    }
}

size_t diag_smem(int k) { return (sizeof(float2) << k) + 2 * (4096 + 4096 + 1024); }

}  // namespace

cudaError_t launch_apply_diag(float2* psi, int n, const int* phys, int k, const float* d_tab, cudaStream_t st,
                              uint64_t* launches) {
    if (k < 1 || k > QSA_MAX_DIAG || k > n || n > QSA_MAX_QUBITS) return cudaErrorInvalidValue;
    DiagArgs a{};
    a.psi = reinterpret_cast<float4*>(psi);
    a.npairs = 1ull << (n - 1);
    a.d = reinterpret_cast<const float2*>(d_tab);
    a.k = k;
    for (int j = 0; j < k; ++j) a.p[j] = phys[j];
    {
        cudaError_t e = set_smem_attr(reinterpret_cast<const void*>(k_apply_diag),
                                      static_cast<int>(diag_smem(QSA_MAX_DIAG)));
        if (e != cudaSuccess) return e;
    }
    const size_t sm = diag_smem(k);
    int occ = 0;
    cudaError_t e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, k_apply_diag, kDiagThreads, sm);
    if (e != cudaSuccess) return e;
    if (occ < 1) return cudaErrorInvalidConfiguration;
    const uint64_t need = (a.npairs + kDiagThreads - 1) / kDiagThreads;
    const uint64_t grid = std::min<uint64_t>(static_cast<uint64_t>(num_sms()) * occ, need);
    k_apply_diag<<<static_cast<unsigned>(grid), kDiagThreads, sm, st>>>(a);
    ++*launches;
    return cudaGetLastError();
}

}  // namespace qsa
