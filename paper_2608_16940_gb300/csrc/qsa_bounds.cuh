// Debug-build bounds checks on the state's global accesses.
//
// Built with -DQSA_DEBUG_BOUNDS (build.py --debug-bounds, which writes
// libqsa_debug.so beside libqsa.so), a checked access whose index lies outside
// the state is skipped and the first such event of the translation unit is
// recorded as (code << 48) | index; qsa_debug_bounds_status() returns the
// first record it finds.  No check traps or asserts: the kernel runs on, so a
// wrong index shows up as a record (and a wrong result), never as a device
// fault.  Without the flag every check is the constant true and compiles away.
#pragma once

#include <cuda_runtime.h>

#include <cstdint>

namespace qsa {
namespace dbg {

#ifdef QSA_DEBUG_BOUNDS
static __device__ unsigned long long g_fail = 0;

// [first, first + count) must lie in [0, limit).
__device__ __forceinline__ bool in_bounds(uint64_t first, uint64_t count, uint64_t limit, unsigned code) {
    if (first + count <= limit) return true;
    atomicCAS(&g_fail, 0ull, (static_cast<unsigned long long>(code) << 48) | (first & 0xffffffffffffull));
    return false;
}

static inline uint64_t read_fail() {
    unsigned long long v = 0;
    if (cudaMemcpyFromSymbol(&v, g_fail, sizeof(v)) != cudaSuccess) return ~0ull;
    return v;
}
#else
__device__ __forceinline__ bool in_bounds(uint64_t, uint64_t, uint64_t, unsigned) { return true; }
static inline uint64_t read_fail() { return 0; }
#endif

}  // namespace dbg
}  // namespace qsa

// A translation unit with checks defines its reader (declared in
// qsa_internal.h) with this macro, inside namespace qsa.
#define QSA_BOUNDS_READER(name) \
    uint64_t name() { return dbg::read_fail(); }
