/*
 * qsa_oracle.c — TEST INFRASTRUCTURE ONLY.
 *
 * A plain, slow, single-threaded FP64 state-vector simulator used to check
 * the CUDA library.  Only tests/, __graft_entry__.smoke() and bench.py's
 * cpu_baseline / reference leg may load it.  It shares no code, header or
 * table with the CUDA path.  Every loop is written straight from the
 * definition it cites, with no blocking, fusion or reordering.
 *
 * Conventions (paper §II, "State and layout notation"):
 *   - amplitude psi_x is stored interleaved: psi[2x] = Re, psi[2x+1] = Im;
 *   - bit p of the flat index x is qubit / position p, position 0 least
 *     significant;
 *   - a k-qubit matrix G acts on the ordered tuple V = (q_0..q_{k-1}); q_j
 *     supplies bit j of the row and column index (little-endian within the
 *     tuple, §II "Fused gates and requests").  G is row-major, G[r][c] at
 *     mat[2*(r*2^k + c)] (+1 for Im).
 *
 * The oracle always works in canonical logical order (layout = identity);
 * the layout map enters only where the paper says the consumer decodes
 * through it (the sampler, §IV-D "terminal computational-basis count
 * sampling decodes logical output bits through the final map").
 */
#include <stdint.h>
#include <stddef.h>
#include <stdlib.h>
#include <string.h>
#include <math.h>

#define ORC_OK 0
#define ORC_EARG 1

/* spread(c) = sum_j bit_j(c) << q_j : the basis index offset selected by row /
 * column index c of G under the little-endian tuple convention (§II). */
static uint64_t spread_bits(uint64_t c, const int* targets, int k) {
    uint64_t off = 0;
    for (int j = 0; j < k; ++j)
        if ((c >> j) & 1u) off |= (uint64_t)1 << targets[j];
    return off;
}

/*
 * apply(G, V): for every basis index x whose target bits are all zero, gather
 * v[c] = psi[x | spread(c)], then psi[x | spread(r)] = sum_c G[r][c] v[c].
 * This is the left multiplication by G of the 2^k x 2^(N-k) view in §IV-B
 * ("left multiplication by G applies the fused gate independently to every
 * column"), written without the permutation: the column is the assignment x
 * of the non-target bits.
 */
int orc_apply(double* psi, int n, const int* targets, int k, const double* mat) {
    if (n < 1 || n > 34 || k < 1 || k > 10 || k > n) return ORC_EARG;
    uint64_t tmask = 0;
    for (int j = 0; j < k; ++j) {
        if (targets[j] < 0 || targets[j] >= n) return ORC_EARG;
        if (tmask & ((uint64_t)1 << targets[j])) return ORC_EARG;
        tmask |= (uint64_t)1 << targets[j];
    }
    const uint64_t d = (uint64_t)1 << k;
    double* v = (double*)malloc(sizeof(double) * 2 * d);
    if (!v) return ORC_EARG;
    const uint64_t dim = (uint64_t)1 << n;
    for (uint64_t x = 0; x < dim; ++x) {
        if (x & tmask) continue;
        for (uint64_t c = 0; c < d; ++c) {
            uint64_t idx = x | spread_bits(c, targets, k);
            v[2 * c] = psi[2 * idx];
            v[2 * c + 1] = psi[2 * idx + 1];
        }
        for (uint64_t r = 0; r < d; ++r) {
            double re = 0.0, im = 0.0;
            for (uint64_t c = 0; c < d; ++c) {
                double gr = mat[2 * (r * d + c)], gi = mat[2 * (r * d + c) + 1];
                re += gr * v[2 * c] - gi * v[2 * c + 1];
                im += gr * v[2 * c + 1] + gi * v[2 * c];
            }
            uint64_t idx = x | spread_bits(r, targets, k);
            psi[2 * idx] = re;
            psi[2 * idx + 1] = im;
        }
    }
    free(v);
    return ORC_OK;
}

/* p(x) = |psi_x|^2 (§IV-E "Sampling"), canonical order. */
void orc_probabilities(const double* psi, int n, double* p) {
    const uint64_t dim = (uint64_t)1 << n;
    for (uint64_t x = 0; x < dim; ++x)
        p[x] = psi[2 * x] * psi[2 * x] + psi[2 * x + 1] * psi[2 * x + 1];
}

/* <Z_mask> = sum_x (-1)^{popcount(x & mask)} |psi_x|^2; mask = 0 gives the norm. */
double orc_expect_z(const double* psi, int n, uint64_t mask) {
    const uint64_t dim = (uint64_t)1 << n;
    double s = 0.0;
    for (uint64_t x = 0; x < dim; ++x) {
        double p = psi[2 * x] * psi[2 * x] + psi[2 * x + 1] * psi[2 * x + 1];
        int par = 0;
        for (uint64_t m = x & mask; m; m >>= 1) par ^= (int)(m & 1u);
        s += par ? -p : p;
    }
    return s;
}

/*
 * Philox4x64-10 (Salmon, Moraes, Dror, Shaw, "Parallel random numbers: as easy
 * as 1, 2, 3", SC'11): ten rounds of the 4x64 S-box; the key is bumped by the
 * Weyl constants between rounds.  Used as the counter-based generator of the
 * sampler; the CUDA side has its own implementation of the same definition.
 */
static void mulhilo64(uint64_t a, uint64_t b, uint64_t* hi, uint64_t* lo) {
    unsigned __int128 p = (unsigned __int128)a * (unsigned __int128)b;
    *hi = (uint64_t)(p >> 64);
    *lo = (uint64_t)p;
}

void orc_philox4x64_10(const uint64_t ctr_in[4], const uint64_t key_in[2], uint64_t out[4]) {
    const uint64_t M0 = 0xD2E7470EE14C6C93ull, M1 = 0xCA5A826395121157ull;
    const uint64_t W0 = 0x9E3779B97F4A7C15ull, W1 = 0xBB67AE8584CAA73Bull;
    uint64_t x0 = ctr_in[0], x1 = ctr_in[1], x2 = ctr_in[2], x3 = ctr_in[3];
    uint64_t k0 = key_in[0], k1 = key_in[1];
    for (int round = 0; round < 10; ++round) {
        if (round > 0) { k0 += W0; k1 += W1; }
        uint64_t hi0, lo0, hi1, lo1;
        mulhilo64(M0, x0, &hi0, &lo0);
        mulhilo64(M1, x2, &hi1, &lo1);
        uint64_t y0 = hi1 ^ x1 ^ k0, y1 = lo1, y2 = hi0 ^ x3 ^ k1, y3 = lo0;
        x0 = y0; x1 = y1; x2 = y2; x3 = y3;
    }
    out[0] = x0; out[1] = x1; out[2] = x2; out[3] = x3;
}

/*
 * Sampling (§IV-E "Sampling", App. B "Numerical configuration", §IV-D).
 * Draw physical outcome y with probability p(y) through the cumulative
 * distribution, using a strict upper bound so a zero-probability bin is
 * never chosen, then decode the logical outcome through the layout map.
 *
 * Reading fixed here (the paper keeps FP64 block sums, whose value depends on
 * the summation order): the weight of a physical index is the integer
 * P_y = floor(re^2 * 2^60) + floor(im^2 * 2^60), each term the exact square
 * truncated to 60 fractional bits (|amplitude| < 2 assumed); the CDF is the
 * integer prefix sum C_y = sum_{y' <= y} P_y', so it is exact and independent
 * of summation order.
 * Shot s of stream t draws r = Philox4x64-10(ctr = (s, t, 0, 0),
 * key = (seed, 0)).word0, maps it to u = floor(r * C_last / 2^64) in
 * [0, C_last) (multiply-high range reduction: u moves by less than the change
 * of C_last when the weights change slightly), and takes the first y with
 * C_y > u.  The logical outcome x has x_q = y_{L(q)}.
 *
 *   amps_logical: FP64 interleaved amplitudes in canonical logical order;
 *   phys_of_logical: L(q) for q < n; the physical amplitude at index y is the
 *                    logical one at decode(y).
 *   near_frac: a draw is flagged when u lies within near_frac * 2^60 of the
 *              cumulative value on either side of the chosen bin.
 * Returns ORC_OK, or ORC_EARG if every weight is zero.
 */
/* floor(v^2 * 2^60) exactly: v = M * 2^(e-53) with a 53-bit integer M, so
 * v^2 * 2^60 = M^2 * 2^(2e-46), formed in 128-bit integers. */
static uint64_t sq_fixed60(double v) {
    if (v == 0.0) return 0;
    int e;
    double fr = frexp(fabs(v), &e);                 /* fr in [0.5, 1) */
    uint64_t M = (uint64_t)ldexp(fr, 53);           /* exact */
    unsigned __int128 sq = (unsigned __int128)M * (unsigned __int128)M;
    int s = 2 * e - 46;
    if (s >= 0) return (uint64_t)(sq << s);
    if (-s >= 128) return 0;
    return (uint64_t)(sq >> (-s));
}

static uint64_t decode_phys(uint64_t y, const int* phys_of_logical, int n) {
    uint64_t x = 0;
    for (int q = 0; q < n; ++q)
        if ((y >> phys_of_logical[q]) & 1u) x |= (uint64_t)1 << q;
    return x;
}

int orc_sample(const double* amps_logical, int n, const int* phys_of_logical,
               uint64_t shots, uint64_t seed, uint64_t stream, double near_frac,
               uint64_t* outcomes_logical, uint8_t* flagged) {
    const uint64_t dim = (uint64_t)1 << n;
    uint64_t* cum = (uint64_t*)malloc(sizeof(uint64_t) * dim);
    if (!cum) return ORC_EARG;
    const double two60 = 1152921504606846976.0; /* 2^60 */
    uint64_t run = 0;
    for (uint64_t y = 0; y < dim; ++y) {
        uint64_t x = decode_phys(y, phys_of_logical, n);
        run += sq_fixed60(amps_logical[2 * x]) + sq_fixed60(amps_logical[2 * x + 1]);
        cum[y] = run;
    }
    const uint64_t total = run;
    if (total == 0) { free(cum); return ORC_EARG; }
    const double near_abs = near_frac * two60;
    for (uint64_t s = 0; s < shots; ++s) {
        uint64_t ctr[4] = {s, stream, 0, 0}, key[2] = {seed, 0}, out[4];
        orc_philox4x64_10(ctr, key, out);
        uint64_t u = (uint64_t)(((unsigned __int128)out[0] * (unsigned __int128)total) >> 64);
        /* first y with cum[y] > u (binary search over a non-decreasing array) */
        uint64_t lo = 0, hi = dim - 1;
        while (lo < hi) {
            uint64_t mid = lo + (hi - lo) / 2;
            if (cum[mid] > u) hi = mid; else lo = mid + 1;
        }
        outcomes_logical[s] = decode_phys(lo, phys_of_logical, n);
        if (flagged) {
            uint64_t below = lo ? cum[lo - 1] : 0;
            double d1 = (double)(u - below), d2 = (double)(cum[lo] - u);
            flagged[s] = (d1 < near_abs || d2 <= near_abs) ? 1 : 0;
        }
    }
    free(cum);
    return ORC_OK;
}
