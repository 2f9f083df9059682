// Ranking a tile of consecutive (Morton-ordered) particles by the length of
// their neighbour lists, for the one-thread-per-particle list walks (the
// density solve and the gradient sums).  A warp runs until its longest list
// is done; on clustered particle sets the list lengths vary several-fold
// between neighbouring particles, so a warp of consecutive particles idles
// most of its lanes.  Sorting the tile's particles by length and handing
// rank r of round k to thread r of that round gives each warp lists of
// nearly equal length; a tile larger than the CTA (R rounds of 128) evens
// them further, while the tile stays a compact piece of the Morton curve, so
// the gathers keep their locality.
#pragma once

#include <stdint.h>

namespace hyd {

constexpr int RANK_THREADS = 128;
constexpr int RANK_MAX_ROUNDS = 8;

// rounds per CTA for n particles: the largest of 8, 4, 2, 1 that still
// leaves at least eight CTAs per SM of the 152 to spread over the GPU
inline int rank_rounds(int64_t n) {
    int r = RANK_MAX_ROUNDS;
    while (r > 1 && (n + (int64_t)RANK_THREADS * r - 1) / ((int64_t)RANK_THREADS * r) < 152 * 8)
        r >>= 1;
    return r;
}

// key[0 .. 128 rounds) = (list length << lb) | tile index, ascending, for the
// tile of particles [base, base + 128 rounds) (rounds a power of two, lb its
// log2 + 7); particles at or beyond n sort first with length 0.  Every
// thread of the 128-thread CTA takes part (it synchronises the block).
__device__ __forceinline__ void rank_tile(unsigned *key, int rounds, const int32_t *cnt,
                                          int64_t base, int64_t n) {
    const int G = RANK_THREADS * rounds;
    const int lb = 7 + __ffs(rounds) - 1;
    const unsigned lmax = (1u << (32 - lb)) - 1u;
    for (int t = threadIdx.x; t < G; t += RANK_THREADS) {
        const int64_t s = base + t;
        const unsigned len = s < n ? min((unsigned)max(cnt[s], 0), lmax) : 0u;
        key[t] = (len << lb) | (unsigned)t;
    }
    __syncthreads();
    // bitonic sort: each thread takes the compare-exchanges of its indices
    for (int k = 2; k <= G; k <<= 1) {
        for (int j = k >> 1; j > 0; j >>= 1) {
            for (int t = threadIdx.x; t < G; t += RANK_THREADS) {
                const int u = t ^ j;
                if (u > t) {
                    const unsigned x = key[t], y = key[u];
                    if ((x > y) == ((t & k) == 0)) { key[t] = y; key[u] = x; }
                }
            }
            __syncthreads();
        }
    }
}

// the tile index held by a key of a tile of 128 rounds particles
__device__ __forceinline__ int rank_index(unsigned key, int rounds) {
    return (int)(key & (unsigned)(RANK_THREADS * rounds - 1));
}

}  // namespace hyd
