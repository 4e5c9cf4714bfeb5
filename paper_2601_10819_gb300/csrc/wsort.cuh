// Sorting networks in registers shared by the deterministic backward paths (sm_103a).
#pragma once

#include <stdint.h>

namespace msda {

// Ascending bitonic sort of one value per lane across the warp.
__device__ __forceinline__ uint32_t warp_sort32(uint32_t x, int lane) {
#pragma unroll
    for (int k = 2; k <= 32; k <<= 1) {
#pragma unroll
        for (int j = k >> 1; j > 0; j >>= 1) {
            const uint32_t y = __shfl_xor_sync(0xffffffffu, x, j);
            const bool up = (lane & k) == 0, low = (lane & j) == 0;
            x = (up == low) ? min(x, y) : max(x, y);
        }
    }
    return x;
}

// Ascending bitonic sort of 32 * E values held E per lane, element index lane * E + e: partners closer than E
// sit in the same lane's registers, farther ones in lane ^ (j / E).
template <int E>
__device__ __forceinline__ void warp_sort_regs(uint32_t (&v)[E], int lane) {
#pragma unroll
    for (int k = 2; k <= 32 * E; k <<= 1) {
#pragma unroll
        for (int j = k >> 1; j > 0; j >>= 1) {
            if (j < E) {
#pragma unroll
                for (int e = 0; e < E; ++e) {
                    if ((e & j) == 0) {
                        const bool up = ((lane * E + e) & k) == 0;
                        const uint32_t a = v[e], b = v[e + j];
                        v[e] = up ? min(a, b) : max(a, b);
                        v[e + j] = up ? max(a, b) : min(a, b);
                    }
                }
            } else {
                const int lj = j / E;
#pragma unroll
                for (int e = 0; e < E; ++e) {
                    const uint32_t y = __shfl_xor_sync(0xffffffffu, v[e], lj);
                    const bool up = ((lane * E + e) & k) == 0, low = (lane & lj) == 0;
                    v[e] = (up == low) ? min(v[e], y) : max(v[e], y);
                }
            }
        }
    }
}

// Ascending odd-even transposition sort of N values held by one thread (N rounds of neighbour exchanges).
template <int N>
__device__ __forceinline__ void thread_sort(uint32_t (&v)[N]) {
#pragma unroll
    for (int rd = 0; rd < N; ++rd) {
#pragma unroll
        for (int j = rd & 1; j + 1 < N; j += 2) {
            const uint32_t lo = min(v[j], v[j + 1]), hi = max(v[j], v[j + 1]);
            v[j] = lo;
            v[j + 1] = hi;
        }
    }
}

}  // namespace msda
