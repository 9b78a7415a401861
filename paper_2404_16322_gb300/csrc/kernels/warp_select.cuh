// Warp-level selection helpers shared by the top-nprobe select and the top-K
// merge.
#pragma once

#include <stdint.h>

namespace dade {

// The k-th smallest (1-based, k <= n) 32-bit pattern among keys(i), i < n,
// by an MSD radix select over 8-bit digits, one warp.  `hist` is the warp's
// 256-int scratch in shared memory.  Keys of non-negative floats compare as
// their bit patterns.
template <class Key>
__device__ uint32_t warp_kth_key(Key keys, int n, int k, int* hist, int lane) {
    uint32_t prefix = 0, mask = 0;
    for (int shift = 24; shift >= 0; shift -= 8) {
        for (int b = lane; b < 256; b += 32) hist[b] = 0;
        __syncwarp();
        for (int i = lane; i < n; i += 32) {
            const uint32_t key = keys(i);
            if ((key & mask) == prefix) atomicAdd(&hist[(key >> shift) & 255u], 1);
        }
        __syncwarp();
        // lane j owns bins [8j, 8j + 8): find the bin where the count reaches k
        int h[8], s = 0;
#pragma unroll
        for (int u = 0; u < 8; ++u) {
            h[u] = hist[lane * 8 + u];
            s += h[u];
        }
        int incl = s;
#pragma unroll
        for (int off = 1; off < 32; off <<= 1) {
            const int o = __shfl_up_sync(0xffffffffu, incl, off);
            if (lane >= off) incl += o;
        }
        const int excl = incl - s;
        const unsigned hit = __ballot_sync(0xffffffffu, excl < k && incl >= k);
        const int src = __ffs(hit) - 1;
        int digit = 0, below = 0;
        if (lane == src) {
            int cum = excl;
#pragma unroll
            for (int u = 0; u < 8; ++u) {
                if (cum + h[u] >= k) {
                    digit = lane * 8 + u;
                    break;
                }
                cum += h[u];
            }
            below = cum;
        }
        digit = __shfl_sync(0xffffffffu, digit, src);
        below = __shfl_sync(0xffffffffu, below, src);
        k -= below;
        prefix |= (uint32_t)digit << shift;
        mask |= 255u << shift;
        __syncwarp();
    }
    return prefix;
}

}  // namespace dade
