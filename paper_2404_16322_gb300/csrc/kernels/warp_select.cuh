// Warp-level selection helpers shared by the top-nprobe select and the top-K
// merge.
#pragma once

#include <climits>
#include <math.h>
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

// ------------------------------------------------------------ 128 in registers
// A warp holds 128 (key, id) entries, entry e = 32 r + lane in slot r of
// lane `lane`, ordered by (key, id).  Bitonic networks over them exchange
// across lanes with shuffles and across slots with swaps.
// Ent carries a 64-bit id; Ent32 a 32-bit one (fewer shuffles and
// registers) where every id fits.
struct Ent {
    float d;
    long long id;
};
struct Ent32 {
    float d;
    int id;
};
template <class E>
__device__ __forceinline__ bool ent_less(const E& a, const E& b) { return a.d < b.d || (a.d == b.d && a.id < b.id); }
template <class E>
__device__ __forceinline__ E shfl_xor_ent(const E& x, int m) {
    E y;
    y.d = __shfl_xor_sync(0xffffffffu, x.d, m);
    y.id = __shfl_xor_sync(0xffffffffu, x.id, m);
    return y;
}
template <class E>
__device__ __forceinline__ E shfl_ent(const E& x, int src) {
    E y;
    y.d = __shfl_sync(0xffffffffu, x.d, src);
    y.id = __shfl_sync(0xffffffffu, x.id, src);
    return y;
}
// the padding entry (after every real one)
template <class E>
__device__ __forceinline__ E ent_pad() {
    E y;
    y.d = INFINITY;
    y.id = sizeof(y.id) == 8 ? (decltype(y.id))LLONG_MAX : (decltype(y.id))INT_MAX;
    return y;
}

// Entry e of the 128 (slot e / 32 of lane e % 32), to every lane; the slot
// is chosen with selects, not an indexed register array.
template <class E>
__device__ __forceinline__ E entry_at(const E (&v)[4], int e) {
    const int r = e >> 5;
    E x = v[0];
    if (r == 1) x = v[1];
    if (r == 2) x = v[2];
    if (r == 3) x = v[3];
    return shfl_ent(x, e & 31);
}

// One compare-exchange level (distance j) of a bitonic network over the 128
// entries; `up(e)` tells whether the block containing entry e sorts upward.
template <class E, class Up>
__device__ __forceinline__ void bitonic_level(E (&v)[4], int j, int lane, Up up) {
    if (j >= 32) {
        const int js = j >> 5;
#pragma unroll
        for (int r = 0; r < 4; ++r) {
            const int p = r ^ js;
            if (p > r) {
                const bool asc = up(r * 32 + lane);
                const bool sw = asc ? ent_less(v[p], v[r]) : ent_less(v[r], v[p]);
                if (sw) {
                    const E t = v[r];
                    v[r] = v[p];
                    v[p] = t;
                }
            }
        }
    } else {
#pragma unroll
        for (int r = 0; r < 4; ++r) {
            const int e = r * 32 + lane;
            const E o = shfl_xor_ent(v[r], j);
            const bool lower = (lane & j) == 0;
            const bool asc = up(e);
            // the lower entry of an upward pair keeps the smaller one
            const bool take_min = lower == asc;
            const bool o_less = ent_less(o, v[r]);
            if (take_min ? o_less : !o_less && (o.d != v[r].d || o.id != v[r].id)) v[r] = o;
        }
    }
}

template <class E>
__device__ __forceinline__ void bitonic_sort128(E (&v)[4], int lane) {
#pragma unroll
    for (int k = 2; k <= 128; k <<= 1)
#pragma unroll
        for (int j = k >> 1; j > 0; j >>= 1) bitonic_level(v, j, lane, [k](int e) { return (e & k) == 0; });
}


// (key, 32-bit payload) pairs, 128 per warp (slot r of lane l = entry 32 r + l),
// sorted by a bitonic network: the same network as bitonic_sort128 with a
// 32-bit payload (two shuffles per exchange instead of three).
struct KV {
    float d;
    int c;
};
__device__ __forceinline__ bool kv_less(const KV& a, const KV& b) { return a.d < b.d || (a.d == b.d && a.c < b.c); }

__device__ __forceinline__ void kv_sort128(KV (&v)[4], int lane) {
#pragma unroll
    for (int k = 2; k <= 128; k <<= 1) {
#pragma unroll
        for (int j = k >> 1; j > 0; j >>= 1) {
            if (j >= 32) {
                const int js = j >> 5;
#pragma unroll
                for (int r = 0; r < 4; ++r) {
                    const int p = r ^ js;
                    if (p > r) {
                        const bool asc = ((r * 32 + lane) & k) == 0;
                        if (asc ? kv_less(v[p], v[r]) : kv_less(v[r], v[p])) {
                            const KV t = v[r];
                            v[r] = v[p];
                            v[p] = t;
                        }
                    }
                }
            } else {
#pragma unroll
                for (int r = 0; r < 4; ++r) {
                    KV o;
                    o.d = __shfl_xor_sync(0xffffffffu, v[r].d, j);
                    o.c = __shfl_xor_sync(0xffffffffu, v[r].c, j);
                    const bool asc = ((r * 32 + lane) & k) == 0;
                    const bool take_min = ((lane & j) == 0) == asc;
                    const bool o_less = kv_less(o, v[r]);
                    if (take_min ? o_less : !o_less && (o.d != v[r].d || o.c != v[r].c)) v[r] = o;
                }
            }
        }
    }
}

}  // namespace dade
