// Top-nprobe bucket selection (Section II-A: a query probes its nprobe
// nearest centroids).  nprobe <= 128: select128_kernel (registers, below).
// Larger nprobe: one warp per query, an MSD radix select over the
// 32-bit patterns of the non-negative FP32 distances (monotone as unsigned
// integers) finds the nprobe-th smallest key; the keys below it and the
// lowest-id keys equal to it are gathered in column order and sorted by
// (distance, list id) with a bitonic network.
#include "../dade_internal.h"
#include "warp_select.cuh"

namespace dade {
namespace {

constexpr int NT = 256;
constexpr int PMAX = 1024;

__device__ __forceinline__ bool key_less(uint32_t ka, int ia, uint32_t kb, int ib) {
    return ka < kb || (ka == kb && ia < ib);
}

constexpr int kSelWarps = 8;

struct RowKeys {
    const float* row;
    __device__ uint32_t operator()(int i) const { return __float_as_uint(row[i]); }
};

// One warp per query: the np-th smallest key by a warp radix select, then
// the keys below it and the lowest-column keys equal to it, gathered in
// column order with ballots and sorted by (key, column) with a warp bitonic
// network.  No CTA-wide barrier.
__global__ void __launch_bounds__(kSelWarps * 32) select_kernel(const float* __restrict__ scores, int64_t B,
                                                               int n, const int32_t* __restrict__ nprobe, int P,
                                                               int32_t* __restrict__ probes,
                                                               int32_t* __restrict__ status) {
    extern __shared__ __align__(16) unsigned char ssm[];
    __shared__ int hist[kSelWarps][256];
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const int64_t b = (int64_t)blockIdx.x * kSelWarps + warp;
    if (b >= B) return;  // whole warps past the last row (no CTA barrier follows)
    const int Pp = 1 << (32 - __clz(P - 1 > 0 ? P - 1 : 1));  // next power of two >= P (>= 2)
    uint32_t* sel_key = reinterpret_cast<uint32_t*>(ssm) + (size_t)warp * 2 * Pp;
    int* sel_id = reinterpret_cast<int*>(sel_key + Pp);
    const float* row = scores + b * (int64_t)n;
    int32_t* out = probes + b * (int64_t)P;
    const int np = nprobe[b];
    if (np < 1 || np > P || np > n) {
        // nprobe = 0 marks an inactive query slot; other values are errors
        if (lane == 0 && status && np != 0) atomicCAS(status, 0, (int)DADE_EINVAL);
        for (int r = lane; r < P; r += 32) out[r] = -1;
        return;
    }
    const uint32_t kth = warp_kth_key(RowKeys{row}, n, np, hist[warp], lane);
    // count the keys below kth to know how many equal keys are needed
    int n_lt = 0;
    for (int i = lane; i < n; i += 32) n_lt += __float_as_uint(row[i]) < kth;
    for (int off = 16; off; off >>= 1) n_lt += __shfl_xor_sync(0xffffffffu, n_lt, off);
    const int need_eq = np - n_lt;
    int c_lt = 0, c_eq = 0;
    for (int base = 0; base < n; base += 32) {
        const int i = base + lane;
        const uint32_t key = i < n ? __float_as_uint(row[i]) : 0xffffffffu;
        const bool lt = i < n && key < kth, eq = i < n && key == kth;
        const unsigned blt = __ballot_sync(0xffffffffu, lt), beq = __ballot_sync(0xffffffffu, eq);
        const unsigned below = (1u << lane) - 1u;
        if (lt) {
            const int pos = c_lt + __popc(blt & below);
            sel_key[pos] = key;
            sel_id[pos] = i;
        }
        if (eq) {
            const int r = c_eq + __popc(beq & below);
            if (r < need_eq) {
                sel_key[n_lt + r] = key;
                sel_id[n_lt + r] = i;
            }
        }
        c_lt += __popc(blt);
        c_eq += __popc(beq);
    }
    int M = 1;
    while (M < np) M <<= 1;
    for (int i = np + lane; i < M; i += 32) {
        sel_key[i] = 0xffffffffu;
        sel_id[i] = 0x7fffffff;
    }
    __syncwarp();
    for (int size = 2; size <= M; size <<= 1) {
        for (int stride = size >> 1; stride > 0; stride >>= 1) {
            for (int i = lane; i < M; i += 32) {
                const int j = i ^ stride;
                if (j > i) {
                    const bool up = (i & size) == 0;
                    const bool sw = up ? key_less(sel_key[j], sel_id[j], sel_key[i], sel_id[i])
                                       : key_less(sel_key[i], sel_id[i], sel_key[j], sel_id[j]);
                    if (sw) {
                        const uint32_t tk = sel_key[i];
                        sel_key[i] = sel_key[j];
                        sel_key[j] = tk;
                        const int ti = sel_id[i];
                        sel_id[i] = sel_id[j];
                        sel_id[j] = ti;
                    }
                }
            }
            __syncwarp();
        }
    }
    for (int r = lane; r < P; r += 32) out[r] = r < np ? sel_id[r] : -1;
}

// nprobe <= 128: one warp per query, the selection in registers.  The
// scores are binned linearly between their minimum and maximum (512 bins);
// only the bins up to the one where the count reaches nprobe can hold the
// nprobe smallest.  Those scores stream in chunks of up to 128 (also not
// above the current nprobe-th entry), each chunk sorted by (score, column)
// with a bitonic network over shuffles and merged with the sorted best.
constexpr int kSelBins = 512;

// One row (a warp): the np smallest of row[0, n) by (score, column) into
// out[0, np), -1 up to P.  h: kSelBins ints, sd / si: 128 entries, all of
// this warp.
__device__ void select128_row(const float* __restrict__ row, int n, int np, int P, int32_t* __restrict__ out,
                              int* h, float* sd, long long* si, int lane) {
    float mn = INFINITY, mx = -INFINITY;
    for (int i = lane; i < n; i += 32) {
        const float d = row[i];
        mn = fminf(mn, d);
        mx = fmaxf(mx, d);
    }
    for (int o = 16; o; o >>= 1) {
        mn = fminf(mn, __shfl_xor_sync(0xffffffffu, mn, o));
        mx = fmaxf(mx, __shfl_xor_sync(0xffffffffu, mx, o));
    }
    float scale = 0.f;
    int kbin = kSelBins;  // no bin filter (all scores equal, or not finite)
    if (mx > mn && isfinite(mx) && isfinite(mn)) {
        scale = (float)kSelBins / (mx - mn);
        
        for (int u = lane; u < kSelBins; u += 32) h[u] = 0;
        __syncwarp();
        for (int i = lane; i < n; i += 32) atomicAdd(&h[min(kSelBins - 1, (int)((row[i] - mn) * scale))], 1);
        __syncwarp();
        constexpr int PER = kSelBins / 32;
        int hs[PER], sum = 0;
#pragma unroll
        for (int u = 0; u < PER; ++u) {
            hs[u] = h[lane * PER + u];
            sum += hs[u];
        }
        int incl = sum;
        for (int o = 1; o < 32; o <<= 1) {
            const int y = __shfl_up_sync(0xffffffffu, incl, o);
            if (lane >= o) incl += y;
        }
        const int excl = incl - sum;
        const unsigned hit = __ballot_sync(0xffffffffu, excl < np && incl >= np);
        const int src = __ffs(hit) - 1;
        int kb = 0;
        if (lane == src) {
            int c = excl;
#pragma unroll
            for (int u = 0; u < PER; ++u) {
                c += hs[u];
                if (c >= np) { kb = lane * PER + u; break; }
            }
        }
        kbin = __shfl_sync(0xffffffffu, kb, src);
    }
    Ent32 a[4];
#pragma unroll
    for (int r = 0; r < 4; ++r) {
        a[r].d = INFINITY;
        a[r].id = INT_MAX;
    }
    int total = 0, i0 = 0;
    while (i0 < n) {
        Ent32 kth;
        kth.d = INFINITY;
        kth.id = INT_MAX;
        if (total >= np) kth = entry_at(a, np - 1);
        int m = 0;
        for (; i0 < n && m < 128; i0 += 32) {
            const int i = i0 + lane;
            Ent32 x;
            x.d = INFINITY;
            x.id = INT_MAX;
            bool keep = false;
            if (i < n) {
                x.d = row[i];
                x.id = i;
                keep = (kbin == kSelBins || min(kSelBins - 1, (int)((x.d - mn) * scale)) <= kbin) && !ent_less(kth, x);
            }
            const unsigned bal = __ballot_sync(0xffffffffu, keep);
            const int pos = m + __popc(bal & ((1u << lane) - 1u));
            if (keep && pos < 128) {
                sd[pos] = x.d;
                si[pos] = x.id;
            }
            const int got = __popc(bal);
            if (m + got > 128) {
                // the chunk is full: resume at the first kept lane not taken
                const int take = 128 - m;
                int seen = 0, resume = 32;
                for (int l2 = 0; l2 < 32; ++l2) {
                    if ((bal >> l2) & 1u) {
                        if (seen == take) { resume = l2; break; }
                        ++seen;
                    }
                }
                m = 128;
                i0 += resume;
                break;
            }
            m += got;
        }
        __syncwarp();
        if (m == 0) break;
        Ent32 c[4];
#pragma unroll
        for (int r = 0; r < 4; ++r) {
            const int e = r * 32 + lane;
            c[r].d = e < m ? sd[e] : INFINITY;
            c[r].id = e < m ? si[e] : INT_MAX;
        }
        __syncwarp();
        bitonic_sort128(c, lane);
#pragma unroll
        for (int r = 0; r < 4; ++r) {
            const Ent32 cr = shfl_ent(c[3 - r], 31 - lane);
            if (ent_less(cr, a[r])) a[r] = cr;
        }
#pragma unroll
        for (int j = 64; j > 0; j >>= 1) bitonic_level(a, j, lane, [](int) { return true; });
        total = min(128, total + m);
    }
#pragma unroll
    for (int r = 0; r < 4; ++r) {
        const int e = r * 32 + lane;
        if (e < P) out[e] = e < np ? (int32_t)a[r].id : -1;
    }
}

__global__ void __launch_bounds__(kSelWarps * 32) select128_kernel(const float* __restrict__ scores, int64_t B, int n,
                                                                  const int32_t* __restrict__ nprobe, int P,
                                                                  int32_t* __restrict__ probes,
                                                                  int32_t* __restrict__ status) {
    __shared__ int s_h[kSelWarps][kSelBins];
    __shared__ float s_d[kSelWarps][128];
    __shared__ long long s_i[kSelWarps][128];
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const int64_t b = (int64_t)blockIdx.x * kSelWarps + warp;
    if (b >= B) return;
    int32_t* out = probes + b * (int64_t)P;
    const int np = nprobe[b];
    if (np < 1 || np > P || np > n) {
        if (lane == 0 && status && np != 0) atomicCAS(status, 0, (int)DADE_EINVAL);
        for (int r = lane; r < P; r += 32) out[r] = -1;
        return;
    }
    select128_row(scores + b * (int64_t)n, n, np, P, out, s_h[warp], s_d[warp], s_i[warp], lane);
}

// nprobe <= 128 with per-tile minima from the centroid-distance kernel:
// tmin holds, per query and 128-centroid tile, the tile's 4 smallest
// distances (the same FP32 values as the score row).  Their np-th smallest,
// theta, is at least the row's np-th smallest (a subset's np-th smallest
// cannot be smaller), so the np smallest of the row are among the scores
// <= theta: one pass gathers those (with their columns), one bitonic sort
// orders them by (score, column).  When more than 128 scores are <= theta
// (ties) the row goes through select128_row instead.
__global__ void __launch_bounds__(kSelWarps * 32) select_thr_kernel(const float* __restrict__ scores,
                                                                   const float* __restrict__ tmin, int nct, int64_t B,
                                                                   int n, const int32_t* __restrict__ nprobe, int P,
                                                                   int32_t* __restrict__ probes,
                                                                   int32_t* __restrict__ status) {
    __shared__ int s_h[kSelWarps][kSelBins];
    __shared__ float s_d[kSelWarps][128];
    __shared__ long long s_i[kSelWarps][128];
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const int64_t b = (int64_t)blockIdx.x * kSelWarps + warp;
    if (b >= B) return;
    const float* row = scores + b * (int64_t)n;
    int32_t* out = probes + b * (int64_t)P;
    const int np = nprobe[b];
    if (np < 1 || np > P || np > n) {
        if (lane == 0 && status && np != 0) atomicCAS(status, 0, (int)DADE_EINVAL);
        for (int r = lane; r < P; r += 32) out[r] = -1;
        return;
    }
    // theta: the np-th smallest of the tiles' 4 smallest (4 * nct <= 128 values)
    // (non-negative FP32 distances order as their bit patterns: the
    // np-th smallest is the largest pattern with fewer than np below it,
    // found bit by bit from the top)
    const float* tm = tmin + b * (int64_t)nct * 4;
    uint32_t key[4];
#pragma unroll
    for (int r = 0; r < 4; ++r) {
        const int e = r * 32 + lane;
        key[r] = __float_as_uint(e < 4 * nct ? tm[e] : INFINITY);
    }
    uint32_t prefix = 0u;
#pragma unroll 1
    for (int bit = 30; bit >= 0; --bit) {
        const uint32_t cand = prefix | (1u << bit);
        int below = 0;
#pragma unroll
        for (int r = 0; r < 4; ++r) below += __popc(__ballot_sync(0xffffffffu, key[r] < cand));
        if (below < np) prefix = cand;
    }
    const float theta = __uint_as_float(prefix);
    bool fallback = !(theta < INFINITY);
    // the scores <= theta, with their columns, in column order
    int m = 0;
    if (!fallback) {
        const bool vec = (n & 3) == 0;
        for (int base = 0; base < n && !fallback; base += 128) {
            float x[4];
            const int c0 = base + lane * 4;
            if (vec && c0 + 3 < n) {
                const float4 f = __ldg(reinterpret_cast<const float4*>(row + c0));
                x[0] = f.x; x[1] = f.y; x[2] = f.z; x[3] = f.w;
            } else {
#pragma unroll
                for (int j = 0; j < 4; ++j) x[j] = c0 + j < n ? row[c0 + j] : INFINITY;
            }
            int c = 0;
#pragma unroll
            for (int j = 0; j < 4; ++j) c += (c0 + j < n && x[j] <= theta) ? 1 : 0;
            int incl = c;
#pragma unroll
            for (int o = 1; o < 32; o <<= 1) {
                const int y = __shfl_up_sync(0xffffffffu, incl, o);
                if (lane >= o) incl += y;
            }
            const int tot = __shfl_sync(0xffffffffu, incl, 31);
            if (m + tot > 128) {
                fallback = true;
                break;
            }
            int pos = m + incl - c;
#pragma unroll
            for (int j = 0; j < 4; ++j) {
                if (c0 + j < n && x[j] <= theta) {
                    s_d[warp][pos] = x[j];
                    s_i[warp][pos] = c0 + j;
                    ++pos;
                }
            }
            m += tot;
        }
    }
    __syncwarp();
    if (fallback) {
        select128_row(row, n, np, P, out, s_h[warp], s_d[warp], s_i[warp], lane);
        return;
    }
    KV a[4];
#pragma unroll
    for (int r = 0; r < 4; ++r) {
        const int e = r * 32 + lane;
        a[r].d = e < m ? s_d[warp][e] : INFINITY;
        a[r].c = e < m ? (int)s_i[warp][e] : INT_MAX;
    }
    kv_sort128(a, lane);
#pragma unroll
    for (int r = 0; r < 4; ++r) {
        const int e = r * 32 + lane;
        if (e < P) out[e] = e < np ? a[r].c : -1;
    }
}

}  // namespace

cudaError_t launch_select_probes(const float* scores, int64_t B, int n, const int32_t* nprobe,
                                 int P, int32_t* probes, int32_t* status, cudaStream_t st, const float* tmin) {
    if (B <= 0) return cudaSuccess;
    if (P > PMAX || P < 1) return cudaErrorInvalidValue;
    const int nct = (n + 127) / 128;
    if (tmin && P <= 128 && 4 * nct <= 128 && P <= 4 * nct) {
        select_thr_kernel<<<(unsigned)ceil_div(B, kSelWarps), kSelWarps * 32, 0, st>>>(scores, tmin, nct, B, n, nprobe,
                                                                                      P, probes, status);
        return cudaGetLastError();
    }
    if (P <= 128) {
        select128_kernel<<<(unsigned)ceil_div(B, kSelWarps), kSelWarps * 32, 0, st>>>(scores, B, n, nprobe, P, probes,
                                                                                     status);
        return cudaGetLastError();
    }
    int Pp = 2;
    while (Pp < P) Pp <<= 1;
    const int smem = kSelWarps * 2 * Pp * (int)sizeof(uint32_t);
    static int configured = 0;
    if (smem > configured) {
        cudaError_t e = cudaFuncSetAttribute(select_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, smem);
        if (e != cudaSuccess) return e;
        configured = smem;
    }
    select_kernel<<<(unsigned)ceil_div(B, kSelWarps), kSelWarps * 32, smem, st>>>(scores, B, n, nprobe, P, probes,
                                                                                  status);
    return cudaGetLastError();
}

}  // namespace dade
