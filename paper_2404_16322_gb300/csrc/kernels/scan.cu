// Refinement kernels around the wave scan: work units per wave (counting
// sort of (bucket, query) items, prefix scans, unit descriptors), the
// per-query top-K merge, the output, the replay that collects training
// samples for the correction, and the launchers.  The estimate-and-prune
// scan itself is the template in scan_steps.cuh; this file instantiates its
// learned-table and full-scan variants (scan_res.cu the RES ones).
//
// Method (arXiv 2404.16322): a candidate's distance is accumulated Delta_d
// rotated dimensions at a time (the loop of Algorithm 2); after each step the
// learned test m1_s * dis' + beta_s > tau prunes it (Section V-A; one
// classifier per step, Section V-B "Incremental Correction"); survivors get
// the exact distance and join the result queue whose largest entry is tau
// (Section I).  tau is frozen per wave of probe ranks so that all
// (bucket, query) pairs of a wave run in parallel.
#include "scan_steps.cuh"
#include "warp_select.cuh"

namespace dade {
namespace {


// ------------------------------------------------------------ merge
// One warp per query.  The wave's candidates are streamed in chunks of up to
// kMergeChunk, each chunk sorted (warp bitonic sort in shared memory) and
// merged with the sorted top-K by rank: an element's place is its index plus
// the number of elements of the other list that precede it in (distance, id)
// order.  When there are many candidates (a wave whose tau was +inf appends
// all of them), a warp radix select first finds the K-th smallest distance v
// among them and only candidates with distance <= v are merged: at least K of
// the candidates are <= v, so no other candidate can enter the top-K.
constexpr int kMergeWarps = 8;
constexpr int kMergeChunk = 256;

__device__ __forceinline__ bool pair_less(float da, long long ia, float db, long long ib) {
    return da < db || (da == db && ia < ib);
}

// number of entries of the sorted list (d, id)[0, n) that precede (x, xi)
__device__ __forceinline__ int count_before(const float* d, const long long* id, int n, float x, long long xi) {
    int lo = 0, hi = n;
    while (lo < hi) {
        int mid = (lo + hi) >> 1;
        if (pair_less(d[mid], id[mid], x, xi)) lo = mid + 1; else hi = mid;
    }
    return lo;
}

struct CandKeys {
    const float* d;
    __device__ uint32_t operator()(int i) const { return __float_as_uint(d[i]); }
};

__device__ __forceinline__ void warp_sort(float* bd, long long* bi, int M, int lane) {
    for (int size = 2; size <= M; size <<= 1) {
        for (int stride = size >> 1; stride > 0; stride >>= 1) {
            for (int i = lane; i < M; i += 32) {
                const int j = i ^ stride;
                if (j > i) {
                    const bool up = (i & size) == 0;
                    const bool sw = up ? pair_less(bd[j], bi[j], bd[i], bi[i])
                                       : pair_less(bd[i], bi[i], bd[j], bi[j]);
                    if (sw) {
                        float x = bd[i];
                        bd[i] = bd[j];
                        bd[j] = x;
                        long long y = bi[i];
                        bi[i] = bi[j];
                        bi[j] = y;
                    }
                }
            }
            __syncwarp();
        }
    }
}

// Sort the chunk b[0, m) and merge it into a[0, cur) keeping the best
// min(K, cur + m); returns the new count (result in a).
__device__ int merge_chunk(float* ad, long long* ai, int cur, float* bd, long long* bi, int m, float* od,
                           long long* oi, int K, int lane) {
    int M = 1;
    while (M < m) M <<= 1;
    for (int i = m + lane; i < M; i += 32) {
        bd[i] = INFINITY;
        bi[i] = LLONG_MAX;
    }
    __syncwarp();
    warp_sort(bd, bi, M, lane);
    const int nout = min(K, cur + m);
    for (int i = lane; i < cur; i += 32) {
        const int r = i + count_before(bd, bi, m, ad[i], ai[i]);
        if (r < nout) {
            od[r] = ad[i];
            oi[r] = ai[i];
        }
    }
    for (int i = lane; i < m; i += 32) {
        const int r = i + count_before(ad, ai, cur, bd[i], bi[i]);
        if (r < nout) {
            od[r] = bd[i];
            oi[r] = bi[i];
        }
    }
    __syncwarp();
    for (int i = lane; i < nout; i += 32) {
        ad[i] = od[i];
        ai[i] = oi[i];
    }
    __syncwarp();
    return nout;
}

__global__ void __launch_bounds__(kMergeWarps * 32) merge_kernel(IndexView ix, WaveView wv, int w) {
    extern __shared__ __align__(16) unsigned char msmem[];
    __shared__ int s_hist[kMergeWarps][256];
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const int64_t q = (int64_t)blockIdx.x * kMergeWarps + warp;
    if (q >= wv.B) return;
    const int cap_k = wv.Kmax;
    const int region = 2 * cap_k + kMergeChunk;  // top list, chunk, output
    float* rd = reinterpret_cast<float*>(msmem) + (size_t)warp * region;
    long long* ri = reinterpret_cast<long long*>(msmem + sizeof(float) * (size_t)kMergeWarps * region) +
                    (size_t)warp * region;
    float* ad = rd;
    long long* ai = ri;
    float* bd = rd + cap_k;
    long long* bi = ri + cap_k;
    float* od = rd + cap_k + kMergeChunk;
    long long* oi = ri + cap_k + kMergeChunk;

    const int64_t* co = wv.cand_off + (int64_t)w * (wv.B + 1);
    const int64_t off = co[q], cap = co[q + 1] - off;
    const int cnt = (int)((int64_t)wv.cand_cnt[q] < cap ? (int64_t)wv.cand_cnt[q] : cap);
    const int K = wv.K[q];
    if (cnt == 0 || K < 1 || K > wv.Kmax) {
        if (lane == 0) wv.cand_cnt[q] = 0;
        return;
    }
    const float* cd = wv.cand_d + off;
    const int32_t* cp = wv.cand_pos + off;
    float* td = wv.top_d + q * wv.Kmax;
    int64_t* ti = wv.top_id + q * wv.Kmax;
    int cur = wv.top_n[q];
    for (int i = lane; i < cur; i += 32) {
        ad[i] = td[i];
        ai[i] = ti[i];
    }
    // candidates above the K-th smallest of this wave cannot enter the top-K
    const uint32_t thr = cnt > max(K, kMergeChunk) ? warp_kth_key(CandKeys{cd}, cnt, K, s_hist[warp], lane) : 0xffffffffu;
    int m = 0;  // filled part of the chunk
    for (int base = 0; base < cnt; base += 32) {
        const int i = base + lane;
        const bool keep = i < cnt && __float_as_uint(cd[i]) <= thr;
        const unsigned bal = __ballot_sync(0xffffffffu, keep);
        if (keep) {
            const int pos = m + __popc(bal & lanemask_lt());
            bd[pos] = cd[i];
            bi[pos] = ix.ids[cp[i]];
        }
        m += __popc(bal);
        __syncwarp();
        if (m > kMergeChunk - 32) {
            cur = merge_chunk(ad, ai, cur, bd, bi, m, od, oi, K, lane);
            m = 0;
        }
    }
    if (m > 0) cur = merge_chunk(ad, ai, cur, bd, bi, m, od, oi, K, lane);
    for (int i = lane; i < cur; i += 32) {
        td[i] = ad[i];
        ti[i] = ai[i];
    }
    if (lane == 0) {
        wv.top_n[q] = cur;
        wv.tau_run[q] = cur == K ? ad[K - 1] : INFINITY;
        wv.cand_cnt[q] = 0;
    }
}

// ------------------------------------------------------------ merge, K <= 128
// The top-K of a query (K <= 128) kept in registers: 128 entries per warp,
// entry e = 32 r + lane in slot r of lane `lane`, ordered by (distance, id).
// New candidates are streamed in chunks of up to 128 -- only those that can
// still enter, i.e. not above the current K-th entry -- each chunk sorted by
// a bitonic network (shuffles across lanes, swaps across slots) and merged
// with the top by taking the elementwise minimum with the reversed chunk
// (a bitonic sequence holding the 128 smallest) and sorting that.
constexpr int kM128Warps = 8;

constexpr int kM128Bins = 512;

// E: Ent (64-bit ids) or Ent32 (every id of the index fits in 31 bits).
template <class E>
__global__ void __launch_bounds__(kM128Warps * 32) merge128_kernel(IndexView ix, WaveView wv, int w) {
    __shared__ float s_d[kM128Warps][128];
    __shared__ long long s_i[kM128Warps][128];
    __shared__ int s_h[kM128Warps][kM128Bins];
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const int64_t q = (int64_t)blockIdx.x * kM128Warps + warp;
    if (q >= wv.B) return;
    const int64_t* co = wv.cand_off + (int64_t)w * (wv.B + 1);
    const int64_t off = co[q], cap = co[q + 1] - off;
    const int cnt = (int)((int64_t)wv.cand_cnt[q] < cap ? (int64_t)wv.cand_cnt[q] : cap);
    const int K = wv.K[q];
    if (cnt == 0 || K < 1 || K > wv.Kmax) {
        if (lane == 0) wv.cand_cnt[q] = 0;
        return;
    }
    const float* cd = wv.cand_d + off;
    const int32_t* cp = wv.cand_pos + off;
    float* td = wv.top_d + q * wv.Kmax;
    int64_t* ti = wv.top_id + q * wv.Kmax;
    const int cur = wv.top_n[q];
    E a[4];
#pragma unroll
    for (int r = 0; r < 4; ++r) {
        const int e = r * 32 + lane;
        a[r].d = e < cur ? td[e] : INFINITY;
        a[r].id = e < cur ? (decltype(a[r].id))ti[e] : ent_pad<E>().id;
    }
    int total = cur;  // entries held (up to 128)
    // Many new candidates: only the K smallest of them can enter.  Their
    // distances are binned linearly between their minimum and maximum; the
    // bins up to the one where the count reaches K hold them all, and only
    // those candidates are streamed below (bin(d) is monotone in d).
    float lo = 0.f, scale = 0.f;
    int kbin = kM128Bins;  // no bin filter
    if (cnt > K) {
        float mn = INFINITY, mx = -INFINITY;
        for (int i = lane; i < cnt; i += 32) {
            const float d = cd[i];
            mn = fminf(mn, d);
            mx = fmaxf(mx, d);
        }
        for (int o = 16; o; o >>= 1) {
            mn = fminf(mn, __shfl_xor_sync(0xffffffffu, mn, o));
            mx = fmaxf(mx, __shfl_xor_sync(0xffffffffu, mx, o));
        }
        if (mx > mn && isfinite(mx)) {
            lo = mn;
            scale = (float)kM128Bins / (mx - mn);
            int* h = s_h[warp];
            for (int b = lane; b < kM128Bins; b += 32) h[b] = 0;
            __syncwarp();
            for (int i = lane; i < cnt; i += 32)
                atomicAdd(&h[min(kM128Bins - 1, (int)((cd[i] - lo) * scale))], 1);
            __syncwarp();
            constexpr int PER = kM128Bins / 32;  // bins per lane, contiguous
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
            const unsigned hit = __ballot_sync(0xffffffffu, excl < K && incl >= K);
            const int src = __ffs(hit) - 1;
            int kb = 0;
            if (lane == src) {
                int c = excl;
#pragma unroll
                for (int u = 0; u < PER; ++u) {
                    c += hs[u];
                    if (c >= K) { kb = lane * PER + u; break; }
                }
            }
            kbin = __shfl_sync(0xffffffffu, kb, src);
        }
    }
    int i0 = 0;
    while (i0 < cnt) {
        // the current K-th entry bounds what can still enter
        E kth = ent_pad<E>();
        if (total >= K) kth = entry_at(a, K - 1);
        // gather up to 128 candidates that are not above the K-th entry's
        // distance (four loads in flight; their ids are looked up after)
        int m = 0;
        while (i0 < cnt && m < 128) {
            float xv[4];
#pragma unroll
            for (int u = 0; u < 4; ++u) {
                const int i = i0 + 32 * u + lane;
                xv[u] = i < cnt ? cd[i] : INFINITY;
            }
            bool stop = false;
#pragma unroll
            for (int u = 0; u < 4; ++u) {
                if (stop) break;
                const int i = i0 + 32 * u + lane;
                const bool keep = i < cnt && xv[u] <= kth.d &&
                                  (kbin == kM128Bins || min(kM128Bins - 1, (int)((xv[u] - lo) * scale)) <= kbin);
                const unsigned bal = __ballot_sync(0xffffffffu, keep);
                const int pos = m + __popc(bal & lanemask_lt());
                if (keep && pos < 128) {
                    s_d[warp][pos] = xv[u];
                    s_i[warp][pos] = i;  // the candidate's index; its id below
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
                    i0 += 32 * u + resume;
                    stop = true;
                } else {
                    m += got;
                }
            }
            if (!stop) i0 += 128;
        }
        __syncwarp();
        if (m == 0) break;
        {  // ids of the gathered candidates, four independent lookups per lane
            int slot[4];
#pragma unroll
            for (int r = 0; r < 4; ++r) {
                const int e = r * 32 + lane;
                slot[r] = e < m ? cp[(int)s_i[warp][e]] : 0;
            }
#pragma unroll
            for (int r = 0; r < 4; ++r) {
                const int e = r * 32 + lane;
                if (e < m) s_i[warp][e] = (long long)ix.ids[slot[r]];
            }
        }
        __syncwarp();
        E b[4];
#pragma unroll
        for (int r = 0; r < 4; ++r) {
            const int e = r * 32 + lane;
            b[r].d = e < m ? s_d[warp][e] : INFINITY;
            b[r].id = e < m ? (decltype(b[r].id))s_i[warp][e] : ent_pad<E>().id;
        }
        __syncwarp();
        bitonic_sort128(b, lane);
        if (total == 0) {
            // nothing kept yet: the sorted chunk is the list
#pragma unroll
            for (int r = 0; r < 4; ++r) a[r] = b[r];
        } else {
            // a ascending, b reversed descending: the elementwise minimum is a
            // bitonic sequence of the 128 smallest of both
#pragma unroll
            for (int r = 0; r < 4; ++r) {
                const E br = shfl_ent(b[3 - r], 31 - lane);
                if (ent_less(br, a[r])) a[r] = br;
            }
#pragma unroll
            for (int j = 64; j > 0; j >>= 1) bitonic_level(a, j, lane, [](int) { return true; });
        }
        total = min(128, total + m);
    }
    const int n_out = min(K, total);
#pragma unroll
    for (int r = 0; r < 4; ++r) {
        const int e = r * 32 + lane;
        if (e < n_out) {
            td[e] = a[r].d;
            ti[e] = a[r].id;
        }
    }
    if (lane == 0) {
        wv.top_n[q] = n_out;
        wv.cand_cnt[q] = 0;
    }
    const E kth = entry_at(a, K - 1);
    if (lane == 0) wv.tau_run[q] = n_out == K ? kth.d : INFINITY;
}

// One warp per query: its K results (padding -1 / +inf up to its slots).
__global__ void output_kernel(WaveView wv, int64_t* ids, float* dists, const int64_t* offsets) {
    const int64_t q = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const int lane = threadIdx.x & 31;
    if (q >= wv.B) return;
    const int K = wv.K[q];
    const int64_t off = offsets ? offsets[q] : q * wv.Kmax;
    const int kk = offsets ? (int)(offsets[q + 1] - offsets[q]) : wv.Kmax;
    const int n = (K >= 1 && K <= wv.Kmax) ? wv.top_n[q] : 0;
    for (int k = lane; k < kk; k += 32) {
        bool v = k < n && k < K;
        ids[off + k] = v ? wv.top_id[q * wv.Kmax + k] : -1;
        dists[off + k] = v ? wv.top_d[q * wv.Kmax + k] : INFINITY;
    }
}

// ------------------------------------------------------------ work units
// One warp per query (lane = probe rank, 32 at a time): per (pass, bucket)
// the number of queries probing it, and per (pass, query) the query's
// candidate count (lanes of the same pass are contiguous: their sizes are
// summed with one warp reduction and added by the first of them).
__global__ void count_kernel(IndexView ix, WaveView wv) {
    const int64_t b = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const int lane = threadIdx.x & 31;
    if (b >= wv.B) return;
    const int np = wv.nprobe[b];
    const int K = wv.K[b];
    if (np < 1 || np > wv.P || K < 1 || K > wv.Kmax) {
        // nprobe = 0 or K = 0 marks an inactive query slot (no work, padded
        // output); anything else out of range is an error
        if (lane == 0 && !((np == 0 && K >= 0 && K <= wv.Kmax) || (K == 0 && np >= 0 && np <= wv.P)))
            atomicCAS(wv.status, 0, (int)DADE_EINVAL);
        return;
    }
    for (int r0 = 0; r0 < np; r0 += 32) {
        const int r = r0 + lane;
        int wr = -1;
        uint32_t size = 0;
        if (r < np) {
            const int l = wv.probes[b * wv.P + r];
            if (l < 0 || l >= ix.nlist) {
                atomicCAS(wv.status, 0, (int)DADE_EINVAL);
            } else {
                wr = pass_of_rank(wv, r);
                atomicAdd(&wv.cnt_wl[wr * ix.nlist + l], 1);
                size = (uint32_t)ix.list_size[l];
            }
        }
        const unsigned grp = __match_any_sync(0xffffffffu, wr);
        const uint32_t tot = __reduce_add_sync(grp, size);
        if (wr >= 0 && lane == __ffs(grp) - 1) wv.cand_off[(int64_t)wr * (wv.B + 1) + b] += tot;
        __syncwarp();  // the next 32 ranks may add to the same pass's count from another lane
    }
}

// One warp per query: each probed (pass, bucket) list gets the query once.
__global__ void scatter_kernel(IndexView ix, WaveView wv) {
    const int64_t b = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const int lane = threadIdx.x & 31;
    if (b >= wv.B) return;
    const int np = wv.nprobe[b];
    const int K = wv.K[b];
    if (np < 1 || np > wv.P || K < 1 || K > wv.Kmax) return;
    for (int r = lane; r < np; r += 32) {
        const int l = wv.probes[b * wv.P + r];
        if (l < 0 || l >= ix.nlist) continue;
        const int wr = pass_of_rank(wv, r);
        const int key = wr * ix.nlist + l;
        const int pos = atomicAdd(&wv.fill_wl[key], 1);
        wv.items[wv.off_wl[key] + pos] = (int32_t)b;
    }
}

// Exclusive scan of one segment per CTA: out[seg*ostride + i] for i < len
// and the total at i = len.  In-place use is safe (each chunk is read
// before any of it is written).
template <class Load, class T>
__global__ void __launch_bounds__(1024) seg_scan_kernel(Load load, T* out, int64_t len, int64_t ostride) {
    __shared__ T warp_tot[32];
    __shared__ T s_carry;
    const int seg = blockIdx.x, tid = threadIdx.x, lane = tid & 31, wid = tid >> 5;
    if (tid == 0) s_carry = 0;
    __syncthreads();
    for (int64_t base = 0; base < len; base += 4096) {
        T v[4], sum = 0;
#pragma unroll
        for (int u = 0; u < 4; ++u) {
            int64_t i = base + tid * 4 + u;
            v[u] = i < len ? load(seg, i) : (T)0;
            sum += v[u];
        }
        T incl = sum;
#pragma unroll
        for (int off = 1; off < 32; off <<= 1) {
            T o = __shfl_up_sync(0xffffffffu, incl, off);
            if (lane >= off) incl += o;
        }
        if (lane == 31) warp_tot[wid] = incl;
        __syncthreads();
        if (wid == 0) {
            T x = warp_tot[lane];
            T xi = x;
#pragma unroll
            for (int off = 1; off < 32; off <<= 1) {
                T o = __shfl_up_sync(0xffffffffu, xi, off);
                if (lane >= off) xi += o;
            }
            warp_tot[lane] = xi - x;  // exclusive warp offsets
        }
        __syncthreads();
        T run = s_carry + warp_tot[wid] + incl - sum;
#pragma unroll
        for (int u = 0; u < 4; ++u) {
            int64_t i = base + tid * 4 + u;
            if (i < len) out[seg * ostride + i] = run;
            run += v[u];
        }
        __syncthreads();
        if (tid == 1023) s_carry = run;
        __syncthreads();
    }
    if (tid == 0) out[seg * ostride + len] = s_carry;
}

struct LoadI32 {
    const int32_t* p;
    __device__ int32_t operator()(int, int64_t i) const { return p[i]; }
};
struct LoadUnits {
    const int32_t* cnt;
    const int32_t* size;
    int nlist;
    int32_t qgroup[kMaxPasses];
    __device__ int32_t operator()(int seg, int64_t l) const {
        int c = cnt[(int64_t)seg * nlist + l];
        int s = size[l];
        const int qg = qgroup[seg];
        return c > 0 ? ((c + qg - 1) / qg) * ((s + kT - 1) / kT) : 0;
    }
};
struct LoadCap {
    const int64_t* p;
    int64_t stride;
    __device__ int64_t operator()(int seg, int64_t i) const { return p[seg * stride + i]; }
};

// One thread per (wave, bucket): write the descriptors of the bucket's units
// in this wave, in the order of unit_off (group-major, then tile).  The cnt
// queries probing the bucket form ceil(cnt / qgroup) groups of balanced size.
__global__ void expand_units_kernel(IndexView ix, WaveView wv) {
    const int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (e >= (int64_t)wv.n_waves * ix.nlist) return;
    const int w = (int)(e / ix.nlist), l = (int)(e % ix.nlist);
    const int cnt = wv.cnt_wl[e];
    if (cnt == 0) return;
    const int nl = ix.list_size[l];
    const int ntile = (nl + kT - 1) / kT;
    const int qg = wv.qgroup[w];
    const int ng = (cnt + qg - 1) / qg;
    const int base = cnt / ng, rem = cnt % ng;
    int4* out = wv.units + wv.ubase[w] + wv.unit_off[(int64_t)w * (ix.nlist + 1) + l];
    const int item0 = wv.off_wl[e];
    for (int g = 0; g < ng; ++g) {
        const int nq = base + (g < rem ? 1 : 0);
        const int first = item0 + g * base + min(g, rem);
        for (int t = 0; t < ntile; ++t) {
            const int nt = min(kT, nl - t * kT);
            out[g * ntile + t] = make_int4(l, t, first, (nq << 16) | nt);
        }
    }
}

__global__ void prepare_queries_kernel(const float* Q, int64_t B, int32_t D, int32_t Dpad, float* qpad) {
    int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= B * Dpad) return;
    int64_t b = i / Dpad;
    int d = (int)(i % Dpad);
    qpad[i] = d < D ? Q[b * D + d] : 0.f;
}

__global__ void fill_kernel(float* p, int64_t n, float v) {
    int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i < n) p[i] = v;
}

// ------------------------------------------------------------ collect
// Replay of a wave with pruning off, emitting labelled training samples.
template <int DT>
__global__ void __launch_bounds__(kScanThreads) collect_kernel(IndexView ix, WaveView wv, int w, int dd,
                                                               int S, CollectArgs ca, int64_t qoff) {
    using E = typename Elem<DT>::T;
    __shared__ int s_unit;
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    const int total = wv.unit_off[(int64_t)w * (ix.nlist + 1) + ix.nlist];
    const int nblk = dd / kBlock;
    for (;;) {
        if (tid == 0) s_unit = atomicAdd(&wv.work[wv.n_waves + w], 1);
        __syncthreads();
        const int u = s_unit;
        if (u >= total) break;
        const Unit un = unpack_unit(wv.units[wv.ubase[w] + u]);
        const int64_t slot_l = ix.list_slot[un.l];
        const int64_t npad = ix.list_slot[un.l + 1] - slot_l;
        const int64_t ebase = slot_l * ix.Dpad;
        for (int g = warp; g < un.nq; g += kWarps) {
            const int q = wv.items[un.item + g];
            const float tau = wv.tau[q];
            if (isinf(tau) && !ca.keep_all) continue;
            const int K = ca.topk_ids ? wv.K[q] : 0;
            const float* qp = wv.qpad + (int64_t)q * ix.Dpad;
            const float* qr = wv.qrot + (int64_t)q * ix.Dpad;
            for (int base = 0; base < un.nt; base += 32) {
                const int c = base + lane;
                const bool valid = c < un.nt;
                bool lab0 = false, lab1 = false;
                int64_t id = -1;
                if (valid) {
                    const int64_t pos = (int64_t)un.t * kT + c;
                    const float d = exact_distance(ix.orig + ebase + pos * kBlock, npad, qp, ix.nb);
                    id = ix.ids[slot_l + pos];
                    for (int k = 0; k < K; ++k) lab0 |= ca.topk_ids[(int64_t)q * ca.topk_stride + k] == id;
                    lab1 = !lab0 && d > tau;
                }
                if (ca.pass == 0) {
                    unsigned bal = __ballot_sync(0xffffffffu, lab1);
                    if (lane == 0 && bal) atomicAdd(ca.n_label1, (unsigned long long)__popc(bal));
                    continue;
                }
                bool emit = lab0 || (ca.keep_all && valid);
                if (lab1 && !emit) {
                    // SplitMix64-derived uniform of (seed, query, id)
                    uint64_t key = ((uint64_t)(qoff + q) << 32) ^ (uint64_t)id;
                    auto mix = [](uint64_t z) {
                        z += 0x9E3779B97F4A7C15ull;
                        z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
                        z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
                        return z ^ (z >> 31);
                    };
                    uint64_t z = mix(ca.seed ^ mix(key));
                    double uu = (double)(z >> 11) * 0x1.0p-53;
                    emit = uu < ca.keep_rate;
                }
                if (!emit) continue;
                unsigned long long row = atomicAdd(ca.n_rows, 1ull);
                if ((int64_t)row >= ca.row_cap) continue;
                const int64_t pos = (int64_t)un.t * kT + c;
                if (ca.query) ca.query[row] = qoff + q;
                if (ca.id) ca.id[row] = id;
                if (ca.pq_m > 0) {
                    // OPQ-L rows: the asymmetric distance and the quantisation error
                    const int64_t slot = slot_l + pos;
                    const float* t = ca.pq_lut + (int64_t)q * ca.pq_m * 256;
                    float dis = 0.f;
                    for (int j = 0; j < ca.pq_m; ++j) dis += t[j * 256 + ca.pq_codes[(int64_t)j * ix.total_slots + slot]];
                    ca.partials[(int64_t)row * 2] = dis;
                    ca.partials[(int64_t)row * 2 + 1] = ca.pq_err[slot];
                    ca.tau[row] = tau;
                    ca.label[row] = lab0 ? 0 : lab1 ? 1 : 2;
                    continue;
                }
                const E* xs = reinterpret_cast<const E*>(ix.slab) + ebase + pos * kBlock;
                float p = 0.f;
                for (int k = 0; k + 1 < S; ++k) {
                    const int b0 = k * nblk, nbk = min(nblk, ix.nb - b0);
                    for (int bb = 0; bb < nbk; ++bb) {
                        float x[8], qv[8], sc[8];
                        if (DT == DADE_SLAB_FP8E4M3) load_q8(ix.scale + (b0 + bb) * kBlock, sc);
                        load8(xs + (int64_t)(b0 + bb) * npad * kBlock, sc, x);
                        load_q8(qr + (b0 + bb) * kBlock, qv);
                        p += block_sq(qv, x);
                    }
                    ca.partials[(int64_t)row * (S - 1) + k] = p;
                }
                if (ca.tau) ca.tau[row] = tau;
                if (ca.label) ca.label[row] = lab0 ? 0 : lab1 ? 1 : 2;
            }
        }
        __syncthreads();
    }
}


}  // namespace

cudaError_t launch_prepare_queries(const float* Q, int64_t B, int32_t D, int32_t Dpad, float* qpad,
                                   cudaStream_t st) {
    int64_t n = B * Dpad;
    if (n == 0) return cudaSuccess;
    prepare_queries_kernel<<<(unsigned)ceil_div(n, 256), 256, 0, st>>>(Q, B, D, Dpad, qpad);
    return cudaGetLastError();
}

cudaError_t launch_fill(float* p, int64_t n, float v, cudaStream_t st) {
    if (n == 0) return cudaSuccess;
    fill_kernel<<<(unsigned)ceil_div(n, 256), 256, 0, st>>>(p, n, v);
    return cudaGetLastError();
}

cudaError_t launch_build_units(const IndexView& ix, const WaveView& wv, cudaStream_t st) {
    const unsigned gb = (unsigned)ceil_div(wv.B * 32, 256);  // a warp per query
    count_kernel<<<gb, 256, 0, st>>>(ix, wv);
    const int64_t nwl = (int64_t)wv.n_waves * ix.nlist;
    seg_scan_kernel<<<1, 1024, 0, st>>>(LoadI32{wv.cnt_wl}, wv.off_wl, nwl, 0);
    LoadUnits lu{wv.cnt_wl, ix.list_size, ix.nlist, {}};
    for (int w = 0; w < kMaxPasses; ++w) lu.qgroup[w] = wv.qgroup[w];
    seg_scan_kernel<<<wv.n_waves, 1024, 0, st>>>(lu, wv.unit_off, (int64_t)ix.nlist, (int64_t)ix.nlist + 1);
    seg_scan_kernel<<<wv.n_waves, 1024, 0, st>>>(LoadCap{wv.cand_off, wv.B + 1}, wv.cand_off, wv.B,
                                                 wv.B + 1);
    scatter_kernel<<<gb, 256, 0, st>>>(ix, wv);
    expand_units_kernel<<<(unsigned)ceil_div(nwl, 128), 128, 0, st>>>(ix, wv);
    return cudaGetLastError();
}

cudaError_t launch_wave_scan(const IndexView& ix, const WaveView& wv, int w, bool full,
                             int delta_d, const float* m1, const float* beta, int S,
                             cudaStream_t st) {
    if (full) return launch_scan_t<DADE_SLAB_F32, 4, true, false, false>(ix, wv, w, m1, beta, S, st);
    if (wv.est) return launch_wave_scan_res(ix, wv, w, delta_d, S, st);
#define DADE_SCAN_CASE(DT, NB)                                                                      \
    if (ix.dtype == DT && delta_d == NB * kBlock)                                                   \
        return wv.final_test ? launch_scan_t<DT, NB, false, true, false>(ix, wv, w, m1, beta, S, st)   \
                             : launch_scan_t<DT, NB, false, false, false>(ix, wv, w, m1, beta, S, st);
    DADE_SCAN_CASE(DADE_SLAB_F32, 1)
    DADE_SCAN_CASE(DADE_SLAB_F32, 2)
    DADE_SCAN_CASE(DADE_SLAB_F32, 4)
    DADE_SCAN_CASE(DADE_SLAB_BF16, 1)
    DADE_SCAN_CASE(DADE_SLAB_BF16, 2)
    DADE_SCAN_CASE(DADE_SLAB_BF16, 4)
    DADE_SCAN_CASE(DADE_SLAB_FP8E4M3, 1)
    DADE_SCAN_CASE(DADE_SLAB_FP8E4M3, 2)
    DADE_SCAN_CASE(DADE_SLAB_FP8E4M3, 4)
#undef DADE_SCAN_CASE
    return cudaErrorInvalidValue;
}

cudaError_t launch_merge(const IndexView& ix, const WaveView& wv, int w, cudaStream_t st) {
    if (wv.B == 0) return cudaSuccess;
    if (wv.Kmax <= 128) {
        if (ix.ids32)
            merge128_kernel<Ent32><<<(unsigned)ceil_div(wv.B, kM128Warps), kM128Warps * 32, 0, st>>>(ix, wv, w);
        else
            merge128_kernel<Ent><<<(unsigned)ceil_div(wv.B, kM128Warps), kM128Warps * 32, 0, st>>>(ix, wv, w);
        return cudaGetLastError();
    }
    const int smem = kMergeWarps * (2 * wv.Kmax + kMergeChunk) * (int)(sizeof(float) + sizeof(long long));
    static int configured = 0;
    if (smem > configured) {
        cudaError_t e = cudaFuncSetAttribute(merge_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, smem);
        if (e != cudaSuccess) return e;
        configured = smem;
    }
    merge_kernel<<<(unsigned)ceil_div(wv.B, kMergeWarps), kMergeWarps * 32, smem, st>>>(ix, wv, w);
    return cudaGetLastError();
}

cudaError_t launch_output(const WaveView& wv, int64_t* ids, float* dists, const int64_t* offsets,
                          cudaStream_t st) {
    if (wv.B == 0) return cudaSuccess;
    output_kernel<<<(unsigned)ceil_div(wv.B * 32, 256), 256, 0, st>>>(wv, ids, dists, offsets);
    return cudaGetLastError();
}

cudaError_t launch_collect(const IndexView& ix, const WaveView& wv, int w, int delta_d, int S,
                           const CollectArgs& ca, int64_t qoff, cudaStream_t st) {
    int dev = 0, sms = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    const unsigned grid = (unsigned)sms * 4;
    if (ix.dtype == DADE_SLAB_F32)
        collect_kernel<DADE_SLAB_F32><<<grid, kScanThreads, 0, st>>>(ix, wv, w, delta_d, S, ca, qoff);
    else if (ix.dtype == DADE_SLAB_BF16)
        collect_kernel<DADE_SLAB_BF16><<<grid, kScanThreads, 0, st>>>(ix, wv, w, delta_d, S, ca, qoff);
    else
        collect_kernel<DADE_SLAB_FP8E4M3><<<grid, kScanThreads, 0, st>>>(ix, wv, w, delta_d, S, ca, qoff);
    return cudaGetLastError();
}

}  // namespace dade

