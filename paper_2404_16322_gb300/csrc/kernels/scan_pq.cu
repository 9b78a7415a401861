// OPQ-L (arXiv 2404.16322, Section V-B "Approximate Distances"): the
// approximate distance is OPQ's asymmetric distance dis' = sum_j
// lut_q[j][code_j] (the query exact, the vector its product-quantised
// reconstruction), and the learned correction has a third feature, the
// vector's quantisation error e: a candidate is pruned iff
// m1 dis' + m3 e + beta > tau, before its exact distance.  There is one
// test (the paper notes that the quantised distance cannot be refined
// incrementally).
//
// The product quantiser is OPQ's parametric form on the index's PCA basis:
// subspace j holds rotated dims perm[j*ds .. (j+1)*ds), 256 centroids each.
//
// Kernels: encoding of every slot's stored vector (codes and e), the
// per-query tables, and the wave scan.  The scan is query-major: a work item
// is (query, run of up to rpi consecutive probe ranks of the wave, rpi chosen
// so that there are a few items per CTA); a
// CTA stages the query's table (m x 256 floats) in shared memory and walks
// the candidates of the item's buckets, kPqThreads at a time; codes are
// stored subspace-major so that a chunk's code for one subspace is one
// coalesced read.
#include "scan_steps.cuh"

namespace dade {
namespace {

// FP32 value of element (slot, dim) of the blocked slab, dequantised.
__device__ __forceinline__ float slab_value(const void* slab, int dtype, const float* scale, int64_t s0, int64_t npad,
                                            int64_t i, int32_t Dpad, int d) {
    const int64_t e = s0 * Dpad + ((int64_t)(d / kBlock) * npad + i) * kBlock + (d % kBlock);
    if (dtype == DADE_SLAB_F32) return static_cast<const float*>(slab)[e];
    if (dtype == DADE_SLAB_BF16) return __bfloat162float(static_cast<const __nv_bfloat16*>(slab)[e]);
    const __nv_fp8_storage_t u = static_cast<const __nv_fp8_storage_t*>(slab)[e];
    return __half2float(__half(__nv_cvt_fp8_to_halfraw(u, __NV_E4M3))) * scale[d];
}

// One thread per slot: the nearest centroid of every subspace (the lower
// index on a tie) and e = sqrt(sum of the nearest squared distances).
// Padding slots get code 0 and e = 0.
__global__ void pq_encode_kernel(const void* __restrict__ slab, int dtype, const float* __restrict__ scale,
                                 const int64_t* __restrict__ list_slot, int nlist, int64_t total_slots, int32_t Dpad,
                                 const int32_t* __restrict__ perm, const float* __restrict__ cb, int m, int ds,
                                 uint8_t* __restrict__ codes, float* __restrict__ err) {
    const int64_t slot = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (slot >= total_slots) return;
    int lo = 0, hi = nlist - 1;
    while (lo < hi) {
        const int mid = (lo + hi + 1) >> 1;
        if (list_slot[mid] <= slot) lo = mid; else hi = mid - 1;
    }
    const int64_t s0 = list_slot[lo], npad = list_slot[lo + 1] - s0, i = slot - s0;
    float e2 = 0.f;
    constexpr int kMaxDs = 64;
    float x[kMaxDs];
    for (int j = 0; j < m; ++j) {
        for (int t = 0; t < ds; ++t) x[t] = slab_value(slab, dtype, scale, s0, npad, i, Dpad, perm[j * ds + t]);
        float best = INFINITY;
        int arg = 0;
        const float* c = cb + (int64_t)j * 256 * ds;
        for (int k = 0; k < 256; ++k) {
            float d = 0.f;
            for (int t = 0; t < ds; ++t) {
                const float u = x[t] - c[k * ds + t];
                d = fmaf(u, u, d);
            }
            if (d < best) {
                best = d;
                arg = k;
            }
        }
        codes[(int64_t)j * total_slots + slot] = (uint8_t)arg;
        e2 += best;
    }
    err[slot] = sqrtf(e2);
}

// lut[(b * m + j) * 256 + k] = ||q'_j - c_jk||^2, one thread per entry.
__global__ void pq_lut_kernel(const float* __restrict__ qrot, int64_t B, int32_t Dpad, const int32_t* __restrict__ perm,
                              const float* __restrict__ cb, int m, int ds, float* __restrict__ lut) {
    const int64_t id = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (id >= B * m * 256) return;
    const int k = (int)(id & 255);
    const int64_t bj = id >> 8;
    const int j = (int)(bj % m);
    const int64_t b = bj / m;
    const float* q = qrot + b * Dpad;
    const float* c = cb + ((int64_t)j * 256 + k) * ds;
    float d = 0.f;
    for (int t = 0; t < ds; ++t) {
        const float u = q[perm[j * ds + t]] - c[t];
        d = fmaf(u, u, d);
    }
    lut[id] = d;
}

constexpr int kPqThreads = 256;

// Persistent over the wave's work items (query b, probe ranks
// [r0 + rpi c, r0 + rpi (c + 1)) clipped to the wave and nprobe).
__global__ void __launch_bounds__(kPqThreads) pq_scan_kernel(IndexView ix, WaveView wv, int w, PQView pv, int rpi) {
    extern __shared__ __align__(16) float s_lut[];
    __shared__ unsigned long long s_st[4];
    __shared__ int64_t s_item;
    const int tid = threadIdx.x, lane = tid & 31;
    const int nlut = pv.m * 256;
    const int r0 = wv.pass_begin[w];
    const int r1 = wv.pass_begin[w + 1];
    const int nch = (min(r1, wv.P) - r0 + rpi - 1) / rpi;  // items per query in this wave
    const int64_t n_items = nch > 0 ? wv.B * nch : 0;
    const bool want_stats = wv.stats != nullptr;
    for (;;) {
        if (tid == 0) s_item = atomicAdd((unsigned long long*)&wv.work[2 * wv.n_waves], 1ull);
        if (tid < 4) s_st[tid] = 0ull;
        __syncthreads();
        const int64_t item = s_item;
        if (item >= n_items) break;
        const int64_t b = item / nch;
        const int ch = (int)(item % nch);
        const int np = wv.nprobe[b];
        const int K = wv.K[b];
        const int rb = r0 + ch * rpi, re = min(min(rb + rpi, r1), np);
        if (K > 0 && np > 0 && rb < re) {
            for (int i = tid; i < nlut; i += kPqThreads) s_lut[i] = pv.lut[b * nlut + i];
            __syncthreads();
            const float tau = wv.tau[b];
            const float* qp = wv.qpad + b * ix.Dpad;
            for (int r = rb; r < re; ++r) {
                const int l = wv.probes[b * wv.P + r];
                const int64_t s0 = ix.list_slot[l];
                const int64_t npad = ix.list_slot[l + 1] - s0;
                const int n = ix.list_size[l];
                for (int c0 = 0; c0 < n; c0 += kPqThreads) {
                    const int c = c0 + tid;
                    const bool valid = c < n;
                    const int64_t slot = s0 + c;
                    bool keep = false;
                    if (valid) {
                        float dis = 0.f;
                        for (int j = 0; j < pv.m; ++j) dis += s_lut[j * 256 + pv.codes[(int64_t)j * pv.total_slots + slot]];
                        keep = !(fmaf(pv.m1, dis, fmaf(pv.m3, pv.err[slot], pv.beta)) > tau);
                    }
                    float d = 0.f;
                    if (keep) d = exact_distance(ix.orig + s0 * ix.Dpad + (int64_t)c * kBlock, npad, qp, ix.nb);
                    append_uniform(wv, w, (int)b, keep && d <= tau, d, (int32_t)slot, lane);
                    if (want_stats) {
                        const unsigned bv = __ballot_sync(0xffffffffu, valid);
                        const unsigned bk = __ballot_sync(0xffffffffu, keep);
                        if (lane == 0) {
                            atomicAdd(&s_st[0], (unsigned long long)__popc(bv));
                            atomicAdd(&s_st[1], (unsigned long long)__popc(bv & ~bk));
                            atomicAdd(&s_st[2], (unsigned long long)__popc(bk));
                            atomicAdd(&s_st[3], (unsigned long long)__popc(bk) * ix.D);
                        }
                    }
                }
            }
        }
        __syncthreads();
        if (want_stats && tid < 4 && s_st[tid]) atomicAdd((unsigned long long*)&wv.stats[b * 4 + tid], s_st[tid]);
        __syncthreads();
    }
}

}  // namespace

cudaError_t launch_pq_encode(const void* slab, int dtype, const float* scale, const int64_t* list_slot, int nlist,
                             int64_t total_slots, int32_t Dpad, const int32_t* perm, const float* cb, int m, int ds,
                             uint8_t* codes, float* err, cudaStream_t st) {
    if (total_slots == 0) return cudaSuccess;
    if (ds > 64) return cudaErrorInvalidValue;
    pq_encode_kernel<<<(unsigned)ceil_div(total_slots, 128), 128, 0, st>>>(slab, dtype, scale, list_slot, nlist,
                                                                          total_slots, Dpad, perm, cb, m, ds, codes,
                                                                          err);
    return cudaGetLastError();
}

cudaError_t launch_pq_lut(const float* qrot, int64_t B, int32_t Dpad, const int32_t* perm, const float* cb, int m,
                          int ds, float* lut, cudaStream_t st) {
    const int64_t n = B * m * 256;
    if (n == 0) return cudaSuccess;
    pq_lut_kernel<<<(unsigned)ceil_div(n, 256), 256, 0, st>>>(qrot, B, Dpad, perm, cb, m, ds, lut);
    return cudaGetLastError();
}

cudaError_t launch_pq_scan(const IndexView& ix, const WaveView& wv, int w, const PQView& pv, cudaStream_t st) {
    const int smem = pv.m * 256 * (int)sizeof(float);
    static int configured = 0;
    if (smem > configured) {
        cudaError_t e = cudaFuncSetAttribute(pq_scan_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, smem);
        if (e != cudaSuccess) return e;
        configured = smem;
    }
    int dev = 0, sms = 0, per = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    cudaError_t e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per, pq_scan_kernel, kPqThreads, smem);
    if (e != cudaSuccess) return e;
    // the item counter (one 64-bit word after the 2 x n_waves scan and
    // collect counters) starts at zero for every wave
    e = cudaMemsetAsync(wv.work + 2 * wv.n_waves, 0, sizeof(unsigned long long), st);
    if (e != cudaSuccess) return e;
    const int64_t grid = (int64_t)sms * std::max(per, 1);
    const int r0 = wv.pass_begin[w];
    const int nranks = std::max(0, std::min(wv.pass_begin[w + 1], (int)wv.P) - r0);
    const int rpi = (int)std::max<int64_t>(1, std::min<int64_t>(std::max(nranks, 1),
                                                                ceil_div(wv.B * nranks, 4 * grid)));
    pq_scan_kernel<<<(unsigned)grid, kPqThreads, smem, st>>>(ix, wv, w, pv, rpi);
    return cudaGetLastError();
}

}  // namespace dade
