// Top-nprobe bucket selection (Section II-A: a query probes its nprobe
// nearest centroids).  One CTA per query: an MSD radix select over the
// 32-bit patterns of the non-negative FP32 distances (monotone as unsigned
// integers) finds the nprobe-th smallest key; the keys below it and the
// lowest-id keys equal to it are gathered in column order and sorted by
// (distance, list id) with a bitonic network.
#include "../dade_internal.h"

namespace dade {
namespace {

constexpr int NT = 256;
constexpr int PMAX = 1024;

__device__ __forceinline__ bool key_less(uint32_t ka, int ia, uint32_t kb, int ib) {
    return ka < kb || (ka == kb && ia < ib);
}

// Exclusive prefix of `flag` over the CTA in thread order; returns the
// thread's offset and writes the CTA total to *total.
__device__ int block_excl_scan(int flag, int* warp_sums, int* total) {
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    unsigned bal = __ballot_sync(0xffffffffu, flag);
    int pre = __popc(bal & ((1u << lane) - 1u));
    if (lane == 0) warp_sums[wid] = __popc(bal);
    __syncthreads();
    int base = 0, tot = 0;
    for (int w = 0; w < NT / 32; ++w) {
        int v = warp_sums[w];
        if (w < wid) base += v;
        tot += v;
    }
    __syncthreads();
    *total = tot;
    return base + pre;
}

// STAGED: the row is first copied to shared memory (n <= kStageMax).
constexpr int kStageMax = 16384;

template <bool STAGED>
__global__ void __launch_bounds__(NT) select_kernel(const float* __restrict__ scores, int n,
                                                    const int32_t* __restrict__ nprobe, int P,
                                                    int32_t* __restrict__ probes,
                                                    int32_t* __restrict__ status) {
    extern __shared__ float srow[];
    __shared__ int hist[256];
    __shared__ int warp_sums[NT / 32];
    __shared__ uint32_t sel_key[PMAX];
    __shared__ int sel_id[PMAX];
    __shared__ int s_digit, s_below;
    const int64_t b = blockIdx.x;
    const float* grow = scores + b * (int64_t)n;
    int32_t* out = probes + b * (int64_t)P;
    const int tid = threadIdx.x;
    if (STAGED) {
        for (int i = tid; i < n; i += NT) srow[i] = grow[i];
        __syncthreads();
    }
    const float* row = STAGED ? srow : grow;
    int np = nprobe[b];
    if (np < 1 || np > P || np > n) {
        // nprobe = 0 marks an inactive query slot; other values are errors
        if (tid == 0 && status && np != 0) atomicCAS(status, 0, (int)DADE_EINVAL);
        for (int r = tid; r < P; r += NT) out[r] = -1;
        return;
    }
    int k = np;  // rank (1-based) still to locate inside the current prefix
    uint32_t prefix = 0, mask = 0;
    for (int shift = 24; shift >= 0; shift -= 8) {
        for (int i = tid; i < 256; i += NT) hist[i] = 0;
        __syncthreads();
        for (int i = tid; i < n; i += NT) {
            uint32_t key = __float_as_uint(row[i]);
            if ((key & mask) == prefix) atomicAdd(&hist[(key >> shift) & 255u], 1);
        }
        __syncthreads();
        if (tid == 0) {
            int cum = 0, d = 0;
            for (; d < 256; ++d) {
                if (cum + hist[d] >= k) break;
                cum += hist[d];
            }
            s_digit = d;
            s_below = cum;
        }
        __syncthreads();
        k -= s_below;
        prefix |= (uint32_t)s_digit << shift;
        mask |= 255u << shift;
        __syncthreads();
    }
    // prefix is the np-th smallest key; k of the keys equal to it are needed
    const uint32_t kth = prefix;
    const int need_eq = k;
    int n_lt = 0, n_eq = 0;
    for (int base = 0; base < n; base += NT) {
        int i = base + tid;
        uint32_t key = i < n ? __float_as_uint(row[i]) : 0xffffffffu;
        int lt = i < n && key < kth;
        int eq = i < n && key == kth;
        int tot_lt, tot_eq;
        int off_lt = block_excl_scan(lt, warp_sums, &tot_lt);
        int off_eq = block_excl_scan(eq, warp_sums, &tot_eq);
        if (lt) {
            sel_key[n_lt + off_lt] = key;
            sel_id[n_lt + off_lt] = i;
        }
        if (eq && n_eq + off_eq < need_eq) {
            int pos = (np - need_eq) + n_eq + off_eq;
            sel_key[pos] = key;
            sel_id[pos] = i;
        }
        n_lt += tot_lt;
        n_eq += tot_eq;
    }
    __syncthreads();
    int M = 1;
    while (M < np) M <<= 1;
    for (int i = np + tid; i < M; i += NT) {
        sel_key[i] = 0xffffffffu;
        sel_id[i] = 0x7fffffff;
    }
    __syncthreads();
    for (int size = 2; size <= M; size <<= 1) {
        for (int stride = size >> 1; stride > 0; stride >>= 1) {
            for (int i = tid; i < M; i += NT) {
                int j = i ^ stride;
                if (j > i) {
                    bool up = (i & size) == 0;
                    bool sw = up ? key_less(sel_key[j], sel_id[j], sel_key[i], sel_id[i])
                                 : key_less(sel_key[i], sel_id[i], sel_key[j], sel_id[j]);
                    if (sw) {
                        uint32_t tk = sel_key[i];
                        sel_key[i] = sel_key[j];
                        sel_key[j] = tk;
                        int ti = sel_id[i];
                        sel_id[i] = sel_id[j];
                        sel_id[j] = ti;
                    }
                }
            }
            __syncthreads();
        }
    }
    for (int r = tid; r < P; r += NT) out[r] = r < np ? sel_id[r] : -1;
}

}  // namespace

cudaError_t launch_select_probes(const float* scores, int64_t B, int n, const int32_t* nprobe,
                                 int P, int32_t* probes, int32_t* status, cudaStream_t st) {
    if (B <= 0) return cudaSuccess;
    if (P > PMAX) return cudaErrorInvalidValue;
    if (n <= kStageMax) {
        static bool configured = false;
        if (!configured) {
            cudaError_t e = cudaFuncSetAttribute(select_kernel<true>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                                 kStageMax * (int)sizeof(float));
            if (e != cudaSuccess) return e;
            configured = true;
        }
        select_kernel<true><<<(unsigned)B, NT, n * sizeof(float), st>>>(scores, n, nprobe, P, probes, status);
    } else {
        select_kernel<false><<<(unsigned)B, NT, 0, st>>>(scores, n, nprobe, P, probes, status);
    }
    return cudaGetLastError();
}

}  // namespace dade
