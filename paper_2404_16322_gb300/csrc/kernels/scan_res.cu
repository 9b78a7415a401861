// The Gaussian-bound (RES) variant of the estimate-and-prune scan, after
// Section IV-C (Algorithms 1-2) of arXiv 2404.16322: the candidate's
// distance is estimated from the partial distance over the scanned rotated
// dims plus the residual norms of the stored vector and of the query over
// the rest (Eq. 1), and corrected by m sigma with
// sigma^2 = 4 sum_{i >= d} q'_i^2 var_i (Eq. 2); the candidate is pruned iff
// the corrected estimate exceeds tau.
//
// The per-candidate residual norms are precomputed per slot and block at
// index build; the per-query part (||q'_r||^2 - m sigma after each step) is
// computed once per batch by res_terms_kernel.  This file holds the RES
// instantiations of the scan template so that they compile in parallel with
// the learned ones (scan.cu).
#include "scan_steps.cuh"

namespace dade {
namespace {

// One warp per query.  Walks the steps from the last to the first, adding
// the dims [d_s, d_{s+1}) (at most 32, one per lane) to FP64 suffix sums of
// q'_i^2 and q'_i^2 var_i.
__global__ void res_terms_kernel(const float* __restrict__ qrot, int64_t B, int32_t D, int32_t Dpad,
                                 const float* __restrict__ var, int delta_d, int S, float m,
                                 float* __restrict__ res_q) {
    const int lane = threadIdx.x & 31;
    const int64_t b = (int64_t)blockIdx.x * (blockDim.x / 32) + (threadIdx.x >> 5);
    if (b >= B) return;
    const float* q = qrot + b * Dpad;
    double rq = 0.0, sg = 0.0;
    int hi = D;
    for (int s = S - 2; s >= 0; --s) {
        const int lo = min((s + 1) * delta_d, D);
        double a = 0.0, c = 0.0;
        for (int j = lo + lane; j < hi; j += 32) {
            const double qj = q[j];
            a += qj * qj;
            c += qj * qj * (double)var[j];
        }
#pragma unroll
        for (int off = 16; off > 0; off >>= 1) {
            a += __shfl_xor_sync(0xffffffffu, a, off);
            c += __shfl_xor_sync(0xffffffffu, c, off);
        }
        rq += a;
        sg += c;
        if (lane == 0) res_q[b * (S - 1) + s] = (float)(rq - (double)m * 2.0 * sqrt(sg));
        hi = lo;
    }
}

}  // namespace

cudaError_t launch_wave_scan_res(const IndexView& ix, const WaveView& wv, int w, int delta_d, int S,
                                 cudaStream_t st) {
#define DADE_SCAN_CASE(DT, NB)                                                                            \
    if (ix.dtype == DT && delta_d == NB * kBlock)                                                         \
        return wv.final_test ? launch_scan_t<DT, NB, false, true, true>(ix, wv, w, nullptr, nullptr, S, st) \
                             : launch_scan_t<DT, NB, false, false, true>(ix, wv, w, nullptr, nullptr, S, st);
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

cudaError_t launch_res_terms(const float* qrot, int64_t B, int32_t D, int32_t Dpad, const float* var,
                             int delta_d, int S, float m, float* res_q, cudaStream_t st) {
    if (B == 0 || S <= 1) return cudaSuccess;
    constexpr int kWarpsPerBlock = 4;
    res_terms_kernel<<<(unsigned)ceil_div(B, kWarpsPerBlock), kWarpsPerBlock * 32, 0, st>>>(
        qrot, B, D, Dpad, var, delta_d, S, m, res_q);
    return cudaGetLastError();
}

}  // namespace dade
