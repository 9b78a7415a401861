// Bucket-sharded search (the multi-GPU layout of an IVF index): the buckets
// are split over n shards, each shard holds only its own buckets' vectors
// (with every centroid, so a query probes the same buckets everywhere), each
// shard runs the whole search over what it holds -- its waves and tau stay
// local -- and the shards' top-K lists are merged by (distance, id).  With
// pruning off the merged result is the exact top-K over the probed buckets,
// i.e. the unsharded result; with pruning on each shard's tau is its own.
#include <memory>
#include <numeric>

#include "dade_internal.h"

namespace dade {

std::vector<int32_t> shard_owners(const std::vector<int64_t>& list_size, int n_shards) {
    const int nl = (int)list_size.size();
    std::vector<int> order(nl);
    std::iota(order.begin(), order.end(), 0);
    std::stable_sort(order.begin(), order.end(), [&](int a, int b) { return list_size[a] > list_size[b]; });
    std::vector<int64_t> load((size_t)n_shards, 0);
    std::vector<int32_t> owner((size_t)nl, 0);
    for (int l : order) {
        int best = 0;
        for (int s = 1; s < n_shards; ++s)
            if (load[(size_t)s] < load[(size_t)best]) best = s;
        owner[(size_t)l] = best;
        load[(size_t)best] += list_size[(size_t)l];
    }
    return owner;
}

namespace {

// One warp per query: lane p < n_parts holds the head of part p's list
// (sorted by (distance, id); ids < 0 are padding); K rounds of a warp
// argmin emit the merged list.
__global__ void merge_topk_kernel(int n_parts, int64_t B, int Kmax, const int32_t* __restrict__ K,
                                  const int64_t* __restrict__ ids, const float* __restrict__ dists,
                                  int64_t* __restrict__ ids_out, float* __restrict__ dists_out) {
    const int lane = threadIdx.x & 31;
    const int64_t b = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    if (b >= B) return;
    const int k_b = min(max(K[b], 0), Kmax);
    int cur = 0;
    auto head = [&](float& d, long long& id) {
        d = INFINITY;
        id = LLONG_MAX;
        if (lane < n_parts && cur < k_b) {
            const int64_t e = ((int64_t)lane * B + b) * Kmax + cur;
            const int64_t x = ids[e];
            if (x >= 0) {
                d = dists[e];
                id = x;
            }
        }
    };
    float hd;
    long long hi;
    head(hd, hi);
    for (int k = 0; k < Kmax; ++k) {
        float bd = hd;
        long long bi = hi;
        int bl = lane;
        for (int off = 16; off; off >>= 1) {
            const float od = __shfl_xor_sync(0xffffffffu, bd, off);
            const long long oi = __shfl_xor_sync(0xffffffffu, bi, off);
            const int ol = __shfl_xor_sync(0xffffffffu, bl, off);
            if (od < bd || (od == bd && (oi < bi || (oi == bi && ol < bl)))) {
                bd = od;
                bi = oi;
                bl = ol;
            }
        }
        if (lane == 0) {
            const bool real = k < k_b && bi != LLONG_MAX;
            ids_out[b * Kmax + k] = real ? (int64_t)bi : -1;
            dists_out[b * Kmax + k] = real ? bd : INFINITY;
        }
        if (lane == bl && bi != LLONG_MAX) {
            ++cur;
            head(hd, hi);
        }
    }
}

}  // namespace

cudaError_t launch_merge_topk(int n_parts, int64_t B, int Kmax, const int32_t* K, const int64_t* ids,
                              const float* dists, int64_t* ids_out, float* dists_out, cudaStream_t st) {
    if (B == 0 || Kmax == 0) return cudaSuccess;
    merge_topk_kernel<<<(unsigned)ceil_div(B * 32, 256), 256, 0, st>>>(n_parts, B, Kmax, K, ids, dists, ids_out,
                                                                        dists_out);
    return cudaGetLastError();
}

}  // namespace dade

using namespace dade;

extern "C" dade_status dade_shard_owners(const int64_t* list_size_host, int32_t nlist, int32_t n_shards,
                                         int32_t* owner_out_host) {
    clear_error();
    if (!list_size_host || !owner_out_host || nlist < 1) return fail(DADE_EINVAL, "null argument or nlist < 1");
    if (n_shards < 1 || n_shards > nlist) return fail(DADE_EINVAL, "n_shards must be in [1, nlist]");
    for (int l = 0; l < nlist; ++l)
        if (list_size_host[l] < 0) return fail(DADE_EINVAL, "negative bucket size");
    const std::vector<int32_t> o = shard_owners(std::vector<int64_t>(list_size_host, list_size_host + nlist), n_shards);
    std::copy(o.begin(), o.end(), owner_out_host);
    return DADE_OK;
}

extern "C" dade_status dade_index_shard(const dade_index* idx, int32_t n_shards, int32_t shard, dade_index** out) {
    clear_error();
    if (!idx || !out) return fail(DADE_EINVAL, "null argument");
    if (n_shards < 1 || n_shards > idx->nlist) return fail(DADE_EINVAL, "n_shards must be in [1, nlist]");
    if (shard < 0 || shard >= n_shards) return fail(DADE_EINVAL, "shard must be in [0, n_shards)");
    const std::vector<int32_t> owner = shard_owners(idx->list_size, n_shards);
    std::unique_ptr<dade_index> sh(new dade_index());
    cudaGetDevice(&sh->device);
    sh->D = idx->D;
    sh->Dpad = idx->Dpad;
    sh->nb = idx->nb;
    sh->nlist = idx->nlist;
    sh->dtype = idx->dtype;
    sh->mean = idx->mean;
    sh->R = idx->R;
    sh->centroids = idx->centroids;
    sh->fp8_scale = idx->fp8_scale;
    sh->var = idx->var;
    for (int64_t i = 0; i < idx->N; ++i) {
        const int32_t l = idx->assign[(size_t)i];
        if (owner[(size_t)l] != shard) continue;
        sh->assign.push_back(l);
        sh->ids.push_back(idx->ids[(size_t)i]);
    }
    sh->N = (int64_t)sh->assign.size();
    DADE_TRY(upload_index_arrays(sh.get()));
    // the owned buckets' device ranges (members keep their order)
    const size_t es = idx->dtype == DADE_SLAB_F32 ? 4 : idx->dtype == DADE_SLAB_BF16 ? 2 : 1;
    const int64_t Dp = idx->Dpad;
    for (int l = 0; l < idx->nlist; ++l) {
        if (owner[(size_t)l] != shard) continue;
        const int64_t s0 = idx->list_slot[(size_t)l], n = idx->list_slot[(size_t)l + 1] - s0;
        const int64_t d0 = sh->list_slot[(size_t)l];
        if (n == 0) continue;
        if (sh->list_slot[(size_t)l + 1] - d0 != n) return fail(DADE_ESTATE, "shard layout mismatch");
        DADE_CUDA_TRY(cudaMemcpy(static_cast<char*>(sh->slab_dev.p) + d0 * Dp * es,
                                 static_cast<const char*>(idx->slab_dev.p) + s0 * Dp * es, n * Dp * es,
                                 cudaMemcpyDefault));
        DADE_CUDA_TRY(cudaMemcpy(sh->orig_dev.as<float>() + d0 * Dp, idx->orig_dev.as<float>() + s0 * Dp,
                                 sizeof(float) * n * Dp, cudaMemcpyDefault));
        DADE_CUDA_TRY(cudaMemcpy(sh->ids_dev.as<int64_t>() + d0, idx->ids_dev.as<int64_t>() + s0,
                                 sizeof(int64_t) * n, cudaMemcpyDefault));
        if (idx->dtype != DADE_SLAB_F32)
            DADE_CUDA_TRY(cudaMemcpy(sh->eps_dev.as<float>() + d0, idx->eps_dev.as<float>() + s0,
                                     sizeof(float) * n, cudaMemcpyDefault));
    }
    auto dup = [](DevBuf& dst, const DevBuf& src) -> dade_status {
        if (!src.p) return DADE_OK;
        DADE_TRY(dst.alloc(src.bytes));
        DADE_CUDA_TRY(cudaMemcpy(dst.p, src.p, src.bytes, cudaMemcpyDefault));
        return DADE_OK;
    };
    DADE_TRY(dup(sh->R_dev, idx->R_dev));
    DADE_TRY(dup(sh->mean_dev, idx->mean_dev));
    DADE_TRY(dup(sh->cent_dev, idx->cent_dev));
    DADE_TRY(dup(sh->cnorm_dev, idx->cnorm_dev));
    DADE_TRY(dup(sh->scale_dev, idx->scale_dev));
    DADE_TRY(dup(sh->var_dev, idx->var_dev));
    DADE_TRY(build_residual_norms(sh.get()));
    DADE_TRY(build_tc_operands(sh.get()));
    for (const auto& kv : idx->tables)
        DADE_TRY(install_table_public(sh.get(), kv.first, kv.second.S, kv.second.m1.data(), kv.second.beta.data()));
    *out = sh.release();
    return DADE_OK;
}

extern "C" dade_status dade_merge_topk(int32_t n_parts, int64_t B, int32_t max_K, const int32_t* K_dev,
                                       const int64_t* ids_dev, const float* dists_dev, int64_t* ids_out_dev,
                                       float* dists_out_dev, void* cuda_stream) {
    clear_error();
    if (n_parts < 1 || n_parts > 32) return fail(DADE_EINVAL, "n_parts must be in [1, 32]");
    if (B < 0 || max_K < 0 || max_K > kMaxK) return fail(DADE_EINVAL, "B >= 0 and max_K in [0, %d] required", kMaxK);
    if (B > 0 && max_K > 0 && (!K_dev || !ids_dev || !dists_dev || !ids_out_dev || !dists_out_dev))
        return fail(DADE_EINVAL, "null argument");
    DADE_CUDA_TRY(launch_merge_topk(n_parts, B, max_K, K_dev, ids_dev, dists_dev, ids_out_dev, dists_out_dev,
                                    static_cast<cudaStream_t>(cuda_stream)));
    return DADE_OK;
}
