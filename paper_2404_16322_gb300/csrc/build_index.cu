// ivf_build: rotate the database on the device, cluster it with Lloyd
// k-means in the rotated space (Section II-A IVF), and lay out each bucket as
// dimension-blocked rotated slabs plus the original FP32 vectors.
#include <string.h>

#include <algorithm>
#include <memory>
#include <thread>
#include <vector>

#include "dade_internal.h"

namespace dade {
namespace {

// Seeded sample of k distinct rows of [0, n): partial Fisher-Yates driven
// by SplitMix64 of (seed + i).
std::vector<int64_t> sample_rows(int64_t n, int64_t k, uint64_t seed) {
    std::vector<int64_t> perm((size_t)n);
    for (int64_t i = 0; i < n; ++i) perm[(size_t)i] = i;
    for (int64_t i = 0; i < k; ++i) {
        uint64_t r = splitmix64(seed + (uint64_t)i);
        int64_t j = i + (int64_t)(r % (uint64_t)(n - i));
        std::swap(perm[(size_t)i], perm[(size_t)j]);
    }
    perm.resize((size_t)k);
    return perm;
}

// New centroids = FP64 mean of the assigned rotated rows; an empty bucket
// keeps its centroid.  Rows are split over threads; partial sums are added in
// thread order.
void update_centroids(const float* xr, int64_t N, int Dpad, int D, const int32_t* assign, int nlist,
                      std::vector<float>& cent /* nlist x Dpad */) {
    unsigned hw = std::max(1u, std::thread::hardware_concurrency());
    int nt = (int)std::min<int64_t>(hw, std::max<int64_t>(1, N / 4096));
    std::vector<std::vector<double>> sums(nt);
    std::vector<std::vector<int64_t>> cnts(nt);
    std::vector<std::thread> th;
    for (int t = 0; t < nt; ++t)
        th.emplace_back([&, t] {
            sums[t].assign((size_t)nlist * D, 0.0);
            cnts[t].assign((size_t)nlist, 0);
            int64_t a = N * t / nt, b = N * (t + 1) / nt;
            for (int64_t i = a; i < b; ++i) {
                int l = assign[i];
                const float* x = xr + i * Dpad;
                double* s = &sums[t][(size_t)l * D];
                for (int j = 0; j < D; ++j) s[j] += x[j];
                cnts[t][l]++;
            }
        });
    for (auto& x : th) x.join();
    for (int l = 0; l < nlist; ++l) {
        int64_t c = 0;
        for (int t = 0; t < nt; ++t) c += cnts[t][l];
        if (c == 0) continue;
        for (int j = 0; j < D; ++j) {
            double s = 0;
            for (int t = 0; t < nt; ++t) s += sums[t][(size_t)l * D + j];
            cent[(size_t)l * Dpad + j] = (float)(s / (double)c);
        }
    }
}

dade_status assign_device(const float* xrot, int64_t N, int Dpad, const float* cent, int nlist,
                          DevBuf& amin, std::vector<unsigned long long>& host, cudaStream_t st) {
    DADE_CUDA_TRY(cudaMemsetAsync(amin.p, 0xff, sizeof(unsigned long long) * N, st));
    DADE_CUDA_TRY(launch_gemm_argmin(xrot, Dpad, cent, Dpad, amin.as<unsigned long long>(), N, nlist,
                                     Dpad, st));
    DADE_CUDA_TRY(cudaMemcpyAsync(host.data(), amin.p, sizeof(unsigned long long) * N,
                                  cudaMemcpyDeviceToHost, st));
    DADE_CUDA_TRY(cudaStreamSynchronize(st));
    return DADE_OK;
}

}  // namespace


}  // namespace dade

extern "C" dade_status ivf_build(const float* X, int64_t N, int32_t D, const double* mean,
                                 const double* R, const dade_build_params* p, dade_index** out) {
    using namespace dade;
    clear_error();
    if (!X || !mean || !R || !p || !out) return fail(DADE_EINVAL, "null argument");
    if (N < 1 || N > (int64_t)1 << 31) return fail(DADE_EINVAL, "N out of range");
    if (D < 1 || D > kMaxD) return fail(DADE_EINVAL, "D out of range");
    if (p->nlist < 1 || p->nlist > 65536 || p->nlist > N) return fail(DADE_EINVAL, "nlist out of range");
    if (p->dtype < DADE_SLAB_F32 || p->dtype > DADE_SLAB_FP8E4M3) return fail(DADE_EINVAL, "bad dtype");
    if (p->assign && !p->centroids) return fail(DADE_EINVAL, "assign needs centroids");
    if (p->assign)
        for (int64_t i = 0; i < N; ++i)
            if (p->assign[i] < 0 || p->assign[i] >= p->nlist) return fail(DADE_EINVAL, "assign out of range");

    std::unique_ptr<dade_index> idx(new dade_index());
    DADE_CUDA_TRY(cudaGetDevice(&idx->device));
    idx->N = N;
    idx->D = D;
    idx->Dpad = (int32_t)round_up(D, kBlock);
    idx->nb = idx->Dpad / kBlock;
    idx->nlist = p->nlist;
    idx->dtype = p->dtype;
    idx->mean.assign(mean, mean + D);
    idx->R.assign(R, R + (size_t)D * D);
    const int Dp = idx->Dpad, nl = p->nlist;

    cudaStream_t st;
    DADE_CUDA_TRY(cudaStreamCreateWithFlags(&st, cudaStreamNonBlocking));
    struct StreamGuard {
        cudaStream_t s;
        ~StreamGuard() { cudaStreamDestroy(s); }
    } guard{st};

    // rotation and mean on the device, FP32
    {
        std::vector<float> Rf((size_t)Dp * Dp, 0.f), mf((size_t)Dp, 0.f);
        for (int i = 0; i < D; ++i) {
            mf[i] = (float)mean[i];
            for (int j = 0; j < D; ++j) Rf[(size_t)i * Dp + j] = (float)R[(size_t)i * D + j];
        }
        DADE_TRY(idx->R_dev.alloc(sizeof(float) * Rf.size()));
        DADE_TRY(idx->mean_dev.alloc(sizeof(float) * mf.size()));
        DADE_CUDA_TRY(cudaMemcpy(idx->R_dev.p, Rf.data(), sizeof(float) * Rf.size(), cudaMemcpyHostToDevice));
        DADE_CUDA_TRY(cudaMemcpy(idx->mean_dev.p, mf.data(), sizeof(float) * mf.size(), cudaMemcpyHostToDevice));
    }
    // X in device memory of this device is read in place; host rows are
    // copied up (pageable or pinned)
    bool x_on_device = false;
    {
        cudaPointerAttributes pa{};
        if (cudaPointerGetAttributes(&pa, X) == cudaSuccess &&
            (pa.type == cudaMemoryTypeDevice || pa.type == cudaMemoryTypeManaged)) {
            if (pa.device != idx->device)
                return fail(DADE_EINVAL, "X is in the memory of device %d, the current device is %d", pa.device,
                            idx->device);
            x_on_device = true;
        }
        cudaGetLastError();
    }
    DevBuf x_dev, xr_dev, amin;
    if (!x_on_device) DADE_TRY(x_dev.alloc(sizeof(float) * N * D));
    DADE_TRY(xr_dev.alloc(sizeof(float) * N * Dp));
    DADE_TRY(amin.alloc(sizeof(unsigned long long) * N));
    if (!x_on_device)
        DADE_CUDA_TRY(cudaMemcpyAsync(x_dev.p, X, sizeof(float) * N * D, cudaMemcpyHostToDevice, st));
    const float* xd = x_on_device ? X : x_dev.as<float>();
    DADE_CUDA_TRY(launch_tc_dot(xd, D, idx->mean_dev.as<float>(), idx->R_dev.as<float>(), Dp,
                                xr_dev.as<float>(), Dp, N, Dp, D, nullptr, st));

    // centroids (rotated space)
    std::vector<float> cent((size_t)nl * Dp, 0.f);
    DADE_TRY(idx->cent_dev.alloc(sizeof(float) * cent.size()));
    std::vector<unsigned long long> amin_h((size_t)N);
    std::vector<int32_t> assign((size_t)N);
    std::vector<float> xr_h;
    if (p->centroids) {
        for (int l = 0; l < nl; ++l)
            for (int j = 0; j < D; ++j) cent[(size_t)l * Dp + j] = p->centroids[(size_t)l * D + j];
    } else {
        std::vector<int64_t> init = sample_rows(N, nl, p->seed);
        xr_h.resize((size_t)N * Dp);
        DADE_CUDA_TRY(cudaMemcpyAsync(xr_h.data(), xr_dev.p, sizeof(float) * N * Dp,
                                      cudaMemcpyDeviceToHost, st));
        DADE_CUDA_TRY(cudaStreamSynchronize(st));
        for (int l = 0; l < nl; ++l)
            memcpy(&cent[(size_t)l * Dp], &xr_h[(size_t)init[l] * Dp], sizeof(float) * Dp);
        for (int it = 0; it < p->kmeans_iters; ++it) {
            DADE_CUDA_TRY(cudaMemcpyAsync(idx->cent_dev.p, cent.data(), sizeof(float) * cent.size(),
                                          cudaMemcpyHostToDevice, st));
            DADE_TRY(assign_device(xr_dev.as<float>(), N, Dp, idx->cent_dev.as<float>(), nl, amin, amin_h, st));
            for (int64_t i = 0; i < N; ++i) assign[(size_t)i] = (int32_t)(amin_h[(size_t)i] & 0xffffffffull);
            update_centroids(xr_h.data(), N, Dp, D, assign.data(), nl, cent);
        }
    }
    DADE_CUDA_TRY(cudaMemcpyAsync(idx->cent_dev.p, cent.data(), sizeof(float) * cent.size(),
                                  cudaMemcpyHostToDevice, st));
    DADE_TRY(idx->cnorm_dev.alloc(sizeof(float) * nl));
    DADE_CUDA_TRY(launch_row_norms(idx->cent_dev.as<float>(), Dp, nl, Dp, idx->cnorm_dev.as<float>(), st));
    if (p->assign) {
        memcpy(assign.data(), p->assign, sizeof(int32_t) * N);
    } else {
        DADE_TRY(assign_device(xr_dev.as<float>(), N, Dp, idx->cent_dev.as<float>(), nl, amin, amin_h, st));
        for (int64_t i = 0; i < N; ++i) assign[(size_t)i] = (int32_t)(amin_h[(size_t)i] & 0xffffffffull);
    }
    idx->centroids.resize((size_t)nl * D);
    for (int l = 0; l < nl; ++l)
        for (int j = 0; j < D; ++j) idx->centroids[(size_t)l * D + j] = cent[(size_t)l * Dp + j];
    idx->assign = assign;
    idx->ids.resize((size_t)N);
    for (int64_t i = 0; i < N; ++i) idx->ids[(size_t)i] = p->ids ? p->ids[i] : i;

    // FP8 per-dimension scale from the rotated FP32 values
    if (idx->dtype == DADE_SLAB_FP8E4M3) {
        DADE_TRY(idx->scale_dev.alloc(sizeof(float) * Dp));
        DADE_CUDA_TRY(launch_amax(xr_dev.as<float>(), N, Dp, idx->scale_dev.as<float>(), st));
        DADE_CUDA_TRY(launch_fp8_scale(idx->scale_dev.as<float>(), Dp, st));
        idx->fp8_scale.resize((size_t)Dp);
        DADE_CUDA_TRY(cudaMemcpyAsync(idx->fp8_scale.data(), idx->scale_dev.p, sizeof(float) * Dp,
                                      cudaMemcpyDeviceToHost, st));
    }
    DADE_CUDA_TRY(cudaStreamSynchronize(st));
    // bucket layout and device arrays (shared with dade_index_load)
    DADE_TRY(upload_index_arrays(idx.get()));
    {
        // slot -> source row map, then the blocked layout kernel
        std::vector<int32_t> slot_row((size_t)idx->total_slots, -1), slot_list((size_t)idx->total_slots);
        std::vector<int64_t> cursor(idx->list_slot.begin(), idx->list_slot.end() - 1);
        for (int64_t i = 0; i < N; ++i) slot_row[(size_t)cursor[(size_t)assign[(size_t)i]]++] = (int32_t)i;
        for (int l = 0; l < nl; ++l)
            for (int64_t s = idx->list_slot[l]; s < idx->list_slot[l + 1]; ++s) slot_list[(size_t)s] = l;
        DevBuf srow, slist;
        DADE_TRY(srow.alloc(sizeof(int32_t) * std::max<int64_t>(1, idx->total_slots)));
        DADE_TRY(slist.alloc(sizeof(int32_t) * std::max<int64_t>(1, idx->total_slots)));
        DADE_CUDA_TRY(cudaMemcpyAsync(srow.p, slot_row.data(), sizeof(int32_t) * idx->total_slots,
                                      cudaMemcpyHostToDevice, st));
        DADE_CUDA_TRY(cudaMemcpyAsync(slist.p, slot_list.data(), sizeof(int32_t) * idx->total_slots,
                                      cudaMemcpyHostToDevice, st));
        LayoutArgs la;
        la.xrot = xr_dev.as<float>();
        la.x = xd;
        la.slot_row = srow.as<int32_t>();
        la.slot_list = slist.as<int32_t>();
        la.list_slot = idx->list_slot_dev.as<int64_t>();
        la.total_slots = idx->total_slots;
        la.D = D;
        la.Dpad = Dp;
        la.dtype = idx->dtype;
        la.scale = idx->scale_dev.as<float>();
        la.slab = idx->slab_dev.p;
        la.orig = idx->orig_dev.as<float>();
        la.eps = idx->dtype == DADE_SLAB_F32 ? nullptr : idx->eps_dev.as<float>();
        DADE_CUDA_TRY(launch_layout(la, st));
        DADE_CUDA_TRY(launch_quant_error(la, st));
        DADE_TRY(idx->var_dev.alloc(sizeof(float) * Dp));
        DADE_CUDA_TRY(launch_dim_var(xr_dev.as<float>(), N, Dp, idx->var_dev.as<float>(), st));
        idx->var.resize((size_t)Dp);
        DADE_CUDA_TRY(cudaMemcpyAsync(idx->var.data(), idx->var_dev.p, sizeof(float) * Dp, cudaMemcpyDeviceToHost, st));
        std::vector<int64_t> slot_ids((size_t)idx->total_slots, -1);
        for (int64_t s = 0; s < idx->total_slots; ++s)
            if (slot_row[(size_t)s] >= 0) slot_ids[(size_t)s] = idx->ids[(size_t)slot_row[(size_t)s]];
        DADE_CUDA_TRY(cudaMemcpyAsync(idx->ids_dev.p, slot_ids.data(), sizeof(int64_t) * idx->total_slots,
                                      cudaMemcpyHostToDevice, st));
        DADE_CUDA_TRY(cudaStreamSynchronize(st));
    }
    DADE_TRY(build_residual_norms(idx.get()));
    DADE_TRY(build_tc_operands(idx.get()));
    *out = idx.release();
    return DADE_OK;
}
