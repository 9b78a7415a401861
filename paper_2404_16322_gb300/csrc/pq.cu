// OPQ-L's product quantiser on an index (arXiv 2404.16322, Section V-B
// "Approximate Distances"; OPQ by its parametric solution, Ge, He, Ke and
// Sun 2014): dimension allocation from the index's per-dimension variances,
// codebooks by host FP64 k-means on a sample, encoding of every slot on the
// device, and the three-feature correction (its fit is in fit.cu).
#include <math.h>
#include <string.h>

#include <algorithm>
#include <numeric>
#include <thread>
#include <vector>

#include "dade_internal.h"

using namespace dade;

namespace {

constexpr int kKsub = 256;

// OPQ's eigenvalue allocation dealt round by round: the dims, in decreasing
// variance, m per round, one to each subspace, the larger variances to the
// subspaces of smaller product of variances so far (lower subspace on a
// tie); the round structure keeps the rule independent of the variances'
// scale.  Subspace j's dims, ascending, at perm[j*ds .. (j+1)*ds).
std::vector<int32_t> allocate_dims(const std::vector<float>& var, int D, int m) {
    const int ds = D / m;
    std::vector<int32_t> order((size_t)D);
    std::iota(order.begin(), order.end(), 0);
    std::stable_sort(order.begin(), order.end(), [&](int a, int b) { return (double)var[a] > (double)var[b]; });
    std::vector<double> logp((size_t)m, 0.0);
    std::vector<std::vector<int32_t>> groups((size_t)m);
    for (int t = 0; t < ds; ++t) {
        std::vector<int> subs((size_t)m);
        std::iota(subs.begin(), subs.end(), 0);
        std::stable_sort(subs.begin(), subs.end(), [&](int a, int b) { return logp[a] < logp[b]; });
        for (int u = 0; u < m; ++u) {
            const int d = order[(size_t)t * m + u], j = subs[(size_t)u];
            groups[(size_t)j].push_back(d);
            logp[(size_t)j] += log(std::max((double)var[d], 1e-300));
        }
    }
    std::vector<int32_t> perm;
    perm.reserve((size_t)D);
    for (auto& g : groups) {
        std::sort(g.begin(), g.end());
        perm.insert(perm.end(), g.begin(), g.end());
    }
    return perm;
}

// Lloyd k-means in FP64 on the n x ds rows of one subspace, from the rows
// init[0..255]; the nearest centroid with the lower index on a tie; an empty
// cluster keeps its centroid.
void kmeans_sub(const double* X, int64_t n, int ds, const int64_t* init, int iters, double* C) {
    for (int k = 0; k < kKsub; ++k)
        for (int t = 0; t < ds; ++t) C[k * ds + t] = X[init[k] * ds + t];
    std::vector<int> a((size_t)n);
    std::vector<double> sum((size_t)kKsub * ds);
    std::vector<int64_t> cnt(kKsub);
    for (int it = 0; it < iters; ++it) {
        for (int64_t i = 0; i < n; ++i) {
            double best = INFINITY;
            int arg = 0;
            for (int k = 0; k < kKsub; ++k) {
                double d = 0;
                for (int t = 0; t < ds; ++t) {
                    const double u = X[i * ds + t] - C[k * ds + t];
                    d += u * u;
                }
                if (d < best) {
                    best = d;
                    arg = k;
                }
            }
            a[(size_t)i] = arg;
        }
        std::fill(sum.begin(), sum.end(), 0.0);
        std::fill(cnt.begin(), cnt.end(), 0);
        for (int64_t i = 0; i < n; ++i) {
            cnt[a[(size_t)i]]++;
            for (int t = 0; t < ds; ++t) sum[(size_t)a[(size_t)i] * ds + t] += X[i * ds + t];
        }
        for (int k = 0; k < kKsub; ++k)
            if (cnt[k])
                for (int t = 0; t < ds; ++t) C[k * ds + t] = sum[(size_t)k * ds + t] / (double)cnt[k];
    }
}

}  // namespace

extern "C" dade_status dade_pq_set(dade_index* idx, int32_t m, const int32_t* perm, const float* codebooks) {
    clear_error();
    if (!idx || !perm || !codebooks) return fail(DADE_EINVAL, "null argument");
    const int D = idx->D;
    if (m < 1 || D % m != 0) return fail(DADE_EINVAL, "m must divide D (%d)", D);
    const int ds = D / m;
    if (ds > 64) return fail(DADE_EINVAL, "at most 64 dims per subspace (D / m = %d)", ds);
    std::vector<char> seen((size_t)D, 0);
    for (int d = 0; d < D; ++d) {
        if (perm[d] < 0 || perm[d] >= D || seen[(size_t)perm[d]]) return fail(DADE_EINVAL, "perm is not a permutation");
        seen[(size_t)perm[d]] = 1;
    }
    idx->pq_perm.assign(perm, perm + D);
    idx->pq_cb.assign(codebooks, codebooks + (size_t)m * kKsub * ds);
    idx->pq_m = m;
    idx->pq_ds = ds;
    idx->pq_has_table = false;
    DADE_TRY(idx->pq_perm_dev.alloc(sizeof(int32_t) * D));
    DADE_TRY(idx->pq_cb_dev.alloc(sizeof(float) * idx->pq_cb.size()));
    DADE_TRY(idx->pq_codes_dev.alloc((size_t)m * std::max<int64_t>(1, idx->total_slots)));
    DADE_TRY(idx->pq_err_dev.alloc(sizeof(float) * std::max<int64_t>(1, idx->total_slots)));
    DADE_CUDA_TRY(cudaMemcpy(idx->pq_perm_dev.p, perm, sizeof(int32_t) * D, cudaMemcpyHostToDevice));
    DADE_CUDA_TRY(cudaMemcpy(idx->pq_cb_dev.p, idx->pq_cb.data(), sizeof(float) * idx->pq_cb.size(),
                             cudaMemcpyHostToDevice));
    DADE_CUDA_TRY(launch_pq_encode(idx->slab_dev.p, idx->dtype, idx->scale_dev.as<float>(),
                                   idx->list_slot_dev.as<int64_t>(), idx->nlist, idx->total_slots, idx->Dpad,
                                   idx->pq_perm_dev.as<int32_t>(), idx->pq_cb_dev.as<float>(), m, ds,
                                   idx->pq_codes_dev.as<uint8_t>(), idx->pq_err_dev.as<float>(), 0));
    DADE_CUDA_TRY(cudaDeviceSynchronize());
    return DADE_OK;
}

extern "C" dade_status dade_pq_train(dade_index* idx, const float* X, int64_t n, int32_t m, int32_t iters,
                                     uint64_t seed, int32_t* perm_out, float* codebooks_out) {
    clear_error();
    if (!idx || !X) return fail(DADE_EINVAL, "null argument");
    const int D = idx->D;
    if (m < 1 || D % m != 0) return fail(DADE_EINVAL, "m must divide D (%d)", D);
    const int ds = D / m;
    if (ds > 64) return fail(DADE_EINVAL, "at most 64 dims per subspace (D / m = %d)", ds);
    if (n < kKsub) return fail(DADE_EINVAL, "need at least %d training rows", kKsub);
    if (iters < 0) return fail(DADE_EINVAL, "iters < 0");
    // rotated training rows, x' = R (x - mean), FP64, subspace-major
    const std::vector<int32_t> perm = allocate_dims(idx->var, D, m);
    std::vector<double> Xs((size_t)n * D);
    {
        const unsigned hw = std::max(1u, std::thread::hardware_concurrency());
        const int nt = (int)std::min<int64_t>(hw, std::max<int64_t>(1, n / 1024));
        std::vector<std::thread> th;
        for (int w = 0; w < nt; ++w)
            th.emplace_back([&, w] {
                std::vector<double> xc((size_t)D);
                for (int64_t i = w; i < n; i += nt) {
                    for (int d = 0; d < D; ++d) xc[(size_t)d] = (double)X[i * D + d] - idx->mean[(size_t)d];
                    for (int j = 0; j < m; ++j)
                        for (int t = 0; t < ds; ++t) {
                            const int r = perm[(size_t)j * ds + t];
                            double s = 0;
                            for (int d = 0; d < D; ++d) s += idx->R[(size_t)r * D + d] * xc[(size_t)d];
                            Xs[((size_t)j * n + i) * ds + t] = s;
                        }
                }
            });
        for (auto& t : th) t.join();
    }
    // initial centroids: the first 256 rows of a seeded partial Fisher-Yates shuffle
    std::vector<int64_t> init((size_t)kKsub);
    {
        std::vector<int64_t> p((size_t)n);
        std::iota(p.begin(), p.end(), 0);
        for (int k = 0; k < kKsub; ++k) {
            const int64_t j = k + (int64_t)(splitmix64(seed + (uint64_t)k) % (uint64_t)(n - k));
            std::swap(p[(size_t)k], p[(size_t)j]);
        }
        std::copy(p.begin(), p.begin() + kKsub, init.begin());
    }
    std::vector<double> C((size_t)m * kKsub * ds);
    {
        const unsigned hw = std::max(1u, std::thread::hardware_concurrency());
        std::vector<std::thread> th;
        for (unsigned w = 0; w < std::min<unsigned>(hw, (unsigned)m); ++w)
            th.emplace_back([&, w] {
                for (int j = (int)w; j < m; j += (int)std::min<unsigned>(hw, (unsigned)m))
                    kmeans_sub(&Xs[(size_t)j * n * ds], n, ds, init.data(), iters, &C[(size_t)j * kKsub * ds]);
            });
        for (auto& t : th) t.join();
    }
    std::vector<float> cbf(C.size());
    for (size_t i = 0; i < C.size(); ++i) cbf[i] = (float)C[i];
    if (perm_out) std::copy(perm.begin(), perm.end(), perm_out);
    if (codebooks_out) std::copy(cbf.begin(), cbf.end(), codebooks_out);
    return dade_pq_set(idx, m, perm.data(), cbf.data());
}

extern "C" dade_status dade_pq_set_correction(dade_index* idx, float m1, float m3, float beta) {
    clear_error();
    if (!idx) return fail(DADE_EINVAL, "null index");
    if (idx->pq_m <= 0) return fail(DADE_ESTATE, "the index has no product quantiser");
    if (isnan(m1) || isnan(m3) || isnan(beta)) return fail(DADE_EINVAL, "NaN coefficient");
    idx->pq_m1 = m1;
    idx->pq_m3 = m3;
    idx->pq_beta = beta;
    idx->pq_has_table = true;
    return DADE_OK;
}

extern "C" dade_status dade_pq_get(const dade_index* idx, int32_t* m_out, float* correction3, uint8_t* codes,
                                   float* err) {
    clear_error();
    if (!idx) return fail(DADE_EINVAL, "null index");
    if (idx->pq_m <= 0) return fail(DADE_ESTATE, "the index has no product quantiser");
    if (m_out) *m_out = idx->pq_m;
    if (correction3) {
        if (!idx->pq_has_table) return fail(DADE_ESTATE, "no OPQ-L correction");
        correction3[0] = idx->pq_m1;
        correction3[1] = idx->pq_m3;
        correction3[2] = idx->pq_beta;
    }
    if (codes || err) {
        // device slots -> input rows: bucket l's rows, in increasing row
        // order, occupy slots list_slot[l], list_slot[l] + 1, ...
        const int m = idx->pq_m;
        const int64_t T = idx->total_slots;
        std::vector<uint8_t> cd((size_t)m * std::max<int64_t>(1, T));
        std::vector<float> ed((size_t)std::max<int64_t>(1, T));
        DADE_CUDA_TRY(cudaMemcpy(cd.data(), idx->pq_codes_dev.p, (size_t)m * T, cudaMemcpyDeviceToHost));
        DADE_CUDA_TRY(cudaMemcpy(ed.data(), idx->pq_err_dev.p, sizeof(float) * T, cudaMemcpyDeviceToHost));
        std::vector<int64_t> fill(idx->list_slot.begin(), idx->list_slot.end() - 1);
        for (int64_t r = 0; r < idx->N; ++r) {
            const int64_t slot = fill[(size_t)idx->assign[(size_t)r]]++;
            if (codes)
                for (int j = 0; j < m; ++j) codes[r * m + j] = cd[(size_t)j * T + slot];
            if (err) err[r] = ed[(size_t)slot];
        }
    }
    return DADE_OK;
}

extern "C" dade_status dade_pq_fit_samples(const double* dis, const double* err, const double* tau,
                                           const int8_t* label, int64_t n, double target_recall, int32_t min_label0,
                                           double* out3) {
    clear_error();
    if (n < 0 || (n > 0 && (!dis || !err || !tau || !label)) || !out3) return fail(DADE_EINVAL, "null argument");
    if (!(target_recall > 0 && target_recall <= 1)) return fail(DADE_EINVAL, "target_recall in (0, 1]");
    return fit_pq_host(dis, err, tau, label, n, target_recall, min_label0, out3);
}
