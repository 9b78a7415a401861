// dade_fit_correction: learn the per-step table (m1_s, beta'_s) of the
// data-driven correction (Section V-A "Parameter Learning", "Adaptive
// Adjustment"; one classifier per step, Section V-B; labels as in
// Section VII-A).
//
// The training queries are searched three times on the device with pruning
// off, under the same wave schedule as dade_search: (A) the exact top-K per
// query; (B) a replay counting label-1 candidates; (C) a replay emitting the
// kept samples (every label-0 candidate, label-1 candidates thinned to about
// label1_cap by a SplitMix64 draw).  The samples' partial distances come from
// the stored slabs with the same arithmetic as the search.  The fit itself is
// host FP64 (fit_tables).
#include <math.h>

#include <algorithm>
#include <numeric>
#include <vector>

#include "dade_internal.h"

using namespace dade;

namespace {

// Training samples of a replay: ncols values per row (the partial distances
// dis'_1..dis'_{S-1}, or OPQ-L's (dis', e)), tau at the test and the label,
// sorted so that the fit does not depend on the device's atomic order.
struct Samples {
    int64_t n = 0;
    std::vector<double> P, T;
    std::vector<int8_t> L;
    std::vector<int64_t> Qi, Id;  // training query and candidate id of each row (if keys were asked for)
};

dade_status replay_samples(dade_index* idx, const float* Tq, int64_t nt, int32_t K, int32_t nprobe, int32_t delta_d,
                           uint64_t seed, int64_t label1_cap, int32_t estimator, int ncols, Samples* out,
                           bool keys = false) {
    cudaStream_t st;
    DADE_CUDA_TRY(cudaStreamCreateWithFlags(&st, cudaStreamNonBlocking));
    struct G {
        dade_index* idx;
        cudaStream_t s;
        ~G() {
            idx->ws.drop(s);  // the replays' scratch on this stream
            cudaStreamDestroy(s);
        }
    } guard{idx, st};

    const int64_t Bc = std::min<int64_t>(nt, 4096);
    const int D = idx->D;
    DevBuf q, kk, np, top_all, dists, cnt, status;
    DADE_TRY(q.alloc(sizeof(float) * Bc * D));
    DADE_TRY(kk.alloc(sizeof(int32_t) * Bc));
    DADE_TRY(np.alloc(sizeof(int32_t) * Bc));
    DADE_TRY(top_all.alloc(sizeof(int64_t) * nt * K));
    DADE_TRY(dists.alloc(sizeof(float) * Bc * K));
    DADE_TRY(cnt.alloc(sizeof(unsigned long long) * 2));
    DADE_TRY(status.alloc(sizeof(int32_t)));
    {
        std::vector<int32_t> kh((size_t)Bc, K), nh((size_t)Bc, nprobe);
        DADE_CUDA_TRY(cudaMemcpy(kk.p, kh.data(), sizeof(int32_t) * Bc, cudaMemcpyHostToDevice));
        DADE_CUDA_TRY(cudaMemcpy(np.p, nh.data(), sizeof(int32_t) * Bc, cudaMemcpyHostToDevice));
        DADE_CUDA_TRY(cudaMemset(cnt.p, 0, sizeof(unsigned long long) * 2));
        DADE_CUDA_TRY(cudaMemset(status.p, 0, sizeof(int32_t)));
    }
    dade_search_opts o{};
    o.mode = DADE_SCAN_FULL;
    o.max_K = K;
    o.max_nprobe = nprobe;
    o.first_wave = 1;
    o.status_dev = status.as<int32_t>();
    o.estimator = estimator;

    CollectArgs ca{};
    ca.seed = seed;
    ca.topk_stride = K;
    ca.n_label1 = cnt.as<unsigned long long>();
    ca.n_rows = cnt.as<unsigned long long>() + 1;

    // The collect replays write their own top-K to a scratch output.
    DevBuf scratch_ids;
    DADE_TRY(scratch_ids.alloc(sizeof(int64_t) * Bc * K));
    auto replay = [&](int pass) -> dade_status {
        for (int64_t b0 = 0; b0 < nt; b0 += Bc) {
            const int64_t B = std::min(Bc, nt - b0);
            DADE_CUDA_TRY(cudaMemcpyAsync(q.p, Tq + b0 * D, sizeof(float) * B * D, cudaMemcpyHostToDevice, st));
            int64_t* top = top_all.as<int64_t>() + b0 * K;
            if (pass < 0) {
                DADE_TRY(search_impl(idx, q.as<float>(), B, kk.as<int32_t>(), np.as<int32_t>(), delta_d, o, top,
                                     dists.as<float>(), nullptr, st, nullptr));
            } else {
                ca.pass = pass;
                ca.topk_ids = top;
                ca.query_offset = b0;
                DADE_TRY(search_impl(idx, q.as<float>(), B, kk.as<int32_t>(), np.as<int32_t>(), delta_d, o,
                                     scratch_ids.as<int64_t>(), dists.as<float>(), nullptr, st, &ca));
            }
        }
        DADE_CUDA_TRY(cudaStreamSynchronize(st));
        return DADE_OK;
    };

    DADE_TRY(replay(-1));  // (A) exact top-K
    DADE_TRY(replay(0));   // (B) count label-1
    unsigned long long counts[2] = {0, 0};
    DADE_CUDA_TRY(cudaMemcpy(counts, cnt.p, sizeof counts, cudaMemcpyDeviceToHost));
    const double n1 = (double)counts[0];
    ca.keep_rate = n1 > (double)label1_cap ? (double)label1_cap / n1 : 1.0;
    ca.row_cap = nt * K + label1_cap + (int64_t)(6.0 * sqrt((double)label1_cap)) + 1024;
    DevBuf rp, rt, rl, rq, ri;
    DADE_TRY(rp.alloc(sizeof(float) * ca.row_cap * ncols));
    DADE_TRY(rt.alloc(sizeof(float) * ca.row_cap));
    DADE_TRY(rl.alloc(sizeof(int8_t) * ca.row_cap));
    ca.partials = rp.as<float>();
    ca.tau = rt.as<float>();
    ca.label = rl.as<int8_t>();
    if (keys) {
        DADE_TRY(rq.alloc(sizeof(int64_t) * ca.row_cap));
        DADE_TRY(ri.alloc(sizeof(int64_t) * ca.row_cap));
        ca.query = rq.as<int64_t>();
        ca.id = ri.as<int64_t>();
    }
    DADE_TRY(replay(1));   // (C) emit samples
    DADE_CUDA_TRY(cudaMemcpy(counts, cnt.p, sizeof counts, cudaMemcpyDeviceToHost));
    int32_t dev_status = 0;
    DADE_CUDA_TRY(cudaMemcpy(&dev_status, status.p, sizeof dev_status, cudaMemcpyDeviceToHost));
    if (dev_status) return fail((dade_status)dev_status, "device status %d during the replay", dev_status);
    const int64_t n = std::min<int64_t>((int64_t)counts[1], ca.row_cap);
    std::vector<float> pf((size_t)n * ncols), tf((size_t)n);
    std::vector<int8_t> lab((size_t)n);
    DADE_CUDA_TRY(cudaMemcpy(pf.data(), rp.p, sizeof(float) * pf.size(), cudaMemcpyDeviceToHost));
    DADE_CUDA_TRY(cudaMemcpy(tf.data(), rt.p, sizeof(float) * tf.size(), cudaMemcpyDeviceToHost));
    DADE_CUDA_TRY(cudaMemcpy(lab.data(), rl.p, sizeof(int8_t) * lab.size(), cudaMemcpyDeviceToHost));
    std::vector<int64_t> qk, ik;
    if (keys) {
        qk.resize((size_t)n);
        ik.resize((size_t)n);
        DADE_CUDA_TRY(cudaMemcpy(qk.data(), rq.p, sizeof(int64_t) * (size_t)n, cudaMemcpyDeviceToHost));
        DADE_CUDA_TRY(cudaMemcpy(ik.data(), ri.p, sizeof(int64_t) * (size_t)n, cudaMemcpyDeviceToHost));
    }
    // rows arrive in atomic order: sort them so the fit is reproducible
    std::vector<int64_t> ord((size_t)n);
    std::iota(ord.begin(), ord.end(), 0);
    std::sort(ord.begin(), ord.end(), [&](int64_t a, int64_t b) {
        if (lab[a] != lab[b]) return lab[a] < lab[b];
        if (tf[a] != tf[b]) return tf[a] < tf[b];
        for (int s = 0; s < ncols; ++s) {
            float x = pf[(size_t)a * ncols + s], y = pf[(size_t)b * ncols + s];
            if (x != y) return x < y;
        }
        return false;
    });
    out->n = n;
    out->P.assign((size_t)n * ncols, 0.0);
    out->T.assign((size_t)n, 0.0);
    out->L.assign((size_t)n, 0);
    if (keys) {
        out->Qi.assign((size_t)n, 0);
        out->Id.assign((size_t)n, 0);
    }
    for (int64_t i = 0; i < n; ++i) {
        int64_t o2 = ord[(size_t)i];
        for (int s = 0; s < ncols; ++s) out->P[(size_t)i * ncols + s] = pf[(size_t)o2 * ncols + s];
        out->T[(size_t)i] = tf[(size_t)o2];
        out->L[(size_t)i] = lab[(size_t)o2];
        if (keys) {
            out->Qi[(size_t)i] = qk[(size_t)o2];
            out->Id[(size_t)i] = ik[(size_t)o2];
        }
    }
    return DADE_OK;
}

dade_status check_fit_args(const dade_index* idx, const float* Tq, int64_t nt, int32_t K, int32_t nprobe,
                           double target_recall, int64_t label1_cap) {
    if (!idx || !Tq) return fail(DADE_EINVAL, "null argument");
    if (nt < 1) return fail(DADE_EINVAL, "need training queries");
    if (K < 1 || K > kMaxK) return fail(DADE_EINVAL, "K out of range");
    if (nprobe < 1 || nprobe > std::min(idx->nlist, 1024)) return fail(DADE_EINVAL, "nprobe out of range");
    if (!(target_recall > 0 && target_recall <= 1)) return fail(DADE_EINVAL, "target_recall in (0, 1]");
    if (label1_cap < 1) return fail(DADE_EINVAL, "label1_cap must be >= 1");
    return DADE_OK;
}

}  // namespace

extern "C" dade_status dade_fit_correction(dade_index* idx, const float* Tq, int64_t nt, int32_t K,
                                           int32_t nprobe, int32_t delta_d, double target_recall,
                                           uint64_t seed, int64_t label1_cap, float* m1_out,
                                           float* beta_out) {
    clear_error();
    DADE_TRY(check_fit_args(idx, Tq, nt, K, nprobe, target_recall, label1_cap));
    if (delta_d != 8 && delta_d != 16 && delta_d != 32) return fail(DADE_EINVAL, "delta_d must be 8, 16 or 32");
    const int S = (int)ceil_div(idx->Dpad, delta_d);
    std::vector<float> m1f((size_t)std::max(1, S - 1), 0.f), btf((size_t)std::max(1, S - 1), -INFINITY);
    if (S <= 1) return install_table_public(idx, delta_d, S, m1f.data(), btf.data());
    Samples sm;
    DADE_TRY(replay_samples(idx, Tq, nt, K, nprobe, delta_d, seed, label1_cap, DADE_EST_LEARNED, S - 1, &sm));
    std::vector<double> m1d((size_t)S - 1), btd((size_t)S - 1);
    DADE_TRY(fit_tables(sm.P.data(), sm.T.data(), sm.L.data(), sm.n, S, target_recall, 100, m1d.data(), btd.data()));
    for (int s = 0; s < S - 1; ++s) {
        m1f[(size_t)s] = (float)m1d[(size_t)s];
        btf[(size_t)s] = (float)btd[(size_t)s];
    }
    DADE_TRY(install_table_public(idx, delta_d, S, m1f.data(), btf.data()));
    if (m1_out) std::copy(m1f.begin(), m1f.begin() + (S - 1), m1_out);
    if (beta_out) std::copy(btf.begin(), btf.begin() + (S - 1), beta_out);
    return DADE_OK;
}

extern "C" dade_status dade_fit_collect(dade_index* idx, const float* Tq, int64_t nt, int32_t K, int32_t nprobe,
                                        int32_t delta_d, uint64_t seed, int64_t label1_cap, int64_t max_rows,
                                        int64_t* n_rows, float* partials, float* tau, int8_t* label, int64_t* query,
                                        int64_t* id) {
    clear_error();
    DADE_TRY(check_fit_args(idx, Tq, nt, K, nprobe, 0.5, label1_cap));
    if (delta_d != 8 && delta_d != 16 && delta_d != 32) return fail(DADE_EINVAL, "delta_d must be 8, 16 or 32");
    if (!n_rows) return fail(DADE_EINVAL, "null n_rows");
    const int S = (int)ceil_div(idx->Dpad, delta_d);
    if (S <= 1) {
        *n_rows = 0;
        return DADE_OK;
    }
    Samples sm;
    DADE_TRY(replay_samples(idx, Tq, nt, K, nprobe, delta_d, seed, label1_cap, DADE_EST_LEARNED, S - 1, &sm, true));
    *n_rows = sm.n;
    if (sm.n > max_rows) return fail(DADE_EINVAL, "the replay kept %lld rows; max_rows is %lld", (long long)sm.n,
                                     (long long)max_rows);
    if (sm.n > 0 && (!partials || !tau || !label || !query || !id)) return fail(DADE_EINVAL, "null output");
    std::vector<int64_t> ord((size_t)sm.n);
    std::iota(ord.begin(), ord.end(), 0);
    std::sort(ord.begin(), ord.end(), [&](int64_t a, int64_t b) {
        if (sm.Qi[(size_t)a] != sm.Qi[(size_t)b]) return sm.Qi[(size_t)a] < sm.Qi[(size_t)b];
        return sm.Id[(size_t)a] < sm.Id[(size_t)b];
    });
    for (int64_t i = 0; i < sm.n; ++i) {
        const size_t o2 = (size_t)ord[(size_t)i];
        for (int s = 0; s < S - 1; ++s) partials[i * (S - 1) + s] = (float)sm.P[o2 * (S - 1) + s];
        tau[i] = (float)sm.T[o2];
        label[i] = sm.L[o2];
        query[i] = sm.Qi[o2];
        id[i] = sm.Id[o2];
    }
    return DADE_OK;
}

extern "C" dade_status dade_partials_collect(const dade_index* idx, const float* Q_host, int64_t nq, int32_t nprobe,
                                             int32_t delta_d, int64_t max_rows, int64_t* n_rows, float* partials,
                                             int64_t* query, int64_t* id) {
    clear_error();
    if (!idx || !n_rows) return fail(DADE_EINVAL, "null index or n_rows");
    if (nq < 0 || max_rows < 0) return fail(DADE_EINVAL, "nq and max_rows must be >= 0");
    if (nq > 0 && !Q_host) return fail(DADE_EINVAL, "null queries");
    if (nprobe < 1 || nprobe > idx->nlist) return fail(DADE_EINVAL, "nprobe must be in [1, nlist]");
    if (delta_d != 8 && delta_d != 16 && delta_d != 32) return fail(DADE_EINVAL, "delta_d must be 8, 16 or 32");
    *n_rows = 0;
    const int S = (int)ceil_div(idx->Dpad, delta_d);
    if (nq == 0 || S <= 1) return DADE_OK;
    if (max_rows > 0 && (!partials || !query || !id)) return fail(DADE_EINVAL, "null output");

    cudaStream_t st;
    DADE_CUDA_TRY(cudaStreamCreateWithFlags(&st, cudaStreamNonBlocking));
    struct G {
        const dade_index* idx;
        cudaStream_t s;
        ~G() {
            idx->ws.drop(s);
            cudaStreamDestroy(s);
        }
    } guard{idx, st};
    const int64_t Bc = std::min<int64_t>(nq, 1024);
    const int D = idx->D;
    const int64_t cap = std::max<int64_t>(1, max_rows);
    DevBuf q, kk, np, ids, dists, cnt, status, rp, rq, ri;
    DADE_TRY(q.alloc(sizeof(float) * Bc * D));
    DADE_TRY(kk.alloc(sizeof(int32_t) * Bc));
    DADE_TRY(np.alloc(sizeof(int32_t) * Bc));
    DADE_TRY(ids.alloc(sizeof(int64_t) * Bc));
    DADE_TRY(dists.alloc(sizeof(float) * Bc));
    DADE_TRY(cnt.alloc(sizeof(unsigned long long) * 2));
    DADE_TRY(status.alloc(sizeof(int32_t)));
    DADE_TRY(rp.alloc(sizeof(float) * cap * (S - 1)));
    DADE_TRY(rq.alloc(sizeof(int64_t) * cap));
    DADE_TRY(ri.alloc(sizeof(int64_t) * cap));
    {
        std::vector<int32_t> kh((size_t)Bc, 1), nh((size_t)Bc, nprobe);
        DADE_CUDA_TRY(cudaMemcpy(kk.p, kh.data(), sizeof(int32_t) * Bc, cudaMemcpyHostToDevice));
        DADE_CUDA_TRY(cudaMemcpy(np.p, nh.data(), sizeof(int32_t) * Bc, cudaMemcpyHostToDevice));
        DADE_CUDA_TRY(cudaMemset(cnt.p, 0, sizeof(unsigned long long) * 2));
        DADE_CUDA_TRY(cudaMemset(status.p, 0, sizeof(int32_t)));
    }
    // one wave over all nprobe buckets, pruning off: every candidate is
    // visited once and emitted with its partial distances
    dade_search_opts o{};
    o.mode = DADE_SCAN_FULL;
    o.max_K = 1;
    o.max_nprobe = nprobe;
    o.first_wave = nprobe;
    o.status_dev = status.as<int32_t>();
    CollectArgs ca{};
    ca.pass = 1;
    ca.keep_all = 1;
    ca.keep_rate = 1.0;
    ca.n_label1 = cnt.as<unsigned long long>();
    ca.n_rows = cnt.as<unsigned long long>() + 1;
    ca.row_cap = max_rows;
    ca.partials = rp.as<float>();
    ca.query = rq.as<int64_t>();
    ca.id = ri.as<int64_t>();
    for (int64_t b0 = 0; b0 < nq; b0 += Bc) {
        const int64_t B = std::min(Bc, nq - b0);
        DADE_CUDA_TRY(cudaMemcpyAsync(q.p, Q_host + b0 * D, sizeof(float) * B * D, cudaMemcpyHostToDevice, st));
        ca.query_offset = b0;
        DADE_TRY(search_impl(idx, q.as<float>(), B, kk.as<int32_t>(), np.as<int32_t>(), delta_d, o,
                             ids.as<int64_t>(), dists.as<float>(), nullptr, st, &ca));
        DADE_CUDA_TRY(cudaStreamSynchronize(st));
    }
    unsigned long long counts[2] = {0, 0};
    DADE_CUDA_TRY(cudaMemcpy(counts, cnt.p, sizeof counts, cudaMemcpyDeviceToHost));
    int32_t dev_status = 0;
    DADE_CUDA_TRY(cudaMemcpy(&dev_status, status.p, sizeof dev_status, cudaMemcpyDeviceToHost));
    if (dev_status) return fail((dade_status)dev_status, "device status %d during the collection", dev_status);
    const int64_t n = (int64_t)counts[1];
    *n_rows = n;
    if (n > max_rows) return fail(DADE_EINVAL, "%lld candidate rows; max_rows is %lld", (long long)n,
                                  (long long)max_rows);
    std::vector<float> pf((size_t)n * (S - 1));
    std::vector<int64_t> qh((size_t)n), ih((size_t)n);
    if (n > 0) {
        DADE_CUDA_TRY(cudaMemcpy(pf.data(), rp.p, sizeof(float) * n * (S - 1), cudaMemcpyDeviceToHost));
        DADE_CUDA_TRY(cudaMemcpy(qh.data(), rq.p, sizeof(int64_t) * n, cudaMemcpyDeviceToHost));
        DADE_CUDA_TRY(cudaMemcpy(ih.data(), ri.p, sizeof(int64_t) * n, cudaMemcpyDeviceToHost));
    }
    std::vector<int64_t> ord((size_t)n);
    std::iota(ord.begin(), ord.end(), 0);
    std::sort(ord.begin(), ord.end(), [&](int64_t a, int64_t b) {
        if (qh[(size_t)a] != qh[(size_t)b]) return qh[(size_t)a] < qh[(size_t)b];
        return ih[(size_t)a] < ih[(size_t)b];
    });
    for (int64_t i = 0; i < n; ++i) {
        const size_t o2 = (size_t)ord[(size_t)i];
        std::copy(pf.begin() + o2 * (S - 1), pf.begin() + (o2 + 1) * (S - 1), partials + i * (S - 1));
        query[i] = qh[o2];
        id[i] = ih[o2];
    }
    return DADE_OK;
}

extern "C" dade_status dade_pq_fit_correction(dade_index* idx, const float* Tq, int64_t nt, int32_t K, int32_t nprobe,
                                              double target_recall, uint64_t seed, int64_t label1_cap, float* out3) {
    clear_error();
    DADE_TRY(check_fit_args(idx, Tq, nt, K, nprobe, target_recall, label1_cap));
    if (idx->pq_m <= 0) return fail(DADE_ESTATE, "the index has no product quantiser");
    Samples sm;
    DADE_TRY(replay_samples(idx, Tq, nt, K, nprobe, 16, seed, label1_cap, DADE_EST_PQ, 2, &sm));
    std::vector<double> dis((size_t)sm.n), err((size_t)sm.n);
    for (int64_t i = 0; i < sm.n; ++i) {
        dis[(size_t)i] = sm.P[(size_t)i * 2];
        err[(size_t)i] = sm.P[(size_t)i * 2 + 1];
    }
    double th[3];
    DADE_TRY(fit_pq_host(dis.data(), err.data(), sm.T.data(), sm.L.data(), sm.n, target_recall, 100, th));
    idx->pq_m1 = (float)th[0];
    idx->pq_m3 = (float)th[1];
    idx->pq_beta = (float)th[2];
    idx->pq_has_table = true;
    if (out3) {
        out3[0] = idx->pq_m1;
        out3[1] = idx->pq_m3;
        out3[2] = idx->pq_beta;
    }
    return DADE_OK;
}
