// dade_search: the batched search pipeline on one stream.
//   rotate queries (GEMM) -> centroid distances (GEMM) -> top-nprobe select
//   -> work units per wave -> per wave: estimate-and-prune scan, top-K merge
//   -> output.
// Every launch goes to the caller's stream; nothing synchronises the host.
#include <algorithm>
#include <mutex>
#include <utility>
#include <vector>

#include "dade_internal.h"
#include "kernels/scan.cuh"

namespace dade {
namespace {

// Stage timing state (process-wide): event pairs around scan launches and a
// device counter of staged bytes.
struct StageTiming {
    std::mutex mu;
    bool on = false;
    bool only_tensor = false;  // time the tensor-core scan launches alone
    std::vector<std::pair<cudaEvent_t, cudaEvent_t>> ev;
    unsigned long long* bytes = nullptr;
};
StageTiming& timing() {
    static StageTiming t;
    return t;
}

struct Carve {
    char* base;
    size_t off = 0;
    template <class T> T* take(size_t n) {
        off = (size_t)round_up((int64_t)off, 256);
        T* p = base ? reinterpret_cast<T*>(base + off) : nullptr;
        off += n * sizeof(T);
        return p;
    }
};

struct Plan {
    WaveView wv{};
    int pass_wave[kMaxPasses] = {};   // the wave of each pass
    bool pass_new[kMaxPasses] = {};   // the pass starts its wave (tau is taken then)
    float* pq_lut = nullptr;   // B x m x 256 (OPQ-L)
    float* scores = nullptr;
    float* qnorm = nullptr;
    bool cent_tc = false;        // centroid distances by the pipelined kernel on pre-split operands
    float* qtc = nullptr;        // query TF32 parts in canonical chunks
    float* tmin = nullptr;       // B x ceil(nlist / 128) x 4: each centroid tile's 4 smallest distances
    char* zero_begin = nullptr;
    size_t zero_bytes = 0;
    int32_t* status_internal = nullptr;
    int64_t cand_cap = 0;
};

// Upper bound of a query's candidates in a pass of n probe ranks: the sum
// of the n largest bucket sizes.
int64_t pass_bound(const dade_index* idx, int n) { return idx->sizes_desc_prefix[std::max(0, std::min(n, idx->nlist))]; }

// Default bound of the candidate buffer (distance and slot, 8 bytes per
// entry): a wave whose worst case exceeds it is scanned in several passes.
constexpr int64_t kDefaultCandidateBudget = int64_t(8) << 30;

// The passes of the wave schedule: every wave [b, e) of probe ranks is cut
// into the fewest passes of equal width (up to one rank) whose worst-case
// candidates for B queries fit the budget (at least one rank per pass); if
// that makes more than kMaxPasses passes the budget is doubled.
void make_passes(const dade_index* idx, int64_t B, int P, int f, int g, int64_t budget, WaveView& v, Plan* pl) {
    const int nw = num_waves(P, f, g);
    for (;;) {
        int np = 0;
        bool fits = true;
        for (int w = 0; w < nw && fits; ++w) {
            const int b0 = wave_begin(w, f, g), b1 = std::min(P, wave_begin(w + 1, f, g));
            const int width = std::max(0, b1 - b0);
            auto fits_in = [&](int h) { return (double)B * (double)pass_bound(idx, h) * 8.0 <= (double)budget; };
            int lo = 1, hi = std::max(1, width);  // largest width that fits (1 if none)
            while (lo < hi) {
                const int mid = (lo + hi + 1) / 2;
                if (fits_in(mid)) lo = mid; else hi = mid - 1;
            }
            const int npass = (width + lo - 1) / std::max(1, lo);
            const int h = npass > 0 ? (width + npass - 1) / npass : 1;
            for (int r = b0; r < b1; r += h) {
                if (np == kMaxPasses) {
                    fits = false;
                    break;
                }
                v.pass_begin[np] = r;
                pl->pass_wave[np] = w;
                pl->pass_new[np] = r == b0;
                ++np;
            }
        }
        if (fits) {
            v.pass_begin[np] = P;
            v.n_waves = np;
            return;
        }
        budget *= 2;
    }
}

// The RES test is in use (PRUNE mode with estimator RES).
bool uses_res(const dade_search_opts& o) { return o.mode == DADE_SCAN_PRUNE && o.estimator == DADE_EST_RES; }

// Steps of the estimate: ceil(Dpad / delta_d); OPQ-L has one test (S = 2).
int n_steps(const dade_index* idx, int32_t delta_d, const dade_search_opts& o) {
    if (o.estimator == DADE_EST_PQ) return 2;
    return (int)ceil_div(idx->Dpad, delta_d > 0 ? delta_d : idx->Dpad);
}

// The tensor-core kernel can run the learned test's waves of this search.
bool tc_eligible(const dade_index* idx, int32_t delta_d, const dade_search_opts& o) {
    return o.mode == DADE_SCAN_PRUNE && o.estimator == DADE_EST_LEARNED && idx->tcslab_dev.p &&
           tc_scan_supported(delta_d);
}

enum WaveKernel { WK_EXACT = 0, WK_CUDA = 1, WK_TENSOR = 2, WK_PQ = 3 };

// Which kernel scans wave w: every candidate's exact distance (a full scan,
// a wave whose tau is +inf for every query, or no test to run), the OPQ-L
// scan, or the learned / RES test on the CUDA cores or the tensor cores.
int wave_kernel(const dade_index* idx, int32_t delta_d, const dade_search_opts& o, int wave) {
    const int S = n_steps(idx, delta_d, o);
    if (o.mode == DADE_SCAN_FULL || S <= 1 || (wave == 0 && o.tau_dev == nullptr)) return WK_EXACT;
    if (o.estimator == DADE_EST_PQ) return WK_PQ;
    if (tc_eligible(idx, delta_d, o) && o.scan_kernel != DADE_KERNEL_CUDA) return WK_TENSOR;
    return WK_CUDA;
}

// Queries per work unit of a wave: the tensor-core kernel takes up to 128
// or 256 (its MMA N), the CUDA-core kernels kG.
int wave_qgroup(int kernel, int32_t delta_d, int32_t requested) {
    const int qmax = kernel == WK_TENSOR ? tc_scan_qmax(delta_d) : kG;
    return requested > 0 ? std::min<int>(requested, qmax) : qmax;
}

size_t carve(const dade_index* idx, int64_t B, int32_t delta_d, const dade_search_opts& o, char* base, Plan* pl) {
    const int P = o.max_nprobe, Kmax = o.max_K;
    const bool frozen = o.tau_dev != nullptr;
    const int f = frozen ? P : std::max(1, o.first_wave);
    const int g = std::max(1, o.wave_growth_log2);
    const int64_t nl = idx->nlist;
    Carve c{base};
    WaveView& v = pl->wv;
    make_passes(idx, B, P, f, g, o.candidate_budget_bytes > 0 ? o.candidate_budget_bytes : kDefaultCandidateBudget, v,
                pl);
    const int nw = v.n_waves;  // passes
    int64_t cap_per_q = 0;
    for (int w = 0; w < nw; ++w) cap_per_q = std::max(cap_per_q, pass_bound(idx, v.pass_begin[w + 1] - v.pass_begin[w]));
    v.B = B;
    v.P = P;
    v.Kmax = Kmax;
    v.final_test = o.final_test != 0;
    v.est = uses_res(o) ? 1 : 0;
    v.res_stride = v.est ? (int)ceil_div(idx->Dpad, delta_d) - 1 : 0;
    {
        const int all = delta_d > 0 ? (int)ceil_div(idx->Dpad, delta_d) - 1 : 0;
        v.test_steps = o.test_steps > 0 ? std::min(all, (int)o.test_steps) : all;
    }
    v.qrot = c.take<float>((size_t)B * idx->Dpad);
    v.qpad = c.take<float>((size_t)B * idx->Dpad);
    pl->scores = o.probe_in_dev ? nullptr : c.take<float>((size_t)B * nl);
    pl->qnorm = o.probe_in_dev ? nullptr : c.take<float>((size_t)B);
    pl->cent_tc = !o.probe_in_dev && idx->cent_tc_dev.p && centroid_tc_supported(idx->Dpad);
    if (pl->cent_tc) {
        pl->qtc = c.take<float>((size_t)ceil_div(B, 128) * (idx->Dpad / 8) * 2 * 1024);
        pl->tmin = c.take<float>((size_t)B * ceil_div(nl, 128) * 4);
    }
    v.probes = c.take<int32_t>((size_t)B * P);
    v.off_wl = c.take<int32_t>((size_t)nw * nl + 1);
    v.items = c.take<int32_t>((size_t)B * P);
    v.unit_off = c.take<int32_t>((size_t)nw * (nl + 1));
    // unit descriptors: a wave has at most (items / kG + buckets touched) groups,
    // each with ceil(largest bucket / kT) tiles
    const int64_t ntile_max = std::max<int64_t>(1, ceil_div(idx->max_list, kT));
    int64_t ucap = 0;
    for (int w = 0; w < nw; ++w) {
        const int64_t width = v.pass_begin[w + 1] - v.pass_begin[w];
        const int qg = wave_qgroup(wave_kernel(idx, delta_d, o, pl->pass_wave[w]), delta_d, o.queries_per_unit);
        v.ubase[w] = ucap;
        v.qgroup[w] = qg;
        ucap += (ceil_div(B * width, qg) + std::min<int64_t>(nl, B * width)) * ntile_max;
    }
    v.units = c.take<int4>((size_t)std::max<int64_t>(1, ucap));
    pl->cand_cap = B * cap_per_q;
    v.cand_d = c.take<float>((size_t)std::max<int64_t>(1, pl->cand_cap));
    v.cand_pos = c.take<int32_t>((size_t)std::max<int64_t>(1, pl->cand_cap));
    v.top_d = c.take<float>((size_t)B * Kmax);
    v.top_id = c.take<int64_t>((size_t)B * Kmax);
    v.tau = c.take<float>((size_t)B);
    v.tau_run = c.take<float>((size_t)B);
    v.res_q = v.res_stride > 0 ? c.take<float>((size_t)B * v.res_stride) : nullptr;
    pl->pq_lut = o.estimator == DADE_EST_PQ ? c.take<float>((size_t)B * idx->pq_m * 256) : nullptr;
    // zero-initialised block
    c.off = (size_t)round_up((int64_t)c.off, 256);
    size_t z0 = c.off;
    v.cnt_wl = c.take<int32_t>((size_t)nw * nl);
    v.fill_wl = c.take<int32_t>((size_t)nw * nl);
    v.cand_off = c.take<int64_t>((size_t)nw * (B + 1));
    v.cand_cnt = c.take<int32_t>((size_t)B);
    v.top_n = c.take<int32_t>((size_t)B);
    v.work = c.take<int32_t>((size_t)2 * nw + 4);  // + one 8-byte item counter of the OPQ-L scan
    pl->status_internal = c.take<int32_t>(1);
    pl->zero_begin = base ? base + z0 : nullptr;
    pl->zero_bytes = c.off - z0;
    return c.off + 256;
}

}  // namespace

dade_status check_args(const dade_index* idx, int64_t B, int32_t delta_d, const dade_search_opts& o) {
    if (!idx) return fail(DADE_EINVAL, "null index");
    if (B < 0 || B > (int64_t)1 << 24) return fail(DADE_EINVAL, "B out of range: %lld", (long long)B);
    if (o.max_K < 1 || o.max_K > kMaxK) return fail(DADE_EINVAL, "max_K must be in [1, %d]", kMaxK);
    if (o.max_nprobe < 1 || o.max_nprobe > std::min(idx->nlist, 1024))
        return fail(DADE_EINVAL, "max_nprobe must be in [1, min(nlist, 1024)]");
    if (o.mode != DADE_SCAN_PRUNE && o.mode != DADE_SCAN_FULL) return fail(DADE_EINVAL, "bad mode");
    if (o.first_wave < 0) return fail(DADE_EINVAL, "first_wave < 0");
    if (o.candidate_budget_bytes < 0) return fail(DADE_EINVAL, "candidate_budget_bytes < 0");
    if (o.queries_per_unit < 0) return fail(DADE_EINVAL, "queries_per_unit < 0");
    if (o.wave_growth_log2 < 0 || o.wave_growth_log2 > 30) return fail(DADE_EINVAL, "wave_growth_log2 must be in [0, 30]");
    if (o.estimator != DADE_EST_LEARNED && o.estimator != DADE_EST_RES && o.estimator != DADE_EST_PQ)
        return fail(DADE_EINVAL, "bad estimator");
    if (o.estimator == DADE_EST_PQ) {
        if (idx->pq_m <= 0) return fail(DADE_ESTATE, "the index has no product quantiser (dade_pq_train / dade_pq_set)");
        if (o.mode == DADE_SCAN_PRUNE && !idx->pq_has_table)
            return fail(DADE_ESTATE, "no OPQ-L correction (dade_pq_fit_correction / dade_pq_set_correction)");
        if (o.mode == DADE_SCAN_PRUNE && (o.final_test || o.test_steps))
            return fail(DADE_ENOTIMPL, "OPQ-L has one test: no final_test or test_steps");
    }
    if (o.scan_kernel < DADE_KERNEL_AUTO || o.scan_kernel > DADE_KERNEL_TENSOR) return fail(DADE_EINVAL, "bad scan_kernel");
    if (o.scan_kernel == DADE_KERNEL_TENSOR && o.mode == DADE_SCAN_PRUNE && !tc_eligible(idx, delta_d, o))
        return fail(DADE_ENOTIMPL, "the tensor-core scan runs the learned test (tables or ADS) only");
    if (o.test_steps < 0) return fail(DADE_EINVAL, "test_steps < 0");
    if (o.test_steps > 0 && o.final_test && o.mode == DADE_SCAN_PRUNE)
        return fail(DADE_ENOTIMPL, "test_steps with final_test");
    if (o.estimator == DADE_EST_RES && !(o.res_m >= 0.f && o.res_m < INFINITY))
        return fail(DADE_EINVAL, "res_m must be finite and >= 0");
    if (o.mode == DADE_SCAN_PRUNE && o.estimator != DADE_EST_PQ) {
        if (delta_d != 8 && delta_d != 16 && delta_d != 32)
            return fail(DADE_EINVAL, "delta_d must be 8, 16 or 32 (got %d)", delta_d);
        int S = (int)ceil_div(idx->Dpad, delta_d);
        if (S > 1 && o.estimator == DADE_EST_LEARNED && !idx->tables.count(delta_d))
            return fail(DADE_ESTATE, "no correction table for delta_d = %d", delta_d);
    }
    return DADE_OK;
}

size_t workspace_bytes(const dade_index* idx, int64_t B, int32_t delta_d, const dade_search_opts& o,
                       const CollectArgs*) {
    Plan pl;
    return carve(idx, B, delta_d, o, nullptr, &pl);
}

dade_status search_impl(const dade_index* idx, const float* Q, int64_t B, const int32_t* K_dev,
                        const int32_t* nprobe_dev, int32_t delta_d, const dade_search_opts& o,
                        int64_t* ids_dev, float* dists_dev, const int64_t* offsets, cudaStream_t st,
                        const CollectArgs* collect) {
    DADE_TRY(check_args(idx, B, delta_d, o));
    if (B == 0) return DADE_OK;
    if (!Q || !K_dev || !nprobe_dev || !ids_dev || !dists_dev) return fail(DADE_EINVAL, "null buffer");
    Plan pl;
    size_t need = carve(idx, B, delta_d, o, nullptr, &pl);
    char* base;
    std::unique_lock<std::mutex> ws_lock;
    if (o.workspace) {
        if (o.workspace_bytes < need)
            return fail(DADE_EINVAL, "workspace too small: %zu < %zu bytes", o.workspace_bytes, need);
        base = static_cast<char*>(o.workspace);
    } else {
        // this stream's own scratch, held until every launch is enqueued
        StreamWorkspaces::Buf* wb = idx->ws.of(st);
        ws_lock = std::unique_lock<std::mutex>(wb->mu);
        if (wb->bytes < need) {
            if (wb->p) DADE_CUDA_TRY(cudaFreeAsync(wb->p, st));
            wb->p = nullptr;
            wb->bytes = 0;
            cudaError_t e = cudaMallocAsync(&wb->p, need, st);
            if (e != cudaSuccess) {
                wb->p = nullptr;
                cudaGetLastError();
                return fail(DADE_ENOMEM, "cudaMallocAsync(%zu) failed: %s", need, cudaGetErrorString(e));
            }
            wb->bytes = need;
        }
        base = static_cast<char*>(wb->p);
    }
    base = reinterpret_cast<char*>(round_up(reinterpret_cast<int64_t>(base), 256));
    carve(idx, B, delta_d, o, base, &pl);
    WaveView& v = pl.wv;
    v.nprobe = nprobe_dev;
    v.K = K_dev;
    v.status = o.status_dev ? o.status_dev : pl.status_internal;
    v.stats = o.stats_dev;
    StageTiming& tm = timing();
    const bool timed = tm.on && !collect;
    v.staged_bytes = timed ? tm.bytes : nullptr;

    IndexView ix;
    ix.slab = idx->slab_dev.p;
    ix.orig = idx->orig_dev.as<float>();
    ix.ids = idx->ids_dev.as<int64_t>();
    ix.list_slot = idx->list_slot_dev.as<int64_t>();
    ix.list_size = idx->list_size_dev.as<int32_t>();
    ix.scale = idx->scale_dev.as<float>();
    ix.eps = idx->dtype == DADE_SLAB_F32 ? nullptr : idx->eps_dev.as<float>();
    ix.sfx = idx->sfx_dev.as<float>();
    ix.tcslab = idx->tcslab_dev.as<float>();
    ix.tile_base = idx->tile_base_dev.as<int64_t>();
    ix.total_slots = idx->total_slots;
    ix.D = idx->D;
    ix.Dpad = idx->Dpad;
    ix.nb = idx->nb;
    ix.nlist = idx->nlist;
    ix.dtype = idx->dtype;
    ix.tc_parts = idx->tc_parts;
    ix.ids32 = idx->ids32;

    const bool full = o.mode == DADE_SCAN_FULL;
    const bool pq = o.estimator == DADE_EST_PQ;
    // OPQ-L has one test whatever delta_d is (S = 2: one test, then the exact distance)
    const int S = n_steps(idx, delta_d, o);
    const float *m1 = nullptr, *beta = nullptr;
    if (!full && S > 1 && !v.est && !pq) {
        const CorrectionTable& tb = idx->tables.at(delta_d);
        m1 = tb.m1_dev;
        beta = tb.beta_dev;
    }

    DADE_CUDA_TRY(cudaMemsetAsync(pl.zero_begin, 0, pl.zero_bytes, st));
    if (o.tau_dev)
        DADE_CUDA_TRY(cudaMemcpyAsync(v.tau, o.tau_dev, sizeof(float) * B, cudaMemcpyDeviceToDevice, st));
    else
        DADE_CUDA_TRY(launch_fill(v.tau, B, INFINITY, st));
    DADE_CUDA_TRY(launch_fill(v.tau_run, B, INFINITY, st));

    // 1. q' = R (q - mean); the original query zero-padded to Dpad
    DADE_CUDA_TRY(launch_tc_dot(Q, idx->D, idx->mean_dev.as<float>(), idx->R_dev.as<float>(), idx->Dpad,
                                const_cast<float*>(v.qrot), idx->Dpad, B, idx->Dpad, idx->D, v.status, st));
    DADE_CUDA_TRY(launch_prepare_queries(Q, B, idx->D, idx->Dpad, const_cast<float*>(v.qpad), st));
    if (pq)
        DADE_CUDA_TRY(launch_pq_lut(v.qrot, B, idx->Dpad, idx->pq_perm_dev.as<int32_t>(), idx->pq_cb_dev.as<float>(),
                                    idx->pq_m, idx->pq_ds, pl.pq_lut, st));
    if (v.est)
        DADE_CUDA_TRY(launch_res_terms(v.qrot, B, idx->D, idx->Dpad, idx->var_dev.as<float>(), delta_d, S, o.res_m,
                                       const_cast<float*>(v.res_q), st));
    if (o.qrot_out_dev) {
        DADE_CUDA_TRY(cudaMemcpy2DAsync(o.qrot_out_dev, sizeof(float) * idx->D, v.qrot,
                                        sizeof(float) * idx->Dpad, sizeof(float) * idx->D, B,
                                        cudaMemcpyDeviceToDevice, st));
    }
    // 2. buckets to probe
    if (o.probe_in_dev) {
        DADE_CUDA_TRY(cudaMemcpyAsync(const_cast<int32_t*>(v.probes), o.probe_in_dev,
                                      sizeof(int32_t) * B * v.P, cudaMemcpyDeviceToDevice, st));
    } else {
        DADE_CUDA_TRY(launch_row_norms(v.qrot, idx->Dpad, B, idx->Dpad, pl.qnorm, st));
        if (pl.cent_tc) {
            DADE_CUDA_TRY(launch_split_tc(v.qrot, idx->Dpad, B, idx->Dpad, pl.qtc, st));
            DADE_CUDA_TRY(launch_centroid_dist_tc(pl.qtc, idx->cent_tc_dev.as<float>(), pl.qnorm,
                                                  idx->cnorm_dev.as<float>(), B, idx->nlist, idx->Dpad, pl.scores,
                                                  pl.tmin, v.status, st));
        } else {
            DADE_CUDA_TRY(launch_tc_l2(v.qrot, idx->Dpad, pl.qnorm, idx->cent_dev.as<float>(), idx->Dpad,
                                       idx->cnorm_dev.as<float>(), pl.scores, idx->nlist, B, idx->nlist, idx->Dpad,
                                       v.status, st));
        }
        DADE_CUDA_TRY(launch_select_probes(pl.scores, B, idx->nlist, nprobe_dev, v.P,
                                           const_cast<int32_t*>(v.probes), v.status, st, pl.tmin));
    }
    if (o.probe_out_dev)
        DADE_CUDA_TRY(cudaMemcpyAsync(o.probe_out_dev, v.probes, sizeof(int32_t) * B * v.P,
                                      cudaMemcpyDeviceToDevice, st));
    // 3. work units of every wave
    DADE_CUDA_TRY(launch_build_units(ix, v, st));
    // 4-5. waves
    for (int w = 0; w < v.n_waves; ++w) {
        // a new wave tests against the top-K's K-th distance as the previous
        // waves left it; the passes of one wave share that tau
        if (w > 0 && pl.pass_new[w] && !o.tau_dev)
            DADE_CUDA_TRY(cudaMemcpyAsync(v.tau, v.tau_run, sizeof(float) * B, cudaMemcpyDeviceToDevice, st));
        if (collect) {
            CollectArgs ca = *collect;
            if (pq) {
                ca.pq_m = idx->pq_m;
                ca.pq_codes = idx->pq_codes_dev.as<uint8_t>();
                ca.pq_err = idx->pq_err_dev.as<float>();
                ca.pq_lut = pl.pq_lut;
            }
            DADE_CUDA_TRY(launch_collect(ix, v, w, delta_d, S, ca, collect->query_offset, st));
        }
        // wave 0 has tau = +inf for every query (no frozen tau): every
        // candidate's exact distance, through the full-scan kernel
        const int wk = wave_kernel(idx, delta_d, o, pl.pass_wave[w]);
        const bool timed_here = timed && (tm.only_tensor == 0 || wk == WK_TENSOR);
        v.staged_bytes = timed_here ? tm.bytes : nullptr;
        cudaEvent_t e0 = nullptr, e1 = nullptr;
        if (timed_here) {
            DADE_CUDA_TRY(cudaEventCreate(&e0));
            DADE_CUDA_TRY(cudaEventCreate(&e1));
            DADE_CUDA_TRY(cudaEventRecord(e0, st));
        }
        if (wk == WK_PQ) {
            PQView pv{idx->pq_codes_dev.as<uint8_t>(), idx->pq_err_dev.as<float>(), pl.pq_lut, idx->total_slots,
                      idx->pq_m, idx->pq_m1, idx->pq_m3, idx->pq_beta};
            DADE_CUDA_TRY(launch_pq_scan(ix, v, w, pv, st));
        } else if (wk == WK_TENSOR) {
            DADE_CUDA_TRY(launch_wave_scan_tc(ix, v, w, delta_d, m1, beta, v.final_test ? S : v.test_steps,
                                              idx->tc_parts, v.final_test != 0, st));
        } else {
            DADE_CUDA_TRY(launch_wave_scan(ix, v, w, wk == WK_EXACT, delta_d, m1, beta, S, st));
        }
        if (timed_here) {
            DADE_CUDA_TRY(cudaEventRecord(e1, st));
            std::lock_guard<std::mutex> lk(tm.mu);
            tm.ev.emplace_back(e0, e1);
        }
        DADE_CUDA_TRY(launch_merge(ix, v, w, st));
    }
    DADE_CUDA_TRY(launch_output(v, ids_dev, dists_dev, offsets, st));
    return DADE_OK;
}

}  // namespace dade

extern "C" dade_status dade_search(const dade_index* idx, const float* Q_dev, int64_t B,
                                   const int32_t* K_dev, const int32_t* nprobe_dev, int32_t delta_d,
                                   const dade_search_opts* opts, int64_t* ids_dev, float* dists_dev,
                                   const int64_t* out_offsets_dev, void* cuda_stream) {
    dade::clear_error();
    if (!opts) return dade::fail(DADE_EINVAL, "opts is required (max_K, max_nprobe)");
    return dade::search_impl(idx, Q_dev, B, K_dev, nprobe_dev, delta_d, *opts, ids_dev, dists_dev,
                             out_offsets_dev, static_cast<cudaStream_t>(cuda_stream), nullptr);
}

extern "C" dade_status dade_search_kernel_count(const dade_index* idx, const float* Q_dev, int64_t B,
                                               const int32_t* K_dev, const int32_t* nprobe_dev, int32_t delta_d,
                                               const dade_search_opts* opts, int64_t* ids_dev, float* dists_dev,
                                               const int64_t* out_offsets_dev, int64_t* count) {
    dade::clear_error();
    if (!opts || !count) return dade::fail(DADE_EINVAL, "opts and count are required");
    if (!opts->workspace) return dade::fail(DADE_EINVAL, "a workspace is required to count launches");
    cudaStream_t st = nullptr;
    DADE_CUDA_TRY(cudaStreamCreateWithFlags(&st, cudaStreamNonBlocking));
    cudaGraph_t g = nullptr;
    cudaError_t e = cudaStreamBeginCapture(st, cudaStreamCaptureModeThreadLocal);
    dade_status s = DADE_OK;
    if (e == cudaSuccess) {
        s = dade::search_impl(idx, Q_dev, B, K_dev, nprobe_dev, delta_d, *opts, ids_dev, dists_dev,
                              out_offsets_dev, st, nullptr);
        e = cudaStreamEndCapture(st, &g);
    }
    int64_t n = 0;
    if (e == cudaSuccess && s == DADE_OK && g) {
        size_t nn = 0;
        e = cudaGraphGetNodes(g, nullptr, &nn);
        std::vector<cudaGraphNode_t> nodes(nn);
        if (e == cudaSuccess && nn) e = cudaGraphGetNodes(g, nodes.data(), &nn);
        for (size_t i = 0; e == cudaSuccess && i < nn; ++i) {
            cudaGraphNodeType t;
            e = cudaGraphNodeGetType(nodes[i], &t);
            if (e == cudaSuccess && t == cudaGraphNodeTypeKernel) ++n;
        }
    }
    if (g) cudaGraphDestroy(g);
    cudaStreamDestroy(st);
    if (s != DADE_OK) return s;
    if (e != cudaSuccess) {
        cudaGetLastError();
        return dade::fail(DADE_ECUDA, "graph capture for the launch count: %s", cudaGetErrorString(e));
    }
    *count = n;
    return DADE_OK;
}

extern "C" dade_status dade_stage_timing(int32_t enable) {
    dade::clear_error();
    dade::StageTiming& t = dade::timing();
    std::lock_guard<std::mutex> lk(t.mu);
    if (enable && !t.bytes) {
        DADE_CUDA_TRY(cudaMalloc(&t.bytes, sizeof(unsigned long long)));
        DADE_CUDA_TRY(cudaMemset(t.bytes, 0, sizeof(unsigned long long)));
    }
    t.on = enable != 0;
    t.only_tensor = enable == 2;
    return DADE_OK;
}

extern "C" dade_status dade_stage_timing_read(double* scan_ms, int64_t* launches, double* bytes) {
    dade::clear_error();
    dade::StageTiming& t = dade::timing();
    std::lock_guard<std::mutex> lk(t.mu);
    double ms = 0;
    for (auto& e : t.ev) {
        DADE_CUDA_TRY(cudaEventSynchronize(e.second));
        float x = 0;
        DADE_CUDA_TRY(cudaEventElapsedTime(&x, e.first, e.second));
        ms += x;
        cudaEventDestroy(e.first);
        cudaEventDestroy(e.second);
    }
    if (launches) *launches = (int64_t)t.ev.size();
    t.ev.clear();
    unsigned long long b = 0;
    if (t.bytes) {
        DADE_CUDA_TRY(cudaMemcpy(&b, t.bytes, sizeof b, cudaMemcpyDeviceToHost));
        DADE_CUDA_TRY(cudaMemset(t.bytes, 0, sizeof b));
    }
    if (scan_ms) *scan_ms = ms;
    if (bytes) *bytes = (double)b;
    return DADE_OK;
}

extern "C" size_t dade_search_workspace_size(const dade_index* idx, int64_t B, int32_t delta_d,
                                             const dade_search_opts* opts) {
    if (!idx || !opts || B < 0) return 0;
    if (dade::check_args(idx, B, delta_d, *opts) != DADE_OK) return 0;
    return dade::workspace_bytes(idx, B, delta_d, *opts, nullptr);
}
