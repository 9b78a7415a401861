// C ABI glue: status/error plumbing, index lifetime, inspection, correction
// tables, persistence, and the host-side rotation training.
#include <climits>
#include <math.h>
#include <stdarg.h>
#include <stdio.h>
#include <string.h>

#include <algorithm>
#include <memory>
#include <vector>

#include "dade_internal.h"

namespace dade {

static thread_local std::string g_last_error;

dade_status fail(dade_status st, const char* fmt, ...) {
    char buf[1024];
    va_list ap;
    va_start(ap, fmt);
    vsnprintf(buf, sizeof buf, fmt, ap);
    va_end(ap);
    g_last_error = buf;
    return st;
}

void clear_error() { g_last_error.clear(); }

dade_status DevBuf::alloc(size_t n) {
    release();
    if (n == 0) n = 1;
    cudaError_t e = cudaMalloc(&p, n);
    if (e != cudaSuccess) {
        p = nullptr;
        cudaGetLastError();
        return fail(DADE_ENOMEM, "cudaMalloc(%zu) failed: %s", n, cudaGetErrorString(e));
    }
    bytes = n;
    return DADE_OK;
}

void DevBuf::release() {
    if (p) cudaFree(p);
    p = nullptr;
    bytes = 0;
}

static size_t elem_size(dade_slab_dtype t) { return t == DADE_SLAB_F32 ? 4 : t == DADE_SLAB_BF16 ? 2 : 1; }

// Bucket metadata from idx->assign, and allocation of the bucket arrays.
dade_status upload_index_arrays(dade_index* idx) {
    const int nl = idx->nlist;
    idx->list_size.assign((size_t)nl, 0);
    for (int32_t a : idx->assign) idx->list_size[(size_t)a]++;
    idx->list_slot.assign((size_t)nl + 1, 0);
    for (int l = 0; l < nl; ++l)
        idx->list_slot[(size_t)l + 1] = idx->list_slot[(size_t)l] + round_up(idx->list_size[(size_t)l], kListAlign);
    idx->total_slots = idx->list_slot[(size_t)nl];
    std::vector<int64_t> desc(idx->list_size);
    std::sort(desc.begin(), desc.end(), std::greater<int64_t>());
    idx->max_list = nl ? desc[0] : 0;
    idx->sizes_desc_prefix.assign((size_t)nl + 1, 0);
    for (int l = 0; l < nl; ++l) idx->sizes_desc_prefix[(size_t)l + 1] = idx->sizes_desc_prefix[(size_t)l] + desc[(size_t)l];
    std::vector<int32_t> sz32(idx->list_size.begin(), idx->list_size.end());
    DADE_TRY(idx->list_size_dev.alloc(sizeof(int32_t) * nl));
    DADE_TRY(idx->list_slot_dev.alloc(sizeof(int64_t) * (nl + 1)));
    DADE_CUDA_TRY(cudaMemcpy(idx->list_size_dev.p, sz32.data(), sizeof(int32_t) * nl, cudaMemcpyHostToDevice));
    DADE_CUDA_TRY(cudaMemcpy(idx->list_slot_dev.p, idx->list_slot.data(), sizeof(int64_t) * (nl + 1),
                             cudaMemcpyHostToDevice));
    const size_t n = (size_t)idx->total_slots * idx->Dpad;
    DADE_TRY(idx->slab_dev.alloc(n * elem_size(idx->dtype)));
    DADE_TRY(idx->orig_dev.alloc(n * sizeof(float)));
    DADE_TRY(idx->ids_dev.alloc(sizeof(int64_t) * std::max<int64_t>(1, idx->total_slots)));
    if (idx->dtype != DADE_SLAB_F32)
        DADE_TRY(idx->eps_dev.alloc(sizeof(float) * std::max<int64_t>(1, idx->total_slots)));
    return DADE_OK;
}

static dade_status install_table(dade_index* idx, int delta_d, int S, const float* m1, const float* beta) {
    CorrectionTable& t = idx->tables[delta_d];
    if (t.m1_dev) cudaFree(t.m1_dev);
    if (t.beta_dev) cudaFree(t.beta_dev);
    t.m1_dev = t.beta_dev = nullptr;
    t.S = S;
    t.m1.assign(m1, m1 + (S - 1));
    t.beta.assign(beta, beta + (S - 1));
    size_t nb = sizeof(float) * std::max(1, S - 1);
    DADE_CUDA_TRY(cudaMalloc(&t.m1_dev, nb));
    DADE_CUDA_TRY(cudaMalloc(&t.beta_dev, nb));
    if (S > 1) {
        DADE_CUDA_TRY(cudaMemcpy(t.m1_dev, m1, sizeof(float) * (S - 1), cudaMemcpyHostToDevice));
        DADE_CUDA_TRY(cudaMemcpy(t.beta_dev, beta, sizeof(float) * (S - 1), cudaMemcpyHostToDevice));
    }
    return DADE_OK;
}

dade_status build_residual_norms(dade_index* idx) {
    const int64_t n = (int64_t)(idx->nb + 1) * std::max<int64_t>(1, idx->total_slots);
    DADE_TRY(idx->sfx_dev.alloc(sizeof(float) * n));
    DADE_CUDA_TRY(launch_residual_norms(idx->slab_dev.p, idx->dtype, idx->scale_dev.as<float>(),
                                        idx->list_slot_dev.as<int64_t>(), idx->nlist, idx->total_slots, idx->Dpad,
                                        idx->sfx_dev.as<float>(), 0));
    DADE_CUDA_TRY(cudaDeviceSynchronize());
    return DADE_OK;
}

dade_status build_tc_operands(dade_index* idx) {
    const int nl = idx->nlist;
    idx->tile_base.assign((size_t)nl + 1, 0);
    for (int l = 0; l < nl; ++l)
        idx->tile_base[(size_t)l + 1] = idx->tile_base[(size_t)l] + ceil_div(idx->list_size[(size_t)l], kTcRows);
    const int64_t ntiles = idx->tile_base[(size_t)nl];
    idx->tc_parts = idx->dtype == DADE_SLAB_BF16 ? 1 : 2;
    DADE_TRY(idx->tile_base_dev.alloc(sizeof(int64_t) * (nl + 1)));
    DADE_CUDA_TRY(cudaMemcpy(idx->tile_base_dev.p, idx->tile_base.data(), sizeof(int64_t) * (nl + 1),
                             cudaMemcpyHostToDevice));
    DADE_TRY(idx->tcslab_dev.alloc(sizeof(float) * 1024 * (size_t)std::max<int64_t>(1, ntiles) * idx->nb *
                                   idx->tc_parts));
    DADE_CUDA_TRY(launch_tc_slab(idx->slab_dev.p, idx->dtype, idx->scale_dev.as<float>(),
                                 idx->list_slot_dev.as<int64_t>(), idx->list_size_dev.as<int32_t>(),
                                 idx->tile_base_dev.as<int64_t>(), nl, idx->Dpad, idx->tc_parts, ntiles,
                                 idx->tcslab_dev.as<float>(), 0));
    {  // may the merges carry 32-bit ids?
        std::vector<int64_t> h((size_t)idx->total_slots);
        if (idx->total_slots > 0)
            DADE_CUDA_TRY(cudaMemcpy(h.data(), idx->ids_dev.p, sizeof(int64_t) * idx->total_slots,
                                     cudaMemcpyDeviceToHost));
        bool fit = true;
        for (int64_t v : h) fit = fit && (v == -1 || (v >= 0 && v < (int64_t)INT_MAX));
        idx->ids32 = fit ? 1 : 0;
    }
    if (centroid_tc_supported(idx->Dpad)) {
        DADE_TRY(idx->cent_tc_dev.alloc(sizeof(float) * 2 * 1024 * (size_t)ceil_div(nl, 128) * (idx->Dpad / 8)));
        DADE_CUDA_TRY(launch_split_tc(idx->cent_dev.as<float>(), idx->Dpad, nl, idx->Dpad,
                                      idx->cent_tc_dev.as<float>(), 0));
    }
    DADE_CUDA_TRY(cudaDeviceSynchronize());
    return DADE_OK;
}

dade_status install_table_public(dade_index* idx, int delta_d, int S, const float* m1, const float* beta) {
    return install_table(idx, delta_d, S, m1, beta);
}

// ---------------------------------------------------------------- persistence
namespace {

struct Fnv {
    uint64_t h = 1469598103934665603ull;
    void add(const void* p, size_t n) {
        const unsigned char* c = static_cast<const unsigned char*>(p);
        for (size_t i = 0; i < n; ++i) {
            h ^= c[i];
            h *= 1099511628211ull;
        }
    }
};

struct Writer {
    FILE* f;
    Fnv fnv;
    bool ok = true;
    void put(const void* p, size_t n) {
        if (!n) return;
        fnv.add(p, n);
        ok = ok && fwrite(p, 1, n, f) == n;
    }
    template <class T> void pod(const T& v) { put(&v, sizeof v); }
};

struct Reader {
    FILE* f;
    Fnv fnv;
    bool ok = true;
    void get(void* p, size_t n) {
        if (!n) return;
        ok = ok && fread(p, 1, n, f) == n;
        if (ok) fnv.add(p, n);
    }
    template <class T> void pod(T& v) { get(&v, sizeof v); }
};

const char kMagic[8] = {'D', 'A', 'D', 'E', 'I', 'D', 'X', '1'};
const uint32_t kVersion = 4;

}  // namespace

}  // namespace dade

using namespace dade;

extern "C" const char* dade_last_error(void) { return g_last_error.c_str(); }

extern "C" void dade_index_free(dade_index* idx) {
    if (!idx) return;
    int cur = 0;
    cudaGetDevice(&cur);
    cudaSetDevice(idx->device);
    for (auto& kv : idx->tables) {
        if (kv.second.m1_dev) cudaFree(kv.second.m1_dev);
        if (kv.second.beta_dev) cudaFree(kv.second.beta_dev);
    }
    delete idx;
    cudaSetDevice(cur);
}

extern "C" dade_status dade_index_info_get(const dade_index* idx, dade_index_info* out) {
    clear_error();
    if (!idx || !out) return fail(DADE_EINVAL, "null argument");
    out->N = idx->N;
    out->D = idx->D;
    out->Dpad = idx->Dpad;
    out->nlist = idx->nlist;
    out->dtype = idx->dtype;
    out->max_list = idx->max_list;
    out->device_bytes = (int64_t)(idx->slab_dev.bytes + idx->orig_dev.bytes + idx->ids_dev.bytes +
                                  idx->cent_dev.bytes + idx->R_dev.bytes + idx->eps_dev.bytes + idx->var_dev.bytes +
                                  idx->sfx_dev.bytes + idx->pq_codes_dev.bytes + idx->pq_err_dev.bytes +
                                  idx->pq_cb_dev.bytes + idx->pq_perm_dev.bytes + idx->tcslab_dev.bytes +
                                  idx->cent_tc_dev.bytes);
    return DADE_OK;
}

extern "C" dade_status dade_index_centroids(const dade_index* idx, float* out) {
    clear_error();
    if (!idx || !out) return fail(DADE_EINVAL, "null argument");
    memcpy(out, idx->centroids.data(), sizeof(float) * idx->centroids.size());
    return DADE_OK;
}

extern "C" dade_status dade_index_assignment(const dade_index* idx, int32_t* out) {
    clear_error();
    if (!idx || !out) return fail(DADE_EINVAL, "null argument");
    memcpy(out, idx->assign.data(), sizeof(int32_t) * idx->assign.size());
    return DADE_OK;
}

extern "C" dade_status dade_index_list_sizes(const dade_index* idx, int64_t* out) {
    clear_error();
    if (!idx || !out) return fail(DADE_EINVAL, "null argument");
    memcpy(out, idx->list_size.data(), sizeof(int64_t) * idx->list_size.size());
    return DADE_OK;
}

extern "C" dade_status dade_index_stored(const dade_index* idx, int64_t row0, int64_t nrows, float* out) {
    clear_error();
    if (!idx || (!out && nrows > 0)) return fail(DADE_EINVAL, "null argument");
    if (row0 < 0 || nrows < 0 || row0 > idx->N || nrows > idx->N - row0)
        return fail(DADE_EINVAL, "rows [%lld, %lld) outside [0, %lld)", (long long)row0,
                    (long long)(row0 + nrows), (long long)idx->N);
    if (nrows == 0) return DADE_OK;
    // slot of input row i: its bucket's first slot plus its rank among the
    // bucket's earlier rows (rows are laid out in input order per bucket)
    std::vector<int64_t> rank((size_t)idx->nlist, 0), base((size_t)nrows), npad((size_t)nrows);
    for (int64_t i = 0; i < row0 + nrows; ++i) {
        const int l = idx->assign[(size_t)i];
        const int64_t k = rank[(size_t)l]++;
        if (i < row0) continue;
        const int64_t s0 = idx->list_slot[(size_t)l];
        base[(size_t)(i - row0)] = s0 * idx->Dpad + k * kBlock;
        npad[(size_t)(i - row0)] = idx->list_slot[(size_t)l + 1] - s0;
    }
    int cur = 0;
    DADE_CUDA_TRY(cudaGetDevice(&cur));
    DADE_CUDA_TRY(cudaSetDevice(idx->device));
    struct Restore {
        int d;
        ~Restore() { cudaSetDevice(d); }
    } restore{cur};
    DevBuf b, n, o;
    DADE_TRY(b.alloc(sizeof(int64_t) * nrows));
    DADE_TRY(n.alloc(sizeof(int64_t) * nrows));
    DADE_TRY(o.alloc(sizeof(float) * nrows * idx->D));
    DADE_CUDA_TRY(cudaMemcpy(b.p, base.data(), sizeof(int64_t) * nrows, cudaMemcpyHostToDevice));
    DADE_CUDA_TRY(cudaMemcpy(n.p, npad.data(), sizeof(int64_t) * nrows, cudaMemcpyHostToDevice));
    DADE_CUDA_TRY(launch_stored_gather(idx->slab_dev.p, idx->dtype, idx->scale_dev.as<float>(), b.as<int64_t>(),
                                       n.as<int64_t>(), nrows, idx->D, o.as<float>(), 0));
    DADE_CUDA_TRY(cudaMemcpy(out, o.p, sizeof(float) * nrows * idx->D, cudaMemcpyDeviceToHost));
    return DADE_OK;
}

extern "C" dade_status dade_set_correction(dade_index* idx, int32_t delta_d, const float* m1,
                                           const float* beta) {
    clear_error();
    if (!idx) return fail(DADE_EINVAL, "null index");
    if (delta_d < 8 || delta_d % 8) return fail(DADE_EINVAL, "delta_d must be a positive multiple of 8");
    int S = (int)ceil_div(idx->Dpad, delta_d);
    if (S > 1 && (!m1 || !beta)) return fail(DADE_EINVAL, "null table");
    for (int s = 0; s + 1 < S; ++s)
        if (isnan(m1[s]) || isnan(beta[s]) || isinf(m1[s])) return fail(DADE_EINVAL, "table entry %d is not finite", s);
    int cur = 0;
    cudaGetDevice(&cur);
    cudaSetDevice(idx->device);
    dade_status st = install_table(idx, delta_d, S, m1, beta);
    cudaSetDevice(cur);
    return st;
}

extern "C" dade_status dade_get_correction(const dade_index* idx, int32_t delta_d, float* m1, float* beta) {
    clear_error();
    if (!idx) return fail(DADE_EINVAL, "null index");
    auto it = idx->tables.find(delta_d);
    if (it == idx->tables.end()) return fail(DADE_ESTATE, "no table for delta_d = %d", delta_d);
    if (m1) memcpy(m1, it->second.m1.data(), sizeof(float) * it->second.m1.size());
    if (beta) memcpy(beta, it->second.beta.data(), sizeof(float) * it->second.beta.size());
    return DADE_OK;
}

extern "C" dade_status dade_index_save(const dade_index* idx, const char* path) {
    clear_error();
    if (!idx || !path) return fail(DADE_EINVAL, "null argument");
    FILE* f = fopen(path, "wb");
    if (!f) return fail(DADE_EIO, "cannot open %s for writing", path);
    Writer w{f};
    w.put(kMagic, sizeof kMagic);
    w.pod(kVersion);
    w.pod(idx->N);
    w.pod(idx->D);
    w.pod(idx->nlist);
    int32_t dt = idx->dtype;
    w.pod(dt);
    w.put(idx->mean.data(), sizeof(double) * idx->mean.size());
    w.put(idx->R.data(), sizeof(double) * idx->R.size());
    w.put(idx->centroids.data(), sizeof(float) * idx->centroids.size());
    w.put(idx->assign.data(), sizeof(int32_t) * idx->assign.size());
    w.put(idx->ids.data(), sizeof(int64_t) * idx->ids.size());
    if (idx->dtype == DADE_SLAB_FP8E4M3) w.put(idx->fp8_scale.data(), sizeof(float) * idx->fp8_scale.size());
    w.put(idx->var.data(), sizeof(float) * idx->var.size());
    // device contents
    std::vector<char> host;
    auto dump = [&](const DevBuf& b, size_t n) {
        host.resize(n);
        if (n && cudaMemcpy(host.data(), b.p, n, cudaMemcpyDeviceToHost) != cudaSuccess) w.ok = false;
        w.put(host.data(), n);
    };
    const size_t n = (size_t)idx->total_slots * idx->Dpad;
    dump(idx->slab_dev, n * elem_size(idx->dtype));
    dump(idx->orig_dev, n * sizeof(float));
    dump(idx->ids_dev, sizeof(int64_t) * idx->total_slots);
    if (idx->dtype != DADE_SLAB_F32) dump(idx->eps_dev, sizeof(float) * idx->total_slots);
    int32_t nt = (int32_t)idx->tables.size();
    w.pod(nt);
    for (auto& kv : idx->tables) {
        int32_t dd = kv.first, S = kv.second.S;
        w.pod(dd);
        w.pod(S);
        w.put(kv.second.m1.data(), sizeof(float) * kv.second.m1.size());
        w.put(kv.second.beta.data(), sizeof(float) * kv.second.beta.size());
    }
    // OPQ-L quantiser (the codes are recomputed from the slabs at load)
    int32_t pm = idx->pq_m;
    w.pod(pm);
    if (pm > 0) {
        w.put(idx->pq_perm.data(), sizeof(int32_t) * idx->pq_perm.size());
        w.put(idx->pq_cb.data(), sizeof(float) * idx->pq_cb.size());
        int32_t ht = idx->pq_has_table ? 1 : 0;
        w.pod(ht);
        w.pod(idx->pq_m1);
        w.pod(idx->pq_m3);
        w.pod(idx->pq_beta);
    }
    uint64_t h = w.fnv.h;
    bool ok = w.ok && fwrite(&h, sizeof h, 1, f) == 1;
    ok = (fclose(f) == 0) && ok;
    return ok ? DADE_OK : fail(DADE_EIO, "write to %s failed", path);
}

extern "C" dade_status dade_index_load(const char* path, dade_index** out) {
    clear_error();
    if (!path || !out) return fail(DADE_EINVAL, "null argument");
    FILE* f = fopen(path, "rb");
    if (!f) return fail(DADE_EIO, "cannot open %s", path);
    struct Closer {
        FILE* f;
        ~Closer() { fclose(f); }
    } closer{f};
    Reader r{f};
    char magic[8];
    uint32_t ver = 0;
    r.get(magic, 8);
    r.pod(ver);
    if (!r.ok || memcmp(magic, kMagic, 8) || ver != kVersion) return fail(DADE_EIO, "%s: not a dade index file", path);
    std::unique_ptr<dade_index> idx(new dade_index());
    int32_t dt = 0;
    r.pod(idx->N);
    r.pod(idx->D);
    r.pod(idx->nlist);
    r.pod(dt);
    if (!r.ok || idx->N < 1 || idx->D < 1 || idx->D > kMaxD || idx->nlist < 1 || dt < 0 || dt > 2)
        return fail(DADE_EIO, "%s: bad header", path);
    idx->dtype = (dade_slab_dtype)dt;
    idx->Dpad = (int32_t)round_up(idx->D, kBlock);
    idx->nb = idx->Dpad / kBlock;
    cudaGetDevice(&idx->device);
    const int D = idx->D, Dp = idx->Dpad, nl = idx->nlist;
    idx->mean.resize((size_t)D);
    idx->R.resize((size_t)D * D);
    idx->centroids.resize((size_t)nl * D);
    idx->assign.resize((size_t)idx->N);
    idx->ids.resize((size_t)idx->N);
    r.get(idx->mean.data(), sizeof(double) * D);
    r.get(idx->R.data(), sizeof(double) * D * D);
    r.get(idx->centroids.data(), sizeof(float) * nl * D);
    r.get(idx->assign.data(), sizeof(int32_t) * idx->N);
    r.get(idx->ids.data(), sizeof(int64_t) * idx->N);
    if (!r.ok) return fail(DADE_EIO, "%s: truncated", path);
    for (int32_t a : idx->assign)
        if (a < 0 || a >= nl) return fail(DADE_EIO, "%s: bad assignment", path);
    if (idx->dtype == DADE_SLAB_FP8E4M3) {
        idx->fp8_scale.resize((size_t)Dp);
        r.get(idx->fp8_scale.data(), sizeof(float) * Dp);
    }
    idx->var.resize((size_t)Dp);
    r.get(idx->var.data(), sizeof(float) * Dp);
    DADE_TRY(upload_index_arrays(idx.get()));
    std::vector<char> host;
    auto fill = [&](DevBuf& b, size_t n) -> dade_status {
        host.resize(n);
        r.get(host.data(), n);
        if (!r.ok) return fail(DADE_EIO, "%s: truncated", path);
        if (n) DADE_CUDA_TRY(cudaMemcpy(b.p, host.data(), n, cudaMemcpyHostToDevice));
        return DADE_OK;
    };
    const size_t n = (size_t)idx->total_slots * Dp;
    DADE_TRY(fill(idx->slab_dev, n * elem_size(idx->dtype)));
    DADE_TRY(fill(idx->orig_dev, n * sizeof(float)));
    DADE_TRY(fill(idx->ids_dev, sizeof(int64_t) * idx->total_slots));
    if (idx->dtype != DADE_SLAB_F32) DADE_TRY(fill(idx->eps_dev, sizeof(float) * idx->total_slots));
    int32_t ntab = 0;
    r.pod(ntab);
    if (!r.ok || ntab < 0 || ntab > 64) return fail(DADE_EIO, "%s: bad table count", path);
    for (int i = 0; i < ntab; ++i) {
        int32_t dd = 0, S = 0;
        r.pod(dd);
        r.pod(S);
        if (!r.ok || dd < 8 || S < 1 || S != (int)ceil_div(Dp, dd)) return fail(DADE_EIO, "%s: bad table", path);
        std::vector<float> m1((size_t)S - 1), beta((size_t)S - 1);
        r.get(m1.data(), sizeof(float) * (S - 1));
        r.get(beta.data(), sizeof(float) * (S - 1));
        DADE_TRY(install_table(idx.get(), dd, S, m1.data(), beta.data()));
    }
    int32_t pm = 0, pq_ht = 0;
    std::vector<int32_t> pq_perm;
    std::vector<float> pq_cb;
    float pq_c[3] = {0.f, 0.f, -INFINITY};
    r.pod(pm);
    if (!r.ok || pm < 0 || (pm > 0 && (D % pm != 0 || D / pm > 64))) return fail(DADE_EIO, "%s: bad quantiser", path);
    if (pm > 0) {
        pq_perm.resize((size_t)D);
        pq_cb.resize((size_t)pm * 256 * (D / pm));
        r.get(pq_perm.data(), sizeof(int32_t) * D);
        r.get(pq_cb.data(), sizeof(float) * pq_cb.size());
        r.pod(pq_ht);
        for (float& c : pq_c) r.pod(c);
    }
    uint64_t want = r.fnv.h, got = 0;
    if (!r.ok || fread(&got, sizeof got, 1, f) != 1 || got != want) return fail(DADE_EIO, "%s: checksum mismatch", path);
    // rotation, mean, centroids on the device
    std::vector<float> Rf((size_t)Dp * Dp, 0.f), mf((size_t)Dp, 0.f), cf((size_t)nl * Dp, 0.f);
    for (int i = 0; i < D; ++i) {
        mf[i] = (float)idx->mean[i];
        for (int j = 0; j < D; ++j) Rf[(size_t)i * Dp + j] = (float)idx->R[(size_t)i * D + j];
    }
    for (int l = 0; l < nl; ++l)
        for (int j = 0; j < D; ++j) cf[(size_t)l * Dp + j] = idx->centroids[(size_t)l * D + j];
    DADE_TRY(idx->R_dev.alloc(sizeof(float) * Rf.size()));
    DADE_TRY(idx->mean_dev.alloc(sizeof(float) * mf.size()));
    DADE_TRY(idx->cent_dev.alloc(sizeof(float) * cf.size()));
    DADE_CUDA_TRY(cudaMemcpy(idx->R_dev.p, Rf.data(), sizeof(float) * Rf.size(), cudaMemcpyHostToDevice));
    DADE_CUDA_TRY(cudaMemcpy(idx->mean_dev.p, mf.data(), sizeof(float) * mf.size(), cudaMemcpyHostToDevice));
    DADE_CUDA_TRY(cudaMemcpy(idx->cent_dev.p, cf.data(), sizeof(float) * cf.size(), cudaMemcpyHostToDevice));
    DADE_TRY(idx->cnorm_dev.alloc(sizeof(float) * nl));
    DADE_CUDA_TRY(launch_row_norms(idx->cent_dev.as<float>(), Dp, nl, Dp, idx->cnorm_dev.as<float>(), 0));
    DADE_CUDA_TRY(cudaDeviceSynchronize());
    if (idx->dtype == DADE_SLAB_FP8E4M3) {
        DADE_TRY(idx->scale_dev.alloc(sizeof(float) * Dp));
        DADE_CUDA_TRY(cudaMemcpy(idx->scale_dev.p, idx->fp8_scale.data(), sizeof(float) * Dp, cudaMemcpyHostToDevice));
    }
    DADE_TRY(idx->var_dev.alloc(sizeof(float) * Dp));
    DADE_CUDA_TRY(cudaMemcpy(idx->var_dev.p, idx->var.data(), sizeof(float) * Dp, cudaMemcpyHostToDevice));
    DADE_TRY(build_residual_norms(idx.get()));
    DADE_TRY(build_tc_operands(idx.get()));
    if (pm > 0) {
        DADE_TRY(dade_pq_set(idx.get(), pm, pq_perm.data(), pq_cb.data()));
        if (pq_ht) DADE_TRY(dade_pq_set_correction(idx.get(), pq_c[0], pq_c[1], pq_c[2]));
    }
    *out = idx.release();
    return DADE_OK;
}

// ---------------------------------------------------------------- rotation
extern "C" dade_status dade_train_rotation(const float* X, int64_t n, int32_t D, int64_t sample_n,
                                           uint64_t seed, double* mean_out, double* R_out,
                                           double* eig_out) {
    clear_error();
    if (!X || !mean_out || !R_out || !eig_out) return fail(DADE_EINVAL, "null argument");
    if (n < 2) return fail(DADE_EINVAL, "need at least 2 rows");
    if (D < 1 || D > kMaxD) return fail(DADE_EINVAL, "D out of range");
    std::vector<int64_t> rows;
    int64_t m = n;
    if (sample_n > 0 && sample_n < n) {
        if (sample_n < 2) return fail(DADE_EINVAL, "sample_n must be >= 2");
        // seeded partial Fisher-Yates, then increasing row order
        std::vector<int64_t> perm((size_t)n);
        for (int64_t i = 0; i < n; ++i) perm[(size_t)i] = i;
        for (int64_t i = 0; i < sample_n; ++i) {
            int64_t j = i + (int64_t)(splitmix64(seed + (uint64_t)i) % (uint64_t)(n - i));
            std::swap(perm[(size_t)i], perm[(size_t)j]);
        }
        rows.assign(perm.begin(), perm.begin() + sample_n);
        std::sort(rows.begin(), rows.end());
        m = sample_n;
    }
    std::vector<double> cov((size_t)D * D);
    DADE_TRY(covariance_fp64(X, n, D, rows.empty() ? nullptr : rows.data(), m, mean_out, cov.data()));
    return jacobi_eigh(D, cov.data(), eig_out, R_out);
}

extern "C" dade_status dade_random_rotation(int32_t D, uint64_t seed, double* R_out) {
    clear_error();
    if (!R_out) return fail(DADE_EINVAL, "null argument");
    if (D < 1 || D > kMaxD) return fail(DADE_EINVAL, "D out of range");
    return haar_rotation(D, seed, R_out);
}

extern "C" dade_status dade_ads_table(int32_t D, int32_t delta_d, double eps0, float* m1_out, float* beta_out) {
    clear_error();
    if (!m1_out || !beta_out) return fail(DADE_EINVAL, "null argument");
    if (D < 1 || D > kMaxD || delta_d < 1) return fail(DADE_EINVAL, "D or delta_d out of range");
    if (!(eps0 >= 0.0 && eps0 < INFINITY)) return fail(DADE_EINVAL, "eps0 must be finite and >= 0");
    const int S = (int)ceil_div(D, delta_d);
    for (int s = 1; s < S; ++s) {
        const double d = (double)std::min<int64_t>((int64_t)s * delta_d, D);
        m1_out[s - 1] = (float)((double)D / d / (1.0 + eps0 / sqrt(d)));
        beta_out[s - 1] = 0.f;
    }
    return DADE_OK;
}

extern "C" dade_status dade_fit_samples(const double* partials, const double* tau, const int8_t* label,
                                        int64_t n, int32_t D, int32_t delta_d, double target_recall,
                                        int32_t min_label0, double* m1_out, double* beta_out) {
    clear_error();
    if (n < 0 || (n > 0 && (!partials || !tau || !label)) || !m1_out || !beta_out)
        return fail(DADE_EINVAL, "null argument");
    if (delta_d < 8 || delta_d % 8 || D < 1) return fail(DADE_EINVAL, "bad D / delta_d");
    if (!(target_recall > 0 && target_recall <= 1)) return fail(DADE_EINVAL, "target_recall in (0, 1]");
    int S = (int)ceil_div(round_up(D, kBlock), delta_d);
    return fit_tables(partials, tau, label, n, S, target_recall, min_label0, m1_out, beta_out);
}
