// Internal declarations of the GB300 library behind include/dade.h.
#pragma once

#include <cuda_runtime.h>
#include <math.h>
#include <stdint.h>

#include <algorithm>
#include <map>
#include <memory>
#include <mutex>
#include <string>
#include <vector>

#include "dade.h"

namespace dade {

// ---------------------------------------------------------------- errors
dade_status fail(dade_status st, const char* fmt, ...);
void clear_error();

#define DADE_CUDA_TRY(expr)                                                                   \
    do {                                                                                      \
        cudaError_t e_ = (expr);                                                              \
        if (e_ != cudaSuccess)                                                                \
            return ::dade::fail(DADE_ECUDA, "%s failed: %s (%s:%d)", #expr,                  \
                                cudaGetErrorString(e_), __FILE__, __LINE__);                  \
    } while (0)

#define DADE_TRY(expr)                                                                        \
    do {                                                                                      \
        dade_status s_ = (expr);                                                              \
        if (s_ != DADE_OK) return s_;                                                         \
    } while (0)

constexpr int kBlock = 8;        // dimensions per layout block
constexpr int kListAlign = 32;   // bucket sizes are padded to a multiple of this
constexpr int kMaxK = 1024;
constexpr int kTcRows = 128;     // candidates per tile of the tensor-core scan (MMA M)
constexpr int kMaxD = 4096;
// Relative slack of the test on the completed rotated distance (a candidate
// is reranked iff dis'_S <= (sqrt(tau) + e_x)^2 (1 + kFinalRel)): covers the
// FP32 rounding of the rotation and of the accumulated sums.
constexpr float kFinalRel = 1e-3f;

inline int64_t ceil_div(int64_t a, int64_t b) { return (a + b - 1) / b; }
inline int64_t round_up(int64_t a, int64_t b) { return ceil_div(a, b) * b; }

// Wave schedule with first wave f and growth 2^g: wave 0 holds probe ranks
// [0, f), wave w >= 1 holds [f 2^(g(w-1)), f 2^(gw)).
inline int wave_of_rank_host(int r, int f, int g) {
    if (r < f) return 0;
    int q = r / f, lg = -1;
    while (q) { q >>= 1; ++lg; }
    return 1 + lg / g;
}
inline int num_waves(int nprobe, int f, int g) { return nprobe <= 0 ? 0 : wave_of_rank_host(nprobe - 1, f, g) + 1; }
inline int wave_begin(int w, int f, int g) {
    if (w == 0) return 0;
    const int64_t sh = (int64_t)g * (w - 1);
    return sh >= 30 ? (1 << 30) : (int)std::min<int64_t>((int64_t)f << sh, 1 << 30);
}

struct CorrectionTable {
    int32_t S = 0;
    std::vector<float> m1, beta;  // S - 1 each
    float* m1_dev = nullptr;
    float* beta_dev = nullptr;
};

// Device buffer with RAII release.
struct DevBuf {
    void* p = nullptr;
    size_t bytes = 0;
    DevBuf() = default;
    DevBuf(const DevBuf&) = delete;
    DevBuf& operator=(const DevBuf&) = delete;
    ~DevBuf() { release(); }
    dade_status alloc(size_t n);
    void release();
    template <class T> T* as() const { return static_cast<T*>(p); }
};

// Scratch of the dade_search calls that pass no workspace: one buffer per
// stream, so that searches of one index on different streams never share
// or free each other's scratch.  A buffer grows stream-ordered (the old one
// is released with cudaFreeAsync on the same stream, after the kernels that
// use it), and a search holds its stream's lock while it enqueues.
struct StreamWorkspaces {
    struct Buf {
        std::mutex mu;
        void* p = nullptr;
        size_t bytes = 0;
    };
    std::mutex mu;
    std::map<cudaStream_t, std::unique_ptr<Buf>> by_stream;
    Buf* of(cudaStream_t st) {
        std::lock_guard<std::mutex> lk(mu);
        std::unique_ptr<Buf>& b = by_stream[st];
        if (!b) b.reset(new Buf);
        return b.get();
    }
    // Release a stream's buffer, ordered after its queued work (before the
    // caller destroys that stream).
    void drop(cudaStream_t st) {
        std::lock_guard<std::mutex> lk(mu);
        auto it = by_stream.find(st);
        if (it == by_stream.end()) return;
        if (it->second->p) cudaFreeAsync(it->second->p, st);
        by_stream.erase(it);
    }
    ~StreamWorkspaces() {
        for (auto& kv : by_stream)
            if (kv.second->p) cudaFree(kv.second->p);
    }
};

}  // namespace dade

struct dade_index {
    int device = 0;
    int64_t N = 0;
    int32_t D = 0, Dpad = 0, nb = 0, nlist = 0;
    dade_slab_dtype dtype = DADE_SLAB_F32;
    std::vector<double> mean, R;       // host FP64 (D, D x D)
    std::vector<float> centroids;      // host nlist x D (rotated space)
    std::vector<int32_t> assign;       // host N: bucket of each input row
    std::vector<int64_t> ids;          // host N: id of each input row
    std::vector<int64_t> list_size;    // nlist
    std::vector<int64_t> list_slot;    // nlist + 1: first slot of each bucket
    std::vector<int64_t> sizes_desc_prefix;  // prefix sums of bucket sizes, largest first
    std::vector<float> fp8_scale;      // Dpad (FP8 only)
    int64_t total_slots = 0, max_list = 0;
    // device copies
    dade::DevBuf R_dev;        // Dpad x Dpad FP32 (zero beyond D)
    dade::DevBuf mean_dev;     // Dpad FP32
    dade::DevBuf cent_dev;     // nlist x Dpad FP32
    dade::DevBuf cnorm_dev;    // nlist FP32: ||c||^2
    dade::DevBuf list_size_dev;  // nlist int32
    dade::DevBuf list_slot_dev;  // nlist + 1 int64
    dade::DevBuf slab_dev;     // total_slots x Dpad elements of dtype, blocked
    dade::DevBuf orig_dev;     // total_slots x Dpad FP32, blocked
    dade::DevBuf ids_dev;      // total_slots int64 (-1 on padding)
    dade::DevBuf scale_dev;    // Dpad FP32 (FP8 only)
    dade::DevBuf eps_dev;      // total_slots FP32: quantisation error norm (BF16/FP8 only)
    dade::DevBuf var_dev;      // Dpad FP32: variance of each rotated dimension (RES)
    dade::DevBuf sfx_dev;      // (nb + 1) x total_slots FP32: residual norms from block b on (RES)
    std::vector<float> var;    // host copy of var_dev
    // tensor-core scan operand: per bucket tile of kTcRows candidates, per
    // 8-dim block, the stored values' TF32 parts (tc_parts of them: 1 for
    // BF16, else 2) in 4 KB canonical-layout chunks
    int32_t tc_parts = 0;
    std::vector<int64_t> tile_base;    // nlist + 1: first tile of each bucket
    dade::DevBuf tile_base_dev;
    dade::DevBuf tcslab_dev;
    int32_t ids32 = 0;         // every slot's id is -1 (padding) or in [0, 2^31 - 1)
    dade::DevBuf cent_tc_dev;  // centroid TF32 parts in canonical chunks (probe step; Dpad <= 128)
    // OPQ-L: product quantisation of the stored rotated vectors
    int32_t pq_m = 0, pq_ds = 0;
    std::vector<int32_t> pq_perm;      // D: rotated dims of subspace j at [j*ds, (j+1)*ds)
    std::vector<float> pq_cb;          // m x 256 x ds codebooks
    dade::DevBuf pq_perm_dev, pq_cb_dev;
    dade::DevBuf pq_codes_dev;         // m x total_slots uint8 (subspace-major)
    dade::DevBuf pq_err_dev;           // total_slots FP32: ||x~ - reconstruction||
    bool pq_has_table = false;
    float pq_m1 = 0.f, pq_m3 = 0.f, pq_beta = -INFINITY;
    std::map<int, dade::CorrectionTable> tables;  // by delta_d
    // internal scratch used when the caller gives no workspace, per stream
    mutable dade::StreamWorkspaces ws;
};

namespace dade {

// ----------------------------------------------------------- host math
dade_status covariance_fp64(const float* X, int64_t n, int32_t D, const int64_t* rows,
                            int64_t m, double* mean, double* cov);
dade_status jacobi_eigh(int32_t D, const double* A, double* eigvals, double* R);
dade_status haar_rotation(int32_t D, uint64_t seed, double* R_out);
dade_status fit_tables(const double* partials, const double* tau, const int8_t* label,
                       int64_t n, int32_t S, double target_recall, int32_t min_label0,
                       double* m1_out, double* beta_out);
// OPQ-L's three-feature classifier (m1, m3, beta'): prune iff
// m1 dis' + m3 e + beta' > tau; out = {0, 0, -inf} when the fit fails.
dade_status fit_pq_host(const double* dis, const double* err, const double* tau, const int8_t* label,
                        int64_t n, double target_recall, int32_t min_label0, double* out3);
uint64_t splitmix64(uint64_t z);
double sample_uniform(uint64_t seed, uint64_t query, uint64_t id);

// ----------------------------------------------------------- kernels
enum GemmOp { GEMM_DOT = 0, GEMM_L2 = 1 };
// C[M x N] = op(A - sub, B): DOT = sum (a - sub) b, L2 = sum (a - b)^2 over k < Kd.
cudaError_t launch_gemm_store(int op, const float* A, int64_t lda, const float* sub,
                              const float* B, int64_t ldb, float* C, int64_t ldc, int64_t M,
                              int64_t N, int Kd, cudaStream_t st);
// out[m] = min over n of (bits(L2(A_m, B_n)) << 32 | n), atomically (out preset to ~0).
cudaError_t launch_gemm_argmin(const float* A, int64_t lda, const float* B, int64_t ldb,
                               unsigned long long* out, int64_t M, int64_t N, int Kd,
                               cudaStream_t st);
// Tensor-core (tcgen05, split-TF32) GEMMs: C = (A - sub) B^T, and
// C = max(0, an + bn - 2 A B^T) (squared distances from norms).
cudaError_t launch_tc_dot(const float* A, int64_t lda, const float* sub, const float* B, int64_t ldb,
                          float* C, int64_t ldc, int64_t M, int64_t N, int Kd, int32_t* status,
                          cudaStream_t st);
cudaError_t launch_tc_l2(const float* A, int64_t lda, const float* an, const float* B, int64_t ldb,
                         const float* bn, float* C, int64_t ldc, int64_t M, int64_t N, int Kd,
                         int32_t* status, cudaStream_t st);
cudaError_t launch_row_norms(const float* X, int64_t ld, int64_t M, int n, float* out, cudaStream_t st);
// Per row b: the nprobe[b] smallest of scores[b, 0:n] ordered by (score, column).
// The centroid distances of the probe step on the tensor cores (pre-split
// operands, the query tile resident, pipelined): available for Dpad <= 128.
bool centroid_tc_supported(int Dpad);
cudaError_t launch_split_tc(const float* X, int64_t ld, int64_t nrows, int Dpad, float* out, cudaStream_t st);
cudaError_t launch_centroid_dist_tc(const float* qtc, const float* ctc, const float* qn, const float* cn, int64_t B,
                                    int nlist, int Dpad, float* scores, float* tmin, int32_t* status,
                                    cudaStream_t st);
// tmin (optional): per query and 128-centroid tile the tile's 4 smallest
// distances (from launch_centroid_dist_tc); with it, nprobe <= 128 and at most
// 32 tiles, the selection takes one pass over each score row.
cudaError_t launch_select_probes(const float* scores, int64_t B, int n, const int32_t* nprobe,
                                 int P, int32_t* probes, int32_t* status, cudaStream_t st,
                                 const float* tmin = nullptr);

struct LayoutArgs {
    const float* xrot;       // N x Dpad rotated FP32 rows
    const float* x;          // N x D original rows
    const int32_t* slot_row; // total_slots: source row or -1
    const int32_t* slot_list;
    const int64_t* list_slot;
    int64_t total_slots;
    int32_t D, Dpad;
    int dtype;
    const float* scale;      // FP8 per-dim scale
    void* slab;
    float* orig;
    float* eps;              // total_slots: ||x' - stored x'|| (BF16/FP8 only, else null)
};
cudaError_t launch_layout(const LayoutArgs& a, cudaStream_t st);
cudaError_t launch_quant_error(const LayoutArgs& a, cudaStream_t st);
cudaError_t launch_tc_slab(const void* slab, int dtype, const float* scale, const int64_t* list_slot,
                           const int32_t* list_size, const int64_t* tile_base, int nlist, int32_t Dpad, int parts,
                           int64_t ntiles, float* out, cudaStream_t st);
// The tensor-core scan's operand copy of idx's slabs (tc_slab_kernel).
dade_status build_tc_operands(dade_index* idx);
cudaError_t launch_stored_gather(const void* slab, int dtype, const float* scale, const int64_t* base,
                                 const int64_t* npad, int64_t nrows, int32_t D, float* out, cudaStream_t st);
cudaError_t launch_dim_var(const float* xrot, int64_t N, int32_t Dpad, float* var, cudaStream_t st);
cudaError_t launch_residual_norms(const void* slab, int dtype, const float* scale, const int64_t* list_slot,
                                  int nlist, int64_t total_slots, int32_t Dpad, float* sfx, cudaStream_t st);
// The per-slot residual norms of idx's slabs (RES), computed on the device.
dade_status build_residual_norms(dade_index* idx);
// OPQ-L kernels (kernels/pq.cu).
cudaError_t launch_pq_encode(const void* slab, int dtype, const float* scale, const int64_t* list_slot,
                             int nlist, int64_t total_slots, int32_t Dpad, const int32_t* perm, const float* cb,
                             int m, int ds, uint8_t* codes, float* err, cudaStream_t st);
cudaError_t launch_pq_lut(const float* qrot, int64_t B, int32_t Dpad, const int32_t* perm, const float* cb, int m,
                          int ds, float* lut, cudaStream_t st);
cudaError_t launch_amax(const float* xrot, int64_t N, int32_t Dpad, float* amax_bits_as_float,
                        cudaStream_t st);
cudaError_t launch_fp8_scale(float* amax_to_scale, int32_t Dpad, cudaStream_t st);

// ----------------------------------------------------------- search
struct SearchPlan;  // defined in search.cu
dade_status search_impl(const dade_index* idx, const float* Q_dev, int64_t B,
                        const int32_t* K_dev, const int32_t* nprobe_dev, int32_t delta_d,
                        const dade_search_opts& opts, int64_t* ids_dev, float* dists_dev,
                        const int64_t* out_offsets_dev, cudaStream_t st,
                        const struct CollectArgs* collect);
// Host-side argument checks of dade_search (status and message as it returns them).
dade_status check_args(const dade_index* idx, int64_t B, int32_t delta_d, const dade_search_opts& opts);
size_t workspace_bytes(const dade_index* idx, int64_t B, int32_t delta_d,
                       const dade_search_opts& opts, const struct CollectArgs* collect);

// Bucket metadata from idx->assign and allocation of the per-slot device
// arrays (abi.cu); installation of a correction table.
dade_status upload_index_arrays(dade_index* idx);
dade_status install_table_public(dade_index* idx, int delta_d, int S, const float* m1, const float* beta);
// Owner shard of every bucket (sizes balanced greedily, largest first).
std::vector<int32_t> shard_owners(const std::vector<int64_t>& list_size, int n_shards);
cudaError_t launch_merge_topk(int n_parts, int64_t B, int Kmax, const int32_t* K, const int64_t* ids,
                              const float* dists, int64_t* ids_out, float* dists_out, cudaStream_t st);

// Sample collection for the correction fit (replay with pruning off).
struct CollectArgs {
    int32_t pass;             // 0: count label-1 rows; 1: emit rows
    const int64_t* topk_ids;  // B x K_max sorted ids of the exact top-K
    int32_t topk_stride;
    uint64_t seed;
    int64_t query_offset;     // index of the batch's first query in the training set
    double keep_rate;         // label-1 keep probability (pass 1)
    unsigned long long* n_label1;  // pass 0 counter
    unsigned long long* n_rows;    // pass 1 counter
    int64_t row_cap;
    float* partials;          // row_cap x (S - 1); OPQ-L: row_cap x 2 (dis', e)
    int32_t pq_m;             // > 0: OPQ-L rows from the codes and tables below
    const uint8_t* pq_codes;
    const float* pq_err;
    const float* pq_lut;
    float* tau;               // row_cap
    int8_t* label;            // row_cap
    int64_t* query;           // row_cap or null: training-query index of each row
    int64_t* id;              // row_cap or null: id of each row's candidate
    int32_t keep_all;         // emit every candidate (also where tau is +inf);
                              // label 2 = neither label 0 nor label 1
};

}  // namespace dade
