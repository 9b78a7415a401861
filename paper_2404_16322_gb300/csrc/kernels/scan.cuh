// Device views shared by the refinement kernels (scan.cu) and the search
// orchestration (search.cu).
#pragma once

#include "../dade_internal.h"

namespace dade {

constexpr int kG = 16;             // queries per work unit
constexpr int kT = 128;            // candidates per tile of a bucket (one per thread in dense steps)
constexpr int kScanThreads = 128;  // 4 warps

struct IndexView {
    const void* slab;          // rotated vectors, blocked, slab dtype
    const float* orig;         // original vectors, blocked, FP32
    const int64_t* ids;        // per slot
    const int64_t* list_slot;  // nlist + 1
    const int32_t* list_size;  // nlist
    const float* scale;        // FP8 per-dimension scale (Dpad)
    const float* eps;          // per slot: quantisation error norm (null for FP32 slabs)
    const float* sfx;          // (nb + 1) x total_slots: sum of the stored x_i^2 over blocks >= b
    const float* tcslab;       // tensor-core operand copy of the slabs (build_tc_operands)
    const int64_t* tile_base;  // nlist + 1: first kTcRows-candidate tile of each bucket
    int64_t total_slots;
    int32_t D, Dpad, nb, nlist, dtype, tc_parts;
    int32_t ids32;             // every id is in [0, 2^31 - 1): the merges sort 32-bit ids
};

// A wave of probe ranks (tested against one tau) is scanned in one or more
// passes of consecutive ranks; the candidate buffer holds one pass.
constexpr int kMaxPasses = 128;

struct WaveView {
    int64_t B;
    int32_t P, Kmax, n_waves;  // n_waves: passes (below)
    int32_t final_test;       // PRUNE: test the completed rotated distance before the exact one
    int32_t est;              // PRUNE: 0 learned tables, 1 the Gaussian-bound (RES) test
    int32_t res_stride;       // S - 1: entries of res_q per query
    int32_t test_steps;       // PRUNE without final_test: steps tested (<= S - 1)
    const float* res_q;       // B x (S - 1): ||q'_r||^2 - m sigma after each step (RES)
    const float* qrot;        // B x Dpad rotated queries
    const float* qpad;        // B x Dpad original queries, zero padded
    const int32_t* probes;    // B x P
    const int32_t* nprobe;    // B
    const int32_t* K;         // B
    int32_t* cnt_wl;          // passes x nlist: queries probing (pass, bucket)
    int32_t* off_wl;          // passes x nlist + 1: exclusive prefix of cnt_wl
    int32_t* fill_wl;         // passes x nlist: scatter cursors
    int32_t* items;           // B x P query ids grouped by (wave, bucket)
    int32_t* unit_off;        // passes x (nlist + 1): work units per pass, prefix
    int4* units;              // unit descriptors {bucket, tile, first item, nq << 16 | nt}
    int64_t ubase[kMaxPasses];    // first descriptor of each pass in `units`
    int32_t qgroup[kMaxPasses];   // queries per unit at most, per pass (the queries probing a
                                  // bucket in a pass are split into balanced groups)
    int32_t pass_begin[kMaxPasses + 1];  // probe ranks [pass_begin[p], pass_begin[p + 1]) of pass p
    int64_t* cand_off;        // passes x (B + 1): candidate capacity per query, prefix
    int32_t* cand_cnt;        // B: candidates appended in the current pass
    float* cand_d;            // candidate buffer (capacity of the largest pass)
    int32_t* cand_pos;
    float* top_d;             // B x Kmax current top-K distances (sorted)
    int64_t* top_id;          // B x Kmax
    int32_t* top_n;           // B
    float* tau;               // B: the tau the current wave tests against (the top-K's K-th
                              // distance when the wave began; +inf while fewer than K)
    float* tau_run;           // B: the top-K's current K-th distance (written by the merges)
    int32_t* work;            // 2 x passes work counters (scan, collect), then an 8-byte counter
    int32_t* status;          // device status word
    int64_t* stats;           // B x 4 or null
    unsigned long long* staged_bytes;  // bytes staged by the scan, or null
};

// The pass that scans probe rank r (0 <= r < P).
__device__ __forceinline__ int pass_of_rank(const WaveView& wv, int r) {
    int lo = 0, hi = wv.n_waves;  // pass_begin[lo] <= r < pass_begin[hi]
    while (hi - lo > 1) {
        const int mid = (lo + hi) >> 1;
        if (wv.pass_begin[mid] <= r) lo = mid; else hi = mid;
    }
    return lo;
}

cudaError_t launch_prepare_queries(const float* Q, int64_t B, int32_t D, int32_t Dpad,
                                   float* qpad, cudaStream_t st);
cudaError_t launch_fill(float* p, int64_t n, float v, cudaStream_t st);
cudaError_t launch_build_units(const IndexView& ix, const WaveView& wv, cudaStream_t st);
cudaError_t launch_wave_scan(const IndexView& ix, const WaveView& wv, int w, bool full,
                             int delta_d, const float* m1, const float* beta, int S,
                             cudaStream_t st);
// OPQ-L: the product-quantisation codes of every slot (subspace-major), the
// quantisation errors, the per-query tables and the learned test.
struct PQView {
    const uint8_t* codes;     // m x total_slots
    const float* err;         // total_slots
    const float* lut;         // B x m x 256
    int64_t total_slots;
    int32_t m;
    float m1, m3, beta;       // prune iff m1 dis' + m3 e + beta > tau
};
// The wave scan of OPQ-L (scan_pq.cu): one test on the asymmetric distance,
// then the exact distance.
cudaError_t launch_pq_scan(const IndexView& ix, const WaveView& wv, int w, const PQView& pv, cudaStream_t st);

// The RES variants of launch_wave_scan (scan_res.cu), and the per-query RES
// terms res_q[b][s] = sum_{i >= d_s} q'_i^2 - m 2 sqrt(sum_{i >= d_s} q'_i^2 var_i),
// d_s = min((s + 1) delta_d, D), for s < S - 1.
cudaError_t launch_wave_scan_res(const IndexView& ix, const WaveView& wv, int w, int delta_d, int S,
                                 cudaStream_t st);
cudaError_t launch_res_terms(const float* qrot, int64_t B, int32_t D, int32_t Dpad, const float* var,
                             int delta_d, int S, float m, float* res_q, cudaStream_t st);
// The tensor-core estimate-and-prune scan of the learned test (scan_tc.cu):
// units of up to kTcRows candidates x 128 queries, nsteps steps (the last
// one the final test on the completed distance when final_test).
bool tc_scan_supported(int delta_d);
int tc_scan_qmax(int delta_d);  // queries per unit of the tensor-core scan
cudaError_t launch_wave_scan_tc(const IndexView& ix, const WaveView& wv, int w, int delta_d, const float* m1,
                                const float* beta, int nsteps, int parts, bool final_test, cudaStream_t st);
cudaError_t launch_merge(const IndexView& ix, const WaveView& wv, int w, cudaStream_t st);
cudaError_t launch_output(const WaveView& wv, int64_t* ids, float* dists,
                          const int64_t* offsets, cudaStream_t st);
cudaError_t launch_collect(const IndexView& ix, const WaveView& wv, int w, int delta_d, int S,
                           const CollectArgs& ca, int64_t query_offset, cudaStream_t st);

}  // namespace dade
