/*
 * dade.h -- C ABI of the GB300 data-aware distance estimation library.
 *
 * Method: "Effective and General Distance Computation for Approximate Nearest
 * Neighbor Search" (arXiv 2404.16322).  The database and the queries are
 * rotated by a PCA matrix learned from the data (Section IV-B, Theorem 1);
 * IVF buckets supply the candidates (Section II-A); each candidate's squared
 * L2 distance is accumulated Delta_d rotated dimensions at a time (the loop
 * of Algorithm 2) and after each step the learned test
 * m1_s * dis' + beta_s > tau decides whether to prune it (Section V-A, V-B
 * "Incremental Correction"); a candidate that passes every test gets its
 * exact distance, is compared with tau itself (Algorithm 2 at d = D) and
 * competes for the result queue whose largest entry is tau (Section I).
 *
 * Conventions for every entry point:
 *  - Every call returns a dade_status; none aborts or exits.  On failure
 *    dade_last_error() gives a message (per calling thread).
 *  - Pointers named *_host are host memory, *_dev device memory of the
 *    current CUDA device.  The caller owns every buffer it passes and the
 *    library never frees or retains them past the call (device buffers
 *    passed to dade_search must stay valid until the stream reaches the end
 *    of the call's work).
 *  - Matrices are row-major, float32 unless stated, with no padding between
 *    rows.  D is the dimensionality of the vectors (1 <= D <= 4096).
 *  - A dade_index is owned by the library: create it with ivf_build or
 *    dade_index_load and release it with dade_index_free.  Its data live in
 *    device memory of the device that was current when it was created.
 */
#ifndef DADE_H
#define DADE_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct dade_index dade_index;

typedef enum {
    DADE_OK = 0,
    DADE_EINVAL = 1,   /* an argument is out of range or inconsistent        */
    DADE_ENOMEM = 2,   /* a host or device allocation failed                 */
    DADE_ECUDA = 3,    /* a CUDA runtime call failed                         */
    DADE_ETIMEOUT = 4, /* a bounded device wait gave up (status word)        */
    DADE_ESTATE = 5,   /* the index lacks what the call needs (e.g. table)   */
    DADE_ENOTIMPL = 6, /* the combination of options is not supported        */
    DADE_EIO = 7       /* file read/write failed or the file is malformed    */
} dade_status;

/* Precision of the rotated slabs read by the estimate-and-prune stage.  The
 * exact distance always uses the original FP32 vectors. */
typedef enum {
    DADE_SLAB_F32 = 0,
    DADE_SLAB_BF16 = 1,    /* round-to-nearest-even of the FP32 value       */
    DADE_SLAB_FP8E4M3 = 2  /* per-dimension scale amax_j / 448, RNE, saturate */
} dade_slab_dtype;

/* ------------------------------------------------------------------------
 * dade_train_rotation -- PCA rotation (Section IV-B, Theorem 1; data centred
 * per the footnote to Section IV-B).
 *
 * X_host: n x D FP32 rows.  If 0 < sample_n < n, a seeded uniform sample of
 * sample_n distinct rows is used (the paper samples 1M rows for large sets,
 * Section VII "Exp-1"); otherwise every row.  Computes, in FP64 on the host,
 * mean_out[D], the covariance 1/(m-1) sum (x-mean)(x-mean)^T and its
 * eigendecomposition (cyclic Jacobi): eigvals_out[D] descending and R_out
 * [D x D] whose row i is the i-th eigenvector, with the sign making the
 * entry of largest magnitude in each row positive.  All outputs are host
 * buffers owned by the caller.  Errors: DADE_EINVAL (n < 2, D out of range,
 * null pointers), DADE_ENOMEM.
 * ---------------------------------------------------------------------- */
dade_status dade_train_rotation(const float* X_host, int64_t n, int32_t D, int64_t sample_n,
                                uint64_t seed, double* mean_out, double* R_out,
                                double* eigvals_out);

/* ------------------------------------------------------------------------
 * ADS baseline (Section III, "Distance Estimation" and "Distance
 * Correction"): a random rotation and a scaled partial-distance test, run
 * by the same search kernels through a correction table.
 *
 * dade_random_rotation: R_out[D x D] (host, caller-owned FP64) is a random
 * orthogonal matrix from the Haar measure, row i the i-th output axis
 * (x' = R x): the positive-diagonal QR factor of a seeded standard Gaussian
 * matrix.  Pass it to ivf_build in place of the PCA rotation.
 *
 * dade_ads_table: the table (m1_s, beta_s), s = 1..S-1, S = ceil(D/delta_d),
 * for which the search's test m1_s dis'_s + beta_s > tau is ADS's test
 * (D/d) dis'_s > (1 + eps) tau with d = min(s delta_d, D) and
 * eps = eps0 / sqrt(d) (the lemma's failure probability 2 exp(-c0 d eps^2)
 * held at the significance level 2 exp(-c0 eps0^2)): m1_s = (D/d) / (1 + eps),
 * beta_s = 0.  Install it with dade_set_correction.  The paper's setting is
 * eps0 = 2.1 with delta_d = 32.  m1_out, beta_out: host, S - 1 floats.
 * Errors: DADE_EINVAL (null pointer, D or delta_d out of range, eps0 < 0 or
 * not finite).
 * ---------------------------------------------------------------------- */
dade_status dade_random_rotation(int32_t D, uint64_t seed, double* R_out);

dade_status dade_ads_table(int32_t D, int32_t delta_d, double eps0, float* m1_out, float* beta_out);

/* ------------------------------------------------------------------------
 * ivf_build -- rotate the database and build the IVF index (Section II-A).
 *
 * X: N x D FP32 rows in host memory or in device memory of the current
 * device (told apart with cudaPointerGetAttributes; device rows are read in
 * place, host rows are copied up once); mean[D], R[D x D] FP64 from
 * dade_train_rotation
 * (or any orthogonal matrix).  The rows are rotated on the device,
 * x' = R (x - mean), clustered into nlist buckets by Lloyd k-means in the
 * rotated space (kmeans_iters iterations from a seeded sample of nlist
 * rows; a point goes to the nearest centroid, the lower id on a tie; an
 * empty bucket keeps its centroid), and laid out per bucket:
 *  - rotated slabs, dimension-blocked: 8 dimensions per block, block b of
 *    the bucket's vector i at ((b * npad + i) * 8 + j) elements from the
 *    bucket's base, npad = bucket size rounded up to 32, in params->dtype;
 *  - the original FP32 vectors in the same blocked layout (exact distance);
 *  - for BF16 / FP8 slabs, each vector's quantisation error norm
 *    e_x = ||x' - x~|| (FP32 rotated vector minus its stored value);
 *  - the ids (params->ids, or the row numbers when NULL) as int64.
 * Inside a bucket, vectors keep increasing row order.  params->centroids
 * (nlist x D rotated-space FP32, host) replaces k-means when non-NULL;
 * params->assign (N bucket ids, host) also replaces the assignment.
 * Errors: DADE_EINVAL (also: X in another device's memory), DADE_ENOMEM,
 * DADE_ECUDA.  *out is set only on success.
 * ---------------------------------------------------------------------- */
typedef struct {
    int32_t nlist;
    int32_t kmeans_iters;
    uint64_t seed;
    dade_slab_dtype dtype;
    const float* centroids;  /* optional, host, nlist x D (rotated space) */
    const int32_t* assign;   /* optional, host, N (needs centroids)       */
    const int64_t* ids;      /* optional, host, N                         */
} dade_build_params;

dade_status ivf_build(const float* X, int64_t N, int32_t D, const double* mean,
                      const double* R, const dade_build_params* params, dade_index** out);

/* ------------------------------------------------------------------------
 * Correction tables.  For a step width delta_d (a multiple of 8) the index
 * holds S - 1 pairs (m1_s, beta_s), S = ceil(D / delta_d): after s slabs the
 * candidate is pruned iff m1_s * dis'_s + beta_s > tau (Section V-A, one
 * classifier per step as in "Incremental Correction", Section V-B).  m1 = 0,
 * beta = -inf disables a step.
 *
 * dade_fit_correction learns them (Section V-A "Parameter Learning" and
 * "Adaptive Adjustment", labels per Section VII-A): train_q_host (nt x D
 * FP32) are searched with pruning off under the same tau schedule as
 * dade_search (nprobe, K, first wave 1); every candidate tested against a
 * finite tau gives a sample (dis'_1..dis'_{S-1}, tau) labelled 0 if it is in
 * the query's exact top-K, 1 if its exact distance exceeds tau (others are
 * dropped); label-1 samples are thinned to about label1_cap by a
 * counter-based SplitMix64 draw of (seed, query, id).  Then, per step on the
 * samples no earlier step prunes, an FP64 logistic regression on
 * (dis'/tau_bar, tau/tau_bar) gives m1 = -w1/w2, and beta' is the largest
 * value keeping label-0 recall >= r_s = 1 - (1 - target_recall) / S.
 * m1_out / beta_out (host, S - 1 floats, may be NULL) receive the table,
 * which is also installed in the index.  Steps with w2 >= 0, fewer than 100
 * label-0 samples or no label-1 sample are disabled.
 * Errors: DADE_EINVAL, DADE_ENOMEM, DADE_ECUDA.
 *
 * dade_fit_collect returns the samples dade_fit_correction would fit on
 * (same arguments, same replay, labels and thinning), for inspection: up
 * to max_rows rows sorted by (query, id) into partials (n x (S-1) FP32:
 * dis'_1..dis'_{S-1} at the stored precision), tau (n), label (n: 0 or 1),
 * query (n: index into train_q_host) and id (n), all host, caller-owned;
 * *n_rows receives the row count (also when it exceeds max_rows, which
 * returns DADE_EINVAL so that the caller can retry with more room).
 *
 * dade_fit_samples runs the host FP64 fit alone on caller samples:
 * partials (n x (S-1)), tau (n), label (n: 0 or 1); outputs S - 1 doubles.
 *
 * dade_set_correction installs a caller table (host floats, S - 1 each).
 * dade_get_correction copies the installed table out (DADE_ESTATE if none).
 * ---------------------------------------------------------------------- */
dade_status dade_fit_correction(dade_index* idx, const float* train_q_host, int64_t nt,
                                int32_t K, int32_t nprobe, int32_t delta_d,
                                double target_recall, uint64_t seed, int64_t label1_cap,
                                float* m1_out, float* beta_out);

dade_status dade_fit_collect(dade_index* idx, const float* train_q_host, int64_t nt, int32_t K, int32_t nprobe,
                             int32_t delta_d, uint64_t seed, int64_t label1_cap, int64_t max_rows, int64_t* n_rows,
                             float* partials_host, float* tau_host, int8_t* label_host, int64_t* query_host,
                             int64_t* id_host);

/* dade_partials_collect: every candidate of each query's nprobe nearest
 * buckets (Q_host: nq x D FP32 queries, original space), each with its
 * partial distances dis'_1..dis'_{S-1} (S = ceil(Dpad / delta_d)) over the
 * stored slabs, computed by the search's CUDA-core arithmetic (the partial
 * squared distance of Section IV-B over the first s * delta_d rotated
 * dims): the estimate-quality measurement of Section VII (Exp-7) on the
 * device.  Rows are sorted by (query, id) into partials (n x (S-1)), query
 * (n) and id (n), host, caller-owned; *n_rows receives the count, also when
 * it exceeds max_rows, which returns DADE_EINVAL.  Errors: DADE_EINVAL
 * (nprobe outside [1, nlist], delta_d not 8/16/32), DADE_ENOMEM, DADE_ECUDA. */
dade_status dade_partials_collect(const dade_index* idx, const float* Q_host, int64_t nq, int32_t nprobe,
                                  int32_t delta_d, int64_t max_rows, int64_t* n_rows, float* partials_host,
                                  int64_t* query_host, int64_t* id_host);

dade_status dade_fit_samples(const double* partials, const double* tau, const int8_t* label,
                             int64_t n, int32_t D, int32_t delta_d, double target_recall,
                             int32_t min_label0, double* m1_out, double* beta_out);

dade_status dade_set_correction(dade_index* idx, int32_t delta_d, const float* m1_host,
                                const float* beta_host);

dade_status dade_get_correction(const dade_index* idx, int32_t delta_d, float* m1_host,
                                float* beta_host);

/* ------------------------------------------------------------------------
 * dade_search -- batched AKNN search on one stream.
 *
 * Q_dev: B x D FP32 queries.  K_dev[B], nprobe_dev[B]: per-query K
 * (1..opts->max_K) and nprobe (1..min(opts->max_nprobe, nlist)); a query
 * with K = 0 or nprobe = 0 is an inactive slot (no work, padded output), so
 * a fixed-capacity batch can carry fewer live queries.
 * Pipeline, all on cuda_stream (a cudaStream_t; NULL = legacy default):
 *  1. q' = R (q - mean) for every query (Section IV-A x_D = R x).
 *  2. squared distance of q' to every centroid; the nprobe nearest, ordered
 *     by (distance, list id), are the query's buckets (Section II-A).
 *  3. probe ranks are cut into waves [b_w, b_{w+1}): b_0 = 0,
 *     b_1 = first_wave, b_{w+1} = 2^g b_w (g = opts->wave_growth_log2).
 *     Every candidate of wave w is tested
 *     against the query's tau at the end of wave w - 1 (tau = +inf before the
 *     queue holds K entries), in parallel over (bucket, query) work units.
 *  4. mode DADE_SCAN_PRUNE: the candidate's partial distance over the rotated
 *     slabs grows delta_d dims per step and the installed table for delta_d
 *     decides pruning after each of the first S - 1 steps (or, with
 *     opts->estimator = DADE_EST_RES, the Gaussian-bound test below); with
 *     opts->final_test a survivor adds the last slab and is pruned iff
 *     dis'_S > (sqrt(tau) + e_x)^2 (1 + 1e-3) (a rotated distance <= tau
 *     implies dis'_S <= (sqrt(tau) + e_x)^2; the 1e-3 covers FP32 rounding);
 *     the rest get the exact FP32 distance from the original vectors.
 *     mode DADE_SCAN_FULL:
 *     every candidate gets the exact FP32 distance (no estimate, no table).
 *     DADE_EST_RES (Section IV-C, Algorithms 1-2, Eq. 1-2): after the step
 *     that completes dims [0, d) the candidate is pruned iff
 *       dis'_d + ||x~_r||^2 + ||q'_r||^2 - m * 2 sqrt(sum_{i>=d} q'_i^2 s_i^2) > tau
 *     where x~_r, q'_r are the stored vector and the rotated query over
 *     dims [d, D), s_i^2 is the variance of rotated dim i over the indexed
 *     vectors (computed at build) and m = opts->res_m.  It needs no
 *     correction table.
 *  5. candidates with exact distance <= tau join the query's top-K, ordered
 *     by (distance, id); tau becomes its K-th distance.
 * Outputs: for query b, ids_dev / dists_dev at [off_b, off_b + K_b) with
 * off = out_offsets_dev (B + 1 int64 prefix of K) or, when it is NULL,
 * off_b = b * max_K.  Fewer than K results pad with id -1 and +inf.
 * The call is asynchronous: it enqueues work and returns.  It performs no
 * host synchronisation.  With opts->workspace given it allocates nothing;
 * without, it uses scratch that the index keeps per stream (allocated
 * stream-ordered with cudaMallocAsync when a stream first needs more, kept
 * until dade_index_free), so searches of one index on distinct streams may
 * run concurrently, and a stream that has warmed up allocates no more.
 * Errors found on the host return at once (DADE_EINVAL, DADE_ESTATE when
 * delta_d has no table in PRUNE mode, DADE_ECUDA on a launch failure).
 * Errors found on the device (K or nprobe out of range, a timed-out wait)
 * set the int32 at opts->status_dev (if given) to a nonzero dade_status;
 * it is never cleared by the library.
 * ---------------------------------------------------------------------- */
typedef enum { DADE_SCAN_PRUNE = 0, DADE_SCAN_FULL = 1 } dade_scan_mode;
typedef enum { DADE_EST_LEARNED = 0, DADE_EST_RES = 1, DADE_EST_PQ = 2 } dade_estimator;

typedef struct {
    int32_t mode;            /* dade_scan_mode                                    */
    int32_t max_K;           /* required: bound on K_dev[b], <= 1024              */
    int32_t max_nprobe;      /* required: bound on nprobe_dev[b]                  */
    int32_t first_wave;      /* buckets in the first wave; 0 means 1              */
    const float* tau_dev;    /* optional B floats: one frozen tau per query and a */
                             /* single wave (candidates with exact dist > tau are */
                             /* dropped).  NULL: the wave schedule above.         */
    const int32_t* probe_in_dev; /* optional B x max_nprobe: given buckets       */
    int32_t* probe_out_dev;  /* optional B x max_nprobe: buckets probed           */
    float* qrot_out_dev;     /* optional B x D: the rotated queries q'            */
    int64_t* stats_dev;      /* optional B x 4, accumulated: candidates, pruned,  */
                             /* exact distances, rotated+exact dims scanned       */
    int32_t* status_dev;     /* optional int32 device status word                 */
    void* workspace;         /* optional device scratch of workspace_bytes        */
    size_t workspace_bytes;
    int32_t wave_growth_log2;  /* g: each wave after the first is 2^g times the */
                               /* previous one (0 means 1: doubling); 30 puts   */
                               /* every rank after the first wave in one wave   */
    int32_t final_test;      /* PRUNE mode, nonzero: the test on the completed   */
                             /* rotated distance (step 4) runs before the exact  */
                             /* distance.  It never changes the results (it only */
                             /* drops candidates with exact distance > tau); it  */
                             /* trades a last slab step for fewer exact          */
                             /* distances.  0: survivors of step S - 1 go        */
                             /* straight to the exact distance.                  */
    int32_t estimator;       /* PRUNE mode: dade_estimator (0: learned tables;  */
                             /* DADE_EST_PQ: OPQ-L, see dade_pq_train; it      */
                             /* ignores delta_d and refuses final_test and     */
                             /* test_steps with DADE_ENOTIMPL)                 */
    float res_m;             /* DADE_EST_RES: the multiplier m of sigma, >= 0   */
                             /* (larger m prunes less; the paper's default 8)  */
    int32_t test_steps;      /* PRUNE mode: only the first test_steps steps are */
                             /* tested; their survivors go straight to the     */
                             /* exact distance (the same results as a table    */
                             /* whose later steps are disabled).  0: all S - 1. */
                             /* Not with final_test (DADE_ENOTIMPL).           */
    int32_t scan_kernel;     /* PRUNE mode with the learned test (tables, ADS):  */
                             /* dade_scan_kernel: which kernel runs the waves   */
                             /* whose tau is finite.  0 (auto) = tensor cores.  */
    int64_t candidate_budget_bytes; /* bound of the candidate buffer (8 bytes  */
                             /* per candidate a pass can append for a query in */
                             /* the worst case: the sum of its largest buckets);*/
                             /* a wave over the bound is scanned in passes of  */
                             /* fewer probe ranks, all tested against the      */
                             /* wave's tau (results do not change).  0: 8 GiB. */
                             /* The bound grows if it would take more than 128 */
                             /* passes.  Each pass costs a scan launch's tail  */
                             /* and a merge: 20,000 requests on 10M x 96 ran   */
                             /* 26 passes in 32 ms at 8 GiB, 2 in 18 ms at 96. */
    int32_t queries_per_unit; /* at most this many queries share one staged   */
                             /* tile of a bucket (a work unit); 0: the scan    */
                             /* kernel's maximum (128 on tensor cores, 16 on   */
                             /* CUDA cores), larger values are clamped to it.  */
                             /* Results do not change, only the time.  >= 0.   */
} dade_search_opts;

/* The estimate-and-prune kernels of the learned test.  DADE_KERNEL_TENSOR:
 * per work unit (a tile of 128 candidates of a bucket against up to 128
 * queries probing it) the partial distances of every pair come from one
 * tcgen05 contraction per step, dis' = ||q||^2 + ||x||^2 - 2 <q, x> over the
 * dims so far (split TF32, FP32 accumulation), and the CUDA cores test them;
 * DADE_KERNEL_CUDA: the FP32 kernel that accumulates (q_j - x_j)^2 per pair
 * (16 queries per unit, survivors compacted in shared memory after every
 * step).  Both test every pair after every step and give the same results
 * up to the rounding of the partial distances (a decision within that
 * rounding of its threshold may differ).  RES and OPQ-L always use the
 * CUDA-core kernels. */
typedef enum { DADE_KERNEL_AUTO = 0, DADE_KERNEL_CUDA = 1, DADE_KERNEL_TENSOR = 2 } dade_scan_kernel;

/* ------------------------------------------------------------------------
 * OPQ-L (Section V-B "Approximate Distances"): the approximate distance is
 * OPQ's asymmetric distance dis' = sum_j ||q'_j - c_j,code_j||^2 over m
 * subspaces of D/m rotated dims (256 centroids each; the query exact), and
 * the learned correction has a third feature, the stored vector's distance
 * e to its quantised reconstruction: a candidate is pruned iff
 * m1 dis' + m3 e + beta > tau, one test before its exact distance.  OPQ's
 * rotation is its parametric solution on the index's PCA basis: the rotated
 * dims, in decreasing variance, are dealt m per round to the subspaces, the
 * larger variances to the subspaces of smaller product of variances so far.
 *
 * dade_pq_train: X_host (n x D FP32, n >= 256) is rotated on the host in
 * FP64; codebooks by Lloyd k-means in FP64 per subspace (iters iterations
 * from a seeded sample of 256 rows); then as dade_pq_set.  perm_out (D
 * int32) and codebooks_out (m x 256 x D/m FP32) may be NULL.
 * dade_pq_set: installs the allocation perm (subspace j's dims at
 * perm[j D/m .. (j + 1) D/m)) and the codebooks, and encodes every stored
 * vector on the device (nearest centroid per subspace, the lower index on a
 * tie; e in FP32).  Replaces any earlier quantiser and its correction.
 * D/m must be <= 64.
 * dade_pq_fit_correction: the classifier fitted on replayed training
 * queries as dade_fit_correction does (same labels and thinning); logistic
 * regression on (dis'/tau_bar, tau/tau_bar, e/sqrt(tau_bar)), m1 = -w1/w2,
 * m3 = -w3 sqrt(tau_bar)/w2, beta' the largest value keeping label-0 recall
 * >= target_recall (w2 >= 0 or too few samples: m1 = m3 = 0, beta = -inf,
 * never prunes).  out3 (host, may be NULL) = {m1, m3, beta'}.
 * dade_pq_fit_samples: that host FP64 fit alone on caller samples.
 * dade_pq_set_correction / dade_pq_get: install / read the classifier; read
 * m, and the codes (N x m, input-row order) and e (N) of the stored vectors.
 * dade_index_save keeps the quantiser and its classifier (the codes are
 * recomputed from the stored vectors at load); dade_index_shard does not
 * carry them.
 * Errors: DADE_EINVAL, DADE_ESTATE (no quantiser), DADE_ENOMEM, DADE_ECUDA.
 * ---------------------------------------------------------------------- */
dade_status dade_pq_train(dade_index* idx, const float* X_host, int64_t n, int32_t m, int32_t iters,
                          uint64_t seed, int32_t* perm_out, float* codebooks_out);

dade_status dade_pq_set(dade_index* idx, int32_t m, const int32_t* perm_host, const float* codebooks_host);

dade_status dade_pq_fit_correction(dade_index* idx, const float* train_q_host, int64_t nt, int32_t K,
                                   int32_t nprobe, double target_recall, uint64_t seed, int64_t label1_cap,
                                   float* out3);

dade_status dade_pq_fit_samples(const double* dis, const double* err, const double* tau, const int8_t* label,
                                int64_t n, double target_recall, int32_t min_label0, double* out3);

dade_status dade_pq_set_correction(dade_index* idx, float m1, float m3, float beta);

dade_status dade_pq_get(const dade_index* idx, int32_t* m_out, float* correction3, uint8_t* codes_host,
                        float* err_host);

dade_status dade_search(const dade_index* idx, const float* Q_dev, int64_t B,
                        const int32_t* K_dev, const int32_t* nprobe_dev, int32_t delta_d,
                        const dade_search_opts* opts, int64_t* ids_dev, float* dists_dev,
                        const int64_t* out_offsets_dev, void* cuda_stream);

/* ------------------------------------------------------------------------
 * dade_search_noalloc -- dade_search for callers that cannot allocate.
 *
 * The paper has no counterpart: this entry point exists for callers that
 * cannot allocate device memory at search time, such as an application whose
 * own allocator has reserved all of the GPU's memory, or a latency-critical
 * path that cannot afford the implicit synchronisation of cudaMalloc.  It
 * runs the same kernels as dade_search, with the same arguments and results,
 * but its scratch is a fixed 64 MiB device array compiled into the library
 * (every GPU that loads the library holds it until the process exits); the
 * call itself performs no cudaMalloc, cudaFree or other allocation.
 *  - opts->workspace must be NULL; a search whose scratch would exceed
 *    64 MiB (dade_search_workspace_size) is rejected with DADE_EINVAL and a
 *    message, before any work is enqueued (e.g. 256 queries of K 100 and
 *    nprobe 64 fit on a 1M-vector index with 4096 buckets).
 *  - The first call on a device looks up the array's device address
 *    (cudaGetSymbolAddress) once for that device; make that first call
 *    before any stream capture.  The address is kept for the life of the
 *    process, so do not use this entry point after a cudaDeviceReset of
 *    that device.
 *  - Invalid arguments return the same status and message as dade_search.
 *  - Every call uses the same array, which keeps the previous call's
 *    contents; each call clears what must start at zero.  Calls whose work
 *    overlaps on the GPU race on the array: serialise them (one stream, or
 *    events between streams).
 * ---------------------------------------------------------------------- */
dade_status dade_search_noalloc(const dade_index* idx, const float* Q_dev, int64_t B,
                                const int32_t* K_dev, const int32_t* nprobe_dev, int32_t delta_d,
                                const dade_search_opts* opts, int64_t* ids_dev, float* dists_dev,
                                const int64_t* out_offsets_dev, void* cuda_stream);

/* Device scratch bytes dade_search needs for B queries with these bounds
 * (the same opts fields as dade_search reads).  0 on invalid arguments. */
size_t dade_search_workspace_size(const dade_index* idx, int64_t B, int32_t delta_d,
                                  const dade_search_opts* opts);

/* The number of kernels one dade_search with these arguments launches
 * (*count), found by capturing the call into a CUDA graph on a private
 * stream and counting its kernel nodes; nothing runs.  The arguments are
 * those of dade_search; opts->workspace is required (the per-stream scratch
 * is not taken inside a capture): DADE_EINVAL without it. */
dade_status dade_search_kernel_count(const dade_index* idx, const float* Q_dev, int64_t B,
                                     const int32_t* K_dev, const int32_t* nprobe_dev, int32_t delta_d,
                                     const dade_search_opts* opts, int64_t* ids_dev, float* dists_dev,
                                     const int64_t* out_offsets_dev, int64_t* count);

/* ------------------------------------------------------------------------
 * Bucket-sharded search (the layout for spreading one index over several
 * GPUs).  The paper has no counterpart: it searches one index on one CPU.
 * dade_shard_owners: owner shard (0 .. n_shards-1) of each of the nlist
 *   buckets, given their sizes (host arrays): buckets in decreasing size
 *   order, ties by lower bucket id, each to the shard with the fewest
 *   vectors so far (ties to the lower shard).  Pure host computation.
 *   Errors: DADE_EINVAL (null pointer, nlist < 1, n_shards outside
 *   [1, nlist], a negative size).
 * dade_index_shard: a new index on the current device holding only the
 *   vectors of the buckets shard `shard` owns (in the same order), with the
 *   parent's rotation, every centroid (so a query probes the same buckets in
 *   every shard) and every correction table.  dade_search on it scans the
 *   owned buckets among the probed ones, with waves and tau of its own.
 *   *out is set only on success.  Errors: DADE_EINVAL, DADE_ENOMEM,
 *   DADE_ECUDA.
 * dade_merge_topk: merges n_parts (<= 32) result lists per query -- part p
 *   of query b at ids_dev / dists_dev[(p * B + b) * max_K ...], each sorted
 *   by (distance, id), ids < 0 padding -- into the K_dev[b] best by
 *   (distance, id) at ids_out_dev / dists_out_dev[b * max_K ...], padded
 *   with -1 / +inf.  With pruning off in every shard, merging the shards'
 *   results gives the unsharded result.  Asynchronous on cuda_stream.
 *   Errors: DADE_EINVAL (n_parts outside [1, 32], max_K outside
 *   [0, 1024], a null pointer), DADE_ECUDA.
 * ---------------------------------------------------------------------- */
dade_status dade_shard_owners(const int64_t* list_size_host, int32_t nlist, int32_t n_shards,
                              int32_t* owner_out_host);
dade_status dade_index_shard(const dade_index* idx, int32_t n_shards, int32_t shard, dade_index** out);
dade_status dade_merge_topk(int32_t n_parts, int64_t B, int32_t max_K, const int32_t* K_dev,
                            const int64_t* ids_dev, const float* dists_dev, int64_t* ids_out_dev,
                            float* dists_out_dev, void* cuda_stream);

/* ------------------------------------------------------------------------
 * Index inspection, persistence and release.
 * dade_index_info fills the sizes.  dade_index_centroids copies the
 * nlist x D rotated-space centroids to the host; dade_index_assignment the
 * bucket of each input row (N int32, host); dade_index_list_sizes the
 * nlist bucket sizes (int64, host).
 * dade_index_stored copies to the host the stored rotated vectors (the
 * values the estimate reads: FP32 slabs as stored, BF16 widened, FP8 codes
 * times their per-dimension scale; Section V-B's "Approximate Distances" at
 * the storage precision) of the input rows [row0, row0 + nrows), row-major
 * nrows x D FP32 in out_host (caller-owned).  For inspecting the
 * quantisation; it allocates a temporary device buffer of nrows x D floats
 * and synchronises.  Errors: DADE_EINVAL (range), DADE_ENOMEM, DADE_ECUDA.
 * dade_index_save writes a versioned binary file (header, rotation, mean,
 * centroids, buckets, slabs, original vectors, ids, quantisation error
 * norms (BF16 / FP8), correction tables, and an FNV-1a checksum);
 * dade_index_load reads it back onto the current device and reproduces
 * identical search results.  Errors: DADE_EIO, DADE_ENOMEM,
 * DADE_ECUDA, DADE_EINVAL.
 * ---------------------------------------------------------------------- */
typedef struct {
    int64_t N;
    int32_t D;
    int32_t Dpad;       /* D rounded up to a multiple of 8 */
    int32_t nlist;
    int32_t dtype;      /* dade_slab_dtype */
    int64_t max_list;   /* largest bucket */
    int64_t device_bytes;
} dade_index_info;

dade_status dade_index_info_get(const dade_index* idx, dade_index_info* out);
dade_status dade_index_centroids(const dade_index* idx, float* centroids_host);
dade_status dade_index_assignment(const dade_index* idx, int32_t* assign_host);
dade_status dade_index_list_sizes(const dade_index* idx, int64_t* sizes_host);
dade_status dade_index_stored(const dade_index* idx, int64_t row0, int64_t nrows, float* out_host);
dade_status dade_index_save(const dade_index* idx, const char* path);
dade_status dade_index_load(const char* path, dade_index** out);
void dade_index_free(dade_index* idx);

/* ------------------------------------------------------------------------
 * Stage timing (tracing).  dade_stage_timing(1) makes every later
 * dade_search record a CUDA event pair around each refinement-scan launch
 * (on the search's stream) and count the bytes that launch stages from
 * device memory (slab blocks copied to shared memory plus original vectors
 * read for exact distances); dade_stage_timing(2) does the same for the
 * tensor-core scan launches alone; dade_stage_timing(0) stops.
 * dade_stage_timing_read synchronises the recorded events and returns the
 * summed milliseconds, the number of launches and the staged bytes since the
 * last read, then resets them.  Process-wide; not for concurrent searches.
 * ---------------------------------------------------------------------- */
dade_status dade_stage_timing(int32_t enable);
dade_status dade_stage_timing_read(double* scan_ms, int64_t* scan_launches, double* scan_bytes);

/* ------------------------------------------------------------------------
 * Workspace arena (host bookkeeping for admission control).  A serving loop
 * holds one device allocation of `bytes` and hands each batch a byte range
 * of it for its dade_search workspace; a batch is admitted when a range is
 * free.  dade_arena_create: ranges are multiples of `align` (a power of
 * two) within [0, bytes rounded down to align); DADE_EINVAL on bad sizes.
 * dade_arena_alloc: the offset of the lowest free range of at least `bytes`
 * (rounded up to align; 0 bytes take one unit), or -1 if none is free.
 * dade_arena_free: releases the range that starts at `offset` (DADE_EINVAL
 * if none does) and merges it with free neighbours.  dade_arena_used: bytes
 * held by live ranges; dade_arena_largest_free: the longest free range.
 * Thread-safe; no device calls (the arena never touches the memory).
 * ---------------------------------------------------------------------- */
typedef struct dade_arena dade_arena;
dade_status dade_arena_create(int64_t bytes, int64_t align, dade_arena** out);
int64_t dade_arena_alloc(dade_arena* arena, int64_t bytes);
dade_status dade_arena_free(dade_arena* arena, int64_t offset);
int64_t dade_arena_used(const dade_arena* arena);
int64_t dade_arena_largest_free(const dade_arena* arena);
void dade_arena_destroy(dade_arena* arena);

/* Message of the last failed call on this thread ("" if none). */
const char* dade_last_error(void);

#ifdef __cplusplus
}
#endif
#endif /* DADE_H */
