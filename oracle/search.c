/*
 * Oracle refinement loop, FP64, plain C.  TEST INFRASTRUCTURE ONLY: the
 * product path never links or calls this file.
 *
 * What it computes (arXiv 2404.16322):
 *  - Candidates of a query are the members of its probed IVF buckets
 *    (Section II-A), visited in canonical order: probe rank, then bucket
 *    storage order.
 *  - For a candidate x, the partial distance after s steps is
 *    dis'_s = sum_{j < s*dd} (q'_j - x'_j)^2 over the rotated query and the
 *    stored rotated vector: the plain PCA partial distance of Section V-B
 *    ("Approximate Distances"), grown dd dimensions at a time as in the loop
 *    of Algorithm 2.
 *  - After each step s < S the learned test of Section V-A is applied:
 *    prune iff m1_s * dis'_s + beta_s > tau ("Incremental Correction" gives
 *    one classifier per step).  A disabled step has m1 = 0, beta = -inf.
 *  - Or (RES) the Gaussian-bound test of Section IV-C and Algorithms 1-2:
 *    with d = s*dd, the estimate C1 - C2 of Eq. 1 -- here dis'_s plus the
 *    residual norms ||x_r||^2 + ||q_r||^2 over dims [d, D) -- is corrected by
 *    m * sigma, sigma^2 = 4 sum_{i >= d} q_i^2 sigma_i^2 (Eq. 2), and the
 *    candidate is pruned iff C1 - C2 - m sigma > tau.  sigma_i^2 is the
 *    variance of rotated dimension i over the indexed vectors; x_r is taken
 *    at the stored precision, like dis'_s, so the estimate is exact at d = D.
 *  - Or (ADS) the test of Section III (Distance Estimation / Distance
 *    Correction): over a random rotation, dis' = (D/d) dis'_s estimates dis
 *    from the first d dims, and the candidate is pruned iff
 *    dis' > (1 + eps) tau.  eps = eps0 / sqrt(d): the lemma's failure
 *    probability 2 exp(-c0 d eps^2) equals the significance level
 *    2 exp(-c0 eps0^2) of the test exactly when d eps^2 = eps0^2.
 *  - Or (OPQ-L, Section V-B "Approximate Distances") one test before the
 *    exact distance, on the asymmetric distance dis' = sum_j lut_q[j][code_j]
 *    of the vector's product-quantisation codes and its quantisation error
 *    e: pruned iff m1 dis' + m3 e + beta > tau (the learned classifier with
 *    three features); a pruned candidate scans no rotated dimension.
 *  - A candidate that passes every test adds the last slab, which completes
 *    the rotated distance dis'_S at the stored precision.  At d = D
 *    Algorithm 2's test has no residual term and compares the distance with
 *    tau itself; here the candidate is kept iff
 *    dis'_S <= (sqrt(tau) + e_x)^2 (1 + final_rel), where e_x = ||x' - x~||
 *    is the stored vector's quantisation error (0 for FP32 slabs): by the
 *    triangle inequality a rotated distance <= tau implies that bound, and
 *    final_rel covers floating-point rounding.
 *  - A kept candidate gets its exact distance sum_j (x_j - q_j)^2 from the
 *    original FP32 vectors (Section II-A), and enters the result queue iff
 *    it beats the queue's largest entry (Section I: tau is the largest
 *    distance in the queue).  Ties are ordered by id; tau = +inf while the
 *    queue holds fewer than K.
 *
 * tau schedules (the paper updates tau after every insertion and is silent
 * on parallel order):
 *  - SEQUENTIAL: tau is re-read before every candidate (Section I heap loop).
 *  - WAVES: probe ranks are cut into waves [b_w, b_{w+1}) with b_0 = 0,
 *    b_1 = first_wave, b_{w+1} = 2^g b_w (g >= 1); every candidate of a wave
 *    is tested against the tau left by the previous waves; survivors are
 *    then merged.
 *  - FROZEN: every candidate is tested against a given tau_q; survivors with
 *    exact distance <= tau_q form the result (top-K by (distance, id)).
 */
#include <math.h>
#include <omp.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

enum { MODE_SEQUENTIAL = 0, MODE_WAVES = 1, MODE_FROZEN = 2 };

typedef struct {
    double d;
    int64_t id;
} entry;

static int entry_less(entry a, entry b) { return a.d < b.d || (a.d == b.d && a.id < b.id); }

/* Result queue: the K best entries so far, kept sorted ascending. */
typedef struct {
    entry* e;
    int n;
    int K;
} result_queue;

static double queue_tau(const result_queue* q) { return q->n < q->K ? INFINITY : q->e[q->K - 1].d; }

static void queue_offer(result_queue* q, entry x)
{
    if (q->K <= 0) return;
    if (q->n == q->K) {
        if (!entry_less(x, q->e[q->n - 1])) return;
        q->n--;
    }
    int i = q->n;
    while (i > 0 && entry_less(x, q->e[i - 1])) {
        q->e[i] = q->e[i - 1];
        i--;
    }
    q->e[i] = x;
    q->n++;
}

static double exact_distance(const float* x, const float* q, int D)
{
    double s = 0.0;
    for (int j = 0; j < D; j++) {
        double t = (double)x[j] - (double)q[j];
        s += t * t;
    }
    return s;
}

/* Terms of the RES and ADS tests.  kind 1 (RES): a query's suffix sums
 * over dims [d, D) of q_i^2 and of q_i^2 sigma_i^2 (arrays of D + 1), the
 * multiplier m, and a candidate scratch of 2 (D + 1) doubles for its suffix
 * sums of x_i^2 (and of their deviation bounds, see rounding below).  kind 2
 * (ADS): eps0. */
typedef struct {
    int kind;
    const double* rq;
    const double* sg;
    double m;
    double* rx;
    double eps0;
} res_terms;

/* How far another implementation of the same arithmetic may stray.  A test
 * "prune iff L > T(tau)" (T increasing in tau) is CERTAIN when it comes out
 * the same for every tau' in [tau_lo, tau_hi] (the range of tau the other
 * side can hold, see search_one) and every L' within
 *     slack = amb * tau_hi + (the test's weight) * flip
 * of L: amb is a band relative to tau for FP32 rounding; flip bounds the
 * change of the partial distance if the other side's stored value of
 * coordinate j lies anywhere in xs_j +- xdev_j (its rotation, rounded
 * differently, may cross a rounding midpoint of the storage format, or move
 * a per-dimension scale) and its rotated query coordinate in qr_j +- qdev_j:
 * sum over the dims so far of 2 |q_j - xs_j| e_j + e_j^2, e_j = xdev_j +
 * qdev_j.  NULL: no deviation. */
typedef struct {
    double amb;
    const double* xdev;
    const double* qdev;  /* D: the same for the rotated query, or NULL */
    double norm_eps;     /* the other side computes dis' as ||q||^2 + ||x~||^2 - 2 <q, x~> over the d dims
                            so far: slack norm_eps * max(d, 16) * (||q||^2 + ||x~||^2) */
} rounding;

/* Decision of one test for the oracle's own tau (returns 1 = prune) and
 * whether it is certain under the rounding model. */
static int decide(double L, double slack, double T_own, double T_lo, double T_hi, int* uncertain)
{
    int prune = L > T_own;
    int sure = prune ? (L - slack > T_hi) : (L + slack < T_lo);
    if (!sure) *uncertain = 1;
    return prune;
}

/* Steps s = 1..S-1 of the estimate-and-test loop.  tau3 = {own tau, tau_lo,
 * tau_hi}.  Returns the number of steps taken (the step at which the
 * candidate was pruned, or S when it passed every test); *pruned tells
 * which and *uncertain whether any decision taken could differ under the
 * rounding model.  partials (may be NULL) receives dis'_s for every step. */
static int estimate_and_test(const double* qr, const double* qdev, const double* xs, const double* xdev, int D,
                             int dd, int S,
                             const double* m1, const double* beta, const double* tau3, double xerr,
                             double final_rel, int* pruned, double* partials, const rounding* rd,
                             int* uncertain, const res_terms* res)
{
    const double tau = tau3[0], tlo = tau3[1], thi = tau3[2];
    double p = 0.0, f = 0.0, qn = 0.0, xn = 0.0;
    const double ne = rd ? rd->norm_eps : 0.0;
    double band = 0.0;
    if (rd && rd->amb > 0.0) {
        double tb = isfinite(thi) ? thi : tlo;
        band = isfinite(tb) ? rd->amb * tb : 0.0;
    }
    *pruned = 0;
    if (res && res->kind == 1) {
        double* fx = res->rx + (D + 1);
        res->rx[D] = 0.0;
        fx[D] = 0.0;
        for (int j = D - 1; j >= 0; j--) {
            res->rx[j] = res->rx[j + 1] + xs[j] * xs[j];
            fx[j] = fx[j + 1] + (xdev ? 2.0 * fabs(xs[j]) * xdev[j] + xdev[j] * xdev[j] : 0.0);
        }
    }
    for (int s = 1; s < S; s++) {
        int j1 = s * dd < D ? s * dd : D;
        for (int j = (s - 1) * dd; j < j1; j++) {
            double t = qr[j] - xs[j];
            p += t * t;
            if (xdev || qdev) {
                double e = (xdev ? xdev[j] : 0.0) + (qdev ? qdev[j] : 0.0);
                f += 2.0 * fabs(t) * e + e * e;
            }
            if (ne > 0.0) {
                qn += qr[j] * qr[j];
                xn += xs[j] * xs[j];
            }
        }
        if (partials) partials[s - 1] = p;
        double L, w = 1.0, c = 1.0, fl = f + ne * (double)(j1 > 16 ? j1 : 16) * (qn + xn);
        if (res && res->kind == 1) {
            L = p + res->rx[j1] + res->rq[j1] - res->m * 2.0 * sqrt(res->sg[j1]);
            fl = f + res->rx[D + 1 + j1];
        } else if (res && res->kind == 2) {
            w = (double)D / (double)j1;
            L = w * p;
            c = 1.0 + res->eps0 / sqrt((double)j1);
        } else {
            w = fabs(m1[s - 1]);
            L = m1[s - 1] * p + beta[s - 1];
        }
        if (decide(L, band + w * fl, c * tau, c * tlo, c * thi, uncertain)) {
            *pruned = 1;
            return s;
        }
    }
    /* d = D: the last slab, then the test on the whole rotated distance */
    for (int j = (S - 1) * dd; j < D; j++) {
        double t = qr[j] - xs[j];
        p += t * t;
        if (xdev || qdev) {
            double e = (xdev ? xdev[j] : 0.0) + (qdev ? qdev[j] : 0.0);
            f += 2.0 * fabs(t) * e + e * e;
        }
        if (ne > 0.0) {
            qn += qr[j] * qr[j];
            xn += xs[j] * xs[j];
        }
    }
    f += ne * (double)(D > 16 ? D : 16) * (qn + xn);
    if (isfinite(final_rel)) {
        double T[3];
        for (int i = 0; i < 3; i++) {
            double r = sqrt(tau3[i]) + xerr;
            T[i] = isfinite(tau3[i]) ? r * r * (1.0 + final_rel) : INFINITY;
        }
        if (decide(p, band + f, T[0], T[1], T[2], uncertain)) {
            *pruned = 1;
            return S;
        }
    }
    return S;
}

static int64_t wave_end(int64_t b, int first_wave, int g)
{
    if (b == 0) return first_wave;
    return g >= 30 ? ((int64_t)1 << 40) : b << g;
}

typedef struct {
    int32_t D, dd, S, P, Kmax, mode, first_wave, growth;
    double amb, norm_eps, final_rel;
    const double* xerr;
    int32_t est;            /* 0: learned tables, 1: RES, 2: ADS, 3: OPQ-L */
    double est_param;       /* RES: m; ADS: eps0; OPQ-L: m3 */
    int32_t pq_m;           /* OPQ-L: subspaces */
    const uint8_t* pq_codes; /* OPQ-L: N x pq_m codes (rows as Xs) */
    const double* pq_err;   /* OPQ-L: N quantisation errors */
    const double* pq_lut;   /* OPQ-L: B x pq_m x 256 tables */
    const double* var;      /* D: sigma_i^2 (RES) */
    const double* Qr;
    const double* Qdev;     /* B x D bound on the other side's rotated-query deviation, or NULL */
    const float* Q;
    const double* Xs;
    const double* Xdev;     /* N x D bound on the other side's stored-value deviation, or NULL */
    const uint8_t* unc_rows; /* N: 1 = the other side may represent this row otherwise (its every
                                decision is uncertain), or NULL */
    const float* X;
    const int64_t* ids;
    const int64_t* list_off;
    const int64_t* members;
    const int32_t* probes;
    const int32_t* nprobe;
    const int32_t* K;
    const double* m1;
    const double* beta;
    const double* tau_in;
    int64_t* out_ids;
    double* out_d;
    int64_t* stats;  /* per query: candidates, pruned, exact, dims scanned, uncertain candidates */
    double* amb_d;   /* per query: smallest exact distance of an uncertain candidate (+inf: none), or NULL */
} oracle_args;

/* One candidate: estimate, test, and if it survives, its exact distance.
 * tau3 = {own tau, tau_lo, tau_hi}.  Returns 1 if the oracle keeps it;
 * *unc = 1 if another rounding could decide otherwise (then out->d is set
 * even for a pruned candidate). */
static int visit(const oracle_args* a, int64_t b, int64_t pos, const double* tau3, entry* out, int64_t* st,
                 const res_terms* res, int* unc)
{
    const double* qr = a->Qr + b * a->D;
    int pruned;
    int steps;
    rounding rd = {a->amb, a->Xdev, a->Qdev ? a->Qdev + b * a->D : NULL, a->norm_eps};
    *unc = 0;
    if (a->est == 3) {
        const double* t = a->pq_lut + b * (int64_t)a->pq_m * 256;
        const uint8_t* c = a->pq_codes + pos * a->pq_m;
        double dis = 0.0;
        for (int j = 0; j < a->pq_m; j++) dis += t[j * 256 + c[j]];
        double lhs = a->m1[0] * dis + a->est_param * a->pq_err[pos] + a->beta[0];
        double tb = isfinite(tau3[2]) ? tau3[2] : tau3[1];
        pruned = decide(lhs, isfinite(tb) ? a->amb * tb : 0.0, tau3[0], tau3[1], tau3[2], unc);
        steps = 0;
    } else {
        steps = estimate_and_test(qr, rd.qdev, a->Xs + pos * a->D, a->Xdev ? a->Xdev + pos * a->D : NULL, a->D, a->dd,
                                  a->S, a->m1, a->beta, tau3, a->xerr ? a->xerr[pos] : 0.0, a->final_rel,
                                  &pruned, NULL, &rd, unc, res);
    }
    if (a->unc_rows && a->unc_rows[pos]) *unc = 1;
    st[0] += 1;
    if (*unc) st[4] += 1;
    if (pruned || *unc) {
        out->d = exact_distance(a->X + pos * a->D, a->Q + b * a->D, a->D);
        out->id = a->ids[pos];
    }
    if (pruned) {
        int64_t dims = (int64_t)steps * a->dd;
        st[1] += 1;
        st[3] += dims < a->D ? dims : a->D;
        return 0;
    }
    st[2] += 1;
    st[3] += a->D;
    out->d = exact_distance(a->X + pos * a->D, a->Q + b * a->D, a->D);
    out->id = a->ids[pos];
    return 1;
}

/* One query.  Beside the oracle's own result queue q, two more queues bound
 * the tau another implementation can hold when its roundings decide the
 * uncertain candidates otherwise: q_hi holds only the candidates kept with
 * certainty (the fewest entries, so the largest tau), q_lo also every
 * uncertain candidate (the most entries, the smallest tau).  Every later
 * test is judged certain only if it holds for the whole range [tau_lo,
 * tau_hi].  So every candidate not marked uncertain is decided the same way
 * by both sides, and below the smallest exact distance of an uncertain
 * candidate (amb_d) both results hold exactly the same entries. */
static void search_one(const oracle_args* a, int64_t b)
{
    int K = a->K[b];
    int np = a->nprobe[b];
    const int32_t* pr = a->probes + b * a->P;
    int64_t* st = a->stats + 5 * b;
    st[0] = st[1] = st[2] = st[3] = st[4] = 0;
    double amb_d = INFINITY;
    result_queue q, qlo, qhi;
    q.K = qlo.K = qhi.K = K;
    q.n = qlo.n = qhi.n = 0;
    q.e = (entry*)malloc(sizeof(entry) * (size_t)(K > 0 ? K : 1));
    qlo.e = (entry*)malloc(sizeof(entry) * (size_t)(K > 0 ? K : 1));
    qhi.e = (entry*)malloc(sizeof(entry) * (size_t)(K > 0 ? K : 1));
    res_terms rt, *res = NULL;
    double* rbuf = NULL;
    if (a->est == 2) {
        rt.kind = 2;
        rt.eps0 = a->est_param;
        res = &rt;
    }
    if (a->est == 1) {
        const int D = a->D;
        const double* qr = a->Qr + b * D;
        rbuf = (double*)malloc(sizeof(double) * 4 * (size_t)(D + 1));
        double* rq = rbuf;
        double* sg = rbuf + (D + 1);
        rq[D] = 0.0;
        sg[D] = 0.0;
        for (int j = D - 1; j >= 0; j--) {
            rq[j] = rq[j + 1] + qr[j] * qr[j];
            sg[j] = sg[j + 1] + qr[j] * qr[j] * a->var[j];
        }
        rt.rq = rq;
        rt.sg = sg;
        rt.kind = 1;
        rt.m = a->est_param;
        rt.rx = rbuf + 2 * (D + 1);
        res = &rt;
    }

    if (a->mode == MODE_SEQUENTIAL) {
        for (int r = 0; r < np; r++) {
            int l = pr[r];
            for (int64_t m = a->list_off[l]; m < a->list_off[l + 1]; m++) {
                entry e;
                int unc;
                double tau3[3] = {queue_tau(&q), queue_tau(&qlo), queue_tau(&qhi)};
                int kept = visit(a, b, a->members[m], tau3, &e, st, res, &unc);
                if (kept) queue_offer(&q, e);
                if (unc) {
                    if (e.d < amb_d) amb_d = e.d;
                    queue_offer(&qlo, e);
                } else if (kept) {
                    queue_offer(&qlo, e);
                    queue_offer(&qhi, e);
                }
            }
        }
    } else {
        int64_t b0 = 0;
        while (b0 < np) {
            int64_t b1 = a->mode == MODE_FROZEN ? np : wave_end(b0, a->first_wave, a->growth);
            if (b1 > np) b1 = np;
            double tau3[3];
            if (a->mode == MODE_FROZEN) {
                tau3[0] = tau3[1] = tau3[2] = a->tau_in[b];
            } else {
                tau3[0] = queue_tau(&q);
                tau3[1] = queue_tau(&qlo);
                tau3[2] = queue_tau(&qhi);
            }
            int64_t cap = 0;
            for (int64_t r = b0; r < b1; r++) cap += a->list_off[pr[r] + 1] - a->list_off[pr[r]];
            entry* surv = (entry*)malloc(sizeof(entry) * (size_t)(cap > 0 ? cap : 1));
            int8_t* flag = (int8_t*)malloc((size_t)(cap > 0 ? cap : 1));  /* bit 0 kept, bit 1 uncertain */
            int64_t ns = 0;
            for (int64_t r = b0; r < b1; r++) {
                int l = pr[r];
                for (int64_t m = a->list_off[l]; m < a->list_off[l + 1]; m++) {
                    int unc;
                    int kept = visit(a, b, a->members[m], tau3, &surv[ns], st, res, &unc);
                    if (kept && a->mode == MODE_FROZEN) {
                        /* a frozen search keeps an exact distance iff it is <= tau */
                        double t = tau3[0];
                        if (isfinite(t) && fabs(surv[ns].d - t) <= a->amb * t) unc = 1;
                        kept = surv[ns].d <= t;
                    }
                    if (kept || unc) {
                        flag[ns] = (int8_t)((kept ? 1 : 0) | (unc ? 2 : 0));
                        ns++;
                    }
                }
            }
            for (int64_t i = 0; i < ns; i++) {
                if (flag[i] & 1) queue_offer(&q, surv[i]);
                if (flag[i] & 2) {
                    if (surv[i].d < amb_d) amb_d = surv[i].d;
                    queue_offer(&qlo, surv[i]);
                } else {
                    queue_offer(&qlo, surv[i]);
                    queue_offer(&qhi, surv[i]);
                }
            }
            free(surv);
            free(flag);
            b0 = b1;
        }
    }
    for (int k = 0; k < a->Kmax; k++) {
        a->out_ids[b * a->Kmax + k] = k < q.n ? q.e[k].id : -1;
        a->out_d[b * a->Kmax + k] = k < q.n ? q.e[k].d : INFINITY;
    }
    if (a->amb_d) a->amb_d[b] = amb_d;
    free(q.e);
    free(qlo.e);
    free(qhi.e);
    free(rbuf);
}

int oracle_search(int64_t B, int32_t D, int32_t delta_d, int32_t S, int32_t P, int32_t Kmax,
                  int32_t mode, int32_t first_wave, int32_t growth, double amb, double norm_eps, double final_rel,
                  int32_t est, double est_param, const double* var,
                  int32_t pq_m, const uint8_t* pq_codes, const double* pq_err, const double* pq_lut,
                  const double* Qr, const double* Qdev, const float* Q, const double* Xs, const double* Xdev, const uint8_t* unc_rows,
                  const double* xerr, const float* X, const int64_t* ids, const int64_t* list_off,
                  const int64_t* members, const int32_t* probes, const int32_t* nprobe,
                  const int32_t* K, const double* m1, const double* beta, const double* tau_in,
                  int64_t* out_ids, double* out_d, int64_t* stats, double* amb_d)
{
    if (delta_d <= 0 || S < 1 || first_wave < 1 || growth < 1 || mode < 0 || mode > 2 || !(final_rel >= 0.0) ||
        !(amb >= 0.0) || !(norm_eps >= 0.0) || est < 0 || est > 3 || (est == 1 && (!var || !(est_param >= 0.0))) ||
        (est == 2 && !(est_param >= 0.0 && est_param < INFINITY)) ||
        (est == 3 && (pq_m < 1 || !pq_codes || !pq_err || !pq_lut || !m1 || !beta)))
        return 1;
    oracle_args a = {D, delta_d, S, P, Kmax, mode, first_wave, growth, amb, norm_eps, final_rel, xerr, est, est_param,
                     pq_m, pq_codes, pq_err, pq_lut, var, Qr, Qdev, Q, Xs, Xdev, unc_rows, X, ids, list_off, members, probes,
                     nprobe, K, m1, beta, tau_in, out_ids, out_d, stats, amb_d};
#pragma omp parallel for schedule(dynamic, 1)
    for (int64_t b = 0; b < B; b++) search_one(&a, b);
    return 0;
}

/* Replay with pruning off under the WAVES schedule and record, for every
 * candidate, its partial distances dis'_1..dis'_{S-1}, the tau it would be
 * tested against, its exact distance, query index and id.  Row offsets per
 * query are given by the caller (row_off[b] = first row of query b). */
int oracle_collect(int64_t B, int32_t D, int32_t delta_d, int32_t S, int32_t P, int32_t first_wave, int32_t growth,
                   const double* Qr, const float* Q, const double* Xs, const float* X,
                   const int64_t* ids, const int64_t* list_off, const int64_t* members,
                   const int32_t* probes, const int32_t* nprobe, const int32_t* K,
                   const int64_t* row_off, double* partials, double* tau_out, double* dis_out,
                   int64_t* id_out)
{
    if (delta_d <= 0 || S < 1 || first_wave < 1 || growth < 1) return 1;
    double* never = (double*)malloc(sizeof(double) * (size_t)(S > 1 ? S - 1 : 1));
    for (int s = 0; s < S - 1; s++) never[s] = 0.0;
#pragma omp parallel for schedule(dynamic, 1)
    for (int64_t b = 0; b < B; b++) {
        const int32_t* pr = probes + b * P;
        int np = nprobe[b];
        result_queue q;
        q.K = K[b];
        q.n = 0;
        q.e = (entry*)malloc(sizeof(entry) * (size_t)(q.K > 0 ? q.K : 1));
        int64_t row = row_off[b];
        int64_t b0 = 0;
        double* neg_inf = (double*)malloc(sizeof(double) * (size_t)(S > 1 ? S - 1 : 1));
        for (int s = 0; s < S - 1; s++) neg_inf[s] = -INFINITY;
        while (b0 < np) {
            int64_t b1 = wave_end(b0, first_wave, growth);
            if (b1 > np) b1 = np;
            double tau = queue_tau(&q);
            int64_t row0 = row;
            for (int64_t r = b0; r < b1; r++) {
                int l = pr[r];
                for (int64_t m = list_off[l]; m < list_off[l + 1]; m++) {
                    int64_t pos = members[m];
                    int pruned, unc = 0;
                    const double tau3[3] = {tau, tau, tau};
                    estimate_and_test(Qr + b * D, NULL, Xs + pos * D, NULL, D, delta_d, S, never, neg_inf, tau3, 0.0,
                                      INFINITY, &pruned, partials + row * (S > 1 ? S - 1 : 0), NULL, &unc, NULL);
                    tau_out[row] = tau;
                    dis_out[row] = exact_distance(X + pos * D, Q + b * D, D);
                    id_out[row] = ids[pos];
                    row++;
                }
            }
            for (int64_t i = row0; i < row; i++) {
                entry e = {dis_out[i], id_out[i]};
                queue_offer(&q, e);
            }
            b0 = b1;
        }
        free(neg_inf);
        free(q.e);
    }
    free(never);
    return 0;
}

void oracle_set_threads(int n) { omp_set_num_threads(n > 0 ? n : 1); }

int oracle_max_threads(void) { return omp_get_max_threads(); }
