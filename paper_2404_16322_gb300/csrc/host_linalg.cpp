// Host FP64 pieces of the library: sample covariance and its symmetric
// eigendecomposition (the PCA rotation of Section IV-B, Theorem 1), and the
// per-step logistic fit with the beta' adjustment (Section V-A).
#include <math.h>
#include <string.h>

#include <algorithm>
#include <thread>
#include <vector>

#include "dade_internal.h"

namespace dade {

uint64_t splitmix64(uint64_t z) {
    // SplitMix64 output function (Steele, Lea, Flood 2014).
    z += 0x9E3779B97F4A7C15ull;
    z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
    z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
    return z ^ (z >> 31);
}

double sample_uniform(uint64_t seed, uint64_t query, uint64_t id) {
    uint64_t z = splitmix64(seed ^ splitmix64((query << 32) ^ id));
    return (double)(z >> 11) * 0x1.0p-53;
}

// ---------------------------------------------------------------------------
// Covariance: mean and 1/(m-1) sum (x - mean)(x - mean)^T over the rows
// listed in `rows` (or all n rows when rows == nullptr), in FP64.  Rows are
// split over host threads; each thread accumulates the upper triangle of its
// share in blocks of 32 rows, and the shares are added in thread order so the
// result does not depend on timing.
dade_status covariance_fp64(const float* X, int64_t n, int32_t D, const int64_t* rows, int64_t m,
                            double* mean, double* cov) {
    if (!rows) m = n;
    unsigned hw = std::max(1u, std::thread::hardware_concurrency());
    int nt = (int)std::min<int64_t>(hw, std::max<int64_t>(1, m / 256));
    auto row_ptr = [&](int64_t i) { return X + (rows ? rows[i] : i) * (int64_t)D; };

    std::vector<std::vector<double>> part_mean(nt, std::vector<double>(D, 0.0));
    std::vector<std::thread> th;
    auto span = [&](int t, int64_t& a, int64_t& b) { a = m * t / nt; b = m * (t + 1) / nt; };
    for (int t = 0; t < nt; ++t)
        th.emplace_back([&, t] {
            int64_t a, b;
            span(t, a, b);
            double* pm = part_mean[t].data();
            for (int64_t i = a; i < b; ++i) {
                const float* x = row_ptr(i);
                for (int j = 0; j < D; ++j) pm[j] += x[j];
            }
        });
    for (auto& x : th) x.join();
    th.clear();
    for (int j = 0; j < D; ++j) {
        double s = 0;
        for (int t = 0; t < nt; ++t) s += part_mean[t][j];
        mean[j] = s / (double)m;
    }

    std::vector<std::vector<double>> part(nt);
    for (int t = 0; t < nt; ++t)
        th.emplace_back([&, t] {
            std::vector<double>& C = part[t];
            C.assign((size_t)D * D, 0.0);
            const int RB = 32;
            std::vector<double> blk((size_t)RB * D);
            int64_t a, b;
            span(t, a, b);
            for (int64_t i0 = a; i0 < b; i0 += RB) {
                int r = (int)std::min<int64_t>(RB, b - i0);
                for (int k = 0; k < r; ++k) {
                    const float* x = row_ptr(i0 + k);
                    for (int j = 0; j < D; ++j) blk[(size_t)j * RB + k] = (double)x[j] - mean[j];
                }
                for (int p = 0; p < D; ++p) {
                    const double* bp = &blk[(size_t)p * RB];
                    double* Cp = &C[(size_t)p * D];
                    for (int q = p; q < D; ++q) {
                        const double* bq = &blk[(size_t)q * RB];
                        double s = 0;
                        for (int k = 0; k < r; ++k) s += bp[k] * bq[k];
                        Cp[q] += s;
                    }
                }
            }
        });
    for (auto& x : th) x.join();
    for (int p = 0; p < D; ++p)
        for (int q = p; q < D; ++q) {
            double s = 0;
            for (int t = 0; t < nt; ++t) s += part[t][(size_t)p * D + q];
            s /= (double)(m - 1);
            cov[(size_t)p * D + q] = s;
            cov[(size_t)q * D + p] = s;
        }
    return DADE_OK;
}

// ---------------------------------------------------------------------------
// Cyclic Jacobi eigenvalue method for a symmetric matrix (Jacobi 1846;
// Golub and Van Loan, "Matrix Computations", Sec. 8.5): sweep over all
// off-diagonal pairs (p, q), apply the plane rotation that zeroes a_pq, and
// accumulate the rotations in V, until the off-diagonal mass is negligible.
// Outputs eigenvalues descending and R with row i = i-th eigenvector, the
// sign of each row chosen so that its entry of largest magnitude is positive.
dade_status jacobi_eigh(int32_t D, const double* Ain, double* eigvals, double* R) {
    std::vector<double> A(Ain, Ain + (size_t)D * D), V((size_t)D * D, 0.0);
    for (int i = 0; i < D; ++i) V[(size_t)i * D + i] = 1.0;
    auto a = [&](int i, int j) -> double& { return A[(size_t)i * D + j]; };
    double scale = 0;
    for (int i = 0; i < D; ++i) scale = std::max(scale, fabs(a(i, i)));
    if (scale == 0) scale = 1;
    for (int sweep = 0; sweep < 100; ++sweep) {
        double off = 0;
        for (int p = 0; p < D; ++p)
            for (int q = p + 1; q < D; ++q) off = std::max(off, fabs(a(p, q)));
        if (off <= 1e-17 * scale) break;
        for (int p = 0; p < D - 1; ++p) {
            for (int q = p + 1; q < D; ++q) {
                double apq = a(p, q);
                if (apq == 0.0) continue;
                double app = a(p, p), aqq = a(q, q);
                if (fabs(apq) < 1e-18 * sqrt(fabs(app * aqq)) && fabs(apq) < 1e-30 * scale) {
                    a(p, q) = a(q, p) = 0;
                    continue;
                }
                double theta = (aqq - app) / (2.0 * apq);
                double t = (theta >= 0 ? 1.0 : -1.0) / (fabs(theta) + sqrt(theta * theta + 1.0));
                double c = 1.0 / sqrt(t * t + 1.0), s = t * c;
                for (int k = 0; k < D; ++k) {
                    if (k == p || k == q) continue;
                    double akp = a(k, p), akq = a(k, q);
                    double nkp = c * akp - s * akq, nkq = s * akp + c * akq;
                    a(k, p) = a(p, k) = nkp;
                    a(k, q) = a(q, k) = nkq;
                }
                a(p, p) = app - t * apq;
                a(q, q) = aqq + t * apq;
                a(p, q) = a(q, p) = 0.0;
                for (int k = 0; k < D; ++k) {
                    double vkp = V[(size_t)k * D + p], vkq = V[(size_t)k * D + q];
                    V[(size_t)k * D + p] = c * vkp - s * vkq;
                    V[(size_t)k * D + q] = s * vkp + c * vkq;
                }
            }
        }
    }
    std::vector<int> order(D);
    for (int i = 0; i < D; ++i) order[i] = i;
    std::stable_sort(order.begin(), order.end(), [&](int x, int y) { return a(x, x) > a(y, y); });
    for (int i = 0; i < D; ++i) {
        int c = order[i];
        eigvals[i] = a(c, c);
        int piv = 0;
        double best = -1;
        for (int k = 0; k < D; ++k) {
            double v = fabs(V[(size_t)k * D + c]);
            if (v > best) { best = v; piv = k; }
        }
        double sg = V[(size_t)piv * D + c] < 0 ? -1.0 : 1.0;
        for (int k = 0; k < D; ++k) R[(size_t)i * D + k] = sg * V[(size_t)k * D + c];
    }
    return DADE_OK;
}

// ---------------------------------------------------------------------------
// Logistic regression P(label 1) = sigmoid(w1 f1 + w2 f2 + b), minimising the
// mean binary cross-entropy + ridge/2 (w1^2 + w2^2) by Newton steps with step
// halving (Section V-A: a linear classifier trained with cross-entropy).
namespace {

struct LogitFit {
    double th[3];
    int iters;
    double grad;
};

void loss_grad(const std::vector<double>& f1, const std::vector<double>& f2,
               const std::vector<double>& y, const double th[3], double ridge, double* loss,
               double g[3], double H[9], bool want_h) {
    size_t n = y.size();
    double L = 0, G[3] = {0, 0, 0}, HH[9] = {0};
    for (size_t i = 0; i < n; ++i) {
        double z = th[0] * f1[i] + th[1] * f2[i] + th[2];
        // log(1 + e^z) without overflow
        double l1p = z > 0 ? z + log1p(exp(-z)) : log1p(exp(z));
        L += l1p - y[i] * z;
        double p = z >= 0 ? 1.0 / (1.0 + exp(-z)) : exp(z) / (1.0 + exp(z));
        double r = p - y[i];
        double a[3] = {f1[i], f2[i], 1.0};
        for (int u = 0; u < 3; ++u) G[u] += r * a[u];
        if (want_h) {
            double w = p * (1 - p);
            for (int u = 0; u < 3; ++u)
                for (int v = 0; v < 3; ++v) HH[u * 3 + v] += w * a[u] * a[v];
        }
    }
    double inv = 1.0 / (double)n;
    *loss = L * inv + 0.5 * ridge * (th[0] * th[0] + th[1] * th[1]);
    for (int u = 0; u < 3; ++u) g[u] = G[u] * inv + (u < 2 ? ridge * th[u] : 0.0);
    if (want_h) {
        for (int u = 0; u < 9; ++u) H[u] = HH[u] * inv;
        H[0] += ridge;
        H[4] += ridge;
    }
}

bool solve3(const double H[9], const double g[3], double x[3]) {
    double M[3][4];
    for (int i = 0; i < 3; ++i) {
        for (int j = 0; j < 3; ++j) M[i][j] = H[i * 3 + j];
        M[i][3] = g[i];
    }
    for (int c = 0; c < 3; ++c) {
        int piv = c;
        for (int r = c + 1; r < 3; ++r)
            if (fabs(M[r][c]) > fabs(M[piv][c])) piv = r;
        if (M[piv][c] == 0) return false;
        for (int j = 0; j < 4; ++j) std::swap(M[c][j], M[piv][j]);
        for (int r = 0; r < 3; ++r) {
            if (r == c) continue;
            double f = M[r][c] / M[c][c];
            for (int j = c; j < 4; ++j) M[r][j] -= f * M[c][j];
        }
    }
    for (int i = 0; i < 3; ++i) x[i] = M[i][3] / M[i][i];
    return true;
}

LogitFit fit_logistic(const std::vector<double>& f1, const std::vector<double>& f2,
                      const std::vector<double>& y) {
    const double ridge = 1e-8, tol = 1e-10;
    LogitFit out{{0, 0, 0}, 0, 0};
    double loss, g[3], H[9];
    loss_grad(f1, f2, y, out.th, ridge, &loss, g, H, true);
    auto gmax = [](const double* v) { return std::max(fabs(v[0]), std::max(fabs(v[1]), fabs(v[2]))); };
    int it = 0;
    for (; it < 50 && gmax(g) >= tol; ++it) {
        double step[3];
        if (!solve3(H, g, step)) break;
        double t = 1.0, cand[3], l2, g2[3], H2[9];
        while (true) {
            for (int u = 0; u < 3; ++u) cand[u] = out.th[u] - t * step[u];
            loss_grad(f1, f2, y, cand, ridge, &l2, g2, H2, true);
            if (l2 <= loss || gmax(g2) < gmax(g) || t < 1e-10) break;
            t *= 0.5;
        }
        memcpy(out.th, cand, sizeof cand);
        loss = l2;
        memcpy(g, g2, sizeof g2);
        memcpy(H, H2, sizeof H2);
    }
    out.iters = it;
    out.grad = gmax(g);
    return out;
}

}  // namespace

// Sequential per-step fit (Section V-A "Parameter Learning" and "Adaptive
// Adjustment", one classifier per step as in Section V-B "Incremental
// Correction"): step s uses the samples no earlier step prunes.
dade_status fit_tables(const double* partials, const double* tau, const int8_t* label, int64_t n,
                       int32_t S, double target_recall, int32_t min_label0, double* m1_out,
                       double* beta_out) {
    const double r_s = 1.0 - (1.0 - target_recall) / (double)S;
    std::vector<char> active((size_t)n, 1);
    for (int s = 1; s < S; ++s) {
        m1_out[s - 1] = 0.0;
        beta_out[s - 1] = -INFINITY;
        int64_t n0 = 0, n1 = 0;
        double tsum = 0;
        for (int64_t i = 0; i < n; ++i)
            if (active[i]) {
                (label[i] == 0 ? n0 : n1)++;
                tsum += tau[i];
            }
        if (n0 < min_label0 || n1 == 0) continue;
        double tb = tsum / (double)(n0 + n1);
        std::vector<double> f1, f2, y;
        f1.reserve(n0 + n1);
        f2.reserve(n0 + n1);
        y.reserve(n0 + n1);
        for (int64_t i = 0; i < n; ++i)
            if (active[i]) {
                f1.push_back(partials[i * (S - 1) + (s - 1)] / tb);
                f2.push_back(tau[i] / tb);
                y.push_back(label[i] ? 1.0 : 0.0);
            }
        LogitFit lf = fit_logistic(f1, f2, y);
        double w1 = lf.th[0], w2 = lf.th[1];
        if (!(w2 < 0)) continue;
        double m1 = -w1 / w2;
        std::vector<double> v;
        v.reserve(n0);
        for (int64_t i = 0; i < n; ++i)
            if (active[i] && label[i] == 0) v.push_back(tau[i] - m1 * partials[i * (S - 1) + (s - 1)]);
        std::sort(v.begin(), v.end());
        int64_t f = (int64_t)floor((1.0 - r_s) * (double)v.size());
        if (f > (int64_t)v.size() - 1) f = (int64_t)v.size() - 1;
        double bp = v[(size_t)f];
        m1_out[s - 1] = m1;
        beta_out[s - 1] = bp;
        for (int64_t i = 0; i < n; ++i)
            if (active[i] && m1 * partials[i * (S - 1) + (s - 1)] + bp > tau[i]) active[i] = 0;
    }
    return DADE_OK;
}

// ---------------------------------------------------------------------------
// OPQ-L's classifier (Section V-B "Approximate Distances": the asymmetric
// distance, the threshold and the quantisation error as features; one
// classifier): full-batch Newton logistic regression on
// (dis'/tau_bar, tau/tau_bar, e/sqrt(tau_bar)) with ridge 1e-8 on the
// weights, step halving, <= 50 iterations, max|gradient| < 1e-10; then
// m1 = -w1/w2, m3 = -w3 sqrt(tau_bar)/w2 (w2 < 0 required) and beta' the
// largest value keeping label-0 recall >= target_recall.
namespace {

bool solve_n(int n, std::vector<double> M /* n x (n + 1) */, double* x) {
    for (int c = 0; c < n; ++c) {
        int piv = c;
        for (int r = c + 1; r < n; ++r)
            if (fabs(M[r * (n + 1) + c]) > fabs(M[piv * (n + 1) + c])) piv = r;
        if (M[piv * (n + 1) + c] == 0) return false;
        for (int j = 0; j <= n; ++j) std::swap(M[c * (n + 1) + j], M[piv * (n + 1) + j]);
        for (int r = 0; r < n; ++r) {
            if (r == c) continue;
            const double f = M[r * (n + 1) + c] / M[c * (n + 1) + c];
            for (int j = c; j <= n; ++j) M[r * (n + 1) + j] -= f * M[c * (n + 1) + j];
        }
    }
    for (int i = 0; i < n; ++i) x[i] = M[i * (n + 1) + n] / M[i * (n + 1) + i];
    return true;
}

// mean cross-entropy + ridge/2 |w|^2 of sigmoid(A theta), gradient and Hessian;
// A is n x k (the last column the bias)
void loss_grad_k(const std::vector<double>& A, const std::vector<double>& y, int k, const double* th, double ridge,
                 double* loss, double* g, double* H) {
    const int64_t n = (int64_t)y.size();
    double L = 0;
    std::vector<double> G((size_t)k, 0.0), HH((size_t)k * k, 0.0);
    for (int64_t i = 0; i < n; ++i) {
        const double* a = &A[(size_t)i * k];
        double z = 0;
        for (int u = 0; u < k; ++u) z += a[u] * th[u];
        L += (z > 0 ? z + log1p(exp(-z)) : log1p(exp(z))) - y[i] * z;
        const double p = z >= 0 ? 1.0 / (1.0 + exp(-z)) : exp(z) / (1.0 + exp(z));
        const double r = p - y[i], w = p * (1 - p);
        for (int u = 0; u < k; ++u) {
            G[u] += r * a[u];
            for (int v = 0; v < k; ++v) HH[u * k + v] += w * a[u] * a[v];
        }
    }
    const double inv = 1.0 / (double)n;
    double reg = 0;
    for (int u = 0; u + 1 < k; ++u) reg += th[u] * th[u];
    *loss = L * inv + 0.5 * ridge * reg;
    for (int u = 0; u < k; ++u) g[u] = G[u] * inv + (u + 1 < k ? ridge * th[u] : 0.0);
    for (int u = 0; u < k * k; ++u) H[u] = HH[u] * inv;
    for (int u = 0; u + 1 < k; ++u) H[u * k + u] += ridge;
}

}  // namespace

dade_status fit_pq_host(const double* dis, const double* err, const double* tau, const int8_t* label, int64_t n,
                        double target_recall, int32_t min_label0, double* out3) {
    out3[0] = 0.0;
    out3[1] = 0.0;
    out3[2] = -INFINITY;
    int64_t n0 = 0, n1 = 0;
    double tsum = 0;
    for (int64_t i = 0; i < n; ++i) {
        (label[i] == 0 ? n0 : n1)++;
        tsum += tau[i];
    }
    if (n0 < min_label0 || n1 == 0) return DADE_OK;
    const double tb = tsum / (double)n, sq = sqrt(tb);
    constexpr int k = 4;
    std::vector<double> A((size_t)n * k), y((size_t)n);
    for (int64_t i = 0; i < n; ++i) {
        A[(size_t)i * k + 0] = dis[i] / tb;
        A[(size_t)i * k + 1] = tau[i] / tb;
        A[(size_t)i * k + 2] = err[i] / sq;
        A[(size_t)i * k + 3] = 1.0;
        y[(size_t)i] = label[i] ? 1.0 : 0.0;
    }
    const double ridge = 1e-8, tol = 1e-10;
    double th[k] = {0, 0, 0, 0}, loss, g[k], H[k * k];
    loss_grad_k(A, y, k, th, ridge, &loss, g, H);
    auto gmax = [](const double* v) {
        double m = 0;
        for (int u = 0; u < k; ++u) m = std::max(m, fabs(v[u]));
        return m;
    };
    for (int it = 0; it < 50 && gmax(g) >= tol; ++it) {
        std::vector<double> M((size_t)k * (k + 1));
        for (int i = 0; i < k; ++i) {
            for (int j = 0; j < k; ++j) M[i * (k + 1) + j] = H[i * k + j];
            M[i * (k + 1) + k] = g[i];
        }
        double step[k];
        if (!solve_n(k, M, step)) break;
        double t = 1.0, cand[k], l2, g2[k], H2[k * k];
        while (true) {
            for (int u = 0; u < k; ++u) cand[u] = th[u] - t * step[u];
            loss_grad_k(A, y, k, cand, ridge, &l2, g2, H2);
            if (l2 <= loss || gmax(g2) < gmax(g) || t < 1e-10) break;
            t *= 0.5;
        }
        memcpy(th, cand, sizeof cand);
        loss = l2;
        memcpy(g, g2, sizeof g2);
        memcpy(H, H2, sizeof H2);
    }
    const double w1 = th[0], w2 = th[1], w3 = th[2];
    if (!(w2 < 0)) return DADE_OK;
    const double m1 = -w1 / w2, m3 = -w3 * sq / w2;
    std::vector<double> v;
    v.reserve((size_t)n0);
    for (int64_t i = 0; i < n; ++i)
        if (label[i] == 0) v.push_back(tau[i] - m1 * dis[i] - m3 * err[i]);
    std::sort(v.begin(), v.end());
    int64_t f = (int64_t)floor((1.0 - target_recall) * (double)v.size());
    if (f > (int64_t)v.size() - 1) f = (int64_t)v.size() - 1;
    out3[0] = m1;
    out3[1] = m3;
    out3[2] = v[(size_t)f];
    return DADE_OK;
}

// ---------------------------------------------------------------------------
// Haar-random rotation (the random projection of ADS, Section III "Distance
// Estimation"): a D x D standard Gaussian matrix (Box-Muller on counter-based
// SplitMix64 uniforms of (seed, index)), its Householder QR in FP64
// (Golub and Van Loan, Sec. 5.2), and Q with column j times sign(R_jj), the
// QR factor with a positive diagonal, which is Haar distributed for a
// Gaussian input (Mezzadri 2007).  R_out's row i is Q's column i.
dade_status haar_rotation(int32_t D, uint64_t seed, double* R_out) {
    const size_t n = (size_t)D;
    std::vector<double> A(n * n);  // column-major: A[j * n + i] = A(i, j)
    const double two_pi = 6.283185307179586476925286766559;
    for (size_t k = 0; k < n * n; k += 2) {
        const uint64_t z1 = splitmix64(seed ^ splitmix64(2 * (uint64_t)k));
        const uint64_t z2 = splitmix64(seed ^ splitmix64(2 * (uint64_t)k + 1));
        const double u1 = ((double)(z1 >> 11) + 1.0) * 0x1.0p-53;  // (0, 1]
        const double u2 = (double)(z2 >> 11) * 0x1.0p-53;          // [0, 1)
        const double r = sqrt(-2.0 * log(u1));
        A[k] = r * cos(two_pi * u2);
        if (k + 1 < n * n) A[k + 1] = r * sin(two_pi * u2);
    }
    // Householder: column k is reduced by H_k = I - 2 v v^T (|v| = 1);
    // vs[k] holds v (entries k..n-1), diag[k] = R_kk
    std::vector<double> vs(n * n, 0.0), diag(n);
    for (size_t k = 0; k < n; ++k) {
        double* a = &A[k * n];
        double nrm = 0.0;
        for (size_t i = k; i < n; ++i) nrm += a[i] * a[i];
        nrm = sqrt(nrm);
        const double alpha = a[k] > 0 ? -nrm : nrm;  // avoids cancellation in v_k
        double* v = &vs[k * n];
        for (size_t i = k; i < n; ++i) v[i] = a[i];
        v[k] -= alpha;
        double vn = 0.0;
        for (size_t i = k; i < n; ++i) vn += v[i] * v[i];
        vn = sqrt(vn);
        diag[k] = alpha;
        if (vn == 0.0) continue;  // column already reduced (measure zero)
        for (size_t i = k; i < n; ++i) v[i] /= vn;
        for (size_t j = k; j < n; ++j) {
            double* c = &A[j * n];
            double dot = 0.0;
            for (size_t i = k; i < n; ++i) dot += v[i] * c[i];
            for (size_t i = k; i < n; ++i) c[i] -= 2.0 * dot * v[i];
        }
    }
    // Q = H_0 H_1 ... H_{n-1} I, built from the right: Q e_j for every j
    std::vector<double> Q(n * n, 0.0);  // column-major
    for (size_t j = 0; j < n; ++j) {
        double* q = &Q[j * n];
        q[j] = 1.0;
        for (size_t kk = n; kk-- > 0;) {
            const double* v = &vs[kk * n];
            double dot = 0.0;
            for (size_t i = kk; i < n; ++i) dot += v[i] * q[i];
            if (dot != 0.0)
                for (size_t i = kk; i < n; ++i) q[i] -= 2.0 * dot * v[i];
        }
    }
    for (size_t j = 0; j < n; ++j) {
        const double sg = diag[j] < 0 ? -1.0 : 1.0;
        for (size_t i = 0; i < n; ++i) R_out[j * n + i] = sg * Q[j * n + i];
    }
    return DADE_OK;
}

}  // namespace dade

