// Dense contractions of the path: the query / database rotation
// x' = R (x - mean) (Section IV-A: x_D = R x, after centring) and the squared
// distance of rotated vectors to every IVF centroid (Section II-A), the
// latter either stored (query probing) or reduced to an argmin (k-means
// assignment).  FP32 FMA accumulation in k order, 64 x 64 output tile per CTA,
// 4 x 4 outputs per thread.
#include "../dade_internal.h"

namespace dade {
namespace {

constexpr int TM = 64, TN = 64, TK = 16, NT = 256;

template <int OP, bool ARGMIN>
__global__ void __launch_bounds__(NT) gemm_kernel(const float* __restrict__ A, int64_t lda,
                                                  const float* __restrict__ sub,
                                                  const float* __restrict__ Bm, int64_t ldb,
                                                  float* __restrict__ C, int64_t ldc,
                                                  unsigned long long* __restrict__ amin,
                                                  int64_t M, int64_t N, int Kd) {
    __shared__ float As[TK][TM + 4];
    __shared__ float Bs[TK][TN + 4];
    const int tid = threadIdx.x;
    const int64_t m0 = (int64_t)blockIdx.x * TM;
    const int64_t n0 = (int64_t)blockIdx.y * TN;
    const int tr = tid >> 4, tc = tid & 15;
    float acc[4][4];
#pragma unroll
    for (int i = 0; i < 4; ++i)
#pragma unroll
        for (int j = 0; j < 4; ++j) acc[i][j] = 0.f;

    for (int k0 = 0; k0 < Kd; k0 += TK) {
#pragma unroll
        for (int u = 0; u < 4; ++u) {
            int e = tid + u * NT;
            int r = e / TK, c = e % TK;
            int64_t gm = m0 + r, gn = n0 + r;
            int gk = k0 + c;
            float a = 0.f, b = 0.f;
            if (gm < M && gk < Kd) {
                a = A[gm * lda + gk];
                if (sub) a -= sub[gk];
            }
            if (gn < N && gk < Kd) b = Bm[gn * ldb + gk];
            As[c][r] = a;
            Bs[c][r] = b;
        }
        __syncthreads();
#pragma unroll
        for (int kk = 0; kk < TK; ++kk) {
            float a[4], b[4];
#pragma unroll
            for (int i = 0; i < 4; ++i) a[i] = As[kk][tr + 16 * i];
#pragma unroll
            for (int j = 0; j < 4; ++j) b[j] = Bs[kk][tc + 16 * j];
#pragma unroll
            for (int i = 0; i < 4; ++i)
#pragma unroll
                for (int j = 0; j < 4; ++j) {
                    if (OP == GEMM_DOT) {
                        acc[i][j] = fmaf(a[i], b[j], acc[i][j]);
                    } else {
                        float t = a[i] - b[j];
                        acc[i][j] = fmaf(t, t, acc[i][j]);
                    }
                }
        }
        __syncthreads();
    }

    if (!ARGMIN) {
#pragma unroll
        for (int i = 0; i < 4; ++i) {
            int64_t gm = m0 + tr + 16 * i;
            if (gm >= M) continue;
#pragma unroll
            for (int j = 0; j < 4; ++j) {
                int64_t gn = n0 + tc + 16 * j;
                if (gn < N) C[gm * ldc + gn] = acc[i][j];
            }
        }
    } else {
#pragma unroll
        for (int i = 0; i < 4; ++i) {
            unsigned long long best = ~0ull;
#pragma unroll
            for (int j = 0; j < 4; ++j) {
                int64_t gn = n0 + tc + 16 * j;
                if (gn < N) {
                    unsigned long long key =
                        ((unsigned long long)__float_as_uint(acc[i][j]) << 32) | (unsigned long long)gn;
                    best = key < best ? key : best;
                }
            }
            // the 16 threads of a row are lanes [0,16) or [16,32) of the warp
#pragma unroll
            for (int off = 8; off >= 1; off >>= 1) {
                unsigned long long o = __shfl_xor_sync(0xffffffffu, best, off);
                best = o < best ? o : best;
            }
            int64_t gm = m0 + tr + 16 * i;
            if (tc == 0 && gm < M && best != ~0ull) atomicMin(&amin[gm], best);
        }
    }
}

}  // namespace

cudaError_t launch_gemm_store(int op, const float* A, int64_t lda, const float* sub,
                              const float* B, int64_t ldb, float* C, int64_t ldc, int64_t M,
                              int64_t N, int Kd, cudaStream_t st) {
    if (M <= 0 || N <= 0) return cudaSuccess;
    dim3 grid((unsigned)ceil_div(M, TM), (unsigned)ceil_div(N, TN));
    if (op == GEMM_DOT)
        gemm_kernel<GEMM_DOT, false><<<grid, NT, 0, st>>>(A, lda, sub, B, ldb, C, ldc, nullptr, M, N, Kd);
    else
        gemm_kernel<GEMM_L2, false><<<grid, NT, 0, st>>>(A, lda, nullptr, B, ldb, C, ldc, nullptr, M, N, Kd);
    return cudaGetLastError();
}

cudaError_t launch_gemm_argmin(const float* A, int64_t lda, const float* B, int64_t ldb,
                               unsigned long long* out, int64_t M, int64_t N, int Kd,
                               cudaStream_t st) {
    if (M <= 0 || N <= 0) return cudaSuccess;
    dim3 grid((unsigned)ceil_div(M, TM), (unsigned)ceil_div(N, TN));
    gemm_kernel<GEMM_L2, true><<<grid, NT, 0, st>>>(A, lda, nullptr, B, ldb, nullptr, 0, out, M, N, Kd);
    return cudaGetLastError();
}

}  // namespace dade
