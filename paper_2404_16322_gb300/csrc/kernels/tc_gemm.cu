// Tensor-core (tcgen05) GEMMs of the path: the query rotation
// q' = R (q - mean) (Section IV-A, x_D = R x after centring) and the squared
// distance of rotated queries to every IVF centroid (Section II-A),
// ||q'||^2 + ||c||^2 - 2 q'.c, clamped at 0.
//
// C[M x N] = A[M x K] . B[N x K]^T with both operands K-major (rows of A and
// of B are contiguous in K).  One CTA of 128 threads computes a 128 x 128 tile:
//  - K is consumed in blocks of 32; the threads load a block of A and B and
//    split every value into TF32 parts (round to nearest): A into three,
//    a = hi + mid + lo exactly (11 + 11 + the last <= 3 bits), B into two,
//    b ~ hi + mid; the parts go to shared memory in the canonical K-major
//    layout without swizzle: 8-row x 16-byte core matrices, core matrices
//    adjacent in K 128 bytes apart (LBO), 8-row groups 1024 bytes apart (SBO);
//  - one thread issues, per K = 8 step, four tcgen05.mma kind::tf32
//    (Ah.Bh + Ah.Bm + Am.Bh + Al.Bh) into an FP32 accumulator of 128 lanes
//    x 128 columns in tensor memory -- every product of B's parts with A is
//    kept except terms below 2^-22 of the result, and a product by an exact
//    TF32 b (such as a permutation matrix) is exact -- then tcgen05.commit
//    to an mbarrier that the threads wait on (bounded);
//  - the accumulator covers one K block: the 4 warps read their 32 lanes
//    (rows) with tcgen05.ld.32x32b after every block and add them to FP32
//    registers, so the tensor core's own accumulation rounding stays that
//    of 32-term sums (the error of a long K would otherwise grow with K);
//    the epilogue then works from those registers.
#include "../dade_internal.h"

namespace dade {
namespace {

constexpr int TM = 128, TN = 128, TKB = 32;          // tile and K block (TF32 elements)
constexpr int TILE_BYTES = TM * TKB * 4;             // 16 KB per operand part
constexpr uint32_t LBO = 128, SBO = 1024;            // byte strides of core matrices

__device__ __forceinline__ uint32_t smem_u32(const void* p) {
    return (uint32_t)__cvta_generic_to_shared(p);
}

// Byte offset of element (r, j) of a 128 x 32 K-major tile.
__device__ __forceinline__ uint32_t tile_off(int r, int j) {
    return (uint32_t)((r >> 3) * SBO + (j >> 2) * LBO + (r & 7) * 16 + (j & 3) * 4);
}

// tcgen05 shared memory descriptor: start >> 4 in [0,14), LBO >> 4 in
// [16,30), SBO >> 4 in [32,46), version 1 in [46,48), no swizzle.
__device__ __forceinline__ uint64_t smem_desc(uint32_t addr) {
    return (uint64_t)((addr >> 4) & 0x3FFFu) | ((uint64_t)((LBO >> 4) & 0x3FFFu) << 16) |
           ((uint64_t)((SBO >> 4) & 0x3FFFu) << 32) | ((uint64_t)1 << 46);
}

// Instruction descriptor: D FP32, A and B TF32, both K-major, N = 128, M = 128.
constexpr uint32_t kIdesc = (1u << 4) | (2u << 7) | (2u << 10) | ((uint32_t)(TN >> 3) << 17) |
                            ((uint32_t)(TM >> 4) << 24);

__device__ __forceinline__ float to_tf32(float x) {
    uint32_t r;
    asm("cvt.rna.tf32.f32 %0, %1;" : "=r"(r) : "f"(x));
    return __uint_as_float(r);
}

__device__ __forceinline__ void mma_tf32(uint32_t tmem, uint64_t a, uint64_t b, uint32_t acc) {
    asm volatile(
        "{\n .reg .pred p;\n setp.ne.b32 p, %4, 0;\n"
        " tcgen05.mma.cta_group::1.kind::tf32 [%0], %1, %2, %3, p;\n}\n" ::"r"(tmem),
        "l"(a), "l"(b), "r"(kIdesc), "r"(acc)
        : "memory");
}

// A waiting thread sleeps until the phase completes or this many ns pass
// (then it re-checks), rather than spinning on the barrier.
constexpr uint32_t kWaitHintNs = 200000;

__device__ __forceinline__ bool bar_try_wait(uint64_t* bar, uint32_t parity) {
    uint32_t ok;
    asm volatile(
        "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2, %3;\n selp.u32 %0, 1, 0, p;\n}"
        : "=r"(ok)
        : "r"(smem_u32(bar)), "r"(parity), "r"(kWaitHintNs)
        : "memory");
    return ok != 0;
}

__device__ __forceinline__ bool bar_wait(uint64_t* bar, uint32_t parity, int32_t* status) {
    if (bar_try_wait(bar, parity)) return true;
    uint64_t t0;
    asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t0));
    for (;;) {
        if (bar_try_wait(bar, parity)) return true;
        uint64_t t;
        asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
        if (t - t0 > 2000000000ull) {
            if (status) atomicCAS(status, 0, (int)DADE_ETIMEOUT);
            return false;
        }
    }
}

enum Epi { EPI_STORE = 0, EPI_L2 = 1 };

// Loads the 128 x 32 K-block at (row0, k0) of a row-major operand and stores
// its TF32 parts: hi, mid and (when lo != nullptr) lo = the exact rest.  VEC: float4 loads (rows 16-byte aligned, K a
// multiple of 4); element f of the 1024 float4s of the block maps to row
// (f / 64) * 8 + f % 8 and float4 column (f / 8) % 8, so the 8 lanes of a
// quarter warp store to 8 different rows of one core-matrix column (distinct
// banks) and each row is read in 64-byte runs.
template <bool VEC>
__device__ __forceinline__ void load_split(const float* __restrict__ X, int64_t ld, const float* __restrict__ sub,
                                           int64_t row0, int64_t nrows, int k0, int Kd,
                                           unsigned char* hi, unsigned char* mid, unsigned char* lo, int tid) {
    if (VEC) {
#pragma unroll
        for (int i = 0; i < 8; ++i) {
            const int f = tid + 128 * i;
            const int r = (f >> 6) * 8 + (f & 7), c4 = (f >> 3) & 7;
            const int64_t gr = row0 + r;
            const int gk = k0 + c4 * 4;
            float4 v = make_float4(0.f, 0.f, 0.f, 0.f);
            if (gr < nrows && gk < Kd) {
                v = __ldg(reinterpret_cast<const float4*>(X + gr * ld + gk));
                if (sub) {
                    const float4 m = __ldg(reinterpret_cast<const float4*>(sub + gk));
                    v.x -= m.x; v.y -= m.y; v.z -= m.z; v.w -= m.w;
                }
            }
            float4 h, m;
            h.x = to_tf32(v.x); h.y = to_tf32(v.y); h.z = to_tf32(v.z); h.w = to_tf32(v.w);
            m.x = to_tf32(v.x - h.x); m.y = to_tf32(v.y - h.y); m.z = to_tf32(v.z - h.z); m.w = to_tf32(v.w - h.w);
            const uint32_t o = tile_off(r, c4 * 4);
            *reinterpret_cast<float4*>(hi + o) = h;
            *reinterpret_cast<float4*>(mid + o) = m;
            if (lo) {
                float4 l;
                l.x = (v.x - h.x) - m.x; l.y = (v.y - h.y) - m.y; l.z = (v.z - h.z) - m.z; l.w = (v.w - h.w) - m.w;
                *reinterpret_cast<float4*>(lo + o) = l;
            }
        }
    } else {
        for (int e = tid; e < TM * TKB; e += 128) {
            const int r = e / TKB, j = e % TKB;
            const int64_t gr = row0 + r;
            const int gk = k0 + j;
            float v = 0.f;
            if (gr < nrows && gk < Kd) {
                v = X[gr * ld + gk];
                if (sub) v -= sub[gk];
            }
            const float h = to_tf32(v);
            const float m = to_tf32(v - h);
            const uint32_t o = tile_off(r, j);
            *reinterpret_cast<float*>(hi + o) = h;
            *reinterpret_cast<float*>(mid + o) = m;
            if (lo) *reinterpret_cast<float*>(lo + o) = (v - h) - m;
        }
    }
}

// A: M x Kd (lda), optionally minus sub[k]; B: N x Kd (ldb).
// EPI_STORE: C = dot.  EPI_L2: C = max(0, an[m] + bn[n] - 2 dot).
template <int EPI, bool VA, bool VB>
__global__ void __launch_bounds__(128, 1) tc_gemm_kernel(const float* __restrict__ A, int64_t lda,
                                                         const float* __restrict__ sub,
                                                         const float* __restrict__ Bm, int64_t ldb,
                                                         const float* __restrict__ an,
                                                         const float* __restrict__ bn,
                                                         float* __restrict__ C, int64_t ldc, int64_t M,
                                                         int64_t N, int Kd, int32_t* status) {
    extern __shared__ __align__(1024) unsigned char tsm[];
    __shared__ __align__(8) uint64_t bar;
    __shared__ uint32_t s_taddr;
    __shared__ int s_ok;
    unsigned char* base = reinterpret_cast<unsigned char*>((reinterpret_cast<uintptr_t>(tsm) + 1023) & ~uintptr_t(1023));
    unsigned char* a_hi = base;
    unsigned char* a_md = base + TILE_BYTES;
    unsigned char* a_lo = base + 2 * TILE_BYTES;
    unsigned char* b_hi = base + 3 * TILE_BYTES;
    unsigned char* b_md = base + 4 * TILE_BYTES;
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    const int64_t m0 = (int64_t)blockIdx.x * TM, n0 = (int64_t)blockIdx.y * TN;

    if (warp == 0) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(&s_taddr)),
                     "r"(TN)
                     : "memory");
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
    }
    if (tid == 0) {
        asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(&bar)), "r"(1) : "memory");
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
        s_ok = 1;
    }
    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
    __syncthreads();
    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
    const uint32_t tmem = s_taddr;

    uint32_t phase = 0;
    const int nkb = (Kd + TKB - 1) / TKB;
    // the accumulator restarts at every K block and the block results are
    // summed here in FP32 (round to nearest): the tensor core's FP32
    // accumulation then spans 32 products, not all of K
    float acc[TN];
#pragma unroll
    for (int j = 0; j < TN; ++j) acc[j] = 0.f;
    const uint32_t trow = tmem + ((uint32_t)(warp * 32) << 16);
    for (int kb = 0; kb < nkb; ++kb) {
        const int k0 = kb * TKB;
        load_split<VA>(A, lda, sub, m0, M, k0, Kd, a_hi, a_md, a_lo, tid);
        load_split<VB>(Bm, ldb, nullptr, n0, N, k0, Kd, b_hi, b_md, nullptr, tid);
        // make the generic-proxy stores visible to the tensor core (and
        // order the previous block's tensor-memory reads before its MMAs)
        asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
        asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
        __syncthreads();
        if (tid == 0) {
            asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
            const uint32_t ah = smem_u32(a_hi), am = smem_u32(a_md), al = smem_u32(a_lo);
            const uint32_t bh = smem_u32(b_hi), bm = smem_u32(b_md);
#pragma unroll
            for (int s = 0; s < TKB / 8; ++s) {
                const uint32_t step = (uint32_t)s * 2 * LBO;  // K = 8 = two core matrices
                const uint32_t first = s == 0 ? 0u : 1u;
                mma_tf32(tmem, smem_desc(ah + step), smem_desc(bh + step), first);
                mma_tf32(tmem, smem_desc(ah + step), smem_desc(bm + step), 1u);
                mma_tf32(tmem, smem_desc(am + step), smem_desc(bh + step), 1u);
                mma_tf32(tmem, smem_desc(al + step), smem_desc(bh + step), 1u);
            }
            asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(
                             smem_u32(&bar))
                         : "memory");
        }
        const bool got = bar_wait(&bar, phase, status);
        phase ^= 1u;
        if (!got) s_ok = 0;
        asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
        __syncthreads();
        if (!s_ok) break;
        // this block's products: warp w reads its 32 accumulator lanes (rows)
#pragma unroll
        for (int c0 = 0; c0 < TN; c0 += 16) {
            uint32_t v[16];
            asm volatile(
                "tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0, %1, %2, %3, %4, %5, %6, %7, %8, %9, %10, %11, "
                "%12, %13, %14, %15}, [%16];"
                : "=r"(v[0]), "=r"(v[1]), "=r"(v[2]), "=r"(v[3]), "=r"(v[4]), "=r"(v[5]), "=r"(v[6]),
                  "=r"(v[7]), "=r"(v[8]), "=r"(v[9]), "=r"(v[10]), "=r"(v[11]), "=r"(v[12]), "=r"(v[13]),
                  "=r"(v[14]), "=r"(v[15])
                : "r"(trow + (uint32_t)c0));
            asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
#pragma unroll
            for (int j = 0; j < 16; ++j) acc[c0 + j] += __uint_as_float(v[j]);
        }
    }

    if (s_ok) {
        // epilogue: warp w owns accumulator lanes (rows) [32w, 32w + 32); a
        // 32 x 16 block goes through shared memory (the operand area, free
        // now) so that global stores run along rows
        float* stage = reinterpret_cast<float*>(base) + warp * 32 * 17;
        const int r = warp * 32 + lane;
        const int64_t gm = m0 + r;
        const float arow = (EPI == EPI_L2 && gm < M) ? an[gm] : 0.f;
#pragma unroll
        for (int c0 = 0; c0 < TN; c0 += 16) {
#pragma unroll
            for (int j = 0; j < 16; ++j) {
                const float dot = acc[c0 + j];
                float out;
                if (EPI == EPI_L2) out = fmaxf(0.f, arow + (n0 + c0 + j < N ? bn[n0 + c0 + j] : 0.f) - 2.f * dot);
                else out = dot;
                stage[lane * 17 + j] = out;
            }
            __syncwarp();
#pragma unroll
            for (int i = 0; i < 16; ++i) {
                const int e = i * 32 + lane, rr = e >> 4, cc = e & 15;
                const int64_t grow = m0 + warp * 32 + rr, gcol = n0 + c0 + cc;
                if (grow < M && gcol < N) C[grow * ldc + gcol] = stage[rr * 17 + cc];
            }
            __syncwarp();
        }
    }
    if (!s_ok) {
        // a wait gave up: give the MMAs in flight one more bounded wait
        // before the accumulator's tensor memory is released
        bar_wait(&bar, phase ^ 1u, nullptr);
    }
    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
    __syncthreads();
    if (warp == 0) {
        asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
        asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(TN) : "memory");
    }
}

// ||row||^2 of the first n columns of each of M rows (FP32): one warp per
// row, lane l summing columns l, l + 32, ... in order, then a butterfly sum
// (a fixed order, so the same row always gets the same bits).
__global__ void row_norms_kernel(const float* __restrict__ X, int64_t ld, int64_t M, int n,
                                 float* __restrict__ out) {
    const int64_t r = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const int lane = threadIdx.x & 31;
    if (r >= M) return;
    float s = 0.f;
    for (int j = lane; j < n; j += 32) {
        const float v = X[r * ld + j];
        s = fmaf(v, v, s);
    }
#pragma unroll
    for (int o = 16; o; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
    if (lane == 0) out[r] = s;
}

constexpr int kSmem = 5 * TILE_BYTES + 1024;  // five operand parts + alignment slack

template <int EPI, bool VA, bool VB>
cudaError_t launch_v(const float* A, int64_t lda, const float* sub, const float* B, int64_t ldb,
                     const float* an, const float* bn, float* C, int64_t ldc, int64_t M, int64_t N, int Kd,
                     int32_t* status, cudaStream_t st) {
    static bool configured = false;
    auto kern = tc_gemm_kernel<EPI, VA, VB>;
    if (!configured) {
        cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, kSmem);
        if (e != cudaSuccess) return e;
        configured = true;
    }
    dim3 grid((unsigned)ceil_div(M, TM), (unsigned)ceil_div(N, TN));
    kern<<<grid, 128, kSmem, st>>>(A, lda, sub, B, ldb, an, bn, C, ldc, M, N, Kd, status);
    return cudaGetLastError();
}

// float4 loads need 16-byte aligned rows and K (and the subtrahend) in
// whole float4s
bool vec_ok(const float* X, int64_t ld, int Kd) {
    return (reinterpret_cast<uintptr_t>(X) & 15) == 0 && ld % 4 == 0 && Kd % 4 == 0;
}

template <int EPI>
cudaError_t launch_t(const float* A, int64_t lda, const float* sub, const float* B, int64_t ldb,
                     const float* an, const float* bn, float* C, int64_t ldc, int64_t M, int64_t N, int Kd,
                     int32_t* status, cudaStream_t st) {
    if (M <= 0 || N <= 0) return cudaSuccess;
    const bool va = vec_ok(A, lda, Kd) && (!sub || (reinterpret_cast<uintptr_t>(sub) & 15) == 0);
    const bool vb = vec_ok(B, ldb, Kd);
    if (va && vb) return launch_v<EPI, true, true>(A, lda, sub, B, ldb, an, bn, C, ldc, M, N, Kd, status, st);
    if (vb) return launch_v<EPI, false, true>(A, lda, sub, B, ldb, an, bn, C, ldc, M, N, Kd, status, st);
    return launch_v<EPI, false, false>(A, lda, sub, B, ldb, an, bn, C, ldc, M, N, Kd, status, st);
}

}  // namespace

cudaError_t launch_tc_dot(const float* A, int64_t lda, const float* sub, const float* B, int64_t ldb, float* C,
                          int64_t ldc, int64_t M, int64_t N, int Kd, int32_t* status, cudaStream_t st) {
    return launch_t<EPI_STORE>(A, lda, sub, B, ldb, nullptr, nullptr, C, ldc, M, N, Kd, status, st);
}

cudaError_t launch_tc_l2(const float* A, int64_t lda, const float* an, const float* B, int64_t ldb,
                         const float* bn, float* C, int64_t ldc, int64_t M, int64_t N, int Kd, int32_t* status,
                         cudaStream_t st) {
    return launch_t<EPI_L2>(A, lda, nullptr, B, ldb, an, bn, C, ldc, M, N, Kd, status, st);
}

cudaError_t launch_row_norms(const float* X, int64_t ld, int64_t M, int n, float* out, cudaStream_t st) {
    if (M <= 0) return cudaSuccess;
    row_norms_kernel<<<(unsigned)ceil_div(M * 32, 256), 256, 0, st>>>(X, ld, M, n, out);
    return cudaGetLastError();
}

}  // namespace dade
