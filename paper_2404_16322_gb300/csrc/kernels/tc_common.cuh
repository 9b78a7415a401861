// tcgen05 helpers shared by the tensor-core kernels of the search: the
// canonical K-major operand chunk (128 rows x 8 FP32 dims = 4 KB, no
// swizzle: 8-row x 16-byte core matrices, the two K halves 128 bytes apart,
// 8-row groups 256 bytes apart), its shared-memory descriptor, the TF32
// instruction descriptor (M = 128), the MMA, tensor-memory loads and
// bounded mbarrier waits.
#pragma once
#include "scan_steps.cuh"

namespace dade {
namespace {

constexpr int kChunkF = 1024;        // floats per 4 KB operand chunk (128 rows x 8 dims)
constexpr uint32_t kTcLBO = 128;     // bytes between the two K halves of a chunk
constexpr uint32_t kTcSBO = 256;     // bytes between 8-row groups

// offset (floats) of element (row r, dim j) in a chunk (of any row count)
__device__ __forceinline__ int chunk_off(int r, int j) { return (r >> 3) * 64 + (j >> 2) * 32 + (r & 7) * 4 + (j & 3); }

// tcgen05 shared memory descriptor of a chunk: no swizzle, version 1.
__device__ __forceinline__ uint64_t tc_desc(uint32_t addr) {
    return (uint64_t)((addr >> 4) & 0x3FFFu) | ((uint64_t)((kTcLBO >> 4) & 0x3FFFu) << 16) |
           ((uint64_t)((kTcSBO >> 4) & 0x3FFFu) << 32) | ((uint64_t)1 << 46);
}
// Instruction descriptor: D FP32, A and B TF32, both K-major, M = 128, N = n.
__device__ __forceinline__ uint32_t tc_idesc(int n) {
    return (1u << 4) | (2u << 7) | (2u << 10) | ((uint32_t)(n >> 3) << 17) | ((uint32_t)(kTcRows >> 4) << 24);
}
__device__ __forceinline__ void tc_mma(uint32_t tmem, uint64_t a, uint64_t b, uint32_t idesc, uint32_t acc) {
    asm volatile(
        "{\n .reg .pred p;\n setp.ne.b32 p, %4, 0;\n"
        " tcgen05.mma.cta_group::1.kind::tf32 [%0], %1, %2, %3, p;\n}\n" ::"r"(tmem),
        "l"(a), "l"(b), "r"(idesc), "r"(acc)
        : "memory");
}
__device__ __forceinline__ float tf32_rna(float x) {
    uint32_t r;
    asm("cvt.rna.tf32.f32 %0, %1;" : "=r"(r) : "f"(x));
    return __uint_as_float(r);
}
__device__ __forceinline__ void tc_fence_after() { asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory"); }
__device__ __forceinline__ void tc_fence_before() { asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory"); }

// 32 or 16 accumulator columns of this warp's 32 lanes (one row per lane).
__device__ __forceinline__ void tmem_ld32(uint32_t taddr, uint32_t (&v)[32]) {
    asm volatile(
        "tcgen05.ld.sync.aligned.32x32b.x32.b32 {%0, %1, %2, %3, %4, %5, %6, %7, %8, %9, %10, %11, %12, %13, "
        "%14, %15, %16, %17, %18, %19, %20, %21, %22, %23, %24, %25, %26, %27, %28, %29, %30, %31}, [%32];"
        : "=r"(v[0]), "=r"(v[1]), "=r"(v[2]), "=r"(v[3]), "=r"(v[4]), "=r"(v[5]), "=r"(v[6]), "=r"(v[7]),
          "=r"(v[8]), "=r"(v[9]), "=r"(v[10]), "=r"(v[11]), "=r"(v[12]), "=r"(v[13]), "=r"(v[14]), "=r"(v[15]),
          "=r"(v[16]), "=r"(v[17]), "=r"(v[18]), "=r"(v[19]), "=r"(v[20]), "=r"(v[21]), "=r"(v[22]), "=r"(v[23]),
          "=r"(v[24]), "=r"(v[25]), "=r"(v[26]), "=r"(v[27]), "=r"(v[28]), "=r"(v[29]), "=r"(v[30]), "=r"(v[31])
        : "r"(taddr));
}
__device__ __forceinline__ void tmem_ld16(uint32_t taddr, uint32_t (&v)[32]) {
    asm volatile(
        "tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0, %1, %2, %3, %4, %5, %6, %7, %8, %9, %10, %11, %12, %13, "
        "%14, %15}, [%16];"
        : "=r"(v[0]), "=r"(v[1]), "=r"(v[2]), "=r"(v[3]), "=r"(v[4]), "=r"(v[5]), "=r"(v[6]), "=r"(v[7]),
          "=r"(v[8]), "=r"(v[9]), "=r"(v[10]), "=r"(v[11]), "=r"(v[12]), "=r"(v[13]), "=r"(v[14]), "=r"(v[15])
        : "r"(taddr));
#pragma unroll
    for (int j = 16; j < 32; ++j) v[j] = 0u;
}

// A bounded wait on an mbarrier, taken by lane 0 and shared with the warp
// (so that the warp-collective tensor-memory loads stay converged).
__device__ __forceinline__ bool warp_wait(uint64_t* bar, uint32_t parity, int32_t* status, int lane) {
    int ok = 1;
    if (lane == 0) ok = mbar_wait(bar, parity, status) ? 1 : 0;
    return __shfl_sync(0xffffffffu, ok, 0) != 0;
}

// Bounded wait that polls (mbarrier.test_wait, the thread is never
// suspended): for waits expected to end within a few hundred cycles.
__device__ __forceinline__ bool mbar_test(uint64_t* bar, uint32_t parity) {
    uint32_t ok;
    asm volatile(
        "{\n .reg .pred p;\n mbarrier.test_wait.parity.shared::cta.b64 p, [%1], %2;\n selp.u32 %0, 1, 0, p;\n}"
        : "=r"(ok)
        : "r"(smem_u32(bar)), "r"(parity)
        : "memory");
    return ok != 0;
}
__device__ __forceinline__ bool mbar_wait_spin(uint64_t* bar, uint32_t parity, int32_t* status) {
    if (mbar_test(bar, parity)) return true;
    const uint64_t t0 = globaltimer();
    for (uint32_t n = 0;; ++n) {
        if (mbar_test(bar, parity)) return true;
        if ((n & 255u) == 255u && globaltimer() - t0 > 2000000000ull) {
            if (status) atomicCAS(status, 0, (int)DADE_ETIMEOUT);
            return false;
        }
    }
}
__device__ __forceinline__ bool warp_wait_spin(uint64_t* bar, uint32_t parity, int32_t* status, int lane) {
    int ok = 1;
    if (lane == 0) ok = mbar_wait_spin(bar, parity, status) ? 1 : 0;
    return __shfl_sync(0xffffffffu, ok, 0) != 0;
}
__device__ __forceinline__ void mbar_arrive(uint64_t* bar) {
    asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(smem_u32(bar)) : "memory");
}

}  // namespace
}  // namespace dade
