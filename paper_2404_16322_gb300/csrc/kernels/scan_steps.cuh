// The estimate-and-prune wave scan as a template over slab type, step width
// and test, included by the translation units that instantiate it (scan.cu:
// learned tables and the full scan; scan_res.cu: the Gaussian-bound test of
// Section IV-C).
//
// Method (arXiv 2404.16322): a candidate's distance is accumulated Delta_d
// rotated dimensions at a time (the loop of Algorithm 2); after each step a
// test prunes it against tau, the result queue's largest entry (Section I);
// survivors get the exact distance from the original vector.
//
// Work unit = (bucket l, tile of up to kT candidates, group of up to kG
// queries probing l in this wave).  The unit's Delta_d slab of the tile is
// one bulk copy per 8-dim block (cp.async.bulk into shared memory, double
// buffered, completion on an mbarrier) and is shared by every query of the
// group.  Step 0 is dense (thread c scores candidate c against every query);
// the surviving (query, candidate) pairs then live in per-warp lists that
// are compacted with warp ballots after every later test.
//
// Distance arithmetic (identical in every path, so a pair's distance does
// not depend on which path computed it): per 8-dim block b, the even and the
// odd dims each form an FMA chain of (q_j - x_j)^2 in dim order (packed FP32
// pairs), s_b = even + odd; the distance adds s_b in block order.
#pragma once

#include <climits>

#include <cuda_bf16.h>
#include <cuda_fp8.h>

#include "scan.cuh"

namespace dade {
namespace {


constexpr int kWarps = kScanThreads / 32;

// ------------------------------------------------------------------ PTX
__device__ __forceinline__ uint32_t smem_u32(const void* p) {
    return (uint32_t)__cvta_generic_to_shared(p);
}
__device__ __forceinline__ void mbar_init(uint64_t* bar, uint32_t count) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(bar)), "r"(count) : "memory");
}
__device__ __forceinline__ void fence_mbar_init() {
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
}
__device__ __forceinline__ void fence_proxy_async() {
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
}
__device__ __forceinline__ void mbar_expect_tx(uint64_t* bar, uint32_t bytes) {
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_u32(bar)),
                 "r"(bytes)
                 : "memory");
}
__device__ __forceinline__ void bulk_g2s(void* dst, const void* src, uint32_t bytes, uint64_t* bar) {
    asm volatile(
        "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(
            smem_u32(dst)),
        "l"(src), "r"(bytes), "r"(smem_u32(bar))
        : "memory");
}
// A waiting thread sleeps until the phase completes or this many ns pass
// (then it re-checks), rather than spinning on the barrier.
constexpr uint32_t kWaitHintNs = 200000;
__device__ __forceinline__ bool mbar_try_wait(uint64_t* bar, uint32_t parity) {
    uint32_t ok;
    asm volatile(
        "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2, %3;\n selp.u32 %0, 1, 0, p;\n}"
        : "=r"(ok)
        : "r"(smem_u32(bar)), "r"(parity), "r"(kWaitHintNs)
        : "memory");
    return ok != 0;
}
__device__ __forceinline__ uint64_t globaltimer() {
    uint64_t t;
    asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
    return t;
}
// Bounded wait: gives up after ~2 s, records DADE_ETIMEOUT and returns false.
__device__ __forceinline__ bool mbar_wait(uint64_t* bar, uint32_t parity, int32_t* status) {
    if (mbar_try_wait(bar, parity)) return true;
    uint64_t t0 = globaltimer();
    while (!mbar_try_wait(bar, parity)) {
        if (globaltimer() - t0 > 2000000000ull) {
            if (status) atomicCAS(status, 0, (int)DADE_ETIMEOUT);
            return false;
        }
    }
    return true;
}
__device__ __forceinline__ unsigned lanemask_lt() {
    unsigned m;
    asm("mov.u32 %0, %%lanemask_lt;" : "=r"(m));
    return m;
}

// ------------------------------------------------------------ element loads
template <int DT> struct Elem;
template <> struct Elem<DADE_SLAB_F32> { using T = float; };
template <> struct Elem<DADE_SLAB_BF16> { using T = __nv_bfloat16; };
template <> struct Elem<DADE_SLAB_FP8E4M3> { using T = __nv_fp8_storage_t; };

// 8 consecutive elements of one block as FP32 (FP8: times the per-dim scale).
__device__ __forceinline__ void load8(const float* p, const float*, float (&x)[8]) {
    float4 a = reinterpret_cast<const float4*>(p)[0];
    float4 b = reinterpret_cast<const float4*>(p)[1];
    x[0] = a.x; x[1] = a.y; x[2] = a.z; x[3] = a.w;
    x[4] = b.x; x[5] = b.y; x[6] = b.z; x[7] = b.w;
}
__device__ __forceinline__ void load8(const __nv_bfloat16* p, const float*, float (&x)[8]) {
    uint4 u = *reinterpret_cast<const uint4*>(p);
    const uint32_t w[4] = {u.x, u.y, u.z, u.w};
#pragma unroll
    for (int i = 0; i < 4; ++i) {
        x[2 * i] = __uint_as_float(w[i] << 16);
        x[2 * i + 1] = __uint_as_float(w[i] & 0xffff0000u);
    }
}
__device__ __forceinline__ void load8(const __nv_fp8_storage_t* p, const float* scale8, float (&x)[8]) {
    uint2 u = *reinterpret_cast<const uint2*>(p);
    const uint32_t w[2] = {u.x, u.y};
#pragma unroll
    for (int i = 0; i < 2; ++i) {
#pragma unroll
        for (int h = 0; h < 2; ++h) {
            __nv_fp8x2_storage_t pair = (__nv_fp8x2_storage_t)((w[i] >> (16 * h)) & 0xffffu);
            __half2_raw hr = __nv_cvt_fp8x2_to_halfraw2(pair, __NV_E4M3);
            float2 f = __half22float2(*reinterpret_cast<__half2*>(&hr));
            int j = 4 * i + 2 * h;
            x[j] = f.x * scale8[j];
            x[j + 1] = f.y * scale8[j + 1];
        }
    }
}

__device__ __forceinline__ unsigned long long pack2(float a, float b) {
    unsigned long long r;
    asm("mov.b64 %0, {%1, %2};" : "=l"(r) : "f"(a), "f"(b));
    return r;
}

// s_b = sum over the block's 8 dims of (q - x)^2 with packed FP32 pairs:
// the even and the odd dims each form an FMA chain in dim order (the first
// term a product), and s_b = even + odd.  Every path uses this function, so
// a pair's distance does not depend on the path that computed it.
__device__ __forceinline__ float block_sq(const float (&q)[8], const float (&x)[8]) {
    unsigned long long acc, t;
    asm("sub.rn.f32x2 %0, %1, %2;" : "=l"(t) : "l"(pack2(q[0], q[1])), "l"(pack2(x[0], x[1])));
    asm("mul.rn.f32x2 %0, %1, %1;" : "=l"(acc) : "l"(t));
#pragma unroll
    for (int j = 2; j < 8; j += 2) {
        asm("sub.rn.f32x2 %0, %1, %2;" : "=l"(t) : "l"(pack2(q[j], q[j + 1])), "l"(pack2(x[j], x[j + 1])));
        asm("fma.rn.f32x2 %0, %1, %1, %2;" : "=l"(acc) : "l"(t), "l"(acc));
    }
    float e, o;
    asm("mov.b64 {%0, %1}, %2;" : "=f"(e), "=f"(o) : "l"(acc));
    return e + o;
}

// 8 FP32 values of one block from the shared-memory slab buffer.  A block
// is 32 bytes; lanes whose bit 2 is set read its second half first, so each
// 16-byte load of a quarter warp touches all 32 banks once.
__device__ __forceinline__ void load8_staged(const float* p, const float*, float (&x)[8]) {
    const float4* p4 = reinterpret_cast<const float4*>(p);
    const int sw = (threadIdx.x >> 2) & 1;
    float4 a = p4[sw], b = p4[sw ^ 1];
    if (sw) {
        const float4 t = a;
        a = b;
        b = t;
    }
    x[0] = a.x; x[1] = a.y; x[2] = a.z; x[3] = a.w;
    x[4] = b.x; x[5] = b.y; x[6] = b.z; x[7] = b.w;
}
__device__ __forceinline__ void load8_staged(const __nv_bfloat16* p, const float* sc, float (&x)[8]) {
    load8(p, sc, x);
}
__device__ __forceinline__ void load8_staged(const __nv_fp8_storage_t* p, const float* sc, float (&x)[8]) {
    load8(p, sc, x);
}

__device__ __forceinline__ void load_q8(const float* p, float (&q)[8]) {
    float4 a = __ldg(reinterpret_cast<const float4*>(p));
    float4 b = __ldg(reinterpret_cast<const float4*>(p) + 1);
    q[0] = a.x; q[1] = a.y; q[2] = a.z; q[3] = a.w;
    q[4] = b.x; q[5] = b.y; q[6] = b.z; q[7] = b.w;
}

// Exact distance of one candidate from the original blocked FP32 vector:
// d += s_b over the blocks in order (the staged paths' order), two blocks'
// loads in flight at a time.
__device__ __forceinline__ void load8_ro(const float* p, float (&x)[8]) {
    float4 a = __ldg(reinterpret_cast<const float4*>(p));
    float4 b = __ldg(reinterpret_cast<const float4*>(p) + 1);
    x[0] = a.x; x[1] = a.y; x[2] = a.z; x[3] = a.w;
    x[4] = b.x; x[5] = b.y; x[6] = b.z; x[7] = b.w;
}

__device__ __forceinline__ float exact_distance(const float* xo, int64_t npad, const float* qp, int nb) {
    float d = 0.f;
    const int64_t stride = npad * kBlock;
    int b = 0;
    for (; b + 4 <= nb; b += 4) {
        float x0[8], x1[8], x2[8], x3[8], q0[8], q1[8], q2[8], q3[8];
        load8_ro(xo + (int64_t)b * stride, x0);
        load8_ro(xo + (int64_t)(b + 1) * stride, x1);
        load8_ro(xo + (int64_t)(b + 2) * stride, x2);
        load8_ro(xo + (int64_t)(b + 3) * stride, x3);
        load_q8(qp + b * kBlock, q0);
        load_q8(qp + (b + 1) * kBlock, q1);
        load_q8(qp + (b + 2) * kBlock, q2);
        load_q8(qp + (b + 3) * kBlock, q3);
        d += block_sq(q0, x0);
        d += block_sq(q1, x1);
        d += block_sq(q2, x2);
        d += block_sq(q3, x3);
    }
    for (; b < nb; ++b) {
        float x0[8], q0[8];
        load8_ro(xo + (int64_t)b * stride, x0);
        load_q8(qp + b * kBlock, q0);
        d += block_sq(q0, x0);
    }
    return d;
}

// ------------------------------------------------------------ unit decode
// A work unit is (bucket l, tile t of up to kT candidates, group of up to kG
// queries probing l in the wave); its descriptor is built by expand_units.
struct Unit {
    int l, t, nq, nt, item;
};

__device__ __forceinline__ Unit unpack_unit(int4 d) {
    Unit r;
    r.l = d.x;
    r.t = d.y;
    r.item = d.z;
    r.nq = d.w >> 16;
    r.nt = d.w & 0xffff;
    return r;
}

// ------------------------------------------------------------ step pipeline
// A unit's first step is dense (thread c scores candidate c of the tile
// against every query of the unit).  The (query, candidate) pairs that
// survive it live in one list per warp: the survivors of (warp w's
// candidates, query g) go to list (w + g) mod kWarps, so the lists are about
// equally long, and each warp compacts its own list after every later test,
// keeping its 32-lane chunks full whichever queries the live pairs belong
// to.  A pair is stored as the key g << 8 | c (kT <= 256) and its partial
// distance.
constexpr int kQs = 4 * kBlock;     // widest step (Delta_d = 32) in floats
constexpr int kQsPad = kQs + 4;     // query rows 16 B apart in bank terms
constexpr int kWarpCap = kG * kT / kWarps;

struct StepShared {
    unsigned char* buf0;        // two slab buffers at buf0 and buf0 + buf_bytes
    int buf_bytes;
    uint64_t* bar;
    uint16_t* key;              // kWarps x kWarpCap pair keys
    float* part;                // kWarps x kWarpCap partial distances
    int* n;                     // live pairs per warp
    unsigned long long* st;     // per query: candidates, pruned, exact, dims
    float* qs;                  // kG x kQsPad: the step's query values
    float* sc;                  // kQs: the step's FP8 scales
    const int* q;               // kG query ids
    const float* tau;           // kG
    float* rx;                  // kT: the tile's stored residual norms after the step (RES)
    float* rq;                  // kG: the queries' residual terms after the step (RES)
};

// RES inputs of one tile: the residual norm of slot s from block b on is
// sfx[b * stride + s] (sfx points at the tile's first slot); query q's term
// after step k is rq[q * rq_stride + k] for k < rq_stride.
struct ResTile {
    const float* sfx;
    int64_t stride;
    const float* rq;
    int rq_stride;
};

// Runs `nsteps` slab steps over the tile: slab k covers blocks
// [k*NBLK, min((k+1)*NBLK, nb)) of the source (rotated slabs in PRUNE mode,
// original vectors otherwise).
//  * Without PRUNE every step is dense: thread (warp, lane) owns candidate
//    c = 32 warp + lane of the tile and accumulates pd[g] for every query g
//    of the unit in registers; the unit's queries are read as broadcasts.
//  * With PRUNE step 0 is dense as well.  Every pair is tested after it and
//    the survivors go to the per-warp lists (warp w keeps its own
//    candidates' survivors, query by query); later steps walk those lists,
//    testing and compacting after each slab.  The test after slab k is the
//    learned one, m1_k dis' + beta_k > tau (Section V-A); with FINAL the
//    last slab (k = nsteps - 1) completes the rotated distance and the test
//    is dis'_S > (sqrt(tau) + e_x)^2 (1 + kFinalRel) (e_x = eps_tile[c], 0
//    without eps_tile).  With EST the test after slab k < S - 1 is the
//    Gaussian-bound one of Section IV-C (Algorithm 2 with Eq. 1-2):
//    dis'_k + ||x~_r||^2 + (||q'_r||^2 - m sigma) > tau, the last two read
//    from `res` (sh.rx per candidate, sh.rq per query; staged like the query
//    values).  A pair whose query has tau = +inf is never pruned.
// Partial sums grow block by block in block order on every path, so a pair
// gets the same value whichever path computed it.  Returns false if a
// bounded wait gave up.
template <class E, int NBLK, bool PRUNE, bool FINAL, bool EST>
__device__ __forceinline__ bool run_steps(const E* src, int64_t npad, int t, int nt, int nq, int nsteps,
                                          int nb, int D, const StepShared& sh, uint32_t& phase_bits,
                                          const float* qsrc, int Dpad, const float* m1,
                                          const float* beta, const float* scale,
                                          const float* eps_tile, const ResTile& res, int32_t* status,
                                          unsigned long long* staged, bool want_stats, float (&pd)[kG]) {
    static_assert(!EST || kScanThreads == kT, "a thread stages one candidate's residual norm");
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    const int nt_copy = (nt + 31) & ~31;
    const uint32_t blk_bytes = (uint32_t)nt_copy * kBlock * sizeof(E);
    // phase_bits bit b is the parity to wait for on buffer b
    auto issue = [src, npad, t, nb, blk_bytes, staged, &sh](int k) {
        int b0 = k * NBLK, nbk = min(NBLK, nb - b0);
        unsigned char* dst = sh.buf0 + (k & 1) * sh.buf_bytes;
        fence_proxy_async();
        mbar_expect_tx(sh.bar + (k & 1), blk_bytes * nbk);
        for (int bb = 0; bb < nbk; ++bb)
            bulk_g2s(dst + (size_t)bb * kT * kBlock * sizeof(E),
                     src + ((int64_t)(b0 + bb) * npad + (int64_t)t * kT) * kBlock, blk_bytes,
                     sh.bar + (k & 1));
        if (staged) atomicAdd(staged, (unsigned long long)blk_bytes * nbk);
    };
#pragma unroll
    for (int g = 0; g < kG; ++g) pd[g] = 0.f;
    if (PRUNE && tid < kWarps) sh.n[tid] = 0;  // step 0 appends with atomics
    if (nsteps <= 0) return true;
    if (tid == 0) issue(0);
    int k = 0;
    bool pending_next = false;
    uint16_t* key = sh.key + warp * kWarpCap;
    float* part = sh.part + warp * kWarpCap;
    const int c_own = warp * 32 + lane;
    const bool own_valid = c_own < nt;
    const bool warp_live = warp * 32 < nt;  // warps past the tile's end skip the dense work
    // the query values (and FP8 scales) of step k for every query of the
    // unit: each thread handles kVals values (and one scale); step k + 1's
    // are loaded into registers during step k and stored after its last read
    constexpr int kVals = kG * kQs / kScanThreads;
    static_assert(kScanThreads % kQs == 0, "a thread keeps one column j of the query values");
    float qv_next[kVals], sc_next = 0.f, rx_next = 0.f, rq_next = 0.f;
    // this thread's values: column j = tid % kQs of rows g = tid / kQs + h * (kScanThreads / kQs)
    const int vj = tid % kQs, vg0 = tid / kQs;
    const float* vsrc[kVals];
#pragma unroll
    for (int h = 0; h < kVals; ++h) {
        const int g = vg0 + h * (kScanThreads / kQs);
        vsrc[h] = g < nq ? qsrc + (int64_t)sh.q[g] * Dpad + vj : nullptr;
    }
    auto load_vals = [&](int kk) {
        const int b0 = kk * NBLK, w8 = min(NBLK, nb - b0) * kBlock;
#pragma unroll
        for (int h = 0; h < kVals; ++h)
            qv_next[h] = vsrc[h] && vj < w8 ? __ldg(vsrc[h] + b0 * kBlock) : 0.f;
        if (scale) sc_next = tid < w8 ? __ldg(scale + b0 * kBlock + tid) : 0.f;
        if (EST) {
            const int br = min((kk + 1) * NBLK, nb);
            rx_next = tid < nt ? __ldg(res.sfx + (int64_t)br * res.stride + tid) : 0.f;
            rq_next = tid < nq && kk < res.rq_stride ? __ldg(res.rq + (int64_t)sh.q[tid] * res.rq_stride + kk) : 0.f;
        }
    };
    auto store_vals = [&]() {
#pragma unroll
        for (int h = 0; h < kVals; ++h)
            if (vsrc[h]) sh.qs[(vg0 + h * (kScanThreads / kQs)) * kQsPad + vj] = qv_next[h];
        if (scale && tid < kQs) sh.sc[tid] = sc_next;
        if (EST) {
            sh.rx[tid] = rx_next;
            if (tid < kG) sh.rq[tid] = rq_next;
        }
    };
    load_vals(0);
    store_vals();
    for (; k < nsteps; ++k) {
        const int b0 = k * NBLK, nbk = min(NBLK, nb - b0);
        bool got = mbar_wait(sh.bar + (k & 1), (phase_bits >> (k & 1)) & 1u, status);
        phase_bits ^= 1u << (k & 1);
        if (!__syncthreads_and(got)) return false;
        pending_next = k + 1 < nsteps;
        if (tid == 0 && pending_next) issue(k + 1);
        if (pending_next) load_vals(k + 1);
        const E* bk = reinterpret_cast<const E*>(sh.buf0 + (k & 1) * sh.buf_bytes);
        const int dims_k = min((k + 1) * NBLK * kBlock, D);
        const bool final_k = FINAL && k == nsteps - 1;
        const float mm = PRUNE && !EST && !final_k ? m1[k] : 0.f;
        const float bt = PRUNE && !EST && !final_k ? beta[k] : 0.f;
        int out = 0;
        if (!PRUNE || k == 0) {
            // dense: block by block, this thread's candidate against every
            // query of the unit
#pragma unroll
            for (int bb = 0; bb < NBLK; ++bb) {
                if (warp_live && bb < nbk) {
                    float x[8];
                    load8_staged(bk + ((size_t)bb * kT + c_own) * kBlock, sh.sc + bb * kBlock, x);
#pragma unroll
                    for (int g = 0; g < kG; ++g) {
                        if (g < nq) {
                            float qv[8];
                            load8(sh.qs + g * kQsPad + bb * kBlock, nullptr, qv);
                            pd[g] += block_sq(qv, x);
                        }
                    }
                }
            }
            if (PRUNE && warp_live) {
                // test every pair; the survivors of (this warp, query g) go
                // to list (warp + g) mod kWarps, so every list gets a share
                // of every warp's candidates and of every query.  Pass 1
                // counts them (lane g keeps query g's count) and reserves
                // every query's space with one atomic instruction; pass 2
                // writes them.
                const float e_own = FINAL && final_k && eps_tile && own_valid ? eps_tile[c_own] : 0.f;
                uint32_t keep_bits = 0u;
                int mine = 0;
#pragma unroll
                for (int g = 0; g < kG; ++g) {
                    if (g < nq) {
                        bool cut;
                        if (FINAL && final_k) {
                            const float r = sqrtf(sh.tau[g]) + e_own;
                            cut = pd[g] > r * r * (1.f + kFinalRel);
                        } else if (EST) {
                            cut = pd[g] + sh.rx[c_own] + sh.rq[g] > sh.tau[g];
                        } else {
                            cut = fmaf(mm, pd[g], bt) > sh.tau[g];
                        }
                        const bool keep = own_valid && !cut;
                        keep_bits |= (uint32_t)keep << g;
                        const int cnt = __popc(__ballot_sync(0xffffffffu, keep));
                        if (lane == g) mine = cnt;
                        if (want_stats) {
                            const int np = __popc(__ballot_sync(0xffffffffu, own_valid && cut));
                            if (lane == 0 && np) {
                                atomicAdd(&sh.st[g * 4 + 1], (unsigned long long)np);
                                atomicAdd(&sh.st[g * 4 + 3], (unsigned long long)np * dims_k);
                            }
                        }
                    }
                }
                int base_mine = 0;
                if (lane < nq && mine) base_mine = atomicAdd(&sh.n[(warp + lane) & (kWarps - 1)], mine);
#pragma unroll
                for (int g = 0; g < kG; ++g) {
                    if (g < nq) {
                        const bool keep = (keep_bits >> g) & 1u;
                        const unsigned bal = __ballot_sync(0xffffffffu, keep);
                        const int base = __shfl_sync(0xffffffffu, base_mine, g);
                        if (keep) {
                            const int pos = ((warp + g) & (kWarps - 1)) * kWarpCap + base + __popc(bal & lanemask_lt());
                            sh.key[pos] = (uint16_t)((g << 8) | c_own);
                            sh.part[pos] = pd[g];
                        }
                    }
                }
            }
        } else {
            // sparse: the warp's live pairs, 32 at a time
            const int n = sh.n[warp];
            for (int base = 0; base < n; base += 32) {
                const int i = base + lane;
                const bool valid = i < n;
                int kk = 0, g = 0, c = 0;
                float pv = 0.f;
                if (valid) {
                    kk = key[i];
                    g = kk >> 8;
                    c = kk & 255;
                    pv = part[i];
                    const float* qg = sh.qs + g * kQsPad;
#pragma unroll
                    for (int bb = 0; bb < NBLK; ++bb) {
                        if (bb < nbk) {
                            float x[8], qv[8];
                            load8_staged(bk + ((size_t)bb * kT + c) * kBlock, sh.sc + bb * kBlock, x);
                            load8(qg + bb * kBlock, nullptr, qv);
                            pv += block_sq(qv, x);
                        }
                    }
                }
                bool cut = false;
                if (FINAL && final_k) {
                    if (valid) {
                        const float r = sqrtf(sh.tau[g]) + (eps_tile ? eps_tile[c] : 0.f);
                        cut = pv > r * r * (1.f + kFinalRel);
                    }
                } else if (EST) {
                    cut = pv + sh.rx[c] + sh.rq[g] > sh.tau[g];
                } else {
                    cut = fmaf(mm, pv, bt) > sh.tau[g];
                }
                const bool keep = valid && !cut;
                const unsigned bal = __ballot_sync(0xffffffffu, keep);
                __syncwarp();
                if (keep) {
                    const int pos = out + __popc(bal & lanemask_lt());
                    key[pos] = (uint16_t)kk;
                    part[pos] = pv;
                }
                out += __popc(bal);
                if (want_stats && valid && !keep) {
                    atomicAdd(&sh.st[g * 4 + 1], 1ull);
                    atomicAdd(&sh.st[g * 4 + 3], (unsigned long long)dims_k);
                }
            }
        }
        if (PRUNE && k > 0) {
            __syncwarp();
            if (lane == 0) sh.n[warp] = out;
        }
        __syncthreads();
        if (pending_next) store_vals();  // every read of step k's values is done
        if (PRUNE) {
            int live = 0;
            for (int w = 0; w < kWarps; ++w) live |= sh.n[w];
            if (!live) break;
        }
    }
    if (PRUNE && k < nsteps && pending_next) {
        // the loop left early with the next slab in flight: drain it
        int kn = k + 1;
        bool got = mbar_wait(sh.bar + (kn & 1), (phase_bits >> (kn & 1)) & 1u, status);
        phase_bits ^= 1u << (kn & 1);
        if (!__syncthreads_and(got)) return false;
    }
    return true;
}

// Append (d, slot) to query q's candidate buffer for every lane with app set,
// q the same on every lane of the warp: one atomic for the warp.
__device__ __forceinline__ void append_uniform(const WaveView& wv, int w, int q, bool app, float d,
                                               int32_t slot, int lane) {
    const unsigned bal = __ballot_sync(0xffffffffu, app);
    if (!bal) return;
    int base = 0;
    if (lane == 0) base = atomicAdd(&wv.cand_cnt[q], __popc(bal));
    base = __shfl_sync(0xffffffffu, base, 0);
    if (!app) return;
    const int64_t* co = wv.cand_off + (int64_t)w * (wv.B + 1);
    const int64_t off = co[q], cap = co[q + 1] - off;
    const int s = base + __popc(bal & lanemask_lt());
    if (s < cap) {
        wv.cand_d[off + s] = d;
        wv.cand_pos[off + s] = slot;
    } else {
        atomicCAS(wv.status, 0, (int)DADE_EINVAL);
    }
}

// Append this lane's candidate (slot `slot`, valid or not) against every query
// g < nq of the unit whose distance pd[g] is at most tau[g].  The warp
// reserves every query's space with one atomic instruction (lane g for query
// qs[g]) and reads the queries' buffer offsets in the same round trip, then
// writes query by query.
__device__ __forceinline__ void append_rows(const WaveView& wv, int w, const int* qs, const float* tau, int nq,
                                            bool valid, const float (&pd)[kG], int32_t slot, int lane) {
    static_assert(kG <= 32, "lane g reserves query g's space");
    uint32_t bits = 0u;
    int mine = 0;
#pragma unroll
    for (int g = 0; g < kG; ++g) {
        if (g < nq) {
            const bool app = valid && pd[g] <= tau[g];
            bits |= (uint32_t)app << g;
            const int cnt = __popc(__ballot_sync(0xffffffffu, app));
            if (lane == g) mine = cnt;
        }
    }
    int base_mine = 0;
    long long off_mine = 0, cap_mine = 0;
    if (lane < nq && mine) {
        const int q = qs[lane];
        base_mine = atomicAdd(&wv.cand_cnt[q], mine);
        const int64_t* co = wv.cand_off + (int64_t)w * (wv.B + 1);
        off_mine = co[q];
        cap_mine = co[q + 1] - off_mine;
    }
#pragma unroll
    for (int g = 0; g < kG; ++g) {
        if (g < nq) {
            const bool app = (bits >> g) & 1u;
            const unsigned bal = __ballot_sync(0xffffffffu, app);
            if (bal) {
                const int base = __shfl_sync(0xffffffffu, base_mine, g);
                const long long off = __shfl_sync(0xffffffffu, off_mine, g);
                const long long cap = __shfl_sync(0xffffffffu, cap_mine, g);
                if (app) {
                    const int s = base + __popc(bal & lanemask_lt());
                    if (s < cap) {
                        wv.cand_d[off + s] = pd[g];
                        wv.cand_pos[off + s] = slot;
                    } else {
                        atomicCAS(wv.status, 0, (int)DADE_EINVAL);
                    }
                }
            }
        }
    }
}

// Append (d, slot) to query q's candidate buffer for every lane with app set;
// lanes of the same query share one atomic.
__device__ __forceinline__ void append_any(const WaveView& wv, int w, int q, bool app, float d,
                                           int32_t slot, int lane) {
    if (!__ballot_sync(0xffffffffu, app)) return;
    const unsigned peers = __match_any_sync(0xffffffffu, app ? q : -1);
    if (!app) return;
    const int leader = __ffs(peers) - 1;
    int base = 0;
    if (lane == leader) base = atomicAdd(&wv.cand_cnt[q], __popc(peers));
    base = __shfl_sync(peers, base, leader);
    const int64_t* co = wv.cand_off + (int64_t)w * (wv.B + 1);
    const int64_t off = co[q], cap = co[q + 1] - off;
    const int s = base + __popc(peers & lanemask_lt());
    if (s < cap) {
        wv.cand_d[off + s] = d;
        wv.cand_pos[off + s] = slot;
    } else {
        atomicCAS(wv.status, 0, (int)DADE_EINVAL);
    }
}

// ------------------------------------------------------------ wave scan
// Dynamic shared memory: two slab buffers, and for the pruned path the
// per-warp pair lists (the full-dimension scan has none).
template <int NBLK, bool FULL>
constexpr int scan_smem_bytes() {
    return 2 * NBLK * kT * kBlock * 4 + (FULL ? 0 : kWarps * kWarpCap * (int)(sizeof(uint16_t) + sizeof(float)));
}

template <int DT, int NBLK, bool FULL, bool FIN, bool EST>
__global__ void __launch_bounds__(kScanThreads, (NBLK <= 2 && !FULL && !EST) ? 7 : 6) wave_scan_kernel(IndexView ix, WaveView wv, int w,
                                                                 const float* __restrict__ m1,
                                                                 const float* __restrict__ beta,
                                                                 int S) {
    using E = typename Elem<DT>::T;
    constexpr int BUF = NBLK * kT * kBlock * 4;  // sized for FP32 (original vectors)
    extern __shared__ __align__(128) unsigned char smem[];
    __shared__ __align__(8) uint64_t bar[2];
    __shared__ int s_unit;
    __shared__ int4 s_desc;
    __shared__ int s_q[kG], s_n[kWarps];
    __shared__ float s_tau[kG];
    __shared__ unsigned long long s_st[kG * 4];
    __shared__ __align__(16) float s_qs[kG * kQsPad];
    __shared__ __align__(16) float s_sc[kQs];
    __shared__ float s_rx[EST ? kT : 1], s_rq[EST ? kG : 1];
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;

    StepShared sh;
    sh.buf0 = smem;
    sh.buf_bytes = BUF;
    sh.key = FULL ? nullptr : reinterpret_cast<uint16_t*>(smem + 2 * BUF);
    sh.part = FULL ? nullptr : reinterpret_cast<float*>(smem + 2 * BUF + kWarps * kWarpCap * sizeof(uint16_t));
    sh.bar = bar;
    sh.n = s_n;
    sh.st = s_st;
    sh.qs = s_qs;
    sh.sc = s_sc;
    sh.q = s_q;
    sh.tau = s_tau;
    sh.rx = s_rx;
    sh.rq = s_rq;
    if (tid == 0) {
        mbar_init(&bar[0], 1);
        mbar_init(&bar[1], 1);
        fence_mbar_init();
    }
    __syncthreads();
    uint32_t ph = 0u;
    const int total = wv.unit_off[(int64_t)w * (ix.nlist + 1) + ix.nlist];
    const int4* units = wv.units + wv.ubase[w];
    const int nsteps_full = (ix.nb + NBLK - 1) / NBLK;
    const bool want_stats = wv.stats != nullptr;
    // thread 0 claims the next unit and loads its descriptor one unit ahead
    int next_u = 0;
    int4 next_d = make_int4(0, 0, 0, 0);
    if (tid == 0) {
        next_u = atomicAdd(&wv.work[w], 1);
        if (next_u < total) next_d = units[next_u];
    }

    for (;;) {
        if (tid == 0) {
            s_unit = next_u;
            s_desc = next_d;
            if (next_u < total) {
                next_u = atomicAdd(&wv.work[w], 1);
                if (next_u < total) next_d = units[next_u];
            }
        }
        __syncthreads();
        if (s_unit >= total) break;
        const Unit un = unpack_unit(s_desc);
        const int l = un.l, t = un.t, nq = un.nq, nt = un.nt;
        // the bucket's extent is read before the barrier below, in the same
        // round trip as the queries' ids and bounds
        const int64_t slot_l = ix.list_slot[l];
        const int64_t npad = ix.list_slot[l + 1] - slot_l;
        bool my_inf = true;
        if (tid < nq) {
            const int q = wv.items[un.item + tid];
            const float tq = wv.tau[q];
            s_q[tid] = q;
            s_tau[tid] = tq;
            my_inf = isinf(tq);
            s_st[tid * 4 + 0] = (unsigned long long)nt;
            s_st[tid * 4 + 1] = s_st[tid * 4 + 2] = s_st[tid * 4 + 3] = 0ull;
        }
        const bool all_inf = __syncthreads_and(my_inf);
        const int64_t ebase = slot_l * ix.Dpad;
        const int32_t slot0 = (int32_t)(slot_l + (int64_t)t * kT);
        const uint16_t* key = sh.key + warp * kWarpCap;
        float pd[kG];
        bool ok;
        if (FULL || all_inf || (S <= 1 && !FIN)) {
            // every pair's exact distance through the staged pipeline (with
            // no test to run, that is also the pruned search's result)
            ok = run_steps<float, NBLK, false, false, false>(ix.orig + ebase, npad, t, nt, nq, nsteps_full,
                                                             ix.nb, ix.D, sh, ph, wv.qpad, ix.Dpad, nullptr,
                                                             nullptr, nullptr, nullptr, ResTile{}, wv.status,
                                                             wv.staged_bytes, want_stats, pd);
            if (!ok) break;
            const int c = warp * 32 + lane;
            append_rows(wv, w, s_q, s_tau, nq, c < nt, pd, slot0 + c, lane);
            if (want_stats && tid < nq) {
                s_st[tid * 4 + 2] += (unsigned long long)nt;
                s_st[tid * 4 + 3] += (unsigned long long)nt * ix.D;
            }
        } else {
            const E* slab = reinterpret_cast<const E*>(ix.slab) + ebase;
            const float* scl = DT == DADE_SLAB_FP8E4M3 ? ix.scale : nullptr;
            ResTile rt{};
            if (EST) rt = ResTile{ix.sfx + slot0, ix.total_slots, wv.res_q, wv.res_stride};
            if (FIN)
                ok = run_steps<E, NBLK, true, true, EST>(slab, npad, t, nt, nq, S, ix.nb, ix.D, sh, ph, wv.qrot,
                                                         ix.Dpad, m1, beta, scl, ix.eps ? ix.eps + slot0 : nullptr,
                                                         rt, wv.status, wv.staged_bytes, want_stats, pd);
            else
                ok = run_steps<E, NBLK, true, false, EST>(slab, npad, t, nt, nq, wv.test_steps, ix.nb, ix.D, sh, ph,
                                                          wv.qrot, ix.Dpad, m1, beta, scl, nullptr, rt, wv.status,
                                                          wv.staged_bytes, want_stats, pd);
            if (!ok) break;
            // survivors: exact distance from the original vector, one lane each
            const int n = s_n[warp];
            for (int base = 0; base < n; base += 32) {
                const int i = base + lane;
                const bool valid = i < n;
                const int kk = valid ? key[i] : 0;
                const int g = kk >> 8, c = kk & 255;
                const int q = s_q[g];
                float d = 0.f;
                if (valid)
                    d = exact_distance(ix.orig + ebase + ((int64_t)t * kT + c) * kBlock, npad,
                                       wv.qpad + (int64_t)q * ix.Dpad, ix.nb);
                append_any(wv, w, q, valid && d <= s_tau[g], d, slot0 + c, lane);
                if (want_stats && valid) {
                    atomicAdd(&s_st[g * 4 + 2], 1ull);
                    atomicAdd(&s_st[g * 4 + 3], (unsigned long long)ix.D);
                }
            }
            if (wv.staged_bytes && lane == 0 && n)
                atomicAdd(wv.staged_bytes, (unsigned long long)n * ix.nb * kBlock * sizeof(float));
        }
        __syncthreads();
        if (want_stats && tid < nq * 4) {
            if (s_st[tid]) atomicAdd((unsigned long long*)&wv.stats[(int64_t)s_q[tid / 4] * 4 + (tid % 4)], s_st[tid]);
        }
        __syncthreads();
    }
}

// ------------------------------------------------------------ launchers
template <int DT, int NBLK, bool FULL, bool FIN, bool EST>
cudaError_t launch_scan_t(const IndexView& ix, const WaveView& wv, int w, const float* m1,
                          const float* beta, int S, cudaStream_t st) {
    constexpr int SMEM = scan_smem_bytes<NBLK, FULL>();
    static int grid = 0;
    auto kern = wave_scan_kernel<DT, NBLK, FULL, FIN, EST>;
    if (grid == 0) {
        cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, SMEM);
        if (e != cudaSuccess) return e;
        int dev = 0, sms = 0, per = 0;
        cudaGetDevice(&dev);
        cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
        e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per, kern, kScanThreads, SMEM);
        if (e != cudaSuccess) return e;
        grid = sms * (per > 0 ? per : 1);
    }
    kern<<<grid, kScanThreads, SMEM, st>>>(ix, wv, w, m1, beta, S);
    return cudaGetLastError();
}

}  // namespace
}  // namespace dade
