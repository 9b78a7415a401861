// The estimate-and-prune wave scan on the tensor cores (tcgen05).
//
// Method (arXiv 2404.16322): a candidate's partial distance is accumulated
// Delta_d rotated dimensions at a time (the loop of Algorithm 2) and after
// each step the learned test m1_s dis'_s + beta_s > tau prunes it
// (Section V-A; one classifier per step, Section V-B "Incremental
// Correction"); survivors get the exact distance (Section II-A) and join the
// result queue whose largest entry is tau (Section I).
//
// Here a work unit is (bucket l, tile of up to 128 candidates, group of up
// to QW = 128 queries probing l in the wave), and the partial distances of
// the whole tile x group are one dense contraction per step:
//   dis'_s(q, x) = ||q_{<d}||^2 + ||x_{<d}||^2 - 2 <q_{<d}, x_{<d}>,  d = s Delta_d,
// with the cumulative dot product accumulated step by step in tensor memory
// (M = 128 candidates, N = the group's queries rounded up to 16, K = 8 per
// MMA, split TF32: the candidate values' parts hi + mid (mid = 0 for BF16,
// which TF32 holds exactly) against the query values' parts hi + mid,
// products hi.hi + hi.mid + mid.hi, FP32 accumulation).
//  - The candidate operand comes from the index's pre-split copy
//    (build_tc_operands): one cp.async.bulk per step, double buffered.
//  - The query operand is gathered by the threads (thread i loads query i's
//    step values, splits them, stores them in the canonical layout) while
//    they also sum the squares of their query's values.
//  - One thread issues the MMAs and commits to an mbarrier.  A CTA has QW
//    threads: warp w reads accumulator lanes (candidates) 32 (w % 4) ..
//    32 (w % 4) + 31 and columns (queries) 128 (w / 4) .. 128 (w / 4) + 127
//    (tcgen05.ld), and each thread tests its candidate against those
//    queries:
//      m1 dis' + beta - tau = m1 ||x||^2 + (m1 ||q||^2 + beta - tau) - 2 m1 <q, x>  > 0,
//    keeping one alive bit per pair in registers.
//  - With the final test, one more step completes the rotated distance and
//    a pair is kept iff dis'_S <= (sqrt(tau) + e_x)^2 (1 + kFinalRel).
//  - After the last step the surviving pairs are listed per warp in shared
//    memory and get the exact FP32 distance, one lane each.
// Every device wait is bounded (about 2 s, then DADE_ETIMEOUT).
#include "scan_steps.cuh"
#include "tc_common.cuh"

namespace dade {
namespace {

// exact_distance with eight blocks' loads in flight at a time (the same
// arithmetic: block sums added in block order).
__device__ __forceinline__ float exact_distance8(const float* xo, int64_t npad, const float* qp, int nb) {
    float d = 0.f;
    const int64_t stride = npad * kBlock;
    int b = 0;
    for (; b + 8 <= nb; b += 8) {
        float x[8][8];
#pragma unroll
        for (int i = 0; i < 8; ++i) load8_ro(xo + (int64_t)(b + i) * stride, x[i]);
#pragma unroll
        for (int i = 0; i < 8; ++i) {
            float q[8];
            load_q8(qp + (b + i) * kBlock, q);
            d += block_sq(q, x[i]);
        }
    }
    for (; b < nb; ++b) {
        float x0[8], q0[8];
        load8_ro(xo + (int64_t)b * stride, x0);
        load_q8(qp + b * kBlock, q0);
        d += block_sq(q0, x0);
    }
    return d;
}

// Queries per unit: 128 (four CTAs of four warps per SM, so that one CTA's
// tests overlap the others' MMAs and copies; 256-query units with eight
// warps and two CTAs per SM measured slower on the SIFT-shaped workload).
template <int NBLK> constexpr int tc_qw() { return 128; }

template <int NBLK, int PARTS, int QW>
constexpr int tc_smem_bytes() {
    // two candidate-operand buffers, one query-operand buffer (QW rows per
    // chunk), alignment slack
    return (2 * NBLK * PARTS) * 4096 + 2 * NBLK * QW * 32 + 1024;
}

// With FIN the last step (k = nsteps - 1) completes the rotated distance
// and its test is the one on the whole distance: a candidate is kept iff
// dis'_S <= (sqrt(tau) + e_x)^2 (1 + kFinalRel), e_x its stored vector's
// quantisation error (0 for FP32 slabs).
template <int NBLK, int PARTS, int QW, bool FIN>
__global__ void __launch_bounds__(QW, 512 / QW) tc_scan_kernel(IndexView ix, WaveView wv, int w,
                                                               const float* __restrict__ m1,
                                                               const float* __restrict__ beta, int nsteps) {
    static_assert(QW == 128 || QW == 256, "one or two warps per accumulator lane quarter");
    constexpr int ACH = NBLK * PARTS;       // chunks per candidate-operand buffer
    constexpr int BCH = QW * kBlock;        // floats per query-operand chunk (QW rows x 8 dims)
    constexpr int NW = 4;                   // alive words per thread: 128 columns
    extern __shared__ __align__(1024) unsigned char tsm[];
    __shared__ __align__(8) uint64_t bar_a[2];
    __shared__ __align__(8) uint64_t bar_m;
    __shared__ uint32_t s_taddr;
    __shared__ int s_unit, s_fail;
    __shared__ int4 s_desc;
    __shared__ int s_q[QW];
    __shared__ float s_tau[QW];
    __shared__ __align__(16) float s_a[2][QW];
    __shared__ __align__(16) float s_rt[FIN ? QW : 1];  // sqrt(tau) per query (the final test)
    __shared__ unsigned s_st[QW * 4];
    unsigned char* base = reinterpret_cast<unsigned char*>((reinterpret_cast<uintptr_t>(tsm) + 1023) & ~uintptr_t(1023));
    float* abuf = reinterpret_cast<float*>(base);
    float* bbuf = abuf + 2 * ACH * kChunkF;
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    const int row = (warp & 3) * 32 + lane;   // this thread's candidate (accumulator lane)
    const int cb0 = (warp >> 2) * 128;        // its first column (query)

    if (warp == 0) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(&s_taddr)),
                     "r"(QW)
                     : "memory");
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
    }
    if (tid == 0) {
        mbar_init(&bar_a[0], 1);
        mbar_init(&bar_a[1], 1);
        mbar_init(&bar_m, 1);
        fence_mbar_init();
        s_fail = 0;
    }
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    const uint32_t tmem = s_taddr;
    const uint32_t tmem_row = tmem + ((uint32_t)((warp & 3) * 32) << 16) + (uint32_t)cb0;

    uint32_t ph_a = 0u, ph_m = 0u;  // parity to wait for: bit b for bar_a[b]; bar_m
    const int total = wv.unit_off[(int64_t)w * (ix.nlist + 1) + ix.nlist];
    const int4* units = wv.units + wv.ubase[w];
    const int nb = ix.nb;
    const bool want_stats = wv.stats != nullptr;
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
        if (s_unit >= total || s_fail) break;
        const Unit un = unpack_unit(s_desc);
        const int l = un.l, t = un.t, nq = un.nq, nt = un.nt;
        const int ncols = (nq + 15) & ~15;
        const int mycols = min(128, max(0, ncols - cb0));   // this warp's columns
        const int myq = min(128, max(0, nq - cb0));
        const int64_t slot_l = ix.list_slot[l];
        const int64_t npad = ix.list_slot[l + 1] - slot_l;
        const int32_t slot0 = (int32_t)(slot_l + (int64_t)t * kTcRows);
        const float* asrc = ix.tcslab + ((ix.tile_base[l] + t) * nb) * (int64_t)PARTS * kChunkF;
        auto a_bytes = [nb](int k) { return (uint32_t)(min(NBLK, nb - k * NBLK) * PARTS * 4096); };
        auto issue_a = [&](int k) {
            fence_proxy_async();
            mbar_expect_tx(&bar_a[k & 1], a_bytes(k));
            bulk_g2s(abuf + (k & 1) * ACH * kChunkF, asrc + (int64_t)k * NBLK * PARTS * kChunkF, a_bytes(k),
                     &bar_a[k & 1]);
            if (wv.staged_bytes) atomicAdd(wv.staged_bytes, (unsigned long long)a_bytes(k));
        };
        // the candidate operand of step k is copied while step k - 1 runs
        if (tid == 0 && nsteps > 0) issue_a(0);
        float tq = 0.f, qn = 0.f, xn = 0.f;
        const float* qsrc = nullptr;
        if (tid < nq) {
            const int q = wv.items[un.item + tid];
            tq = wv.tau[q];
            s_q[tid] = q;
            s_tau[tid] = tq;
            if (FIN) s_rt[tid] = sqrtf(tq);
            qsrc = wv.qrot + (int64_t)q * ix.Dpad;
        }
        const float ex = (FIN && ix.eps && row < nt) ? ix.eps[slot0 + row] : 0.f;
        if (want_stats)
            for (int i = tid; i < nq * 4; i += QW) s_st[i] = (i & 3) == 0 ? (unsigned)nt : 0u;
        // alive bit j of word c4: the pair (this thread's candidate, query cb0 + 32 c4 + j)
        uint32_t alive[NW];
#pragma unroll
        for (int c4 = 0; c4 < NW; ++c4) {
            const int n = min(32, max(0, myq - c4 * 32));
            alive[c4] = (row < nt && n > 0) ? (n == 32 ? 0xffffffffu : ((1u << n) - 1u)) : 0u;
        }
        float qv[NBLK * kBlock];
        auto load_q = [&](int k) {
            const int b0 = k * NBLK, nbk = min(NBLK, nb - b0);
#pragma unroll
            for (int bb = 0; bb < NBLK; ++bb) {
                float4 u = make_float4(0.f, 0.f, 0.f, 0.f), v = u;
                if (qsrc && bb < nbk) {
                    u = __ldg(reinterpret_cast<const float4*>(qsrc + (b0 + bb) * kBlock));
                    v = __ldg(reinterpret_cast<const float4*>(qsrc + (b0 + bb) * kBlock) + 1);
                }
                qv[bb * 8 + 0] = u.x; qv[bb * 8 + 1] = u.y; qv[bb * 8 + 2] = u.z; qv[bb * 8 + 3] = u.w;
                qv[bb * 8 + 4] = v.x; qv[bb * 8 + 5] = v.y; qv[bb * 8 + 6] = v.z; qv[bb * 8 + 7] = v.w;
            }
        };
        load_q(0);
        int k = 0;
        bool mma_failed = false;
        for (; k < nsteps; ++k) {
            const int b0 = k * NBLK, nbk = min(NBLK, nb - b0);
            const bool fin_k = FIN && k == nsteps - 1;
            const float mk = fin_k ? 1.f : m1[k], bk = fin_k ? 0.f : beta[k];
            // 1. the step's query operand, the query norms and the test constants
            if (tid < nq) {
#pragma unroll
                for (int bb = 0; bb < NBLK; ++bb) {
                    if (bb < nbk) {
                        float h[8], m[8];
#pragma unroll
                        for (int j = 0; j < 8; ++j) {
                            const float x = qv[bb * 8 + j];
                            h[j] = tf32_rna(x);
                            m[j] = tf32_rna(x - h[j]);
                            qn = fmaf(x, x, qn);
                        }
                        float* ch = bbuf + (bb * 2) * BCH + chunk_off(tid, 0);
                        float* cm = ch + BCH;
                        *reinterpret_cast<float4*>(ch) = make_float4(h[0], h[1], h[2], h[3]);
                        *reinterpret_cast<float4*>(ch + 32) = make_float4(h[4], h[5], h[6], h[7]);
                        *reinterpret_cast<float4*>(cm) = make_float4(m[0], m[1], m[2], m[3]);
                        *reinterpret_cast<float4*>(cm + 32) = make_float4(m[4], m[5], m[6], m[7]);
                    }
                }
                s_a[k & 1][tid] = fin_k ? qn : fmaf(mk, qn, bk) - tq;
            }
            fence_proxy_async();
            // 2. the candidate operand of the step has landed
            const bool ok = warp_wait(&bar_a[k & 1], (ph_a >> (k & 1)) & 1u, wv.status, lane);
            ph_a ^= 1u << (k & 1);
            if (!ok && lane == 0) s_fail = 1;
            uint32_t any = 0u;
#pragma unroll
            for (int c4 = 0; c4 < NW; ++c4) any |= alive[c4];
            // every thread is done with step k - 1 here: its candidate buffer
            // is free, and the tensor core has finished reading the operands
            const int live = __syncthreads_or(any != 0u);
            if (s_fail || !live) break;
            // 3. the MMAs of the step, issued by one thread, and the copy of
            //    the next step's candidate operand into the other buffer
            if (tid == 0) {
                if (k + 1 < nsteps) issue_a(k + 1);
                tc_fence_after();
                const uint32_t idesc = tc_idesc(ncols);
                const uint32_t a0 = smem_u32(abuf + (k & 1) * ACH * kChunkF), bq = smem_u32(bbuf);
#pragma unroll
                for (int bb = 0; bb < NBLK; ++bb) {
                    if (bb < nbk) {
                        const uint32_t ah = a0 + (uint32_t)(bb * PARTS) * 4096u, am = ah + 4096u;
                        const uint32_t bh = bq + (uint32_t)(bb * 2) * (BCH * 4u), bm = bh + BCH * 4u;
                        tc_mma(tmem, tc_desc(ah), tc_desc(bh), idesc, (k > 0 || bb > 0) ? 1u : 0u);
                        tc_mma(tmem, tc_desc(ah), tc_desc(bm), idesc, 1u);
                        if (PARTS > 1) tc_mma(tmem, tc_desc(am), tc_desc(bh), idesc, 1u);
                    }
                }
                asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(
                                 smem_u32(&bar_m))
                             : "memory");
            }
            // 4. meanwhile: the next step's query values, this step's candidate norms
            if (k + 1 < nsteps) load_q(k + 1);
            if (row < nt && mycols > 0) {
                const float* ar = abuf + (k & 1) * ACH * kChunkF + chunk_off(row, 0);
#pragma unroll
                for (int bb = 0; bb < NBLK; ++bb) {
                    if (bb < nbk) {
                        const float* ch = ar + (bb * PARTS) * kChunkF;
                        float4 h0 = *reinterpret_cast<const float4*>(ch), h1 = *reinterpret_cast<const float4*>(ch + 32);
                        if (PARTS > 1) {
                            const float4 m0 = *reinterpret_cast<const float4*>(ch + kChunkF);
                            const float4 m1v = *reinterpret_cast<const float4*>(ch + kChunkF + 32);
                            h0.x += m0.x; h0.y += m0.y; h0.z += m0.z; h0.w += m0.w;
                            h1.x += m1v.x; h1.y += m1v.y; h1.z += m1v.z; h1.w += m1v.w;
                        }
                        xn = fmaf(h0.x, h0.x, xn); xn = fmaf(h0.y, h0.y, xn);
                        xn = fmaf(h0.z, h0.z, xn); xn = fmaf(h0.w, h0.w, xn);
                        xn = fmaf(h1.x, h1.x, xn); xn = fmaf(h1.y, h1.y, xn);
                        xn = fmaf(h1.z, h1.z, xn); xn = fmaf(h1.w, h1.w, xn);
                    }
                }
            }
            const float xm = mk * xn, m2 = -2.f * mk;
            const unsigned dims_k = (unsigned)min((k + 1) * NBLK * kBlock, ix.D);
            // 5. the accumulator is complete (a warp whose wait gave up skips
            //    the tests; the CTA leaves together at the next barrier)
            const bool okm = warp_wait(&bar_m, ph_m, wv.status, lane);
            ph_m ^= 1u;
            if (!okm) {
                mma_failed = true;
                if (lane == 0) s_fail = 1;
            }
            tc_fence_after();
            // 6. the tests of every (candidate, query) pair of this warp's columns
#pragma unroll
            for (int c4 = 0; c4 < NW; ++c4) {
                if (okm && c4 * 32 < mycols) {
                    uint32_t v[32];
                    if (mycols - c4 * 32 >= 32) tmem_ld32(tmem_row + (uint32_t)(c4 * 32), v);
                    else tmem_ld16(tmem_row + (uint32_t)(c4 * 32), v);
                    asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
                    uint32_t newly = 0u;
                    if (alive[c4] && !fin_k) {
                        // the learned test: m1 dis' + beta - tau > 0
                        const float4* ap = reinterpret_cast<const float4*>(&s_a[k & 1][cb0 + c4 * 32]);
                        uint32_t prune = 0u;
#pragma unroll
                        for (int j4 = 0; j4 < 8; ++j4) {
                            if (c4 * 32 + j4 * 4 >= myq) break;  // the group's columns only
                            const float4 a4 = ap[j4];
                            const float av[4] = {a4.x, a4.y, a4.z, a4.w};
#pragma unroll
                            for (int i = 0; i < 4; ++i) {
                                const int j = j4 * 4 + i;
                                const float tv = fmaf(m2, __uint_as_float(v[j]), xm + av[i]);
                                prune |= (tv > 0.f ? 1u : 0u) << j;
                            }
                        }
                        newly = alive[c4] & prune;
                        alive[c4] &= ~prune;
                    } else if (FIN && alive[c4]) {
                        // the test on the completed rotated distance
                        const float4* ap = reinterpret_cast<const float4*>(&s_a[k & 1][cb0 + c4 * 32]);
                        const float4* rp = reinterpret_cast<const float4*>(&s_rt[cb0 + c4 * 32]);
                        uint32_t prune = 0u;
#pragma unroll
                        for (int j4 = 0; j4 < 8; ++j4) {
                            if (c4 * 32 + j4 * 4 >= myq) break;
                            const float4 a4 = ap[j4], r4 = rp[j4];
                            const float av[4] = {a4.x, a4.y, a4.z, a4.w}, rv[4] = {r4.x, r4.y, r4.z, r4.w};
#pragma unroll
                            for (int i = 0; i < 4; ++i) {
                                const int j = j4 * 4 + i;
                                const float r = rv[i] + ex;
                                const float dis = fmaf(-2.f, __uint_as_float(v[j]), xn + av[i]);
                                prune |= (dis > r * r * (1.f + kFinalRel) ? 1u : 0u) << j;
                            }
                        }
                        newly = alive[c4] & prune;
                        alive[c4] &= ~prune;
                    }
                    if (want_stats) {
                        for (int j = 0; j < 32; ++j) {
                            const int np = __popc(__ballot_sync(0xffffffffu, (newly >> j) & 1u));
                            if (lane == 0 && np) {
                                atomicAdd(&s_st[(cb0 + c4 * 32 + j) * 4 + 1], (unsigned)np);
                                atomicAdd(&s_st[(cb0 + c4 * 32 + j) * 4 + 3], (unsigned)np * dims_k);
                            }
                        }
                    }
                }
            }
            tc_fence_before();
        }
        // No copy is in flight here: the copy of step k + 1 is issued only
        // after the barrier of step k has let the step run.  MMAs whose wait
        // gave up get one more bounded wait before the CTA stops.
        if (mma_failed) warp_wait(&bar_m, ph_m ^ 1u, nullptr, lane);
        __syncthreads();
        if (s_fail) break;
        // 7. survivors: the exact distance from the original vector, one lane
        //    each, listed per warp (the query buffer is free now)
        uint16_t* list = reinterpret_cast<uint16_t*>(bbuf) + warp * 1024;
        unsigned long long ex_bytes = 0;
#pragma unroll
        for (int c4 = 0; c4 < NW; ++c4) {
            if (c4 * 32 >= mycols) continue;
            uint32_t bits = alive[c4];
            const int cnt = __popc(bits);
            int incl = cnt;
#pragma unroll
            for (int o = 1; o < 32; o <<= 1) {
                const int y = __shfl_up_sync(0xffffffffu, incl, o);
                if (lane >= o) incl += y;
            }
            const int tot = __shfl_sync(0xffffffffu, incl, 31);
            if (tot == 0) continue;
            int pos = incl - cnt;
            while (bits) {
                const int j = __ffs(bits) - 1;
                bits &= bits - 1u;
                list[pos++] = (uint16_t)(((cb0 + c4 * 32 + j) << 7) | row);
            }
            __syncwarp();
            for (int b = 0; b < tot; b += 32) {
                const int i = b + lane;
                const bool valid = i < tot;
                const int key = valid ? list[i] : 0;
                const int g = key >> 7, c = key & 127;
                const int q = s_q[g];
                float d = 0.f;
                if (valid)
                    d = exact_distance8(ix.orig + slot_l * ix.Dpad + ((int64_t)t * kTcRows + c) * kBlock, npad,
                                        wv.qpad + (int64_t)q * ix.Dpad, nb);
                append_any(wv, w, q, valid && d <= s_tau[g], d, slot0 + c, lane);
                if (want_stats && valid) {
                    atomicAdd(&s_st[g * 4 + 2], 1u);
                    atomicAdd(&s_st[g * 4 + 3], (unsigned)ix.D);
                }
            }
            ex_bytes += (unsigned long long)tot * ix.Dpad * sizeof(float);
            __syncwarp();
        }
        if (wv.staged_bytes && lane == 0 && ex_bytes) atomicAdd(wv.staged_bytes, ex_bytes);
        __syncthreads();
        if (want_stats)
            for (int i = tid; i < nq * 4; i += QW)
                if (s_st[i])
                    atomicAdd((unsigned long long*)&wv.stats[(int64_t)s_q[i >> 2] * 4 + (i & 3)],
                              (unsigned long long)s_st[i]);
        __syncthreads();
    }
    tc_fence_before();
    __syncthreads();
    if (warp == 0) {
        tc_fence_after();
        asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(QW) : "memory");
    }
}

template <int NBLK, int PARTS, bool FIN>
cudaError_t launch_tc_t(const IndexView& ix, const WaveView& wv, int w, const float* m1, const float* beta,
                        int nsteps, cudaStream_t st) {
    constexpr int QW = tc_qw<NBLK>();
    static int grid = 0, smem = 0;
    auto kern = tc_scan_kernel<NBLK, PARTS, QW, FIN>;
    if (grid == 0) {
        int dev = 0, sms = 0, per = 0;
        cudaError_t e = cudaGetDevice(&dev);
        if (e != cudaSuccess) return e;
        e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
        if (e != cudaSuccess) return e;
        // each CTA holds QW of the SM's 512 tensor-memory columns for its
        // whole life: request enough shared memory that at most 512 / QW
        // CTAs are resident on an SM, so that no allocation waits
        int bytes = tc_smem_bytes<NBLK, PARTS, QW>();
        for (;;) {
            e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, bytes);
            if (e != cudaSuccess) return e;
            e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per, kern, QW, bytes);
            if (e != cudaSuccess) return e;
            if (per <= 512 / QW) break;
            bytes += 8192;
        }
        smem = bytes;
        // the occupancy query can report fewer resident CTAs than registers and
        // shared memory allow (it does not know how much tensor memory a CTA
        // takes); the scan is persistent, so a launch of 512 / QW CTAs per SM
        // is safe either way: CTAs that are not resident start later and find
        // the work taken
        grid = sms * (512 / QW);
    }
    kern<<<grid, QW, smem, st>>>(ix, wv, w, m1, beta, nsteps);
    return cudaGetLastError();
}

}  // namespace

bool tc_scan_supported(int delta_d) { return delta_d == 8 || delta_d == 16 || delta_d == 32; }

int tc_scan_qmax(int delta_d) { return delta_d == 8 ? tc_qw<1>() : delta_d == 16 ? tc_qw<2>() : tc_qw<4>(); }

cudaError_t launch_wave_scan_tc(const IndexView& ix, const WaveView& wv, int w, int delta_d, const float* m1,
                                const float* beta, int nsteps, int parts, bool final_test, cudaStream_t st) {
#define DADE_TC_CASE(NB, PT)                                                                        \
    if (delta_d == NB * kBlock && parts == PT)                                                      \
        return final_test ? launch_tc_t<NB, PT, true>(ix, wv, w, m1, beta, nsteps, st)             \
                          : launch_tc_t<NB, PT, false>(ix, wv, w, m1, beta, nsteps, st);
    DADE_TC_CASE(1, 1)
    DADE_TC_CASE(2, 1)
    DADE_TC_CASE(4, 1)
    DADE_TC_CASE(1, 2)
    DADE_TC_CASE(2, 2)
    DADE_TC_CASE(4, 2)
#undef DADE_TC_CASE
    return cudaErrorInvalidValue;
}

}  // namespace dade
