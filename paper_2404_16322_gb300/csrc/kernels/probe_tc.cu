// The centroid distances of the IVF probe step on the tensor cores
// (Section II-A: ||q'||^2 + ||c||^2 - 2 q'.c, clamped at 0, for every query
// and centroid), written as the B x nlist score matrix that the top-nprobe
// selection reads.
//
// Operands: the rotated queries and the centroids are split once into TF32
// parts (hi + mid, round to nearest) and laid out as canonical K-major
// chunks (128 rows x 8 dims, 4 KB per part): the centroids at index build,
// the queries per search (split_tc_kernel).  The 128 x 128 (queries x
// centroids) tiles, query-tile major, are dealt to the CTAs in contiguous
// ranges of equal length (so a CTA meets at most a few query tiles):
//  - warp 4, one lane: the producer.  It copies the CTA's current query
//    tile (all its chunks, both parts: at most 128 KB for Dpad <= 128) into
//    shared memory once, and streams the centroid chunks, two per copy,
//    through kPStages stages with cp.async.bulk (mbarrier "full",
//    expect_tx), up to kPStages - 2 stages ahead; per chunk it issues the
//    three products hi.hi + hi.mid + mid.hi (tcgen05.mma kind::tf32,
//    M = 128 queries, N = 128 centroids, K = 8) into one of two
//    tensor-memory accumulators; tcgen05.commit frees the stage ("empty")
//    and, after a tile's last chunk, hands the accumulator to the epilogue
//    ("acc full").  Its cursors advance by counting (no integer division in
//    the loop: a 64-bit division per chunk cost more than the chunk's MMAs);
//  - warps 0-3: the epilogue.  Thread t of warp w reads accumulator lane
//    (query) 32 w + t (tcgen05.ld), forms its distances and stores them as
//    float4 runs of its query's row, and the tile's 4 smallest of them (for
//    the selection's threshold); then the warp releases the accumulator
//    ("acc empty"), so the producer's next tile overlaps the stores.
// Every wait is bounded (about 2 s, then DADE_ETIMEOUT, and the CTA's loops
// stop; the MMAs issued are drained before the tensor memory is freed).
#include "tc_common.cuh"

namespace dade {
namespace {

constexpr int kPSC = 2;                          // chunks per centroid-operand stage
constexpr int kPStages = 4;                      // centroid-operand stages (kPSC chunks each)
constexpr int kPEpiWarps = 4;                    // epilogue warps (32 accumulator lanes each)
constexpr int kPThreads = (kPEpiWarps + 1) * 32; // + the producer warp
constexpr uint32_t kPChunk2 = 2 * 4096;          // one chunk, both parts (hi, mid)
constexpr int kPMaxChunks = 16;                  // Dpad <= 128: the resident query tile
constexpr int kPSmem = (kPMaxChunks + kPStages * kPSC) * kPChunk2 + 1024;

struct DistArgs {
    const float* qtc;      // query tiles: [qtile][chunk][part 2][1024]
    const float* ctc;      // centroid tiles: [ctile][chunk][part 2][1024]
    const float* qn;       // B: ||q'||^2
    const float* cn;       // nlist: ||c||^2
    int64_t B;
    int nlist, nchunks, nqtile, nctile;
    float* scores;         // B x nlist
    float* tmin;           // B x nctile x 4: each tile's 4 smallest distances per query (or null)
    int32_t* status;
};

__device__ __forceinline__ void tc_commit(uint64_t* bar) {
    asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(smem_u32(bar))
                 : "memory");
}

__global__ void __launch_bounds__(kPThreads, 1) centroid_dist_kernel(DistArgs a) {
    extern __shared__ __align__(1024) unsigned char psm[];
    __shared__ __align__(8) uint64_t full[kPStages], empty[kPStages], accf[2], acce[2], qfull, qfree, drain;
    __shared__ uint32_t s_taddr;
    __shared__ int s_abort;
    __shared__ __align__(16) float s_cn[kPEpiWarps][128];
    volatile int* abort_flag = &s_abort;
    unsigned char* base = reinterpret_cast<unsigned char*>((reinterpret_cast<uintptr_t>(psm) + 1023) & ~uintptr_t(1023));
    float* qres = reinterpret_cast<float*>(base);                              // resident query tile
    float* stages = reinterpret_cast<float*>(base + kPMaxChunks * kPChunk2);  // kPStages x kPSC chunks
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    // this CTA's tiles: [t0, t1) of the nqtile * nctile tiles, query-tile major
    const int64_t T = (int64_t)a.nqtile * a.nctile;
    const int64_t t0 = T * blockIdx.x / gridDim.x, t1 = T * (blockIdx.x + 1) / gridDim.x;

    if (warp == 0) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(&s_taddr)),
                     "r"(256)
                     : "memory");
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
    }
    if (tid == 0) {
        for (int i = 0; i < kPStages; ++i) {
            mbar_init(&full[i], 1);
            mbar_init(&empty[i], 1);
        }
        for (int i = 0; i < 2; ++i) {
            mbar_init(&accf[i], 1);
            mbar_init(&acce[i], kPEpiWarps);
        }
        mbar_init(&qfull, 1);
        mbar_init(&qfree, 1);
        mbar_init(&drain, 1);
        fence_mbar_init();
        s_abort = 0;
    }
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    const uint32_t tmem = s_taddr;

    if (warp == kPEpiWarps) {
        // ------------------------------------------------------ producer
        if (lane == 0 && t1 > t0) {
            const int spt = (a.nchunks + kPSC - 1) / kPSC;  // stages per tile
            int c_ct = (int)(t0 % a.nctile), c_s = 0;       // copy cursor: centroid tile, stage
            int64_t c_left = t1 - t0;                       // tiles the copy cursor has not finished
            int m_ct = c_ct, m_qt = (int)(t0 / a.nctile), m_s = 0;  // MMA cursor
            int64_t m_left = t1 - t0;
            uint32_t ncopy = 0, nmma = 0, lt = 0, nq = 0;
            int cur_qt = -1;
            const uint32_t idesc = tc_idesc(128);
            bool ok = true;
            while (m_left > 0 && !*abort_flag) {
                if (m_s == 0 && m_qt != cur_qt) {
                    // a new query tile, once the MMAs on the previous one are done
                    if (nq > 0) {
                        tc_commit(&qfree);
                        ok = mbar_wait_spin(&qfree, (nq - 1) & 1u, a.status);
                        if (!ok) break;
                    }
                    cur_qt = m_qt;
                    const uint32_t qbytes = (uint32_t)a.nchunks * kPChunk2;
                    mbar_expect_tx(&qfull, qbytes);
                    bulk_g2s(qres, a.qtc + (int64_t)cur_qt * a.nchunks * 2 * kChunkF, qbytes, &qfull);
                    ++nq;
                }
                // centroid stages up to kPStages - 2 ahead of the MMAs: the slot
                // of copy n is free once the MMAs of stage n - kPStages are done
                while (c_left > 0 && ncopy <= nmma + kPStages - 2) {
                    const int slot = (int)(ncopy % kPStages);
                    if (ncopy >= kPStages) ok = mbar_wait_spin(&empty[slot], ((ncopy / kPStages) - 1) & 1u, a.status);
                    if (!ok) break;
                    const int k0 = c_s * kPSC, nk = min(kPSC, a.nchunks - k0);
                    const uint32_t bytes = (uint32_t)nk * kPChunk2;
                    mbar_expect_tx(&full[slot], bytes);
                    bulk_g2s(stages + (size_t)slot * kPSC * (kPChunk2 / 4),
                             a.ctc + ((int64_t)c_ct * a.nchunks + k0) * 2 * kChunkF, bytes, &full[slot]);
                    ++ncopy;
                    if (++c_s == spt) {
                        c_s = 0;
                        --c_left;
                        if (++c_ct == a.nctile) c_ct = 0;
                    }
                }
                if (!ok) break;
                const int ab = (int)(lt & 1);
                if (m_s == 0 && lt >= 2)  // the epilogue has read this accumulator's previous tile
                    ok = mbar_wait_spin(&acce[ab], ((lt >> 1) - 1) & 1u, a.status);
                if (ok && m_s == 0) ok = mbar_wait_spin(&qfull, (nq - 1) & 1u, a.status);
                const int slot = (int)(nmma % kPStages);
                if (ok) ok = mbar_wait_spin(&full[slot], (nmma / kPStages) & 1u, a.status);
                if (!ok) break;
                tc_fence_after();
                const int k0 = m_s * kPSC, nk = min(kPSC, a.nchunks - k0);
                const uint32_t acc = tmem + (uint32_t)(ab * 128);
                const uint32_t qa = smem_u32(qres) + (uint32_t)k0 * kPChunk2;
                const uint32_t ca = smem_u32(stages) + (uint32_t)slot * kPSC * kPChunk2;
                for (int k = 0; k < nk; ++k) {
                    const uint32_t qh = qa + (uint32_t)k * kPChunk2, qm = qh + 4096u;
                    const uint32_t ch = ca + (uint32_t)k * kPChunk2, cm = ch + 4096u;
                    tc_mma(acc, tc_desc(qh), tc_desc(ch), idesc, (k0 + k) > 0 ? 1u : 0u);
                    tc_mma(acc, tc_desc(qh), tc_desc(cm), idesc, 1u);
                    tc_mma(acc, tc_desc(qm), tc_desc(ch), idesc, 1u);
                }
                tc_commit(&empty[slot]);
                ++nmma;
                if (++m_s == spt) {
                    tc_commit(&accf[ab]);
                    m_s = 0;
                    ++lt;
                    --m_left;
                    if (++m_ct == a.nctile) {
                        m_ct = 0;
                        ++m_qt;
                    }
                }
            }
            if (!ok) *abort_flag = 1;
            // every MMA issued has completed before the accumulators are freed
            tc_commit(&drain);
            mbar_wait_spin(&drain, 0u, a.status);
        }
    } else {
        // ------------------------------------------------------ epilogue
        const uint32_t trow = tmem + ((uint32_t)(warp * 32) << 16);
        float* cnw = s_cn[warp];
        const bool vec = (a.nlist & 3) == 0;
        uint32_t lt = 0;
        int ct = (int)(t0 % a.nctile);
        int64_t qbase = (t0 / a.nctile) * 128;
        for (int64_t tile = t0; tile < t1; ++tile, ++lt) {
            const int ab = (int)(lt & 1);
            const int c0 = ct * 128;
            const int64_t q = qbase + warp * 32 + lane;
            {  // this tile's centroid norms, a warp-private copy
                const int cc = c0 + lane * 4;
                float4 v4;
                v4.x = cc < a.nlist ? __ldg(a.cn + cc) : 0.f;
                v4.y = cc + 1 < a.nlist ? __ldg(a.cn + cc + 1) : 0.f;
                v4.z = cc + 2 < a.nlist ? __ldg(a.cn + cc + 2) : 0.f;
                v4.w = cc + 3 < a.nlist ? __ldg(a.cn + cc + 3) : 0.f;
                *reinterpret_cast<float4*>(cnw + lane * 4) = v4;
            }
            const float qnq = q < a.B ? a.qn[q] : 0.f;
            const bool ok = !*abort_flag && warp_wait_spin(&accf[ab], (lt >> 1) & 1u, a.status, lane);
            if (!ok) {
                if (lane == 0) *abort_flag = 1;
                break;  // warp-uniform; no barrier among the epilogue warps follows
            }
            tc_fence_after();
            __syncwarp();
            float* row = a.scores + q * (int64_t)a.nlist;
            // the tile's 4 smallest distances of this query, ascending
            float r0 = INFINITY, r1 = INFINITY, r2 = INFINITY, r3 = INFINITY;
            auto keep4 = [&](float x) {
                float t = fminf(r0, x);
                x = fmaxf(r0, x);
                r0 = t;
                t = fminf(r1, x);
                x = fmaxf(r1, x);
                r1 = t;
                t = fminf(r2, x);
                x = fmaxf(r2, x);
                r2 = t;
                r3 = fminf(r3, x);
            };
#pragma unroll 1
            for (int j0 = 0; j0 < 128; j0 += 32) {
                uint32_t v[32];
                tmem_ld32(trow + (uint32_t)(ab * 128 + j0), v);
                asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
                if (q >= a.B) continue;
                const int cb = c0 + j0;
                if (vec && cb + 32 <= a.nlist) {
#pragma unroll
                    for (int j = 0; j < 32; j += 4) {
                        const float4 cv = *reinterpret_cast<const float4*>(cnw + j0 + j);
                        float4 o;
                        o.x = fmaxf(0.f, qnq + cv.x - 2.f * __uint_as_float(v[j]));
                        o.y = fmaxf(0.f, qnq + cv.y - 2.f * __uint_as_float(v[j + 1]));
                        o.z = fmaxf(0.f, qnq + cv.z - 2.f * __uint_as_float(v[j + 2]));
                        o.w = fmaxf(0.f, qnq + cv.w - 2.f * __uint_as_float(v[j + 3]));
                        *reinterpret_cast<float4*>(row + cb + j) = o;
                        keep4(o.x);
                        keep4(o.y);
                        keep4(o.z);
                        keep4(o.w);
                    }
                } else {
#pragma unroll
                    for (int j = 0; j < 32; ++j)
                        if (cb + j < a.nlist) {
                            const float o = fmaxf(0.f, qnq + cnw[j0 + j] - 2.f * __uint_as_float(v[j]));
                            row[cb + j] = o;
                            keep4(o);
                        }
                }
            }
            if (a.tmin && q < a.B)
                *reinterpret_cast<float4*>(a.tmin + (q * a.nctile + ct) * 4) = make_float4(r0, r1, r2, r3);
            tc_fence_before();
            __syncwarp();
            if (lane == 0) mbar_arrive(&acce[ab]);
            if (++ct == a.nctile) {
                ct = 0;
                qbase += 128;
            }
        }
    }
    tc_fence_before();
    __syncthreads();
    if (warp == 0) {
        tc_fence_after();
        asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(256) : "memory");
    }
}

// The canonical chunks of the TF32 parts (hi, mid) of rows [0, nrows) of a
// row-major FP32 matrix (ld floats per row, the first nchunks * 8 columns),
// zero beyond nrows: out[tile][chunk][part][1024].
__global__ void split_tc_kernel(const float* __restrict__ X, int64_t ld, int64_t nrows, int nchunks, int64_t total,
                                float* __restrict__ out) {
    const int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;  // one element of one chunk
    if (e >= total) return;
    const int64_t tc = e >> 10;  // (tile, chunk)
    const int in = (int)(e & 1023), r = in >> 3, j = in & 7;
    const int64_t tile = tc / nchunks;
    const int c = (int)(tc % nchunks);
    const int64_t row = tile * 128 + r;
    const float v = row < nrows ? X[row * ld + c * 8 + j] : 0.f;
    const float h = tf32_rna(v);
    const float m = tf32_rna(v - h);
    float* o = out + tc * 2 * kChunkF + chunk_off(r, j);
    o[0] = h;
    o[kChunkF] = m;
}

}  // namespace

bool centroid_tc_supported(int Dpad) { return Dpad % 8 == 0 && Dpad / 8 <= kPMaxChunks; }

cudaError_t launch_split_tc(const float* X, int64_t ld, int64_t nrows, int Dpad, float* out, cudaStream_t st) {
    const int nchunks = Dpad / 8;
    const int64_t total = ceil_div(nrows, 128) * nchunks * 1024;
    if (total == 0) return cudaSuccess;
    split_tc_kernel<<<(unsigned)ceil_div(total, 256), 256, 0, st>>>(X, ld, nrows, nchunks, total, out);
    return cudaGetLastError();
}

cudaError_t launch_centroid_dist_tc(const float* qtc, const float* ctc, const float* qn, const float* cn, int64_t B,
                                    int nlist, int Dpad, float* scores, float* tmin, int32_t* status,
                                    cudaStream_t st) {
    if (B == 0 || nlist == 0) return cudaSuccess;
    static int sms = 0;
    if (sms == 0) {
        int dev = 0, n = 0;
        cudaError_t e = cudaGetDevice(&dev);
        if (e == cudaSuccess) e = cudaDeviceGetAttribute(&n, cudaDevAttrMultiProcessorCount, dev);
        if (e == cudaSuccess)
            e = cudaFuncSetAttribute(centroid_dist_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, kPSmem);
        if (e != cudaSuccess) return e;
        sms = n;
    }
    DistArgs a;
    a.qtc = qtc;
    a.ctc = ctc;
    a.qn = qn;
    a.cn = cn;
    a.B = B;
    a.nlist = nlist;
    a.nchunks = Dpad / 8;
    a.nqtile = (int)ceil_div(B, 128);
    a.nctile = (int)ceil_div(nlist, 128);
    a.scores = scores;
    a.tmin = tmin;
    a.status = status;
    const int64_t tiles = (int64_t)a.nqtile * a.nctile;
    const unsigned grid = (unsigned)std::min<int64_t>(tiles, sms);
    centroid_dist_kernel<<<grid, kPThreads, kPSmem, st>>>(a);
    return cudaGetLastError();
}

}  // namespace dade
