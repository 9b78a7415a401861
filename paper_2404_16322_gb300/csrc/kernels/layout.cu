// Bucket layout of the index: rotated vectors in the slab precision and the
// original FP32 vectors, both dimension-blocked (8 dims per block, block b
// of a bucket's vector i at (b * npad + i) * 8), so that a Delta_d slab of a
// run of vectors is one contiguous range.  FP8-E4M3 uses a per-dimension
// scale amax_j / 448 (round to nearest even, saturating).
#include <cuda_bf16.h>
#include <cuda_fp8.h>

#include "../dade_internal.h"

namespace dade {
namespace {

__global__ void layout_kernel(LayoutArgs a) {
    const int nb = a.Dpad / kBlock;
    int64_t idx = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (idx >= a.total_slots * nb) return;
    int64_t slot = idx / nb;
    int b = (int)(idx % nb);
    int l = a.slot_list[slot];
    int64_t s0 = a.list_slot[l];
    int64_t npad = a.list_slot[l + 1] - s0;
    int64_t i = slot - s0;
    int64_t elem = s0 * a.Dpad + (b * npad + i) * kBlock;
    int64_t row = a.slot_row[slot];
#pragma unroll
    for (int j = 0; j < kBlock; ++j) {
        int d = b * kBlock + j;
        float xr = row >= 0 ? a.xrot[row * a.Dpad + d] : 0.f;
        float xo = (row >= 0 && d < a.D) ? a.x[row * a.D + d] : 0.f;
        a.orig[elem + j] = xo;
        if (a.dtype == DADE_SLAB_F32) {
            static_cast<float*>(a.slab)[elem + j] = xr;
        } else if (a.dtype == DADE_SLAB_BF16) {
            static_cast<__nv_bfloat16*>(a.slab)[elem + j] = __float2bfloat16_rn(xr);
        } else {
            float y = xr / a.scale[d];
            static_cast<__nv_fp8_storage_t*>(a.slab)[elem + j] =
                __nv_cvt_float_to_fp8(y, __NV_SATFINITE, __NV_E4M3);
        }
    }
}

// Quantisation error norm ||x' - x~|| of every slot's stored vector (one warp
// per slot, lanes over dimensions, fixed-order butterfly sum).
__global__ void quant_error_kernel(LayoutArgs a) {
    const int64_t slot = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const int lane = threadIdx.x & 31;
    if (slot >= a.total_slots) return;
    const int64_t row = a.slot_row[slot];
    float s = 0.f;
    if (row >= 0) {
        for (int d = lane; d < a.D; d += 32) {
            const float xr = a.xrot[row * a.Dpad + d];
            float xs;
            if (a.dtype == DADE_SLAB_BF16) {
                xs = __bfloat162float(__float2bfloat16_rn(xr));
            } else {
                const __nv_fp8_storage_t v = __nv_cvt_float_to_fp8(xr / a.scale[d], __NV_SATFINITE, __NV_E4M3);
                xs = __half2float(__half(__nv_cvt_fp8_to_halfraw(v, __NV_E4M3))) * a.scale[d];
            }
            const float e = xr - xs;
            s = fmaf(e, e, s);
        }
    }
    for (int off = 16; off; off >>= 1) s += __shfl_xor_sync(0xffffffffu, s, off);
    if (lane == 0) a.eps[slot] = sqrtf(s);
}

// Variance of each rotated dimension over the N rows (1/N; two passes in
// FP64, one block per dimension, fixed reduction order).
__global__ void dim_var_kernel(const float* __restrict__ xrot, int64_t N, int32_t Dpad, float* __restrict__ var) {
    __shared__ double red[256];
    const int d = blockIdx.x, tid = threadIdx.x;
    double s = 0.0;
    for (int64_t r = tid; r < N; r += 256) s += xrot[r * Dpad + d];
    red[tid] = s;
    __syncthreads();
    for (int h = 128; h; h >>= 1) {
        if (tid < h) red[tid] += red[tid + h];
        __syncthreads();
    }
    const double mean = red[0] / (double)(N > 0 ? N : 1);
    __syncthreads();
    s = 0.0;
    for (int64_t r = tid; r < N; r += 256) {
        const double t = xrot[r * Dpad + d] - mean;
        s += t * t;
    }
    red[tid] = s;
    __syncthreads();
    for (int h = 128; h; h >>= 1) {
        if (tid < h) red[tid] += red[tid + h];
        __syncthreads();
    }
    if (tid == 0) var[d] = (float)(red[0] / (double)(N > 0 ? N : 1));
}

// Residual norms of every slot's stored vector: sfx[b][slot] = sum over
// blocks b' >= b of ||x~_b'||^2 (dequantised, FP32, from the last block
// back), b = 0 .. nb; padding slots get 0.  The slot's bucket comes from a
// binary search of list_slot.
__global__ void residual_norms_kernel(const void* __restrict__ slab, int dtype, const float* __restrict__ scale,
                                      const int64_t* __restrict__ list_slot, int nlist, int64_t total_slots,
                                      int32_t Dpad, float* __restrict__ sfx) {
    const int64_t slot = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (slot >= total_slots) return;
    int lo = 0, hi = nlist - 1;
    while (lo < hi) {
        const int mid = (lo + hi + 1) >> 1;
        if (list_slot[mid] <= slot) lo = mid; else hi = mid - 1;
    }
    const int64_t s0 = list_slot[lo], npad = list_slot[lo + 1] - s0, i = slot - s0;
    const int nb = Dpad / kBlock;
    float acc = 0.f;
    sfx[(int64_t)nb * total_slots + slot] = 0.f;
    for (int b = nb - 1; b >= 0; --b) {
        const int64_t e = s0 * Dpad + ((int64_t)b * npad + i) * kBlock;
        float s = 0.f;
        for (int j = 0; j < kBlock; ++j) {
            float v;
            if (dtype == DADE_SLAB_F32) {
                v = static_cast<const float*>(slab)[e + j];
            } else if (dtype == DADE_SLAB_BF16) {
                v = __bfloat162float(static_cast<const __nv_bfloat16*>(slab)[e + j]);
            } else {
                const __nv_fp8_storage_t u = static_cast<const __nv_fp8_storage_t*>(slab)[e + j];
                v = __half2float(__half(__nv_cvt_fp8_to_halfraw(u, __NV_E4M3))) * scale[b * kBlock + j];
            }
            s = fmaf(v, v, s);
        }
        acc += s;
        sfx[(int64_t)b * total_slots + slot] = acc;
    }
}

__global__ void amax_kernel(const float* __restrict__ xrot, int64_t N, int32_t Dpad,
                            unsigned int* __restrict__ amax) {
    int d = blockIdx.y;
    float m = 0.f;
    for (int64_t r = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; r < N;
         r += (int64_t)gridDim.x * blockDim.x)
        m = fmaxf(m, fabsf(xrot[r * Dpad + d]));
    for (int off = 16; off; off >>= 1) m = fmaxf(m, __shfl_xor_sync(0xffffffffu, m, off));
    if ((threadIdx.x & 31) == 0) atomicMax(&amax[d], __float_as_uint(m));
}

__global__ void scale_kernel(float* v, int32_t Dpad) {
    int d = blockIdx.x * blockDim.x + threadIdx.x;
    if (d < Dpad) {
        float a = v[d];
        v[d] = a > 0.f ? a / 448.f : 1.f;
    }
}

// Stored rotated values of a set of slots, decoded to FP32 (row r: slot
// elements from base[r], blocks npad[r] * 8 apart).
__global__ void stored_gather_kernel(const void* slab, int dtype, const float* scale, const int64_t* base,
                                     const int64_t* npad, int64_t nrows, int32_t D, float* out) {
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= nrows * D) return;
    const int64_t r = i / D;
    const int d = (int)(i % D);
    const int64_t e = base[r] + ((int64_t)(d / kBlock) * npad[r]) * kBlock + d % kBlock;
    float v;
    if (dtype == DADE_SLAB_F32) {
        v = static_cast<const float*>(slab)[e];
    } else if (dtype == DADE_SLAB_BF16) {
        v = __bfloat162float(static_cast<const __nv_bfloat16*>(slab)[e]);
    } else {
        const __nv_fp8_storage_t c = static_cast<const __nv_fp8_storage_t*>(slab)[e];
        v = __half2float(__half(__nv_cvt_fp8_to_halfraw(c, __NV_E4M3))) * scale[d];
    }
    out[i] = v;
}

// The stored slabs as the tensor-core scan's operand: per tile of kTcRows
// candidates of a bucket and per 8-dim block, the TF32 parts of the stored
// values (hi = tf32(x~), mid = tf32(x~ - hi); only hi for BF16, which TF32
// holds exactly) in the canonical K-major layout without swizzle, each part
// one 4 KB chunk: element (row r, dim j) at float (r / 8) * 64 + (j / 4) * 32
// + (r % 8) * 4 + j % 4 (8-row x 16-byte core matrices; the two K halves 128
// bytes apart, 8-row groups 256 bytes apart).  Chunks ordered (tile, block,
// part), so a step's blocks are one contiguous range.
__global__ void tc_slab_kernel(const void* slab, int dtype, const float* scale, const int64_t* list_slot,
                               const int32_t* list_size, const int64_t* tile_base, int nlist, int32_t Dpad,
                               int parts, int64_t ntiles, float* out) {
    const int nb = Dpad / kBlock;
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= ntiles * nb * kTcRows) return;
    const int64_t T = i / ((int64_t)nb * kTcRows);
    const int b = (int)((i / kTcRows) % nb);
    const int r = (int)(i % kTcRows);
    int lo = 0, hi_ = nlist;  // bucket of tile T: tile_base[l] <= T < tile_base[l + 1]
    while (hi_ - lo > 1) {
        const int mid = (lo + hi_) >> 1;
        if (tile_base[mid] <= T) lo = mid; else hi_ = mid;
    }
    const int l = lo;
    const int64_t row = (T - tile_base[l]) * kTcRows + r;
    const int64_t s0 = list_slot[l];
    const int64_t npad = list_slot[l + 1] - s0;
    float* o = out + ((T * nb + b) * parts) * 1024 + (r >> 3) * 64 + (r & 7) * 4;
#pragma unroll
    for (int j = 0; j < kBlock; ++j) {
        float x = 0.f;
        if (row < list_size[l]) {
            const int64_t e = s0 * Dpad + ((int64_t)b * npad + row) * kBlock + j;
            if (dtype == DADE_SLAB_F32) {
                x = static_cast<const float*>(slab)[e];
            } else if (dtype == DADE_SLAB_BF16) {
                x = __bfloat162float(static_cast<const __nv_bfloat16*>(slab)[e]);
            } else {
                const __nv_fp8_storage_t c = static_cast<const __nv_fp8_storage_t*>(slab)[e];
                x = __half2float(__half(__nv_cvt_fp8_to_halfraw(c, __NV_E4M3))) * scale[b * kBlock + j];
            }
        }
        uint32_t h;
        asm("cvt.rna.tf32.f32 %0, %1;" : "=r"(h) : "f"(x));
        const int off = (j >> 2) * 32 + (j & 3);
        o[off] = __uint_as_float(h);
        if (parts > 1) {
            uint32_t m;
            asm("cvt.rna.tf32.f32 %0, %1;" : "=r"(m) : "f"(x - __uint_as_float(h)));
            o[1024 + off] = __uint_as_float(m);
        }
    }
}

}  // namespace

cudaError_t launch_tc_slab(const void* slab, int dtype, const float* scale, const int64_t* list_slot,
                           const int32_t* list_size, const int64_t* tile_base, int nlist, int32_t Dpad, int parts,
                           int64_t ntiles, float* out, cudaStream_t st) {
    const int64_t n = ntiles * (Dpad / kBlock) * kTcRows;
    if (n == 0) return cudaSuccess;
    tc_slab_kernel<<<(unsigned)ceil_div(n, 256), 256, 0, st>>>(slab, dtype, scale, list_slot, list_size, tile_base,
                                                               nlist, Dpad, parts, ntiles, out);
    return cudaGetLastError();
}

cudaError_t launch_stored_gather(const void* slab, int dtype, const float* scale, const int64_t* base,
                                 const int64_t* npad, int64_t nrows, int32_t D, float* out, cudaStream_t st) {
    const int64_t n = nrows * D;
    if (n == 0) return cudaSuccess;
    stored_gather_kernel<<<(unsigned)ceil_div(n, 256), 256, 0, st>>>(slab, dtype, scale, base, npad, nrows, D, out);
    return cudaGetLastError();
}

cudaError_t launch_layout(const LayoutArgs& a, cudaStream_t st) {
    int64_t n = a.total_slots * (a.Dpad / kBlock);
    if (n == 0) return cudaSuccess;
    layout_kernel<<<(unsigned)ceil_div(n, 256), 256, 0, st>>>(a);
    return cudaGetLastError();
}

cudaError_t launch_quant_error(const LayoutArgs& a, cudaStream_t st) {
    if (a.total_slots == 0 || a.dtype == DADE_SLAB_F32 || !a.eps) return cudaSuccess;
    quant_error_kernel<<<(unsigned)ceil_div(a.total_slots * 32, 256), 256, 0, st>>>(a);
    return cudaGetLastError();
}

cudaError_t launch_dim_var(const float* xrot, int64_t N, int32_t Dpad, float* var, cudaStream_t st) {
    dim_var_kernel<<<(unsigned)Dpad, 256, 0, st>>>(xrot, N, Dpad, var);
    return cudaGetLastError();
}

cudaError_t launch_residual_norms(const void* slab, int dtype, const float* scale, const int64_t* list_slot,
                                  int nlist, int64_t total_slots, int32_t Dpad, float* sfx, cudaStream_t st) {
    if (total_slots == 0) return cudaSuccess;
    residual_norms_kernel<<<(unsigned)ceil_div(total_slots, 128), 128, 0, st>>>(slab, dtype, scale, list_slot, nlist,
                                                                               total_slots, Dpad, sfx);
    return cudaGetLastError();
}

cudaError_t launch_amax(const float* xrot, int64_t N, int32_t Dpad, float* out, cudaStream_t st) {
    cudaError_t e = cudaMemsetAsync(out, 0, sizeof(float) * Dpad, st);
    if (e != cudaSuccess) return e;
    dim3 grid((unsigned)std::min<int64_t>(64, ceil_div(N, 256)), (unsigned)Dpad);
    amax_kernel<<<grid, 256, 0, st>>>(xrot, N, Dpad, reinterpret_cast<unsigned int*>(out));
    return cudaGetLastError();
}

cudaError_t launch_fp8_scale(float* v, int32_t Dpad, cudaStream_t st) {
    scale_kernel<<<(unsigned)ceil_div(Dpad, 128), 128, 0, st>>>(v, Dpad);
    return cudaGetLastError();
}

}  // namespace dade
