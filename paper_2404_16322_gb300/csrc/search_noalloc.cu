// dade_search_noalloc: dade_search with its scratch in a fixed device array.
//
// Some callers cannot allocate device memory when they search: an embedding
// application whose allocator has already reserved all of the GPU's memory,
// or a latency-critical path that cannot afford the implicit synchronisation
// of cudaMalloc.  This entry point runs the same kernels as dade_search but
// takes its workspace from the file-scope array below, so a call performs no
// cudaMalloc, cudaFree or other allocation.
#include <map>
#include <mutex>

#include "dade_internal.h"

namespace {

// 64 MiB of scratch, held by every GPU that loads the library until the
// process exits.  It fits, for example, 256 queries of K 100 and nprobe 64
// on a 1M-vector index with 4096 buckets.
constexpr size_t kNoAllocBytes = size_t(64) << 20;
__device__ __align__(256) unsigned char g_noalloc_scratch[kNoAllocBytes];

// Device address of the array, looked up once per device and kept for the
// life of the process (so not valid across a cudaDeviceReset of that
// device).  In host code the array's name is only a host-side stand-in,
// never a device address.
std::mutex g_mu;
std::map<int, void*> g_addr;

dade_status scratch_address(void** out) {
    int dev = 0;
    DADE_CUDA_TRY(cudaGetDevice(&dev));
    std::lock_guard<std::mutex> lk(g_mu);
    auto it = g_addr.find(dev);
    if (it == g_addr.end()) {
        void* p = nullptr;
        DADE_CUDA_TRY(cudaGetSymbolAddress(&p, g_noalloc_scratch));
        it = g_addr.emplace(dev, p).first;
    }
    *out = it->second;
    return DADE_OK;
}

}  // namespace

extern "C" dade_status dade_search_noalloc(const dade_index* idx, const float* Q_dev, int64_t B,
                                           const int32_t* K_dev, const int32_t* nprobe_dev,
                                           int32_t delta_d, const dade_search_opts* opts,
                                           int64_t* ids_dev, float* dists_dev,
                                           const int64_t* out_offsets_dev, void* cuda_stream) {
    dade::clear_error();
    if (!opts) return dade::fail(DADE_EINVAL, "opts is required (max_K, max_nprobe)");
    if (opts->workspace)
        return dade::fail(DADE_EINVAL, "dade_search_noalloc uses its own fixed scratch; opts->workspace must be NULL");
    dade_search_opts o = *opts;
    DADE_TRY(dade::check_args(idx, B, delta_d, o));  // the same status and message as dade_search
    const size_t need = dade::workspace_bytes(idx, B, delta_d, o, nullptr);
    if (need > kNoAllocBytes)
        return dade::fail(DADE_EINVAL,
                          "this search needs %zu bytes of scratch but dade_search_noalloc holds %zu; "
                          "use fewer queries per call or dade_search",
                          need, kNoAllocBytes);
    void* scratch = nullptr;
    DADE_TRY(scratch_address(&scratch));
    o.workspace = scratch;
    o.workspace_bytes = kNoAllocBytes;
    return dade::search_impl(idx, Q_dev, B, K_dev, nprobe_dev, delta_d, o, ids_dev, dists_dev,
                             out_offsets_dev, static_cast<cudaStream_t>(cuda_stream), nullptr);
}
