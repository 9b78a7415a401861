// Host bookkeeping of one device memory arena for the serving loop's
// admission control: first-fit allocation of aligned byte ranges of
// [0, size), coalescing on free.  The device memory itself belongs to the
// caller (one allocation); the arena only hands out offsets into it, so a
// batch is admitted exactly when a free range holds its workspace.
#include <stdint.h>

#include <iterator>
#include <map>
#include <mutex>
#include <new>

#include "dade.h"

struct dade_arena {
    int64_t size = 0, align = 256, used = 0;
    std::map<int64_t, int64_t> free_;  // offset -> length of each free range (disjoint, not adjacent)
    std::map<int64_t, int64_t> live;   // offset -> length of each allocation
    mutable std::mutex mu;
};

namespace {

int64_t round_up(int64_t x, int64_t a) { return (x + a - 1) / a * a; }

}  // namespace

extern "C" dade_status dade_arena_create(int64_t bytes, int64_t align, dade_arena** out) {
    if (!out || bytes < 0 || align < 1 || (align & (align - 1)) != 0) return DADE_EINVAL;
    dade_arena* a = new (std::nothrow) dade_arena;
    if (!a) return DADE_ENOMEM;
    a->size = bytes / align * align;
    a->align = align;
    if (a->size > 0) a->free_[0] = a->size;
    *out = a;
    return DADE_OK;
}

extern "C" int64_t dade_arena_alloc(dade_arena* a, int64_t bytes) {
    if (!a || bytes < 0) return -1;
    std::lock_guard<std::mutex> lk(a->mu);
    const int64_t need = round_up(bytes > 0 ? bytes : 1, a->align);
    for (auto it = a->free_.begin(); it != a->free_.end(); ++it) {
        if (it->second < need) continue;
        const int64_t off = it->first, len = it->second;
        a->free_.erase(it);
        if (len > need) a->free_[off + need] = len - need;
        a->live[off] = need;
        a->used += need;
        return off;
    }
    return -1;
}

extern "C" dade_status dade_arena_free(dade_arena* a, int64_t offset) {
    if (!a) return DADE_EINVAL;
    std::lock_guard<std::mutex> lk(a->mu);
    auto it = a->live.find(offset);
    if (it == a->live.end()) return DADE_EINVAL;
    int64_t off = it->first, len = it->second;
    a->live.erase(it);
    a->used -= len;
    // merge with the free neighbours on both sides
    auto nx = a->free_.lower_bound(off);
    if (nx != a->free_.end() && off + len == nx->first) {
        len += nx->second;
        nx = a->free_.erase(nx);
    }
    if (nx != a->free_.begin()) {
        auto pv = std::prev(nx);
        if (pv->first + pv->second == off) {
            pv->second += len;
            return DADE_OK;
        }
    }
    a->free_[off] = len;
    return DADE_OK;
}

extern "C" int64_t dade_arena_used(const dade_arena* a) {
    if (!a) return -1;
    std::lock_guard<std::mutex> lk(a->mu);
    return a->used;
}

extern "C" int64_t dade_arena_largest_free(const dade_arena* a) {
    if (!a) return -1;
    std::lock_guard<std::mutex> lk(a->mu);
    int64_t m = 0;
    for (const auto& f : a->free_) m = f.second > m ? f.second : m;
    return m;
}

extern "C" void dade_arena_destroy(dade_arena* a) { delete a; }
