// arena.cpp -- first-fit sub-allocator over one device memory budget.
//
// The serving loop owns one large device buffer (the HBM budget) and carves
// request buffers out of it; the arena only does the bookkeeping of byte
// offsets, so it never calls CUDA.  Free blocks are kept in an ordered map
// (offset -> size); allocation takes the first block that fits (aligned),
// freeing merges a block with its free neighbours.  All calls are serialised
// by one mutex.
#include <iterator>
#include <map>
#include <mutex>
#include <new>

#include "pencil.h"

struct pencil_arena {
    size_t capacity = 0;
    size_t align = 256;
    size_t free_bytes = 0;
    std::map<size_t, size_t> free_blocks;  // offset -> size
    std::map<size_t, size_t> used;         // offset -> size
    std::mutex mu;
};

namespace {

size_t round_up(size_t x, size_t a) { return (x + a - 1) / a * a; }

}  // namespace

extern "C" {

int pencil_arena_create(size_t capacity, size_t align, pencil_arena **out) {
    if (!out) return PENCIL_ERR_NULL;
    *out = nullptr;
    if (capacity == 0 || align == 0 || (align & (align - 1)) != 0) return PENCIL_ERR_ARG;
    pencil_arena *a = new (std::nothrow) pencil_arena;
    if (!a) return PENCIL_ERR_NOMEM;
    a->align = align;
    a->capacity = capacity / align * align;
    if (a->capacity == 0) {
        delete a;
        return PENCIL_ERR_ARG;
    }
    a->free_bytes = a->capacity;
    a->free_blocks[0] = a->capacity;
    *out = a;
    return PENCIL_OK;
}

int pencil_arena_alloc(pencil_arena *a, size_t bytes, size_t *offset) {
    if (!a || !offset) return PENCIL_ERR_NULL;
    if (bytes == 0) return PENCIL_ERR_ARG;
    const size_t need = round_up(bytes, a->align);
    if (need < bytes) return PENCIL_ERR_NOMEM;
    std::lock_guard<std::mutex> lk(a->mu);
    for (auto it = a->free_blocks.begin(); it != a->free_blocks.end(); ++it) {
        if (it->second < need) continue;
        const size_t off = it->first, size = it->second;
        a->free_blocks.erase(it);
        if (size > need) a->free_blocks[off + need] = size - need;
        a->used[off] = need;
        a->free_bytes -= need;
        *offset = off;
        return PENCIL_OK;
    }
    return PENCIL_ERR_NOMEM;
}

int pencil_arena_free(pencil_arena *a, size_t offset) {
    if (!a) return PENCIL_ERR_NULL;
    std::lock_guard<std::mutex> lk(a->mu);
    auto u = a->used.find(offset);
    if (u == a->used.end()) return PENCIL_ERR_ARG;
    size_t off = u->first, size = u->second;
    a->used.erase(u);
    a->free_bytes += size;
    auto next = a->free_blocks.lower_bound(off);
    if (next != a->free_blocks.end() && off + size == next->first) {
        size += next->second;
        next = a->free_blocks.erase(next);
    }
    if (next != a->free_blocks.begin()) {
        auto prev = std::prev(next);
        if (prev->first + prev->second == off) {
            prev->second += size;
            return PENCIL_OK;
        }
    }
    a->free_blocks[off] = size;
    return PENCIL_OK;
}

size_t pencil_arena_free_bytes(pencil_arena *a) {
    if (!a) return 0;
    std::lock_guard<std::mutex> lk(a->mu);
    return a->free_bytes;
}

size_t pencil_arena_largest_free(pencil_arena *a) {
    if (!a) return 0;
    std::lock_guard<std::mutex> lk(a->mu);
    size_t m = 0;
    for (const auto &b : a->free_blocks) m = b.second > m ? b.second : m;
    return m;
}

void pencil_arena_destroy(pencil_arena *a) { delete a; }

}  // extern "C"
