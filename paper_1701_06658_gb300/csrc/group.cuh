// Step groups on the device: the work items of several contexts in one
// launch.  A group kernel walks the concatenation of its members' lists of one
// kind; each CTA first takes the exclusive prefix of the members' item counts
// into shared memory, and each item then finds its member by a binary search
// over that prefix.
#pragma once

#include "lsgg_internal.cuh"

namespace lsgg {

// The lists a kernel walks: plane, column-chunk or slab items of a tier, the
// boxes, the domain tiles.
enum : int { kItemPlanes = 0, kItemChunks = 1, kItemSlabs = 2, kItemBoxes = 3, kItemTiles = 4, kItemBoxChunks = 5,
             kItemBoxChunksGo = 6 };

__device__ __forceinline__ int list_count(const StepBuffers& B, int list, int tier) {
    switch (list) {
        case kItemPlanes: return B.st->n_planes[tier];
        case kItemChunks: return B.st->n_chunks[tier];
        case kItemSlabs: return B.st->n_slabs[tier];
        case kItemBoxes: return B.n_boxes;
        case kItemBoxChunks: return (B.n_boxes + kBuChunk - 1) / kBuChunk;
        case kItemBoxChunksGo: return B.st->bu_go ? (B.n_boxes + kBuChunk - 1) / kBuChunk : 0;
        default: return B.n_tiles;
    }
}

// A member takes part in the group's step: not halted, and (with `limit`)
// below its step limit.  The box update's item writer ignores the limit, so
// that a member that reaches it keeps valid work items for later steps.
__device__ __forceinline__ bool group_live(const StepBuffers& B, bool limit) {
    return *(volatile int*)&B.st->halt == 0 && (!limit || B.st->steps_done < B.st->step_limit);
}

// Exclusive prefix s[0..n] of the live members' item counts, in shared memory
// (kMaxGroup + 1 entries); called by every thread (a barrier); returns the total.
__device__ inline int group_scan(const GroupRef& g, int list, int tier, bool limit, int* s) {
    if (threadIdx.x < 32) {
        const int l = threadIdx.x;
        int a = 0, b = 0;
        if (l < g.n && group_live(g.B[l], limit)) a = list_count(g.B[l], list, tier);
        if (l + 32 < g.n && group_live(g.B[l + 32], limit)) b = list_count(g.B[l + 32], list, tier);
#pragma unroll
        for (int d = 1; d < 32; d <<= 1) {
            const int x = __shfl_up_sync(0xffffffffu, a, d), y = __shfl_up_sync(0xffffffffu, b, d);
            if (l >= d) { a += x; b += y; }
        }
        const int ta = __shfl_sync(0xffffffffu, a, 31);
        s[l + 1] = a;
        s[l + 33] = ta + b;
        if (l == 0) s[0] = 0;
    }
    __syncthreads();
    return s[g.n];
}

// The member holding group item i (the largest k with s[k] <= i), its index
// in that member's list in `local`; without a group, the launch's own buffers.
template <bool GRP>
__device__ __forceinline__ const StepBuffers& member(const StepBuffers& B1, const GroupRef& g, const int* s, int i,
                                                     int& local) {
    if constexpr (GRP) {
        int lo = 0, hi = g.n;
        while (hi - lo > 1) {
            const int mid = (lo + hi) >> 1;
            if (s[mid] <= i) lo = mid; else hi = mid;
        }
        local = i - s[lo];
        return g.B[lo];
    } else {
        local = i;
        return B1;
    }
}

// Item `local` of a member's list (group), or entry i of the launch's list.
template <bool GRP>
__device__ __forceinline__ int2 list_item(const StepBuffers& B, const int2* items1, int list, int tier, int i,
                                          int local) {
    if constexpr (GRP) {
        if (list == kItemPlanes) return B.plane_items[B.st->plane_base[tier] + local];
        if (list == kItemChunks) return B.chunk_items[B.st->chunk_base[tier] + local];
        return B.slab_items[B.st->slab_base[tier] + local];
    } else {
        return items1[i];
    }
}

}  // namespace lsgg
