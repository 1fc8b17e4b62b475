// Neighbour tables for the velocity correction of Eq. (10).
//
// The paper refreshes a grain's neighbourhood from its points of contact and
// keeps, per cell, the nearest other grain in the ID-field (Sec. 3.1).  Here a
// grain's table is exactly the set of grain ids present in its ID-field: the
// pairs the next predictor can meet.  k_collect_neighbours rebuilds it from the
// state's ID-field before every predictor: the first kNbCap ids with their
// Read-Shockley weights in a fixed table per grain, and, on the pass path,
// every id of the box (up to kPoolKeys) with its weight and mobility in the
// step's pool, which the z pass turns into a shared-memory hash per box, so
// that no cell searches or evaluates a pair.
#include <cooperative_groups.h>

#include "kernels_common.cuh"

namespace lsgg {

namespace cg = cooperative_groups;

constexpr int kHashSlots = kPoolKeys;
static_assert((kHashSlots & (kHashSlots - 1)) == 0, "hash slots: a power of two");

// Key j enters the box's hash (shared, kHashSlots open-addressing slots);
// a full table sets the overflow flag.
__device__ __forceinline__ void collect_key(int* keys, int* n_keys, int* overflow, int j) {
    unsigned h = ((unsigned)j * 2654435761u) >> 23;   // 9 bits
    for (int probe = 0; probe < kHashSlots; ++probe) {
        const int slot = (int)((h + probe) & (kHashSlots - 1));
        const int cur = keys[slot];
        if (cur == j) return;
        if (cur == -1) {
            const int prevk = atomicCAS(&keys[slot], -1, j);
            if (prevk == -1) { atomicAdd(n_keys, 1); return; }
            if (prevk == j) return;
        }
    }
    *overflow = 1;
}

constexpr int kCollectThreads = 256;
constexpr int kCollectLoads = 4;     // 16-byte loads in flight per thread

// The box's ID-field as (plane, group of four consecutive cells) items (box
// planes start on 32-byte boundaries), kCollectLoads items per thread loaded
// together; a cell probes the hash only where a run of equal ids starts and
// its thread has not entered that id last.  I: the index type (32-bit
// divisions whenever the items fit).
template <class I>
__device__ __forceinline__ void collect_walk(const int* base, int A, int ps, int nz, int part, int parts, int* keys,
                                             int* n_keys, int* overflow) {
    const I nq = (I)((A + 3) >> 2);
    const I all = nq * (I)nz;
    const I first = all / (I)parts * (I)part + min((I)part, all % (I)parts);     // this part's items
    const I items = first + all / (I)parts + ((I)part < all % (I)parts ? 1 : 0);
    int last = -1;
    const int lane = threadIdx.x & 31;
    // the loop is uniform across each warp (its lanes exchange values below)
    for (I w0 = first + threadIdx.x - lane; w0 < items; w0 += (I)kCollectLoads * blockDim.x) {
        const I i0 = w0 + lane;
        int v[kCollectLoads][4];
#pragma unroll
        for (int k = 0; k < kCollectLoads; ++k) {
            const I it = i0 + (I)k * blockDim.x;
            const I z = it < items ? it / nq : 0;
            const int q = it < items ? 4 * (int)(it - z * nq) : 0;
            const int* pl = base + (long long)z * ps;
            if (it < items && q + 3 < A) {
                const int4 w4 = *reinterpret_cast<const int4*>(pl + q);
                v[k][0] = w4.x; v[k][1] = w4.y; v[k][2] = w4.z; v[k][3] = w4.w;
            } else {
#pragma unroll
                for (int u = 0; u < 4; ++u) v[k][u] = it < items && q + u < A ? pl[q + u] : -1;
            }
        }
        // a value equal to the cell before it (the lane's own previous cell, or
        // the previous lane's last one: lanes hold consecutive groups) is
        // already entered or being entered: only the starts of runs probe
#pragma unroll
        for (int k = 0; k < kCollectLoads; ++k) {
            int before = __shfl_up_sync(0xffffffffu, v[k][3], 1);
            if (lane == 0) before = -1;
#pragma unroll
            for (int u = 0; u < 4; ++u) {
                const int j = v[k][u];
                const bool run_start = j != (u == 0 ? before : v[k][u - 1]);
                if (j < 0 || !run_start || j == last) continue;
                last = j;
                collect_key(keys, n_keys, overflow, j);
            }
        }
    }
}

constexpr int kCollectCluster = 4;    // CTAs per box: a thread-block cluster

// A cluster of kCollectCluster CTAs per box: each walks a part of the box's
// ID-field and enters its ids into the hash in the shared memory of the
// cluster's first CTA (distributed shared memory), which then does the rest.
__global__ void __cluster_dims__(kCollectCluster, 1, 1) __launch_bounds__(kCollectThreads)
k_collect_neighbours(PhysicsDev phys, StepState* st, const Box* __restrict__ prev, const int* __restrict__ IDF,
                     int* __restrict__ tab, int* __restrict__ cnt, float* __restrict__ tw, float* __restrict__ tm) {
    __shared__ int keys[kHashSlots];
    __shared__ int n_keys, overflow;
    cg::cluster_group cluster = cg::this_cluster();
    const int part = (int)cluster.block_rank();
    const int b = blockIdx.x / kCollectCluster;
    const Box ob = prev[b];
    if (part == 0) {
        for (int k = threadIdx.x; k < kHashSlots; k += blockDim.x) keys[k] = -1;
        if (threadIdx.x == 0) { n_keys = 0; overflow = 0; }
    }
    cluster.sync();                                  // the first CTA's hash is clear before any entry
    if (ob.nx > 0) {
        int* const k0 = cluster.map_shared_rank(keys, 0);
        int* const n0 = cluster.map_shared_rank(&n_keys, 0);
        int* const o0 = cluster.map_shared_rank(&overflow, 0);
        const int A = ob.nx * ob.ny;
        const int ps = plane_stride(ob.nx, ob.ny);
        if ((long long)((A + 3) >> 2) * ob.nz < (1LL << 31) - 4LL * kCollectLoads * kCollectThreads)
            collect_walk<unsigned>(IDF + ob.off, A, ps, ob.nz, part, kCollectCluster, k0, n0, o0);
        else
            collect_walk<long long>(IDF + ob.off, A, ps, ob.nz, part, kCollectCluster, k0, n0, o0);
    }
    cluster.sync();                                  // every entry is in; the other CTAs are done
    if (part != 0) return;
    // the box's place in this step's pool (every key, or none when they overflowed)
    __shared__ int pool_base;
    // this step's pool and the previous step's (the parity of the steps done)
    const bool odd = phys.pool_ent[0] && (st->steps_done & 1);
    int2* const pool_box = odd ? phys.pool_box[1] : phys.pool_box[0];
    int4* const pool_ent = odd ? phys.pool_ent[1] : phys.pool_ent[0];
    const int2* const prev_box = odd ? phys.pool_box[0] : phys.pool_box[1];
    const int4* const prev_pool = odd ? phys.pool_ent[0] : phys.pool_ent[1];
    const bool pooled = pool_ent != nullptr && !overflow;
    if (threadIdx.x == 0) {
        int base = -1;
        if (pooled && n_keys > 0) {
            base = atomicAdd(&st->pool_used, n_keys);
            if (base > phys.pool_cap - n_keys) base = -1;
        }
        pool_base = base;
        if (pool_ent) pool_box[b] = make_int2(base < 0 ? 0 : base, n_keys == 0 ? 0 : (base < 0 ? -1 : n_keys));
    }
    // the keys in consecutive entries, then ranked (ascending) among
    // themselves, so that the weights below are evaluated by full warps
    __shared__ int packed[kHashSlots], sorted[kHashSlots];
    __shared__ int n_packed;
    if (threadIdx.x == 0) n_packed = 0;
    __syncthreads();
    for (int k = threadIdx.x; k < kHashSlots; k += blockDim.x)
        if (keys[k] >= 0) packed[atomicAdd(&n_packed, 1)] = keys[k];
    __syncthreads();
    const int np = n_packed;
    for (int k = threadIdx.x; k < np; k += blockDim.x) {
        const int j = packed[k];
        int rank = 0;
        for (int q = 0; q < np; ++q) rank += packed[q] < j;
        sorted[rank] = j;
    }
    __syncthreads();
    const bool rs = phys.kind == LSGG_PHYSICS_READ_SHOCKLEY;
    // the first kNbCap in the grain's table, all of them in the pool, each
    // with its pair weights: the previous step's list of the box (the other
    // pool) gives those of the pairs it held, the rest are evaluated (FP64
    // disorientation)
    const int2 prev_list = pool_ent ? prev_box[b] : make_int2(0, 0);
    const int4* prev_ent = pool_ent ? prev_pool + prev_list.x : nullptr;
    const int n_eval = pool_base >= 0 ? n_keys : min(n_keys, kNbCap);
    for (int rank = threadIdx.x; rank < n_eval; rank += blockDim.x) {
        const int j = sorted[rank];
        float w = 1.0f, m = 1.0f;
        if (rs) {
            int lo = 0, hi = prev_list.y - 1;             // count -1: no list
            bool hit = false;
            while (lo <= hi) {
                const int mid = (lo + hi) >> 1;
                const int4 e = prev_ent[mid];
                if (e.x == j) { w = __int_as_float(e.y); m = __int_as_float(e.z); hit = true; break; }
                if (e.x < j) lo = mid + 1; else hi = mid - 1;
            }
            if (!hit) rs_pair(phys, b, j, w, m);
        }
        if (rs && rank < kNbCap) {
            tab[(size_t)b * kNbCap + rank] = j;
            tw[(size_t)b * kNbCap + rank] = w;
            tm[(size_t)b * kNbCap + rank] = m;
        }
        if (pool_base >= 0) pool_ent[pool_base + rank] = make_int4(j, __float_as_int(w), __float_as_int(m), 0);
    }
    if (threadIdx.x == 0 && rs) cnt[b] = (overflow || n_keys > kNbCap) ? kNbCap + 1 : n_keys;
}

// Contact neighbours of each box from the neighbour-max field of the last step:
// per cell the largest other grain above -eps (the step's ID-field).
__global__ void __launch_bounds__(256)
k_field_neighbours(Domain D, const Box* __restrict__ boxes, const unsigned long long* __restrict__ T, int cap,
                   int* __restrict__ tab, int* __restrict__ cnt) {
    __shared__ int keys[kHashSlots];
    __shared__ int n_keys, overflow;
    const int b = blockIdx.x;
    const Box nb = boxes[b];
    for (int k = threadIdx.x; k < kHashSlots; k += blockDim.x) keys[k] = -1;
    if (threadIdx.x == 0) { n_keys = 0; overflow = 0; }
    __syncthreads();
    if (nb.nx > 0) {
        const long long A = (long long)nb.nx * nb.ny, n = A * nb.nz;
        int last = -1;
        for (long long c = threadIdx.x; c < n; c += blockDim.x) {
            const int z = (int)(c / A);
            const int rem = (int)(c - (long long)z * A);
            const int y = rem / nb.nx, x = rem - y * nb.nx;
            const long long g = ((long long)pmod(nb.oz + z, D.nz) * D.ny + pmod(nb.oy + y, D.ny)) * D.nx +
                                pmod(nb.ox + x, D.nx);
            const unsigned long long k1 = T[2 * g], k2 = T[2 * g + 1];
            const int id1 = key_id(k1);
            const unsigned long long kk = id1 != b ? k1 : k2;
            if (!kk || !(key_val(kk, D.eps) > -D.eps)) continue;
            const int j = key_id(kk);
            if (j == last) continue;
            last = j;
            unsigned h = ((unsigned)j * 2654435761u) >> 23;
            for (int probe = 0; probe < kHashSlots; ++probe) {
                const int slot = (int)((h + probe) & (kHashSlots - 1));
                const int cur = keys[slot];
                if (cur == j) break;
                if (cur == -1) {
                    const int prevk = atomicCAS(&keys[slot], -1, j);
                    if (prevk == -1) { atomicAdd(&n_keys, 1); break; }
                    if (prevk == j) break;
                }
                if (probe == kHashSlots - 1) overflow = 1;
            }
        }
    }
    __syncthreads();
    for (int k = threadIdx.x; k < kHashSlots; k += blockDim.x) {
        const int j = keys[k];
        if (j < 0) continue;
        int rank = 0;
        for (int q = 0; q < kHashSlots; ++q) rank += (unsigned)keys[q] < (unsigned)j && keys[q] >= 0;
        if (rank < cap) tab[(size_t)b * cap + rank] = j;
    }
    if (threadIdx.x == 0) cnt[b] = overflow ? cap + 1 : n_keys;
}

cudaError_t launch_field_neighbours(const StepBuffers& B, const Box* boxes, int cap, int* tab, int* cnt,
                                    cudaStream_t s) {
    k_field_neighbours<<<B.n_boxes, 256, 0, s>>>(B.dom, boxes, B.T, cap, tab, cnt);
    return cudaGetLastError();
}

cudaError_t launch_collect_neighbours(const StepBuffers& B, const PhysicsDev& phys, cudaStream_t s) {
    if (phys.pool_ent[0]) {
        const cudaError_t e = cudaMemsetAsync(&B.st->pool_used, 0, sizeof(int), s);
        if (e != cudaSuccess) return e;
    }
    k_collect_neighbours<<<B.n_boxes * kCollectCluster, kCollectThreads, 0, s>>>(phys, B.st, B.prev, B.IDF, const_cast<int*>(phys.nb_tab),
                                                     const_cast<int*>(phys.nb_cnt), const_cast<float*>(phys.nb_w),
                                                     const_cast<float*>(phys.nb_m));
    return cudaGetLastError();
}

}  // namespace lsgg
