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
#include "kernels_common.cuh"

namespace lsgg {

constexpr int kHashSlots = kPoolKeys;
static_assert((kHashSlots & (kHashSlots - 1)) == 0, "hash slots: a power of two");

__global__ void __launch_bounds__(256)
k_collect_neighbours(PhysicsDev phys, StepState* st, const Box* __restrict__ prev, const int* __restrict__ IDF,
                     int* __restrict__ tab, int* __restrict__ cnt, float* __restrict__ tw, float* __restrict__ tm) {
    __shared__ int keys[kHashSlots];
    __shared__ int n_keys, overflow;
    const int b = blockIdx.x;
    const Box ob = prev[b];
    for (int k = threadIdx.x; k < kHashSlots; k += blockDim.x) keys[k] = -1;
    if (threadIdx.x == 0) { n_keys = 0; overflow = 0; }
    __syncthreads();
    if (ob.nx > 0) {
        const long long A = (long long)ob.nx * ob.ny, n = A * ob.nz;
        const int ps = plane_stride(ob.nx, ob.ny);
        int last = -1;
        for (long long c = threadIdx.x; c < n; c += blockDim.x) {
            const long long z = c / A, rem = c - z * A;
            const int j = IDF[ob.off + z * ps + rem];
            if (j < 0 || j == last) continue;
            last = j;
            unsigned h = ((unsigned)j * 2654435761u) >> 23;   // 9 bits
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
    // the box's place in the pool (every key, or none when they overflowed)
    __shared__ int pool_base;
    const bool pooled = phys.pool_ent != nullptr && !overflow;
    if (threadIdx.x == 0) {
        int base = -1;
        if (pooled && n_keys > 0) {
            base = atomicAdd(&st->pool_used, n_keys);
            if (base > phys.pool_cap - n_keys) base = -1;
        }
        pool_base = base;
        if (phys.pool_ent) phys.pool_box[b] = make_int2(base < 0 ? 0 : base, n_keys == 0 ? 0 : (base < 0 ? -1 : n_keys));
    }
    __syncthreads();
    const bool rs = phys.kind == LSGG_PHYSICS_READ_SHOCKLEY;
    // rank-sort the keys (ascending): the first kNbCap in the grain's table,
    // all of them in the pool, each with its pair weights (FP64
    // disorientation, once per grain, pair and step)
    for (int k = threadIdx.x; k < kHashSlots; k += blockDim.x) {
        const int j = keys[k];
        if (j < 0) continue;
        int rank = 0;
        for (int q = 0; q < kHashSlots; ++q) rank += (unsigned)keys[q] < (unsigned)j && keys[q] >= 0;
        if (rank >= kNbCap && pool_base < 0) continue;
        float w = 1.0f, m = 1.0f;
        if (rs) rs_pair(phys, b, j, w, m);
        if (rs && rank < kNbCap) {
            tab[(size_t)b * kNbCap + rank] = j;
            tw[(size_t)b * kNbCap + rank] = w;
            tm[(size_t)b * kNbCap + rank] = m;
        }
        if (pool_base >= 0) phys.pool_ent[pool_base + rank] = make_int4(j, __float_as_int(w), __float_as_int(m), 0);
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
    if (phys.pool_ent) {
        const cudaError_t e = cudaMemsetAsync(&B.st->pool_used, 0, sizeof(int), s);
        if (e != cudaSuccess) return e;
    }
    k_collect_neighbours<<<B.n_boxes, 256, 0, s>>>(phys, B.st, B.prev, B.IDF, const_cast<int*>(phys.nb_tab),
                                                     const_cast<int*>(phys.nb_cnt), const_cast<float*>(phys.nb_w),
                                                     const_cast<float*>(phys.nb_m));
    return cudaGetLastError();
}

}  // namespace lsgg
