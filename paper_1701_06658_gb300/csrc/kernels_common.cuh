// Device helpers shared by the batched kernels (step.cu) and the per-grain
// comparator kernels (plain.cu), so both paths do the same arithmetic.
#pragma once

#include "lsgg_internal.cuh"
#include "../../include/lsgg.h"

namespace lsgg {

__device__ __forceinline__ bool sgn_pos(float v) { return !(__float_as_uint(v) >> 31); }

__device__ __forceinline__ float pair_blend(const PhysicsDev& phys, int gid, int j, float phi, float c) {
    // Eq. (10): phi + w (c - phi) + M (e_j - e_i) dt; w = 1, no bulk when j < 0.
    if (j < 0) return c;
    float w = 1.0f, m = 1.0f;
    if (phys.kind == LSGG_PHYSICS_READ_SHOCKLEY) {
        int lo = phys.nb_start[gid], hi = phys.nb_start[gid + 1] - 1;
        while (lo <= hi) {
            int mid = (lo + hi) >> 1;
            int jj = phys.nb[mid].j;
            if (jj == j) { w = phys.nb[mid].w; m = phys.nb[mid].m; break; }
            if (jj < j) lo = mid + 1; else hi = mid - 1;
        }
    }
    float bulk = 0.0f;
    if (phys.energy) bulk = m * (phys.energy[j] - phys.energy[gid]) * phys.dt;
    return phi + w * (c - phi) + bulk;
}

// Along one line of n cells (stride `stride` in `in`), the sign-blocked
// taxicab min-plus over +-kRedistReach of cell `i`: min over cells reachable
// through same-sign cells of |v| + steps.  `wrap` for a periodic line.
__device__ __forceinline__ float line_min(const float* in, int i, int n, int stride, bool wrap) {
    const float v = in[i * stride];
    const bool s = sgn_pos(v);
    float best = fabsf(v);
#pragma unroll
    for (int k = 1; k <= kRedistReach; ++k) {
        int j = i - k;
        if (j < 0) { if (!wrap) break; j += n; }
        float u = in[j * stride];
        if (sgn_pos(u) != s) break;
        best = fminf(best, fabsf(u) + (float)k);
    }
#pragma unroll
    for (int k = 1; k <= kRedistReach; ++k) {
        int j = i + k;
        if (j >= n) { if (!wrap) break; j -= n; }
        float u = in[j * stride];
        if (sgn_pos(u) != s) break;
        best = fminf(best, fabsf(u) + (float)k);
    }
    return s ? best : -best;
}

__device__ __forceinline__ void opp_delta(float a, bool pos, float nbv, float& dmin) {
    if ((nbv > 0.0f) != pos) {
        float d = a / (a + fabsf(nbv));
        dmin = fminf(dmin, d);
    }
}

// Pull the next box of class `cls` for kernel `which`; -1 when the queue is empty.
__device__ __forceinline__ int pull_box(const StepBuffers& B, int which, int cls, int* s_box) {
    if (threadIdx.x == 0) {
        int b = -1;
        if (!*(volatile int*)&B.st->halt) {
            int w = atomicAdd(&B.st->queue[which][cls], 1);
            if (w < B.st->class_count[cls]) b = B.worklist[cls * B.n_boxes + w];
        }
        *s_box = b;
    }
    __syncthreads();
    int b = *s_box;
    __syncthreads();
    return b;
}

}  // namespace lsgg
