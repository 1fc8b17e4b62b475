// Device helpers shared by the batched kernels (step.cu) and the per-grain
// comparator kernels (plain.cu), so both paths do the same arithmetic.
#pragma once

#include "lsgg_internal.cuh"
#include "../../include/lsgg.h"

namespace lsgg {

__device__ __forceinline__ bool sgn_pos(float v) { return !(__float_as_uint(v) >> 31); }

// Division of non-negative ints below 2^16 by a divisor d set once: q = (t *
// ceil(2^32 / d)) >> 32 is exact in that range (two instructions).  The
// multiplier of every divisor up to kDivTable comes from a table in constant
// memory (one load, uniform across the warp); larger divisors compute it.
constexpr int kDivTable = 256;
struct DivMagic {
    unsigned m[kDivTable + 1];
};
constexpr DivMagic make_div_magic() {
    DivMagic t{};
    for (int d = 1; d <= kDivTable; ++d) t.m[d] = (unsigned)((0x100000000ULL + d - 1) / d);
    return t;
}
static __constant__ DivMagic c_div_magic = make_div_magic();

struct Div16 {
    unsigned m;
    __device__ __forceinline__ explicit Div16(int d)
        : m(d <= kDivTable ? c_div_magic.m[d] : (unsigned)((0x100000000ULL + d - 1) / d)) {}
    // d = 1: the multiplier 2^32 does not fit and is stored as 0
    __device__ __forceinline__ int operator()(int t) const { return m ? (int)__umulhi((unsigned)t, m) : t; }
};

// a mod n for a within one period of [0, n) (the usual case of box and
// domain offsets), falling back to the general form otherwise.
__device__ __forceinline__ int wrap_near(int a, int n) {
    if (a < 0) a += n;
    else if (a >= n) a -= n;
    return (unsigned)a < (unsigned)n ? a : pmod(a, n);
}

// Disorientation angle (radians) of two cubic crystals: with q = conj(qa) qb
// and |q| components sorted c0 >= c1 >= c2 >= c3, the largest |w| over the 24
// proper rotations of the cube applied to q is max(c0, (c0 + c1)/sqrt 2,
// (c0 + c1 + c2 + c3)/2) (identity and half turns about the axes; quarter
// turns and half turns about face diagonals; third turns about body
// diagonals); the angle is 2 acos of it.
__device__ __forceinline__ double cubic_disorientation(const double* qa, const double* qb) {
    const double aw = qa[0], ax = -qa[1], ay = -qa[2], az = -qa[3];
    const double bw = qb[0], bx = qb[1], by = qb[2], bz = qb[3];
    double c0 = fabs(aw * bw - ax * bx - ay * by - az * bz);
    double c1 = fabs(aw * bx + ax * bw + ay * bz - az * by);
    double c2 = fabs(aw * by - ax * bz + ay * bw + az * bx);
    double c3 = fabs(aw * bz + ax * by - ay * bx + az * bw);
    double t;
    if (c0 < c1) { t = c0; c0 = c1; c1 = t; }
    if (c2 < c3) { t = c2; c2 = c3; c3 = t; }
    if (c0 < c2) { t = c0; c0 = c2; c2 = t; }
    if (c1 < c3) { t = c1; c1 = c3; c3 = t; }
    if (c1 < c2) { t = c1; c1 = c2; c2 = t; }
    double m = fmax(c0, fmax((c0 + c1) * 0.70710678118654752440, 0.5 * (c0 + c1 + c2 + c3)));
    return 2.0 * acos(fmin(1.0, m));
}

// Read-Shockley pair weight of Eq. (10) (Sec. 4.3): w = max(1e-3, M* gamma*)
// with gamma* = t (1 - ln t), t = theta / theta_max below theta_max, 1 above;
// M* = mob_low below theta_max (step law) or Eq. (20).
__device__ __forceinline__ void rs_pair(const PhysicsDev& phys, int i, int j, float& w, float& m) {
    const double th = cubic_disorientation(phys.quats + 4 * (size_t)i, phys.quats + 4 * (size_t)j);
    double g;
    if (th >= phys.theta_max) g = 1.0;
    else if (th <= 0.0) g = 0.0;
    else { const double t = th / phys.theta_max; g = t * (1.0 - log(t)); }
    double mob;
    if (phys.mob_law == LSGG_MOBILITY_STEP) mob = th < phys.theta_max ? phys.mob_low : 1.0;
    else mob = 1.0 - 0.99 * exp(-5.0 * pow(th / (15.0 * 0.017453292519943295), 9.0));
    const double ww = mob * g;
    w = (float)(ww > 1e-3 ? ww : 1e-3);
    m = (float)mob;
}

// Pair weights of one box, looked up from a shared-memory copy of its
// neighbour table (tj ascending, n entries); computed directly on a miss.
struct PairTable {
    const int* tj;
    const float* tw;
    const float* tm;
    int n;
};

// Pair weight w and mobility M of grain gid against neighbour j (j >= 0).
__device__ __forceinline__ void pair_weights(const PhysicsDev& phys, const PairTable& tab, int gid, int j, float& w,
                                             float& m) {
    w = 1.0f;
    m = 1.0f;
    if (phys.kind == LSGG_PHYSICS_READ_SHOCKLEY) {
        int lo = 0, hi = tab.n - 1;
        bool hit = false;
        while (lo <= hi) {
            const int mid = (lo + hi) >> 1;
            const int jj = tab.tj[mid];
            if (jj == j) { w = tab.tw[mid]; m = tab.tm[mid]; hit = true; break; }
            if (jj < j) lo = mid + 1; else hi = mid - 1;
        }
        if (!hit) rs_pair(phys, gid, j, w, m);
    }
}

// Eq. (10): phi + w (c - phi) + M (e_j - e_i) dt; w = 1, no bulk term when j < 0.
__device__ __forceinline__ float pair_blend(const PhysicsDev& phys, const PairTable& tab, int gid, int j, float phi,
                                            float c) {
    if (j < 0) return c;
    float w, m;
    pair_weights(phys, tab, gid, j, w, m);
    float bulk = 0.0f;
    if (phys.energy) bulk = m * (phys.energy[j] - phys.energy[gid]) * phys.dt;
    return phi + w * (c - phi) + bulk;
}

// pair_blend with the last neighbour's weights and energy kept: along a
// column the neighbour seldom changes, so the table search and the energy
// load run once per run of equal j.  Same arithmetic as pair_blend.
struct PairCache {
    int j = -1;
    float w = 1.0f, m = 1.0f, ej = 0.0f;
};
__device__ __forceinline__ float pair_blend_cached(const PhysicsDev& phys, const PairTable& tab, int gid, int j,
                                                   float phi, float c, float ei, PairCache& pc) {
    if (j < 0) return c;
    if (j != pc.j) {
        pair_weights(phys, tab, gid, j, pc.w, pc.m);
        pc.ej = phys.energy ? phys.energy[j] : 0.0f;
        pc.j = j;
    }
    float bulk = 0.0f;
    if (phys.energy) bulk = pc.m * (pc.ej - ei) * phys.dt;
    return phi + pc.w * (c - phi) + bulk;
}

// Load box `gid`'s neighbour table and its pair weights (evaluated once per
// step when the table is rebuilt) into shared memory (all threads of the CTA;
// caller synchronises afterwards).
__device__ __forceinline__ PairTable load_pair_table(const PhysicsDev& phys, int gid, int* tj, float* tw, float* tm) {
    PairTable t{tj, tw, tm, 0};
    if (phys.kind != LSGG_PHYSICS_READ_SHOCKLEY) return t;
    int n = phys.nb_cnt[gid];
    if (n > kNbCap) n = kNbCap;
    for (int k = threadIdx.x; k < n; k += blockDim.x) {
        const size_t e = (size_t)gid * kNbCap + k;
        tj[k] = phys.nb_tab[e];
        tw[k] = phys.nb_w[e];
        tm[k] = phys.nb_m[e];
    }
    t.n = n;
    return t;
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

// Reference cells of the re-initialisation (Sec. 2.1.6): a cell with a face
// neighbour of the opposite sign.  On an axis whose opposite-sign neighbours
// have largest magnitude n, linear interpolation puts the zero crossing at
// a / (a + n) cells (a = |phi|); the distance to the plane through the
// crossings of all such axes is 1 / sqrt(sum over them of ((a + n) / a)^2).
// opp_max: n for one axis' two neighbours, -1 when neither is opposite.
__device__ __forceinline__ float opp_max(bool pos, float l, float r) {
    float n = -1.0f;
    if ((l > 0.0f) != pos) n = fabsf(l);
    if ((r > 0.0f) != pos) n = fmaxf(n, fabsf(r));
    return n;
}

// Magnitude of phi after classification: eps for cells that are not reference
// cells, else the planar-exact distance (0 when phi = 0).
__device__ __forceinline__ float ref_magnitude(float a, float n0, float n1, float n2, float eps) {
    if (n0 < 0.0f && n1 < 0.0f && n2 < 0.0f) return eps;
    const float ra = __frcp_rn(a);              // = 1 / a rounded to nearest; a = 0: inf, distance 0
    float s = 0.0f;
    if (n0 >= 0.0f) { const float r = fmaf(n0, ra, 1.0f); s = fmaf(r, r, s); }
    if (n1 >= 0.0f) { const float r = fmaf(n1, ra, 1.0f); s = fmaf(r, r, s); }
    if (n2 >= 0.0f) { const float r = fmaf(n2, ra, 1.0f); s = fmaf(r, r, s); }
    return rsqrtf(s);
}

// Signed classified value of a cell from its six face neighbours.
__device__ __forceinline__ float classify_cell(float v, float xl, float xr, float yl, float yr, float zl, float zr,
                                               float eps) {
    const bool pos = v > 0.0f;
    const float mag = ref_magnitude(fabsf(v), opp_max(pos, xl, xr), opp_max(pos, yl, yr), opp_max(pos, zl, zr), eps);
    return pos ? mag : -mag;
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
