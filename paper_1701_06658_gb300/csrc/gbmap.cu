// Anisotropy map of Sec. 2.1.4 on the device: every cell near a grain's
// boundary adopts the grain across the closest point of that boundary, so
// that Eq. (10)'s weight w(i, j) and mobility come from the closest GB point
// rather than from the cell's own ID-field entry (Sec. 4.1 accelerates the
// same search by clustering triple-junction points; here the box-local
// window below plays that role).
//
// The boundary of grain i is the zero level of its box function phi_i,
// triangulated by marching tetrahedra: each cell cube (8 corners) split into
// the six tetrahedra around its main diagonal, one per order of the axes
// (z, y, x), the level linearly interpolated on the edges between corners of
// opposite sign (phi > 0 inside).  A tetrahedron with one corner apart gives a
// triangle, one with two and two a quad (positive corners a < b, the others
// c < d, in the tetrahedron's corner order) split along the diagonal from the
// point on edge (a, c) to the point on edge (b, d).  A triangle faces the
// grain most frequent in the ID-field among its tetrahedron's corners with
// phi <= 0 (lowest id on ties, -1 without any).
//
//   k_gb_map  one CTA per box, threads over its cells.  A cell with
//             |phi| < tube takes the grain of the triangle at the smallest
//             (squared distance, grain) -- the order of the triangles does not
//             matter -- searched over the cubes within r = ceil(tube) + 1 cells
//             per axis; a triangle outside that window lies at distance >= r,
//             so a best distance below r is the box's minimum, and otherwise
//             (a function far from a distance function) every cube of the box
//             is searched.  Every other cell, and every cell of a box with no
//             triangle, copies the ID-field.
//
// Box-local: the cubes are those between the box's own cells; a periodic
// (full) axis is not wrapped, and a box with an axis of one cell has no cubes.
#include <cmath>

#include "lsgg_internal.cuh"
#include "../../include/lsgg.h"

namespace lsgg {

namespace {

struct V3 {
    float z, y, x;
};

__device__ __forceinline__ V3 v3(float z, float y, float x) { return V3{z, y, x}; }
__device__ __forceinline__ V3 operator-(V3 a, V3 b) { return v3(a.z - b.z, a.y - b.y, a.x - b.x); }
__device__ __forceinline__ V3 operator+(V3 a, V3 b) { return v3(a.z + b.z, a.y + b.y, a.x + b.x); }
__device__ __forceinline__ V3 operator*(V3 a, float s) { return v3(a.z * s, a.y * s, a.x * s); }
__device__ __forceinline__ float dot(V3 a, V3 b) { return fmaf(a.z, b.z, fmaf(a.y, b.y, a.x * b.x)); }
__device__ __forceinline__ V3 cross(V3 a, V3 b) {
    return v3(a.y * b.x - a.x * b.y, a.x * b.z - a.z * b.x, a.z * b.y - a.y * b.z);
}

// Squared distance from p to segment [u, v] (the clamped projection).
__device__ __forceinline__ float seg_d2(V3 p, V3 u, V3 v) {
    const V3 e = v - u, w = p - u;
    const float ee = dot(e, e);
    const float t = ee > 0.0f ? fminf(1.0f, fmaxf(0.0f, dot(w, e) / ee)) : 0.0f;
    const V3 d = w - e * t;
    return dot(d, d);
}

// Squared distance from p to triangle (a, b, c): the nearest of its edges, or
// its plane when the foot point lies inside.  A triangle whose two edges from
// a span an angle below about 1e-5 rad is treated as its edges.
__device__ float tri_d2(V3 p, V3 a, V3 b, V3 c) {
    float best = fminf(seg_d2(p, a, b), fminf(seg_d2(p, b, c), seg_d2(p, c, a)));
    const V3 ab = b - a, ac = c - a;
    const V3 n = cross(ab, ac);
    const float nn = dot(n, n);
    if (nn > 1e-10f * dot(ab, ab) * dot(ac, ac)) {
        const float s = dot(p - a, n);
        const V3 f = p - n * (s / nn);
        if (dot(cross(ab, f - a), n) >= 0.0f && dot(cross(c - b, f - b), n) >= 0.0f &&
            dot(cross(a - c, f - c), n) >= 0.0f)
            best = fminf(best, s * s / nn);
    }
    return best;
}

// Zero of the linear interpolant from corner u to corner v.
__device__ __forceinline__ V3 edge_pt(V3 pu, V3 pv, float fu, float fv) { return pu + (pv - pu) * (fu / (fu - fv)); }

struct Best {
    float d2;
    int grain;
    bool any;
};

__device__ __forceinline__ void offer(Best& b, float d2, int g) {
    if (!b.any || d2 < b.d2 || (d2 == b.d2 && g < b.grain)) {
        b.d2 = d2;
        b.grain = g;
        b.any = true;
    }
}

// Corner k of a cube: bit 2 = +z, bit 1 = +y, bit 0 = +x.  The six
// tetrahedra, one per order of the axes: 0, then one, two and three unit steps.
__constant__ unsigned char c_kuhn[6][4] = {
    {0, 4, 6, 7}, {0, 4, 5, 7}, {0, 2, 6, 7}, {0, 2, 3, 7}, {0, 1, 5, 7}, {0, 1, 3, 7}};

// Offer every triangle of cube (z, y, x) (its base corner) to b.
__device__ void offer_cube(Best& b, V3 p, const float* __restrict__ phi, const int* __restrict__ idf, int z,
                           int y, int x, int ny, int nx) {
    float f[8];
    int id[8];
    unsigned posm = 0;
    for (int k = 0; k < 8; ++k) {
        const long long o = ((long long)(z + (k >> 2)) * ny + (y + ((k >> 1) & 1))) * nx + (x + (k & 1));
        f[k] = phi[o];
        id[k] = idf[o];
        posm |= (f[k] > 0.0f ? 1u : 0u) << k;
    }
    if (posm == 0u || posm == 0xffu) return;
    for (int t = 0; t < 6; ++t) {
        int c[4];
        V3 P[4];
        float F[4];
        bool pos[4];
        int np = 0;
        for (int m = 0; m < 4; ++m) {
            c[m] = c_kuhn[t][m];
            P[m] = v3((float)(z + (c[m] >> 2)), (float)(y + ((c[m] >> 1) & 1)), (float)(x + (c[m] & 1)));
            F[m] = f[c[m]];
            pos[m] = F[m] > 0.0f;
            np += pos[m];
        }
        if (np == 0 || np == 4) continue;
        // the grain across: the most frequent id >= 0 among the corners with phi <= 0
        int g = -1, gc = 0;
        for (int m = 0; m < 4; ++m) {
            const int v = id[c[m]];
            if (pos[m] || v < 0) continue;
            int cnt = 0;
            for (int q = 0; q < 4; ++q) cnt += (!pos[q] && id[c[q]] == v);
            if (cnt > gc || (cnt == gc && v < g)) { g = v; gc = cnt; }
        }
        if (np == 1 || np == 3) {
            int k = 0;
            while (pos[k] != (np == 1)) ++k;                 // the corner apart
            V3 e[3];
            int w = 0;
            for (int m = 0; m < 4; ++m)
                if (m != k) e[w++] = edge_pt(P[k], P[m], F[k], F[m]);
            offer(b, tri_d2(p, e[0], e[1], e[2]), g);
        } else {
            int a = -1, bb = -1, cc = -1, d = -1;           // positive a < bb, non-positive cc < d
            for (int m = 0; m < 4; ++m) {
                if (pos[m]) { if (a < 0) a = m; else bb = m; }
                else { if (cc < 0) cc = m; else d = m; }
            }
            const V3 eac = edge_pt(P[a], P[cc], F[a], F[cc]), ead = edge_pt(P[a], P[d], F[a], F[d]);
            const V3 ebd = edge_pt(P[bb], P[d], F[bb], F[d]), ebc = edge_pt(P[bb], P[cc], F[bb], F[cc]);
            offer(b, tri_d2(p, eac, ead, ebd), g);
            offer(b, tri_d2(p, eac, ebd, ebc), g);
        }
    }
}

__device__ __forceinline__ bool gb_box_ok(const lsgg_box& b, long long n_elems) {
    if (b.nx <= 0 || b.ny < 1 || b.nz < 1) return false;
    const long long n = (long long)b.nx * b.ny * b.nz;
    return b.offset >= 0 && b.offset <= n_elems && n <= n_elems - b.offset;
}

__global__ void __launch_bounds__(256)
k_gb_map(const lsgg_box* __restrict__ boxes, const float* __restrict__ phi_all, const int* __restrict__ idf_all,
         long long n_elems, float tube, int r, int* __restrict__ out_all) {
    const lsgg_box bx = boxes[blockIdx.x];
    if (!gb_box_ok(bx, n_elems)) return;
    const int nx = bx.nx, ny = bx.ny, nz = bx.nz;
    const float* phi = phi_all + bx.offset;
    const int* idf = idf_all + bx.offset;
    int* out = out_all + bx.offset;
    const long long A = (long long)nx * ny, n = A * nz;
    const bool cubes = nx >= 2 && ny >= 2 && nz >= 2;
    const float r_in = (float)r - 0.01f;
    for (long long i = threadIdx.x; i < n; i += blockDim.x) {
        int res = idf[i];
        if (cubes && fabsf(phi[i]) < tube) {
            const int z = (int)(i / A), rem = (int)(i - (long long)z * A);
            const int y = rem / nx, x = rem - y * nx;
            const V3 p = v3((float)z, (float)y, (float)x);
            Best b{0.0f, -1, false};
            for (int cz = max(0, z - r); cz <= min(nz - 2, z + r - 1); ++cz)
                for (int cy = max(0, y - r); cy <= min(ny - 2, y + r - 1); ++cy)
                    for (int cx = max(0, x - r); cx <= min(nx - 2, x + r - 1); ++cx)
                        offer_cube(b, p, phi, idf, cz, cy, cx, ny, nx);
            if (!(b.any && b.d2 < r_in * r_in)) {             // not provably the box's minimum: every cube
                b.any = false;
                for (int cz = 0; cz <= nz - 2; ++cz)
                    for (int cy = 0; cy <= ny - 2; ++cy)
                        for (int cx = 0; cx <= nx - 2; ++cx) offer_cube(b, p, phi, idf, cz, cy, cx, ny, nx);
            }
            if (b.any) res = b.grain;
        }
        out[i] = res;
    }
}

}  // namespace

}  // namespace lsgg

extern "C" int lsgg_closest_gb_map(const lsgg_box* boxes_dev, int32_t n_boxes, const float* phi_dev,
                                   const int32_t* idf_dev, int64_t n_elems, float tube, int32_t* out_dev,
                                   void* stream) {
    if (!boxes_dev || !phi_dev || !idf_dev || !out_dev || n_boxes < 0 || n_elems < 0) return LSGG_ERR_INVALID_ARG;
    if (!(tube > 0.0f && tube <= 16.0f)) return LSGG_ERR_INVALID_ARG;
    if (n_boxes == 0) return LSGG_OK;
    const int r = (int)std::ceil(tube) + 1;
    lsgg::k_gb_map<<<n_boxes, 256, 0, (cudaStream_t)stream>>>(boxes_dev, phi_dev, idf_dev, n_elems, tube, r,
                                                             out_dev);
    return cudaGetLastError() == cudaSuccess ? LSGG_OK : LSGG_ERR_CUDA;
}
