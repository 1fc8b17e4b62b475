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
//   k_gb_map  a CTA per box (grid-stride over the boxes).  The box's
//             triangles are built once, into the CTA's scratch in the order of
//             their cubes (x fastest): the cubes' triangle counts, a
//             block-wide prefix sum giving each cube its first triangle, then
//             the triangles themselves.  The cells with |phi| < tube are
//             gathered into a shared-memory list so that every thread
//             searches one of them: the cubes within r = ceil(tube) + 1 cells
//             per axis form, per row of cubes, one contiguous range of
//             triangles; the smallest (squared distance, grain) over them is
//             the box's minimum when its distance is below r (a triangle
//             outside that window lies at least r away), and otherwise
//             (a function far from a distance function, or a tube wider
//             than the band) every triangle of the box is searched -- a
//             bound of cells x triangles.  Every other cell, and every cell
//             of a box with no triangle, copies the ID-field.  A box with
//             more cubes or triangles than the scratch holds takes the same
//             search with the triangles rebuilt from each cube's corners.
//             The same kernel serves the stateless op (packed boxes) and the
//             step (the state arena's layout, FP32 or BF16 state).
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

// A box of the map: its cells (x fastest) start at `base`, planes `ps`
// elements apart; phi is FP32 or the state arena's BF16.
struct GbBox {
    long long base;
    int nx, ny, nz, ps;
};

__device__ __forceinline__ float gb_phi(const float* phi, long long i) { return phi[i]; }
__device__ __forceinline__ float gb_phi(const __nv_bfloat16* phi, long long i) { return __bfloat162float(phi[i]); }

// The triangles of cube (z, y, x) (its base corner): each passed to emit(a, b,
// c, grain).  Returns their number.
template <class T, class Emit>
__device__ int cube_triangles(const GbBox& bx, const T* __restrict__ phi, const int* __restrict__ idf, int z, int y,
                              int x, Emit emit) {
    float f[8];
    int id[8];
    unsigned posm = 0;
    for (int k = 0; k < 8; ++k) {
        const long long o = bx.base + (long long)(z + (k >> 2)) * bx.ps + (long long)(y + ((k >> 1) & 1)) * bx.nx +
                            (x + (k & 1));
        f[k] = gb_phi(phi, o);
        id[k] = idf[o];
        posm |= (f[k] > 0.0f ? 1u : 0u) << k;
    }
    if (posm == 0u || posm == 0xffu) return 0;
    int n = 0;
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
            emit(e[0], e[1], e[2], g);
            n += 1;
        } else {
            int a = -1, bb = -1, cc = -1, d = -1;           // positive a < bb, non-positive cc < d
            for (int m = 0; m < 4; ++m) {
                if (pos[m]) { if (a < 0) a = m; else bb = m; }
                else { if (cc < 0) cc = m; else d = m; }
            }
            const V3 eac = edge_pt(P[a], P[cc], F[a], F[cc]), ead = edge_pt(P[a], P[d], F[a], F[d]);
            const V3 ebd = edge_pt(P[bb], P[d], F[bb], F[d]), ebc = edge_pt(P[bb], P[cc], F[bb], F[cc]);
            emit(eac, ead, ebd, g);
            emit(eac, ebd, ebc, g);
            n += 2;
        }
    }
    return n;
}

// Number of triangles of cube (z, y, x): one per tetrahedron with one or three
// positive corners, two per tetrahedron with two.
template <class T>
__device__ int cube_triangle_count(const GbBox& bx, const T* __restrict__ phi, int z, int y, int x) {
    unsigned posm = 0;
    for (int k = 0; k < 8; ++k) {
        const long long o = bx.base + (long long)(z + (k >> 2)) * bx.ps + (long long)(y + ((k >> 1) & 1)) * bx.nx +
                            (x + (k & 1));
        posm |= (gb_phi(phi, o) > 0.0f ? 1u : 0u) << k;
    }
    if (posm == 0u || posm == 0xffu) return 0;
    int n = 0;
    for (int t = 0; t < 6; ++t) {
        int np = 0;
        for (int m = 0; m < 4; ++m) np += (posm >> c_kuhn[t][m]) & 1u;
        n += np == 2 ? 2 : (np == 1 || np == 3 ? 1 : 0);
    }
    return n;
}

// A stored triangle: three float4 (vertices z, y, x in order, then the grain).
__device__ __forceinline__ void store_tri(float4* t, V3 a, V3 b, V3 c, int g) {
    t[0] = make_float4(a.z, a.y, a.x, b.z);
    t[1] = make_float4(b.y, b.x, c.z, c.y);
    t[2] = make_float4(c.x, __int_as_float(g), 0.0f, 0.0f);
}
__device__ __forceinline__ void offer_tri(Best& best, V3 p, const float4* t) {
    const float4 u = t[0], v = t[1], w = t[2];
    offer(best, tri_d2(p, v3(u.x, u.y, u.z), v3(u.w, v.x, v.y), v3(v.z, v.w, w.x)), __float_as_int(w.y));
}

constexpr int kGbThreads = 256;
constexpr int kGbGather = 8;          // cells a thread tests per round of the band-cell gathering

template <class T>
__device__ void gb_map_box(const GbBox bx, const T* __restrict__ phi, const int* __restrict__ idf, int* __restrict__ out,
                           float tube, int r, int* __restrict__ off, float4* __restrict__ tri, int cap_cubes,
                           int cap_tris) {
    __shared__ int s_list[kGbThreads * kGbGather];
    __shared__ int s_cnt, s_part[kGbThreads / 32];
    const int t = threadIdx.x;
    const int nx = bx.nx, ny = bx.ny, nz = bx.nz;
    const long long A = (long long)nx * ny, n = A * nz;
    const int ncx = nx - 1, ncy = ny - 1, ncz = nz - 1;
    const bool cubes = ncx >= 1 && ncy >= 1 && ncz >= 1;
    const long long ncubes = cubes ? (long long)ncx * ncy * ncz : 0;
    // triangles in scratch: per cube its count, then the exclusive prefix sum
    // (thread-contiguous chunks, a block scan of the chunk sums)
    bool stored = cubes && ncubes <= cap_cubes;
    int total = 0;
    if (stored) {
        const int per = (int)((ncubes + kGbThreads - 1) / kGbThreads);
        const int q0 = (int)min((long long)t * per, ncubes), q1 = (int)min((long long)q0 + per, ncubes);
        int sum = 0;
        for (int q = q0; q < q1; ++q) {
            const int cx = q % ncx, rest = q / ncx, cy = rest % ncy, cz = rest / ncy;
            const int c = cube_triangle_count(bx, phi, cz, cy, cx);
            off[q] = c;
            sum += c;
        }
        // block exclusive scan of the chunk sums
        int incl = sum;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            const int v = __shfl_up_sync(0xffffffffu, incl, o);
            if ((t & 31) >= o) incl += v;
        }
        if ((t & 31) == 31) s_part[t >> 5] = incl;
        __syncthreads();
        if (t == 0) {
            int acc = 0;
            for (int w = 0; w < kGbThreads / 32; ++w) { const int v = s_part[w]; s_part[w] = acc; acc += v; }
            s_cnt = acc;
        }
        __syncthreads();
        int run = s_part[t >> 5] + incl - sum;
        total = s_cnt;
        for (int q = q0; q < q1; ++q) { const int c = off[q]; off[q] = run; run += c; }
        if (t == kGbThreads - 1) off[ncubes] = run;
        stored = total <= cap_tris;
        __syncthreads();
        if (stored) {
            for (int q = t; q < ncubes; q += kGbThreads) {
                const int first = off[q];
                if (off[q + 1] == first) continue;
                const int cx = q % ncx, rest = q / ncx, cy = rest % ncy, cz = rest / ncy;
                int k = first;
                cube_triangles(bx, phi, idf, cz, cy, cx, [&](V3 a, V3 b, V3 c, int g) { store_tri(tri + 3 * (k++), a, b, c, g); });
            }
        }
        __syncthreads();
    }
    const float r_in = (float)r - 0.01f;
    // rounds: every thread tests kGbGather cells; the band cells go to s_list
    for (long long base = 0; base < n; base += (long long)kGbThreads * kGbGather) {
        if (t == 0) s_cnt = 0;
        __syncthreads();
#pragma unroll
        for (int u = 0; u < kGbGather; ++u) {
            const long long i = base + (long long)u * kGbThreads + t;
            if (i >= n) break;
            const int z = (int)(i / A), rem = (int)(i - (long long)z * A);
            const long long o = bx.base + (long long)z * bx.ps + rem;
            if (cubes && fabsf(gb_phi(phi, o)) < tube) s_list[atomicAdd(&s_cnt, 1)] = (int)(i - base);
            else out[o] = idf[o];
        }
        __syncthreads();
        const int cnt = s_cnt;
        for (int k = t; k < cnt; k += kGbThreads) {
            const long long i = base + s_list[k];
            const int z = (int)(i / A), rem = (int)(i - (long long)z * A);
            const int y = rem / nx, x = rem - y * nx;
            const long long o = bx.base + (long long)z * bx.ps + rem;
            const V3 p = v3((float)z, (float)y, (float)x);
            Best best{0.0f, -1, false};
            const int xl = max(0, x - r), xh = min(ncx - 1, x + r - 1);
            for (int cz = max(0, z - r); cz <= min(ncz - 1, z + r - 1); ++cz)
                for (int cy = max(0, y - r); cy <= min(ncy - 1, y + r - 1); ++cy) {
                    if (stored) {
                        const int q = (cz * ncy + cy) * ncx;
                        const int e = off[q + xh + 1];
                        for (int j = off[q + xl]; j < e; ++j) offer_tri(best, p, tri + 3 * j);
                    } else {
                        for (int cx = xl; cx <= xh; ++cx)
                            cube_triangles(bx, phi, idf, cz, cy, cx, [&](V3 a, V3 b, V3 c, int g) { offer(best, tri_d2(p, a, b, c), g); });
                    }
                }
            if (!(best.any && best.d2 < r_in * r_in)) {     // not provably the box's minimum: every triangle
                if (stored) {
                    for (int j = 0; j < total; ++j) offer_tri(best, p, tri + 3 * j);
                } else {
                    for (int cz = 0; cz < ncz; ++cz)
                        for (int cy = 0; cy < ncy; ++cy)
                            for (int cx = 0; cx < ncx; ++cx)
                                cube_triangles(bx, phi, idf, cz, cy, cx, [&](V3 a, V3 b, V3 c, int g) { offer(best, tri_d2(p, a, b, c), g); });
                }
            }
            out[o] = best.any ? best.grain : idf[o];
        }
        __syncthreads();                                  // s_list and s_cnt are reused
    }
}

__device__ __forceinline__ bool gb_box_ok(const lsgg_box& b, long long n_elems) {
    if (b.nx <= 0 || b.ny < 1 || b.nz < 1) return false;
    const long long n = (long long)b.nx * b.ny * b.nz;
    return b.offset >= 0 && b.offset <= n_elems && n <= n_elems - b.offset;
}

// the stateless op: packed boxes, FP32 phi
__global__ void __launch_bounds__(kGbThreads)
k_gb_map(const lsgg_box* __restrict__ boxes, int n_boxes, const float* __restrict__ phi_all,
         const int* __restrict__ idf_all, long long n_elems, float tube, int r, int* __restrict__ out_all,
         int* __restrict__ scratch_off, float4* __restrict__ scratch_tri, int cap_cubes, int cap_tris) {
    int* off = scratch_off + (long long)blockIdx.x * (cap_cubes + 1);
    float4* tri = scratch_tri + (long long)blockIdx.x * 3 * cap_tris;
    for (int b = blockIdx.x; b < n_boxes; b += gridDim.x) {
        const lsgg_box bx = boxes[b];
        if (!gb_box_ok(bx, n_elems)) continue;
        const GbBox g{bx.offset, bx.nx, bx.ny, bx.nz, bx.nx * bx.ny};
        gb_map_box(g, phi_all, idf_all, out_all, tube, r, off, tri, cap_cubes, cap_tris);
        __syncthreads();
    }
}

// The state and its ID-field on the current boxes (the boxes the step writes),
// in their layout: a cell outside the previous box is -eps and -1 (the
// grain's function and ID-field as they enter the step, Sec. 3.1).
__global__ void __launch_bounds__(256)
k_gb_resample(StepBuffers B, float* __restrict__ phi, int* __restrict__ idf) {
    const Domain D = B.dom;
    for (int b = blockIdx.x; b < B.n_boxes; b += gridDim.x) {
        const Box nb = B.cur[b], ob = B.prev[b];
        if (nb.nx <= 0) continue;
        const int A = nb.nx * nb.ny, ps = plane_stride(nb.nx, nb.ny), ops = plane_stride(ob.nx, ob.ny);
        const long long n = (long long)A * nb.nz;
        for (long long i = threadIdx.x; i < n; i += blockDim.x) {
            const int z = (int)(i / A), rem = (int)(i - (long long)z * A);
            const int y = rem / nb.nx, x = rem - y * nb.nx;
            const int lx = pmod(nb.ox + x - ob.ox, D.nx), ly = pmod(nb.oy + y - ob.oy, D.ny);
            const int lz = pmod(nb.oz + z - ob.oz, D.nz);
            float v = -D.eps;
            int j = -1;
            if (lx < ob.nx && ly < ob.ny && lz < ob.nz) {
                const long long o = ob.off + (long long)lz * ops + (long long)ly * ob.nx + lx;
                v = ld_state(B, o);
                j = B.IDF[o];
            }
            const long long d = nb.off + (long long)z * ps + rem;
            phi[d] = v;
            idf[d] = j;
        }
    }
}

// the step: every alive box on its current box, phi and ID-field resampled
// into the layout of `cur`, the map into `map` (same layout)
__global__ void __launch_bounds__(kGbThreads)
k_gb_map_step(StepBuffers B, const float* __restrict__ phi, const int* __restrict__ idf, float tube, int r,
              int* __restrict__ map, int* __restrict__ scratch_off, float4* __restrict__ scratch_tri, int cap_cubes,
              int cap_tris) {
    if (*(volatile int*)&B.st->halt) return;
    int* off = scratch_off + (long long)blockIdx.x * (cap_cubes + 1);
    float4* tri = scratch_tri + (long long)blockIdx.x * 3 * cap_tris;
    for (int b = blockIdx.x; b < B.n_boxes; b += gridDim.x) {
        const Box nb = B.cur[b];
        if (nb.nx <= 0) continue;
        const GbBox g{nb.off, nb.nx, nb.ny, nb.nz, plane_stride(nb.nx, nb.ny)};
        gb_map_box(g, phi, idf, map, tube, r, off, tri, cap_cubes, cap_tris);
        __syncthreads();
    }
}

}  // namespace

// Scratch of the map for `grid` CTAs: per CTA 3 * cap_tris float4 of
// triangles, then cap_cubes + 1 ints of per-cube offsets.
size_t gb_map_scratch_bytes(int grid, int cap_cubes, int cap_tris) {
    return (size_t)grid * ((size_t)cap_tris * 3 * sizeof(float4) + ((size_t)cap_cubes + 1) * sizeof(int));
}

static void gb_scratch(void* scratch, int grid, int cap_tris, int** off, float4** tri) {
    *tri = static_cast<float4*>(scratch);
    *off = reinterpret_cast<int*>(*tri + (size_t)grid * 3 * cap_tris);
}

// The anisotropy map of the step into B.gb_map (layout of `cur`): the state
// and ID-field resampled onto the current boxes into Y and Z (free before the
// predictor's passes write them), then the map.
cudaError_t launch_gb_map_step(const StepBuffers& B, cudaStream_t s) {
    int* off = nullptr;
    float4* tri = nullptr;
    gb_scratch(B.gb_scratch, B.gb_grid, B.gb_cap_tris, &off, &tri);
    int* idf = reinterpret_cast<int*>(B.Z);
    k_gb_resample<<<B.n_sm * 4, 256, 0, s>>>(B, B.Y, idf);
    const int r = (int)ceilf(B.gb_tube) + 1;
    k_gb_map_step<<<B.gb_grid, kGbThreads, 0, s>>>(B, B.Y, idf, B.gb_tube, r, B.gb_map, off, tri, B.gb_cap_cubes,
                                                   B.gb_cap_tris);
    return cudaGetLastError();
}

}  // namespace lsgg

// The stateless op's scratch: boxes of up to 2^17 cubes and 2^15 triangles
// keep their triangles; larger ones rebuild them per cell.
static constexpr int kOpCapCubes = 1 << 17, kOpCapTris = 1 << 15;

extern "C" int lsgg_closest_gb_map(const lsgg_box* boxes_dev, int32_t n_boxes, const float* phi_dev,
                                   const int32_t* idf_dev, int64_t n_elems, float tube, int32_t* out_dev,
                                   void* stream) {
    if (!boxes_dev || !phi_dev || !idf_dev || !out_dev || n_boxes < 0 || n_elems < 0) return LSGG_ERR_INVALID_ARG;
    if (!(tube > 0.0f && tube <= 16.0f)) return LSGG_ERR_INVALID_ARG;
    if (n_boxes == 0) return LSGG_OK;
    int dev = 0, n_sm = 1;
    if (cudaGetDevice(&dev) != cudaSuccess ||
        cudaDeviceGetAttribute(&n_sm, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess) {
        cudaGetLastError();
        return LSGG_ERR_CUDA;
    }
    const int grid = n_boxes < 2 * n_sm ? n_boxes : 2 * n_sm;
    cudaStream_t s = (cudaStream_t)stream;
    void* scratch = nullptr;
    if (cudaMallocAsync(&scratch, lsgg::gb_map_scratch_bytes(grid, kOpCapCubes, kOpCapTris), s) != cudaSuccess) {
        cudaGetLastError();
        return LSGG_ERR_OUT_OF_MEMORY;
    }
    int* off = nullptr;
    float4* tri = nullptr;
    lsgg::gb_scratch(scratch, grid, kOpCapTris, &off, &tri);
    const int r = (int)std::ceil(tube) + 1;
    lsgg::k_gb_map<<<grid, lsgg::kGbThreads, 0, s>>>(boxes_dev, n_boxes, phi_dev, idf_dev, n_elems, tube, r, out_dev,
                                                     off, tri, kOpCapCubes, kOpCapTris);
    const cudaError_t e = cudaGetLastError();
    cudaFreeAsync(scratch, s);
    return e == cudaSuccess ? LSGG_OK : LSGG_ERR_CUDA;
}
