// Grid coarsening (Sec. 4.1, sequential optimizations): as the population
// falls the grid spacing grows, so that a grain keeps about the same number
// of cells, and every grain's function is projected onto the coarser grid by
// trilinear interpolation.
//
// On a periodic domain of N cells per axis coarsened to N' cells (one spacing:
// N'/N is the same on every axis), coarse cell i' of an axis sits at the fine
// index coordinate u = i' N / N', taken exactly as the integer quotient and
// remainder of i' N by N'.  Its value interpolates the fine values at
// floor(u) and floor(u) + 1 of each axis (-eps outside the grain's fine box),
// is scaled by N'/N (distances in coarse cells) and clamped to [-eps, eps].
// The projection leaves a valid band of only eps N'/N coarse cells; the pass
// path's re-initialisation and box update then rebuild it (launch_reinit).
//
//   k_coarsen  boxes grid-strided over CTAs, threads over the cells of a box's
//              coarse (`cur`) layout; the grain's fine function is its box
//              before the coarsening (`fine_boxes`), its values those the
//              state holds in its own layout (`prev`), -eps elsewhere -- the
//              function a step would start from; writes Z.
#include "lsgg_internal.cuh"

namespace lsgg {

namespace {

// Box-local coordinate of global cell c in the box (origin o, extent n) of an
// axis of N cells, -1 outside.
__device__ __forceinline__ int local_in(int c, int o, int n, int N) {
    int l = c - o;
    if (l < 0) l += N;
    return l < n ? l : -1;
}

// One axis of coarse cell g2: the storage-layout coordinates (-1 where the
// grain's function is -eps: outside its fine box or its stored box) of the
// fine corners floor(u) and floor(u) + 1, and the weight of the second.
struct AxisTap {
    int l0, l1;
    float w;
};

__device__ __forceinline__ AxisTap axis_tap(int g2, int N, int N2, int fo, int fn, int so, int sn) {
    const long long num = (long long)g2 * N;
    const int c0 = (int)(num / N2);                  // floor(u), in [0, N)
    const int rem = (int)(num - (long long)c0 * N2);
    const int c1 = c0 + 1 < N ? c0 + 1 : 0;
    AxisTap a;
    a.w = (float)rem / (float)N2;                     // exact quotient rounded once
    a.l0 = local_in(c0, fo, fn, N) >= 0 ? local_in(c0, so, sn, N) : -1;
    a.l1 = local_in(c1, fo, fn, N) >= 0 ? local_in(c1, so, sn, N) : -1;
    return a;
}

__device__ __forceinline__ float lerp(float a, float b, float w) { return fmaf(w, b - a, a); }

__global__ void __launch_bounds__(256)
k_coarsen(StepBuffers B, Domain F, const Box* __restrict__ fine_boxes, const float* __restrict__ X) {
    const Domain D = B.dom;
    const float eps = D.eps;
    const float scale = (float)D.nx / (float)F.nx;
    for (int b = blockIdx.x; b < B.n_boxes; b += gridDim.x) {
        const Box nb = B.cur[b], ob = B.prev[b], fb = fine_boxes[b];
        if (nb.nx <= 0 || ob.nx <= 0 || fb.nx <= 0) continue;
        const int ps = plane_stride(nb.nx, nb.ny), ops = plane_stride(ob.nx, ob.ny);
        const int nxy = nb.nx * nb.ny;
        const long long n = (long long)nxy * nb.nz;
        for (long long i = threadIdx.x; i < n; i += blockDim.x) {
            const int z = (int)(i / nxy), r = (int)(i - (long long)z * nxy);
            const int y = r / nb.nx, x = r - y * nb.nx;
            int gx = nb.ox + x, gy = nb.oy + y, gz = nb.oz + z;
            if (gx >= D.nx) gx -= D.nx;
            if (gy >= D.ny) gy -= D.ny;
            if (gz >= D.nz) gz -= D.nz;
            const AxisTap tx = axis_tap(gx, F.nx, D.nx, fb.ox, fb.nx, ob.ox, ob.nx);
            const AxisTap ty = axis_tap(gy, F.ny, D.ny, fb.oy, fb.ny, ob.oy, ob.ny);
            const AxisTap tz = axis_tap(gz, F.nz, D.nz, fb.oz, fb.nz, ob.oz, ob.nz);
            auto at = [&](int lz, int ly, int lx) -> float {
                if (lz < 0 || ly < 0 || lx < 0) return -eps;
                return X[ob.off + (long long)lz * ops + (long long)ly * ob.nx + lx];
            };
            const float c00 = lerp(at(tz.l0, ty.l0, tx.l0), at(tz.l0, ty.l0, tx.l1), tx.w);
            const float c01 = lerp(at(tz.l0, ty.l1, tx.l0), at(tz.l0, ty.l1, tx.l1), tx.w);
            const float c10 = lerp(at(tz.l1, ty.l0, tx.l0), at(tz.l1, ty.l0, tx.l1), tx.w);
            const float c11 = lerp(at(tz.l1, ty.l1, tx.l0), at(tz.l1, ty.l1, tx.l1), tx.w);
            const float v = lerp(lerp(c00, c01, ty.w), lerp(c10, c11, ty.w), tz.w);
            B.Z[nb.off + (long long)z * ps + (long long)y * nb.nx + x] = fminf(eps, fmaxf(-eps, v * scale));
        }
    }
}

}  // namespace

cudaError_t launch_coarsen(const StepBuffers& B, const Domain& fine, const Box* fine_boxes, const float* state,
                           cudaStream_t s) {
    if (B.n_boxes <= 0) return cudaSuccess;
    const int grid = B.n_boxes < B.n_sm * 8 ? B.n_boxes : B.n_sm * 8;
    k_coarsen<<<grid, 256, 0, s>>>(B, fine, fine_boxes, state);
    return cudaGetLastError();
}

}  // namespace lsgg
