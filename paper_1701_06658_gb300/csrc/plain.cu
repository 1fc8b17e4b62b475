// Comparator path: the same step as step.cu, launched grain by grain.
//
// For every alive grain the host issues separate cell-parallel kernels per
// sub-step of Algorithm 1, each working through global memory:
//   predictor     kp_conv_x, kp_conv_y, kp_conv_z (+ neighbour-max scatter)
//   corrector     kp_compare (after every grain's predictor)
//   re-init       kp_classify, kp_dt_x, kp_dt_y, kp_dt_z (+ positive bbox)
// followed by the batched box update.  Per step that is 8 launches per grain
// in 3D (6 in 2D) plus three: the structure a straightforward port of the
// paper's per-grain loop gives, kept to measure what batching buys.
#include <climits>
#include <vector>

#include "kernels_common.cuh"

namespace lsgg {

struct PlainBox {
    Box nb, ob;      // current (written) and previous (state) layouts
    int gid;
};

__device__ __forceinline__ float masked_state(const Domain& D, const PlainBox& p, const float* X, int xl, int yl,
                                              int zl) {
    // value of grain p at new-box local (xl, yl, zl) possibly outside [0, n): wrap on full axes, -eps outside
    const Box& nb = p.nb;
    const Box& ob = p.ob;
    const bool fx = nb.nx == D.nx, fy = nb.ny == D.ny, fz = nb.nz == D.nz;
    if (fx) xl = pmod(xl, nb.nx); else if (xl < 0 || xl >= nb.nx) return -D.eps;
    if (fy) yl = pmod(yl, nb.ny); else if (yl < 0 || yl >= nb.ny) return -D.eps;
    if (D.dim == 3) { if (fz) zl = pmod(zl, nb.nz); else if (zl < 0 || zl >= nb.nz) return -D.eps; }
    int ox = pmod(nb.ox + xl - ob.ox, D.nx), oy = pmod(nb.oy + yl - ob.oy, D.ny);
    int oz = D.dim == 3 ? pmod(nb.oz + zl - ob.oz, D.nz) : 0;
    if (ox >= ob.nx || oy >= ob.ny || oz >= ob.nz) return -D.eps;
    return X[ob.off + (long long)oz * plane_stride(ob.nx, ob.ny) + oy * ob.nx + ox];
}

__global__ void kp_conv_x(Domain D, PlainBox p, const float* __restrict__ X, float* __restrict__ t1, Taps taps) {
    const int R = taps.radius, W = 2 * R + 1;
    const int nx = p.nb.nx, py = p.nb.ny + 2 * R, pz = D.dim == 3 ? p.nb.nz + 2 * R : 1;
    const long long n = (long long)nx * py * pz;
    for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x) {
        int x = (int)(i % nx);
        int yp = (int)((i / nx) % py);
        int zp = (int)(i / ((long long)nx * py));
        int yl = yp - R, zl = D.dim == 3 ? zp - R : 0;
        float acc = 0.0f;
        for (int k = 0; k < W; ++k) acc = fmaf(taps.g[k], masked_state(D, p, X, x + k - R, yl, zl), acc);
        t1[i] = acc;
    }
}

__global__ void kp_conv_y(Domain D, PlainBox p, const float* __restrict__ t1, float* __restrict__ t2, Taps taps) {
    const int R = taps.radius, W = 2 * R + 1;
    const int nx = p.nb.nx, ny = p.nb.ny, py = ny + 2 * R, pz = D.dim == 3 ? p.nb.nz + 2 * R : 1;
    const long long n = (long long)nx * ny * pz;
    for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x) {
        int x = (int)(i % nx);
        int y = (int)((i / nx) % ny);
        int zp = (int)(i / ((long long)nx * ny));
        float acc = 0.0f;
        for (int k = 0; k < W; ++k) acc = fmaf(taps.g[k], t1[((long long)zp * py + y + k) * nx + x], acc);
        t2[i] = acc;
    }
}

__global__ void kp_conv_z(Domain D, PlainBox p, const float* __restrict__ t2, const float* __restrict__ X,
                          const int* __restrict__ IDF, float* __restrict__ Y, unsigned long long* __restrict__ T,
                          Taps taps, PhysicsDev phys) {
    const int R = taps.radius, W = 2 * R + 1;
    const Box& nb = p.nb;
    const int nx = nb.nx, ny = nb.ny, nz = nb.nz;
    const long long A = (long long)nx * ny, n = A * nz;
    const int ps = plane_stride(nx, ny);
    for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x) {
        int x = (int)(i % nx);
        int y = (int)((i / nx) % ny);
        int z = (int)(i / A);
        float c;
        if (D.dim == 3) {
            c = 0.0f;
            for (int k = 0; k < W; ++k) c = fmaf(taps.g[k], t2[(long long)(z + k) * A + (long long)y * nx + x], c);
        } else {
            c = t2[(long long)y * nx + x];
        }
        float v = c;
        if (phys.kind != LSGG_PHYSICS_IDEAL) {
            const Box& ob = p.ob;
            int ox = pmod(nb.ox + x - ob.ox, D.nx), oy = pmod(nb.oy + y - ob.oy, D.ny);
            int oz = D.dim == 3 ? pmod(nb.oz + z - ob.oz, D.nz) : 0;
            float phi0 = -D.eps;
            int j = -1;
            if (ox < ob.nx && oy < ob.ny && oz < ob.nz) {
                long long o = ob.off + (long long)oz * plane_stride(ob.nx, ob.ny) + oy * ob.nx + ox;
                phi0 = X[o];
                j = IDF[o];
            }
            v = pair_blend(phys, PairTable{nullptr, nullptr, nullptr, 0}, p.gid, j, phi0, c);
        }
        v = fminf(fmaxf(v, -D.eps), D.eps);
        Y[nb.off + (long long)z * ps + (long long)y * nx + x] = v;
        long long g = ((long long)pmod(nb.oz + z, D.nz) * D.ny + pmod(nb.oy + y, D.ny)) * D.nx + pmod(nb.ox + x, D.nx);
        unsigned long long key = make_key(v, p.gid);
        unsigned long long old = atomicMax(&T[2 * g], key);
        if (old) atomicMax(&T[2 * g + 1], old < key ? old : key);
    }
}

__global__ void kp_compare(Domain D, PlainBox p, const float* __restrict__ Y, const unsigned long long* __restrict__ T,
                           float* __restrict__ Cc, int* __restrict__ IDF, int write_idf) {
    const Box& nb = p.nb;
    const long long A = (long long)nb.nx * nb.ny, n = A * nb.nz;
    const int ps = plane_stride(nb.nx, nb.ny);
    for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x) {
        int x = (int)(i % nb.nx);
        int y = (int)((i / nb.nx) % nb.ny);
        int z = (int)(i / A);
        long long o = nb.off + (long long)z * ps + (long long)y * nb.nx + x;
        long long g = ((long long)pmod(nb.oz + z, D.nz) * D.ny + pmod(nb.oy + y, D.ny)) * D.nx + pmod(nb.ox + x, D.nx);
        unsigned long long k1 = T[2 * g], k2 = T[2 * g + 1];
        int id1 = key_id(k1);
        float m;
        int mid;
        if (id1 != p.gid) { m = key_val(k1, D.eps); mid = id1; }
        else { m = key_val(k2, D.eps); mid = key_id(k2); }
        if (!(m > -D.eps)) mid = -1;
        Cc[o] = 0.5f * (Y[o] - m);
        if (write_idf) IDF[o] = mid;
    }
}

__device__ __forceinline__ float box_value(const Domain& D, const Box& nb, const float* A_, int x, int y, int z) {
    // phi_c at local (x, y, z) with wrap on full axes and -eps outside the box
    if (x < 0 || x >= nb.nx) { if (nb.nx != D.nx) return -D.eps; x = pmod(x, nb.nx); }
    if (y < 0 || y >= nb.ny) { if (nb.ny != D.ny) return -D.eps; y = pmod(y, nb.ny); }
    if (z < 0 || z >= nb.nz) { if (nb.nz != D.nz) return -D.eps; z = pmod(z, nb.nz); }
    return A_[nb.off + (long long)z * plane_stride(nb.nx, nb.ny) + (long long)y * nb.nx + x];
}

__global__ void kp_classify(Domain D, PlainBox p, const float* __restrict__ Cc, float* __restrict__ Gg) {
    const Box& nb = p.nb;
    const long long A = (long long)nb.nx * nb.ny, n = A * nb.nz;
    const int ps = plane_stride(nb.nx, nb.ny);
    for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x) {
        int x = (int)(i % nb.nx);
        int y = (int)((i / nb.nx) % nb.ny);
        int z = (int)(i / A);
        const float v = box_value(D, nb, Cc, x, y, z);
        const bool pos = v > 0.0f;
        float n[3] = {-1.0f, -1.0f, -1.0f};
        for (int ax = 0; ax < D.dim; ++ax) {
            const int dx = ax == 0, dy = ax == 1, dz = ax == 2;
            n[ax] = opp_max(pos, box_value(D, nb, Cc, x - dx, y - dy, z - dz), box_value(D, nb, Cc, x + dx, y + dy, z + dz));
        }
        const float mag = ref_magnitude(fabsf(v), n[0], n[1], n[2], D.eps);
        Gg[nb.off + (long long)z * ps + (long long)y * nb.nx + x] = pos ? mag : -mag;
    }
}

// Taxicab min-plus along one axis (0 = x, 1 = y, 2 = z); the z pass writes the
// clamped result and accumulates the positive bounding box.
__global__ void kp_dt(Domain D, PlainBox p, int axis, const float* __restrict__ in, float* __restrict__ out,
                      int final_pass, Bounds* __restrict__ bounds) {
    const Box& nb = p.nb;
    const long long A = (long long)nb.nx * nb.ny, n = A * nb.nz;
    const int ps = plane_stride(nb.nx, nb.ny);
    for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x) {
        int x = (int)(i % nb.nx);
        int y = (int)((i / nb.nx) % nb.ny);
        int z = (int)(i / A);
        const float* base = in + nb.off;
        float v;
        if (axis == 0) v = line_min(base + (long long)z * ps + (long long)y * nb.nx, x, nb.nx, 1, nb.nx == D.nx);
        else if (axis == 1) v = line_min(base + (long long)z * ps + x, y, nb.ny, nb.nx, nb.ny == D.ny);
        else v = line_min(base + (long long)y * nb.nx + x, z, nb.nz, ps, nb.nz == D.nz);
        long long o = nb.off + (long long)z * ps + (long long)y * nb.nx + x;
        if (final_pass) {
            float m = fminf(fabsf(v), D.eps);
            v = sgn_pos(v) ? m : -m;
            if (v > 0.0f) {
                Bounds* bd = bounds + p.gid;
                atomicMin(&bd->lo[0], x); atomicMax(&bd->hi[0], x);
                atomicMin(&bd->lo[1], y); atomicMax(&bd->hi[1], y);
                atomicMin(&bd->lo[2], z); atomicMax(&bd->hi[2], z);
            }
        }
        out[o] = v;
    }
}

__global__ void kp_bounds_init(int G, Bounds* bounds) {
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < G; i += gridDim.x * blockDim.x) {
        Bounds b;
        for (int a = 0; a < 3; ++a) { b.lo[a] = INT_MAX; b.hi[a] = INT_MIN; }
        bounds[i] = b;
    }
}

static int grid_for(long long n) {
    long long b = (n + 255) / 256;
    return (int)(b < 1 ? 1 : (b > 4096 ? 4096 : b));
}

// h_cur / h_prev: host copies of the box tables for this step.
cudaError_t launch_plain_step_impl(const StepBuffers& B, const Taps& taps, const PhysicsDev& phys,
                                   const Box* h_cur, const Box* h_prev, float* t1, float* t2, float* Cc,
                                   float* Gg, float* Hh, cudaStream_t s) {
    const Domain& D = B.dom;
    const int R = taps.radius;
    long long ncell = (long long)D.nx * D.ny * D.nz;
    cudaError_t e = cudaMemsetAsync(B.T, 0, (size_t)ncell * 16, s);
    if (e != cudaSuccess) return e;
    kp_bounds_init<<<grid_for(B.n_boxes), 256, 0, s>>>(B.n_boxes, B.bounds);
    for (int b = 0; b < B.n_boxes; ++b) {
        if (h_cur[b].nx <= 0) continue;
        PlainBox p{h_cur[b], h_prev[b], b};
        long long n1 = (long long)p.nb.nx * (p.nb.ny + 2 * R) * (D.dim == 3 ? p.nb.nz + 2 * R : 1);
        long long n2 = (long long)p.nb.nx * p.nb.ny * (D.dim == 3 ? p.nb.nz + 2 * R : 1);
        long long n3 = (long long)p.nb.nx * p.nb.ny * p.nb.nz;
        kp_conv_x<<<grid_for(n1), 256, 0, s>>>(D, p, B.X, t1, taps);
        kp_conv_y<<<grid_for(n2), 256, 0, s>>>(D, p, t1, t2, taps);
        kp_conv_z<<<grid_for(n3), 256, 0, s>>>(D, p, t2, B.X, B.IDF, B.Y, B.T, taps, phys);
    }
    const int widf = phys.kind != LSGG_PHYSICS_IDEAL;
    for (int b = 0; b < B.n_boxes; ++b) {
        if (h_cur[b].nx <= 0) continue;
        PlainBox p{h_cur[b], h_prev[b], b};
        long long n3 = (long long)p.nb.nx * p.nb.ny * p.nb.nz;
        int gr = grid_for(n3);
        kp_compare<<<gr, 256, 0, s>>>(D, p, B.Y, B.T, Cc, B.IDF, widf);
        kp_classify<<<gr, 256, 0, s>>>(D, p, Cc, Gg);
        kp_dt<<<gr, 256, 0, s>>>(D, p, 0, Gg, Hh, 0, B.bounds);
        if (D.dim == 3) {
            kp_dt<<<gr, 256, 0, s>>>(D, p, 1, Hh, Gg, 0, B.bounds);
            kp_dt<<<gr, 256, 0, s>>>(D, p, 2, Gg, B.X, 1, B.bounds);
        } else {
            kp_dt<<<gr, 256, 0, s>>>(D, p, 1, Hh, B.X, 1, B.bounds);
        }
    }
    e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    return launch_box_update(B, false, s);
}

}  // namespace lsgg
