// Initial microstructure: Algorithm 1, "Initialization" (Sec. 2.1.3; the
// tessellation input of Sec. 3.1).
//
//   k_labels        power-diagram label of each cell: argmin_i |x - s_i|^2 - w_i
//                   with minimum-image displacements, lowest id on ties.  An FP32
//                   pass finds the minimum; candidates within a safe margin are
//                   decided in FP64 with explicitly rounded operations so the
//                   integer result does not depend on FMA contraction.
//   k_face_pairs    grains whose cells touch across a face (bit matrix).
//   k_label_bbox    per grain, min/max of the integer minimum-image offsets of its
//                   cells from its rounded seed.
//   k_init_boxes    box = that bbox grown by the halo (full axis if it reaches N).
//   k_sdf           phi_i(x) = clamp(min_{j in Nb(i)} signed distance of x to the
//                   power bisector of (i, j), -eps, eps) and the minimising j.
#include <cfloat>
#include <climits>

#include "lsgg_internal.cuh"

namespace lsgg {

__device__ __forceinline__ double min_image(double d, double n) {
    // d - n * rint(d / n), each operation rounded on its own
    return __dsub_rn(d, __dmul_rn(n, rint(__ddiv_rn(d, n))));
}

__device__ __forceinline__ float min_image_f(float d, float n) {
    return d - n * rintf(d / n);
}

constexpr int kSeedTile = 512;

__global__ void __launch_bounds__(256)
k_labels(Domain D, int G, const double* __restrict__ seeds, const double* __restrict__ weights,
         int* __restrict__ labels) {
    __shared__ float4 s_f[kSeedTile];
    const long long ncell = (long long)D.nx * D.ny * D.nz;
    const long long cell = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    const bool active = cell < ncell;
    int x = 0, y = 0, z = 0;
    if (active) {
        x = (int)(cell % D.nx);
        y = (int)((cell / D.nx) % D.ny);
        z = (int)(cell / ((long long)D.nx * D.ny));
    }
    const float fnx = (float)D.nx, fny = (float)D.ny, fnz = (float)D.nz;
    // pass 1: FP32 minimum of the power distance
    float best32 = FLT_MAX;
    for (int t0 = 0; t0 < G; t0 += kSeedTile) {
        __syncthreads();
        for (int k = threadIdx.x; k < kSeedTile && t0 + k < G; k += blockDim.x) {
            int i = t0 + k;
            s_f[k] = make_float4((float)seeds[3 * i], (float)seeds[3 * i + 1], (float)seeds[3 * i + 2],
                                 weights ? (float)weights[i] : 0.0f);
        }
        __syncthreads();
        if (active) {
            int n = min(kSeedTile, G - t0);
            for (int k = 0; k < n; ++k) {
                float4 s = s_f[k];
                float dx = min_image_f((float)x - s.x, fnx);
                float dy = min_image_f((float)y - s.y, fny);
                float dz = min_image_f((float)z - s.z, fnz);
                float r = dx * dx + dy * dy + dz * dz - s.w;
                best32 = fminf(best32, r);
            }
        }
    }
    // margin covering FP32 rounding of |d|^2 <= 3 N^2 and of the weights
    float nmax = fmaxf(fnx, fmaxf(fny, fnz));
    const float margin = 0.5f + 4e-6f * nmax * nmax + 1e-5f * fabsf(best32);
    // pass 2: exact FP64 decision among the candidates
    double best = DBL_MAX;
    int arg = -1;
    for (int t0 = 0; t0 < G; t0 += kSeedTile) {
        __syncthreads();
        for (int k = threadIdx.x; k < kSeedTile && t0 + k < G; k += blockDim.x) {
            int i = t0 + k;
            s_f[k] = make_float4((float)seeds[3 * i], (float)seeds[3 * i + 1], (float)seeds[3 * i + 2],
                                 weights ? (float)weights[i] : 0.0f);
        }
        __syncthreads();
        if (active) {
            int n = min(kSeedTile, G - t0);
            for (int k = 0; k < n; ++k) {
                float4 s = s_f[k];
                float dx = min_image_f((float)x - s.x, fnx);
                float dy = min_image_f((float)y - s.y, fny);
                float dz = min_image_f((float)z - s.z, fnz);
                float r = dx * dx + dy * dy + dz * dz - s.w;
                if (r <= best32 + margin) {
                    int i = t0 + k;
                    double ex = min_image(__dsub_rn((double)x, seeds[3 * i]), (double)D.nx);
                    double ey = min_image(__dsub_rn((double)y, seeds[3 * i + 1]), (double)D.ny);
                    double ez = min_image(__dsub_rn((double)z, seeds[3 * i + 2]), (double)D.nz);
                    double rr = __dadd_rn(__dadd_rn(__dmul_rn(ex, ex), __dmul_rn(ey, ey)), __dmul_rn(ez, ez));
                    if (weights) rr = __dsub_rn(rr, weights[i]);
                    if (rr < best) { best = rr; arg = i; }
                }
            }
        }
    }
    if (active) labels[cell] = arg;
}

__global__ void k_face_pairs(Domain D, int G, const int* __restrict__ labels, unsigned* __restrict__ bits,
                             long long words_per_row) {
    const long long ncell = (long long)D.nx * D.ny * D.nz;
    for (long long cell = (long long)blockIdx.x * blockDim.x + threadIdx.x; cell < ncell;
         cell += (long long)gridDim.x * blockDim.x) {
        int x = (int)(cell % D.nx);
        int y = (int)((cell / D.nx) % D.ny);
        int z = (int)(cell / ((long long)D.nx * D.ny));
        int a = labels[cell];
        int nbr[3];
        nbr[0] = labels[((long long)z * D.ny + y) * D.nx + (x + 1) % D.nx];
        nbr[1] = labels[((long long)z * D.ny + (y + 1) % D.ny) * D.nx + x];
        nbr[2] = D.dim == 3 ? labels[((long long)((z + 1) % D.nz) * D.ny + y) * D.nx + x] : a;
        for (int k = 0; k < 3; ++k) {
            int b = nbr[k];
            if (b == a) continue;
            atomicOr(&bits[(long long)a * words_per_row + (b >> 5)], 1u << (b & 31));
            atomicOr(&bits[(long long)b * words_per_row + (a >> 5)], 1u << (a & 31));
        }
    }
}

__device__ __forceinline__ int offset_from(int x, int r, int n) {
    int e = pmod(x - r, n);
    return e > n / 2 ? e - n : e;
}

__global__ void k_bbox_init(int G, int* bb) {
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < G; i += gridDim.x * blockDim.x) {
        for (int a = 0; a < 3; ++a) { bb[6 * i + a] = INT_MAX; bb[6 * i + 3 + a] = INT_MIN; }
    }
}

__global__ void k_label_bbox(Domain D, const int* __restrict__ labels, const double* __restrict__ seeds,
                             int* __restrict__ bb) {
    const long long ncell = (long long)D.nx * D.ny * D.nz;
    for (long long cell = (long long)blockIdx.x * blockDim.x + threadIdx.x; cell < ncell;
         cell += (long long)gridDim.x * blockDim.x) {
        int x = (int)(cell % D.nx);
        int y = (int)((cell / D.nx) % D.ny);
        int z = (int)(cell / ((long long)D.nx * D.ny));
        int i = labels[cell];
        int c[3] = {x, y, z};
        int N[3] = {D.nx, D.ny, D.nz};
        for (int a = 0; a < 3; ++a) {
            int r = pmod((int)rint(seeds[3 * i + a]), N[a]);
            int e = offset_from(c[a], r, N[a]);
            atomicMin(&bb[6 * i + a], e);
            atomicMax(&bb[6 * i + 3 + a], e);
        }
    }
}

__global__ void k_init_boxes(Domain D, int G, const int* __restrict__ bb, const double* __restrict__ seeds,
                             Box* __restrict__ cur) {
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < G; i += gridDim.x * blockDim.x) {
        Box b{};
        if (bb[6 * i] > bb[6 * i + 3]) {       // no cell: extinct from the start
            cur[i] = b;
            continue;
        }
        int N[3] = {D.nx, D.ny, D.nz};
        int o[3], n[3];
        for (int a = 0; a < 3; ++a) {
            if (N[a] == 1) { o[a] = 0; n[a] = 1; continue; }
            int r = pmod((int)rint(seeds[3 * i + a]), N[a]);
            int lo = bb[6 * i + a], hi = bb[6 * i + 3 + a];
            int ext = hi - lo + 1 + 2 * D.halo;
            n[a] = ext < N[a] ? ext : N[a];
            o[a] = pmod(r + lo - D.halo, N[a]);
        }
        b.ox = o[0]; b.oy = o[1]; b.oz = o[2];
        b.nx = n[0]; b.ny = n[1]; b.nz = n[2];
        cur[i] = b;
    }
}

constexpr int kSdfNb = 512;

__device__ __forceinline__ double power_dist(const double* p, const double* s, double w, const double* N,
                                             double& e0, double& e1, double& e2) {
    e0 = min_image(__dsub_rn(p[0], s[0]), N[0]);
    e1 = min_image(__dsub_rn(p[1], s[1]), N[1]);
    e2 = min_image(__dsub_rn(p[2], s[2]), N[2]);
    return __dsub_rn(__dadd_rn(__dadd_rn(__dmul_rn(e0, e0), __dmul_rn(e1, e1)), __dmul_rn(e2, e2)), w);
}

__global__ void __launch_bounds__(256)
k_sdf(Domain D, int G, const Box* __restrict__ boxes, const double* __restrict__ seeds,
      const double* __restrict__ weights, const unsigned* __restrict__ bits, long long words_per_row,
      float* __restrict__ X, int* __restrict__ IDF, int* __restrict__ status) {
    __shared__ int s_nb[kSdfNb];
    __shared__ int s_cnt;
    const int i = blockIdx.x;
    const Box b = boxes[i];
    if (b.nx <= 0) return;
    if (threadIdx.x == 0) {
        int cnt = 0;
        for (long long w = 0; w < words_per_row; ++w) {
            unsigned m = bits[(long long)i * words_per_row + w];
            while (m) {
                int bit = __ffs(m) - 1;
                m &= m - 1;
                if (cnt < kSdfNb) s_nb[cnt] = (int)(w * 32 + bit);
                ++cnt;
            }
        }
        if (cnt > kSdfNb) { atomicExch(status, -8); cnt = kSdfNb; }
        s_cnt = cnt;
    }
    __syncthreads();
    const int cnt = s_cnt;
    const double si[3] = {seeds[3 * i], seeds[3 * i + 1], seeds[3 * i + 2]};
    const double wi = weights ? weights[i] : 0.0;
    const double Nd[3] = {(double)D.nx, (double)D.ny, (double)D.nz};
    const int A = b.nx * b.ny;
    const int ps = plane_stride(b.nx, b.ny);
    const long long ncell = (long long)A * b.nz;
    const double eps = (double)D.eps;
    for (long long idx = threadIdx.x; idx < ncell; idx += blockDim.x) {
        int z = (int)(idx / A);
        int rem = (int)(idx - (long long)z * A);
        int y = rem / b.nx, x = rem - y * b.nx;
        double p[3] = {(double)pmod(b.ox + x, D.nx), (double)pmod(b.oy + y, D.ny), (double)pmod(b.oz + z, D.nz)};
        double a0, a1, a2;
        double pa = power_dist(p, si, wi, Nd, a0, a1, a2);
        double best = DBL_MAX;
        int arg = -1;
        for (int k = 0; k < cnt; ++k) {
            int j = s_nb[k];
            double b0, b1, b2;
            double pb = power_dist(p, seeds + 3 * j, weights ? weights[j] : 0.0, Nd, b0, b1, b2);
            double d0 = __dsub_rn(b0, a0), d1 = __dsub_rn(b1, a1), d2 = __dsub_rn(b2, a2);
            double den = __dmul_rn(2.0, __dsqrt_rn(__dadd_rn(__dadd_rn(__dmul_rn(d0, d0), __dmul_rn(d1, d1)),
                                                             __dmul_rn(d2, d2))));
            double v = __ddiv_rn(__dsub_rn(pb, pa), den);
            if (v < best) { best = v; arg = j; }
        }
        double outv = best == DBL_MAX ? eps : (best < -eps ? -eps : (best > eps ? eps : best));
        long long o = b.off + (long long)z * ps + rem;
        X[o] = (float)outv;
        if (IDF) IDF[o] = arg;
    }
}

cudaError_t launch_init(const Domain& D, int G, const double* d_seeds, const double* d_weights,
                        int* d_labels, unsigned* d_bits, long long words_per_row, int* d_bb,
                        Box* d_cur, cudaStream_t s) {
    const long long ncell = (long long)D.nx * D.ny * D.nz;
    int blocks = (int)((ncell + 255) / 256);
    k_labels<<<blocks, 256, 0, s>>>(D, G, d_seeds, d_weights, d_labels);
    cudaError_t e = cudaMemsetAsync(d_bits, 0, (size_t)G * words_per_row * 4, s);
    if (e != cudaSuccess) return e;
    int gs = (int)((ncell + 255) / 256);
    if (gs > 65535 * 8) gs = 65535 * 8;
    k_face_pairs<<<gs, 256, 0, s>>>(D, G, d_labels, d_bits, words_per_row);
    k_bbox_init<<<(G + 255) / 256, 256, 0, s>>>(G, d_bb);
    k_label_bbox<<<gs, 256, 0, s>>>(D, d_labels, d_seeds, d_bb);
    k_init_boxes<<<(G + 255) / 256, 256, 0, s>>>(D, G, d_bb, d_seeds, d_cur);
    return cudaGetLastError();
}

cudaError_t launch_sdf(const Domain& D, int G, const Box* d_cur, const double* d_seeds, const double* d_weights,
                       const unsigned* d_bits, long long words_per_row, float* X, int* IDF, int* d_status,
                       cudaStream_t s) {
    k_sdf<<<G, 256, 0, s>>>(D, G, d_cur, d_seeds, d_weights, d_bits, words_per_row, X, IDF, d_status);
    return cudaGetLastError();
}

}  // namespace lsgg
