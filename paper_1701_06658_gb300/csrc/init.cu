// Initial microstructure: Algorithm 1, "Initialization" (Sec. 2.1.3; the
// tessellation input of Sec. 3.1).
//
//   k_labels        power-diagram label of each cell: argmin_i |x - s_i|^2 - w_i
//                   with minimum-image displacements, lowest id on ties.  The
//                   seeds are binned on a uniform grid; an FP32 search over the
//                   bins around the cell bounds the minimum, and candidates within
//                   a safe margin of it are decided in FP64 with explicitly
//                   rounded operations, so the integer result does not depend on
//                   FMA contraction or on the search order.
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

// Minimum image d - n * rint(d / n) for |d| < n (cells and seeds in [0, n)):
// rint(d / n) is +1 exactly when d > n / 2 and -1 when d < -n / 2 (n / 2 is
// exact; a double d within half an ulp of 0.5 n is n / 2 itself, whose
// quotient 0.5 rounds to 0), so the division is replaced by comparisons.
// Seeds outside [0, n) take the general form.
__device__ __forceinline__ double min_image(double d, double n) {
    const double h = 0.5 * n;
    if (fabs(d) < n) return d > h ? __dsub_rn(d, n) : (d < -h ? __dadd_rn(d, n) : d);
    return __dsub_rn(d, __dmul_rn(n, rint(__ddiv_rn(d, n))));
}

__device__ __forceinline__ float wrap_half(float d, float n) {
    return d > 0.5f * n ? d - n : (d < -0.5f * n ? d + n : d);
}

// A bin index within one period of [0, nb) (the reach never exceeds a period).
__device__ __forceinline__ int wrap_bin(int i, int nb) { return i < 0 ? i + nb : (i >= nb ? i - nb : i); }

// Bins of one axis to visit around bin c at reach k: [lo, lo + cnt) cyclically.
__device__ __forceinline__ void bin_range(int c, int k, int nb, int& lo, int& cnt) {
    if (2 * k + 1 >= nb) { lo = 0; cnt = nb; }
    else { lo = c - k; cnt = 2 * k + 1; }
}

// Visit every seed in the bin block around (cx, cy, cz) of reach (kx, ky, kz).
template <class F>
__device__ __forceinline__ void for_block(const SeedBins& S, int cx, int cy, int cz, int kx, int ky, int kz, F f) {
    int lx, nx_, ly, ny_, lz, nz_;
    bin_range(cx, kx, S.nb[0], lx, nx_);
    bin_range(cy, ky, S.nb[1], ly, ny_);
    bin_range(cz, kz, S.nb[2], lz, nz_);
    for (int iz = 0; iz < nz_; ++iz) {
        const int bz = wrap_bin(lz + iz, S.nb[2]);
        for (int iy = 0; iy < ny_; ++iy) {
            const int by = wrap_bin(ly + iy, S.nb[1]);
            const int row = (bz * S.nb[1] + by) * S.nb[0];
            for (int ix = 0; ix < nx_; ++ix) {
                const int bin = row + wrap_bin(lx + ix, S.nb[0]);
                for (int q = S.start[bin]; q < S.start[bin + 1]; ++q) f(q);
            }
        }
    }
}

__global__ void __launch_bounds__(256)
k_labels(Domain D, int G, SeedBins S, const double* __restrict__ seeds, const double* __restrict__ weights,
         int* __restrict__ labels) {
    const long long ncell = (long long)D.nx * D.ny * D.nz;
    const long long cell = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (cell >= ncell) return;
    const int x = (int)(cell % D.nx);
    const int y = (int)((cell / D.nx) % D.ny);
    const int z = (int)(cell / ((long long)D.nx * D.ny));
    const float fx = (float)x, fy = (float)y, fz = (float)z;
    const float fnx = (float)D.nx, fny = (float)D.ny, fnz = (float)D.nz;
    const int cx = min(S.nb[0] - 1, (int)(fx / S.size[0]));
    const int cy = min(S.nb[1] - 1, (int)(fy / S.size[1]));
    const int cz = min(S.nb[2] - 1, (int)(fz / S.size[2]));
    auto d32 = [&](int q) {
        const float4 p = S.pts[q];
        const float dx = wrap_half(fx - p.x, fnx), dy = wrap_half(fy - p.y, fny), dz = wrap_half(fz - p.z, fnz);
        return dx * dx + dy * dy + dz * dz - p.w;
    };
    // an upper bound from the neighbouring bins, then every seed that can beat it
    float bound = FLT_MAX;
    for_block(S, cx, cy, cz, 1, 1, 1, [&](int q) { bound = fminf(bound, d32(q)); });
    const float nmax = fmaxf(fnx, fmaxf(fny, fnz));
    // margin covering FP32 rounding of |d|^2 <= 3 N^2, of the seeds and of the weights
    auto margin = [&](float v) { return 0.5f + 4e-6f * nmax * nmax + 1e-5f * fabsf(v); };
    int k[3] = {S.nb[0], S.nb[1], S.nb[2]};
    if (bound < FLT_MAX) {
        const float r = sqrtf(fmaxf(0.0f, bound + margin(bound) + S.wmax)) + 1.0f;   // + 1: bin-edge rounding
        for (int a = 0; a < 3; ++a) k[a] = (int)ceilf(r / S.size[a]) + 1;
    }
    // one pass: the FP32 minimum and the seeds within the margin of the running
    // minimum (a superset of those within the margin of the final one); a
    // full candidate list falls back to a second pass
    constexpr int kCand = 8;
    int cand[kCand];
    float cand_d[kCand];
    int n_cand = 0;
    bool rescan = false;
    float best32 = FLT_MAX;
    for_block(S, cx, cy, cz, k[0], k[1], k[2], [&](int q) {
        const float d = d32(q);
        best32 = fminf(best32, d);
        if (d <= best32 + margin(best32)) {
            if (n_cand < kCand) { cand[n_cand] = q; cand_d[n_cand] = d; ++n_cand; }
            else rescan = true;
        }
    });
    const float lim = best32 + margin(best32);
    double best = DBL_MAX;
    int arg = -1;
    auto exact = [&](int q) {
        const int i = S.ids[q];
        const double ex = min_image(__dsub_rn((double)x, seeds[3 * i]), (double)D.nx);
        const double ey = min_image(__dsub_rn((double)y, seeds[3 * i + 1]), (double)D.ny);
        const double ez = min_image(__dsub_rn((double)z, seeds[3 * i + 2]), (double)D.nz);
        double rr = __dadd_rn(__dadd_rn(__dmul_rn(ex, ex), __dmul_rn(ey, ey)), __dmul_rn(ez, ez));
        if (weights) rr = __dsub_rn(rr, weights[i]);
        if (rr < best || (rr == best && i < arg)) { best = rr; arg = i; }
    };
    if (!rescan) {
        for (int c = 0; c < n_cand; ++c)
            if (cand_d[c] <= lim) exact(cand[c]);
    } else {
        for_block(S, cx, cy, cz, k[0], k[1], k[2], [&](int q) {
            if (d32(q) <= lim) exact(q);
        });
    }
    labels[cell] = arg;
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

// For cell p with displacement a = p - s_i (minimum image) and neighbour j
// with D = s_i - s_j (minimum image), p - s_j = a + D up to one period per
// axis; with d = (p - s_j) - a the bisector distance is
// (d . (d + 2a) - (w_j - w_i)) / (2 |d|).  An FP32 pass over the neighbours
// finds the candidates within a margin of the minimum; those are evaluated in
// FP64 in that well-conditioned form (a reciprocal square root instead of a
// square root and a division): the same value as the definition's
// ((p - s_j)^2 - w_j - (p - s_i)^2 + w_i) / (2 |d|) up to FP64 rounding,
// far below the FP32 result's half unit.
__global__ void __launch_bounds__(256)
k_sdf(Domain D, int G, const Box* __restrict__ boxes, const double* __restrict__ seeds,
      const double* __restrict__ weights, const unsigned* __restrict__ bits, long long words_per_row,
      float* __restrict__ X, int* __restrict__ IDF, int* __restrict__ status) {
    __shared__ int s_nb[kSdfNb];
    __shared__ float4 s_d[kSdfNb];          // D = s_i - s_j (minimum image), w_j - w_i
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
    const float Nf[3] = {(float)D.nx, (float)D.ny, (float)D.nz};
    for (int k = threadIdx.x; k < cnt; k += blockDim.x) {
        const int j = s_nb[k];
        const double wj = weights ? weights[j] : 0.0;
        s_d[k] = make_float4((float)min_image(si[0] - seeds[3 * j], Nd[0]), (float)min_image(si[1] - seeds[3 * j + 1], Nd[1]),
                             (float)min_image(si[2] - seeds[3 * j + 2], Nd[2]), (float)(wj - wi));
    }
    __syncthreads();
    const int A = b.nx * b.ny;
    const int ps = plane_stride(b.nx, b.ny);
    const int ncell = A * b.nz;
    const double eps = (double)D.eps;
    for (int idx = threadIdx.x; idx < ncell; idx += blockDim.x) {
        const int z = idx / A;
        const int rem = idx - z * A;
        const int y = rem / b.nx, x = rem - y * b.nx;
        const double p[3] = {(double)pmod(b.ox + x, D.nx), (double)pmod(b.oy + y, D.ny), (double)pmod(b.oz + z, D.nz)};
        double a0, a1, a2;
        power_dist(p, si, wi, Nd, a0, a1, a2);
        const float af[3] = {(float)a0, (float)a1, (float)a2};
        // FP32 screen: U bounds the exact minimum from above
        const float asum = fabsf(af[0]) + fabsf(af[1]) + fabsf(af[2]);
        auto screen = [&](int k, float& v, float& err) {
            const float4 dk = s_d[k];
            const float dd[3] = {dk.x, dk.y, dk.z};
            float num = -dk.w, den = 0.0f;
            bool near_half = false;                            // image choice too close to call in FP32
#pragma unroll
            for (int c = 0; c < 3; ++c) {
                const float t = af[c] + dd[c];                 // p - s_j before wrapping
                near_half |= fabsf(fabsf(t) - 0.5f * Nf[c]) < 1e-2f;
                const float dc = t > 0.5f * Nf[c] ? dd[c] - Nf[c] : (t < -0.5f * Nf[c] ? dd[c] + Nf[c] : dd[c]);
                num = fmaf(dc, fmaf(2.0f, af[c], dc), num);
                den = fmaf(dc, dc, den);
            }
            const float rinv = rsqrtf(den);
            v = 0.5f * num * rinv;
            // about 64 FP32 ulps of every term of num / (2 |d|), and of v
            err = near_half ? FLT_MAX
                            : 4e-6f * (0.5f * den * rinv + asum + 0.5f * fabsf(dk.w) * rinv + fabsf(v) + 1.0f);
        };
        // one screening pass keeps the neighbours that may still be the minimum
        // (v - err <= the running bound U); a full list falls back to a rescan
        constexpr int kCand = 6;
        int cand[kCand];
        float cand_lo[kCand];
        int n_cand = 0;
        bool rescan = false;
        float U = FLT_MAX;
        for (int k = 0; k < cnt; ++k) {
            float v, err;
            screen(k, v, err);
            U = fminf(U, v + err);
            if (v - err <= U) {
                if (n_cand < kCand) { cand[n_cand] = k; cand_lo[n_cand] = v - err; ++n_cand; }
                else rescan = true;
            }
        }
        // exact evaluation of the candidates (neighbour order decides ties, as in the definition)
        double best = DBL_MAX;
        int arg = -1;
        auto exact = [&](int k) {
            const int j = s_nb[k];
            const double* sj = seeds + 3 * j;
            const double d0 = __dsub_rn(min_image(__dsub_rn(p[0], sj[0]), Nd[0]), a0);
            const double d1 = __dsub_rn(min_image(__dsub_rn(p[1], sj[1]), Nd[1]), a1);
            const double d2 = __dsub_rn(min_image(__dsub_rn(p[2], sj[2]), Nd[2]), a2);
            double num = fma(d0, fma(2.0, a0, d0), fma(d1, fma(2.0, a1, d1), d2 * fma(2.0, a2, d2)));
            if (weights) num -= weights[j] - wi;
            const double ve = num * (0.5 * rsqrt(fma(d0, d0, fma(d1, d1, d2 * d2))));
            if (ve < best) { best = ve; arg = j; }
        };
        if (!rescan) {
            for (int q = 0; q < n_cand; ++q)           // ascending neighbour order
                if (cand_lo[q] <= U) exact(cand[q]);
        } else {
            for (int k = 0; k < cnt; ++k) {
                float v, err;
                screen(k, v, err);
                if (v - err <= U) exact(k);
            }
        }
        const double outv = best == DBL_MAX ? eps : (best < -eps ? -eps : (best > eps ? eps : best));
        const long long o = b.off + (long long)z * ps + rem;
        X[o] = (float)outv;
        if (IDF) IDF[o] = arg;
    }
}

cudaError_t launch_init(const Domain& D, int G, const SeedBins& bins, const double* d_seeds, const double* d_weights,
                        int* d_labels, unsigned* d_bits, long long words_per_row, int* d_bb,
                        Box* d_cur, cudaStream_t s) {
    const long long ncell = (long long)D.nx * D.ny * D.nz;
    int blocks = (int)((ncell + 255) / 256);
    k_labels<<<blocks, 256, 0, s>>>(D, G, bins, d_seeds, d_weights, d_labels);
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
