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

// Visit every seed in the bins that meet [x - r, x + r] on each axis (cyclic;
// a range of a period or more visits the whole axis once).
template <class F>
__device__ __forceinline__ void for_reach(const SeedBins& S, float fx, float fy, float fz, float r, F f) {
    const float c[3] = {fx, fy, fz};
    int lo[3], cnt[3];
#pragma unroll
    for (int a = 0; a < 3; ++a) {
        if (2.0f * r + 2.0f * S.size[a] >= (float)S.nb[a] * S.size[a]) { lo[a] = 0; cnt[a] = S.nb[a]; continue; }
        const int l = (int)floorf((c[a] - r) / S.size[a]);
        const int h = (int)floorf((c[a] + r) / S.size[a]);
        cnt[a] = h - l + 1;
        lo[a] = l;
        if (cnt[a] >= S.nb[a]) { lo[a] = 0; cnt[a] = S.nb[a]; }
        else { lo[a] %= S.nb[a]; if (lo[a] < 0) lo[a] += S.nb[a]; }
    }
    for (int iz = 0; iz < cnt[2]; ++iz) {
        const int bz = wrap_bin(lo[2] + iz, S.nb[2]);
        for (int iy = 0; iy < cnt[1]; ++iy) {
            const int by = wrap_bin(lo[1] + iy, S.nb[1]);
            const int row = (bz * S.nb[1] + by) * S.nb[0];
            for (int ix = 0; ix < cnt[0]; ++ix) {
                const int bin = row + wrap_bin(lo[0] + ix, S.nb[0]);
                for (int q = S.start[bin]; q < S.start[bin + 1]; ++q) f(q);
            }
        }
    }
}

// The label of one cell (see k_labels).
__device__ __forceinline__ int label_cell(const Domain& D, const SeedBins& S, const double* __restrict__ seeds,
                                          const double* __restrict__ weights, long long cell) {
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
    // every seed within the margin of the minimum lies within r of the cell
    const float r = bound < FLT_MAX ? sqrtf(fmaxf(0.0f, bound + margin(bound) + S.wmax)) + 1.0f   // + 1: bin-edge rounding
                                    : FLT_MAX;
    // one pass: the FP32 minimum and the seeds within the margin of the running
    // minimum (a superset of those within the margin of the final one); a
    // full candidate list falls back to a second pass
    constexpr int kCand = 8;
    int cand[kCand];
    float cand_d[kCand];
    int n_cand = 0;
    bool rescan = false;
    float best32 = FLT_MAX;
    for_reach(S, fx, fy, fz, r, [&](int q) {
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
        for_reach(S, fx, fy, fz, r, [&](int q) {
            if (d32(q) <= lim) exact(q);
        });
    }
    return arg;
}

__global__ void __launch_bounds__(256)
k_labels(Domain D, int G, SeedBins S, const double* __restrict__ seeds, const double* __restrict__ weights,
         int* __restrict__ labels) {
    const long long ncell = (long long)D.nx * D.ny * D.nz;
    const long long cell = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (cell >= ncell) return;
    labels[cell] = label_cell(D, S, seeds, weights, cell);
}

// The same labels from a persistent grid whose CTAs first copy the binned
// seeds (points and bin starts) into shared memory: the search's dependent
// loads then come from shared memory instead of L2.
__global__ void __launch_bounds__(512)
k_labels_staged(Domain D, int G, SeedBins S, long long n_bins, const double* __restrict__ seeds,
                const double* __restrict__ weights, int* __restrict__ labels) {
    extern __shared__ __align__(16) unsigned char sm_labels[];
    float4* s_pts = reinterpret_cast<float4*>(sm_labels);
    int* s_start = reinterpret_cast<int*>(s_pts + G);
    for (int i = threadIdx.x; i < G; i += blockDim.x) s_pts[i] = S.pts[i];
    for (long long i = threadIdx.x; i <= n_bins; i += blockDim.x) s_start[i] = S.start[i];
    __syncthreads();
    SeedBins L = S;
    L.pts = s_pts;
    L.start = s_start;
    const long long ncell = (long long)D.nx * D.ny * D.nz;
    for (long long cell = (long long)blockIdx.x * blockDim.x + threadIdx.x; cell < ncell;
         cell += (long long)gridDim.x * blockDim.x)
        labels[cell] = label_cell(D, L, seeds, weights, cell);
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
// (d . (d + 2a) - (w_j - w_i)) / (2 |d|).  Where p - s_j needs no other
// period than D's (every cell of a box small against the domain), d = D and
// the distance is affine in a: n . a + c with n = D / |D| and
// c = |D| / 2 - (w_j - w_i) / (2 |D|), both per pair, computed once per grain
// in FP64.  An FP32 pass over the neighbours (3 FMAs each) finds the
// candidates within a bound of its rounding error of the minimum; those are
// evaluated in FP64 (3 FMAs): the definition's value
// ((p - s_j)^2 - w_j - (p - s_i)^2 + w_i) / (2 |d|) up to FP64 rounding, far
// below the FP32 result's half unit.  Cells where the image of s_j or of s_i
// is too close to call in FP32 take the general form with a per-cell image.
struct SdfPair {
    double n0, n1, n2, c;
};

__global__ void __launch_bounds__(256)
k_sdf(Domain D, int G, const Box* __restrict__ boxes, const double* __restrict__ seeds,
      const double* __restrict__ weights, const unsigned* __restrict__ bits, long long words_per_row,
      float* __restrict__ X, int* __restrict__ IDF, int* __restrict__ status) {
    __shared__ int s_nb[kSdfNb];
    __shared__ float4 s_d[kSdfNb];          // D = s_i - s_j (minimum image), w_j - w_i
    __shared__ float4 s_f[kSdfNb];          // n and c in FP32
    __shared__ SdfPair s_p[kSdfNb];         // n and c in FP64
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
    const int Ni[3] = {D.nx, D.ny, D.nz};
    for (int k = threadIdx.x; k < cnt; k += blockDim.x) {
        const int j = s_nb[k];
        const double wj = weights ? weights[j] : 0.0;
        const double d0 = min_image(si[0] - seeds[3 * j], Nd[0]), d1 = min_image(si[1] - seeds[3 * j + 1], Nd[1]),
                     d2 = min_image(si[2] - seeds[3 * j + 2], Nd[2]);
        s_d[k] = make_float4((float)d0, (float)d1, (float)d2, (float)(wj - wi));
        const double len = sqrt(fma(d0, d0, fma(d1, d1, d2 * d2)));
        SdfPair q;
        q.n0 = d0 / len;
        q.n1 = d1 / len;
        q.n2 = d2 / len;
        q.c = 0.5 * len - 0.5 * (wj - wi) / len;
        s_p[k] = q;
        s_f[k] = make_float4((float)q.n0, (float)q.n1, (float)q.n2, (float)q.c);
    }
    __syncthreads();
    const float sif[3] = {(float)si[0], (float)si[1], (float)si[2]};
    const float nmax = fmaxf(Nf[0], fmaxf(Nf[1], Nf[2]));
    const int A = b.nx * b.ny;
    const int ps = plane_stride(b.nx, b.ny);
    const int ncell = A * b.nz;
    const double eps = (double)D.eps;
    const int o[3] = {b.ox, b.oy, b.oz};
    for (int idx = threadIdx.x; idx < ncell; idx += blockDim.x) {
        const int z = idx / A;
        const int rem = idx - z * A;
        const int y = rem / b.nx, x = rem - y * b.nx;
        const int l[3] = {x, y, z};
        // the cell's global coordinates g and its displacement from s_i: the
        // image decided in FP32 (g - (float)s_i is exact), FP64 only for the value
        int g[3], sh[3];
        float af[3];
        bool amb = false;
#pragma unroll
        for (int c = 0; c < 3; ++c) {
            int gc = o[c] + l[c];
            if (gc >= Ni[c]) gc -= Ni[c];
            g[c] = gc;
            const float raw = (float)gc - sif[c];
            const float h = 0.5f * Nf[c];
            amb |= fabsf(fabsf(raw) - h) < 1e-2f;
            sh[c] = raw > h ? -Ni[c] : (raw < -h ? Ni[c] : 0);
            af[c] = raw + (float)sh[c];
        }
        double a0, a1, a2;
        if (amb) {
            const double p[3] = {(double)g[0], (double)g[1], (double)g[2]};
            power_dist(p, si, wi, Nd, a0, a1, a2);
            af[0] = (float)a0;
            af[1] = (float)a1;
            af[2] = (float)a2;
        } else {
            a0 = __dsub_rn((double)(g[0] + sh[0]), si[0]);
            a1 = __dsub_rn((double)(g[1] + sh[1]), si[1]);
            a2 = __dsub_rn((double)(g[2] + sh[2]), si[2]);
        }
        const float asum = fabsf(af[0]) + fabsf(af[1]) + fabsf(af[2]);
        // whether neighbour k's image for this cell is D's (then the affine form
        // holds); near half a period the general form decides
        auto affine = [&](const float4& dk) {
            bool ok = !amb;
#pragma unroll
            for (int c = 0; c < 3; ++c) {
                const float t = af[c] + (c == 0 ? dk.x : (c == 1 ? dk.y : dk.z));
                ok &= fabsf(t) < 0.5f * Nf[c] - 1e-2f;
            }
            return ok;
        };
        auto screen = [&](int k, float& v, float& err) {
            const float4 dk = s_d[k];
            if (affine(dk)) {
                const float4 f = s_f[k];
                v = fmaf(f.x, af[0], fmaf(f.y, af[1], fmaf(f.z, af[2], f.w)));
                // rounding of s_i, n and c to FP32 and of the three FMAs
                err = 2.4e-7f * (3.0f * nmax + 2.0f * asum + 2.0f * fabsf(f.w) + 4.0f);
                return;
            }
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
            err = near_half || amb ? FLT_MAX
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
            double ve;
            if (affine(s_d[k])) {
                const SdfPair q = s_p[k];
                ve = fma(q.n0, a0, fma(q.n1, a1, fma(q.n2, a2, q.c)));
            } else {
                const double p[3] = {(double)g[0], (double)g[1], (double)g[2]};
                const double* sj = seeds + 3 * j;
                const double d0 = __dsub_rn(min_image(__dsub_rn(p[0], sj[0]), Nd[0]), a0);
                const double d1 = __dsub_rn(min_image(__dsub_rn(p[1], sj[1]), Nd[1]), a1);
                const double d2 = __dsub_rn(min_image(__dsub_rn(p[2], sj[2]), Nd[2]), a2);
                double num = fma(d0, fma(2.0, a0, d0), fma(d1, fma(2.0, a1, d1), d2 * fma(2.0, a2, d2)));
                if (weights) num -= weights[j] - wi;
                ve = num * (0.5 * rsqrt(fma(d0, d0, fma(d1, d1, d2 * d2))));
            }
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
        const long long off = b.off + (long long)z * ps + rem;
        X[off] = (float)outv;
        if (IDF) IDF[off] = arg;
    }
}

cudaError_t launch_init(const Domain& D, int G, const SeedBins& bins, const double* d_seeds, const double* d_weights,
                        int* d_labels, unsigned* d_bits, long long words_per_row, int* d_bb,
                        Box* d_cur, cudaStream_t s) {
    const long long ncell = (long long)D.nx * D.ny * D.nz;
    // the binned seeds in shared memory when they fit, else read from global memory
    const long long n_bins = (long long)bins.nb[0] * bins.nb[1] * bins.nb[2];
    const size_t staged = (size_t)G * sizeof(float4) + (size_t)(n_bins + 1) * sizeof(int);
    int dev = 0, n_sm = 0, optin = 0, occ = 0;
    bool use_staged = cudaGetDevice(&dev) == cudaSuccess &&
                      cudaDeviceGetAttribute(&n_sm, cudaDevAttrMultiProcessorCount, dev) == cudaSuccess &&
                      cudaDeviceGetAttribute(&optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev) == cudaSuccess &&
                      staged <= (size_t)optin &&
                      cudaFuncSetAttribute(k_labels_staged, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                           (int)staged) == cudaSuccess &&
                      cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, k_labels_staged, 512, staged) ==
                          cudaSuccess &&
                      occ > 0;
    if (use_staged) {
        k_labels_staged<<<n_sm * occ, 512, staged, s>>>(D, G, bins, n_bins, d_seeds, d_weights, d_labels);
    } else {
        cudaGetLastError();                      // a refused attribute leaves no error behind
        int blocks = (int)((ncell + 255) / 256);
        k_labels<<<blocks, 256, 0, s>>>(D, G, bins, d_seeds, d_weights, d_labels);
    }
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

// ---------------------------------------------------------------------------
// initialisation from a label field
// ---------------------------------------------------------------------------
// Per grain and axis, the positions holding one of its cells, as bits
// (words of 32 positions per (grain, axis)).
__global__ void k_label_occupancy(Domain D, const int* __restrict__ labels, unsigned* __restrict__ occ, int words) {
    const long long ncell = (long long)D.nx * D.ny * D.nz;
    const int N[3] = {D.nx, D.ny, D.nz};
    for (long long cell = (long long)blockIdx.x * blockDim.x + threadIdx.x; cell < ncell;
         cell += (long long)gridDim.x * blockDim.x) {
        const int c[3] = {(int)(cell % D.nx), (int)((cell / D.nx) % D.ny), (int)(cell / ((long long)D.nx * D.ny))};
        const long long i = labels[cell];
#pragma unroll
        for (int a = 0; a < 3; ++a)
            if (N[a] > 1) atomicOr(&occ[(i * 3 + a) * words + (c[a] >> 5)], 1u << (c[a] & 31));
    }
}

// Grain i's box from its label cells: per axis the shortest cyclic interval
// holding every occupied position -- the complement of the longest run of
// empty positions, the first such run (smallest start) on ties -- grown by
// the halo and capped at the axis; no cell: extinct.
__global__ void k_label_boxes(Domain D, int G, const unsigned* __restrict__ occ, int words, Box* __restrict__ cur) {
    const int N[3] = {D.nx, D.ny, D.nz};
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < G; i += gridDim.x * blockDim.x) {
        const unsigned* ox = occ + ((long long)i * 3) * words;
        bool any = false;
        for (int w = 0; w < words; ++w) any = any || ox[w] != 0u;
        Box b{};
        if (!any) {
            cur[i] = b;
            continue;
        }
        int o[3], n[3];
        for (int a = 0; a < 3; ++a) {
            const int na = N[a];
            if (na == 1) { o[a] = 0; n[a] = 1; continue; }
            const unsigned* bits = occ + ((long long)i * 3 + a) * words;
            auto at = [&](int p) { return (bits[p >> 5] >> (p & 31)) & 1u; };
            int best_start = 0, best_len = -1;
            for (int p = 0; p < na; ++p) {
                if (at(p) || !at(p == 0 ? na - 1 : p - 1)) continue;   // not the first empty position of a run
                int len = 0;
                while (len < na && !at((p + len) % na)) ++len;
                if (len > best_len) { best_start = p; best_len = len; }
            }
            int start = 0, length = na;                            // every position held
            if (best_len > 0) {
                start = (best_start + best_len) % na;
                length = na - best_len;
            }
            n[a] = length + 2 * D.halo < na ? length + 2 * D.halo : na;
            o[a] = pmod(start - D.halo, na);
        }
        b.ox = o[0]; b.oy = o[1]; b.oz = o[2];
        b.nx = n[0]; b.ny = n[1]; b.nz = n[2];
        cur[i] = b;
    }
}

// The starting function before the re-initialisation: +1/2 on the grain's
// label cells and -1/2 on the other cells of its box (`cur` layout, FP32).
__global__ void k_label_phi(Domain D, const Box* __restrict__ cur, const int* __restrict__ labels,
                            float* __restrict__ Z) {
    const int i = blockIdx.x;
    const Box b = cur[i];
    if (b.nx <= 0) return;
    const int ps = plane_stride(b.nx, b.ny);
    const int A = b.nx * b.ny;
    const long long n = (long long)A * b.nz;
    for (long long k = threadIdx.x; k < n; k += blockDim.x) {
        const int z = (int)(k / A), rem = (int)(k - (long long)z * A);
        const int y = rem / b.nx, x = rem - y * b.nx;
        const long long g = ((long long)pmod(b.oz + z, D.nz) * D.ny + pmod(b.oy + y, D.ny)) * D.nx + pmod(b.ox + x, D.nx);
        Z[b.off + (long long)z * ps + rem] = labels[g] == i ? 0.5f : -0.5f;
    }
}

cudaError_t launch_label_boxes(const Domain& D, int G, const int* d_labels, unsigned* d_occ, int words, Box* d_cur,
                               cudaStream_t s) {
    cudaError_t e = cudaMemsetAsync(d_occ, 0, (size_t)G * 3 * words * sizeof(unsigned), s);
    if (e != cudaSuccess) return e;
    const long long ncell = (long long)D.nx * D.ny * D.nz;
    long long gs = (ncell + 255) / 256;
    if (gs > 65535 * 8) gs = 65535 * 8;
    k_label_occupancy<<<(int)gs, 256, 0, s>>>(D, d_labels, d_occ, words);
    k_label_boxes<<<(G + 127) / 128, 128, 0, s>>>(D, G, d_occ, words, d_cur);
    return cudaGetLastError();
}

cudaError_t launch_label_phi(const Domain& D, int G, const Box* d_cur, const int* d_labels, float* Z, cudaStream_t s) {
    k_label_phi<<<G, 256, 0, s>>>(D, d_cur, d_labels, Z);
    return cudaGetLastError();
}

cudaError_t launch_sdf(const Domain& D, int G, const Box* d_cur, const double* d_seeds, const double* d_weights,
                       const unsigned* d_bits, long long words_per_row, float* X, int* IDF, int* d_status,
                       cudaStream_t s) {
    k_sdf<<<G, 256, 0, s>>>(D, G, d_cur, d_seeds, d_weights, d_bits, words_per_row, X, IDF, d_status);
    return cudaGetLastError();
}

}  // namespace lsgg
