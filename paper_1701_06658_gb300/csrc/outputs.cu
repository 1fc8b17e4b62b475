// Outputs of a microstructure.
//
//   k_volumes   V_i = sum_x H(phi_i(x)), H(phi) = clamp(phi + 1/2, 0, 1): one CTA
//               per box over the state's own layout (`prev`), 16-byte loads,
//               four in flight per thread.  Each thread sums its cells in
//               fixed point (H in units of 2^-28 is an integer, exactly for
//               every |phi| >= 2^-5 and to 2^-29 below, so the 64-bit sum is
//               exact); the threads' partials are merged in FP64 with
//               compensated (TwoSum) additions in a fixed tree order.  For a
//               box of fewer than 2^25 cells every partial sum is an integer
//               multiple of 2^-28 below 2^25, exact in FP64, so the result is
//               the exact sum whatever the cells' order; larger boxes keep the
//               compensated sum's rounding, the same on every run.
//   k_owner_*   owner(x) = argmax_i phi_i(x) over boxes covering x, lowest id on
//               ties (64-bit atomicMax of (phi, -id) keys), -1 where uncovered.
//   k_remap     the state phi (stored in the `prev` layout) resampled on the
//               current boxes with -eps where the old box did not reach: the
//               grain functions as they enter the next step (Sec. 3.1 box update).
#include <algorithm>

#include "lsgg_internal.cuh"
#include "../../include/lsgg.h"

namespace lsgg {

__device__ __forceinline__ void two_sum(double a, double b, double& s, double& e) {
    s = __dadd_rn(a, b);
    double bb = __dsub_rn(s, a);
    e = __dadd_rn(__dsub_rn(a, __dsub_rn(s, bb)), __dsub_rn(b, bb));
}

// Value of grain b's function at a cell of its current box (local x, y, z):
// read from the prev layout, -eps outside the prev box.
__device__ __forceinline__ float state_value(const Domain& D, const Box& nb, const Box& ob, const float* X,
                                             int x, int y, int z) {
    int lx = pmod(nb.ox + x - ob.ox, D.nx);
    int ly = pmod(nb.oy + y - ob.oy, D.ny);
    int lz = pmod(nb.oz + z - ob.oz, D.nz);
    if (lx >= ob.nx || ly >= ob.ny || lz >= ob.nz) return -D.eps;
    return X[ob.off + (long long)lz * plane_stride(ob.nx, ob.ny) + ly * ob.nx + lx];
}

// H of one cell in units of 2^-28 (an integer: exact for every |phi| >=
// 2^-5 and to 2^-29 below); no cell (phi = -1 here) gives 0.
__device__ __forceinline__ long long vol_units(float v) {
    constexpr float kScale = 268435456.0f;           // 2^28
    constexpr int kHalf = 1 << 27, kOne = 1 << 28;
    const int q = __float2int_rn(v * kScale);        // |phi| <= eps: no overflow
    return min(max(q + kHalf, 0), kOne);
}

constexpr int kVolLoads = 4;     // 16-byte loads in flight per thread

// Sum of H over one box in its layout (planes of A cells at stride ps, each
// starting on a 32-byte boundary), as (plane, group of four cells) items,
// kVolLoads of them per thread loaded together.  The sum is of integers:
// the same in any order.  I: the index type (32-bit divisions whenever the
// items fit).
template <class I>
__device__ __forceinline__ long long volume_walk(const float* base, int A, int ps, int nz) {
    const I nq = (I)((A + 3) >> 2);
    const I items = nq * (I)nz;
    long long acc = 0;
    for (I i0 = threadIdx.x; i0 < items; i0 += (I)kVolLoads * blockDim.x) {
        float v[kVolLoads][4];
#pragma unroll
        for (int k = 0; k < kVolLoads; ++k) {
            const I it = i0 + (I)k * blockDim.x;
            const I z = it < items ? it / nq : 0;
            const int q = it < items ? 4 * (int)(it - z * nq) : 0;
            const float* pl = base + (long long)z * ps;
            if (it < items && q + 3 < A) {
                const float4 w4 = __ldg(reinterpret_cast<const float4*>(pl + q));
                v[k][0] = w4.x; v[k][1] = w4.y; v[k][2] = w4.z; v[k][3] = w4.w;
            } else {
#pragma unroll
                for (int u = 0; u < 4; ++u) v[k][u] = it < items && q + u < A ? __ldg(pl + q + u) : -1.0f;
            }
        }
#pragma unroll
        for (int k = 0; k < kVolLoads; ++k)
#pragma unroll
            for (int u = 0; u < 4; ++u) acc += vol_units(v[k][u]);
    }
    return acc;
}

// The state lives in the `prev` layout; a cell of the prev box outside the
// current box is at least halo + 1 cells from every positive cell, so its
// phi <= -halo and H = 0: summing the prev box is summing the current box.
__global__ void __launch_bounds__(256)
k_volumes(Domain D, const Box* __restrict__ cur, const Box* __restrict__ prev, const float* __restrict__ X,
          double* __restrict__ out) {
    __shared__ double s_s[256], s_c[256];
    const int b = blockIdx.x;
    constexpr int kOne = 1 << 28;
    long long acc = 0;
    if (cur[b].nx > 0) {
        const Box ob = prev[b];
        const int A = ob.nx * ob.ny, ps = plane_stride(ob.nx, ob.ny);
        if ((long long)((A + 3) >> 2) * ob.nz < (1LL << 31) - 4LL * kVolLoads * 256)
            acc = volume_walk<unsigned>(X + ob.off, A, ps, ob.nz);
        else
            acc = volume_walk<long long>(X + ob.off, A, ps, ob.nz);
    }
    s_s[threadIdx.x] = (double)acc / (double)kOne;   // exact: acc < 2^53
    s_c[threadIdx.x] = 0.0;
    __syncthreads();
    for (int o = blockDim.x / 2; o > 0; o >>= 1) {
        if (threadIdx.x < (unsigned)o) {
            double t, e;
            two_sum(s_s[threadIdx.x], s_s[threadIdx.x + o], t, e);
            s_s[threadIdx.x] = t;
            s_c[threadIdx.x] = __dadd_rn(__dadd_rn(s_c[threadIdx.x], s_c[threadIdx.x + o]), e);
        }
        __syncthreads();
    }
    if (threadIdx.x == 0) out[b] = __dadd_rn(s_s[0], s_c[0]);
}

__global__ void __launch_bounds__(256)
k_owner_scatter(Domain D, const Box* __restrict__ cur, const Box* __restrict__ prev, const float* __restrict__ X,
                unsigned long long* __restrict__ F) {
    const int b = blockIdx.x;
    const Box nb = cur[b];
    if (nb.nx <= 0) return;
    const Box ob = prev[b];
    const long long A = (long long)nb.nx * nb.ny;
    const long long n = A * nb.nz;
    for (long long i = threadIdx.x; i < n; i += blockDim.x) {
        int z = (int)(i / A);
        int rem = (int)(i - z * A);
        int y = rem / nb.nx, x = rem - y * nb.nx;
        float v = state_value(D, nb, ob, X, x, y, z);
        long long g = ((long long)pmod(nb.oz + z, D.nz) * D.ny + pmod(nb.oy + y, D.ny)) * D.nx + pmod(nb.ox + x, D.nx);
        atomicMax(&F[g], make_key(v, b));
    }
}

__global__ void k_owner_decode(long long n, const unsigned long long* __restrict__ F, int* __restrict__ out) {
    for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x)
        out[i] = key_id(F[i]);
}

// Packed copy of the state on the current boxes (grain-id order, x fastest, no padding).
__global__ void __launch_bounds__(256)
k_pack_state(Domain D, const Box* __restrict__ cur, const Box* __restrict__ prev, const float* __restrict__ X,
             const long long* __restrict__ packed_off, float* __restrict__ out) {
    const int b = blockIdx.x;
    const Box nb = cur[b];
    if (nb.nx <= 0) return;
    const Box ob = prev[b];
    const long long A = (long long)nb.nx * nb.ny;
    const long long n = A * nb.nz;
    for (long long i = threadIdx.x; i < n; i += blockDim.x) {
        int z = (int)(i / A);
        int rem = (int)(i - z * A);
        int y = rem / nb.nx, x = rem - y * nb.nx;
        out[packed_off[b] + i] = state_value(D, nb, ob, X, x, y, z);
    }
}

// Packed copy of a cur-layout arena (debug intermediates); `ints` selects int32 data.
__global__ void __launch_bounds__(256)
k_pack_cur(const Box* __restrict__ cur, const void* __restrict__ arena, const long long* __restrict__ packed_off,
           void* __restrict__ out) {
    const int b = blockIdx.x;
    const Box nb = cur[b];
    if (nb.nx <= 0) return;
    const long long A = (long long)nb.nx * nb.ny;
    const long long n = A * nb.nz;
    const int ps = plane_stride(nb.nx, nb.ny);
    const unsigned* src = reinterpret_cast<const unsigned*>(arena);
    unsigned* dst = reinterpret_cast<unsigned*>(out);
    for (long long i = threadIdx.x; i < n; i += blockDim.x) {
        long long z = i / A, rem = i - z * A;
        dst[packed_off[b] + i] = src[nb.off + z * ps + rem];
    }
}

// Unpack host-given state into the arena (cur layout) and set prev = cur.
__global__ void __launch_bounds__(256)
k_unpack_state(const Box* __restrict__ cur, const float* __restrict__ packed, const int* __restrict__ packed_idf,
               const long long* __restrict__ packed_off, float* __restrict__ X, int* __restrict__ IDF) {
    const int b = blockIdx.x;
    const Box nb = cur[b];
    if (nb.nx <= 0) return;
    const long long A = (long long)nb.nx * nb.ny;
    const long long n = A * nb.nz;
    const int ps = plane_stride(nb.nx, nb.ny);
    for (long long i = threadIdx.x; i < n; i += blockDim.x) {
        long long z = i / A, rem = i - z * A;
        long long o = nb.off + z * ps + rem;
        X[o] = packed[packed_off[b] + i];
        if (IDF) IDF[o] = packed_idf ? packed_idf[packed_off[b] + i] : -1;
    }
}

cudaError_t launch_volumes(const Domain& D, int G, const Box* cur, const Box* prev, const float* X, double* out,
                           cudaStream_t s) {
    k_volumes<<<G, 256, 0, s>>>(D, cur, prev, X, out);
    return cudaGetLastError();
}

cudaError_t launch_owner(const Domain& D, int G, const Box* cur, const Box* prev, const float* X,
                         unsigned long long* F, int* out, cudaStream_t s) {
    long long n = (long long)D.nx * D.ny * D.nz;
    cudaError_t e = cudaMemsetAsync(F, 0, (size_t)n * 8, s);
    if (e != cudaSuccess) return e;
    k_owner_scatter<<<G, 256, 0, s>>>(D, cur, prev, X, F);
    int blocks = (int)((n + 255) / 256);
    if (blocks > 65535 * 16) blocks = 65535 * 16;
    k_owner_decode<<<blocks, 256, 0, s>>>(n, F, out);
    return cudaGetLastError();
}

// The status of the steps enqueued so far, read on the device: their error
// code, LSGG_ERR_CAPACITY for a step stopped on a full box arena (lsgg_sync
// grows it and finishes the steps), else 0.
__global__ void k_step_status(const StepState* __restrict__ st, int* __restrict__ out) {
    const int status = *(volatile const int*)&st->status, halt = *(volatile const int*)&st->halt;
    *out = status ? status : (halt ? LSGG_ERR_CAPACITY : 0);
}

cudaError_t launch_step_status(const StepState* st, int* out, cudaStream_t s) {
    k_step_status<<<1, 1, 0, s>>>(st, out);
    return cudaGetLastError();
}

cudaError_t launch_pack_state(const Domain& D, int G, const Box* cur, const Box* prev, const float* X,
                              const long long* packed_off, float* out, cudaStream_t s) {
    k_pack_state<<<G, 256, 0, s>>>(D, cur, prev, X, packed_off, out);
    return cudaGetLastError();
}

cudaError_t launch_pack_cur(int G, const Box* cur, const void* arena, const long long* packed_off, void* out,
                            cudaStream_t s) {
    k_pack_cur<<<G, 256, 0, s>>>(cur, arena, packed_off, out);
    return cudaGetLastError();
}

cudaError_t launch_unpack_state(int G, const Box* cur, const float* packed, const int* packed_idf,
                                const long long* packed_off, float* X, int* IDF, cudaStream_t s) {
    k_unpack_state<<<G, 256, 0, s>>>(cur, packed, packed_idf, packed_off, X, IDF);
    return cudaGetLastError();
}

// Whole-arena conversions of the BF16 state (LSGG_STORAGE_BF16) to and from
// FP32: the outputs and the test hooks read and write FP32 through them.
__global__ void __launch_bounds__(256) k_state_to_f32(const __nv_bfloat16* __restrict__ in, float* __restrict__ out,
                                                      long long n) {
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x)
        out[i] = __bfloat162float(in[i]);
}
__global__ void __launch_bounds__(256) k_f32_to_state(const float* __restrict__ in, __nv_bfloat16* __restrict__ out,
                                                      long long n) {
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x)
        out[i] = __float2bfloat16_rn(in[i]);
}
cudaError_t launch_state_to_f32(const void* bf16_in, float* out, long long n, cudaStream_t s) {
    const long long blocks = std::min<long long>((n + 255) / 256, 4096);
    k_state_to_f32<<<(int)std::max<long long>(blocks, 1), 256, 0, s>>>(static_cast<const __nv_bfloat16*>(bf16_in), out, n);
    return cudaGetLastError();
}
cudaError_t launch_f32_to_state(const float* in, void* bf16_out, long long n, cudaStream_t s) {
    const long long blocks = std::min<long long>((n + 255) / 256, 4096);
    k_f32_to_state<<<(int)std::max<long long>(blocks, 1), 256, 0, s>>>(in, static_cast<__nv_bfloat16*>(bf16_out), n);
    return cudaGetLastError();
}

// Grain statistics (Sec. 5's size analysis) from the volumes, one CTA:
// per-thread partial sums over grains t, t + blockDim, ... in FP64, merged by
// compensated additions in a fixed tree order; bins counted with integer
// atomics (order-free); out = alive, mean V, mean R, rms R, max R, overflow.
constexpr int kStatsThreads = 1024;
constexpr int kStatsMaxBins = 4096;

__global__ void __launch_bounds__(kStatsThreads)
k_grain_stats(const double* __restrict__ vol, int G, int dim, int n_bins, double r_max, double* __restrict__ out,
              double* __restrict__ hist) {
    __shared__ double s_s[4][kStatsThreads], s_c[4][kStatsThreads];
    __shared__ unsigned s_bins[kStatsMaxBins + 1];
    const int t = threadIdx.x;
    // 0: count, 1: sum V, 2: sum R, 3: sum R^2 (running compensated per thread)
    double sum[4] = {0.0, 0.0, 0.0, 0.0}, comp[4] = {0.0, 0.0, 0.0, 0.0}, rmax = 0.0;
    for (int k = t; k <= n_bins; k += blockDim.x) s_bins[k] = 0u;
    for (int i = t; i < G; i += blockDim.x) {
        const double v = vol[i];
        if (!(v > 0.0)) continue;
        const double r = dim == 3 ? cbrt(3.0 * v / (4.0 * 3.14159265358979323846)) : sqrt(v / 3.14159265358979323846);
        const double x[4] = {1.0, v, r, r * r};
#pragma unroll
        for (int q = 0; q < 4; ++q) {
            double s2, e;
            two_sum(sum[q], x[q], s2, e);
            sum[q] = s2;
            comp[q] = __dadd_rn(comp[q], e);
        }
        rmax = fmax(rmax, r);
    }
#pragma unroll
    for (int q = 0; q < 4; ++q) { s_s[q][t] = sum[q]; s_c[q][t] = comp[q]; }
    __syncthreads();
    for (int o = blockDim.x / 2; o > 0; o >>= 1) {
        if (t < o) {
#pragma unroll
            for (int q = 0; q < 4; ++q) {
                double s2, e;
                two_sum(s_s[q][t], s_s[q][t + o], s2, e);
                s_s[q][t] = s2;
                s_c[q][t] = __dadd_rn(__dadd_rn(s_c[q][t], s_c[q][t + o]), e);
            }
        }
        __syncthreads();
    }
    __shared__ double s_max[kStatsThreads];
    s_max[t] = rmax;
    __syncthreads();
    for (int o = blockDim.x / 2; o > 0; o >>= 1) {
        if (t < o) s_max[t] = fmax(s_max[t], s_max[t + o]);
        __syncthreads();
    }
    const double n = __dadd_rn(s_s[0][0], s_c[0][0]);
    const double mean_r = n > 0.0 ? __dadd_rn(s_s[2][0], s_c[2][0]) / n : 0.0;
    for (int i = t; i < G; i += blockDim.x) {
        const double v = vol[i];
        if (!(v > 0.0)) continue;
        const double r = dim == 3 ? cbrt(3.0 * v / (4.0 * 3.14159265358979323846)) : sqrt(v / 3.14159265358979323846);
        const double k = floor(r / mean_r / r_max * (double)n_bins);
        atomicAdd(&s_bins[k < (double)n_bins ? (int)k : n_bins], 1u);
    }
    __syncthreads();
    if (t == 0) {
        out[0] = n;
        out[1] = n > 0.0 ? __dadd_rn(s_s[1][0], s_c[1][0]) / n : 0.0;
        out[2] = mean_r;
        const double msq = n > 0.0 ? __dadd_rn(s_s[3][0], s_c[3][0]) / n : 0.0;
        out[3] = sqrt(msq);
        out[4] = s_max[0];
        out[5] = n > 0.0 ? (double)s_bins[n_bins] / n : 0.0;
        out[6] = msq > 0.0 ? mean_r * mean_r / msq : 0.0;            // rho = <R>^2 / <R^2>
        out[7] = mean_r > 0.0 ? msq / (mean_r * mean_r) - 1.0 : 0.0;  // Var(R / <R>) = 1 / rho - 1
    }
    for (int k = t; k < n_bins; k += blockDim.x) hist[k] = n > 0.0 ? (double)s_bins[k] / n : 0.0;
}

// Texture shares: per class c < n_classes, the summed volume of its grains
// over the summed volume of all grains, each sum compensated (TwoSum) per
// thread and merged in a fixed tree order (deterministic).  One CTA; out:
// n_classes + 1 doubles (the last: the total volume).
__global__ void __launch_bounds__(kStatsThreads)
k_texture_shares(const double* __restrict__ vol, const int* __restrict__ cls, int G, int n_classes,
                 double* __restrict__ out) {
    __shared__ double s_s[kStatsThreads], s_c[kStatsThreads];
    const int t = threadIdx.x;
    for (int c = -1; c < n_classes; ++c) {            // c = -1: all grains
        double sum = 0.0, comp = 0.0;
        for (int i = t; i < G; i += blockDim.x) {
            const double v = vol[i];
            if (!(v > 0.0) || (c >= 0 && cls[i] != c)) continue;
            double s2, e;
            two_sum(sum, v, s2, e);
            sum = s2;
            comp = __dadd_rn(comp, e);
        }
        s_s[t] = sum;
        s_c[t] = comp;
        __syncthreads();
        for (int o = blockDim.x / 2; o > 0; o >>= 1) {
            if (t < o) {
                double s2, e;
                two_sum(s_s[t], s_s[t + o], s2, e);
                s_s[t] = s2;
                s_c[t] = __dadd_rn(__dadd_rn(s_c[t], s_c[t + o]), e);
            }
            __syncthreads();
        }
        if (t == 0) out[c < 0 ? n_classes : c] = __dadd_rn(s_s[0], s_c[0]);
        __syncthreads();
    }
    if (t == 0) {
        const double tot = out[n_classes];
        for (int c = 0; c < n_classes; ++c) out[c] = tot > 0.0 ? out[c] / tot : 0.0;
    }
}

cudaError_t launch_texture_shares(const double* vol, const int* cls, int G, int n_classes, double* out,
                                  cudaStream_t s) {
    k_texture_shares<<<1, kStatsThreads, 0, s>>>(vol, cls, G, n_classes, out);
    return cudaGetLastError();
}

cudaError_t launch_grain_stats(const double* vol, int G, int dim, int n_bins, double r_max, double* out,
                               double* hist, cudaStream_t s) {
    if (n_bins < 1 || n_bins > kStatsMaxBins) return cudaErrorInvalidValue;
    k_grain_stats<<<1, kStatsThreads, 0, s>>>(vol, G, dim, n_bins, r_max, out, hist);
    return cudaGetLastError();
}

}  // namespace lsgg
