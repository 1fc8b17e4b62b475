// One time step of Algorithm 1 on the packed box list (batched path).
//
//   k_predict   Sec. 2.1.4, Eqs. (7)-(10): phi_p = G(dt) * phi (separable,
//               x -> y in shared memory per plane, z over a ring of 2R+1
//               planes while streaming the box along z), optional velocity
//               correction, clamp to [-eps, eps]; the result is written in
//               the box's new layout and scattered into the neighbour-max
//               field T (two 64-bit atomicMax per cell: top-1 and top-2).
//   k_correct   Sec. 2.1.5, Eq. (16) and Sec. 2.1.6: phi_c = (phi_p - m) / 2
//               with m = max_{j != i} phi_p_j read from T; reference cells and
//               their planar-exact distances; taxicab distance as a
//               sign-blocked min-plus transform, x and y in the plane, z as a
//               forward sweep plus a 6-plane backward window; clamp; positive
//               bounding box of the box.
//   k_box_update  Secs. 2.1.3 / 3.1: new box = bbox{phi > 0} + halo, arena
//               offsets by a block-wide scan, size classes and work queues.
//
// One CTA owns one box at a time and streams it plane by plane; CTAs of a
// size class pull boxes from a device queue (persistent grid).  Outside its
// box a grain's function is -eps (Fig. 1 caption); a box axis that spans the
// domain is periodic.
#include <cfloat>
#include <climits>

#include "lsgg_internal.cuh"
#include "group.cuh"
#include "kernels_common.cuh"
#include "../../include/lsgg.h"

namespace lsgg {

constexpr int kThreads = 256;
constexpr int kBoxUpdateThreads = 1024;

// ---------------------------------------------------------------------------
// predictor + neighbour-max scatter
// ---------------------------------------------------------------------------

struct PredictSmem {   // carved from dynamic shared memory (maps) + a float buffer
    int* mapx;         // [nx + 2R] old-box local x (or -1) for padded new-box x
    int* mapy;         // [ny + 2R]
    int* gx;           // [nx] global x of new-box cells
    int* gy;           // [ny]
};

__device__ void predict_box(const StepBuffers& B, const Taps& taps, const PhysicsDev& phys,
                            int b, const PredictSmem& sm, float* buf, const PairTable& tab) {
    const Domain& D = B.dom;
    const Box nb = B.cur[b];
    const Box ob = B.prev[b];
    const int nx = nb.nx, ny = nb.ny, nz = nb.nz;
    const int R = taps.radius;
    const int W = 2 * R + 1;
    const int px = nx + 2 * R, py = ny + 2 * R;
    const int A = nx * ny;
    const bool fx = nx == D.nx, fy = ny == D.ny, fz = nz == D.nz;
    const float eps = D.eps;

    float* P = buf;                       // (ny+2R) x (nx+2R) staged input plane
    float* Xp = P + (size_t)px * py;      // (ny+2R) x nx after the x pass
    float* ring = Xp + (size_t)nx * py;   // W planes of nx*ny after the y pass

    for (int i = threadIdx.x; i < px; i += blockDim.x) {
        int xl = i - R, v = -1;
        bool ok = fx || (xl >= 0 && xl < nx);
        if (ok) {
            if (fx) xl = pmod(xl, nx);
            int ol = pmod(nb.ox + xl - ob.ox, D.nx);
            v = ol < ob.nx ? ol : -1;
        }
        sm.mapx[i] = v;
    }
    for (int i = threadIdx.x; i < py; i += blockDim.x) {
        int yl = i - R, v = -1;
        bool ok = fy || (yl >= 0 && yl < ny);
        if (ok) {
            if (fy) yl = pmod(yl, ny);
            int ol = pmod(nb.oy + yl - ob.oy, D.ny);
            v = ol < ob.ny ? ol : -1;
        }
        sm.mapy[i] = v;
    }
    for (int i = threadIdx.x; i < nx; i += blockDim.x) sm.gx[i] = pmod(nb.ox + i, D.nx);
    for (int i = threadIdx.x; i < ny; i += blockDim.x) sm.gy[i] = pmod(nb.oy + i, D.ny);
    __syncthreads();

    const int ps_old = plane_stride(ob.nx, ob.ny);
    const int ps_new = plane_stride(nx, ny);
    const bool is3d = D.dim == 3;
    const int zlo = is3d ? -R : 0, zhi = is3d ? nz + R : 1;

    for (int zin = zlo; zin < zhi; ++zin) {
        // ---- stage plane zin (new-box local z), masked by both boxes ----
        int zold = -1;
        {
            bool ok = !is3d || fz || (zin >= 0 && zin < nz);
            if (ok) {
                int zl = is3d && fz ? pmod(zin, nz) : zin;
                int ol = is3d ? pmod(nb.oz + zl - ob.oz, D.nz) : 0;
                zold = ol < ob.nz ? ol : -1;
            }
        }
        const long long src = ob.off + (long long)(zold < 0 ? 0 : zold) * ps_old;
        for (int idx = threadIdx.x; idx < px * py; idx += blockDim.x) {
            int yp = idx / px, xp = idx - yp * px;
            int mx = sm.mapx[xp], my = sm.mapy[yp];
            float v = -eps;
            if (zold >= 0 && mx >= 0 && my >= 0) v = ld_state(B, src + my * ob.nx + mx);
            P[idx] = v;
        }
        __syncthreads();
        // ---- x pass ----
        for (int idx = threadIdx.x; idx < nx * py; idx += blockDim.x) {
            int yp = idx / nx, x = idx - yp * nx;
            const float* row = P + yp * px + x;
            float acc = 0.0f;
#pragma unroll
            for (int k = 0; k < kMaxTaps; ++k)
                if (k < W) acc = fmaf(taps.g[k], row[k], acc);
            Xp[idx] = acc;
        }
        __syncthreads();
        // ---- y pass -> ring slot of plane zin ----
        float* slot = ring + (size_t)(is3d ? pmod(zin, W) : 0) * A;
        for (int idx = threadIdx.x; idx < A; idx += blockDim.x) {
            int y = idx / nx, x = idx - y * nx;
            const float* col = Xp + y * nx + x;
            float acc = 0.0f;
#pragma unroll
            for (int k = 0; k < kMaxTaps; ++k)
                if (k < W) acc = fmaf(taps.g[k], col[k * nx], acc);
            slot[idx] = acc;
        }
        __syncthreads();
        // ---- z pass for output plane zo = zin - R ----
        const int zo = is3d ? zin - R : 0;
        if (zo < 0) continue;
        const int gz = is3d ? pmod(nb.oz + zo, D.nz) : 0;
        float* dst = B.Y + nb.off + (long long)zo * ps_new;
        for (int idx = threadIdx.x; idx < A; idx += blockDim.x) {
            float c;
            if (is3d) {
                c = 0.0f;
#pragma unroll
                for (int k = 0; k < kMaxTaps; ++k)
                    if (k < W) c = fmaf(taps.g[k], ring[(size_t)pmod(zo - R + k, W) * A + idx], c);
            } else {
                c = slot[idx];
            }
            int y = idx / nx, x = idx - y * nx;
            float v = c;
            if (phys.kind != LSGG_PHYSICS_IDEAL) {
                int zl = zo;
                int zo_old = is3d ? pmod(nb.oz + zl - ob.oz, D.nz) : 0;
                int mx = sm.mapx[x + R], my = sm.mapy[y + R];
                float phi0 = -eps;
                int j = -1;
                if (zo_old < ob.nz && mx >= 0 && my >= 0) {
                    long long o = ob.off + (long long)zo_old * ps_old + my * ob.nx + mx;
                    phi0 = ld_state(B, o);
                    j = B.IDF[o];
                }
                v = pair_blend(phys, tab, b, j, phi0, c);
            }
            v = fminf(fmaxf(v, -eps), eps);
            dst[idx] = v;
            if (!B.use_passes) {        // the pass path's field pass builds T instead
                long long g = ((long long)gz * D.ny + sm.gy[y]) * D.nx + sm.gx[x];
                unsigned long long key = make_key(v, b);
                unsigned long long old = atomicMax(&B.T[2 * g], key);
                if (old) atomicMax(&B.T[2 * g + 1], old < key ? old : key);
            }
        }
        // no barrier needed: the next writes into `ring` happen after two barriers
    }
    __syncthreads();
}

__global__ void __launch_bounds__(kThreads)
k_predict(StepBuffers B, Taps taps, PhysicsDev phys, int cls) {
    extern __shared__ __align__(16) unsigned char smem_raw[];
    __shared__ int s_box;
    const int side = B.class_side[cls];
    PredictSmem sm;
    sm.mapx = reinterpret_cast<int*>(smem_raw);
    sm.mapy = sm.mapx + side + 2 * kMaxRadius;
    sm.gx = sm.mapy + side + 2 * kMaxRadius;
    sm.gy = sm.gx + side;
    float* buf = reinterpret_cast<float*>(sm.gy + side + 4);
    buf = reinterpret_cast<float*>((reinterpret_cast<uintptr_t>(buf) + 15) & ~uintptr_t(15));
    if (B.mode[cls] == 2) buf = B.scratch + B.scratch_class_off[cls] + (long long)blockIdx.x * B.scratch_per_cta;
    __shared__ int s_tj[kNbCap];
    __shared__ float s_tw[kNbCap], s_tm[kNbCap];
    for (;;) {
        int b = pull_box(B, 0, cls, &s_box);
        if (b < 0) break;
        const PairTable tab = load_pair_table(phys, b, s_tj, s_tw, s_tm);
        predict_box(B, taps, phys, b, sm, buf, tab);
    }
}

// ---------------------------------------------------------------------------
// comparison + re-initialisation
// ---------------------------------------------------------------------------

__device__ void correct_box(const StepBuffers& B, const PhysicsDev& phys, const DebugOut& dbg,
                            int b, int* gx, int* gy, float* buf, int* s_red) {
    const Domain& D = B.dom;
    const Box nb = B.cur[b];
    const int nx = nb.nx, ny = nb.ny, nz = nb.nz;
    const int A = nx * ny;
    const bool fx = nx == D.nx, fy = ny == D.ny, fz = nz == D.nz;
    const bool is3d = D.dim == 3;
    const float eps = D.eps;
    const int ps = plane_stride(nx, ny);

    float* C = buf;                  // 3 planes of phi_c (z-1, z, z+1)
    float* G = C + 3 * (size_t)A;    // reference-classified plane
    float* H = G + A;                // after the x pass
    float* F = H + A;                // 7 planes: forward z sweep

    for (int i = threadIdx.x; i < nx; i += blockDim.x) gx[i] = pmod(nb.ox + i, D.nx);
    for (int i = threadIdx.x; i < ny; i += blockDim.x) gy[i] = pmod(nb.oy + i, D.ny);
    int lo[3] = {INT_MAX, INT_MAX, INT_MAX}, hi[3] = {INT_MIN, INT_MIN, INT_MIN};

    // stream bounds (see the pipeline description in the file header)
    int z_first, z_last;
    if (!is3d) { z_first = 0; z_last = 0; }
    else if (fz) { z_first = -(kRedistReach + 1); z_last = nz + kRedistReach; }
    else {
        z_first = 0; z_last = nz + kRedistReach;
        float* pre = C + (size_t)pmod(-1, 3) * A;       // plane -1: outside, -eps
        for (int i = threadIdx.x; i < A; i += blockDim.x) pre[i] = -eps;
    }
    __syncthreads();

    for (int zin = z_first; zin <= z_last; ++zin) {
        // ---- A: phi_c of plane zin ----
        {
            float* Cz = C + (size_t)pmod(zin, 3) * A;
            bool inside = !is3d || fz || (zin >= 0 && zin < nz);
            bool want = is3d ? (fz ? true : zin <= nz) : true;
            if (want) {
                if (!inside) {
                    for (int i = threadIdx.x; i < A; i += blockDim.x) Cz[i] = -eps;
                } else {
                    int zl = is3d && fz ? pmod(zin, nz) : zin;
                    int gz = is3d ? pmod(nb.oz + zl, D.nz) : 0;
                    const float* src = B.Y + nb.off + (long long)zl * ps;
                    bool record = zin >= 0 && zin < nz;
                    for (int i = threadIdx.x; i < A; i += blockDim.x) {
                        int y = i / nx, x = i - y * nx;
                        float pp = src[i];
                        long long g = ((long long)gz * D.ny + gy[y]) * D.nx + gx[x];
                        unsigned long long k1 = B.T[2 * g], k2 = B.T[2 * g + 1];
                        int id1 = key_id(k1);
                        float m;
                        int mid;
                        if (id1 != b) { m = key_val(k1, eps); mid = id1; }
                        else { m = key_val(k2, eps); mid = key_id(k2); }
                        if (!(m > -eps)) mid = -1;
                        float pc = 0.5f * (pp - m);
                        Cz[i] = pc;
                        if (record) {
                            long long o = nb.off + (long long)zl * ps + i;
                            if (phys.kind != LSGG_PHYSICS_IDEAL) B.IDF[o] = mid;
                            if (dbg.m) { dbg.m[o] = m; dbg.idm[o] = mid; dbg.phic[o] = pc; dbg.phip[o] = pp; }
                        }
                    }
                }
            }
        }
        __syncthreads();
        const int zb = zin - 1 + (is3d ? 0 : 1);     // 2D: classify plane 0 right away
        const bool do_b = is3d ? (fz ? zb >= z_first + 1 && zb <= nz + kRedistReach - 1 : zb >= 0 && zb < nz) : true;
        if (do_b) {
            // ---- B: classification of plane zb -> G ----
            const float* Cm = C + (size_t)pmod(zb - 1, 3) * A;
            const float* C0 = C + (size_t)pmod(zb, 3) * A;
            const float* Cp = C + (size_t)pmod(zb + 1, 3) * A;
            for (int i = threadIdx.x; i < A; i += blockDim.x) {
                int y = i / nx, x = i - y * nx;
                const float xl = x > 0 ? C0[i - 1] : (fx ? C0[i + nx - 1] : -eps);
                const float xr = x < nx - 1 ? C0[i + 1] : (fx ? C0[i - nx + 1] : -eps);
                const float yl = y > 0 ? C0[i - nx] : (fy ? C0[i + (ny - 1) * nx] : -eps);
                const float yr = y < ny - 1 ? C0[i + nx] : (fy ? C0[i - (ny - 1) * nx] : -eps);
                // 2D: no z neighbours (on the z axis nothing is opposite)
                const float zl = is3d ? Cm[i] : C0[i], zr = is3d ? Cp[i] : C0[i];
                G[i] = classify_cell(C0[i], xl, xr, yl, yr, zl, zr, eps);
            }
            __syncthreads();
            // ---- C: x pass G -> H, y pass H -> forward z sweep into F ----
            for (int i = threadIdx.x; i < A; i += blockDim.x) {
                int y = i / nx, x = i - y * nx;
                H[i] = line_min(G + y * nx, x, nx, 1, fx);
            }
            __syncthreads();
            float* Fz = F + (size_t)(is3d ? pmod(zb, 7) : 0) * A;
            const float* Fprev = F + (size_t)pmod(zb - 1, 7) * A;
            const bool first = !is3d || zb == (fz ? z_first + 1 : 0);
            for (int i = threadIdx.x; i < A; i += blockDim.x) {
                int y = i / nx, x = i - y * nx;
                float v = line_min(H + x, y, ny, nx, fy);
                if (!first) {
                    float p = Fprev[i];
                    if (sgn_pos(p) == sgn_pos(v)) {
                        float m = fminf(fabsf(v), fabsf(p) + 1.0f);
                        v = sgn_pos(v) ? m : -m;
                    }
                }
                Fz[i] = v;
            }
        }
        __syncthreads();
        // ---- E: backward z window, output plane zo ----
        const int zo = is3d ? zb - kRedistReach : zb;
        if (zo >= 0 && zo < nz && (is3d || zin == 0)) {
            const int ztop = is3d ? (fz ? zb : min(zb, nz - 1)) : zo;
            const long long dst = nb.off + (long long)zo * ps;
            for (int i = threadIdx.x; i < A; i += blockDim.x) {
                float v = F[(size_t)(is3d ? pmod(zo, 7) : 0) * A + i];
                const bool s = sgn_pos(v);
                float best = fabsf(v);
                if (is3d) {
#pragma unroll
                    for (int k = 1; k <= kRedistReach; ++k) {
                        if (zo + k > ztop) break;
                        float u = F[(size_t)pmod(zo + k, 7) * A + i];
                        if (sgn_pos(u) != s) break;
                        best = fminf(best, fabsf(u) + (float)k);
                    }
                }
                best = fminf(best, eps);
                float out = s ? best : -best;
                st_state(B, dst + i, out);
                if (dbg.phin) dbg.phin[nb.off + (long long)zo * ps + i] = out;
                if (out > 0.0f) {
                    int y = i / nx, x = i - y * nx;
                    lo[0] = min(lo[0], x); hi[0] = max(hi[0], x);
                    lo[1] = min(lo[1], y); hi[1] = max(hi[1], y);
                    lo[2] = min(lo[2], zo); hi[2] = max(hi[2], zo);
                }
            }
        }
        // F slot reuse and C slot reuse are separated by the barriers of the next A and B stages
        if (!is3d) break;
    }
    // ---- positive bounding box of this box ----
    for (int a = 0; a < 3; ++a) {
        int l = lo[a], h = hi[a];
        for (int o = 16; o > 0; o >>= 1) {
            l = min(l, __shfl_xor_sync(0xffffffffu, l, o));
            h = max(h, __shfl_xor_sync(0xffffffffu, h, o));
        }
        lo[a] = l; hi[a] = h;
    }
    __syncthreads();
    if (threadIdx.x < 6) s_red[threadIdx.x] = threadIdx.x < 3 ? INT_MAX : INT_MIN;
    __syncthreads();
    if ((threadIdx.x & 31) == 0) {
        for (int a = 0; a < 3; ++a) { atomicMin(&s_red[a], lo[a]); atomicMax(&s_red[3 + a], hi[a]); }
    }
    __syncthreads();
    if (threadIdx.x == 0) {
        Bounds bd;
        for (int a = 0; a < 3; ++a) { bd.lo[a] = s_red[a]; bd.hi[a] = s_red[3 + a]; }
        B.bounds[b] = bd;
    }
    __syncthreads();
}

__global__ void __launch_bounds__(kThreads)
k_correct(StepBuffers B, PhysicsDev phys, DebugOut dbg, int cls) {
    extern __shared__ __align__(16) unsigned char smem_raw[];
    __shared__ int s_box;
    __shared__ int s_red[6];
    const int side = B.class_side[cls];
    int* gx = reinterpret_cast<int*>(smem_raw);
    int* gy = gx + side;
    float* buf = reinterpret_cast<float*>(gy + side + 4);
    buf = reinterpret_cast<float*>((reinterpret_cast<uintptr_t>(buf) + 15) & ~uintptr_t(15));
    if (B.mode[cls] == 2) buf = B.scratch + B.scratch_class_off[cls] + (long long)blockIdx.x * B.scratch_per_cta;
    for (;;) {
        int b = pull_box(B, 1, cls, &s_box);
        if (b < 0) break;
        correct_box(B, phys, dbg, b, gx, gy, buf, s_red);
    }
}

// ---------------------------------------------------------------------------
// box update (single CTA)
// ---------------------------------------------------------------------------

// Block-wide exclusive scan of N ints per thread (thread order): pre = the sum
// over lower threads, tot = the block total.  s: (blockDim / 32) * N ints.
template <int N>
__device__ __forceinline__ void block_exclusive_scan(const int (&v)[N], int (&pre)[N], int (&tot)[N], int* s) {
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nw = blockDim.x >> 5;
    int inc[N];
#pragma unroll
    for (int k = 0; k < N; ++k) {
        int x = v[k];
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            const int y = __shfl_up_sync(0xffffffffu, x, o);
            if (lane >= o) x += y;
        }
        inc[k] = x;
        if (lane == 31) s[warp * N + k] = x;
    }
    __syncthreads();
    if (warp == 0) {
#pragma unroll
        for (int k = 0; k < N; ++k) {
            int x = lane < nw ? s[lane * N + k] : 0;
#pragma unroll
            for (int o = 1; o < 32; o <<= 1) {
                const int y = __shfl_up_sync(0xffffffffu, x, o);
                if (lane >= o) x += y;
            }
            if (lane < nw) s[lane * N + k] = x;          // inclusive prefix over warps
        }
    }
    __syncthreads();
#pragma unroll
    for (int k = 0; k < N; ++k) {
        pre[k] = inc[k] - v[k] + (warp ? s[(warp - 1) * N + k] : 0);
        tot[k] = s[(nw - 1) * N + k];
    }
    __syncthreads();
}

// Block-wide sums of N long longs per thread, the same values on every
// thread afterwards (s: 32 * N long longs, free on entry and on return).
template <int N>
__device__ __forceinline__ void block_sums_ll(long long (&v)[N], long long* s) {
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nw = blockDim.x >> 5;
#pragma unroll
    for (int k = 0; k < N; ++k)
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) v[k] += __shfl_xor_sync(0xffffffffu, v[k], o);
    if (lane == 0)
#pragma unroll
        for (int k = 0; k < N; ++k) s[warp * N + k] = v[k];
    __syncthreads();
#pragma unroll
    for (int k = 0; k < N; ++k) {
        long long t = 0;
        for (int w = 0; w < nw; ++w) t += s[w * N + k];
        v[k] = t;
    }
    __syncthreads();
}

// Block-wide inclusive scan of one long long per thread in thread order
// (warp shuffles; warp 0 scans the warp totals); *total = the block's sum
// (s: 32 long longs, free on entry and on return).
__device__ __forceinline__ long long block_inclusive_scan_ll(long long v, long long* s, long long* total) {
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nw = blockDim.x >> 5;
    long long x = v;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        const long long y = __shfl_up_sync(0xffffffffu, x, o);
        if (lane >= o) x += y;
    }
    if (lane == 31) s[warp] = x;
    __syncthreads();
    if (warp == 0) {
        long long w = lane < nw ? s[lane] : 0;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            const long long y = __shfl_up_sync(0xffffffffu, w, o);
            if (lane >= o) w += y;
        }
        if (lane < nw) s[lane] = w;
    }
    __syncthreads();
    const long long r = x + (warp ? s[warp - 1] : 0);
    *total = s[nw - 1];
    __syncthreads();
    return r;
}

// Size class of a box: the smallest class whose side holds the x and y extents
// of both its new layout and the layout its state is read from.
__device__ __forceinline__ int box_class(const StepBuffers& B, const Box& b, const Box& p) {
    int s = max(max(b.nx, b.ny), max(p.nx, p.ny));
    for (int c = 0; c < kNumClasses - 1; ++c)
        if (s <= B.class_side[c]) return c;
    return kNumClasses - 1;
}

// Tier of a pass-path class: the smallest tier whose side holds the class's side.
__device__ __forceinline__ int pass_tier(const StepBuffers& B, int c) {
    for (int t = 0; t < kTiers - 1; ++t)
        if (B.class_side[c] <= B.tier_side[t]) return t;
    return kTiers - 1;
}

// The box after a step (Secs. 2.1.3, 3.1, reading R6): the bbox of the
// positive cells the re-initialisation collected (box-local bounds bd), grown
// by the halo; an axis reaching the domain becomes full and keeps its origin
// while full; no positive cell: extinct (nx = 0).
__device__ __forceinline__ Box updated_box(const Box& cb, const Bounds& bd, const Domain& D) {
    Box n = cb;
    if (bd.hi[0] < bd.lo[0]) {
        n.nx = n.ny = n.nz = 0;
        return n;
    }
    const int Ns[3] = {D.nx, D.ny, D.nz};
    const int os[3] = {cb.ox, cb.oy, cb.oz};
    const int ns[3] = {cb.nx, cb.ny, cb.nz};
    int no[3], nn[3];
#pragma unroll
    for (int a = 0; a < 3; ++a) {
        if (a == 2 && D.dim == 2) { no[a] = 0; nn[a] = 1; continue; }
        const int ext = bd.hi[a] - bd.lo[a] + 1 + 2 * D.halo;
        const bool was_full = ns[a] == Ns[a];
        if (ext >= Ns[a]) {
            nn[a] = Ns[a];
            no[a] = was_full ? os[a] : pmod(os[a] + bd.lo[a] - D.halo, Ns[a]);
        } else {
            nn[a] = ext;
            no[a] = pmod(os[a] + bd.lo[a] - D.halo, Ns[a]);
        }
    }
    n.ox = no[0]; n.oy = no[1]; n.oz = no[2];
    n.nx = nn[0]; n.ny = nn[1]; n.nz = nn[2];
    return n;
}

// layout_only: offsets and work items for the `cur` boxes as they are;
// otherwise the boxes follow the bounds collected by the re-initialisation,
// and count_step adds the step to the step and cell-update counters (not for
// the re-initialisation of a coarsening).  In a step group, CTA k updates
// member k (if it took part in the step).
template <bool GRP>
__global__ void __launch_bounds__(kBoxUpdateThreads)
k_box_update(StepBuffers B1, GroupRef grp, int layout_only, int count_step) {
    static_assert(2 + kTiers <= 8 && kBoxUpdateThreads <= 1024, "the scratch holds 8 sums of 32 warps");
    __shared__ long long s_part[32 * 8];
    __shared__ int s_scan[(kBoxUpdateThreads / 32) * (kNumClasses + 3 * kTiers)];
    const StepBuffers& B = GRP ? grp.B[blockIdx.x] : B1;
    if (GRP && !group_live(B, true)) return;
    const int G = B.n_boxes;
    const Domain D = B.dom;
    if (*(volatile int*)&B.st->halt && !layout_only) return;
    const int per = (G + blockDim.x - 1) / blockDim.x;
    const int b0 = threadIdx.x * per, b1 = min(G, b0 + per);
    long long sum = 0, done = 0;
    for (int b = b0; b < b1; ++b) {
        Box cb = B.cur[b];
        if (cb.nx > 0) done += (long long)cb.nx * cb.ny * cb.nz;
        if (!layout_only) {
            const Box n = cb.nx > 0 ? updated_box(cb, B.bounds[b], D) : cb;
            B.prev[b] = cb;
            B.cur[b] = n;
            cb = n;
        }
        sum += box_elems(cb);
    }
    // inclusive scan of the per-thread sums (integer: the order does not matter)
    long long total = 0;
    const long long incl = block_inclusive_scan_ll(sum, s_part, &total);
    if (!layout_only && count_step) {
        long long dn[1] = {done};
        block_sums_ll<1>(dn, s_part);
        if (threadIdx.x == 0) {
            B.st->cell_updates += dn[0];
            B.st->steps_done += 1;                  // the step's fields are complete
        }
    }
    if (total > B.cap) {
        if (threadIdx.x == 0) {
            B.st->status = LSGG_ERR_CAPACITY;
            B.st->halt = 1;
            B.st->box_cells = total;
        }
        return;
    }
    long long off = incl - sum;
    // per-thread counts: boxes per class (work lists), pass-path planes,
    // column chunks and slabs per tier; their block-wide exclusive scans place
    // every box's entries in box order
    // (every array below is indexed by unrolled constants only, so that it
    // stays in registers: a class or tier picks its entries by predicates)
    constexpr int NV = kNumClasses + 3 * kTiers;
    int cls_pass[kNumClasses], cls_tier[kNumClasses];
#pragma unroll
    for (int q = 0; q < kNumClasses; ++q) {
        cls_pass[q] = B.mode[q] == 3;
        cls_tier[q] = pass_tier(B, q);
    }
    int cnt[NV];
#pragma unroll
    for (int k = 0; k < NV; ++k) cnt[k] = 0;
    long long cells = 0, alive = 0, tcell[kTiers] = {};
    for (int b = b0; b < b1; ++b) {
        Box cb = B.cur[b];
        cb.off = off;
        off += box_elems(cb);
        B.cur[b] = cb;
        if (cb.nx > 0) {
            const int c = box_class(B, cb, B.prev[b]);
            const long long vol = (long long)cb.nx * cb.ny * cb.nz;
            int pass = 0, t = 0;
#pragma unroll
            for (int q = 0; q < kNumClasses; ++q)
                if (q == c) {
                    cnt[q] += 1;
                    pass = cls_pass[q];
                    t = cls_tier[q];
                }
            if (pass) {
                const int nch = (cb.nx * cb.ny + kPassChunk - 1) / kPassChunk;
                const int nsl = (cb.nz + B.slab - 1) / B.slab;
#pragma unroll
                for (int u = 0; u < kTiers; ++u)
                    if (u == t) {
                        cnt[kNumClasses + u] += cb.nz;
                        cnt[kNumClasses + kTiers + u] += nch;
                        cnt[kNumClasses + 2 * kTiers + u] += nsl;
                        tcell[u] += vol;
                    }
            }
            cells += vol;
            alive += 1;
        }
    }
    int pre[NV], tot[NV];
    block_exclusive_scan<NV>(cnt, pre, tot, s_scan);
    // first entry of each tier's items in the shared lists (kind 0 planes,
    // 1 column chunks, 2 slabs): the totals of the tiers before it
    int tier_base[3][kTiers];
    long long kind_total[3];
#pragma unroll
    for (int kd = 0; kd < 3; ++kd) {
        long long acc = 0;
#pragma unroll
        for (int t = 0; t < kTiers; ++t) {
            tier_base[kd][t] = (int)acc;
            acc += tot[kNumClasses + kd * kTiers + t];
        }
        kind_total[kd] = acc;
    }
    const bool items_fit = kind_total[0] <= B.plane_item_cap && kind_total[1] <= B.chunk_item_cap &&
                           kind_total[2] <= B.slab_item_cap;
    for (int b = b0; b < b1; ++b) {
        const Box cb = B.cur[b];
        if (B.use_passes) B.item_base[b] = make_int4(0, 0, 0, -1);
        if (cb.nx <= 0) continue;
        const int c = box_class(B, cb, B.prev[b]);
        int pass = 0, t = 0, wl = 0;
#pragma unroll
        for (int q = 0; q < kNumClasses; ++q)
            if (q == c) {
                pass = cls_pass[q];
                t = cls_tier[q];
                if (!pass) wl = pre[q]++;
            }
        if (!pass) {
            B.worklist[c * G + wl] = b;
            continue;
        }
        if (!items_fit) continue;
        const int nch = (cb.nx * cb.ny + kPassChunk - 1) / kPassChunk;
        const int nsl = (cb.nz + B.slab - 1) / B.slab;
        int p0 = 0, c0 = 0, s0 = 0;
#pragma unroll
        for (int u = 0; u < kTiers; ++u)
            if (u == t) {
                p0 = tier_base[0][u] + pre[kNumClasses + u];
                c0 = tier_base[1][u] + pre[kNumClasses + kTiers + u];
                s0 = tier_base[2][u] + pre[kNumClasses + 2 * kTiers + u];
                pre[kNumClasses + u] += cb.nz;
                pre[kNumClasses + kTiers + u] += nch;
                pre[kNumClasses + 2 * kTiers + u] += nsl;
            }
        B.item_base[b] = make_int4(p0, c0, s0, t);    // the items themselves: k_write_items
    }
    // reduce cells / alive / tier cells in one pass
    long long red[2 + kTiers];
    red[0] = cells;
    red[1] = alive;
    for (int t = 0; t < kTiers; ++t) red[2 + t] = tcell[t];
    block_sums_ll<2 + kTiers>(red, s_part);
    const long long r_cells = red[0], r_alive = red[1];
    long long r_tc[kTiers];
    for (int t = 0; t < kTiers; ++t) r_tc[t] = red[2 + t];
    if (threadIdx.x == 0) B.st->box_cells = r_cells;
    if (threadIdx.x < kNumClasses) {
        B.st->class_count[threadIdx.x] = tot[threadIdx.x];
        B.st->queue[0][threadIdx.x] = 0;
        B.st->queue[1][threadIdx.x] = 0;
    }
    if (threadIdx.x < kTiers) {
        const int t = threadIdx.x;
        B.st->n_planes[t] = items_fit ? tot[kNumClasses + t] : 0;
        B.st->n_chunks[t] = items_fit ? tot[kNumClasses + kTiers + t] : 0;
        B.st->plane_base[t] = tier_base[0][t];
        B.st->chunk_base[t] = tier_base[1][t];
        B.st->n_slabs[t] = items_fit ? tot[kNumClasses + 2 * kTiers + t] : 0;
        B.st->slab_base[t] = tier_base[2][t];
        B.st->tier_cells[t] = r_tc[t];
    }
    if (threadIdx.x == 0) {
        B.st->alive = r_alive;
        if (!items_fit) { B.st->status = LSGG_ERR_UNSUPPORTED; B.st->halt = 1; }   // not reached: caps are bounds
    }
}

// ---------------------------------------------------------------------------
// host-side launch helpers
// ---------------------------------------------------------------------------

static size_t predict_smem_bytes(int side, int R) {
    size_t ints = (size_t)2 * (side + 2 * kMaxRadius) + 2 * side + 4;
    size_t floats = (size_t)(side + 2 * R) * (side + 2 * R) + (size_t)side * (side + 2 * R) +
                    (size_t)(2 * R + 1) * side * side;
    return ints * 4 + 16 + floats * 4;
}
static size_t correct_smem_bytes(int side) {
    return ((size_t)2 * side + 4) * 4 + 16 + (size_t)12 * side * side * 4;
}

cudaError_t launch_collect_neighbours(const StepBuffers& B, const PhysicsDev& phys, cudaStream_t s);
cudaError_t configure_fast(StepBuffers& B, int cls, int n_sm);
cudaError_t launch_fast(const StepBuffers& B, int which, int cls, const Taps& taps, const PhysicsDev& phys,
                        const DebugOut& dbg, cudaStream_t s);

cudaError_t allow_max_dynamic_smem(const void* fn) {
    int dev = 0, max_optin = 0;
    cudaFuncAttributes fa{};
    cudaError_t e = cudaGetDevice(&dev);
    if (e == cudaSuccess) e = cudaDeviceGetAttribute(&max_optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev);
    if (e == cudaSuccess) e = cudaFuncGetAttributes(&fa, fn);
    if (e == cudaSuccess)        // static shared memory counts against the same limit
        e = cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, max_optin - (int)fa.sharedSizeBytes);
    return e;
}

cudaError_t configure_step_kernels(StepBuffers& B) {
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return e;
    int n_sm = 0, max_optin = 0;
    cudaDeviceGetAttribute(&n_sm, cudaDevAttrMultiProcessorCount, dev);
    cudaDeviceGetAttribute(&max_optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev);
    B.n_sm = n_sm;
    const int R = B.dom.radius;
    int big = B.dom.nx > B.dom.ny ? B.dom.nx : B.dom.ny;
    if (B.dom.nz > big) big = B.dom.nz;
    const bool fast_ok = B.dom.dim == 3 && R == 5;
    const int sides[kNumClasses - 1] = {32, 40, 48, 64};
    for (int c = 0; c < kNumClasses - 1; ++c) B.class_side[c] = sides[c];
    B.class_side[kNumClasses - 1] = big;
    // register-ring kernels for the small classes, shared-memory rings where they fit, global otherwise
    size_t mp = 0, mc = 0;
    const bool passes = B.use_passes && B.dom.dim == 3;
    B.use_passes = passes ? 1 : 0;
    for (int c = 0; c < kNumClasses; ++c) {
        B.block[c] = kThreads;
        if (passes) {                             // pass path (the largest boxes: its general-size tier)
            B.mode[c] = 3;
            continue;
        }
        if (fast_ok && fast_class_side(c) == B.class_side[c]) {
            e = configure_fast(B, c, n_sm);
            if (e != cudaSuccess) return e;
            B.mode[c] = 0;
            continue;
        }
        size_t sp = 0, sc = 0;
        bool fits = c < kNumClasses - 1 && (int)predict_smem_bytes(B.class_side[c], R) <= max_optin &&
                    (int)correct_smem_bytes(B.class_side[c]) <= max_optin;
        if (fits) {
            B.mode[c] = 1;
            sp = predict_smem_bytes(B.class_side[c], R);
            sc = correct_smem_bytes(B.class_side[c]);
        } else {
            B.mode[c] = 2;
            int side = c < kNumClasses - 1 ? B.class_side[c] : big;
            sp = (size_t)(2 * (side + 2 * kMaxRadius) + 2 * side + 4) * 4 + 16;
            sc = ((size_t)2 * side + 4) * 4 + 16;
        }
        B.smem[0][c] = sp;
        B.smem[1][c] = sc;
        if (sp > mp) mp = sp;
        if (sc > mc) mc = sc;
    }
    // the attribute is process-wide: set it to the device limit (never to a
    // context's own need, which would cap another context's launches)
    if (mp > 0 && (e = allow_max_dynamic_smem(reinterpret_cast<const void*>(k_predict))) != cudaSuccess) return e;
    if (mc > 0 && (e = allow_max_dynamic_smem(reinterpret_cast<const void*>(k_correct))) != cudaSuccess) return e;
    if (passes) {
        e = configure_passes(B);
        if (e != cudaSuccess) return e;
    }
    for (int c = 0; c < kNumClasses; ++c) {
        if (B.mode[c] == 0 || B.mode[c] == 3) continue;
        if (B.mode[c] == 2) {
            B.grid[0][c] = B.grid[1][c] = (n_sm + 3) / 4;
            continue;
        }
        int occ_p = 0, occ_c = 0;
        cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ_p, k_predict, kThreads, B.smem[0][c]);
        cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ_c, k_correct, kThreads, B.smem[1][c]);
        B.grid[0][c] = n_sm * (occ_p < 1 ? 1 : occ_p);
        B.grid[1][c] = n_sm * (occ_c < 1 ? 1 : occ_c);
    }
    return cudaSuccess;
}

long long large_class_scratch_floats(const Domain& d) {
    int big = d.nx > d.ny ? d.nx : d.ny;
    long long side = big;
    long long p = (side + 2 * kMaxRadius) * (side + 2 * kMaxRadius) + side * (side + 2 * kMaxRadius) +
                  (long long)(2 * kMaxRadius + 1) * side * side;
    long long c = 12 * side * side;
    long long m = p > c ? p : c;
    return (m + 31) & ~31LL;
}

// The pass path's work items of every box, from the bases k_box_update set:
// a warp per box, lanes along its items (coalesced stores).
// The members of a step group whose box update ran: not halted (a member at
// its step limit after this step still writes its items).
template <bool GRP>
__global__ void __launch_bounds__(256)
k_write_items(StepBuffers B1, GroupRef grp) {
    __shared__ int s_gb[GRP ? kMaxGroup + 1 : 1];
    if (!GRP && *(volatile int*)&B1.st->halt) return;   // the box update stopped the step: no fresh bases
    const int n_all = GRP ? group_scan(grp, kItemBoxes, 0, false, s_gb) : B1.n_boxes;
    const int lane = threadIdx.x & 31;
    const int warps = (blockDim.x >> 5) * gridDim.x;
    for (int gb = (blockIdx.x * blockDim.x + threadIdx.x) >> 5; gb < n_all; gb += warps) {
        int b;
        const StepBuffers& B = member<GRP>(B1, grp, s_gb, gb, b);
        const int4 base = B.item_base[b];
        if (base.w < 0) continue;
        const Box cb = B.cur[b];
        const int nch = (cb.nx * cb.ny + kPassChunk - 1) / kPassChunk;
        const int nsl = (cb.nz + B.slab - 1) / B.slab;
        for (int z = lane; z < cb.nz; z += 32) B.plane_items[base.x + z] = make_int2(b, z);
        for (int k = lane; k < nch; k += 32) B.chunk_items[base.y + k] = make_int2(b, k);
        for (int k = lane; k < nsl; k += 32) B.slab_items[base.z + k] = make_int2(b, k * B.slab);
    }
}

// ---------------------------------------------------------------------------
// the step's box update over the whole GPU
// ---------------------------------------------------------------------------
// The values a box contributes (kBuVals): arena elements of its new box, its
// cells before the update (the step's cell-updates), its cells and 1 if
// alive, one box for its size class, and on the pass path its planes, column
// chunks, slabs and cells for its tier.
enum : int { kVElems = 0, kVDone = 1, kVCells = 2, kVAlive = 3, kVCls = 4, kVPl = kVCls + kNumClasses,
             kVCh = kVPl + kTiers, kVSl = kVCh + kTiers, kVTc = kVSl + kTiers };
static_assert(kVTc + kTiers == kBuVals, "one layout of the box update's values");

__device__ __forceinline__ void box_values(const StepBuffers& B, const Box& cb, const Box& pb, long long done,
                                           long long (&v)[kBuVals], int& cls, int& pass, int& tier) {
#pragma unroll
    for (int q = 0; q < kBuVals; ++q) v[q] = 0;
    v[kVElems] = box_elems(cb);
    v[kVDone] = done;
    cls = 0; pass = 0; tier = 0;
    if (cb.nx <= 0) return;
    const long long vol = (long long)cb.nx * cb.ny * cb.nz;
    v[kVCells] = vol;
    v[kVAlive] = 1;
    cls = box_class(B, cb, pb);
#pragma unroll
    for (int q = 0; q < kNumClasses; ++q)
        if (q == cls) {
            v[kVCls + q] = 1;
            pass = B.mode[q] == 3;
            tier = pass_tier(B, q);
        }
    if (!pass) return;
    const long long nch = (cb.nx * cb.ny + kPassChunk - 1) / kPassChunk;
    const long long nsl = (cb.nz + B.slab - 1) / B.slab;
#pragma unroll
    for (int u = 0; u < kTiers; ++u)
        if (u == tier) {
            v[kVPl + u] = cb.nz;
            v[kVCh + u] = nch;
            v[kVSl + u] = nsl;
            v[kVTc + u] = vol;
        }
}

// Block-wide exclusive scan of N long longs per thread (thread order):
// pre = sum over lower threads; s: (blockDim / 32) * N long longs.
template <int N>
__device__ __forceinline__ void block_exclusive_scan_ll(const long long (&v)[N], long long (&pre)[N], long long* s) {
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nw = blockDim.x >> 5;
#pragma unroll
    for (int k = 0; k < N; ++k) {
        long long x = v[k];
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            const long long y = __shfl_up_sync(0xffffffffu, x, o);
            if (lane >= o) x += y;
        }
        pre[k] = x - v[k];
        if (lane == 31) s[warp * N + k] = x;
    }
    __syncthreads();
    if (warp == 0) {
#pragma unroll
        for (int k = 0; k < N; ++k) {
            long long x = lane < nw ? s[lane * N + k] : 0;
#pragma unroll
            for (int o = 1; o < 32; o <<= 1) {
                const long long y = __shfl_up_sync(0xffffffffu, x, o);
                if (lane >= o) x += y;
            }
            if (lane < nw) s[lane * N + k] = x;       // inclusive prefix over warps
        }
    }
    __syncthreads();
#pragma unroll
    for (int k = 0; k < N; ++k) pre[k] += warp ? s[(warp - 1) * N + k] : 0;
    __syncthreads();
}

// 1. New boxes and per-chunk sums (a CTA per chunk of kBuChunk boxes).
template <bool GRP>
__global__ void __launch_bounds__(kBuChunk)
k_bu_new(StepBuffers B1, GroupRef grp) {
    __shared__ int s_gb[GRP ? kMaxGroup + 1 : 1];
    __shared__ long long s_red[32 * kBuVals];
    const int n_all = GRP ? group_scan(grp, kItemBoxChunks, 0, true, s_gb)
                          : (*(volatile int*)&B1.st->halt ? 0 : (B1.n_boxes + kBuChunk - 1) / kBuChunk);
    for (int gc = blockIdx.x; gc < n_all; gc += gridDim.x) {
        int k;
        const StepBuffers& B = member<GRP>(B1, grp, s_gb, gc, k);
        const int b = k * kBuChunk + threadIdx.x;
        long long v[kBuVals];
        int cls, pass, tier;
        if (b < B.n_boxes) {
            const Box cb = B.cur[b];
            const Box n = cb.nx > 0 ? updated_box(cb, B.bounds[b], B.dom) : cb;
            B.prev[b] = cb;
            B.cur[b] = n;
            box_values(B, n, cb, cb.nx > 0 ? (long long)cb.nx * cb.ny * cb.nz : 0, v, cls, pass, tier);
        } else {
#pragma unroll
            for (int q = 0; q < kBuVals; ++q) v[q] = 0;
        }
        block_sums_ll<kBuVals>(v, s_red);
#pragma unroll
        for (int q = 0; q < kBuVals; ++q)
            if (threadIdx.x == q) B.bu_part[(long long)k * kBuVals + q] = v[q];
    }
}

// 2. The chunk sums scanned into chunk bases (in place), the totals checked
// against the arena and the work-item lists, the step's counters (one CTA per
// context; in a group, CTA k for member k).
constexpr int kBuScanThreads = 128;     // the chunk sums of a context are few (one per 256 boxes)

template <bool GRP>
__global__ void __launch_bounds__(kBuScanThreads)
k_bu_scan(StepBuffers B1, GroupRef grp, int count_step) {
    __shared__ long long s_red[32 * kBuVals];
    const StepBuffers& B = GRP ? grp.B[blockIdx.x] : B1;
    const bool live = GRP ? group_live(B, true) : *(volatile int*)&B.st->halt == 0;
    if (!live) {
        if (threadIdx.x == 0) B.st->bu_go = 0;
        return;
    }
    const int nch = (B.n_boxes + kBuChunk - 1) / kBuChunk;
    const int per = (nch + blockDim.x - 1) / blockDim.x;
    const int c0 = min(nch, (int)threadIdx.x * per), c1 = min(nch, c0 + per);
    long long v[kBuVals], pre[kBuVals];
#pragma unroll
    for (int q = 0; q < kBuVals; ++q) v[q] = 0;
    for (int c = c0; c < c1; ++c)
#pragma unroll
        for (int q = 0; q < kBuVals; ++q) v[q] += B.bu_part[(long long)c * kBuVals + q];
    block_exclusive_scan_ll<kBuVals>(v, pre, s_red);
    for (int c = c0; c < c1; ++c)                    // chunk sums -> chunk bases
#pragma unroll
        for (int q = 0; q < kBuVals; ++q) {
            long long* e = B.bu_part + (long long)c * kBuVals + q;
            const long long x = *e;
            *e = pre[q];
            pre[q] += x;
        }
    // totals: the last thread's running prefix
    __shared__ long long s_tot[kBuVals];
    if (threadIdx.x == blockDim.x - 1)
#pragma unroll
        for (int q = 0; q < kBuVals; ++q) s_tot[q] = pre[q];
    __syncthreads();
    if (threadIdx.x != 0) return;
    StepState* st = B.st;
    if (count_step) {
        st->cell_updates += s_tot[kVDone];
        st->steps_done += 1;                          // the step's fields are complete
    }
    if (s_tot[kVElems] > B.cap) {
        st->status = LSGG_ERR_CAPACITY;
        st->halt = 1;
        st->box_cells = s_tot[kVElems];
        st->bu_go = 0;
        return;
    }
    long long kind_total[3];
#pragma unroll
    for (int kd = 0; kd < 3; ++kd) {
        long long acc = 0;
#pragma unroll
        for (int t = 0; t < kTiers; ++t) {
            if (kd == 0) st->plane_base[t] = (int)acc;
            if (kd == 1) st->chunk_base[t] = (int)acc;
            if (kd == 2) st->slab_base[t] = (int)acc;
            acc += s_tot[kVPl + kd * kTiers + t];
        }
        kind_total[kd] = acc;
    }
    const bool items_fit = kind_total[0] <= B.plane_item_cap && kind_total[1] <= B.chunk_item_cap &&
                           kind_total[2] <= B.slab_item_cap;
    st->box_cells = s_tot[kVCells];
    st->alive = s_tot[kVAlive];
#pragma unroll
    for (int q = 0; q < kNumClasses; ++q) {
        st->class_count[q] = (int)s_tot[kVCls + q];
        st->queue[0][q] = 0;
        st->queue[1][q] = 0;
    }
#pragma unroll
    for (int t = 0; t < kTiers; ++t) {
        st->n_planes[t] = items_fit ? (int)s_tot[kVPl + t] : 0;
        st->n_chunks[t] = items_fit ? (int)s_tot[kVCh + t] : 0;
        st->n_slabs[t] = items_fit ? (int)s_tot[kVSl + t] : 0;
        st->tier_cells[t] = s_tot[kVTc + t];
    }
    if (!items_fit) { st->status = LSGG_ERR_UNSUPPORTED; st->halt = 1; }   // not reached: caps are bounds
    st->bu_go = items_fit ? 1 : 0;
}

// 3. Every box's arena offset, work-list entry and work-item bases: the
// chunk base plus the box's exclusive prefix within its chunk.
template <bool GRP>
__global__ void __launch_bounds__(kBuChunk)
k_bu_place(StepBuffers B1, GroupRef grp) {
    __shared__ int s_gb[GRP ? kMaxGroup + 1 : 1];
    __shared__ long long s_scan[(kBuChunk / 32) * kBuVals];
    const int n_all = GRP ? group_scan(grp, kItemBoxChunksGo, 0, false, s_gb)
                          : (B1.st->bu_go ? (B1.n_boxes + kBuChunk - 1) / kBuChunk : 0);
    for (int gc = blockIdx.x; gc < n_all; gc += gridDim.x) {
        int k;
        const StepBuffers& B = member<GRP>(B1, grp, s_gb, gc, k);
        const int b = k * kBuChunk + threadIdx.x;
        long long v[kBuVals], pre[kBuVals];
        int cls = 0, pass = 0, tier = 0;
        Box cb{};
        if (b < B.n_boxes) {
            cb = B.cur[b];
            box_values(B, cb, B.prev[b], 0, v, cls, pass, tier);
        } else {
#pragma unroll
            for (int q = 0; q < kBuVals; ++q) v[q] = 0;
        }
        block_exclusive_scan_ll<kBuVals>(v, pre, s_scan);
        if (b >= B.n_boxes) continue;
        const long long* base = B.bu_part + (long long)k * kBuVals;
        B.cur[b].off = base[kVElems] + pre[kVElems];
        if (cb.nx <= 0) {
            if (B.use_passes) B.item_base[b] = make_int4(0, 0, 0, -1);
            continue;
        }
        if (!pass) {
            long long pos = 0;
#pragma unroll
            for (int q = 0; q < kNumClasses; ++q)
                if (q == cls) pos = base[kVCls + q] + pre[kVCls + q];
            B.worklist[cls * B.n_boxes + pos] = b;
            if (B.use_passes) B.item_base[b] = make_int4(0, 0, 0, -1);
            continue;
        }
        int p0 = 0, c0 = 0, s0 = 0;
#pragma unroll
        for (int u = 0; u < kTiers; ++u)
            if (u == tier) {
                p0 = B.st->plane_base[u] + (int)(base[kVPl + u] + pre[kVPl + u]);
                c0 = B.st->chunk_base[u] + (int)(base[kVCh + u] + pre[kVCh + u]);
                s0 = B.st->slab_base[u] + (int)(base[kVSl + u] + pre[kVSl + u]);
            }
        B.item_base[b] = make_int4(p0, c0, s0, tier);   // the items themselves: k_write_items
    }
}

cudaError_t launch_box_update(const StepBuffers& B, bool layout_only, cudaStream_t s, bool count_step) {
    const GroupRef none{nullptr, 0};
    cudaError_t e;
    if (layout_only) {
        k_box_update<false><<<1, kBoxUpdateThreads, 0, s>>>(B, none, 1, 0);
    } else {
        const int nch = (B.n_boxes + kBuChunk - 1) / kBuChunk;
        const int grid = nch < 4 * B.n_sm ? nch : 4 * B.n_sm;
        k_bu_new<false><<<grid, kBuChunk, 0, s>>>(B, none);
        e = cudaGetLastError();
        if (e != cudaSuccess) return e;
        k_bu_scan<false><<<1, kBuScanThreads, 0, s>>>(B, none, count_step ? 1 : 0);
        e = cudaGetLastError();
        if (e != cudaSuccess) return e;
        k_bu_place<false><<<grid, kBuChunk, 0, s>>>(B, none);
    }
    e = cudaGetLastError();
    if (e != cudaSuccess || !B.use_passes) return e;
    k_write_items<false><<<B.n_sm * 4, 256, 0, s>>>(B, none);
    return cudaGetLastError();
}

// Each member's step limit (steps_done at which it stops taking part).
__global__ void k_group_limits(GroupRef grp, const long long* __restrict__ lim) {
    const int k = blockIdx.x * blockDim.x + threadIdx.x;
    if (k < grp.n) grp.B[k].st->step_limit = lim[k];
}

cudaError_t launch_group_limits(const GroupRef& grp, const long long* lim, cudaStream_t s) {
    k_group_limits<<<1, kMaxGroup, 0, s>>>(grp, lim);
    return cudaGetLastError();
}

// One step of every member of a step group (ideal growth, taxicab
// re-initialisation, the pass path): the same kernels as launch_step's pass
// path, each launched once over all members.  With side streams the binning
// runs beside the convolution passes and tiers 1.. beside tier 0.
cudaError_t launch_group_step(const StepBuffers& B0, const GroupRef& grp, const Taps& taps, cudaStream_t s,
                              const StepStreams* ss) {
    cudaStream_t bs = ss ? ss->side[kTiers - 1] : s;
    cudaError_t e = cudaSuccess;
    if (bs != s) {
        e = traced(cudaEventRecord(ss->fork, s), "fork record");
        if (e == cudaSuccess) e = traced(cudaStreamWaitEvent(bs, ss->fork, 0), "fork wait");
        if (e != cudaSuccess) return e;
    }
    e = traced(launch_bin_group(B0, grp, bs), "group binning");
    if (e == cudaSuccess && bs != s) e = traced(cudaEventRecord(ss->join[kTiers - 1], bs), "join record");
    if (e != cudaSuccess) return e;
    auto tiers = [&](int which) -> cudaError_t {
        if (ss) {
            cudaError_t r = traced(cudaEventRecord(ss->fork, s), "fork record");
            if (r != cudaSuccess) return r;
        }
        for (int t = 0; t < kTiers; ++t) {
            cudaStream_t ts = s;
            if (ss && t > 0) {
                ts = ss->side[t - 1];
                cudaError_t r = traced(cudaStreamWaitEvent(ts, ss->fork, 0), "fork wait");
                if (r != cudaSuccess) return r;
            }
            cudaError_t r = traced(launch_passes_group(B0, grp, which, t, taps, ts), "group pass kernels");
            if (r != cudaSuccess) return r;
            if (ss && t > 0) {
                r = traced(cudaEventRecord(ss->join[t - 1], ts), "join record");
                if (r == cudaSuccess) r = traced(cudaStreamWaitEvent(s, ss->join[t - 1], 0), "join wait");
                if (r != cudaSuccess) return r;
            }
        }
        return cudaSuccess;
    };
    e = tiers(0);
    if (e != cudaSuccess) return e;
    if (bs != s) {
        e = traced(cudaStreamWaitEvent(s, ss->join[kTiers - 1], 0), "join wait");
        if (e != cudaSuccess) return e;
    }
    e = traced(launch_field_group(B0, grp, s), "group field pass");
    if (e == cudaSuccess) e = tiers(1);
    if (e != cudaSuccess) return e;
    k_bu_new<true><<<4 * B0.n_sm, kBuChunk, 0, s>>>(B0, grp);
    e = cudaGetLastError();
    if (e == cudaSuccess) {
        k_bu_scan<true><<<grp.n, kBuScanThreads, 0, s>>>(B0, grp, 1);
        e = cudaGetLastError();
    }
    if (e == cudaSuccess) {
        k_bu_place<true><<<4 * B0.n_sm, kBuChunk, 0, s>>>(B0, grp);
        e = cudaGetLastError();
    }
    if (e != cudaSuccess) return traced(e, "group box update");
    k_write_items<true><<<B0.n_sm * 4, 256, 0, s>>>(B0, grp);
    return traced(cudaGetLastError(), "group work items");
}

cudaError_t launch_step(const StepBuffers& B, const Taps& taps, const PhysicsDev& phys,
                        const DebugOut* dbg, cudaStream_t s, cudaEvent_t* ev, const StepStreams* ss,
                        cudaEvent_t* cls_ev, cudaEvent_t* pass_ev) {
    long long ncell = (long long)B.dom.nx * B.dom.ny * B.dom.nz;
    cudaEvent_t* bin_ev = pass_ev ? pass_ev + 6 * kTiers : nullptr;
    if (ev) cudaEventRecord(ev[0], s);
    cudaError_t e;
    // binning reads only the boxes and writes only the tile lists and the
    // bounds the re-initialisation collects: with side streams it runs beside
    // the convolution passes and joins before the field pass
    static_assert(kTiers <= kNumClasses, "a side stream for the binning beside the tiers' ones");
    cudaStream_t bs = ss && B.use_passes ? ss->side[kTiers - 1] : s;
    if (B.use_passes) {                 // the field pass stores every cell of T: no clear
        if (bs != s) {
            e = traced(cudaEventRecord(ss->fork, s), "fork record");
            if (e == cudaSuccess) e = traced(cudaStreamWaitEvent(bs, ss->fork, 0), "fork wait");
            if (e != cudaSuccess) return e;
        }
        if (bin_ev) cudaEventRecord(bin_ev[0], s);
        e = traced(launch_bin(B, bs), "tile binning");
        if (bin_ev) cudaEventRecord(bin_ev[1], s);
        if (e == cudaSuccess && bs != s) e = traced(cudaEventRecord(ss->join[kTiers - 1], bs), "join record");
    } else {
        e = traced(cudaMemsetAsync(B.T, 0, (size_t)ncell * 16, s), "field clear");
    }
    if (e != cudaSuccess) return e;
    if (ev) cudaEventRecord(ev[1], s);
    DebugOut d{};
    if (dbg) d = *dbg;
    if (phys.kind == LSGG_PHYSICS_READ_SHOCKLEY || phys.pool_ent[0]) {
        e = traced(launch_collect_neighbours(B, phys, s), "neighbour tables");
        if (e != cudaSuccess) return e;
    }
    if (phys.pair_map) {                // Eq. (10)'s pairs from the closest boundary point (Sec. 2.1.4)
        e = traced(launch_gb_map_step(B, s), "anisotropy map");
        if (e != cudaSuccess) return e;
    }
    // Each phase forks the box-streaming size classes off the step's stream
    // onto their side streams and joins them back.
    auto run_phase = [&](int which) -> cudaError_t {
        bool joined[kNumClasses] = {};
        if (ss) {
            cudaError_t r = traced(cudaEventRecord(ss->fork, s), "fork record");
            if (r != cudaSuccess) return r;
        }
        auto stream_for = [&](int k, cudaStream_t* cs) -> cudaError_t {
            *cs = s;
            if (!ss) return cudaSuccess;
            *cs = ss->side[k];
            return traced(cudaStreamWaitEvent(*cs, ss->fork, 0), "fork wait");
        };
        auto join = [&](int k, cudaStream_t cs) -> cudaError_t {
            if (!ss) return cudaSuccess;
            joined[k] = true;
            return traced(cudaEventRecord(ss->join[k], cs), "join record");
        };
        // pass-path tiers: a tier's passes touch only its own boxes, so with
        // side streams (graph replay) tiers 1.. run on side streams beside
        // tier 0 and the small tiers' launches and every pass's tail overlap
        // the others; profiled steps (no side streams) run them one after
        // another so that each event time is one kernel's
        if (B.use_passes && which == 1 && B.redist != LSGG_REDIST_TAXICAB) {
            // Godunov re-initialisation over all tiers at once; its time is
            // reported as tier 0's re-initialisation passes
            cudaEvent_t* pe = pass_ev ? pass_ev + 3 : nullptr;
            if (pe) cudaEventRecord(pe[0], s);
            cudaError_t r = traced(launch_sweep_redist(B, d, s), "sweep re-initialisation");
            if (r != cudaSuccess) return r;
            if (pe) {
                cudaEventRecord(pe[1], s);
                cudaEventRecord(pe[2], s);
                for (int t = 1; t < kTiers; ++t)
                    for (int k = 0; k < 3; ++k) cudaEventRecord(pass_ev[t * 6 + 3 + k], s);
            }
        } else if (B.use_passes) {
            static_assert(kTiers - 1 <= kNumClasses, "a side stream per tier beyond the first");
            for (int t = 0; t < kTiers; ++t) {
                cudaStream_t ts = s;
                if (ss && t > 0) {
                    ts = ss->side[t - 1];
                    cudaError_t r = traced(cudaStreamWaitEvent(ts, ss->fork, 0), "fork wait");
                    if (r != cudaSuccess) return r;
                }
                cudaError_t r = traced(
                    launch_passes(B, which, t, taps, phys, d, ts, pass_ev ? pass_ev + t * 6 + (which ? 3 : 0) : nullptr),
                    "pass kernels");
                if (r != cudaSuccess) return r;
                if (ss && t > 0) {
                    r = traced(cudaEventRecord(ss->join[t - 1], ts), "join record");
                    if (r == cudaSuccess) r = traced(cudaStreamWaitEvent(s, ss->join[t - 1], 0), "join wait");
                    if (r != cudaSuccess) return r;
                }
            }
        }
        for (int c = 0; c < kNumClasses; ++c) {
            if (B.mode[c] == 3) continue;
            cudaStream_t cs;
            cudaError_t r = stream_for(c, &cs);
            if (r != cudaSuccess) return r;
            if (cls_ev) cudaEventRecord(cls_ev[(which * kNumClasses + c) * 2], cs);
            if (B.mode[c] == 0) r = launch_fast(B, which, c, taps, phys, d, cs);
            else if (which == 0) { k_predict<<<B.grid[0][c], kThreads, B.smem[0][c], cs>>>(B, taps, phys, c); r = cudaGetLastError(); }
            else { k_correct<<<B.grid[1][c], kThreads, B.smem[1][c], cs>>>(B, phys, d, c); r = cudaGetLastError(); }
            if (r != cudaSuccess) return traced(r, "box-streaming kernels");
            if (cls_ev) cudaEventRecord(cls_ev[(which * kNumClasses + c) * 2 + 1], cs);
            r = join(c, cs);
            if (r != cudaSuccess) return r;
        }
        for (int c = 0; c < kNumClasses; ++c)
            if (joined[c]) {
                cudaError_t r = traced(cudaStreamWaitEvent(s, ss->join[c], 0), "join wait");
                if (r != cudaSuccess) return r;
            }
        return cudaSuccess;
    };
    e = run_phase(0);
    if (e != cudaSuccess) return e;
    if (B.use_passes) {
        if (bs != s) {
            e = traced(cudaStreamWaitEvent(s, ss->join[kTiers - 1], 0), "join wait");
            if (e != cudaSuccess) return e;
        }
        if (bin_ev) cudaEventRecord(bin_ev[2], s);
        e = traced(launch_field(B, phys, d, s), "field pass");
        if (e != cudaSuccess) return e;
        if (bin_ev) cudaEventRecord(bin_ev[3], s);
    }
    if (ev) cudaEventRecord(ev[2], s);
    e = run_phase(1);
    if (e != cudaSuccess) return e;
    if (ev) cudaEventRecord(ev[3], s);
    e = traced(launch_box_update(B, false, s), "box update");
    if (ev) cudaEventRecord(ev[4], s);
    return e;
}

// The re-initialisation (pass 3) and box update of a step alone, on the
// phi_c that Z holds in the `cur` layout: the pass path's binning (which
// resets the bounds), its re-initialisation passes of every tier and a box
// update that counts no step.  With id_field, the field pass then runs on the
// re-initialised state (copied to Y as its phi_p) before the box update, so
// that the ID-field the next step's correction reads exists in this layout.
// Used by the grid coarsening.
cudaError_t launch_reinit(const StepBuffers& B, const Taps& taps, const PhysicsDev& phys, bool id_field,
                          cudaStream_t s) {
    if (!B.use_passes) return cudaErrorInvalidValue;
    cudaError_t e = traced(launch_bin(B, s), "tile binning");
    if (e != cudaSuccess) return e;
    const DebugOut d{};
    if (B.redist != LSGG_REDIST_TAXICAB) {
        e = traced(launch_sweep_redist(B, d, s), "sweep re-initialisation");
    } else {
        for (int t = 0; t < kTiers && e == cudaSuccess; ++t)
            e = traced(launch_passes(B, 1, t, taps, phys, d, s, nullptr), "pass kernels");
    }
    if (e == cudaSuccess && id_field) {
        e = B.bf16 ? launch_state_to_f32(B.X, B.Y, B.cap, s)
                   : cudaMemcpyAsync(B.Y, B.X, (size_t)B.cap * sizeof(float), cudaMemcpyDeviceToDevice, s);
        if (e == cudaSuccess) e = traced(launch_field(B, phys, d, s), "field pass");
    }
    if (e != cudaSuccess) return e;
    return traced(launch_box_update(B, false, s, false), "box update");
}

}  // namespace lsgg
