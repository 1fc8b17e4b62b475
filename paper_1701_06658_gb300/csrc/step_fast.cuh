// Register-ring kernels of the batched step for 3D boxes of side <= 48 and a
// kernel radius of 5 (the benchmark configuration); other boxes use step.cu.
//
// Same arithmetic as step.cu (Sec. 2.1.4 predictor, Eq. (16) comparison,
// Sec. 2.1.6 taxicab re-initialisation); what changes is where data lives:
//   * the box's old planes stream into a 3-slot shared-memory ring by
//     cp.async.bulk (TMA bulk copies completing on mbarriers), prefetched two
//     planes ahead, so the CTA never waits on a plain global load;
//   * each thread owns a column segment of V cells (x, y0 .. y0+V-1) for the
//     whole box and keeps the z windows in registers: the 2R+1 planes of the
//     convolution's y-pass output in k_predict_fast, and the 7 planes of the
//     forward z sweep in k_correct_fast;
//   * the x and y passes are register-blocked (a thread loads a window once
//     and produces several outputs), the taxicab passes use a forward and a
//     backward sweep over the window.
// Every wait on an mbarrier is bounded; on expiry the CTA records
// LSGG_ERR_TIMEOUT, halts the step and returns.
#pragma once

#include <cfloat>
#include <climits>

#include "bulk_copy.cuh"
#include "kernels_common.cuh"

namespace lsgg {
namespace fast {

// Division of small non-negative ints (< 2^16) by a per-box divisor d:
// q = (t * ceil(2^32 / d)) >> 32 is exact in that range, two instructions
// instead of an integer-division sequence.
struct FastDiv {
    unsigned m;
    int d;
    __device__ __forceinline__ explicit FastDiv(int dd) : m((unsigned)((0x100000000ULL + dd - 1) / dd)), d(dd) {}
    __device__ __forceinline__ int div(int t) const { return (int)__umulhi((unsigned)t, m); }
};

constexpr int kSlots = 3;
constexpr int kVX = 4;      // outputs per thread in the convolution x pass
constexpr int kVD = 8;      // outputs per thread in the taxicab x pass
constexpr int kReach = kRedistReach;

// Timeout: record it, stop the step, drain (bounded) the copies this CTA may
// still have in flight, and leave.
__device__ inline void give_up(const StepBuffers& B, uint64_t* bar, uint32_t phase) {
    if (threadIdx.x == 0) {
        atomicExch(&B.st->status, LSGG_ERR_TIMEOUT);
        atomicExch(&B.st->halt, 1);
        for (int s = 0; s < kSlots; ++s) mbar_wait(&bar[s], (phase >> s) & 1u);
    }
    __syncthreads();
}

template <int SIDE, int R>
struct PredictLayout {
    static constexpr int PX = SIDE + 2 * R;
    static constexpr int PS = (SIDE * SIDE + 3) & ~3;
    static constexpr size_t raw = 128;
    static constexpr size_t P = raw + sizeof(float) * kSlots * PS;
    static constexpr size_t Xp = P + sizeof(float) * PX * PX;
    static constexpr size_t maps = Xp + sizeof(float) * SIDE * PX;
    static constexpr size_t bytes = maps + sizeof(int) * (2 * PX + 2 * SIDE);
};

// ---------------------------------------------------------------------------
// predictor + neighbour-max scatter
// ---------------------------------------------------------------------------
template <int R, int V, int NT, int SIDE, int MINB>
__global__ void __launch_bounds__(NT, MINB)
k_predict_fast(StepBuffers B, Taps taps, PhysicsDev phys, int cls) {
    constexpr int W = 2 * R + 1;
    using L = PredictLayout<SIDE, R>;
    extern __shared__ __align__(128) unsigned char sm[];
    uint64_t* bar = reinterpret_cast<uint64_t*>(sm);
    float* raw = reinterpret_cast<float*>(sm + L::raw);
    float* P = reinterpret_cast<float*>(sm + L::P);
    float* Xp = reinterpret_cast<float*>(sm + L::Xp);
    int* mapx = reinterpret_cast<int*>(sm + L::maps);
    int* mapy = mapx + L::PX;
    int* gx = mapy + L::PX;
    int* gy = gx + SIDE;
    __shared__ int s_box;
    __shared__ int s_tj[kNbCap];
    __shared__ float s_tw[kNbCap], s_tm[kNbCap];
    const int tid = threadIdx.x;
    if (tid == 0) {
        for (int s = 0; s < kSlots; ++s) mbar_init(&bar[s], 1);
        fence_mbar_init();
    }
    __syncthreads();
    uint32_t phase = 0;
    const Domain D = B.dom;
    const float eps = D.eps;

    for (;;) {
        const int b = pull_box(B, 0, cls, &s_box);
        if (b < 0) break;
        const PairTable tab = load_pair_table(phys, b, s_tj, s_tw, s_tm);
        const Box nb = B.cur[b];
        const Box ob = B.prev[b];
        const int nx = nb.nx, ny = nb.ny, nz = nb.nz;
        const bool fx = nx == D.nx, fy = ny == D.ny, fzf = nz == D.nz;
        const int PXa = nx + 2 * R, PYa = ny + 2 * R;
        for (int i = tid; i < PXa; i += NT) {
            int xl = i - R, v = -1;
            if (fx || (xl >= 0 && xl < nx)) {
                if (fx) xl = pmod(xl, nx);
                int ol = pmod(nb.ox + xl - ob.ox, D.nx);
                v = ol < ob.nx ? ol : -1;
            }
            mapx[i] = v;
        }
        for (int i = tid; i < PYa; i += NT) {
            int yl = i - R, v = -1;
            if (fy || (yl >= 0 && yl < ny)) {
                if (fy) yl = pmod(yl, ny);
                int ol = pmod(nb.oy + yl - ob.oy, D.ny);
                v = ol < ob.ny ? ol : -1;
            }
            mapy[i] = v;
        }
        for (int i = tid; i < nx; i += NT) gx[i] = pmod(nb.ox + i, D.nx);
        for (int i = tid; i < ny; i += NT) gy[i] = pmod(nb.oy + i, D.ny);
        const int ps_old = plane_stride(ob.nx, ob.ny);
        const int ps_new = plane_stride(nx, ny);
        const uint32_t bytes = (uint32_t)ps_old * 4u;
        const int zlo = -R, zhi = nz + R;
        auto zold_of = [&](int zin) -> int {
            if (!fzf && (zin < 0 || zin >= nz)) return -1;
            int zl = fzf ? pmod(zin, nz) : zin;
            int ol = pmod(nb.oz + zl - ob.oz, D.nz);
            return ol < ob.nz ? ol : -1;
        };
        const float* Xold = B.X + ob.off;
        if (tid == 0) {
            fence_async_smem();
            for (int j = 0; j < kSlots; ++j) {
                const int zin = zlo + j;
                if (zin < zhi) {
                    const int zo = zold_of(zin);
                    if (zo >= 0) {
                        mbar_expect(&bar[j], bytes);
                        bulk_load(raw + j * L::PS, Xold + (long long)zo * ps_old, bytes, &bar[j]);
                    }
                }
            }
        }
        __syncthreads();
        const int sx = tid % nx, y0 = (tid / nx) * V;
        const bool own = y0 < ny;
        const int nxs = (nx + kVX - 1) / kVX;
        const FastDiv fdPX(PXa), fdXS(nxs);
        float ring[W][V];
#pragma unroll
        for (int k = 0; k < W; ++k)
#pragma unroll
            for (int v = 0; v < V; ++v) ring[k][v] = 0.0f;
        // second-key atomics of the previous output plane, issued one plane late
        // so the first atomics' return values arrive while this plane is computed
        unsigned long long pend_old[V];
        float pend_val[V];
        int pend_g[V];            // domain cell index (< 2^31)
#pragma unroll
        for (int v = 0; v < V; ++v) { pend_old[v] = 0; pend_val[v] = 0.0f; pend_g[v] = 0; }
        int slot = 0;
        for (int zin = zlo; zin < zhi; ++zin) {
            const int zl = zold_of(zin);
            bool ok = true;
            if (zl >= 0) {
                ok = mbar_wait(&bar[slot], (phase >> slot) & 1u);
                phase ^= 1u << slot;
            }
            const float* rs = raw + slot * L::PS;
            for (int idx = tid; idx < PXa * PYa; idx += NT) {
                const int yp = fdPX.div(idx), xp = idx - yp * PXa;
                const int mx = mapx[xp], my = mapy[yp];
                float v = -eps;
                if (zl >= 0 && mx >= 0 && my >= 0) v = rs[my * ob.nx + mx];
                P[idx] = v;
            }
            if (__syncthreads_or(!ok)) { give_up(B, bar, phase); return; }
            if (tid == 0) {
                const int zn = zin + kSlots;
                if (zn < zhi) {
                    const int zz = zold_of(zn);
                    if (zz >= 0) {
                        fence_async_smem();
                        mbar_expect(&bar[slot], bytes);
                        bulk_load(raw + slot * L::PS, Xold + (long long)zz * ps_old, bytes, &bar[slot]);
                    }
                }
            }
            slot = slot + 1 == kSlots ? 0 : slot + 1;
            // x pass: kVX outputs per thread from one window of the staged row
            for (int t = tid; t < PYa * nxs; t += NT) {
                const int yp = fdXS.div(t), x0 = (t - yp * nxs) * kVX;
                const float* row = P + yp * PXa + x0;
                float in[kVX + 2 * R];
#pragma unroll
                for (int j = 0; j < kVX + 2 * R; ++j) in[j] = x0 + j < PXa ? row[j] : 0.0f;
#pragma unroll
                for (int v = 0; v < kVX; ++v) {
                    float acc = 0.0f;
#pragma unroll
                    for (int k = 0; k < W; ++k) acc = fmaf(taps.g[k], in[v + k], acc);
                    if (x0 + v < nx) Xp[yp * nx + x0 + v] = acc;
                }
            }
            __syncthreads();
            // pending second keys of the previous plane (their first atomics have returned)
#pragma unroll
            for (int v = 0; v < V; ++v)
                if (pend_old[v]) {
                    const unsigned long long k = make_key(pend_val[v], b);
                    atomicMax(&B.T[2 * (long long)pend_g[v] + 1], pend_old[v] < k ? pend_old[v] : k);
                }
            // rotate the ring: ring[k] holds plane zin - (W - 1) + k
#pragma unroll
            for (int k = 0; k < W - 1; ++k)
#pragma unroll
                for (int v = 0; v < V; ++v) ring[k][v] = ring[k + 1][v];
            if (own) {
                float col[V + 2 * R];
#pragma unroll
                for (int j = 0; j < V + 2 * R; ++j) col[j] = y0 + j < PYa ? Xp[(y0 + j) * nx + sx] : 0.0f;
#pragma unroll
                for (int v = 0; v < V; ++v) {
                    float acc = 0.0f;
#pragma unroll
                    for (int k = 0; k < W; ++k) acc = fmaf(taps.g[k], col[v + k], acc);
                    ring[W - 1][v] = acc;
                }
            }
            // z pass for output plane zo = zin - R: ring[0 .. W-1] = planes zo-R .. zo+R
            const int zo = zin - R;
#pragma unroll
            for (int v = 0; v < V; ++v) pend_old[v] = 0;
            if (own && zo >= 0) {
                const int gz = pmod(nb.oz + zo, D.nz);
                float* dst = B.Y + nb.off + (long long)zo * ps_new;
                const long long grow = (long long)gz * D.ny;
#pragma unroll
                for (int v = 0; v < V; ++v) {
                    const int y = y0 + v;
                    if (y < ny) {
                        float c = 0.0f;
#pragma unroll
                        for (int k = 0; k < W; ++k) c = fmaf(taps.g[k], ring[k][v], c);
                        float val = c;
                        if (phys.kind != LSGG_PHYSICS_IDEAL) {
                            const int ozz = pmod(nb.oz + zo - ob.oz, D.nz);
                            const int mx = mapx[sx + R], my = mapy[y + R];
                            float phi0 = -eps;
                            int j = -1;
                            if (ozz < ob.nz && mx >= 0 && my >= 0) {
                                const long long o = ob.off + (long long)ozz * ps_old + my * ob.nx + mx;
                                phi0 = B.X[o];
                                j = B.IDF[o];
                            }
                            val = pair_blend(phys, tab, b, j, phi0, c);
                        }
                        val = fminf(fmaxf(val, -eps), eps);
                        dst[y * nx + sx] = val;
                        const long long g = (grow + gy[y]) * D.nx + gx[sx];
                        const unsigned long long key = make_key(val, b);
                        pend_old[v] = atomicMax(&B.T[2 * g], key);
                        pend_val[v] = val;
                        pend_g[v] = (int)g;
                    }
                }
            }
        }
#pragma unroll
        for (int v = 0; v < V; ++v)
            if (pend_old[v]) {
                const unsigned long long k = make_key(pend_val[v], b);
                atomicMax(&B.T[2 * (long long)pend_g[v] + 1], pend_old[v] < k ? pend_old[v] : k);
            }
        __syncthreads();
    }
}

// ---------------------------------------------------------------------------
// comparison + taxicab re-initialisation
// ---------------------------------------------------------------------------
template <int SIDE>
struct CorrectLayout {
    static constexpr int A = SIDE * SIDE;
    static constexpr int PS = (A + 3) & ~3;
    static constexpr size_t raw = 128;
    static constexpr size_t C = raw + sizeof(float) * kSlots * PS;
    static constexpr size_t G = C + sizeof(float) * 2 * A;
    static constexpr size_t H = G + sizeof(float) * A;
    static constexpr size_t ints = H + sizeof(float) * A;
    static constexpr size_t bytes = ints + sizeof(int) * (2 * SIDE + 8);
};

// Sign-blocked taxicab sweep over a window of N values `w` (valid[j] false
// where the window leaves a non-periodic box): b[j] = min over positions j'
// reachable through same-sign cells of |w[j']| + |j - j'|, signed like w[j].
template <int N>
__device__ __forceinline__ void window_sweep(float (&w)[N], const bool (&valid)[N]) {
    float f[N];
#pragma unroll
    for (int j = 0; j < N; ++j) {
        float a = fabsf(w[j]);
        if (j > 0 && valid[j] && valid[j - 1] && sgn_pos(w[j]) == sgn_pos(w[j - 1])) a = fminf(a, f[j - 1] + 1.0f);
        f[j] = a;
    }
#pragma unroll
    for (int j = N - 2; j >= 0; --j) {
        if (valid[j] && valid[j + 1] && sgn_pos(w[j]) == sgn_pos(w[j + 1])) f[j] = fminf(f[j], f[j + 1] + 1.0f);
    }
#pragma unroll
    for (int j = 0; j < N; ++j) w[j] = sgn_pos(w[j]) ? f[j] : -f[j];
}

template <int V, int NT, int SIDE, int MINB>
__global__ void __launch_bounds__(NT, MINB)
k_correct_fast(StepBuffers B, PhysicsDev phys, DebugOut dbg, int cls) {
    using L = CorrectLayout<SIDE>;
    constexpr int ZR = kReach + 1;        // F ring depth (7)
    constexpr int NY = V + 2 * kReach;    // y-pass window
    constexpr int NXW = kVD + 2 * kReach; // x-pass window
    extern __shared__ __align__(128) unsigned char sm[];
    uint64_t* bar = reinterpret_cast<uint64_t*>(sm);
    float* raw = reinterpret_cast<float*>(sm + L::raw);
    float* Cs = reinterpret_cast<float*>(sm + L::C);
    float* G = reinterpret_cast<float*>(sm + L::G);
    float* H = reinterpret_cast<float*>(sm + L::H);
    int* gx = reinterpret_cast<int*>(sm + L::ints);
    int* gy = gx + SIDE;
    int* red = gy + SIDE;                 // 6 ints: positive bbox
    __shared__ int s_box;
    const int tid = threadIdx.x;
    if (tid == 0) {
        for (int s = 0; s < kSlots; ++s) mbar_init(&bar[s], 1);
        fence_mbar_init();
    }
    __syncthreads();
    uint32_t phase = 0;
    const Domain D = B.dom;
    const float eps = D.eps;

    for (;;) {
        const int b = pull_box(B, 1, cls, &s_box);
        if (b < 0) break;
        const Box nb = B.cur[b];
        const int nx = nb.nx, ny = nb.ny, nz = nb.nz;
        const int A = nx * ny;
        const bool fx = nx == D.nx, fy = ny == D.ny, fzf = nz == D.nz;
        const int ps = plane_stride(nx, ny);
        const uint32_t bytes = (uint32_t)ps * 4u;
        for (int i = tid; i < nx; i += NT) gx[i] = pmod(nb.ox + i, D.nx);
        for (int i = tid; i < ny; i += NT) gy[i] = pmod(nb.oy + i, D.ny);
        if (tid < 6) red[tid] = tid < 3 ? INT_MAX : INT_MIN;
        const int z_first = fzf ? -(kReach + 1) : 0;
        const int z_last = nz + kReach;       // inclusive
        auto a_plane = [&](int zin) -> int {  // local plane of stage A, or -1 (outside: -eps)
            if (fzf) return pmod(zin, nz);
            return (zin >= 0 && zin < nz) ? zin : -1;
        };
        auto a_wanted = [&](int zin) -> bool { return fzf || zin <= nz; };
        const float* Ybox = B.Y + nb.off;
        if (tid == 0) {
            fence_async_smem();
            for (int j = 0; j < kSlots; ++j) {
                const int zin = z_first + j;
                const int zl = a_plane(zin);
                if (zin <= z_last && a_wanted(zin) && zl >= 0) {
                    mbar_expect(&bar[j], bytes);
                    bulk_load(raw + j * L::PS, Ybox + (long long)zl * ps, bytes, &bar[j]);
                }
            }
        }
        __syncthreads();
        const int sx = tid % nx, y0 = (tid / nx) * V;
        const bool own = y0 < ny;
        float c_m[V], c_0[V], c_p[V];
#pragma unroll
        for (int v = 0; v < V; ++v) { c_m[v] = -eps; c_0[v] = -eps; c_p[v] = -eps; }
        float fr[ZR][V];
#pragma unroll
        for (int k = 0; k < ZR; ++k)
#pragma unroll
            for (int v = 0; v < V; ++v) fr[k][v] = -eps;
        int lo[3] = {INT_MAX, INT_MAX, INT_MAX}, hi[3] = {INT_MIN, INT_MIN, INT_MIN};
        const int zb_first = fzf ? z_first + 1 : 0;
        int slot = 0;
        // field records of the owned cells of the next stage-A plane, loaded a plane early
        ulonglong2 tk[V];
#pragma unroll
        for (int v = 0; v < V; ++v) tk[v] = make_ulonglong2(0ull, 0ull);
        auto load_t = [&](int zin) {
            const int zl = a_plane(zin);
            if (!own || zl < 0 || zin > z_last || !a_wanted(zin)) return;
            const long long grow = (long long)pmod(nb.oz + zl, D.nz) * D.ny;
#pragma unroll
            for (int v = 0; v < V; ++v) {
                const int y = y0 + v;
                if (y < ny) tk[v] = __ldg(reinterpret_cast<const ulonglong2*>(B.T) + (grow + gy[y]) * D.nx + gx[sx]);
            }
        };
        load_t(z_first);
        for (int zin = z_first; zin <= z_last; ++zin) {
            // ---- A: phi_c of plane zin for the owned cells ----
            const bool want = a_wanted(zin);
            const int zl = a_plane(zin);
            bool ok = true;
            if (want && zl >= 0) {
                ok = mbar_wait(&bar[slot], (phase >> slot) & 1u);
                phase ^= 1u << slot;
            }
            if (want) {
#pragma unroll
                for (int v = 0; v < V; ++v) { c_m[v] = c_0[v]; c_0[v] = c_p[v]; }
                if (own) {
                    const float* rs = raw + slot * L::PS;
                    float* Cz = Cs + (zin & 1) * A;
                    const bool record = zin >= 0 && zin < nz;
#pragma unroll
                    for (int v = 0; v < V; ++v) {
                        const int y = y0 + v;
                        float pc = -eps;
                        if (y < ny && zl >= 0) {
                            const int i = y * nx + sx;
                            const float pp = rs[i];
                            const int id1 = key_id(tk[v].x);
                            float m;
                            int mid;
                            if (id1 != b) { m = key_val(tk[v].x, eps); mid = id1; }
                            else { m = key_val(tk[v].y, eps); mid = key_id(tk[v].y); }
                            if (!(m > -eps)) mid = -1;
                            pc = 0.5f * (pp - m);
                            Cz[i] = pc;
                            if (record) {
                                const long long o = nb.off + (long long)zl * ps + i;
                                if (phys.kind != LSGG_PHYSICS_IDEAL) B.IDF[o] = mid;
                                if (dbg.m) { dbg.m[o] = m; dbg.idm[o] = mid; dbg.phic[o] = pc; dbg.phip[o] = pp; }
                            }
                        }
                        c_p[v] = pc;
                    }
                }
            }
            // ---- B: classification of plane zb = zin - 1 (its C plane was written an
            //      iteration ago; its z neighbours are the owned registers) ----
            const int zb = zin - 1;
            const bool do_b = zb >= zb_first && (fzf ? zb <= nz + kReach - 1 : zb < nz);
            if (do_b && own) {
                const float* C0 = Cs + (zb & 1) * A;
#pragma unroll
                for (int v = 0; v < V; ++v) {
                    const int y = y0 + v;
                    if (y >= ny) continue;
                    const int i = y * nx + sx;
                    const float val = c_0[v];
                    const float xl = sx > 0 ? C0[i - 1] : (fx ? C0[i + nx - 1] : -eps);
                    const float xr = sx < nx - 1 ? C0[i + 1] : (fx ? C0[i - nx + 1] : -eps);
                    const float yl = y > 0 ? C0[i - nx] : (fy ? C0[i + (ny - 1) * nx] : -eps);
                    const float yr = y < ny - 1 ? C0[i + nx] : (fy ? C0[i - (ny - 1) * nx] : -eps);
                    G[i] = classify_cell(val, xl, xr, yl, yr, c_m[v], c_p[v], eps);
                }
            }
            load_t(zin + 1);
            if (__syncthreads_or(!ok)) { give_up(B, bar, phase); return; }
            if (tid == 0) {
                // refill this slot with the plane kSlots ahead (if it needs a copy)
                const int zn = zin + kSlots;
                const int zz = a_plane(zn);
                if (zn <= z_last && a_wanted(zn) && zz >= 0) {
                    fence_async_smem();
                    mbar_expect(&bar[slot], bytes);
                    bulk_load(raw + slot * L::PS, Ybox + (long long)zz * ps, bytes, &bar[slot]);
                }
            }
            slot = slot + 1 == kSlots ? 0 : slot + 1;
            if (do_b) {
                // ---- x pass: G -> H, kVD outputs per thread ----
                const int nxs = (nx + kVD - 1) / kVD;
                const FastDiv fdXD(nxs);
                for (int t = tid; t < ny * nxs; t += NT) {
                    const int y = fdXD.div(t), x0 = (t - y * nxs) * kVD;
                    const float* row = G + y * nx;
                    float w[NXW];
                    bool valid[NXW];
                    if (!fx) {
#pragma unroll
                        for (int j = 0; j < NXW; ++j) {
                            const int x = x0 - kReach + j;
                            valid[j] = x >= 0 && x < nx;
                            w[j] = valid[j] ? row[x] : 0.0f;
                        }
                    } else {
#pragma unroll
                        for (int j = 0; j < NXW; ++j) {
                            valid[j] = true;
                            w[j] = row[pmod(x0 - kReach + j, nx)];
                        }
                    }
                    window_sweep<NXW>(w, valid);
#pragma unroll
                    for (int v = 0; v < kVD; ++v)
                        if (x0 + v < nx) H[y * nx + x0 + v] = w[kReach + v];
                }
            }
            __syncthreads();
            // ---- y pass (owned column segment) + forward z sweep: fr[ZR-1] = plane zb ----
            if (do_b) {
#pragma unroll
                for (int k = 0; k < ZR - 1; ++k)
#pragma unroll
                    for (int v = 0; v < V; ++v) fr[k][v] = fr[k + 1][v];
                if (own) {
                    float w[NY];
                    bool valid[NY];
                    if (!fy) {
#pragma unroll
                        for (int j = 0; j < NY; ++j) {
                            const int y = y0 - kReach + j;
                            valid[j] = y >= 0 && y < ny;
                            w[j] = valid[j] ? H[y * nx + sx] : 0.0f;
                        }
                    } else {
#pragma unroll
                        for (int j = 0; j < NY; ++j) {
                            valid[j] = true;
                            w[j] = H[pmod(y0 - kReach + j, ny) * nx + sx];
                        }
                    }
                    window_sweep<NY>(w, valid);
                    const bool first = zb == zb_first;
#pragma unroll
                    for (int v = 0; v < V; ++v) {
                        float val = w[kReach + v];
                        const float p = fr[ZR - 2][v];
                        if (!first && sgn_pos(p) == sgn_pos(val)) {
                            const float mm = fminf(fabsf(val), fabsf(p) + 1.0f);
                            val = sgn_pos(val) ? mm : -mm;
                        }
                        fr[ZR - 1][v] = val;
                    }
                }
            } else {
                // planes past the box end: shift so that fr[0] stays plane zb - kReach
#pragma unroll
                for (int k = 0; k < ZR - 1; ++k)
#pragma unroll
                    for (int v = 0; v < V; ++v) fr[k][v] = fr[k + 1][v];
            }
            // ---- E: backward z window over fr[0 .. 6] = planes zo .. zo + 6 ----
            const int zo = zb - kReach;
            if (own && zo >= 0 && zo < nz) {
                const int ztop = fzf ? zb : min(zb, nz - 1);
                float* dst = B.X + nb.off + (long long)zo * ps;
#pragma unroll
                for (int v = 0; v < V; ++v) {
                    const int y = y0 + v;
                    if (y >= ny) continue;
                    const float val = fr[0][v];
                    const bool sg = sgn_pos(val);
                    float best = fabsf(val);
                    bool go = true;
#pragma unroll
                    for (int k = 1; k <= kReach; ++k) {
                        const float u = fr[k][v];
                        go = go && (zo + k <= ztop) && (sgn_pos(u) == sg);
                        if (go) best = fminf(best, fabsf(u) + (float)k);
                    }
                    best = fminf(best, eps);
                    const float out = sg ? best : -best;
                    const int i = y * nx + sx;
                    dst[i] = out;
                    if (dbg.phin) dbg.phin[nb.off + (long long)zo * ps + i] = out;
                    if (out > 0.0f) {
                        lo[0] = min(lo[0], sx); hi[0] = max(hi[0], sx);
                        lo[1] = min(lo[1], y); hi[1] = max(hi[1], y);
                        lo[2] = min(lo[2], zo); hi[2] = max(hi[2], zo);
                    }
                }
            }
        }
        // ---- positive bounding box of the box ----
#pragma unroll
        for (int a = 0; a < 3; ++a) {
            int l = lo[a], h = hi[a];
#pragma unroll
            for (int o = 16; o > 0; o >>= 1) {
                l = min(l, __shfl_xor_sync(0xffffffffu, l, o));
                h = max(h, __shfl_xor_sync(0xffffffffu, h, o));
            }
            if ((tid & 31) == 0) { atomicMin(&red[a], l); atomicMax(&red[3 + a], h); }
        }
        __syncthreads();
        if (tid == 0) {
            Bounds bd;
            for (int a = 0; a < 3; ++a) { bd.lo[a] = red[a]; bd.hi[a] = red[3 + a]; }
            B.bounds[b] = bd;
        }
        __syncthreads();
    }
}

}  // namespace fast

// One compiled (V, NT) instance of both kernels for a size class.
struct FastKernel {
    const void* fn;
    size_t smem;
    int threads;
};

}  // namespace lsgg
