// Pass path of the batched step for 3D boxes whose x and y sides are at most
// 64: passes over (box, plane), (box, column chunk) and domain-tile work items.
//
// Same arithmetic as the box-streaming kernels (Sec. 2.1.4 predictor, Eq. (16)
// comparison, Sec. 2.1.6 taxicab re-initialisation), arranged so that every
// pass is a persistent grid striding over the work items of all boxes at once:
// the many short, independent items keep every SM busy where one CTA per box
// serialised a whole box along z.  The fields between passes go through HBM:
//   k_bin       per box: list it in every domain tile it overlaps; reset its
//               positive bounding box
//   p_conv_xy   (box, plane): stage the plane of phi (old box -> new box, -eps
//               outside), x and y passes in shared memory   -> Z = xy-convolved
//   p_conv_z    (box, columns): z pass over a register window, velocity
//               correction, clamp                                -> Y = phi_p
//   p_field     (domain tile): top-2 keys (phi_p, -id) over the tile's boxes
//               in registers -> T; then phi_c = (phi_p - m) / 2 and the
//               ID-field for every box cell of the tile          -> Z = phi_c
//   p_redist_xy (box, plane): reference cells with their planar-exact
//               distances, x and y sign-blocked taxicab passes   -> Y
//   p_redist_z  (box, columns): forward sweep + 6-plane backward window along
//               z, clamp, positive bounding box                  -> X = phi
// The field pass replaces the box-streaming kernels' atomic scatter: each
// domain cell's top-2 is built by the one thread that owns the cell, so the
// step has no atomics on the field.  The work-item lists are written by the
// box update; boxes of x, y side <= 32 (tier 0) and <= 64 (tier 1) have their
// own lists and launches, so the plane passes of small boxes run with small
// CTAs and high occupancy.  A non-periodic box's planes outside it are -eps;
// their xy convolution is the constant that p_conv_z recomputes with the FMA
// sequence p_conv_xy would use.
#include <cfloat>
#include <climits>

#include "kernels_common.cuh"

namespace lsgg {

constexpr int kPVX = 4;              // convolution x-pass outputs per task
constexpr int kPVD = 8;              // taxicab x-pass outputs per task
constexpr int kPVY = 8;              // taxicab y-pass outputs per task
constexpr int kPCY = 4;              // convolution y-pass outputs per task
constexpr int kZB = 8;               // planes loaded ahead by the column passes
constexpr int kReachP = kRedistReach;
constexpr int kColThreads = kPassChunk;

__device__ __forceinline__ bool halted(const StepBuffers& B) { return *(volatile int*)&B.st->halt != 0; }

// xy convolution of a plane that is -eps everywhere (the W-tap FMA chains of p_conv_xy)
template <int R>
__device__ __forceinline__ float conv_xy_of_const(const float (&g)[2 * R + 1], float v) {
    float a = 0.0f;
#pragma unroll
    for (int k = 0; k < 2 * R + 1; ++k) a = fmaf(g[k], v, a);
    float c = 0.0f;
#pragma unroll
    for (int k = 0; k < 2 * R + 1; ++k) c = fmaf(g[k], a, c);
    return c;
}

// ---------------------------------------------------------------------------
// pass 1: xy convolution of one plane
// ---------------------------------------------------------------------------
template <int R>
__global__ void __launch_bounds__(256)
p_conv_xy(StepBuffers B, Taps taps, int tier) {
    constexpr int W = 2 * R + 1;
    extern __shared__ __align__(16) float sm[];
    if (halted(B)) return;
    const Domain D = B.dom;
    float g[W];
#pragma unroll
    for (int k = 0; k < W; ++k) g[k] = taps.g[k];
    const int side = B.tier_side[tier];
    float* P = sm;                                          // (side+2R)^2 staged plane
    float* Xp = P + (side + 2 * R) * (side + 2 * R);        // (side+2R) rows x side after the x pass
    int* mapx = reinterpret_cast<int*>(Xp + side * (side + 2 * R));
    int* mapy = mapx + side + 2 * R;
    const int n_items = B.st->n_planes[tier];
    const int2* items = B.plane_items + B.st->plane_base[tier];
    for (int item = blockIdx.x; item < n_items; item += gridDim.x) {
        const int2 it = items[item];
        const int b = it.x, z = it.y;
        const Box nb = B.cur[b], ob = B.prev[b];
        const int nx = nb.nx, ny = nb.ny;
        const bool fx = nx == D.nx, fy = ny == D.ny;
        const int PXa = nx + 2 * R, PYa = ny + 2 * R;
        __syncthreads();                                    // previous item done with the buffers
        for (int i = threadIdx.x; i < PXa; i += blockDim.x) {
            int xl = i - R, v = -1;
            if (fx || (xl >= 0 && xl < nx)) {
                if (fx) xl = pmod(xl, nx);
                const int ol = pmod(nb.ox + xl - ob.ox, D.nx);
                v = ol < ob.nx ? ol : -1;
            }
            mapx[i] = v;
        }
        for (int i = threadIdx.x; i < PYa; i += blockDim.x) {
            int yl = i - R, v = -1;
            if (fy || (yl >= 0 && yl < ny)) {
                if (fy) yl = pmod(yl, ny);
                const int ol = pmod(nb.oy + yl - ob.oy, D.ny);
                v = ol < ob.ny ? ol : -1;
            }
            mapy[i] = v;
        }
        const int ozl = pmod(nb.oz + z - ob.oz, D.nz);
        const int zold = ozl < ob.nz ? ozl : -1;
        const float* src = B.X + ob.off + (long long)(zold < 0 ? 0 : zold) * plane_stride(ob.nx, ob.ny);
        const Div16 dPX(PXa);
        __syncthreads();
        for (int idx = threadIdx.x; idx < PXa * PYa; idx += blockDim.x) {
            const int yp = dPX(idx), xp = idx - yp * PXa;
            const int mx = mapx[xp], my = mapy[yp];
            P[idx] = (zold >= 0 && mx >= 0 && my >= 0) ? src[my * ob.nx + mx] : -D.eps;
        }
        __syncthreads();
        const int nxs = (nx + kPVX - 1) / kPVX;
        const Div16 dXS(nxs);
        for (int t = threadIdx.x; t < PYa * nxs; t += blockDim.x) {
            const int yp = dXS(t), x0 = (t - yp * nxs) * kPVX;
            const float* row = P + yp * PXa + x0;
            float in[kPVX + 2 * R];
#pragma unroll
            for (int j = 0; j < kPVX + 2 * R; ++j) in[j] = x0 + j < PXa ? row[j] : 0.0f;
#pragma unroll
            for (int v = 0; v < kPVX; ++v) {
                float acc = 0.0f;
#pragma unroll
                for (int k = 0; k < W; ++k) acc = fmaf(g[k], in[v + k], acc);
                if (x0 + v < nx) Xp[yp * nx + x0 + v] = acc;
            }
        }
        __syncthreads();
        float* dst = B.Z + nb.off + (long long)z * plane_stride(nx, ny);
        const Div16 dNX(nx);
        const int nys = (ny + kPCY - 1) / kPCY;
        for (int t = threadIdx.x; t < nx * nys; t += blockDim.x) {
            const int ys = dNX(t), x = t - ys * nx;
            const int y0 = ys * kPCY;
            const float* col = Xp + y0 * nx + x;
            float in[kPCY + 2 * R];
#pragma unroll
            for (int j = 0; j < kPCY + 2 * R; ++j) in[j] = y0 + j < PYa ? col[j * nx] : 0.0f;
#pragma unroll
            for (int v = 0; v < kPCY; ++v) {
                float acc = 0.0f;
#pragma unroll
                for (int k = 0; k < W; ++k) acc = fmaf(g[k], in[v + k], acc);
                if (y0 + v < ny) dst[(y0 + v) * nx + x] = acc;
            }
        }
    }
}

// ---------------------------------------------------------------------------
// pass 2: z convolution per column, velocity correction, clamp
// ---------------------------------------------------------------------------
template <int R, bool PHYS>
__global__ void __launch_bounds__(kColThreads)
p_conv_z(StepBuffers B, Taps taps, PhysicsDev phys, int tier) {
    constexpr int W = 2 * R + 1;
    __shared__ int s_tj[PHYS ? kNbCap : 1];
    __shared__ float s_tw[PHYS ? kNbCap : 1], s_tm[PHYS ? kNbCap : 1];
    if (halted(B)) return;
    const Domain D = B.dom;
    float g[W];
#pragma unroll
    for (int k = 0; k < W; ++k) g[k] = taps.g[k];
    const float cconst = conv_xy_of_const<R>(g, -D.eps);
    const int n_items = B.st->n_chunks[tier];
    const int2* items = B.chunk_items + B.st->chunk_base[tier];
    const bool rs = PHYS && phys.kind == LSGG_PHYSICS_READ_SHOCKLEY;
    int last_b = -1;
    PairTable tab{s_tj, s_tw, s_tm, 0};
    for (int item = blockIdx.x; item < n_items; item += gridDim.x) {
        const int2 it = items[item];
        const int b = it.x;
        if (rs && b != last_b) {                           // uniform across the CTA
            __syncthreads();
            tab = load_pair_table(phys, b, s_tj, s_tw, s_tm);
            __syncthreads();
        }
        last_b = b;
        const Box nb = B.cur[b], ob = B.prev[b];
        const int nx = nb.nx, ny = nb.ny, nz = nb.nz;
        const bool fz = nz == D.nz;
        const int c = it.y * kPassChunk + threadIdx.x;
        if (c >= nx * ny) continue;
        const int ps = plane_stride(nx, ny);
        const float* zc = B.Z + nb.off + c;
        float* yc = B.Y + nb.off + c;
        int oxl = 0, oyl = 0;
        bool in_old_xy = false;
        if (PHYS) {
            const int y = c / nx, x = c - y * nx;
            oxl = pmod(nb.ox + x - ob.ox, D.nx);
            oyl = pmod(nb.oy + y - ob.oy, D.ny);
            in_old_xy = oxl < ob.nx && oyl < ob.ny;
        }
        const int ps_old = plane_stride(ob.nx, ob.ny);
        float win[W];                                      // planes zo-R .. zo+R
#pragma unroll
        for (int k = 0; k < W; ++k) win[k] = cconst;
        const int n_in = nz + 2 * R;                       // input planes -R .. nz+R-1
        for (int base = 0; base < n_in; base += kZB) {
            float v[kZB];
#pragma unroll
            for (int u = 0; u < kZB; ++u) {
                const int zin = base + u - R;
                v[u] = cconst;
                if (base + u < n_in) {
                    if (fz) v[u] = zc[(long long)pmod(zin, nz) * ps];
                    else if (zin >= 0 && zin < nz) v[u] = zc[(long long)zin * ps];
                }
            }
#pragma unroll
            for (int u = 0; u < kZB; ++u) {
                if (base + u >= n_in) break;
#pragma unroll
                for (int k = 0; k < W - 1; ++k) win[k] = win[k + 1];
                win[W - 1] = v[u];
                const int zo = base + u - 2 * R;
                if (zo < 0) continue;
                float acc = 0.0f;
#pragma unroll
                for (int k = 0; k < W; ++k) acc = fmaf(g[k], win[k], acc);
                float val = acc;
                if (PHYS) {
                    const int ozl = pmod(nb.oz + zo - ob.oz, D.nz);
                    float phi0 = -D.eps;
                    int j = -1;
                    if (in_old_xy && ozl < ob.nz) {
                        const long long o = ob.off + (long long)ozl * ps_old + (long long)oyl * ob.nx + oxl;
                        phi0 = B.X[o];
                        j = B.IDF[o];
                    }
                    val = pair_blend(phys, tab, b, j, phi0, acc);
                }
                val = fminf(fmaxf(val, -D.eps), D.eps);
                yc[(long long)zo * ps] = val;
            }
        }
    }
}

// ---------------------------------------------------------------------------
// tile lists: every alive box in every domain tile it overlaps
// ---------------------------------------------------------------------------

// Tiles of one axis met by the cyclic cell interval [o, o + n) (0 <= o < N):
// tc tiles from ts on, cyclically.
__device__ __forceinline__ void axis_tiles(int o, int n, int N, int T, int nt, int& ts, int& tc) {
    if (n >= N) { ts = 0; tc = nt; return; }
    const int last = o + n - 1;
    ts = o / T;
    const int te = (last >= N ? last - N : last) / T;
    if (last >= N && te >= ts) { ts = 0; tc = nt; return; }   // wraps into its own first tile
    tc = te >= ts ? te - ts + 1 : te + nt - ts + 1;
}

__global__ void __launch_bounds__(256)
k_bin(StepBuffers B) {
    if (halted(B)) return;
    const Domain D = B.dom;
    const int lane = threadIdx.x & 31;
    const int warps = (blockDim.x >> 5) * gridDim.x;
    for (int b = (blockIdx.x * blockDim.x + threadIdx.x) >> 5; b < B.n_boxes; b += warps) {
        const Box bx = B.cur[b];
        if (bx.nx <= 0) continue;
        if (lane == 0) {
            Bounds bd;
            for (int a = 0; a < 3; ++a) { bd.lo[a] = INT_MAX; bd.hi[a] = INT_MIN; }
            B.bounds[b] = bd;
        }
        int ts[3], tc[3];
        axis_tiles(bx.ox, bx.nx, D.nx, kTileX, B.ntile[0], ts[0], tc[0]);
        axis_tiles(bx.oy, bx.ny, D.ny, kTileY, B.ntile[1], ts[1], tc[1]);
        axis_tiles(bx.oz, bx.nz, D.nz, kTileZ, B.ntile[2], ts[2], tc[2]);
        const int n = tc[0] * tc[1] * tc[2];
        for (int k = lane; k < n; k += 32) {
            const int i = k % tc[0], j = (k / tc[0]) % tc[1], l = k / (tc[0] * tc[1]);
            const int tx = (ts[0] + i) % B.ntile[0], ty = (ts[1] + j) % B.ntile[1], tz = (ts[2] + l) % B.ntile[2];
            const int t = (tz * B.ntile[1] + ty) * B.ntile[0] + tx;
            const int slot = atomicAdd(&B.tile_cnt[t], 1);
            if (slot < kTileCap) B.tile_list[(long long)t * kTileCap + slot] = b;
        }
    }
}

// ---------------------------------------------------------------------------
// field pass: top-2 per domain cell, then the comparison step (Eq. (16))
// ---------------------------------------------------------------------------
// Thread (x, y) of a tile owns the column of kTileZ cells at (x, y); for each
// box covering the column it loads the box's phi_p there and keeps the two
// largest keys (phi_p, -id) per cell in registers -- the same order as the
// box-streaming kernels' atomicMax field, so m and the ID-field are identical.
// Per listed box the CTA first stages, in shared memory, the box-local
// coordinates of the tile's corner and the mask of the tile's planes the box
// covers, so the per-thread work is a compare per column and a load per cell.
struct TileBox {
    long long off;            // arena offset of the box
    int nx, ny;               // box x, y sides
    int dx, dy;               // box-local x, y of the tile corner (cyclic)
    int ps;                   // plane stride
    int id;                   // grain id
    int dz;                   // box-local z of the tile's first plane (cyclic)
    unsigned zmask;           // bit zz: plane zz of the tile lies in the box
};

__device__ __forceinline__ void stage_tile_box(const StepBuffers& B, int b, int tx0, int ty0, int z0, int nzt,
                                               TileBox& t) {
    const Domain& D = B.dom;
    const Box bx = B.cur[b];
    t.off = bx.off;
    t.nx = bx.nx;
    t.ny = bx.ny;
    t.id = b;
    t.ps = plane_stride(bx.nx, bx.ny);
    t.dx = pmod(tx0 - bx.ox, D.nx);
    t.dy = pmod(ty0 - bx.oy, D.ny);
    t.dz = pmod(z0 - bx.oz, D.nz);
    unsigned m = 0;
    if (bx.nx > 0)
        for (int zz = 0; zz < nzt; ++zz) {
            int lz = t.dz + zz;
            if (lz >= D.nz) lz -= D.nz;
            if (lz < bx.nz) m |= 1u << zz;
        }
    t.zmask = m;
}

__global__ void __launch_bounds__(kTileX * kTileY, 2)
p_field(StepBuffers B, PhysicsDev phys, DebugOut dbg) {
    __shared__ TileBox s_tb[kTileCap];
    if (halted(B)) return;
    const Domain D = B.dom;
    const float eps = D.eps;
    const int ntx = B.ntile[0], nty = B.ntile[1];
    const int lx = threadIdx.x % kTileX, ly = threadIdx.x / kTileX;
    for (int tile = blockIdx.x; tile < B.n_tiles; tile += gridDim.x) {
        const int tx = tile % ntx, tyz = tile / ntx, ty = tyz % nty, tz = tyz / nty;
        const int tx0 = tx * kTileX, ty0 = ty * kTileY, z0 = tz * kTileZ;
        const int x = tx0 + lx, y = ty0 + ly;
        const bool col = x < D.nx && y < D.ny;
        const int nzt = min(kTileZ, D.nz - z0);
        const int cnt = B.tile_cnt[tile];
        const bool all = cnt > kTileCap;            // list overflowed: test every box in batches
        const int n_total = all ? B.n_boxes : cnt;
        unsigned long long k1[kTileZ], k2[kTileZ];
#pragma unroll
        for (int zz = 0; zz < kTileZ; ++zz) { k1[zz] = 0ull; k2[zz] = 0ull; }
        // two sweeps over the tile's boxes: 0 builds the top-2, 1 writes phi_c
        for (int sweep = 0; sweep < 2; ++sweep) {
            if (sweep == 1 && col) {
                ulonglong2* T2 = reinterpret_cast<ulonglong2*>(B.T);
#pragma unroll
                for (int zz = 0; zz < kTileZ; ++zz)
                    if (zz < nzt) T2[((long long)(z0 + zz) * D.ny + y) * D.nx + x] = make_ulonglong2(k1[zz], k2[zz]);
            }
            for (int base = 0; base < n_total; base += kTileCap) {
                const int nb = min(kTileCap, n_total - base);
                __syncthreads();                    // previous batch done with s_tb
                for (int k = threadIdx.x; k < nb; k += blockDim.x) {
                    const int b = all ? base + k : B.tile_list[(long long)tile * kTileCap + k];
                    stage_tile_box(B, b, tx0, ty0, z0, nzt, s_tb[k]);
                }
                __syncthreads();
                if (!col) continue;
                for (int k = 0; k < nb; ++k) {
                    const TileBox& t = s_tb[k];
                    if (!t.zmask) continue;
                    int bxl = t.dx + lx, byl = t.dy + ly;
                    if (bxl >= D.nx) bxl -= D.nx;
                    if (byl >= D.ny) byl -= D.ny;
                    if (bxl >= t.nx || byl >= t.ny) continue;
                    const long long o0 = t.off + (long long)byl * t.nx + bxl;
                    const float* src = B.Y + o0;
                    const unsigned zm = t.zmask;
                    const int ps = t.ps, dz = t.dz;
                    float v[kTileZ];
#pragma unroll
                    for (int zz = 0; zz < kTileZ; ++zz) {
                        int lz = dz + zz;
                        if (lz >= D.nz) lz -= D.nz;
                        v[zz] = (zm >> zz) & 1u ? src[lz * ps] : 0.0f;
                    }
                    if (sweep == 0) {
                        const unsigned lo = 0xffffffffu - (unsigned)t.id;
#pragma unroll
                        for (int zz = 0; zz < kTileZ; ++zz) {
                            if (!((zm >> zz) & 1u)) continue;
                            const unsigned long long key = ((unsigned long long)ord_float(v[zz]) << 32) | lo;
                            if (key > k1[zz]) { k2[zz] = k1[zz]; k1[zz] = key; }
                            else if (key > k2[zz]) k2[zz] = key;
                        }
                    } else {
#pragma unroll
                        for (int zz = 0; zz < kTileZ; ++zz) {
                            if (!((zm >> zz) & 1u)) continue;
                            int lz = dz + zz;
                            if (lz >= D.nz) lz -= D.nz;
                            const long long o = o0 + (long long)lz * ps;
                            const int id1 = key_id(k1[zz]);
                            float m;
                            int mid;
                            if (id1 != t.id) { m = key_val(k1[zz], eps); mid = id1; }
                            else { m = key_val(k2[zz], eps); mid = key_id(k2[zz]); }
                            if (!(m > -eps)) mid = -1;
                            const float pc = 0.5f * (v[zz] - m);
                            B.Z[o] = pc;
                            if (phys.kind != LSGG_PHYSICS_IDEAL) B.IDF[o] = mid;
                            if (dbg.m) { dbg.m[o] = m; dbg.idm[o] = mid; dbg.phic[o] = pc; dbg.phip[o] = v[zz]; }
                        }
                    }
                }
            }
        }
    }
}

// ---------------------------------------------------------------------------
// pass 4: classification + x / y taxicab passes of one plane
// ---------------------------------------------------------------------------
template <int N>
__device__ __forceinline__ void sweep_window(float (&w)[N], const bool (&valid)[N]) {
    float f[N];
#pragma unroll
    for (int j = 0; j < N; ++j) {
        float a = fabsf(w[j]);
        if (j > 0 && valid[j] && valid[j - 1] && sgn_pos(w[j]) == sgn_pos(w[j - 1])) a = fminf(a, f[j - 1] + 1.0f);
        f[j] = a;
    }
#pragma unroll
    for (int j = N - 2; j >= 0; --j)
        if (valid[j] && valid[j + 1] && sgn_pos(w[j]) == sgn_pos(w[j + 1])) f[j] = fminf(f[j], f[j + 1] + 1.0f);
#pragma unroll
    for (int j = 0; j < N; ++j) w[j] = sgn_pos(w[j]) ? f[j] : -f[j];
}

__device__ __forceinline__ void axis_inv2(float a, bool pos, float l, float r, float& inv2, bool& zero) {
    float dmin = FLT_MAX;
    opp_delta(a, pos, l, dmin);
    opp_delta(a, pos, r, dmin);
    if (dmin < FLT_MAX) { if (dmin > 0.0f) inv2 += 1.0f / (dmin * dmin); else zero = true; }
}

__global__ void __launch_bounds__(256)
p_redist_xy(StepBuffers B, int tier) {
    extern __shared__ __align__(16) float sm[];
    if (halted(B)) return;
    const Domain D = B.dom;
    const float eps = D.eps;
    const int side = B.tier_side[tier];
    float* C0 = sm;
    float* G = C0 + side * side;
    float* H = G + side * side;
    const int n_items = B.st->n_planes[tier];
    const int2* items = B.plane_items + B.st->plane_base[tier];
    constexpr int NXW = kPVD + 2 * kReachP;
    constexpr int NYW = kPVY + 2 * kReachP;
    for (int item = blockIdx.x; item < n_items; item += gridDim.x) {
        const int2 it = items[item];
        const int b = it.x, z = it.y;
        const Box nb = B.cur[b];
        const int nx = nb.nx, ny = nb.ny, nz = nb.nz, A = nx * ny;
        const bool fx = nx == D.nx, fy = ny == D.ny, fz = nz == D.nz;
        const int ps = plane_stride(nx, ny);
        const float* zb = B.Z + nb.off;
        __syncthreads();                                    // previous item done with the buffers
        for (int i = threadIdx.x; i < A; i += blockDim.x) C0[i] = zb[(long long)z * ps + i];
        const int zm = fz ? pmod(z - 1, nz) : z - 1, zp = fz ? pmod(z + 1, nz) : z + 1;
        const bool has_m = zm >= 0, has_p = zp < nz;
        const Div16 dNX(nx);
        __syncthreads();
        // reference cells (a neighbour of opposite sign) get the planar-exact
        // distance 1 / sqrt(sum over such axes of 1 / d^2); others eps
        for (int i = threadIdx.x; i < A; i += blockDim.x) {
            const int y = dNX(i), x = i - y * nx;
            const float val = C0[i];
            const bool pos = val > 0.0f;
            const float xl = x > 0 ? C0[i - 1] : (fx ? C0[i + nx - 1] : -eps);
            const float xr = x < nx - 1 ? C0[i + 1] : (fx ? C0[i - nx + 1] : -eps);
            const float yl = y > 0 ? C0[i - nx] : (fy ? C0[i + (ny - 1) * nx] : -eps);
            const float yr = y < ny - 1 ? C0[i + nx] : (fy ? C0[i - (ny - 1) * nx] : -eps);
            const float zl = has_m ? zb[(long long)zm * ps + i] : -eps;
            const float zr = has_p ? zb[(long long)zp * ps + i] : -eps;
            const bool any = ((xl > 0.0f) != pos) | ((xr > 0.0f) != pos) | ((yl > 0.0f) != pos) |
                             ((yr > 0.0f) != pos) | ((zl > 0.0f) != pos) | ((zr > 0.0f) != pos);
            float mag = eps;
            if (any) {
                const float a = fabsf(val);
                float inv2 = 0.0f;
                bool zero = false;
                axis_inv2(a, pos, xl, xr, inv2, zero);
                axis_inv2(a, pos, yl, yr, inv2, zero);
                axis_inv2(a, pos, zl, zr, inv2, zero);
                mag = zero ? 0.0f : 1.0f / sqrtf(inv2);
            }
            G[i] = pos ? mag : -mag;
        }
        __syncthreads();
        // x pass G -> H
        const int nxs = (nx + kPVD - 1) / kPVD;
        const Div16 dXS(nxs);
        for (int t = threadIdx.x; t < ny * nxs; t += blockDim.x) {
            const int y = dXS(t), x0 = (t - y * nxs) * kPVD;
            const float* row = G + y * nx;
            float w[NXW];
            bool valid[NXW];
            if (!fx) {
#pragma unroll
                for (int j = 0; j < NXW; ++j) {
                    const int x = x0 - kReachP + j;
                    valid[j] = x >= 0 && x < nx;
                    w[j] = valid[j] ? row[x] : 0.0f;
                }
            } else {
#pragma unroll
                for (int j = 0; j < NXW; ++j) { valid[j] = true; w[j] = row[pmod(x0 - kReachP + j, nx)]; }
            }
            sweep_window<NXW>(w, valid);
#pragma unroll
            for (int v = 0; v < kPVD; ++v)
                if (x0 + v < nx) H[y * nx + x0 + v] = w[kReachP + v];
        }
        __syncthreads();
        // y pass H -> Y
        const int nys = (ny + kPVY - 1) / kPVY;
        float* out = B.Y + nb.off + (long long)z * ps;
        for (int t = threadIdx.x; t < nx * nys; t += blockDim.x) {
            const int ys = dNX(t), x = t - ys * nx;
            const int y0 = ys * kPVY;
            float w[NYW];
            bool valid[NYW];
            if (!fy) {
#pragma unroll
                for (int j = 0; j < NYW; ++j) {
                    const int y = y0 - kReachP + j;
                    valid[j] = y >= 0 && y < ny;
                    w[j] = valid[j] ? H[y * nx + x] : 0.0f;
                }
            } else {
#pragma unroll
                for (int j = 0; j < NYW; ++j) { valid[j] = true; w[j] = H[pmod(y0 - kReachP + j, ny) * nx + x]; }
            }
            sweep_window<NYW>(w, valid);
#pragma unroll
            for (int v = 0; v < kPVY; ++v)
                if (y0 + v < ny) out[(y0 + v) * nx + x] = w[kReachP + v];
        }
    }
}

// ---------------------------------------------------------------------------
// pass 5: z taxicab pass per column, clamp, bounding box of the positive set
// ---------------------------------------------------------------------------
__global__ void __launch_bounds__(kColThreads)
p_redist_z(StepBuffers B, DebugOut dbg, int tier) {
    if (halted(B)) return;
    const Domain D = B.dom;
    const float eps = D.eps;
    constexpr int ZR = kReachP + 1;
    const int n_items = B.st->n_chunks[tier];
    const int2* items = B.chunk_items + B.st->chunk_base[tier];
    for (int item = blockIdx.x; item < n_items; item += gridDim.x) {
        const int2 it = items[item];
        const int b = it.x;
        const Box nb = B.cur[b];
        const int nx = nb.nx, ny = nb.ny, nz = nb.nz;
        const bool fz = nz == D.nz;
        const int c = it.y * kPassChunk + threadIdx.x;
        int lo[3] = {INT_MAX, INT_MAX, INT_MAX}, hi[3] = {INT_MIN, INT_MIN, INT_MIN};
        if (c < nx * ny) {
            const int y = c / nx, x = c - y * nx;
            const int ps = plane_stride(nx, ny);
            const float* hc = B.Y + nb.off + c;
            float* xc = B.X + nb.off + c;
            float fr[ZR];                                  // forward-swept planes zb-6 .. zb
#pragma unroll
            for (int k = 0; k < ZR; ++k) fr[k] = -eps;
            // periodic z: the sweep starts 6 planes early so that plane 0 sees its wrapped predecessors
            const int zb_first = fz ? -kReachP : 0;
            const int n_zb = nz + kReachP - zb_first;      // zb = zb_first .. nz-1+6
            for (int base = 0; base < n_zb; base += kZB) {
                float v[kZB];
#pragma unroll
                for (int u = 0; u < kZB; ++u) {
                    const int zb = zb_first + base + u;
                    v[u] = 0.0f;
                    if (base + u < n_zb && (fz || zb < nz)) v[u] = hc[(long long)(fz ? pmod(zb, nz) : zb) * ps];
                }
#pragma unroll
                for (int u = 0; u < kZB; ++u) {
                    if (base + u >= n_zb) break;
                    const int zb = zb_first + base + u;
#pragma unroll
                    for (int k = 0; k < ZR - 1; ++k) fr[k] = fr[k + 1];
                    if (fz || zb < nz) {
                        float val = v[u];
                        const float p = fr[ZR - 2];
                        if (zb != zb_first && sgn_pos(p) == sgn_pos(val)) {
                            const float mm = fminf(fabsf(val), fabsf(p) + 1.0f);
                            val = sgn_pos(val) ? mm : -mm;
                        }
                        fr[ZR - 1] = val;
                    }
                    const int zo = zb - kReachP;
                    if (zo < 0) continue;
                    const int ztop = fz ? zb : min(zb, nz - 1);
                    const float v0 = fr[0];
                    const bool sg = sgn_pos(v0);
                    float best = fabsf(v0);
                    bool go = true;
#pragma unroll
                    for (int k = 1; k <= kReachP; ++k) {
                        const float w = fr[k];
                        go = go && (zo + k <= ztop) && (sgn_pos(w) == sg);
                        if (go) best = fminf(best, fabsf(w) + (float)k);
                    }
                    best = fminf(best, eps);
                    const float out = sg ? best : -best;
                    xc[(long long)zo * ps] = out;
                    if (dbg.phin) dbg.phin[nb.off + (long long)zo * ps + c] = out;
                    if (out > 0.0f) {
                        lo[0] = min(lo[0], x); hi[0] = max(hi[0], x);
                        lo[1] = min(lo[1], y); hi[1] = max(hi[1], y);
                        lo[2] = min(lo[2], zo); hi[2] = max(hi[2], zo);
                    }
                }
            }
        }
        // every thread of the CTA reaches this point for every item
#pragma unroll
        for (int a = 0; a < 3; ++a) {
            int l = lo[a], h = hi[a];
#pragma unroll
            for (int o = 16; o > 0; o >>= 1) {
                l = min(l, __shfl_xor_sync(0xffffffffu, l, o));
                h = max(h, __shfl_xor_sync(0xffffffffu, h, o));
            }
            if ((threadIdx.x & 31) == 0 && l <= h) {
                atomicMin(&B.bounds[b].lo[a], l);
                atomicMax(&B.bounds[b].hi[a], h);
            }
        }
    }
}

// ---------------------------------------------------------------------------
// host side
// ---------------------------------------------------------------------------
// The radius-specialised convolution kernels (R = 1 .. kMaxRadius); the z pass
// with or without the velocity correction of Eq. (10).
struct PassFns {
    const void* conv_xy;
    const void* conv_z;
};

template <int R>
static PassFns pass_fns_r(bool phys) {
    return PassFns{reinterpret_cast<const void*>(p_conv_xy<R>),
                   phys ? reinterpret_cast<const void*>(p_conv_z<R, true>)
                        : reinterpret_cast<const void*>(p_conv_z<R, false>)};
}

static PassFns pass_fns(int R, bool phys) {
    switch (R) {
        case 1: return pass_fns_r<1>(phys);
        case 2: return pass_fns_r<2>(phys);
        case 3: return pass_fns_r<3>(phys);
        case 4: return pass_fns_r<4>(phys);
        case 5: return pass_fns_r<5>(phys);
        case 6: return pass_fns_r<6>(phys);
        case 7: return pass_fns_r<7>(phys);
        default: return PassFns{nullptr, nullptr};
    }
}

static size_t pass_smem_conv(int side, int R) {
    return sizeof(float) * ((size_t)(side + 2 * R) * (side + 2 * R) + (size_t)side * (side + 2 * R)) +
           sizeof(int) * 2 * (size_t)(side + 2 * R);
}
static size_t pass_smem_redist(int side) { return sizeof(float) * 3 * (size_t)side * side; }

cudaError_t configure_passes(StepBuffers& B) {
    const int sides[kTiers] = {32, 64};
    const int threads[kTiers] = {128, 256};
    for (int t = 0; t < kTiers; ++t) {
        B.tier_side[t] = sides[t];
        B.tier_threads[t] = threads[t];
        B.psmem[t][0] = pass_smem_conv(sides[t], B.dom.radius);
        B.psmem[t][1] = pass_smem_redist(sides[t]);
    }
    const PassFns fn = pass_fns(B.dom.radius, true);
    if (!fn.conv_xy) return cudaErrorInvalidValue;
    cudaError_t e = allow_max_dynamic_smem(fn.conv_xy);
    if (e != cudaSuccess) return e;
    e = allow_max_dynamic_smem(reinterpret_cast<const void*>(p_redist_xy));
    if (e != cudaSuccess) return e;
    for (int t = 0; t < kTiers; ++t) {
        int o[5] = {0, 0, 1, 0, 0};
        e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&o[0], fn.conv_xy, threads[t], B.psmem[t][0]);
        if (e == cudaSuccess) e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&o[1], fn.conv_z, kColThreads, 0);
        if (e == cudaSuccess)
            e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&o[3], p_redist_xy, threads[t], B.psmem[t][1]);
        if (e == cudaSuccess) e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&o[4], p_redist_z, kColThreads, 0);
        if (e != cudaSuccess) return e;
        for (int k = 0; k < 5; ++k) B.pgrid[t][k] = B.n_sm * (o[k] < 1 ? 1 : o[k]);
    }
    int of = 0;
    e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&of, p_field, kTileX * kTileY, 0);
    if (e != cudaSuccess) return e;
    B.field_grid = B.n_sm * (of < 1 ? 1 : of);
    B.bin_grid = B.n_sm;
    const int tsz[3] = {kTileX, kTileY, kTileZ};
    const int dn[3] = {B.dom.nx, B.dom.ny, B.dom.nz};
    for (int a = 0; a < 3; ++a) B.ntile[a] = (dn[a] + tsz[a] - 1) / tsz[a];
    B.n_tiles = B.ntile[0] * B.ntile[1] * B.ntile[2];
    return cudaSuccess;
}

// which = 0: p_conv_xy, p_conv_z; which = 1: p_redist_xy, p_redist_z.
// pass_ev (optional): one event before the first kernel and one after each.
cudaError_t launch_passes(const StepBuffers& B, int which, int tier, const Taps& taps, const PhysicsDev& phys,
                          const DebugOut& dbg, cudaStream_t s, cudaEvent_t* pass_ev) {
    const int nt = B.tier_threads[tier];
    const int* g = B.pgrid[tier];
    int k = 0;
    if (pass_ev) cudaEventRecord(pass_ev[k++], s);
    if (which == 0) {
        const PassFns fn = pass_fns(taps.radius, phys.kind != LSGG_PHYSICS_IDEAL);
        if (!fn.conv_xy) return cudaErrorInvalidValue;
        Taps tp = taps;
        StepBuffers bb = B;
        int tr = tier;
        PhysicsDev ph = phys;
        void* a0[] = {&bb, &tp, &tr};
        cudaError_t e = cudaLaunchKernel(fn.conv_xy, dim3(g[0]), dim3(nt), a0, B.psmem[tier][0], s);
        if (e != cudaSuccess) return e;
        if (pass_ev) cudaEventRecord(pass_ev[k++], s);
        void* a1[] = {&bb, &tp, &ph, &tr};
        e = cudaLaunchKernel(fn.conv_z, dim3(g[1]), dim3(kColThreads), a1, 0, s);
        if (e != cudaSuccess) return e;
        if (pass_ev) cudaEventRecord(pass_ev[k++], s);
    } else {
        p_redist_xy<<<g[3], nt, B.psmem[tier][1], s>>>(B, tier);
        if (pass_ev) cudaEventRecord(pass_ev[k++], s);
        p_redist_z<<<g[4], kColThreads, 0, s>>>(B, dbg, tier);
        if (pass_ev) cudaEventRecord(pass_ev[k++], s);
    }
    return cudaGetLastError();
}

cudaError_t launch_bin(const StepBuffers& B, cudaStream_t s) {
    cudaError_t e = cudaMemsetAsync(B.tile_cnt, 0, sizeof(int) * (size_t)B.n_tiles, s);
    if (e != cudaSuccess) return e;
    k_bin<<<B.bin_grid, 256, 0, s>>>(B);
    return cudaGetLastError();
}

cudaError_t launch_field(const StepBuffers& B, const PhysicsDev& phys, const DebugOut& dbg, cudaStream_t s) {
    p_field<<<B.field_grid, kTileX * kTileY, 0, s>>>(B, phys, dbg);
    return cudaGetLastError();
}

}  // namespace lsgg
