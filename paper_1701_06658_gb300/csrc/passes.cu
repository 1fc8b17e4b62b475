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

constexpr int kZB = 8;               // planes loaded ahead by the column passes
constexpr int kStageU = 8;           // loads in flight per thread when staging a plane
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
// A CTA of SIDE threads takes one (box, plane) item at a time: the plane of
// phi is staged row by row (old box -> new box, -eps outside), then thread x
// walks down column x, convolving each padded row along x from shared memory
// and keeping the last 2R + 1 row results in registers for the y convolution.
template <int R, int SIDE>
__global__ void __launch_bounds__(SIDE)
p_conv_xy(StepBuffers B, Taps taps, int tier) {
    constexpr int W = 2 * R + 1;
    constexpr int PS = SIDE + 2 * R;
    __shared__ float P[(PS + W) * PS];      // W spare rows: the unrolled row loop may read past the plane
    __shared__ int mapx[PS], mapy[PS];
    if (halted(B)) return;
    const Domain D = B.dom;
    float g[W];
#pragma unroll
    for (int k = 0; k < W; ++k) g[k] = taps.g[k];
    const int t = threadIdx.x;
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
        for (int i = t; i < PXa; i += SIDE) {
            int xl = i - R, v = -1;
            if (fx || (xl >= 0 && xl < nx)) {
                if (fx) xl = pmod(xl, nx);
                const int ol = pmod(nb.ox + xl - ob.ox, D.nx);
                v = ol < ob.nx ? ol : -1;
            }
            mapx[i] = v;
        }
        for (int i = t; i < PYa; i += SIDE) {
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
        __syncthreads();
        {   // stage the padded plane, kStageU loads in flight per thread
            const int n = PXa * PYa;
            const Div16 dPX(PXa);
            for (int i0 = t; i0 < n; i0 += SIDE * kStageU) {
                float v[kStageU];
#pragma unroll
                for (int u = 0; u < kStageU; ++u) {
                    const int i = i0 + u * SIDE;
                    v[u] = -D.eps;
                    if (i < n && zold >= 0) {
                        const int yp = dPX(i), xp = i - yp * PXa;
                        const int mx = mapx[xp], my = mapy[yp];
                        if (mx >= 0 && my >= 0) v[u] = src[my * ob.nx + mx];
                    }
                }
#pragma unroll
                for (int u = 0; u < kStageU; ++u)
                    if (i0 + u * SIDE < n) P[i0 + u * SIDE] = v[u];
            }
        }
        __syncthreads();
        if (t < nx) {
            float* dst = B.Z + nb.off + (long long)z * plane_stride(nx, ny) + t;
            const float* prow = P + t;
            float win[W];                                   // x-convolved rows, slot = row mod W
            for (int yb = 0; yb < PYa; yb += W) {
                // W rows per trip without branches, so that their independent FMA
                // chains interleave; rows past the plane are computed and dropped
#pragma unroll
                for (int s = 0; s < W; ++s) {
                    const int yp = yb + s;
                    const float* r = prow + yp * PXa;
                    float acc = 0.0f;
#pragma unroll
                    for (int k = 0; k < W; ++k) acc = fmaf(g[k], r[k], acc);
                    win[s] = acc;
                    float o = 0.0f;                         // output row y = yp - 2R: rows y .. yp
#pragma unroll
                    for (int k = 0; k < W; ++k) o = fmaf(g[k], win[(s + 1 + k) % W], o);
                    if (yp >= 2 * R && yp < PYa) dst[(yp - 2 * R) * nx] = o;
                }
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

__global__ void __launch_bounds__(kTileX * kTileY, 3)
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
// Sign-blocked min-plus along one line of n cells, in place (stride st):
// f_j = min(|v_j|, f_{j-1} + 1) over a run of one sign, forward then backward.
// A periodic line is swept twice around in each direction.  Cells further
// than 6 apart add at least 7 >= eps, so this equals the 6-step window of
// the box-streaming kernels.  `out` (optional) receives the final values.
__device__ __forceinline__ void line_sweep(float* L, int n, int st, bool wrap, float* out, int out_st) {
    const int laps = wrap ? 2 : 1;
    float fp = 0.0f;
    bool sp = false;
    for (int j = 0; j < laps * n; ++j) {
        const int i = j < n ? j : j - n;
        const float v = L[i * st];
        const bool sv = sgn_pos(v);
        float a = fabsf(v);
        if (j > 0 && sv == sp) a = fminf(a, fp + 1.0f);
        L[i * st] = sv ? a : -a;
        fp = a;
        sp = sv;
    }
    for (int j = laps * n - 2; j >= 0; --j) {
        const int i = j < n ? j : j - n;
        const float v = L[i * st];
        const bool sv = sgn_pos(v);
        float a = fabsf(v);
        if (sv == sp) a = fminf(a, fp + 1.0f);
        const float f = sv ? a : -a;
        L[i * st] = f;
        if (out && j < n) out[i * out_st] = f;
        fp = a;
        sp = sv;
    }
    if (out) {                                       // the last cell is final after the forward sweep
        const int i = n - 1;
        if (laps == 1) out[i * out_st] = L[i * st];
    }
}

template <int SIDE>
__global__ void __launch_bounds__(SIDE)
p_redist_xy(StepBuffers B, int tier) {
    constexpr int PG = SIDE + 1;                      // odd pitch: row sweeps hit distinct banks
    constexpr int U = 4;                              // rows classified per trip
    __shared__ float G[(SIDE + U) * PG];              // U spare rows for the unrolled trip
    if (halted(B)) return;
    const Domain D = B.dom;
    const float eps = D.eps;
    const int t = threadIdx.x;
    const int n_items = B.st->n_planes[tier];
    const int2* items = B.plane_items + B.st->plane_base[tier];
    for (int item = blockIdx.x; item < n_items; item += gridDim.x) {
        const int2 it = items[item];
        const int b = it.x, z = it.y;
        const Box nb = B.cur[b];
        const int nx = nb.nx, ny = nb.ny, nz = nb.nz;
        const bool fx = nx == D.nx, fy = ny == D.ny, fz = nz == D.nz;
        const int ps = plane_stride(nx, ny);
        const float* zb = B.Z + nb.off;
        const int zm = fz ? pmod(z - 1, nz) : z - 1, zp = fz ? pmod(z + 1, nz) : z + 1;
        const bool has_m = zm >= 0, has_p = zp < nz;
        __syncthreads();                                    // previous item done with G
        if (t < nx) {                                       // classification, thread = column
            // phi_c of plane z and of its z neighbours, read through L1: row y of
            // the plane is loaded by the whole CTA, so the x neighbours hit L1
            const int x = t;
            const float* c = zb + (long long)z * ps;
            const float* cm = zb + (long long)(has_m ? zm : 0) * ps;
            const float* cp = zb + (long long)(has_p ? zp : 0) * ps;
            const int xl_i = x > 0 ? x - 1 : (fx ? nx - 1 : -1);
            const int xr_i = x < nx - 1 ? x + 1 : (fx ? 0 : -1);
            float c_prev = fy ? __ldg(c + (ny - 1) * nx + x) : -eps;
            float c_cur = __ldg(c + x);
            for (int y0 = 0; y0 < ny; y0 += U) {
                float cv[U + 1], xl[U], xr[U], zl[U], zr[U];
                cv[0] = c_cur;
#pragma unroll
                for (int u = 0; u < U; ++u) {
                    const int y = y0 + u;
                    const bool in = y < ny;
                    const int yn = y + 1 < ny ? y + 1 : (fy ? 0 : -1);
                    cv[u + 1] = in && yn >= 0 ? __ldg(c + yn * nx + x) : -eps;
                    xl[u] = in && xl_i >= 0 ? __ldg(c + y * nx + xl_i) : -eps;
                    xr[u] = in && xr_i >= 0 ? __ldg(c + y * nx + xr_i) : -eps;
                    zl[u] = in && has_m ? __ldg(cm + y * nx + x) : -eps;
                    zr[u] = in && has_p ? __ldg(cp + y * nx + x) : -eps;
                }
#pragma unroll
                for (int u = 0; u < U; ++u) {
                    const float yl = u ? cv[u - 1] : c_prev;
                    G[(y0 + u) * PG + x] = classify_cell(cv[u], xl[u], xr[u], yl, cv[u + 1], zl[u], zr[u], eps);
                }
                c_prev = cv[U - 1];
                c_cur = cv[U];
            }
        }
        __syncthreads();
        if (t < ny) line_sweep(G + t * PG, nx, 1, fx, nullptr, 0);      // x pass, thread = row
        __syncthreads();
        if (t < nx)                                         // y pass, thread = column -> Y
            line_sweep(G + t, ny, PG, fy, B.Y + nb.off + (long long)z * ps + t, nx);
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
// The radius-specialised convolution kernels (R = 1 .. kMaxRadius) per tier
// side; the z pass with or without the velocity correction of Eq. (10).
constexpr int kTierSide[kTiers] = {32, 64};

struct PassFns {
    const void* conv_xy[kTiers];
    const void* conv_z;
    const void* redist_xy[kTiers];
};

template <int R>
static PassFns pass_fns_r(bool phys) {
    static_assert(kTiers == 2, "one instantiation per tier side");
    PassFns f;
    f.conv_xy[0] = reinterpret_cast<const void*>(p_conv_xy<R, 32>);
    f.conv_xy[1] = reinterpret_cast<const void*>(p_conv_xy<R, 64>);
    f.conv_z = phys ? reinterpret_cast<const void*>(p_conv_z<R, true>) : reinterpret_cast<const void*>(p_conv_z<R, false>);
    f.redist_xy[0] = reinterpret_cast<const void*>(p_redist_xy<32>);
    f.redist_xy[1] = reinterpret_cast<const void*>(p_redist_xy<64>);
    return f;
}

static bool pass_fns(int R, bool phys, PassFns* f) {
    switch (R) {
        case 1: *f = pass_fns_r<1>(phys); return true;
        case 2: *f = pass_fns_r<2>(phys); return true;
        case 3: *f = pass_fns_r<3>(phys); return true;
        case 4: *f = pass_fns_r<4>(phys); return true;
        case 5: *f = pass_fns_r<5>(phys); return true;
        case 6: *f = pass_fns_r<6>(phys); return true;
        case 7: *f = pass_fns_r<7>(phys); return true;
        default: return false;
    }
}

cudaError_t configure_passes(StepBuffers& B) {
    PassFns fn;
    if (!pass_fns(B.dom.radius, true, &fn)) return cudaErrorInvalidValue;
    cudaError_t e = cudaSuccess;
    for (int t = 0; t < kTiers; ++t) {
        B.tier_side[t] = kTierSide[t];
        B.tier_threads[t] = kTierSide[t];
        int o[5] = {0, 0, 1, 0, 0};
        e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&o[0], fn.conv_xy[t], kTierSide[t], 0);
        if (e == cudaSuccess) e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&o[1], fn.conv_z, kColThreads, 0);
        if (e == cudaSuccess) e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&o[3], fn.redist_xy[t], kTierSide[t], 0);
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
    PassFns fn;
    if (!pass_fns(taps.radius, phys.kind != LSGG_PHYSICS_IDEAL, &fn)) return cudaErrorInvalidValue;
    const int nt = B.tier_threads[tier];
    const int* g = B.pgrid[tier];
    StepBuffers bb = B;
    Taps tp = taps;
    PhysicsDev ph = phys;
    DebugOut db = dbg;
    int tr = tier;
    int k = 0;
    cudaError_t e;
    if (pass_ev) cudaEventRecord(pass_ev[k++], s);
    if (which == 0) {
        void* a0[] = {&bb, &tp, &tr};
        e = cudaLaunchKernel(fn.conv_xy[tier], dim3(g[0]), dim3(nt), a0, 0, s);
        if (e != cudaSuccess) return e;
        if (pass_ev) cudaEventRecord(pass_ev[k++], s);
        void* a1[] = {&bb, &tp, &ph, &tr};
        e = cudaLaunchKernel(fn.conv_z, dim3(g[1]), dim3(kColThreads), a1, 0, s);
        if (e != cudaSuccess) return e;
        if (pass_ev) cudaEventRecord(pass_ev[k++], s);
    } else {
        void* a3[] = {&bb, &tr};
        e = cudaLaunchKernel(fn.redist_xy[tier], dim3(g[3]), dim3(nt), a3, 0, s);
        if (e != cudaSuccess) return e;
        if (pass_ev) cudaEventRecord(pass_ev[k++], s);
        void* a4[] = {&bb, &db, &tr};
        e = cudaLaunchKernel(reinterpret_cast<const void*>(p_redist_z), dim3(g[4]), dim3(kColThreads), a4, 0, s);
        if (e != cudaSuccess) return e;
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
