// Pass path of the batched step for 3D boxes: passes over (box, plane),
// (box, slab), (box, column chunk) and domain-tile work items.
//
// Same arithmetic as the box-streaming kernels (Sec. 2.1.4 predictor, Eq. (16)
// comparison, Sec. 2.1.6 taxicab re-initialisation), arranged so that every
// pass is a persistent grid striding over the work items of all boxes at once:
// the many short, independent items keep every SM busy where one CTA per box
// serialised a whole box along z.  The fields between passes go through HBM:
//   k_bin       per box: list it in every domain tile it overlaps; reset its
//               positive bounding box
//   p_conv_xy   (box, plane): bulk copy of the plane of phi in the old layout,
//               staged into the new layout (-eps outside), x and y passes in
//               shared memory                                     -> Z = xy-convolved
//   p_conv_z    (box, columns): z pass from the column in registers, velocity
//               correction (Read-Shockley pairs from a per-box hash of the
//               step's neighbour list), clamp                     -> Y = phi_p
//   p_field     (domain tile): the two largest (phi_p, grain) per cell over
//               the tile's boxes in registers (stored in T as (phi_p, -id)
//               keys only on request, B.keep_field); then
//               phi_c = (phi_p - m) / 2 and the ID-field for every box cell of
//               the tile                                          -> Z = phi_c
//   p_redist_xy (box, slab): plane ring filled by bulk copies; reference cells
//               with their planar-exact distances, y and x taxicab scans -> Y
//   p_redist_z  (box, columns): the column in registers, z taxicab scans,
//               signs, positive bounding box                      -> X = phi
// The field pass replaces the box-streaming kernels' atomic scatter: each
// domain cell's top-2 is built by the one thread that owns the cell, so the
// step has no atomics on the field.  The work-item lists are written by the
// box update; boxes of x, y side <= 32, <= 40, <= 48 and <= 64 (tiers 0-3)
// have their own lists and launches, so the plane passes of smaller boxes run
// with smaller shared-memory grids and higher occupancy; larger boxes (tier 4)
// take plane passes through global memory (p_conv_xy_big, p_redist_xy_big).
// A non-periodic box's planes outside it are -eps; their xy convolution is
// the constant that p_conv_z recomputes with the FMA sequence p_conv_xy would
// use.
#include <cfloat>
#include <climits>

#include "bulk_copy.cuh"
#include "group.cuh"
#include "kernels_common.cuh"

namespace lsgg {

constexpr int kZB = 8;               // planes loaded ahead by the column passes
constexpr int kReachP = kRedistReach;
constexpr int kColThreads = kPassChunk;

__device__ __forceinline__ bool halted(const StepBuffers& B) { return *(volatile int*)&B.st->halt != 0; }

// A launch that cannot run records LSGG_ERR_UNSUPPORTED and halts its
// context, or every member of its group.
template <bool GRP>
__device__ __forceinline__ void refuse_launch(const StepBuffers& B1, const GroupRef& g) {
    if constexpr (GRP) {
        for (int k = 0; k < g.n; ++k) {
            atomicExch(&g.B[k].st->status, LSGG_ERR_UNSUPPORTED);
            atomicExch(&g.B[k].st->halt, 1);
        }
    } else {
        atomicExch(&B1.st->status, LSGG_ERR_UNSUPPORTED);
        atomicExch(&B1.st->halt, 1);
    }
}

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
// A CTA of NT threads takes one (box, plane) item at a time:
//   fetch   the plane of phi in the box's previous layout (contiguous,
//           16-byte aligned) arrives in a raw slot by a bulk copy, issued
//           while the CTA still works on the item before;
//   stage   raw -> padded grid P in the new layout (-eps outside the old
//           box), a thread per group of four cells of a padded row; rows
//           outside the old box are left unstaged;
//   x pass  each thread convolves 4 consecutive cells of one padded row from
//           16-byte shared loads -> grid XC (all padded rows; a row outside
//           the old box is the FMA chain over -eps, written directly);
//   y pass  each thread convolves 4 consecutive rows of one column from
//           shared loads of XC and stores them (lanes along x: coalesced).
// The FMA order of both passes is the one conv_xy_of_const repeats.  Every
// wait on a copy is bounded (LSGG_ERR_TIMEOUT, halt, drain, return).
//
// The sizes below are the one definition of the layout: the kernel's
// offsets and the launch's dynamic shared-memory size both derive from them.
// padded rows; 16-byte loads per x window of 4 outputs; pitch of P (room for
// the last group's window); pitch of XC; rows of XC (3 spare rows)
__host__ __device__ constexpr int conv_pyr(int R, int side) { return side + 2 * R; }
__host__ __device__ constexpr int conv_nq(int R) { return (2 * R + 1 + 6) / 4; }
__host__ __device__ constexpr int conv_px(int R, int side) { return ((side + 3) & ~3) + 4 * conv_nq(R); }
__host__ __device__ constexpr int conv_xp(int side) { return (side + 3) & ~3; }
__host__ __device__ constexpr int conv_xr(int R, int side) { return conv_pyr(R, side) + 3; }
__host__ __device__ constexpr int conv_mx(int R, int side) { return (conv_pyr(R, side) + 3) & ~3; }
__host__ __device__ constexpr size_t conv_layout_bytes(int R, int side) {
    return 128 + sizeof(float) * ((size_t)side * side + (size_t)conv_pyr(R, side) * conv_px(R, side) +
                                  (size_t)conv_xr(R, side) * conv_xp(side)) +
           sizeof(int) * (size_t)(conv_mx(R, side) + conv_pyr(R, side));
}
template <int R, int SIDE>
struct ConvXYLayout {
    static constexpr int PYR = conv_pyr(R, SIDE);
    static constexpr int NQ = conv_nq(R);
    static constexpr int PX = conv_px(R, SIDE);              // room for the last group's window
    static constexpr int XP = conv_xp(SIDE);
    static constexpr int XR = conv_xr(R, SIDE);              // the last 4-row group reads 3 rows past PYR
    static constexpr int MX = conv_mx(R, SIDE);               // x map entries: whole 4-cell staging groups
    static constexpr size_t raw = 128;                        // after the barrier
    static constexpr size_t P = raw + sizeof(float) * SIDE * SIDE;
    static constexpr size_t XC = P + sizeof(float) * PYR * PX;
    static constexpr size_t maps = XC + sizeof(float) * XR * XP;
    static constexpr size_t bytes = maps + sizeof(int) * (MX + PYR);
    static_assert(bytes == conv_layout_bytes(R, SIDE), "one definition of the layout");
};

// Dynamic shared memory of the running launch: the plane kernels refuse to
// run (LSGG_ERR_UNSUPPORTED) rather than index past a launch that got less
// than their layout.
__device__ __forceinline__ unsigned dyn_smem_bytes() {
    unsigned r;
    asm volatile("mov.u32 %0, %%dynamic_smem_size;" : "=r"(r));
    return r;
}

__device__ __forceinline__ float to_f32(float v) { return v; }
__device__ __forceinline__ float to_f32(__nv_bfloat16 v) { return __bfloat162float(v); }

// raw plane (old layout) -> padded grid P (new layout): a thread per group of
// four padded cells of a row (16-byte stores; the map has -1 past the row's
// end, so a group's extra cells take the fill).  Rows outside the old box are
// not staged: the x pass writes their result directly.
template <int NT, int PX, class T>
__device__ __forceinline__ void stage_plane(const T* raw, float* P, const int* mapx, const int* mapy, int PXa, int PYa,
                                            int onx, float fill, int t) {
    const int ngp = (PXa + 3) >> 2;
    const Div16 dg(ngp);
    for (int j = t; j < PYa * ngp; j += NT) {
        const int yp = dg(j), xp0 = 4 * (j - yp * ngp);
        const int my = mapy[yp];
        if (my < 0) continue;
        const T* rrow = raw + my * onx;
        float v[4];
#pragma unroll
        for (int u = 0; u < 4; ++u) {
            const int mx = mapx[xp0 + u];
            v[u] = mx >= 0 ? to_f32(rrow[mx]) : fill;
        }
        *reinterpret_cast<float4*>(P + yp * PX + xp0) = make_float4(v[0], v[1], v[2], v[3]);
    }
}

// The plane of item `item` in the box's previous layout: source address and
// bytes (0 when the new plane lies outside the old box).
__device__ __forceinline__ void conv_source(const StepBuffers& B, int2 it, const float** src, uint32_t* bytes) {
    const Box nb = B.cur[it.x], ob = B.prev[it.x];
    const int ozl = pmod(nb.oz + it.y - ob.oz, B.dom.nz);
    const int ps = plane_stride(ob.nx, ob.ny);
    const long long e = ob.off + (long long)(ozl < ob.nz ? ozl : 0) * ps;
    *src = reinterpret_cast<const float*>(reinterpret_cast<const char*>(B.X) + e * state_bytes(B));
    *bytes = ozl < ob.nz ? (uint32_t)(ps * state_bytes(B)) : 0u;
}

template <int R, int SIDE, int NT, bool GRP>
__global__ void __launch_bounds__(NT)
p_conv_xy(StepBuffers B1, GroupRef grp, Taps taps, int tier) {
    constexpr int W = 2 * R + 1;
    using LY = ConvXYLayout<R, SIDE>;
    extern __shared__ __align__(128) unsigned char smc[];   // ConvXYLayout::bytes
    uint64_t* bar = reinterpret_cast<uint64_t*>(smc);
    float* const raw = reinterpret_cast<float*>(smc + LY::raw);
    float* const P = reinterpret_cast<float*>(smc + LY::P);
    float* const XC = reinterpret_cast<float*>(smc + LY::XC);
    int* const mapx = reinterpret_cast<int*>(smc + LY::maps);
    int* const mapy = mapx + LY::MX;
    __shared__ int s_flag;
    __shared__ int s_gb[GRP ? kMaxGroup + 1 : 1];
    const int t = threadIdx.x;
    if (t == 0) {
        const bool fits = dyn_smem_bytes() >= LY::bytes;
        if (fits) {
            mbar_init(bar, 1);
            fence_mbar_init();
        } else {
            refuse_launch<GRP>(B1, grp);
        }
        s_flag = !fits || (!GRP && halted(B1));
    }
    __syncthreads();
    if (s_flag) return;
    const Domain D1 = B1.dom;
    float g[W];
#pragma unroll
    for (int k = 0; k < W; ++k) g[k] = taps.g[k];
    const int n_items = GRP ? group_scan(grp, kItemSlabs, tier, true, s_gb) : B1.st->n_slabs[tier];
    const int2* items = GRP ? nullptr : B1.slab_items + B1.st->slab_base[tier];
    uint32_t phase = 0;
    bool pending = false;
    // bulk copy of plane z of box it.x in its previous layout into raw (none
    // when the plane lies outside the old box)
    auto fetch = [&](const StepBuffers& Bx, int2 itx, int z) {
        const float* src;
        uint32_t bytes;
        conv_source(Bx, make_int2(itx.x, z), &src, &bytes);
        if (bytes) {
            if (t == 0) {
                fence_async_smem();                     // earlier generic accesses to raw come first
                mbar_expect(bar, bytes);
                bulk_load(raw, src, bytes, bar);
            }
            pending = true;
        }
    };
    if (blockIdx.x < n_items) {                         // the first item's first plane
        int lf;
        const StepBuffers& Bf = member<GRP>(B1, grp, s_gb, blockIdx.x, lf);
        const int2 itf = list_item<GRP>(Bf, items, kItemSlabs, tier, blockIdx.x, lf);
        fetch(Bf, itf, itf.y);
    }
    for (int item = blockIdx.x; item < n_items; item += gridDim.x) {
        int local;
        const StepBuffers& B = member<GRP>(B1, grp, s_gb, item, local);
        const Domain D = GRP ? B.dom : D1;
        const int2 it = list_item<GRP>(B, items, kItemSlabs, tier, item, local);
        const int b = it.x, z0 = it.y;
        const Box nb = B.cur[b], ob = B.prev[b];
        const int nx = nb.nx, ny = nb.ny;
        const bool fx = nx == D.nx, fy = ny == D.ny;
        const int PXa = nx + 2 * R, PYa = ny + 2 * R;
        const int z1 = min(z0 + B.slab, nb.nz);
        if (max(max(nx, ny), max(ob.nx, ob.ny)) > SIDE) {    // not this tier's box: refuse, never overrun
            if (t == 0) { atomicExch(&B.st->status, LSGG_ERR_UNSUPPORTED); atomicExch(&B.st->halt, 1); }
            if (pending) { if (t == 0) mbar_wait(bar, phase); }
            return;
        }
        // the new-to-old layout maps of the item's box (the same for all its planes)
        for (int i = t; i < LY::MX + PYa; i += NT) {
            const bool isx = i < LY::MX;
            const int ip = isx ? i : i - LY::MX;
            const int n = isx ? nx : ny, N = isx ? D.nx : D.ny;
            const int o_new = isx ? nb.ox : nb.oy, o_old = isx ? ob.ox : ob.oy, n_old = isx ? ob.nx : ob.ny;
            const bool full = isx ? fx : fy;
            int l = ip - R, v = -1;
            if ((!isx || ip < PXa) && (full || (l >= 0 && l < n))) {
                if (full) l = wrap_near(l, n);
                const int ol = wrap_near(o_new + l - o_old, N);
                v = ol < n_old ? ol : -1;
            }
            if (isx) mapx[ip] = v; else mapy[ip] = v;
        }
        __syncthreads();                                    // the maps are published
        for (int z = z0; z < z1; ++z) {
            const bool have = pending;
            bool ok = true;
            if (pending) {
                ok = mbar_wait(bar, phase, B.wait_limit);
                if (ok) phase ^= 1u;
            }
            if (!__syncthreads_and(ok)) {
                if (t == 0) {
                    atomicExch(&B.st->status, LSGG_ERR_TIMEOUT);
                    atomicExch(&B.st->halt, 1);
                    mbar_wait(bar, phase);
                }
                __syncthreads();
                return;
            }
            pending = false;
            // stage: raw (old layout, FP32 or BF16) -> P (new layout), warp per padded row
            if (have) {
                if (B.bf16) stage_plane<NT, LY::PX>(reinterpret_cast<const __nv_bfloat16*>(raw), P, mapx, mapy, PXa, PYa,
                                                    ob.nx, -D.eps, t);
                else stage_plane<NT, LY::PX>(raw, P, mapx, mapy, PXa, PYa, ob.nx, -D.eps, t);
            }
            __syncthreads();                                // raw is free: fetch the next plane
            if (z + 1 < z1) {
                fetch(B, it, z + 1);
            } else if (item + (int)gridDim.x < n_items) {
                const int nxt = item + gridDim.x;
                int ln;
                const StepBuffers& Bn = member<GRP>(B1, grp, s_gb, nxt, ln);
                const int2 itn = list_item<GRP>(Bn, items, kItemSlabs, tier, nxt, ln);
                fetch(Bn, itn, itn.y);
            }
            // x pass: (padded row, group of 4 outputs)
            const int ngx = (nx + 3) >> 2;
            {
                const Div16 dgx(ngx);
                float cfill = 0.0f;
    #pragma unroll
                for (int k = 0; k < W; ++k) cfill = fmaf(g[k], -D.eps, cfill);
                for (int j = t; j < PYa * ngx; j += NT) {
                    const int yp = dgx(j), x0 = 4 * (j - yp * ngx);
                    if (!have || mapy[yp] < 0) {                // a fill row: the chain over -eps, unstaged
                        *reinterpret_cast<float4*>(XC + yp * LY::XP + x0) = make_float4(cfill, cfill, cfill, cfill);
                        continue;
                    }
                    const float4* r4 = reinterpret_cast<const float4*>(P + yp * LY::PX + x0);
                    float v[4 * LY::NQ];
    #pragma unroll
                    for (int q = 0; q < LY::NQ; ++q) {
                        const float4 a = r4[q];
                        v[4 * q] = a.x; v[4 * q + 1] = a.y; v[4 * q + 2] = a.z; v[4 * q + 3] = a.w;
                    }
                    float o[4];
    #pragma unroll
                    for (int u = 0; u < 4; ++u) {
                        float acc = 0.0f;
    #pragma unroll
                        for (int k = 0; k < W; ++k) acc = fmaf(g[k], v[u + k], acc);
                        o[u] = acc;
                    }
                    *reinterpret_cast<float4*>(XC + yp * LY::XP + x0) = make_float4(o[0], o[1], o[2], o[3]);
                }
            }
            __syncthreads();
            // y pass: (group of 4 rows, column), lanes along x
            {
                float* dst = B.Z + nb.off + (long long)z * plane_stride(nx, ny);
                const int ngy = (ny + 3) >> 2;
                const Div16 dnx(nx);
                for (int j = t; j < ngy * nx; j += NT) {
                    const int gy = dnx(j), x = j - gy * nx, y0 = 4 * gy;
                    const float* col = XC + y0 * LY::XP + x;
                    float v[W + 3];
    #pragma unroll
                    for (int k = 0; k < W + 3; ++k) v[k] = col[k * LY::XP];
    #pragma unroll
                    for (int u = 0; u < 4; ++u) {
                        float acc = 0.0f;
    #pragma unroll
                        for (int k = 0; k < W; ++k) acc = fmaf(g[k], v[u + k], acc);
                        if (y0 + u < ny) dst[(y0 + u) * nx + x] = acc;
                    }
                }
            }
            __syncthreads();                                // XC is free
        }
    }
}

// ---------------------------------------------------------------------------
// pass 2: z convolution per column, velocity correction, clamp
// ---------------------------------------------------------------------------
// z pass of one column of nz <= NZ cells on a non-periodic axis, ideal
// growth: the column in registers (unconditional loads: cells past the column
// re-read its last cell, so all of them are in flight at once), planes
// outside the box are the constant xy convolution of -eps.
template <int R, int NZ>
__device__ __forceinline__ void conv_column(const float* zc, float* yc, int nz, int ps, const float (&g)[2 * R + 1],
                                            float cconst, float eps) {
    constexpr int W = 2 * R + 1;
    float r[NZ + 2 * R];
#pragma unroll
    for (int k = 0; k < R; ++k) r[k] = cconst;
#pragma unroll
    for (int z = 0; z < NZ; ++z) r[R + z] = __ldg(zc + (long long)min(z, nz - 1) * ps);
#pragma unroll
    for (int z = 0; z < NZ + R; ++z)
        if (z >= nz) r[R + z] = cconst;
#pragma unroll
    for (int z = 0; z < NZ; ++z)
        if (z < nz) {
            float acc = 0.0f;
#pragma unroll
            for (int k = 0; k < W; ++k) acc = fmaf(g[k], r[z + k], acc);
            yc[(long long)z * ps] = fminf(fmaxf(acc, -eps), eps);
        }
}

// The z pass's per-box pair hash (Read-Shockley): the box's pool list (every
// grain of its ID-field with w and M) in kZHash open-addressing slots, at
// most half full, so a cell finds its pair's weights with one or two shared
// loads.
constexpr int kZHash = 2 * kPoolKeys;
static_assert((kZHash & (kZHash - 1)) == 0, "pair hash slots: a power of two");
__device__ __forceinline__ unsigned zhash(int j) { return ((unsigned)j * 2654435761u) >> 22; }
static_assert((1u << 10) == kZHash, "zhash yields the slot bits of kZHash");
__device__ __forceinline__ int zslot(const int* hk, int j) {
    unsigned h = zhash(j);
#pragma unroll 1
    for (int p = 0; p < kZHash; ++p) {
        const int k = hk[h];
        if (k == j) return (int)h;
        if (k < 0) return -1;
        h = (h + 1) & (kZHash - 1);
    }
    return -1;
}

constexpr int kColumnRadius = 5;   // the physics z pass keeps its column in registers at this radius

// Read-Shockley weights of a pair missing from the box's hash (a list that
// did not fit the pool): out of line, so that the unrolled column below
// keeps one call per cell instead of the FP64 evaluation.
__device__ __noinline__ void rs_pair_out_of_line(const PhysicsDev& phys, int i, int j, float& w, float& m) {
    rs_pair(phys, i, j, w, m);
}

// z pass with the velocity correction of Eq. (10) for one column of nz <= NZ
// cells on a non-periodic axis: the z convolution from the column in
// registers (as conv_column), then per group of eight cells the previous
// step's phi and pair ids (old layout; -eps and no pair outside the old box)
// loaded together, the bulk energies e_j loaded together, and the blend
// phi + w (c - phi) + M (e_j - e_i) dt with w and M from the box's pair hash
// (Read-Shockley) or 1 (magnetic); cells without a pair take c.
template <int R, int NZ>
__device__ __forceinline__ void conv_column_phys(const StepBuffers& B, const PhysicsDev& phys, const float* zc, float* yc,
                                                 int nz, int ps, const float (&g)[2 * R + 1], float cconst, float eps,
                                                 long long o_old, int ps_old, int ozl0, int onz, int dnz, bool in_old,
                                                 int b, float ei, bool rs, const int* hk, const float* hw,
                                                 const float* hm) {
    constexpr int W = 2 * R + 1;
    constexpr int G8 = 8;
    float r[NZ + 2 * R];
#pragma unroll
    for (int k = 0; k < R; ++k) r[k] = cconst;
#pragma unroll
    for (int z = 0; z < NZ; ++z) r[R + z] = __ldg(zc + (long long)min(z, nz - 1) * ps);
#pragma unroll
    for (int z = 0; z < NZ + R; ++z)
        if (z >= nz) r[R + z] = cconst;
#pragma unroll
    for (int z0 = 0; z0 < NZ; z0 += G8) {
        if (z0 >= nz) break;                               // uniform: one box per CTA item
        float p0[G8], ej[G8];
        int jj[G8];
#pragma unroll
        for (int u = 0; u < G8; ++u) {
            const int z = z0 + u;
            int ozl = ozl0 + z;                            // ozl0 + z < 2 N_z
            if (ozl >= dnz) ozl -= dnz;
            const bool ok = z < nz && in_old && ozl < onz;
            const long long o = o_old + (long long)(ok ? ozl : 0) * ps_old;
            p0[u] = ok ? ld_state(B, o) : -eps;
            jj[u] = ok ? B.IDF[o] : -1;
        }
#pragma unroll
        for (int u = 0; u < G8; ++u) ej[u] = phys.energy && jj[u] >= 0 ? __ldg(phys.energy + jj[u]) : 0.0f;
#pragma unroll
        for (int u = 0; u < G8; ++u) {
            const int z = z0 + u;
            if (z >= nz) break;
            float acc = 0.0f;
#pragma unroll
            for (int k = 0; k < W; ++k) acc = fmaf(g[k], r[z + k], acc);
            float val = acc;
            const int j = jj[u];
            if (j >= 0) {
                float w = 1.0f, m = 1.0f;
                if (rs) {
                    const int h = zslot(hk, j);
                    if (h >= 0) {
                        w = hw[h];
                        m = hm[h];
                    } else {
                        rs_pair_out_of_line(phys, b, j, w, m);
                    }
                }
                float bulk = 0.0f;
                if (phys.energy) bulk = m * (ej[u] - ei) * phys.dt;
                val = p0[u] + w * (acc - p0[u]) + bulk;
            }
            yc[(long long)z * ps] = fminf(fmaxf(val, -eps), eps);
        }
    }
}

template <int R, bool PHYS, bool GRP>
__global__ void __launch_bounds__(kColThreads, PHYS ? 2 : (R < 5 ? 4 : 3))
p_conv_z(StepBuffers B1, GroupRef grp, Taps taps, PhysicsDev phys, int tier) {
    static_assert(!(GRP && PHYS), "step groups run ideal growth");
    constexpr int W = 2 * R + 1;
    __shared__ int s_tj[PHYS ? kNbCap : 1];
    __shared__ float s_tw[PHYS ? kNbCap : 1], s_tm[PHYS ? kNbCap : 1];
    __shared__ int s_hk[PHYS ? kZHash : 1];
    __shared__ float s_hw[PHYS ? kZHash : 1], s_hm[PHYS ? kZHash : 1];
    __shared__ int s_gb[GRP ? kMaxGroup + 1 : 1];
    if (!GRP && halted(B1)) return;
    float g[W];
#pragma unroll
    for (int k = 0; k < W; ++k) g[k] = taps.g[k];
    const float cconst1 = GRP ? 0.0f : conv_xy_of_const<R>(g, -B1.dom.eps);
    const int n_items = GRP ? group_scan(grp, kItemChunks, tier, true, s_gb) : B1.st->n_chunks[tier];
    const int2* items = GRP ? nullptr : B1.chunk_items + B1.st->chunk_base[tier];
    const bool rs = PHYS && phys.kind == LSGG_PHYSICS_READ_SHOCKLEY;
    const bool pooled = PHYS && phys.pool_ent[0] != nullptr && phys.pair_map == nullptr;
    // this step's pool (the parity of the steps done)
    const bool odd = pooled && (B1.st->steps_done & 1);
    const int2* pool_box = PHYS ? (odd ? phys.pool_box[1] : phys.pool_box[0]) : nullptr;
    const int4* pool_ent = PHYS ? (odd ? phys.pool_ent[1] : phys.pool_ent[0]) : nullptr;
    int last_b = -1;
    int hash_n = -1;                                       // the box's pair hash entries, -1: none
    PairTable tab{s_tj, s_tw, s_tm, 0};
    for (int item = blockIdx.x; item < n_items; item += gridDim.x) {
        int local;
        const StepBuffers& B = member<GRP>(B1, grp, s_gb, item, local);
        const Domain D = B.dom;
        const float cconst = GRP ? conv_xy_of_const<R>(g, -D.eps) : cconst1;
        const int2 it = list_item<GRP>(B, items, kItemChunks, tier, item, local);
        const int b = it.x;
        if (PHYS && (rs || pooled) && b != last_b) {       // uniform across the CTA
            __syncthreads();
            hash_n = -1;
            tab.n = 0;
            if (pooled) {
                const int2 pb = pool_box[b];
                if (pb.y >= 0 && pb.y <= kZHash / 2) hash_n = pb.y;
            }
            if (hash_n >= 0) {
                for (int k = threadIdx.x; k < kZHash; k += blockDim.x) s_hk[k] = -1;
                __syncthreads();
                const int2 pb = pool_box[b];
                for (int k = threadIdx.x; k < hash_n; k += blockDim.x) {
                    const int4 e = pool_ent[pb.x + k];
                    unsigned h = zhash(e.x);
                    while (atomicCAS(&s_hk[h], -1, e.x) != -1) h = (h + 1) & (kZHash - 1);
                    s_hw[h] = __int_as_float(e.y);
                    s_hm[h] = __int_as_float(e.z);
                }
            } else if (rs) {
                tab = load_pair_table(phys, b, s_tj, s_tw, s_tm);
            }
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
            oxl = wrap_near(nb.ox + x - ob.ox, D.nx);
            oyl = wrap_near(nb.oy + y - ob.oy, D.ny);
            in_old_xy = oxl < ob.nx && oyl < ob.ny;
        }
        if (!PHYS && !fz && nz <= 64) {                    // uniform across the CTA (one box per item)
            if (nz <= 16) conv_column<R, 16>(zc, yc, nz, ps, g, cconst, D.eps);
            else if (nz <= 32) conv_column<R, 32>(zc, yc, nz, ps, g, cconst, D.eps);
            else if (nz <= 48) conv_column<R, 48>(zc, yc, nz, ps, g, cconst, D.eps);
            else conv_column<R, 64>(zc, yc, nz, ps, g, cconst, D.eps);
            continue;
        }
        const int ps_old = plane_stride(ob.nx, ob.ny);
        // the paper's radius (the column code is instantiated for it alone)
        if constexpr (PHYS && R == kColumnRadius) {
            if (!fz && nz <= 64 && !phys.pair_map && (!rs || hash_n >= 0)) {
                // uniform across the CTA
                const long long o_old = ob.off + (long long)oyl * ob.nx + oxl;
                const int ozl0 = wrap_near(nb.oz - ob.oz, D.nz);
                const float ei = phys.energy ? phys.energy[b] : 0.0f;
                if (nz <= 16)
                    conv_column_phys<R, 16>(B, phys, zc, yc, nz, ps, g, cconst, D.eps, o_old, ps_old, ozl0, ob.nz, D.nz,
                                            in_old_xy, b, ei, rs, s_hk, s_hw, s_hm);
                else if (nz <= 32)
                    conv_column_phys<R, 32>(B, phys, zc, yc, nz, ps, g, cconst, D.eps, o_old, ps_old, ozl0, ob.nz, D.nz,
                                            in_old_xy, b, ei, rs, s_hk, s_hw, s_hm);
                else if (nz <= 48)
                    conv_column_phys<R, 48>(B, phys, zc, yc, nz, ps, g, cconst, D.eps, o_old, ps_old, ozl0, ob.nz, D.nz,
                                            in_old_xy, b, ei, rs, s_hk, s_hw, s_hm);
                else
                    conv_column_phys<R, 64>(B, phys, zc, yc, nz, ps, g, cconst, D.eps, o_old, ps_old, ozl0, ob.nz, D.nz,
                                            in_old_xy, b, ei, rs, s_hk, s_hw, s_hm);
                continue;
            }
        }
        PairCache pcache;
        const float ei = PHYS && phys.energy ? phys.energy[b] : 0.0f;
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
            // the previous step's phi and ID-field of this batch's output planes
            float phi0[PHYS ? kZB : 1];
            int jn[PHYS ? kZB : 1];
            if (PHYS) {
#pragma unroll
                for (int u = 0; u < kZB; ++u) {
                    const int zo = base + u - 2 * R;
                    const int ozl = wrap_near(nb.oz + zo - ob.oz, D.nz);
                    phi0[u] = -D.eps;
                    jn[u] = -1;
                    if (zo >= 0 && zo < nz && in_old_xy && ozl < ob.nz) {
                        const long long o = ob.off + (long long)ozl * ps_old + (long long)oyl * ob.nx + oxl;
                        phi0[u] = ld_state(B, o);
                        jn[u] = B.IDF[o];
                    }
                    if (phys.pair_map && zo >= 0 && zo < nz) jn[u] = phys.pair_map[nb.off + (long long)zo * ps + c];
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
                if (PHYS && hash_n >= 0) {
                    // Eq. (10) with the pair's w and M from the box's hash
                    // (the arithmetic of pair_blend)
                    const int j = jn[u];
                    if (j >= 0) {
                        const int h = zslot(s_hk, j);
                        float w = 1.0f, m = 1.0f;
                        if (h >= 0) {
                            w = s_hw[h];
                            m = s_hm[h];
                        } else if (rs) {                       // not in the box's list: direct
                            rs_pair_out_of_line(phys, b, j, w, m);
                        }
                        const float ej = phys.energy ? phys.energy[j] : 0.0f;
                        float bulk = 0.0f;
                        if (phys.energy) bulk = m * (ej - ei) * phys.dt;
                        val = phi0[u] + w * (acc - phi0[u]) + bulk;
                    }
                } else if (PHYS) {
                    val = pair_blend_cached(phys, tab, b, jn[u], phi0[u], acc, ei, pcache);
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

template <bool GRP>
__global__ void __launch_bounds__(256)
k_bin(StepBuffers B1, GroupRef grp) {
    __shared__ int s_gb[GRP ? kMaxGroup + 1 : 1];
    if (!GRP && halted(B1)) return;
    const int n_all = GRP ? group_scan(grp, kItemBoxes, 0, true, s_gb) : B1.n_boxes;
    const int lane = threadIdx.x & 31;
    const int warps = (blockDim.x >> 5) * gridDim.x;
    for (int gb = (blockIdx.x * blockDim.x + threadIdx.x) >> 5; gb < n_all; gb += warps) {
        int b;
        const StepBuffers& B = member<GRP>(B1, grp, s_gb, gb, b);
        const Domain D = B.dom;
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

// The tile counters of every live member cleared (the group's counterpart of
// the single context's memset before k_bin).
__global__ void __launch_bounds__(256)
k_clear_tiles_group(GroupRef grp) {
    __shared__ int s_gb[kMaxGroup + 1];
    const int n_all = group_scan(grp, kItemTiles, 0, true, s_gb);
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n_all; i += gridDim.x * blockDim.x) {
        int local;
        const StepBuffers& B = member<true>(grp.B[0], grp, s_gb, i, local);
        B.tile_cnt[local] = 0;
    }
}

// ---------------------------------------------------------------------------
// field pass: top-2 per domain cell, then the comparison step (Eq. (16))
// ---------------------------------------------------------------------------
// Thread (x, y) of a tile owns the column of kTileZ cells at (x, y); for each
// box covering the column it loads the box's phi_p there and keeps the two
// largest (phi_p, grain) pairs per cell in registers, ordered by phi_p and,
// at equal phi_p, by the smaller grain id first -- the order of the
// box-streaming kernels' 64-bit keys (phi_p, -id) under atomicMax, so m and
// the ID-field are identical.  Per listed box the CTA first stages, in shared
// memory, how the tile maps into the box: on an axis where the box's cells
// in the tile keep one box-local offset (all but boxes spanning nearly the
// whole domain), the mask of the tile's rows / columns / planes it covers
// and one arena offset for the tile's corner, so that the per-thread work is
// a mask test per column and an add per cell; other boxes take the general
// cyclic path.
struct TileBox {
    long long off;            // affine: arena offset of tile cell (0, 0, 0); general: of the box
    int nx, ny;               // box x, y sides
    int ps;                   // plane stride
    int id;                   // grain id
    unsigned xmask, ymask;    // affine: bit lx / ly: column / row of the tile lies in the box
    unsigned zm;              // bits 0-7: planes (both paths), bit 31: affine
    int dx, dy, dz;           // general: box-local coordinates of the tile corner (cyclic)
};

// One axis of the tile -> box map: tile cells l in [0, T) with box-local
// coordinate l + sh, covered where 0 <= l + sh < n.  False when the box's
// cells in the tile do not share one offset (the uncovered gap of a box
// spanning nearly the whole axis lies inside the tile).
__device__ __forceinline__ bool tile_axis(int t0, int T, int N, int o, int n, int& sh, unsigned& mask) {
    int d = t0 - o;
    if (d < 0) d += N;
    if (d < n && N - d < T) return false;
    sh = d < n ? d : d - N;
    const int lo = max(0, -sh), hi = min(T, n - sh);
    const int w = hi - lo;
    mask = w <= 0 ? 0u : (w >= 32 ? 0xffffffffu : (1u << w) - 1u) << lo;
    return true;
}

__device__ __forceinline__ void stage_tile_box(const StepBuffers& B, int b, int tx0, int ty0, int z0, int ntx, int nty,
                                               int nzt, TileBox& t) {
    const Domain& D = B.dom;
    const Box bx = B.cur[b];
    t.nx = bx.nx;
    t.ny = bx.ny;
    t.id = b;
    t.ps = plane_stride(bx.nx, bx.ny);
    t.dx = wrap_near(tx0 - bx.ox, D.nx);
    t.dy = wrap_near(ty0 - bx.oy, D.ny);
    t.dz = wrap_near(z0 - bx.oz, D.nz);
    int sx, sy, sz;
    unsigned mx, my, mz;
    if (bx.nx <= 0) {
        t.off = 0;
        t.xmask = t.ymask = 0;
        t.zm = 1u << 31;                    // affine and empty
        return;
    }
    if (tile_axis(tx0, ntx, D.nx, bx.ox, bx.nx, sx, mx) && tile_axis(ty0, nty, D.ny, bx.oy, bx.ny, sy, my) &&
        tile_axis(z0, nzt, D.nz, bx.oz, bx.nz, sz, mz)) {
        t.off = bx.off + (long long)sz * t.ps + (long long)sy * bx.nx + sx;
        t.xmask = mx;
        t.ymask = my;
        t.zm = (1u << 31) | mz;
        return;
    }
    unsigned m = 0;
    for (int zz = 0; zz < nzt; ++zz) {
        int lz = t.dz + zz;
        if (lz >= D.nz) lz -= D.nz;
        if (lz < bx.nz) m |= 1u << zz;
    }
    t.off = bx.off;
    t.xmask = t.ymask = 0;
    t.zm = m;
}

// (v, id) enters the top two (v1, i1) >= (v2, i2) of a cell; absent entries
// are (-inf, -1), and v = -inf never enters.
__device__ __forceinline__ void top2_insert(float v, int id, float& v1, int& i1, float& v2, int& i2) {
    const bool c1 = v > v1 || (v == v1 && id < i1);
    const bool c2 = v > v2 || (v == v2 && id < i2);
    v2 = c1 ? v1 : (c2 ? v : v2);
    i2 = c1 ? i1 : (c2 ? id : i2);
    v1 = c1 ? v : v1;
    i1 = c1 ? id : i1;
}

// Four CTAs per SM for the plain field; the ID-field and debug variants keep
// the registers of three.
template <bool IDF, bool DBG, bool GRP>
__global__ void __launch_bounds__(kTileX * kTileY, (IDF || DBG || GRP) ? 3 : 4)
p_field(StepBuffers B1, GroupRef grp, PhysicsDev phys, DebugOut dbg) {
    static_assert(!(GRP && (IDF || DBG)), "step groups run ideal growth without intermediates");
    __shared__ TileBox s_tb[kTileCap];
    __shared__ int s_gb[GRP ? kMaxGroup + 1 : 1];
    if (!GRP && halted(B1)) return;
    const int n_all = GRP ? group_scan(grp, kItemTiles, 0, true, s_gb) : B1.n_tiles;
    const int lx = threadIdx.x % kTileX, ly = threadIdx.x / kTileX;
    for (int gtile = blockIdx.x; gtile < n_all; gtile += gridDim.x) {
        int tile;
        const StepBuffers& B = member<GRP>(B1, grp, s_gb, gtile, tile);
        const Domain D = B.dom;
        const float eps = D.eps;
        const int ntx = B.ntile[0], nty = B.ntile[1];
        const int tx = tile % ntx, tyz = tile / ntx, ty = tyz % nty, tz = tyz / nty;
        const int tx0 = tx * kTileX, ty0 = ty * kTileY, z0 = tz * kTileZ;
        const int x = tx0 + lx, y = ty0 + ly;
        const bool col = x < D.nx && y < D.ny;
        const int ext_x = min(kTileX, D.nx - tx0), ext_y = min(kTileY, D.ny - ty0);
        const int nzt = min(kTileZ, D.nz - z0);
        const int cnt = B.tile_cnt[tile];
        const bool all = cnt > kTileCap;            // list overflowed: test every box in batches
        const int n_total = all ? B.n_boxes : cnt;
        float v1[kTileZ], v2[kTileZ], w1[kTileZ], w2[kTileZ];
        int i1[kTileZ], i2[kTileZ];
#pragma unroll
        for (int zz = 0; zz < kTileZ; ++zz) { v1[zz] = v2[zz] = -INFINITY; i1[zz] = i2[zz] = -1; }
        // two sweeps over the tile's boxes: 0 builds the top two, 1 writes phi_c
#pragma unroll
        for (int sweep = 0; sweep < 2; ++sweep) {
            if (sweep == 1) {
                ulonglong2* T2 = reinterpret_cast<ulonglong2*>(B.T);
                const bool keep = B.keep_field != 0;
#pragma unroll
                for (int zz = 0; zz < kTileZ; ++zz) {
                    if (keep && col && zz < nzt)
                        T2[((long long)(z0 + zz) * D.ny + y) * D.nx + x] =
                            make_ulonglong2(i1[zz] >= 0 ? make_key(v1[zz], i1[zz]) : 0ull,
                                            i2[zz] >= 0 ? make_key(v2[zz], i2[zz]) : 0ull);
                    w1[zz] = i1[zz] >= 0 ? v1[zz] + 0.0f : -eps;
                    w2[zz] = i2[zz] >= 0 ? v2[zz] + 0.0f : -eps;
                }
            }
            for (int base = 0; base < n_total; base += kTileCap) {
                const int nb = min(kTileCap, n_total - base);
                // one batch (the tile's whole list): the first sweep's staging serves both
                if (sweep == 0 || n_total > kTileCap) {
                    __syncthreads();                // previous batch done with s_tb
                    for (int k = threadIdx.x; k < nb; k += blockDim.x) {
                        const int b = all ? base + k : B.tile_list[(long long)tile * kTileCap + k];
                        stage_tile_box(B, b, tx0, ty0, z0, ext_x, ext_y, nzt, s_tb[k]);
                    }
                    __syncthreads();
                }
                if (!col) continue;
                for (int k = 0; k < nb; ++k) {
                    const TileBox& t = s_tb[k];
                    const unsigned zaff = t.zm;
                    const unsigned zm = zaff & 0xffu;
                    const int id = t.id, ps = t.ps;
                    long long o[kTileZ];                // arena offsets of the column's cells
                    if (zaff >> 31) {                   // affine (uniform across the CTA)
                        if (!((t.xmask >> lx) & (t.ymask >> ly) & 1u)) continue;
                        const long long oc = t.off + (long long)(ly * t.nx + lx);
#pragma unroll
                        for (int zz = 0; zz < kTileZ; ++zz) o[zz] = oc + (long long)zz * ps;
                    } else {
                        if (!zm) continue;
                        int bxl = t.dx + lx, byl = t.dy + ly;
                        if (bxl >= D.nx) bxl -= D.nx;
                        if (byl >= D.ny) byl -= D.ny;
                        if (bxl >= t.nx || byl >= t.ny) continue;
                        const long long oc = t.off + (long long)byl * t.nx + bxl;
#pragma unroll
                        for (int zz = 0; zz < kTileZ; ++zz) {
                            int lz = t.dz + zz;
                            if (lz >= D.nz) lz -= D.nz;
                            o[zz] = oc + (long long)lz * ps;
                        }
                    }
                    float v[kTileZ];
                    if (zm == 0xffu) {                  // the whole column (uniform)
#pragma unroll
                        for (int zz = 0; zz < kTileZ; ++zz) v[zz] = B.Y[o[zz]];
                    } else {
#pragma unroll
                        for (int zz = 0; zz < kTileZ; ++zz) v[zz] = (zm >> zz) & 1u ? B.Y[o[zz]] : -INFINITY;
                    }
                    if (sweep == 0) {
#pragma unroll
                        for (int zz = 0; zz < kTileZ; ++zz) top2_insert(v[zz], id, v1[zz], i1[zz], v2[zz], i2[zz]);
                    } else {
#pragma unroll
                        for (int zz = 0; zz < kTileZ; ++zz) {
                            if (!((zm >> zz) & 1u)) continue;
                            const bool top = i1[zz] == id;
                            const float m = top ? w2[zz] : w1[zz];
                            const float pc = 0.5f * (v[zz] - m);
                            B.Z[o[zz]] = pc;
                            if (IDF || DBG) {
                                int mid = top ? i2[zz] : i1[zz];
                                if (!(m > -eps)) mid = -1;
                                if (IDF) B.IDF[o[zz]] = mid;
                                if (DBG) {
                                    dbg.m[o[zz]] = m;
                                    dbg.idm[o[zz]] = mid;
                                    dbg.phic[o[zz]] = pc;
                                    dbg.phip[o[zz]] = v[zz];
                                }
                            }
                        }
                    }
                }
            }
        }
    }
}

// ---------------------------------------------------------------------------
// pass 4: classification + y / x taxicab passes of one plane
// ---------------------------------------------------------------------------
// After classification every cell holds eps or, at a reference cell, its
// planar-exact distance, which is at most 1.  A sign change along a line
// lies between two reference cells, and a value carried across it (at least
// 1 after the crossing) never undercuts the reference value on the far side:
// restricting the taxicab propagation to same-sign neighbours changes
// nothing.  The fixed point of Sec. 2.1.6 is therefore the plain taxicab
// distance transform of the magnitudes with each cell's own sign put back.
// That transform is separable -- a forward and a backward scan
// f_j = min(m_j, f_{j-1} + 1) along x, y and z, in any order -- and a scan of
// the whole line equals the 6-step window because no magnitude exceeds
// eps = 7.

// Forward and backward min-plus scan of N registers.  Entries past the end
// of the line start at eps (not below any magnitude): they only ever carry a
// line value plus a distance, which never undercuts the line's own values.
template <int N>
__device__ __forceinline__ void scan_regs(float (&r)[N]) {
#pragma unroll
    for (int j = 1; j < N; ++j) r[j] = fminf(r[j], r[j - 1] + 1.0f);
#pragma unroll
    for (int j = N - 2; j >= 0; --j) r[j] = fminf(r[j], r[j + 1] + 1.0f);
}

// The scan of n <= N magnitudes in shared memory (stride st) through registers.
template <int N>
__device__ __forceinline__ void scan_line_regs(float* L, int n, int st, float pad) {
    float r[N];
#pragma unroll
    for (int j = 0; j < N; ++j) r[j] = j < n ? L[j * st] : pad;
    scan_regs(r);
#pragma unroll
    for (int j = 0; j < N; ++j)
        if (j < n) L[j * st] = r[j];
}

// The scan of a periodic line of n magnitudes in shared memory: twice around
// in each direction.
__device__ __forceinline__ void scan_line_wrap(float* L, int n, int st) {
    float f = L[0];
    for (int j = 1; j < 2 * n; ++j) {
        const int i = j < n ? j : j - n;
        f = fminf(L[i * st], f + 1.0f);
        L[i * st] = f;
    }
    for (int j = 2 * n - 2; j >= 0; --j) {
        const int i = j < n ? j : j - n;
        f = fminf(L[i * st], f + 1.0f);
        L[i * st] = f;
    }
}

// Segmented min-plus scan of a line held in registers by the LANES
// consecutive lanes that share it: lane `seg` holds cells [seg * L, seg * L +
// L) and scans them forward and backward; between the two directions it
// takes the boundary value of its neighbour segment (forward: the previous
// segment's last cell, backward: the next segment's first) and lowers its
// first / last cells by it.  With L > 6 a segment's boundary cells do not
// depend on the carry coming into it, so one exchange per direction suffices.
// Cells past the line's end hold eps.  All lanes of the warp must call.
template <int L, int LANES>
__device__ __forceinline__ void scan_seg_regs(float (&r)[L], int seg, float eps) {
    static_assert(L > kRedistReach, "one exchange per direction needs segments longer than the reach");
    static_assert(LANES > 1 && 32 % LANES == 0, "a group of lanes lies within one warp");
#pragma unroll
    for (int j = 1; j < L; ++j) r[j] = fminf(r[j], r[j - 1] + 1.0f);
    float cf = __shfl_up_sync(0xffffffffu, r[L - 1], 1);
    if (seg == 0) cf = eps;
#pragma unroll
    for (int j = 0; j < kRedistReach; ++j) r[j] = fminf(r[j], cf + (float)(j + 1));
#pragma unroll
    for (int j = L - 2; j >= 0; --j) r[j] = fminf(r[j], r[j + 1] + 1.0f);
    float cb = __shfl_down_sync(0xffffffffu, r[0], 1);
    if (seg == LANES - 1) cb = eps;
#pragma unroll
    for (int j = 0; j < kRedistReach; ++j) r[L - 1 - j] = fminf(r[L - 1 - j], cb + (float)(j + 1));
}

// Plane pass of the re-initialisation: a CTA of NT = 4 * SIDE threads takes
// one (box, slab of kSlab planes) item at a time and walks its planes in z
// order.  Planes of phi_c stream into a 3-slot shared-memory ring by bulk
// copies (a box plane is contiguous and 16-byte aligned), plane z + 2 being
// fetched while plane z is processed.  Thread (r, s) owns cells [s L, s L +
// L) of row r (L = SIDE / 4) and, for every plane entering the ring, records
// their signs (phi > 0) as an L-bit word W.  A cell is a reference cell when
// a face neighbour's sign differs (outside the box the neighbour is -eps,
// negative): shifts and XORs of the words of its row, of the rows above and
// below and of the same row in planes z - 1 and z + 1 find the reference
// cells of a segment at once, and only those load their neighbours' values
// for the planar-exact distance; every other cell starts at eps.  The x scan
// runs in the owner's registers (one carry exchange between the four lanes
// of a row) and goes to the grid G; thread (c, s) then scans rows [s L, s L +
// L) of column c the same way and stores plane z with the signs of phi_c put
// back.  A full periodic axis takes a serial scan twice around the line by
// one lane.  Every wait on a copy is bounded: on expiry the CTA records
// LSGG_ERR_TIMEOUT, halts the step, drains its copies (bounded) and returns.
constexpr int kRedistLanes = 4;      // lanes per row (x phase) and per column (y phase)
__host__ __device__ constexpr size_t redist_layout_bytes(int side) {  // barriers, 3 plane slots, G, sign words, lists
    return 128 + (size_t)(3 * side * side + side * (side + 1)) * sizeof(float) +
           (size_t)3 * side * kRedistLanes * sizeof(unsigned) + (size_t)side * side * sizeof(unsigned short);
}

// CTAs per SM the register budget is sized for (shared memory allows them)
__host__ __device__ constexpr int redist_min_blocks(int side) { return side <= 32 ? 8 : side <= 40 ? 6 : side <= 48 ? 5 : 2; }

template <int SIDE, int NT, bool GRP>
__global__ void __launch_bounds__(NT, GRP ? (redist_min_blocks(SIDE) > 2 ? redist_min_blocks(SIDE) - 1 : 2)
                                          : redist_min_blocks(SIDE))
p_redist_xy(StepBuffers B1, GroupRef grp, int tier) {
    constexpr int PA = SIDE * SIDE;                   // floats per plane slot
    constexpr int PG = SIDE + 1;                      // pitch of G
    constexpr int LANES = kRedistLanes;
    constexpr int L = SIDE / LANES;                   // cells per segment
    constexpr int WS = SIDE * LANES;                  // sign words per slot
    static_assert(NT == LANES * SIDE && SIDE % LANES == 0, "four lanes per row of the plane");
    static_assert(L <= 32, "a segment's signs fit one word");
    extern __shared__ __align__(128) unsigned char smraw[];    // redist_layout_bytes(SIDE)
    static_assert(128 + sizeof(float) * (3 * PA + SIDE * PG) + sizeof(unsigned) * 3 * WS +
                  sizeof(unsigned short) * PA == redist_layout_bytes(SIDE), "one layout");
    uint64_t* bar = reinterpret_cast<uint64_t*>(smraw);
    float* const slots = reinterpret_cast<float*>(smraw + 128);
    float* const G = slots + 3 * PA;
    unsigned* const W = reinterpret_cast<unsigned*>(G + SIDE * PG);
    // per warp, the reference cells of its rows (row << 8 | x): 32 lanes x L cells
    unsigned short* const RL = reinterpret_cast<unsigned short*>(W + 3 * WS) + (threadIdx.x >> 5) * (32 * L);
    __shared__ int s_flag;
    __shared__ int s_gb[GRP ? kMaxGroup + 1 : 1];
    const int t = threadIdx.x;
    if (t == 0) {
        const bool fits = dyn_smem_bytes() >= redist_layout_bytes(SIDE);
        if (fits) {
            for (int k = 0; k < 3; ++k) mbar_init(&bar[k], 1);
            fence_mbar_init();
        } else {
            refuse_launch<GRP>(B1, grp);
        }
        s_flag = !fits || (!GRP && halted(B1));
    }
    __syncthreads();
    if (s_flag) return;
    const int r = t / LANES, s = t % LANES;           // x phase: row r; y phase: column r
    const int x0 = s * L;                             // first cell of the segment
    uint32_t phase = 0;                               // bit k: parity of slot k's next completion
    uint32_t pending = 0;                             // bit k: a copy into slot k is in flight
    const int n_items = GRP ? group_scan(grp, kItemSlabs, tier, true, s_gb) : B1.st->n_slabs[tier];
    const int2* items = GRP ? nullptr : B1.slab_items + B1.st->slab_base[tier];
    for (int item = blockIdx.x; item < n_items; item += gridDim.x) {
        int local;
        const StepBuffers& B = member<GRP>(B1, grp, s_gb, item, local);
        const Domain D = B.dom;
        const float eps = D.eps;
        const float4 fill = make_float4(-eps, -eps, -eps, -eps);
        const int2 it = list_item<GRP>(B, items, kItemSlabs, tier, item, local);
        const int b = it.x, z0 = it.y;
        const Box nb = B.cur[b];
        const int nx = nb.nx, ny = nb.ny, nz = nb.nz;
        const bool fx = nx == D.nx, fy = ny == D.ny, fz = nz == D.nz;
        const int ps = plane_stride(nx, ny);
        const int n = nx * ny;
        const float* zb = B.Z + nb.off;
        const int z1 = min(z0 + B.slab, nz);
        if (max(nx, ny) > SIDE) {                           // not this tier's box: refuse, never overrun
            if (t == 0) { atomicExch(&B.st->status, LSGG_ERR_UNSUPPORTED); atomicExch(&B.st->halt, 1); }
            return;                                         // no copy is in flight between items
        }
        // cells of this thread's segment inside the row (x phase), its valid bits
        const int nbits = min(max(nx - x0, 0), L);
        const unsigned valid = nbits >= 32 ? 0xffffffffu : (1u << nbits) - 1u;
        // the cell of the last segment holding x = nx - 1, for the periodic wrap
        const int sl = (nx - 1) / L, jl = (nx - 1) - sl * L;
        // plane zz (z0 - 1 <= zz <= z1) lives in slot (zz - z0 + 1) mod 3; a
        // plane outside a non-periodic box is the -eps fill
        auto request = [&](int zz) {
            const int k = (zz - z0 + 1) % 3;
            const int src = fz ? pmod(zz, nz) : zz;
            if (src >= 0 && src < nz) {
                if (t == 0) {
                    fence_async_smem();                 // earlier generic accesses to the slot come first
                    mbar_expect(&bar[k], (uint32_t)ps * 4u);
                    bulk_load(slots + k * PA, zb + (long long)src * ps, (uint32_t)ps * 4u, &bar[k]);
                }
                pending |= 1u << k;
            } else {
                float4* d = reinterpret_cast<float4*>(slots + k * PA);
                for (int q = t; q < ps / 4; q += NT) d[q] = fill;
            }
        };
        __syncthreads();                                    // previous item done with the slots, G and W
        request(z0 - 1);
        request(z0);
        request(z0 + 1);
        unsigned fresh = 7u;                                // slots whose sign words are still to be made
        for (int z = z0; z < z1; ++z) {
            bool ok = true;
#pragma unroll
            for (int k = 0; k < 3; ++k)
                if ((pending >> k) & 1u) {
                    if (mbar_wait(&bar[k], (phase >> k) & 1u, B.wait_limit)) {
                        phase ^= 1u << k;
                        pending &= ~(1u << k);
                    } else {
                        ok = false;
                    }
                }
            if (!__syncthreads_and(ok)) {                   // also publishes the fills
                if (t == 0) {
                    atomicExch(&B.st->status, LSGG_ERR_TIMEOUT);
                    atomicExch(&B.st->halt, 1);
                    for (int k = 0; k < 3; ++k)
                        if ((pending >> k) & 1u) mbar_wait(&bar[k], (phase >> k) & 1u);
                }
                __syncthreads();
                return;
            }
            const int km = (z - z0) % 3, kc = (z - z0 + 1) % 3, kp = (z - z0 + 2) % 3;
            const float* Pm = slots + km * PA;
            const float* Pc = slots + kc * PA;
            const float* Pp = slots + kp * PA;
            // sign words of the planes that entered the ring: plane z + 1, and at
            // the slab's start planes z - 1 and z as well
            fresh |= 1u << kp;
#pragma unroll
            for (int k = 0; k < 3; ++k)
                if ((fresh >> k) & 1u) {
                    // cells past the row's end read a later row or the slot's tail
                    // (in bounds) and are masked off
                    const float* row = slots + k * PA + min(r, ny - 1) * nx + x0;
                    unsigned w = 0u;
#pragma unroll
                    for (int j = 0; j < L; ++j) w |= (row[j] > 0.0f ? 1u : 0u) << j;
                    W[k * WS + t] = r < ny ? w & valid : 0u;
                }
            fresh = 0u;
            __syncthreads();
            // classification and the x scan of row r, segment s
            float rr[L];
            {
                const unsigned* Wc = W + kc * WS;
                unsigned ref = 0u;
                if (r < ny) {
                    const unsigned m0 = Wc[t];
                    unsigned lbit, rbit;
                    if (s > 0) lbit = (Wc[t - 1] >> (L - 1)) & 1u;
                    else lbit = fx ? (Wc[r * LANES + sl] >> jl) & 1u : 0u;
                    if (x0 + L < nx) rbit = Wc[t + 1] & 1u;
                    else rbit = fx ? Wc[r * LANES] & 1u : 0u;
                    const unsigned mL = (m0 << 1) | lbit;
                    const unsigned mR = nbits > 0 ? (m0 >> 1) | (rbit << (nbits - 1)) : 0u;
                    const unsigned mU = r > 0 ? Wc[t - LANES] : (fy ? Wc[(ny - 1) * LANES + s] : 0u);
                    const unsigned mD = r < ny - 1 ? Wc[t + LANES] : (fy ? Wc[s] : 0u);
                    const unsigned mZm = W[km * WS + t], mZp = W[kp * WS + t];
                    ref = ((m0 ^ mL) | (m0 ^ mR) | (m0 ^ mU) | (m0 ^ mD) | (m0 ^ mZm) | (m0 ^ mZp)) & valid;
                }
                // the warp's reference cells into its list (lane order), then
                // spread evenly over its lanes: planar-exact distance from the
                // opposite-sign neighbours -> G
                const int lane = t & 31;
                const int cnt = __popc(ref);
                int pre = cnt;
#pragma unroll
                for (int o = 1; o < 32; o <<= 1) {
                    const int v = __shfl_up_sync(0xffffffffu, pre, o);
                    if (lane >= o) pre += v;
                }
                const int total = __shfl_sync(0xffffffffu, pre, 31);
                pre -= cnt;
                for (unsigned m = ref; m; m &= m - 1u) RL[pre++] = (unsigned short)((r << 8) | (x0 + __ffs(m) - 1));
                __syncwarp();
                for (int q = lane; q < total; q += 32) {
                    const unsigned e = RL[q];
                    const int ry = (int)(e >> 8), x = (int)(e & 0xffu);
                    const int i = ry * nx + x;
                    const float v = Pc[i];
                    const bool pos = v > 0.0f;
                    const float xl = x > 0 ? Pc[i - 1] : (fx ? Pc[i + nx - 1] : -eps);
                    const float xr = x < nx - 1 ? Pc[i + 1] : (fx ? Pc[i - nx + 1] : -eps);
                    const float yl = ry > 0 ? Pc[i - nx] : (fy ? Pc[i + n - nx] : -eps);
                    const float yr = ry < ny - 1 ? Pc[i + nx] : (fy ? Pc[i - n + nx] : -eps);
                    G[ry * PG + x] = ref_magnitude(fabsf(v), opp_max(pos, xl, xr), opp_max(pos, yl, yr),
                                                   opp_max(pos, Pm[i], Pp[i]), eps);
                }
                __syncwarp();
#pragma unroll
                for (int j = 0; j < L; ++j) {
                    const float g = G[r * PG + x0 + j];            // in bounds; used at reference cells only
                    rr[j] = (ref >> j) & 1u ? g : eps;
                }
                if (!fx) scan_seg_regs<L, LANES>(rr, s, eps);
                // rows past ny and cells past nx of G are written but never read
#pragma unroll
                for (int j = 0; j < L; ++j) G[r * PG + x0 + j] = rr[j];
                if (fx) {                                   // periodic x: the row twice around, one lane
                    __syncwarp();
                    if (s == 0 && r < ny) scan_line_wrap(G + r * PG, nx, 1);
                }
            }
            __syncthreads();                                // G holds the x scans; the slot of z - 1 is free
            if (z + 1 < z1) request(z + 2);
            // y scan of column c = r, rows [s L, s L + L), then the signs of plane z back
            {
                const int c = r;
                if (fy) {                                   // periodic y: the column twice around, one lane
                    if (s == 0 && c < nx) scan_line_wrap(G + c, ny, PG);
                    __syncwarp();
                }
#pragma unroll
                for (int j = 0; j < L; ++j) {
                    const float g = G[(x0 + j) * PG + c];          // in bounds; rows past ny are eps
                    rr[j] = x0 + j < ny ? g : eps;
                }
                if (!fy) scan_seg_regs<L, LANES>(rr, s, eps);
                float* dst = B.Y + nb.off + (long long)z * ps + c;
                const float* pcol = Pc + c;
#pragma unroll
                for (int j = 0; j < L; ++j) {
                    const int y = x0 + j;
                    const float sgn = pcol[min(y, ny - 1) * nx];   // in bounds; stored only inside the plane
                    if (c < nx && y < ny) dst[y * nx] = sgn > 0.0f ? rr[j] : -rr[j];
                }
            }
        }
    }
}

// ---------------------------------------------------------------------------
// pass 5: z taxicab pass per column, clamp, bounding box of the positive set
// ---------------------------------------------------------------------------
// Column of nz <= NZ cells on a non-periodic axis, held in registers: the
// magnitudes are scanned forward and backward and the signs put back.
// Returns the mask of positive cells (bit z).
template <int NZ>
__device__ __forceinline__ unsigned long long redist_column(const StepBuffers& B, const float* hc, long long xo,
                                                            float* dc, int nz, int ps, float eps) {
    float r[NZ];
    unsigned long long pm = 0;
    // unconditional loads (cells past the column re-read its last cell), so
    // that all of them are in flight at once
#pragma unroll
    for (int z = 0; z < NZ; ++z) r[z] = __ldg(hc + (long long)min(z, nz - 1) * ps);
#pragma unroll
    for (int z = 0; z < NZ; ++z) {
        if (z < nz && sgn_pos(r[z])) pm |= 1ull << z;
        r[z] = z < nz ? fabsf(r[z]) : eps;
    }
    scan_regs(r);
#pragma unroll
    for (int z = 0; z < NZ; ++z)
        if (z < nz) {
            const float out = (pm >> z) & 1ull ? r[z] : -r[z];
            st_state(B, xo + (long long)z * ps, out);
            if (dc) dc[(long long)z * ps] = out;
        }
    return pm;
}

template <bool GRP>
__global__ void __launch_bounds__(kColThreads, 2)
p_redist_z(StepBuffers B1, GroupRef grp, DebugOut dbg, int tier) {
    __shared__ int s_gb[GRP ? kMaxGroup + 1 : 1];
    if (!GRP && halted(B1)) return;
    constexpr int ZR = kReachP + 1;
    const int n_items = GRP ? group_scan(grp, kItemChunks, tier, true, s_gb) : B1.st->n_chunks[tier];
    const int2* items = GRP ? nullptr : B1.chunk_items + B1.st->chunk_base[tier];
    for (int item = blockIdx.x; item < n_items; item += gridDim.x) {
        int local;
        const StepBuffers& B = member<GRP>(B1, grp, s_gb, item, local);
        const Domain D = B.dom;
        const float eps = D.eps;
        const int2 it = list_item<GRP>(B, items, kItemChunks, tier, item, local);
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
            const long long xo = nb.off + c;
            if (!fz && nz <= 64) {                         // uniform across the CTA (one box per item)
                float* dc = dbg.phin ? dbg.phin + nb.off + c : nullptr;
                const unsigned long long pm = nz <= 16   ? redist_column<16>(B, hc, xo, dc, nz, ps, eps)
                                              : nz <= 32 ? redist_column<32>(B, hc, xo, dc, nz, ps, eps)
                                              : nz <= 48 ? redist_column<48>(B, hc, xo, dc, nz, ps, eps)
                                                         : redist_column<64>(B, hc, xo, dc, nz, ps, eps);
                if (pm) {
                    lo[0] = hi[0] = x;
                    lo[1] = hi[1] = y;
                    lo[2] = __ffsll((long long)pm) - 1;
                    hi[2] = 63 - __clzll((long long)pm);
                }
            } else {
                // periodic or long column: forward scan over a register ring,
                // backward over a 6-plane window
                float fr[ZR];                              // forward-swept planes zb-6 .. zb
#pragma unroll
                for (int k = 0; k < ZR; ++k) fr[k] = -eps;
                // periodic z: the sweep starts 6 planes early so that plane 0 sees its wrapped predecessors
                const int zb_first = fz ? -kReachP : 0;
                const int n_zb = nz + kReachP - zb_first;  // zb = zb_first .. nz-1+6
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
                        st_state(B, xo + (long long)zo * ps, out);
                        if (dbg.phin) dbg.phin[nb.off + (long long)zo * ps + c] = out;
                        if (out > 0.0f) {
                            lo[0] = min(lo[0], x); hi[0] = max(hi[0], x);
                            lo[1] = min(lo[1], y); hi[1] = max(hi[1], y);
                            lo[2] = min(lo[2], zo); hi[2] = max(hi[2], zo);
                        }
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
// Godunov re-initialisation (LSGG_REDIST_GODUNOV)
// ---------------------------------------------------------------------------
// The same reference cells and values as the taxicab scheme; every other cell
// takes the smallest u with sum over the axes whose neighbour minimum a_k is
// below u of (u - a_k)^2 = 1 (the Euclidean first-order upwind update of
// Zhao's fast sweeping), capped at eps.  Non-reference cells have only
// same-sign face neighbours, so no sign test is needed.  The update is not
// separable: Jacobi sweeps over all boxes' columns (kGodunovSweeps, even, so
// the magnitudes end in Y), ping-ponging between Y and X (the state is not
// read after the predictor).  Reference cells are stored as -(1 + |d|) and
// held fixed.  All tiers' column items at once: their lists are contiguous.
constexpr int kGodunovSweeps = 20;     // fixed point to ~1e-8 (FP64 oracle), well inside the 1e-4 tolerance

__device__ __forceinline__ float god_mag(float v) { return v < 0.0f ? -v - 1.0f : v; }

__device__ __forceinline__ float godunov_u(float a, float b, float c) {
    // sort a <= b <= c
    float t;
    if (b < a) { t = a; a = b; b = t; }
    if (c < b) { t = b; b = c; c = t; }
    if (b < a) { t = a; a = b; b = t; }
    float u = a + 1.0f;
    if (u > b) {
        const float d = a - b;
        u = 0.5f * (a + b + sqrtf(2.0f - d * d));
        if (u > c) {
            const float s = a + b + c;
            u = (s + sqrtf(fmaxf(s * s - 3.0f * (a * a + b * b + c * c - 1.0f), 0.0f))) * (1.0f / 3.0f);
        }
    }
    return u;
}

__device__ __forceinline__ int god_n_items(const StepBuffers& B) {
    int n = 0;
#pragma unroll
    for (int t = 0; t < kTiers; ++t) n += B.st->n_chunks[t];
    return n;
}

// classification -> Y (non-reference eps, reference -(1 + distance))
__global__ void __launch_bounds__(kColThreads)
p_god_init(StepBuffers B) {
    if (halted(B)) return;
    const Domain D = B.dom;
    const float eps = D.eps;
    const int n_items = god_n_items(B);
    for (int item = blockIdx.x; item < n_items; item += gridDim.x) {
        const int2 it = B.chunk_items[item];
        const Box nb = B.cur[it.x];
        const int nx = nb.nx, ny = nb.ny, nz = nb.nz;
        const bool fx = nx == D.nx, fy = ny == D.ny, fz = nz == D.nz;
        const int c = it.y * kPassChunk + threadIdx.x;
        if (c >= nx * ny) continue;
        const int y = c / nx, x = c - y * nx;
        const int ps = plane_stride(nx, ny);
        const long long o0 = nb.off + c;
        const int dxl = x > 0 ? -1 : (fx ? nx - 1 : 0), dxr = x < nx - 1 ? 1 : (fx ? 1 - nx : 0);
        const int dyl = y > 0 ? -nx : (fy ? (ny - 1) * nx : 0), dyr = y < ny - 1 ? nx : (fy ? (1 - ny) * nx : 0);
        for (int z = 0; z < nz; ++z) {
            const long long o = o0 + (long long)z * ps;
            const float v = __ldg(B.Z + o);
            const bool pos = v > 0.0f;
            const float xl = dxl ? __ldg(B.Z + o + dxl) : -eps, xr = dxr ? __ldg(B.Z + o + dxr) : -eps;
            const float yl = dyl ? __ldg(B.Z + o + dyl) : -eps, yr = dyr ? __ldg(B.Z + o + dyr) : -eps;
            const int zm = z > 0 ? z - 1 : (fz ? nz - 1 : -1), zp = z < nz - 1 ? z + 1 : (fz ? 0 : -1);
            const float zl = zm >= 0 ? __ldg(B.Z + o0 + (long long)zm * ps) : -eps;
            const float zr = zp >= 0 ? __ldg(B.Z + o0 + (long long)zp * ps) : -eps;
            const float m = ref_magnitude(fabsf(v), opp_max(pos, xl, xr), opp_max(pos, yl, yr), opp_max(pos, zl, zr), eps);
            B.Y[o] = m < eps ? -(1.0f + m) : eps;
        }
    }
}

// one Jacobi sweep src -> dst
__global__ void __launch_bounds__(kColThreads)
p_god_sweep(StepBuffers B, const float* __restrict__ src, float* __restrict__ dst) {
    if (halted(B)) return;
    const Domain D = B.dom;
    const float eps = D.eps;
    const int n_items = god_n_items(B);
    for (int item = blockIdx.x; item < n_items; item += gridDim.x) {
        const int2 it = B.chunk_items[item];
        const Box nb = B.cur[it.x];
        const int nx = nb.nx, ny = nb.ny, nz = nb.nz;
        const bool fx = nx == D.nx, fy = ny == D.ny, fz = nz == D.nz;
        const int c = it.y * kPassChunk + threadIdx.x;
        if (c >= nx * ny) continue;
        const int y = c / nx, x = c - y * nx;
        const int ps = plane_stride(nx, ny);
        const long long o0 = nb.off + c;
        const int dxl = x > 0 ? -1 : (fx ? nx - 1 : 0), dxr = x < nx - 1 ? 1 : (fx ? 1 - nx : 0);
        const int dyl = y > 0 ? -nx : (fy ? (ny - 1) * nx : 0), dyr = y < ny - 1 ? nx : (fy ? (1 - ny) * nx : 0);
        const float inf = __int_as_float(0x7f800000);
        // batches of kZB planes: every load of a batch is issued before any use
        // (indices clamped into the column, the values of absent neighbours
        // replaced afterwards)
        for (int z0 = 0; z0 < nz; z0 += kZB) {
            float col[kZB + 2], xl[kZB], xr[kZB], yl[kZB], yr[kZB];
#pragma unroll
            for (int u = 0; u < kZB + 2; ++u) {
                int z = z0 + u - 1;
                const bool in = z >= 0 && z < nz;
                if (!in && fz) z = z < 0 ? z + nz : z - nz;
                const int zc = min(max(z, 0), nz - 1);
                col[u] = src[o0 + (long long)zc * ps];
                if (!in && !fz) col[u] = -16.0f;           // marker: no neighbour (encoded values are >= -2)
            }
#pragma unroll
            for (int u = 0; u < kZB; ++u) {
                const long long o = o0 + (long long)min(z0 + u, nz - 1) * ps;
                xl[u] = src[o + dxl];
                xr[u] = src[o + dxr];
                yl[u] = src[o + dyl];
                yr[u] = src[o + dyr];
            }
#pragma unroll
            for (int u = 0; u < kZB; ++u) {
                const int z = z0 + u;
                if (z >= nz) break;
                const float v = col[u + 1];
                const long long o = o0 + (long long)z * ps;
                if (v < 0.0f) { dst[o] = v; continue; }
                const float ax = fminf(dxl ? god_mag(xl[u]) : inf, dxr ? god_mag(xr[u]) : inf);
                const float ay = fminf(dyl ? god_mag(yl[u]) : inf, dyr ? god_mag(yr[u]) : inf);
                const float zl = col[u] == -16.0f ? inf : god_mag(col[u]);
                const float zr = col[u + 2] == -16.0f ? inf : god_mag(col[u + 2]);
                dst[o] = fminf(v, fminf(eps, godunov_u(ax, ay, fminf(zl, zr))));
            }
        }
    }
}

// signs of phi_c back -> X, positive bounding box
__global__ void __launch_bounds__(kColThreads)
p_god_final(StepBuffers B, DebugOut dbg) {
    if (halted(B)) return;
    const Domain D = B.dom;
    const int n_items = god_n_items(B);
    for (int item = blockIdx.x; item < n_items; item += gridDim.x) {
        const int2 it = B.chunk_items[item];
        const int b = it.x;
        const Box nb = B.cur[b];
        const int nx = nb.nx, ny = nb.ny, nz = nb.nz;
        const int c = it.y * kPassChunk + threadIdx.x;
        int lo[3] = {INT_MAX, INT_MAX, INT_MAX}, hi[3] = {INT_MIN, INT_MIN, INT_MIN};
        if (c < nx * ny) {
            const int y = c / nx, x = c - y * nx;
            const int ps = plane_stride(nx, ny);
            for (int z = 0; z < nz; ++z) {
                const long long o = nb.off + c + (long long)z * ps;
                const float m = god_mag(B.Y[o]);
                const float out = __ldg(B.Z + o) > 0.0f ? m : -m;
                st_state(B, o, out);
                if (dbg.phin) dbg.phin[o] = out;
                if (out > 0.0f) {
                    lo[0] = min(lo[0], x); hi[0] = max(hi[0], x);
                    lo[1] = min(lo[1], y); hi[1] = max(hi[1], y);
                    lo[2] = min(lo[2], z); hi[2] = max(hi[2], z);
                }
            }
        }
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
// constrained reinitialization of Hartmann et al. (LSGG_REDIST_HARTMANN)
// ---------------------------------------------------------------------------
// Forward-Euler pseudo-time steps of phi_tau + S(phi0) (|grad phi| - 1) =
// beta F from phi0 = phi_c (which stays in Z): S(phi0) = phi0 / sqrt(phi0^2 +
// 1), |grad phi| by Godunov's upwind scheme (per axis, with a = phi_i -
// phi_{i-1} and b = phi_{i+1} - phi_i, max(max(a, 0)^2, min(b, 0)^2) where S >
// 0 and max(min(a, 0)^2, max(b, 0)^2) otherwise), and on a cell with face
// neighbours j of the opposite sign in phi0 (and phi0_j != 0) F = mean over
// them of (phi0_i / phi0_j) phi_j - phi_i, the value that keeps each linearly
// interpolated zero crossing of phi0 in place; every iterate is clamped to
// [-eps, eps], values outside the box are -eps.  A thread walks one column of
// a box along z with the z neighbours of phi and phi0 in registers; the
// steps ping-pong between Y and X (the state is not read after the
// predictor), and the last one stores the state and the positive bounding
// box.  The axes and the neighbours enter the sums in the order z, y, x and
// +1, -1.
constexpr int kHcrIters = 20;         // pseudo-time steps
constexpr float kHcrDtau = 0.5f;      // pseudo-time step (grid units)
constexpr float kHcrBeta = 0.5f;      // weight of the constraint forcing

__device__ __forceinline__ float hcr_axis(float a, float b, bool sp) {
    const float p = sp ? fmaxf(a, 0.0f) : fminf(a, 0.0f);
    const float q = sp ? fminf(b, 0.0f) : fmaxf(b, 0.0f);
    return fmaxf(p * p, q * q);
}

__device__ __forceinline__ void hcr_term(float q0, bool pos0, float nb0, float nbv, float& cons, int& cnt) {
    if ((nb0 > 0.0f) != pos0 && nb0 != 0.0f) {
        cons += (q0 / nb0) * nbv;
        ++cnt;
    }
}

template <bool LAST>
__global__ void __launch_bounds__(kColThreads)
p_hcr_step(StepBuffers B, const float* __restrict__ src, float* __restrict__ dst, DebugOut dbg) {
    if (halted(B)) return;
    const Domain D = B.dom;
    const float eps = D.eps;
    const float* __restrict__ P0 = B.Z;
    const int n_items = god_n_items(B);
    for (int item = blockIdx.x; item < n_items; item += gridDim.x) {
        const int2 it = B.chunk_items[item];
        const int b = it.x;
        const Box nb = B.cur[b];
        const int nx = nb.nx, ny = nb.ny, nz = nb.nz;
        const bool fx = nx == D.nx, fy = ny == D.ny, fz = nz == D.nz;
        const int c = it.y * kPassChunk + threadIdx.x;
        int lo[3] = {INT_MAX, INT_MAX, INT_MAX}, hi[3] = {INT_MIN, INT_MIN, INT_MIN};
        if (c < nx * ny) {
            const int y = c / nx, x = c - y * nx;
            const int ps = plane_stride(nx, ny);
            const long long o0 = nb.off + c;
            const int dxl = x > 0 ? -1 : (fx ? nx - 1 : 0), dxr = x < nx - 1 ? 1 : (fx ? 1 - nx : 0);
            const int dyl = y > 0 ? -nx : (fy ? (ny - 1) * nx : 0), dyr = y < ny - 1 ? nx : (fy ? (1 - ny) * nx : 0);
            // plane zz of a field at this column; -eps outside a non-periodic box
            auto at = [&](const float* f, int zz) -> float {
                if (zz < 0 || zz >= nz) {
                    if (!fz) return -eps;
                    zz = zz < 0 ? zz + nz : zz - nz;
                }
                return f[o0 + (long long)zz * ps];
            };
            float pm = at(src, -1), pc = at(src, 0), qm = at(P0, -1), qc = at(P0, 0);
            for (int z = 0; z < nz; ++z) {
                const float pp = at(src, z + 1), qp = at(P0, z + 1);
                const long long o = o0 + (long long)z * ps;
                const float yl = dyl ? src[o + dyl] : -eps, yr = dyr ? src[o + dyr] : -eps;
                const float xl = dxl ? src[o + dxl] : -eps, xr = dxr ? src[o + dxr] : -eps;
                const float qyl = dyl ? P0[o + dyl] : -eps, qyr = dyr ? P0[o + dyr] : -eps;
                const float qxl = dxl ? P0[o + dxl] : -eps, qxr = dxr ? P0[o + dxr] : -eps;
                const float s0 = qc / sqrtf(qc * qc + 1.0f);
                const bool sp = s0 > 0.0f;
                float g2 = hcr_axis(pc - pm, pp - pc, sp);
                g2 += hcr_axis(pc - yl, yr - pc, sp);
                g2 += hcr_axis(pc - xl, xr - pc, sp);
                const bool pos0 = qc > 0.0f;
                float cons = 0.0f;
                int cnt = 0;
                hcr_term(qc, pos0, qp, pp, cons, cnt);
                hcr_term(qc, pos0, qm, pm, cons, cnt);
                hcr_term(qc, pos0, qyr, yr, cons, cnt);
                hcr_term(qc, pos0, qyl, yl, cons, cnt);
                hcr_term(qc, pos0, qxr, xr, cons, cnt);
                hcr_term(qc, pos0, qxl, xl, cons, cnt);
                const float force = cnt ? cons / (float)cnt - pc : 0.0f;
                float out = pc - kHcrDtau * s0 * (sqrtf(g2) - 1.0f) + kHcrDtau * kHcrBeta * force;
                out = fminf(fmaxf(out, -eps), eps);
                if (LAST) {
                    st_state(B, o, out);
                    if (dbg.phin) dbg.phin[o] = out;
                    if (out > 0.0f) {
                        lo[0] = min(lo[0], x); hi[0] = max(hi[0], x);
                        lo[1] = min(lo[1], y); hi[1] = max(hi[1], y);
                        lo[2] = min(lo[2], z); hi[2] = max(hi[2], z);
                    }
                } else {
                    dst[o] = out;
                }
                pm = pc; pc = pp;
                qm = qc; qc = qp;
            }
        }
        if (LAST) {
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
}

cudaError_t launch_sweep_redist(const StepBuffers& B, const DebugOut& dbg, cudaStream_t s) {
    const int grid = B.pgrid[0][4];
    if (B.redist == LSGG_REDIST_HARTMANN) {
        // step k reads Z (k = 0), Y (k odd) or X (k even), writes Y (k even) or X
        static_assert(kHcrIters % 2 == 0, "the last step reads Y and stores the state");
        for (int k = 0; k < kHcrIters - 1; ++k) {
            const float* src = k == 0 ? B.Z : ((k & 1) ? B.Y : B.X);
            float* dst = (k & 1) ? B.X : B.Y;
            p_hcr_step<false><<<grid, kColThreads, 0, s>>>(B, src, dst, dbg);
        }
        p_hcr_step<true><<<grid, kColThreads, 0, s>>>(B, B.Y, B.X, dbg);
        return cudaGetLastError();
    }
    p_god_init<<<grid, kColThreads, 0, s>>>(B);
    for (int k = 0; k < kGodunovSweeps; ++k) {
        const bool even = (k & 1) == 0;
        p_god_sweep<<<grid, kColThreads, 0, s>>>(B, even ? B.Y : B.X, even ? B.X : B.Y);
    }
    p_god_final<<<grid, kColThreads, 0, s>>>(B, dbg);
    return cudaGetLastError();
}

// ---------------------------------------------------------------------------
// general-size tier: plane passes through global memory
// ---------------------------------------------------------------------------
// Boxes with an x or y side above 64 (the lognormal tail of a power-diagram
// tessellation, grains grown large) exceed every shared-memory plane grid.
// Their plane passes keep one CTA per (box, plane) item and work through
// global memory (L1 / L2) instead: the x pass writes the plane's x-convolved
// rows into its own region of Y, the y pass reads them back after a barrier;
// the re-initialisation classifies into Y, scans rows (a thread per row) and
// columns (a thread per column) in place and puts the signs back.  Same
// arithmetic and FMA order as p_conv_xy; scans as scan_line_wrap without the
// wrap.  The column passes are the shared ones.

// Forward and backward min-plus scan of n magnitudes (stride st), in place.
__device__ __forceinline__ void scan_line_serial(float* L, int n, int st) {
    float f = L[0];
    for (int j = 1; j < n; ++j) {
        f = fminf(L[(long long)j * st], f + 1.0f);
        L[(long long)j * st] = f;
    }
    for (int j = n - 2; j >= 0; --j) {
        f = fminf(L[(long long)j * st], f + 1.0f);
        L[(long long)j * st] = f;
    }
}

template <int R, bool GRP>
__global__ void __launch_bounds__(256)
p_conv_xy_big(StepBuffers B1, GroupRef grp, Taps taps, int tier) {
    constexpr int W = 2 * R + 1;
    constexpr int kChunk = 128;                            // x outputs per staged row segment
    constexpr int kTY = 64;                                // rows per staged column tile
    __shared__ float s_row[8][kChunk + 2 * R];             // per warp: the segment's inputs (old layout, -eps outside)
    __shared__ float s_col[kTY + 2 * R][33];               // a tile of 32 columns of the x-convolved rows (padded)
    __shared__ int s_flag;
    __shared__ int s_gb[GRP ? kMaxGroup + 1 : 1];
    const int t = threadIdx.x, lane = t & 31, warp = t >> 5;
    if (t == 0) s_flag = !GRP && halted(B1);
    __syncthreads();
    if (s_flag) return;
    float g[W];
#pragma unroll
    for (int k = 0; k < W; ++k) g[k] = taps.g[k];
    const int n_items = GRP ? group_scan(grp, kItemPlanes, tier, true, s_gb) : B1.st->n_planes[tier];
    const int2* items = GRP ? nullptr : B1.plane_items + B1.st->plane_base[tier];
    for (int item = blockIdx.x; item < n_items; item += gridDim.x) {
        int local;
        const StepBuffers& B = member<GRP>(B1, grp, s_gb, item, local);
        const Domain D = B.dom;
        float aconst = 0.0f;                              // x convolution of a row of -eps
#pragma unroll
        for (int k = 0; k < W; ++k) aconst = fmaf(g[k], -D.eps, aconst);
        const int2 it = list_item<GRP>(B, items, kItemPlanes, tier, item, local);
        const int b = it.x, z = it.y;
        const Box nb = B.cur[b], ob = B.prev[b];
        const int nx = nb.nx, ny = nb.ny;
        const bool fx = nx == D.nx, fy = ny == D.ny;
        const int ps = plane_stride(nx, ny);
        const int ozl = wrap_near(nb.oz + z - ob.oz, D.nz);
        const bool zin = ozl < ob.nz;
        const long long obase = ob.off + (long long)(zin ? ozl : 0) * plane_stride(ob.nx, ob.ny);
        float* rows = B.Y + nb.off + (long long)z * ps;  // x-convolved rows of this plane (scratch)
        for (int y = warp; y < ny; y += 8) {               // x pass: warp per row, lanes along x
            const int oy = wrap_near(nb.oy + y - ob.oy, D.ny);
            const bool rin = zin && oy < ob.ny;
            const long long rbase = obase + (long long)oy * ob.nx;
            float* sr = s_row[warp];
            for (int x0 = 0; x0 < nx; x0 += kChunk) {      // segments: inputs staged once per warp
                const int nout = min(kChunk, nx - x0);
                for (int q = lane; q < nout + 2 * R; q += 32) {
                    int xl = x0 + q - R;
                    float v = -D.eps;
                    if (fx || (xl >= 0 && xl < nx)) {
                        if (fx) xl = wrap_near(xl, nx);
                        const int ox = wrap_near(nb.ox + xl - ob.ox, D.nx);
                        if (rin && ox < ob.nx) v = ld_state(B, rbase + ox);
                    }
                    sr[q] = v;
                }
                __syncwarp();
                for (int x = lane; x < nout; x += 32) {
                    float acc = 0.0f;
#pragma unroll
                    for (int k = 0; k < W; ++k) acc = fmaf(g[k], sr[x + k], acc);
                    rows[(long long)y * nx + x0 + x] = acc;
                }
                __syncwarp();                               // the segment is read before the next one
            }
        }
        __syncthreads();
        float* dst = B.Z + nb.off + (long long)z * ps;
        for (int x0 = 0; x0 < nx; x0 += 32) {              // y pass: tiles of 32 columns x kTY rows
            const int xc = x0 + lane;
            for (int y0 = 0; y0 < ny; y0 += kTY) {
                const int nrow = min(kTY, ny - y0);
                for (int r = warp; r < nrow + 2 * R; r += 8) {
                    int yl = y0 + r - R;
                    float v = aconst;                       // a row outside the box: the x convolution of -eps
                    if (xc < nx && (fy || (yl >= 0 && yl < ny))) {
                        if (fy) yl = wrap_near(yl, ny);
                        v = rows[(long long)yl * nx + xc];
                    }
                    s_col[r][lane] = v;
                }
                __syncthreads();
                for (int r = warp; r < nrow; r += 8) {
                    if (xc >= nx) continue;
                    float acc = 0.0f;
#pragma unroll
                    for (int k = 0; k < W; ++k) acc = fmaf(g[k], s_col[r + k][lane], acc);
                    dst[(long long)(y0 + r) * nx + xc] = acc;
                }
                __syncthreads();                            // the tile is read before the next one
            }
        }
    }
}

template <bool GRP>
__global__ void __launch_bounds__(256)
p_redist_xy_big(StepBuffers B1, GroupRef grp, int tier) {
    constexpr int R = kRedistReach;
    constexpr int kChunk = 128;                            // x outputs per staged row segment
    constexpr int kTY = 64;                                // rows per staged column tile
    __shared__ float s_row[8][kChunk + 2 * R];             // per warp: a row segment's magnitudes
    __shared__ float s_col[kTY + 2 * R][33];               // a tile of 32 columns (padded)
    __shared__ int s_flag;
    __shared__ int s_gb[GRP ? kMaxGroup + 1 : 1];
    const int t = threadIdx.x, lane = t & 31, warp = t >> 5;
    if (t == 0) s_flag = !GRP && halted(B1);
    __syncthreads();
    if (s_flag) return;
    const Domain D1 = B1.dom;
    const int n_items = GRP ? group_scan(grp, kItemPlanes, tier, true, s_gb) : B1.st->n_planes[tier];
    const int2* items = GRP ? nullptr : B1.plane_items + B1.st->plane_base[tier];
    for (int item = blockIdx.x; item < n_items; item += gridDim.x) {
        int local;
        const StepBuffers& B = member<GRP>(B1, grp, s_gb, item, local);
        const Domain D = GRP ? B.dom : D1;
        const float eps = D.eps;
        const int2 it = list_item<GRP>(B, items, kItemPlanes, tier, item, local);
        const int b = it.x, z = it.y;
        const Box nb = B.cur[b];
        const int nx = nb.nx, ny = nb.ny, nz = nb.nz;
        const bool fx = nx == D.nx, fy = ny == D.ny, fz = nz == D.nz;
        const int ps = plane_stride(nx, ny);
        const int n = nx * ny;
        const float* c = B.Z + nb.off + (long long)z * ps;
        const int zm = fz ? pmod(z - 1, nz) : z - 1, zp = fz ? pmod(z + 1, nz) : z + 1;
        const float* cm = zm >= 0 ? B.Z + nb.off + (long long)zm * ps : nullptr;
        const float* cp = zp < nz ? B.Z + nb.off + (long long)zp * ps : nullptr;
        float* G = B.Y + nb.off + (long long)z * ps;        // magnitudes, then the result
        for (int y = warp; y < ny; y += 8) {               // classification: warp per row
            for (int x = lane; x < nx; x += 32) {
                const long long i = (long long)y * nx + x;
                const float v = __ldg(c + i);
                const bool pos = v > 0.0f;
                const float xl = x > 0 ? __ldg(c + i - 1) : (fx ? __ldg(c + i + nx - 1) : -eps);
                const float xr = x < nx - 1 ? __ldg(c + i + 1) : (fx ? __ldg(c + i - nx + 1) : -eps);
                const float yl = y > 0 ? __ldg(c + i - nx) : (fy ? __ldg(c + i + n - nx) : -eps);
                const float yr = y < ny - 1 ? __ldg(c + i + nx) : (fy ? __ldg(c + i - n + nx) : -eps);
                const float zl = cm ? __ldg(cm + i) : -eps, zr = cp ? __ldg(cp + i) : -eps;
                G[i] = ref_magnitude(fabsf(v), opp_max(pos, xl, xr), opp_max(pos, yl, yr), opp_max(pos, zl, zr), eps);
            }
        }
        __syncthreads();
        // The line transforms as windows: no magnitude exceeds eps = 7, so a
        // cell's taxicab distance along a line is min over |k| <= R = 6 of
        // m(x + k) + |k| (past the ends of a non-periodic line: eps, which
        // never undercuts), and a window over values already transformed
        // gives the same distance.
        for (int y = warp; y < ny; y += 8) {               // x: warp per row, segments staged per warp
            float* row = G + (long long)y * nx;
            float* sr = s_row[warp];
            for (int x0 = 0; x0 < nx; x0 += kChunk) {
                const int nout = min(kChunk, nx - x0);
                for (int q = lane; q < nout + 2 * R; q += 32) {
                    const int xl = x0 + q - R;
                    sr[q] = fx ? row[pmod(xl, nx)] : (xl >= 0 && xl < nx ? row[xl] : eps);
                }
                __syncwarp();
                for (int x = lane; x < nout; x += 32) {
                    float d = sr[x + R];
#pragma unroll
                    for (int k = 1; k <= R; ++k) d = fminf(d, fminf(sr[x + R - k], sr[x + R + k]) + (float)k);
                    row[x0 + x] = d;
                }
                __syncwarp();                               // the segment is read before the next one
            }
        }
        __syncthreads();
        for (int x0 = 0; x0 < nx; x0 += 32) {              // y: tiles of 32 columns x kTY rows, then the signs
            const int xc = x0 + lane;
            for (int y0 = 0; y0 < ny; y0 += kTY) {
                const int nrow = min(kTY, ny - y0);
                for (int r = warp; r < nrow + 2 * R; r += 8) {
                    const int yl = y0 + r - R;
                    float v = eps;
                    if (xc < nx) {
                        if (fy) v = fabsf(G[(long long)pmod(yl, ny) * nx + xc]);
                        else if (yl >= 0 && yl < ny) v = fabsf(G[(long long)yl * nx + xc]);
                    }
                    s_col[r][lane] = v;
                }
                __syncthreads();
                for (int r = warp; r < nrow; r += 8) {
                    if (xc >= nx) continue;
                    float d = s_col[r + R][lane];
#pragma unroll
                    for (int k = 1; k <= R; ++k) d = fminf(d, fminf(s_col[r + R - k][lane], s_col[r + R + k][lane]) + (float)k);
                    const long long i = (long long)(y0 + r) * nx + xc;
                    G[i] = __ldg(c + i) > 0.0f ? d : -d;
                }
                __syncthreads();                            // the tile is read before the next one
            }
        }
    }
}

// ---------------------------------------------------------------------------
// host side
// ---------------------------------------------------------------------------
// The radius-specialised convolution kernels (R = 1 .. kMaxRadius) per tier
// side; the z pass with or without the velocity correction of Eq. (10).
constexpr int kTierSide[kTiers] = {32, 40, 48, 64, 1 << 30};  // the last tier: any size (global-memory plane passes)
constexpr int kRedistThreads[kTiers] = {128, 160, 192, 256, 256};   // threads per CTA of p_redist_xy (4 lanes per line)
constexpr int kConvThreads[kTiers] = {128, 160, 192, 256, 256};     // threads per CTA of p_conv_xy
constexpr int kBigTier = kTiers - 1;
static size_t conv_smem_bytes(int side, int R) {       // ConvXYLayout<R, side>::bytes
    return side > 64 ? 0 : conv_layout_bytes(R, side);   // general-size tier: static shared memory only
}
constexpr size_t redist_smem_bytes(int side) { return side > 64 ? 0 : redist_layout_bytes(side); }

struct PassFns {
    const void* conv_xy[kTiers];
    const void* conv_z;
    const void* redist_xy[kTiers];
};

template <int R, bool GRP = false>
static PassFns pass_fns_r(bool phys) {
    static_assert(kTiers == 5, "one instantiation per tier side");
    PassFns f;
    f.conv_xy[0] = reinterpret_cast<const void*>(p_conv_xy<R, 32, kConvThreads[0], GRP>);
    f.conv_xy[1] = reinterpret_cast<const void*>(p_conv_xy<R, 40, kConvThreads[1], GRP>);
    f.conv_xy[2] = reinterpret_cast<const void*>(p_conv_xy<R, 48, kConvThreads[2], GRP>);
    f.conv_xy[3] = reinterpret_cast<const void*>(p_conv_xy<R, 64, kConvThreads[3], GRP>);
    f.conv_xy[4] = reinterpret_cast<const void*>(p_conv_xy_big<R, GRP>);
    if constexpr (GRP) f.conv_z = reinterpret_cast<const void*>(p_conv_z<R, false, true>);
    else f.conv_z = phys ? reinterpret_cast<const void*>(p_conv_z<R, true, false>)
                         : reinterpret_cast<const void*>(p_conv_z<R, false, false>);
    f.redist_xy[0] = reinterpret_cast<const void*>(p_redist_xy<32, kRedistThreads[0], GRP>);
    f.redist_xy[1] = reinterpret_cast<const void*>(p_redist_xy<40, kRedistThreads[1], GRP>);
    f.redist_xy[2] = reinterpret_cast<const void*>(p_redist_xy<48, kRedistThreads[2], GRP>);
    f.redist_xy[3] = reinterpret_cast<const void*>(p_redist_xy<64, kRedistThreads[3], GRP>);
    f.redist_xy[4] = reinterpret_cast<const void*>(p_redist_xy_big<GRP>);
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
    PassFns fn, fn_ideal;
    if (!pass_fns(B.dom.radius, true, &fn) || !pass_fns(B.dom.radius, false, &fn_ideal)) return cudaErrorInvalidValue;
    cudaError_t e = cudaSuccess;
    for (int t = 0; t < kTiers; ++t) {
        B.tier_side[t] = kTierSide[t];
        B.tier_threads[t] = kTierSide[t];
        int o[5] = {0, 0, 0, 0, 0};       // conv_xy, conv_z (ideal), conv_z (physics), redist_xy, redist_z
        e = t == kBigTier ? cudaSuccess : allow_max_dynamic_smem(fn.conv_xy[t]);
        if (e == cudaSuccess)
            e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&o[0], fn.conv_xy[t], kConvThreads[t],
                                                              conv_smem_bytes(kTierSide[t], B.dom.radius));
        if (e == cudaSuccess) e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&o[1], fn_ideal.conv_z, kColThreads, 0);
        if (e == cudaSuccess) e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&o[2], fn.conv_z, kColThreads, 0);
        if (e == cudaSuccess && t != kBigTier) e = allow_max_dynamic_smem(fn.redist_xy[t]);
        if (e == cudaSuccess)
            e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&o[3], fn.redist_xy[t], kRedistThreads[t],
                                                              redist_smem_bytes(kTierSide[t]));
        if (e == cudaSuccess) e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&o[4], p_redist_z<false>, kColThreads, 0);
        if (e != cudaSuccess) return e;
        for (int k = 0; k < 5; ++k) {
            B.pocc[t][k] = o[k] < 1 ? 1 : o[k];
            B.pgrid[t][k] = B.n_sm * B.pocc[t][k];
        }
    }
    int of = 0;
    e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&of, p_field<false, false, false>, kTileX * kTileY, 0);
    if (e != cudaSuccess) return e;
    B.field_grid[0] = B.n_sm * (of < 1 ? 1 : of);
    e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&of, p_field<true, false, false>, kTileX * kTileY, 0);
    if (e != cudaSuccess) return e;
    B.field_grid[1] = B.n_sm * (of < 1 ? 1 : of);
    B.bin_grid = B.n_sm;
    if (B.slab < kMinSlab) B.slab = kSlab;
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
    const int* g = B.pgrid[tier];
    StepBuffers bb = B;
    Taps tp = taps;
    PhysicsDev ph = phys;
    DebugOut db = dbg;
    int tr = tier;
    int k = 0;
    cudaError_t e;
    GroupRef none{nullptr, 0};
    if (pass_ev) cudaEventRecord(pass_ev[k++], s);
    if (which == 0) {
        void* a0[] = {&bb, &none, &tp, &tr};
        e = cudaLaunchKernel(fn.conv_xy[tier], dim3(g[0]), dim3(kConvThreads[tier]), a0,
                             conv_smem_bytes(kTierSide[tier], taps.radius), s);
        if (e != cudaSuccess) return e;
        if (pass_ev) cudaEventRecord(pass_ev[k++], s);
        void* a1[] = {&bb, &none, &tp, &ph, &tr};
        e = cudaLaunchKernel(fn.conv_z, dim3(g[phys.kind != LSGG_PHYSICS_IDEAL ? 2 : 1]), dim3(kColThreads), a1, 0, s);
        if (e != cudaSuccess) return e;
        if (pass_ev) cudaEventRecord(pass_ev[k++], s);
    } else {
        void* a3[] = {&bb, &none, &tr};
        e = cudaLaunchKernel(fn.redist_xy[tier], dim3(g[3]), dim3(kRedistThreads[tier]), a3,
                             redist_smem_bytes(kTierSide[tier]), s);
        if (e != cudaSuccess) return e;
        if (pass_ev) cudaEventRecord(pass_ev[k++], s);
        void* a4[] = {&bb, &none, &db, &tr};
        e = cudaLaunchKernel(reinterpret_cast<const void*>(p_redist_z<false>), dim3(g[4]), dim3(kColThreads), a4, 0, s);
        if (e != cudaSuccess) return e;
        if (pass_ev) cudaEventRecord(pass_ev[k++], s);
    }
    return cudaGetLastError();
}

cudaError_t launch_bin(const StepBuffers& B, cudaStream_t s) {
    cudaError_t e = cudaMemsetAsync(B.tile_cnt, 0, sizeof(int) * (size_t)B.n_tiles, s);
    if (e != cudaSuccess) return e;
    k_bin<false><<<B.bin_grid, 256, 0, s>>>(B, GroupRef{nullptr, 0});
    return cudaGetLastError();
}

cudaError_t launch_field(const StepBuffers& B, const PhysicsDev& phys, const DebugOut& dbg, cudaStream_t s) {
    const bool idf = phys.kind != LSGG_PHYSICS_IDEAL, dg = dbg.m != nullptr;
    auto k = idf ? (dg ? p_field<true, true, false> : p_field<true, false, false>)
                 : (dg ? p_field<false, true, false> : p_field<false, false, false>);
    k<<<B.field_grid[idf || dg ? 1 : 0], kTileX * kTileY, 0, s>>>(B, GroupRef{nullptr, 0}, phys, dbg);
    return cudaGetLastError();
}

// ---- step groups ----
// Persistent grids of the group kernels (their own occupancy: the group
// variants keep more registers than the single-context ones).
struct GroupShapes {
    int pgrid[kTiers][5];             // as StepBuffers::pgrid (index 2 unused)
    int field, bin, n_sm;
};
static GroupShapes g_group_shapes{};

// The group kernels are instantiated for radius kGroupRadius only; their
// launch shapes are the member B0's (the same device: the same occupancy).
cudaError_t launch_passes_group(const StepBuffers& B0, const GroupRef& grp, int which, int tier, const Taps& taps,
                                cudaStream_t s) {
    if (taps.radius != kGroupRadius) return cudaErrorInvalidValue;
    const PassFns fn = pass_fns_r<kGroupRadius, true>(false);
    const int* g = g_group_shapes.pgrid[tier];
    StepBuffers bb = B0;
    GroupRef gr = grp;
    Taps tp = taps;
    PhysicsDev ph{};
    DebugOut db{};
    int tr = tier;
    cudaError_t e;
    if (which == 0) {
        void* a0[] = {&bb, &gr, &tp, &tr};
        e = cudaLaunchKernel(fn.conv_xy[tier], dim3(g[0]), dim3(kConvThreads[tier]), a0,
                             conv_smem_bytes(kTierSide[tier], taps.radius), s);
        if (e != cudaSuccess) return e;
        void* a1[] = {&bb, &gr, &tp, &ph, &tr};
        e = cudaLaunchKernel(fn.conv_z, dim3(g[1]), dim3(kColThreads), a1, 0, s);
    } else {
        void* a3[] = {&bb, &gr, &tr};
        e = cudaLaunchKernel(fn.redist_xy[tier], dim3(g[3]), dim3(kRedistThreads[tier]), a3,
                             redist_smem_bytes(kTierSide[tier]), s);
        if (e != cudaSuccess) return e;
        void* a4[] = {&bb, &gr, &db, &tr};
        e = cudaLaunchKernel(reinterpret_cast<const void*>(p_redist_z<true>), dim3(g[4]), dim3(kColThreads), a4, 0, s);
    }
    if (e != cudaSuccess) return e;
    return cudaGetLastError();
}

cudaError_t configure_group_kernels(int n_sm) {
    const PassFns fn = pass_fns_r<kGroupRadius, true>(false);
    GroupShapes sh{};
    sh.n_sm = n_sm;
    for (int t = 0; t < kTiers; ++t) {
        cudaError_t e = cudaSuccess;
        if (t + 1 < kTiers) {
            e = allow_max_dynamic_smem(fn.conv_xy[t]);
            if (e == cudaSuccess) e = allow_max_dynamic_smem(fn.redist_xy[t]);
        }
        int o[5] = {0, 0, 0, 0, 0};
        if (e == cudaSuccess)
            e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&o[0], fn.conv_xy[t], kConvThreads[t],
                                                              conv_smem_bytes(kTierSide[t], kGroupRadius));
        if (e == cudaSuccess) e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&o[1], fn.conv_z, kColThreads, 0);
        if (e == cudaSuccess)
            e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&o[3], fn.redist_xy[t], kRedistThreads[t],
                                                              redist_smem_bytes(kTierSide[t]));
        if (e == cudaSuccess) e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&o[4], p_redist_z<true>, kColThreads, 0);
        if (e != cudaSuccess) return e;
        for (int k = 0; k < 5; ++k) sh.pgrid[t][k] = n_sm * (o[k] < 1 ? 1 : o[k]);
    }
    int of = 0;
    cudaError_t e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&of, p_field<false, false, true>, kTileX * kTileY, 0);
    if (e != cudaSuccess) return e;
    sh.field = n_sm * (of < 1 ? 1 : of);
    sh.bin = n_sm;
    g_group_shapes = sh;
    return cudaSuccess;
}

cudaError_t launch_bin_group(const StepBuffers& B0, const GroupRef& grp, cudaStream_t s) {
    k_clear_tiles_group<<<g_group_shapes.n_sm, 256, 0, s>>>(grp);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    k_bin<true><<<g_group_shapes.bin, 256, 0, s>>>(B0, grp);
    return cudaGetLastError();
}

cudaError_t launch_field_group(const StepBuffers& B0, const GroupRef& grp, cudaStream_t s) {
    p_field<false, false, true><<<g_group_shapes.field, kTileX * kTileY, 0, s>>>(B0, grp, PhysicsDev{}, DebugOut{});
    return cudaGetLastError();
}

}  // namespace lsgg
