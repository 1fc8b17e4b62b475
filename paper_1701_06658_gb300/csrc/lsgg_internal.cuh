// Internal declarations of the sm_103a level-set grain-growth library.
//
// Data layout in HBM (one context):
//   boxes      Box[G] x 2 tables: `prev` = layout of the state arena X,
//              `cur` = layout the next step writes (bbox of {phi > 0} + halo).
//   X          state arena: phi between steps, `cap` elements of FP32, or of
//              BF16 with LSGG_STORAGE_BF16 (the allocation keeps the FP32
//              size).  Box b's plane z starts at off + z * ps with ps =
//              round_up(nx * ny, 8), so that a plane is one 16-byte aligned bulk
//              copy in either type; off is a multiple of 32.
//   Y          FP32 box arena (same layout): phi_p and the passes' results.
//   T          neighbour-max field, 2 x u64 per domain cell: key1 = the largest
//              (phi_p, -id) over the boxes covering the cell, key2 = the second.
//              Box-streaming kernels build it with 64-bit atomicMax; the pass
//              path computes it per domain tile in registers and stores it.
//   IDF        int32 ID-field arena (same layout as X) for the physics blend.
//   Z          FP32 box arena (same layout) between the passes of the pass
//              path; aliases IDF when the physics needs no ID-field.
//   classes    per size class a work list of box indices and a queue counter
//              per kernel; persistent CTAs pull boxes from the queue.
//   items      pass path: per tier a list of (box, plane), of (box, slab of
//              kSlab planes) and of (box, column chunk) work items, rebuilt by
//              every box update.
#pragma once

#include <cstdint>
#include <cuda_bf16.h>
#include <cuda_runtime.h>

namespace lsgg {

constexpr int kMaxRadius = 7;
constexpr int kMaxTaps = 2 * kMaxRadius + 1;
constexpr int kNumClasses = 5;          // box side <= 32, 40, 48, 64, larger (global scratch)
constexpr int kRedistReach = 6;         // taxicab steps below eps = 7 (exact fixed point)
constexpr int kTiers = 5;               // pass path: boxes with x, y sides <= 32, <= 40, <= 48, <= 64, larger
constexpr int kPassChunk = 256;         // columns per column item of the pass path
constexpr int kSlab = 8;                // planes per slab item of the pass path (default; autotuned)
constexpr int kMinSlab = 4;             // the smallest slab the autotuner tries (sizes the slab item list)
constexpr int kTileX = 8, kTileY = 32, kTileZ = 8;    // domain tiles of the field pass
constexpr int kTileCap = 128;           // boxes listed per tile (more: the tile scans all boxes)

struct Box {
    int ox, oy, oz;       // origin, each in [0, N)
    int nx, ny, nz;       // dims; nx == 0 marks an extinct grain
    long long off;        // arena offset (elements) of plane 0
};

struct Domain {
    int nx, ny, nz;
    int dim;              // 2 or 3
    float eps;
    int halo;
    int radius;
};

struct Taps {
    float g[kMaxTaps];
    int radius;
};

struct Bounds {           // positive-cell bbox in box-local coordinates
    int lo[3];
    int hi[3];
};

// Physics of Eq. (10) for the blend phi_p = phi + w (c - phi) + M (e_j - e_i) dt.
struct PairEntry {        // neighbour j of grain i: weight w_ij and mobility M_ij
    int j;
    float w;
    float m;
};

constexpr int kNbCap = 96;          // neighbour-table entries per grain
constexpr int kPoolKeys = 512;      // pool list entries per box at most (the collection's hash slots)

struct PhysicsDev {
    int kind;                       // LSGG_PHYSICS_*
    const float* energy;            // per grain bulk energy, grid units (MAGNETIC)
    const double* quats;            // per grain unit quaternion (w, x, y, z) (READ_SHOCKLEY)
    const int* pair_map;            // per cell of `cur` the pair's j (the anisotropy map), or null: the
                                    // previous step's ID-field (`prev` layout) gives j
    const int* nb_tab;              // per grain: the first kNbCap ascending ids of the grains in its ID-field
    const int* nb_cnt;              // per grain: entries (kNbCap + 1: more ids than the table holds)
    const float* nb_w;              // per grain and entry: pair weight w (READ_SHOCKLEY, refreshed with nb_tab)
    const float* nb_m;              // per grain and entry: pair mobility M
    // the pass path's complete neighbour lists of a READ_SHOCKLEY run (every
    // grain of a box's ID-field, ascending, up to kPoolKeys), refreshed
    // before each predictor into the pool of the step's parity (steps_done &
    // 1; the other one holds the previous step's lists, whose weights are
    // reused): entry {j, w, M, 0} (w, M as float bits); per box {first
    // entry, count} with count -1 when the list did not fit
    int4* pool_ent[2];              // null: no pool (the z pass looks pairs up per cell)
    int2* pool_box[2];
    int pool_cap;                   // entries per pool
    double theta_max;               // radians
    double mob_low;
    int mob_law;                    // LSGG_MOBILITY_*
    float dt;
};

struct DebugOut {                   // optional per-cell intermediates (cur layout, FP32)
    float* phip;
    float* m;
    int* idm;
    float* phic;
    float* phin;
};

struct StepState {                  // device-resident control block
    int status;                     // 0 or an LSGG_ERR_* code
    int halt;                       // 1: remaining launches of this step return at once
    long long steps_done;
    long long box_cells;            // sum of box volumes in `cur`
    long long alive;
    long long cell_updates;         // box cells advanced by completed steps (sum over steps)
    int class_count[kNumClasses];
    int queue[2][kNumClasses];      // pull counters of the predictor / corrector kernels
    int n_planes[kTiers];           // pass path: work items per tier and their
    int n_chunks[kTiers];           // first entry in the shared item lists
    int plane_base[kTiers];
    int chunk_base[kTiers];
    long long tier_cells[kTiers];   // box cells per tier in `cur`
    int n_slabs[kTiers];            // pass path: slab items (kSlab planes) per tier
    int slab_base[kTiers];
    long long step_limit;           // step groups: the member takes part while steps_done < step_limit
    int bu_go;                      // the step's box update places offsets and items (set by its scan)
    int pool_used;                  // neighbour-list pool entries taken by this step's lists
};

// The step's box update runs as three grid launches over chunks of
// kBuChunk boxes: new boxes and per-chunk sums of kBuVals values, a scan of
// the chunk sums (one CTA per context), then every box's arena offset and
// work-item bases.
constexpr int kBuChunk = 256;
constexpr int kBuVals = 4 + kNumClasses + 4 * kTiers;

__host__ __device__ inline int plane_stride(int nx, int ny) { return (nx * ny + 7) & ~7; }
__host__ __device__ inline long long box_elems(const Box& b) {
    if (b.nx <= 0) return 0;
    long long s = (long long)plane_stride(b.nx, b.ny) * b.nz;
    return (s + 31) & ~31LL;
}
__host__ __device__ inline int pmod(int a, int n) { int r = a % n; return r < 0 ? r + n : r; }

// ---- order-preserving keys for the neighbour-max field ----
__device__ __forceinline__ unsigned int ord_float(float v) {
    unsigned int u = __float_as_uint(v + 0.0f);          // -0 -> +0
    return (u & 0x80000000u) ? ~u : (u | 0x80000000u);
}
__device__ __forceinline__ float unord_float(unsigned int o) {
    unsigned int u = (o & 0x80000000u) ? (o & 0x7fffffffu) : ~o;
    return __uint_as_float(u);
}
__device__ __forceinline__ unsigned long long make_key(float v, int gid) {
    return ((unsigned long long)ord_float(v) << 32) | (unsigned long long)(0xffffffffu - (unsigned)gid);
}
__device__ __forceinline__ int key_id(unsigned long long k) {
    return k ? (int)(0xffffffffu - (unsigned)(k & 0xffffffffu)) : -1;
}
__device__ __forceinline__ float key_val(unsigned long long k, float eps) {
    return k ? unord_float((unsigned)(k >> 32)) : -eps;
}

// ---- launch helpers (implemented in step.cu / init.cu / outputs.cu) ----
struct StepBuffers {
    Domain dom;
    int n_boxes;
    int bf16;                       // X holds BF16 (LSGG_STORAGE_BF16); arithmetic stays FP32
    int redist;                     // LSGG_REDIST_*: TAXICAB by the pass kernels; GODUNOV and HARTMANN
                                    // by Jacobi sweeps over the boxes' columns
    Box* prev;
    Box* cur;
    Bounds* bounds;
    float* X;
    float* Y;
    int* IDF;
    unsigned long long* T;
    int* worklist;                  // kNumClasses x n_boxes
    StepState* st;
    long long cap;
    float* scratch;                 // global ring buffers of the classes in mode 2
    long long scratch_per_cta;
    long long scratch_class_off[kNumClasses];   // each mode-2 class owns a slice (classes run concurrently)
    int n_sm;
    // anisotropy map of Eq. (10)'s pairs (gb_tube > 0): per cell of `cur`, and
    // the map kernel's per-CTA scratch
    float gb_tube;
    int* gb_map;
    void* gb_scratch;
    int gb_grid, gb_cap_cubes, gb_cap_tris;
    int wait_limit;                 // polls of a pass kernel's wait on its bulk copies (test hook lowers it)
    int keep_field;                 // pass path: the field pass also stores the top-two field in T
    int class_side[kNumClasses];    // largest box side per class (last: whole domain)
    int mode[kNumClasses];          // 0: register-ring kernels, 1: shared-memory ring, 2: global scratch ring,
                                    // 3: pass path
    int block[kNumClasses];         // threads per CTA (shared-memory / global rings)
    int fblock[2][kNumClasses];     // threads per CTA of the register-ring kernels
    int variant[2][kNumClasses];    // tile variant of the register-ring kernels (autotuned)
    static constexpr int kVariants = 3;
    int grid[2][kNumClasses];       // persistent grid per kernel and class
    size_t smem[2][kNumClasses];
    // pass path (mode 3 classes): tiers of box side <= tier_side[t]
    float* Z;
    int2* plane_items;              // (box, local z), tier 0 then tier 1
    int2* chunk_items;              // (box, column chunk of kPassChunk columns)
    int2* slab_items;               // (box, first plane of a slab of kSlab planes)
    int4* item_base;                // per box: first plane / chunk / slab item, tier (-1: no items)
    long long plane_item_cap;       // entries (n_boxes * domain nz: a bound on sum nz)
    long long slab_item_cap;        // entries (n_boxes * ceil(domain nz / kSlab))
    long long chunk_item_cap;       // entries (n_boxes * 64 * 64 / kPassChunk)
    int use_passes;
    int tier_side[kTiers];
    int tier_threads[kTiers];       // threads per CTA of the plane passes (= tier side)
    int pgrid[kTiers][5];           // persistent grid per tier and pass (conv_xy, conv_z ideal, conv_z physics, redist_xy, redist_z)
    int pocc[kTiers][5];            // resident CTAs per SM of those kernels (the grids' upper bound)
    int slab;                       // planes per slab item of p_redist_xy (kSlab unless autotuned)
    long long* bu_part;             // box update: per chunk of kBuChunk boxes kBuVals sums, then their bases
    // field pass: boxes overlapping each domain tile of kTileX x kTileY x kTileZ cells
    int* tile_cnt;                  // [n_tiles]
    int* tile_list;                 // [n_tiles * kTileCap]
    int ntile[3];
    int n_tiles;
    int field_grid[2], bin_grid;      // field grid: plain / ID-field and debug variants
};

// A step group: the StepBuffers of several contexts (one GPU, the pass path,
// ideal growth, taxicab re-initialisation), whose steps run as one set of
// launches.  Each work item finds its context through a per-CTA prefix of the
// members' item counts; a member takes part while it is not halted and its
// steps_done is below its step_limit.
constexpr int kMaxGroup = 64;
struct GroupRef {
    const StepBuffers* B;           // device array of n members
    int n;
};

// Element i of the state arena X as FP32, and its store (round to nearest
// even when the arena holds BF16).
__device__ __forceinline__ float ld_state(const StepBuffers& B, long long i) {
    return B.bf16 ? __bfloat162float(reinterpret_cast<const __nv_bfloat16*>(B.X)[i]) : B.X[i];
}
__device__ __forceinline__ void st_state(const StepBuffers& B, long long i, float v) {
    if (B.bf16) reinterpret_cast<__nv_bfloat16*>(B.X)[i] = __float2bfloat16_rn(v);
    else B.X[i] = v;
}
__host__ __device__ inline int state_bytes(const StepBuffers& B) { return B.bf16 ? 2 : 4; }

// Side streams on which the size-class kernels of one phase run concurrently
// (forked from and joined back into the step's stream by events).
struct StepStreams {
    cudaStream_t side[kNumClasses];
    cudaEvent_t fork;
    cudaEvent_t join[kNumClasses];
};

// ev (optional, 5 events): recorded before the field clear, after it, after the
// predictor launches, after the corrector launches and after the box update.
// ss (optional): run each phase's class kernels concurrently on side streams.
// cls_ev (optional, 4 * kNumClasses events): start / end of each class kernel of
// each phase, recorded on the class's stream: [(which * kNumClasses + c) * 2 + {0, 1}].
// pass_ev (optional, 6 * kTiers + 4 events): per tier, around the pass-path kernels:
// [t * 6 + 0..2] p_conv_xy, p_conv_z; [t * 6 + 3..5] p_redist_xy, p_redist_z;
// [6 * kTiers + 0..1] around k_bin, [6 * kTiers + 2..3] around p_field.
cudaError_t launch_step(const StepBuffers& B, const Taps& taps, const PhysicsDev& phys,
                        const DebugOut* dbg, cudaStream_t s, cudaEvent_t* ev = nullptr,
                        const StepStreams* ss = nullptr, cudaEvent_t* cls_ev = nullptr,
                        cudaEvent_t* pass_ev = nullptr);
cudaError_t launch_box_update(const StepBuffers& B, bool commit_only_layout, cudaStream_t s, bool count_step = true);
cudaError_t launch_reinit(const StepBuffers& B, const Taps& taps, const PhysicsDev& phys, bool id_field,
                          cudaStream_t s);
// grid coarsening (coarsen.cu): every alive grain's function on the domain
// `fine` (its box `fine_boxes`, values from the FP32 state in the `prev`
// layout) projected trilinearly into Z in the `cur` layout on B.dom, scaled by
// the spacing ratio and clamped
cudaError_t launch_texture_shares(const double* vol, const int* cls, int G, int n_classes, double* out,
                                  cudaStream_t s);
cudaError_t launch_coarsen(const StepBuffers& B, const Domain& fine, const Box* fine_boxes, const float* state,
                           cudaStream_t s);

// Seeds sorted into a uniform grid of bins (built on the host) for the
// labelling search of the initialisation.
struct SeedBins {
    const float4* pts;     // per sorted seed: x, y, z wrapped into [0, N), weight (FP32)
    const int* ids;        // per sorted seed: its grain id
    const int* start;      // per bin (x fastest): first sorted seed; [n_bins] = G
    int nb[3];             // bins per axis
    float size[3];         // bin side (cells) per axis
    float wmax;            // largest weight (0 without weights)
};
cudaError_t configure_step_kernels(StepBuffers& B);
// Let `fn` take up to the device's opt-in shared memory per CTA (process-wide).
cudaError_t allow_max_dynamic_smem(const void* fn);
cudaError_t configure_passes(StepBuffers& B);
// Whole-arena conversions of the state between BF16 and FP32 (n elements).
cudaError_t launch_state_to_f32(const void* bf16_in, float* out, long long n, cudaStream_t s);
cudaError_t launch_f32_to_state(const float* in, void* bf16_out, long long n, cudaStream_t s);
cudaError_t launch_passes(const StepBuffers& B, int which, int tier, const Taps& taps, const PhysicsDev& phys,
                          const DebugOut& dbg, cudaStream_t s, cudaEvent_t* pass_ev);
cudaError_t launch_bin(const StepBuffers& B, cudaStream_t s);
// Step groups (radius 5 only): the pass kernels of one tier / the binning /
// the field pass over every member of `grp`; B0 (a member) gives the launch
// shapes.  launch_group_step enqueues a whole step.
constexpr int kGroupRadius = 5;
// shared-memory limits and persistent grids of the group kernels on a GPU of n_sm SMs
cudaError_t configure_group_kernels(int n_sm);
cudaError_t launch_passes_group(const StepBuffers& B0, const GroupRef& grp, int which, int tier, const Taps& taps,
                                cudaStream_t s);
cudaError_t launch_bin_group(const StepBuffers& B0, const GroupRef& grp, cudaStream_t s);
cudaError_t launch_field_group(const StepBuffers& B0, const GroupRef& grp, cudaStream_t s);
cudaError_t launch_group_step(const StepBuffers& B0, const GroupRef& grp, const Taps& taps, cudaStream_t s,
                              const StepStreams* ss);
// member k's step limit := lim[k] (device array of grp.n entries)
cudaError_t launch_group_limits(const GroupRef& grp, const long long* lim, cudaStream_t s);
// LSGG_REDIST_GODUNOV: classification, Jacobi sweeps and signs over all boxes;
// LSGG_REDIST_HARTMANN: the constrained reinitialization's pseudo-time steps.
cudaError_t launch_sweep_redist(const StepBuffers& B, const DebugOut& dbg, cudaStream_t s);
cudaError_t launch_field(const StepBuffers& B, const PhysicsDev& phys, const DebugOut& dbg, cudaStream_t s);
// Anisotropy map (gbmap.cu): the step's map into B.gb_map, and the scratch its
// kernel needs for `grid` CTAs.
cudaError_t launch_gb_map_step(const StepBuffers& B, cudaStream_t s);
size_t gb_map_scratch_bytes(int grid, int cap_cubes, int cap_tris);
constexpr int kPassEvents = 6 * kTiers + 4;
// Error tracing (LSGG_TRACE_ERRORS in the environment): `traced` prints a
// failing call's message and `what` on stderr and returns the error.
bool trace_errors();
cudaError_t traced(cudaError_t e, const char* what);
cudaError_t configure_fast_variant(StepBuffers& B, int which, int cls, int variant);
int fast_class_side(int cls);
cudaError_t launch_plain_step(const StepBuffers& B, const Taps& taps, const PhysicsDev& phys,
                              const int* h_alive_boxes, int n_alive, cudaStream_t s);

}  // namespace lsgg
