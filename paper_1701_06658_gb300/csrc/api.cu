// C ABI of the library (declared in include/lsgg.h): context lifecycle, the
// step loop (eager launches or a captured CUDA graph), arena growth, outputs
// and test hooks.  Host code only marshals sizes and pointers; every
// computation on grain data runs in the kernels of step.cu, init.cu,
// outputs.cu and plain.cu.
#include <algorithm>
#include <chrono>
#include <climits>
#include <cmath>
#include <cstdio>
#include <cstdlib>
#include <cstring>
#include <new>
#include <thread>
#include <vector>

#include "bulk_copy.cuh"
#include "lsgg_internal.cuh"
#include "../../include/lsgg.h"

static_assert(lsgg::kTiers == LSGG_PASS_TIERS, "pass-path tiers of the library and of the ABI");

namespace lsgg {
cudaError_t launch_init(const Domain& D, int G, const SeedBins& bins, const double* d_seeds, const double* d_weights, int* d_labels,
                        unsigned* d_bits, long long words_per_row, int* d_bb, Box* d_cur, cudaStream_t s);
cudaError_t launch_label_boxes(const Domain& D, int G, const int* d_labels, unsigned* d_occ, int words, Box* d_cur,
                               cudaStream_t s);
cudaError_t launch_label_phi(const Domain& D, int G, const Box* d_cur, const int* d_labels, float* Z, cudaStream_t s);
cudaError_t launch_sdf(const Domain& D, int G, const Box* d_cur, const double* d_seeds, const double* d_weights,
                       const unsigned* d_bits, long long words_per_row, float* X, int* IDF, int* d_status,
                       cudaStream_t s);
cudaError_t launch_grain_stats(const double* vol, int G, int dim, int n_bins, double r_max, double* out,
                               double* hist, cudaStream_t s);
cudaError_t launch_volumes(const Domain& D, int G, const Box* cur, const Box* prev, const float* X, double* out,
                           cudaStream_t s);
cudaError_t launch_owner(const Domain& D, int G, const Box* cur, const Box* prev, const float* X,
                         unsigned long long* F, int* out, cudaStream_t s);
cudaError_t launch_step_status(const StepState* st, int* out, cudaStream_t s);
cudaError_t launch_pack_state(const Domain& D, int G, const Box* cur, const Box* prev, const float* X,
                              const long long* packed_off, float* out, cudaStream_t s);
cudaError_t launch_pack_cur(int G, const Box* cur, const void* arena, const long long* packed_off, void* out,
                            cudaStream_t s);
cudaError_t launch_unpack_state(int G, const Box* cur, const float* packed, const int* packed_idf,
                                const long long* packed_off, float* X, int* IDF, cudaStream_t s);
long long large_class_scratch_floats(const Domain& d);
cudaError_t launch_field_neighbours(const StepBuffers& B, const Box* boxes, int cap, int* tab, int* cnt,
                                    cudaStream_t s);
cudaError_t launch_plain_step_impl(const StepBuffers& B, const Taps& taps, const PhysicsDev& phys,
                                   const Box* h_cur, const Box* h_prev, float* t1, float* t2, float* Cc,
                                   float* Gg, float* Hh, cudaStream_t s);
}  // namespace lsgg

using namespace lsgg;

struct lsgg_ctx {
    lsgg_config cfg{};
    int device = 0;
    cudaStream_t stream = nullptr;
    bool own_stream = false;
    Domain dom{};
    int G = 0;
    StepBuffers B{};
    Box* d_boxes = nullptr;          // 2 * G: prev then cur
    double* d_seeds = nullptr;
    double* d_weights = nullptr;
    float* d_energy = nullptr;
    double* d_quats = nullptr;
    int* d_nb_tab = nullptr;
    int* d_nb_cnt = nullptr;
    float* d_nb_w = nullptr;
    float* d_nb_m = nullptr;
    double* d_vol = nullptr;
    long long* d_packed_off = nullptr;
    StepState* h_st = nullptr;       // pinned mirror for status reads
    bool field_valid = false;        // T holds the field of the last completed step
    cudaEvent_t join_in = nullptr;   // _device outputs on a caller stream: after the context's work,
    cudaEvent_t join_out = nullptr;  // and the context's later work after them
    long long steps_target = 0;      // steps requested since creation
    double last_dt = 0.0;
    long long device_bytes = 0;
    PhysicsDev phys{};
    // CUDA graph of one step (batched path)
    cudaGraphExec_t graph = nullptr;
    double graph_dt = -1.0;
    std::vector<void*> allocations;
    // kernel timing (lsgg_profile)
    bool profiling = false;
    std::vector<cudaEvent_t> ev_pool;
    std::vector<std::vector<cudaEvent_t>> ev_pending;
    double acc_ms[4] = {0, 0, 0, 0};
    long long acc_cnt[4] = {0, 0, 0, 0};
    double acc_pass_ms[kTiers * 4 + 2] = {};
    long long acc_pass_cnt[kTiers * 4 + 2] = {};
    StepStreams ss{};
    bool have_ss = false;
    bool separate_z = false;         // pass path with an ID-field: Z has its own arena
    // plain (per-grain) comparator buffers
    float *p_t1 = nullptr, *p_t2 = nullptr, *p_C = nullptr, *p_G = nullptr, *p_H = nullptr;
    long long p_cap = 0;
};

namespace lsgg {

// With LSGG_TRACE_ERRORS set in the environment, CUDA failures are reported
// on stderr with the runtime's message and where they were seen.
bool trace_errors() {
    static const bool on = std::getenv("LSGG_TRACE_ERRORS") != nullptr;
    return on;
}

cudaError_t traced(cudaError_t e, const char* what) {
    if (e != cudaSuccess && trace_errors()) std::fprintf(stderr, "lsgg: CUDA error '%s' in %s\n", cudaGetErrorString(e), what);
    return e;
}

}  // namespace lsgg

namespace {


int trace_cuda(cudaError_t e, int line) {
    if (trace_errors()) std::fprintf(stderr, "lsgg: CUDA error '%s' (api.cu:%d)\n", cudaGetErrorString(e), line);
    return LSGG_ERR_CUDA;
}

int fail_cuda(cudaError_t e) { return trace_cuda(e, 0); }

#define CUDA_FAIL() trace_cuda(cudaPeekAtLastError(), __LINE__)

#define CK(call)                                                 \
    do {                                                         \
        cudaError_t e__ = (call);                                \
        if (e__ != cudaSuccess) return trace_cuda(e__, __LINE__); \
    } while (0)

template <class T>
int dalloc(lsgg_ctx* c, T** p, size_t count) {
    void* q = nullptr;
    size_t bytes = count * sizeof(T);
    if (bytes == 0) bytes = 16;
    cudaError_t e = cudaMalloc(&q, bytes);
    if (e != cudaSuccess) {
        cudaGetLastError();
        return e == cudaErrorMemoryAllocation ? LSGG_ERR_OUT_OF_MEMORY : LSGG_ERR_CUDA;
    }
    c->allocations.push_back(q);
    c->device_bytes += (long long)bytes;
    *p = static_cast<T*>(q);
    return LSGG_OK;
}

void dfree(lsgg_ctx* c, void* p) {
    if (!p) return;
    auto it = std::find(c->allocations.begin(), c->allocations.end(), p);
    if (it != c->allocations.end()) c->allocations.erase(it);
    cudaFree(p);
}

uint64_t splitmix_mix(uint64_t z) {
    z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ULL;
    z = (z ^ (z >> 27)) * 0x94D049BB133111EBULL;
    return z ^ (z >> 31);
}
double u01(uint64_t seed, uint64_t stream, uint64_t index) {
    uint64_t k = (stream << 40) + index;
    uint64_t z = seed + (k + 1) * 0x9E3779B97F4A7C15ULL;
    return (double)(splitmix_mix(z) >> 11) * (1.0 / 9007199254740992.0);
}

Taps make_taps(double dt, int R) {
    Taps t{};
    t.radius = R;
    double sum = 0.0, g[kMaxTaps];
    for (int k = -R; k <= R; ++k) {
        g[k + R] = std::exp(-(double)k * k / (4.0 * dt));
        sum += g[k + R];
    }
    for (int k = 0; k < 2 * R + 1; ++k) t.g[k] = (float)(g[k] / sum);
    return t;
}

long long host_box_elems(const Box& b) { return box_elems(b); }

int read_state(lsgg_ctx* c) {
    CK(cudaMemcpyAsync(c->h_st, c->B.st, sizeof(StepState), cudaMemcpyDeviceToHost, c->stream));
    CK(cudaStreamSynchronize(c->stream));
    return LSGG_OK;
}

// Point the pass path's Z arena at `cap` elements: its own arena when the
// physics keeps an ID-field, else the (then unused) ID-field arena.
int replace_z(lsgg_ctx* c, long long cap) {
    if (!c->B.use_passes) return LSGG_OK;
    if (!c->separate_z) { c->B.Z = reinterpret_cast<float*>(c->B.IDF); return LSGG_OK; }
    float* Z2 = nullptr;
    int r = dalloc(c, &Z2, (size_t)cap);
    if (r != LSGG_OK) return r;
    c->device_bytes -= c->B.cap * 4;
    dfree(c, c->B.Z);
    c->B.Z = Z2;
    return LSGG_OK;
}

int ensure_chunk_cap(lsgg_ctx* c);

// The anisotropy map's arena at `cap` elements (its content is rebuilt by
// every step).
int replace_map(lsgg_ctx* c, long long cap) {
    if (!c->B.gb_map) return LSGG_OK;
    int* M2 = nullptr;
    int r = dalloc(c, &M2, (size_t)cap);
    if (r != LSGG_OK) return r;
    c->device_bytes -= c->B.cap * 4;
    dfree(c, c->B.gb_map);
    c->B.gb_map = M2;
    c->phys.pair_map = M2;
    return LSGG_OK;
}

// Grow the arenas to hold `need` elements, keeping the state (prev layout).
int grow_arena(lsgg_ctx* c, long long need) {
    long long cap = std::max<long long>(need + need / 4, c->B.cap * 2);
    float *X2 = nullptr, *Y2 = nullptr;
    int* I2 = nullptr;
    int r;
    if ((r = dalloc(c, &X2, cap)) != LSGG_OK) return r;
    if ((r = dalloc(c, &Y2, cap)) != LSGG_OK) return r;
    if ((r = dalloc(c, &I2, cap)) != LSGG_OK) return r;
    CK(cudaMemcpyAsync(X2, c->B.X, (size_t)c->B.cap * 4, cudaMemcpyDeviceToDevice, c->stream));
    CK(cudaMemcpyAsync(I2, c->B.IDF, (size_t)c->B.cap * 4, cudaMemcpyDeviceToDevice, c->stream));
    CK(cudaStreamSynchronize(c->stream));
    c->device_bytes -= 3 * c->B.cap * 4;
    dfree(c, c->B.X);
    dfree(c, c->B.Y);
    dfree(c, c->B.IDF);
    c->B.X = X2;
    c->B.Y = Y2;
    c->B.IDF = I2;
    r = replace_z(c, cap);
    if (r == LSGG_OK) r = replace_map(c, cap);
    c->B.cap = cap;
    if (r == LSGG_OK) r = ensure_chunk_cap(c);
    if (c->graph) { cudaGraphExecDestroy(c->graph); c->graph = nullptr; }
    return r;
}

// Column-chunk work items of the pass path: a box of plane area A has
// ceil(A / kPassChunk) <= A / kPassChunk + 1 chunks and the plane areas sum to
// at most the box cells, which the arena capacity bounds.  Reallocated (not
// copied: the next box update rebuilds them) when the arena grows.
int ensure_chunk_cap(lsgg_ctx* c) {
    if (!c->B.use_passes) return LSGG_OK;
    const long long need = (long long)c->G + c->B.cap / kPassChunk + 64;
    if (c->B.chunk_items && c->B.chunk_item_cap >= need) return LSGG_OK;
    if (c->B.chunk_items) {
        c->device_bytes -= c->B.chunk_item_cap * (long long)sizeof(int2);
        dfree(c, c->B.chunk_items);
        c->B.chunk_items = nullptr;
    }
    c->B.chunk_item_cap = need;
    return dalloc(c, &c->B.chunk_items, (size_t)need);
}

// The state as FP32: X itself, or (BF16 storage) its conversion into Y,
// which is free between steps.
cudaError_t state_as_f32(lsgg_ctx* c, const float** out, cudaStream_t s = nullptr) {
    if (!c->B.bf16) { *out = c->B.X; return cudaSuccess; }
    *out = c->B.Y;
    return launch_state_to_f32(c->B.X, c->B.Y, c->B.cap, s ? s : c->stream);
}

// Run an output on caller stream s (the context's own when null): s waits for
// the context's enqueued work before, and the context's stream for s after.
cudaError_t join_caller_stream(lsgg_ctx* c, cudaStream_t s, bool after) {
    if (s == c->stream) return cudaSuccess;
    cudaEvent_t& e = after ? c->join_out : c->join_in;
    if (!e) {
        cudaError_t r = cudaEventCreateWithFlags(&e, cudaEventDisableTiming);
        if (r != cudaSuccess) { e = nullptr; return r; }
    }
    cudaStream_t from = after ? s : c->stream, to = after ? c->stream : s;
    cudaError_t r = cudaEventRecord(e, from);
    return r == cudaSuccess ? cudaStreamWaitEvent(to, e, 0) : r;
}

// Assign arena offsets / classes for the `cur` boxes (no resize), growing if needed.
int relayout(lsgg_ctx* c) {
    for (int attempt = 0; attempt < 4; ++attempt) {
        StepState z{};
        // keep steps_done, clear status/halt
        CK(cudaMemcpyAsync(c->h_st, c->B.st, sizeof(StepState), cudaMemcpyDeviceToHost, c->stream));
        CK(cudaStreamSynchronize(c->stream));
        z = *c->h_st;
        z.status = 0;
        z.halt = 0;
        *c->h_st = z;
        CK(cudaMemcpyAsync(c->B.st, c->h_st, sizeof(StepState), cudaMemcpyHostToDevice, c->stream));
        CK(launch_box_update(c->B, true, c->stream));
        int r = read_state(c);
        if (r != LSGG_OK) return r;
        if (c->h_st->status == LSGG_ERR_CAPACITY) {
            r = grow_arena(c, c->h_st->box_cells);
            if (r != LSGG_OK) return r;
            continue;
        }
        return LSGG_OK;
    }
    return LSGG_ERR_OUT_OF_MEMORY;
}

int enqueue_steps(lsgg_ctx* c, long long n, double dt, const DebugOut* dbg);

// Steps leave the neighbour-max field in T: always off the pass path, on it
// while lsgg_keep_field is on.
bool field_stored(const lsgg_ctx* c) { return !c->B.use_passes || c->B.keep_field; }

}  // namespace

extern "C" {

void lsgg_config_default(lsgg_config* cfg) {
    if (!cfg) return;
    std::memset(cfg, 0, sizeof(*cfg));
    cfg->nx = cfg->ny = cfg->nz = 64;
    cfg->n_grains = 50;
    cfg->seed = 1;
    cfg->halo = 5;
    cfg->radius = 5;
    cfg->eps = 7.0f;
    cfg->init_kind = LSGG_INIT_VORONOI;
    cfg->physics = LSGG_PHYSICS_IDEAL;
    cfg->storage = LSGG_STORAGE_FP32;
    cfg->exec = LSGG_EXEC_BATCHED;
    cfg->mobility_law = LSGG_MOBILITY_STEP;
    cfg->theta_max_deg = 15.0;
    cfg->mob_low = 0.1;
    cfg->lognormal_sigma = 0.5;
    cfg->big_fraction = 0.01;
    cfg->big_volume = 5.0;
    cfg->field_dir[0] = 0.0;
    cfg->field_dir[1] = std::cos(32.0 * M_PI / 180.0);
    cfg->field_dir[2] = std::sin(32.0 * M_PI / 180.0);
    cfg->energy_scale = 0.0;
    cfg->arena_slack = 1.5;
}

const char* lsgg_status_string(int s) {
    switch (s) {
        case LSGG_OK: return "ok";
        case LSGG_ERR_INVALID_ARG: return "invalid argument";
        case LSGG_ERR_OUT_OF_MEMORY: return "out of device memory";
        case LSGG_ERR_OVER_BUDGET: return "over the HBM budget";
        case LSGG_ERR_CUDA: return "CUDA error";
        case LSGG_ERR_TIMEOUT: return "timed out";
        case LSGG_ERR_NOT_READY: return "not ready";
        case LSGG_ERR_CAPACITY: return "buffer too small";
        case LSGG_ERR_UNSUPPORTED: return "unsupported";
        default: return "unknown status";
    }
}

void* lsgg_get_stream(lsgg_ctx* c) { return c ? (void*)c->stream : nullptr; }

size_t lsgg_abi_config_size(void) { return sizeof(lsgg_config); }

int lsgg_generate_seeds(uint64_t seed, int32_t n, int32_t nx, int32_t ny, int32_t nz, double* out) {
    if (!out || n <= 0 || nx <= 0 || ny <= 0 || nz <= 0) return LSGG_ERR_INVALID_ARG;
    const double N[3] = {(double)nx, (double)ny, (double)nz};
    for (int i = 0; i < n; ++i)
        for (int a = 0; a < 3; ++a) out[3 * i + a] = u01(seed, 0, 3 * (uint64_t)i + a) * N[a];
    if (nz == 1)
        for (int i = 0; i < n; ++i) out[3 * i + 2] = 0.0;
    return LSGG_OK;
}

int lsgg_destroy(lsgg_ctx* c) {
    if (!c) return LSGG_ERR_INVALID_ARG;
    cudaSetDevice(c->device);
    if (c->stream) cudaStreamSynchronize(c->stream);
    if (c->graph) cudaGraphExecDestroy(c->graph);
    if (c->have_ss) {
        for (int k = 0; k < kNumClasses; ++k) {
            cudaStreamDestroy(c->ss.side[k]);
            cudaEventDestroy(c->ss.join[k]);
        }
        cudaEventDestroy(c->ss.fork);
    }
    for (auto& v : c->ev_pending)
        for (cudaEvent_t e : v) c->ev_pool.push_back(e);
    for (cudaEvent_t e : c->ev_pool) cudaEventDestroy(e);
    if (c->join_in) cudaEventDestroy(c->join_in);
    if (c->join_out) cudaEventDestroy(c->join_out);
    for (void* p : c->allocations) cudaFree(p);
    if (c->h_st) cudaFreeHost(c->h_st);
    if (c->own_stream && c->stream) cudaStreamDestroy(c->stream);
    delete c;
    return LSGG_OK;
}

static int create_impl(const lsgg_config* cfg, void* stream, lsgg_ctx** out);

int lsgg_create_microstructure(const lsgg_config* cfg, void* stream, lsgg_ctx** out) {
    if (!cfg || !out) return LSGG_ERR_INVALID_ARG;
    *out = nullptr;
    int r = create_impl(cfg, stream, out);
    return r;
}

static int validate(const lsgg_config* cfg) {
    if (cfg->nx < 2 || cfg->ny < 2 || cfg->nz < 1) return LSGG_ERR_INVALID_ARG;
    if ((long long)cfg->nx * cfg->ny * cfg->nz > (1LL << 31)) return LSGG_ERR_INVALID_ARG;
    if (cfg->n_grains < 1 || cfg->n_grains > (1 << 24)) return LSGG_ERR_INVALID_ARG;
    if (cfg->halo < 1 || cfg->radius < 1 || cfg->radius > kMaxRadius) return LSGG_ERR_INVALID_ARG;
    if (!(cfg->eps > 1.0f) || cfg->eps > 64.0f) return LSGG_ERR_INVALID_ARG;
    if (cfg->init_kind != LSGG_INIT_VORONOI && cfg->init_kind != LSGG_INIT_LAGUERRE &&
        cfg->init_kind != LSGG_INIT_LABELS)
        return LSGG_ERR_INVALID_ARG;
    if (cfg->init_kind == LSGG_INIT_LABELS) {
        // the label field starts through the pass path's re-initialisation (3D, batched)
        if (!cfg->labels) return LSGG_ERR_INVALID_ARG;
        if (cfg->exec != LSGG_EXEC_BATCHED || cfg->nz == 1) return LSGG_ERR_UNSUPPORTED;
        const long long n = (long long)cfg->nx * cfg->ny * cfg->nz;
        for (long long k = 0; k < n; ++k)
            if (cfg->labels[k] < 0 || cfg->labels[k] >= cfg->n_grains) return LSGG_ERR_INVALID_ARG;
    }
    if (cfg->physics < LSGG_PHYSICS_IDEAL || cfg->physics > LSGG_PHYSICS_MAGNETIC) return LSGG_ERR_INVALID_ARG;
    if (cfg->storage != LSGG_STORAGE_FP32 && cfg->storage != LSGG_STORAGE_BF16) return LSGG_ERR_INVALID_ARG;
    // BF16 state storage: the batched path's kernels (pass path, shared /
    // global-ring box streaming) read and write it; the comparator and the
    // register-ring kernels keep FP32 only
    if (cfg->storage == LSGG_STORAGE_BF16 && cfg->exec != LSGG_EXEC_BATCHED) return LSGG_ERR_UNSUPPORTED;
    if (cfg->redist != LSGG_REDIST_TAXICAB && cfg->redist != LSGG_REDIST_GODUNOV && cfg->redist != LSGG_REDIST_HARTMANN)
        return LSGG_ERR_INVALID_ARG;
    // the Godunov and Hartmann sweeps run on the pass path's column items (3D, batched)
    if (cfg->redist != LSGG_REDIST_TAXICAB && (cfg->exec != LSGG_EXEC_BATCHED || cfg->nz == 1))
        return LSGG_ERR_UNSUPPORTED;
    if (cfg->exec != LSGG_EXEC_BATCHED && cfg->exec != LSGG_EXEC_PLAIN && cfg->exec != LSGG_EXEC_STREAMED)
        return LSGG_ERR_INVALID_ARG;
    if (cfg->physics == LSGG_PHYSICS_READ_SHOCKLEY &&
        (!(cfg->theta_max_deg > 0.0) || !(cfg->mob_low > 0.0) ||
         (cfg->mobility_law != LSGG_MOBILITY_STEP && cfg->mobility_law != LSGG_MOBILITY_EQ20)))
        return LSGG_ERR_INVALID_ARG;
    if (!(cfg->arena_slack >= 1.0)) return LSGG_ERR_INVALID_ARG;
    // the anisotropy map: a tube inside the band, physics that reads pairs,
    // the pass path's z pass
    if (!(cfg->gb_map_tube >= 0.0) || cfg->gb_map_tube >= cfg->eps) return LSGG_ERR_INVALID_ARG;
    if (cfg->gb_map_tube > 0.0 &&
        (cfg->physics == LSGG_PHYSICS_IDEAL || cfg->exec != LSGG_EXEC_BATCHED || cfg->nz == 1))
        return LSGG_ERR_UNSUPPORTED;
    // taxicab reach is fixed to the default band: eps = 7 gives 6 exact steps
    if (std::fabs(cfg->eps - 7.0f) > 1e-6f) return LSGG_ERR_UNSUPPORTED;
    return LSGG_OK;
}

static int create_impl(const lsgg_config* cfg_in, void* stream, lsgg_ctx** out) {
    int r = validate(cfg_in);
    if (r != LSGG_OK) return r;
    int ndev = 0;
    if (cudaGetDeviceCount(&ndev) != cudaSuccess || ndev <= 0) { cudaGetLastError(); return CUDA_FAIL(); }
    if (cfg_in->device < 0 || cfg_in->device >= ndev) return LSGG_ERR_INVALID_ARG;
    lsgg_ctx* c = new (std::nothrow) lsgg_ctx();
    if (!c) return LSGG_ERR_OUT_OF_MEMORY;
    c->cfg = *cfg_in;
    c->cfg.seeds = c->cfg.weights = c->cfg.quats = c->cfg.energy = nullptr;
    c->cfg.labels = nullptr;
    c->device = cfg_in->device;
    auto bail = [&](int code) { lsgg_destroy(c); return code; };
    if (cudaSetDevice(c->device) != cudaSuccess) return bail(CUDA_FAIL());
    if (stream) c->stream = (cudaStream_t)stream;
    else {
        if (cudaStreamCreateWithFlags(&c->stream, cudaStreamNonBlocking) != cudaSuccess) return bail(CUDA_FAIL());
        c->own_stream = true;
    }
    if (cudaMallocHost(&c->h_st, sizeof(StepState)) != cudaSuccess) return bail(LSGG_ERR_OUT_OF_MEMORY);
    std::memset(c->h_st, 0, sizeof(StepState));
    const int G = cfg_in->n_grains;
    c->G = G;
    Domain& D = c->dom;
    D.nx = cfg_in->nx; D.ny = cfg_in->ny; D.nz = cfg_in->nz;
    D.dim = cfg_in->nz == 1 ? 2 : 3;
    D.eps = cfg_in->eps;
    D.halo = cfg_in->halo;
    D.radius = cfg_in->radius;

    // ---- seeds / weights / energies (host marshalling of given or generated inputs) ----
    const bool from_labels = cfg_in->init_kind == LSGG_INIT_LABELS;
    std::vector<double> seeds(3 * (size_t)G), weights, energy;
    if (cfg_in->seeds) std::memcpy(seeds.data(), cfg_in->seeds, seeds.size() * 8);
    else if (!from_labels) lsgg_generate_seeds(cfg_in->seed, G, D.nx, D.ny, D.nz, seeds.data());
    if (cfg_in->init_kind == LSGG_INIT_LAGUERRE) {
        weights.resize(G);
        if (cfg_in->weights) std::memcpy(weights.data(), cfg_in->weights, (size_t)G * 8);
        else {
            // lognormal radii with enlarged grains, weight = radius^2 (same recipe as the inputs module)
            std::vector<double> rad(G);
            double mean = 0.0;
            for (int i = 0; i < G; ++i) {
                double a = u01(cfg_in->seed, 1, 2 * (uint64_t)i), b = u01(cfg_in->seed, 1, 2 * (uint64_t)i + 1);
                double z = std::sqrt(-2.0 * std::log1p(-a)) * std::cos(2.0 * M_PI * b);
                double rr = std::exp(cfg_in->lognormal_sigma * z);
                if (u01(cfg_in->seed, 2, (uint64_t)i) < cfg_in->big_fraction) rr *= std::pow(cfg_in->big_volume, 1.0 / D.dim);
                rad[i] = rr;
                mean += rr;
            }
            mean /= G;
            double spacing = std::pow((double)D.nx * D.ny * D.nz / G, 1.0 / D.dim);
            for (int i = 0; i < G; ++i) { double rr = rad[i] * 0.5 * spacing / mean; weights[i] = rr * rr; }
        }
    }
    std::vector<double> quats;
    if (cfg_in->physics != LSGG_PHYSICS_IDEAL) {
        // unit quaternions: given, or Shoemake's method on SplitMix64 stream 3 (as the inputs module)
        quats.resize(4 * (size_t)G);
        for (int i = 0; i < G; ++i) {
            double* q = quats.data() + 4 * (size_t)i;
            if (cfg_in->quats) std::memcpy(q, cfg_in->quats + 4 * (size_t)i, 32);
            else {
                double a = u01(cfg_in->seed, 3, 3 * (uint64_t)i), b = u01(cfg_in->seed, 3, 3 * (uint64_t)i + 1),
                       cc = u01(cfg_in->seed, 3, 3 * (uint64_t)i + 2);
                double s1 = std::sqrt(1 - a), s2 = std::sqrt(a);
                q[0] = s2 * std::cos(2 * M_PI * cc); q[1] = s1 * std::sin(2 * M_PI * b);
                q[2] = s1 * std::cos(2 * M_PI * b); q[3] = s2 * std::sin(2 * M_PI * cc);
            }
        }
    }
    if (cfg_in->physics == LSGG_PHYSICS_MAGNETIC) {
        energy.resize(G);
        if (cfg_in->energy) std::memcpy(energy.data(), cfg_in->energy, (size_t)G * 8);
        else {
            double f[3] = {cfg_in->field_dir[0], cfg_in->field_dir[1], cfg_in->field_dir[2]};
            double fn = std::sqrt(f[0] * f[0] + f[1] * f[1] + f[2] * f[2]);
            if (!(fn > 0)) return bail(LSGG_ERR_INVALID_ARG);
            for (int i = 0; i < G; ++i) {
                const double* q = quats.data() + 4 * (size_t)i;
                double ax = 2 * (q[1] * q[3] + q[0] * q[2]), ay = 2 * (q[2] * q[3] - q[0] * q[1]),
                       az = 1 - 2 * (q[1] * q[1] + q[2] * q[2]);
                double cs = (ax * f[0] + ay * f[1] + az * f[2]) / fn;
                energy[i] = cfg_in->energy_scale * cs * cs;
            }
        }
    }

    // ---- device allocations for initialisation ----
    const long long ncell = (long long)D.nx * D.ny * D.nz;
    const long long wpr = (G + 31) / 32;
    int* d_labels = nullptr;
    unsigned* d_bits = nullptr;
    int* d_bb = nullptr;
    if ((r = dalloc(c, &c->d_seeds, seeds.size())) != LSGG_OK) return bail(r);
    if (!weights.empty() && (r = dalloc(c, &c->d_weights, weights.size())) != LSGG_OK) return bail(r);
    if ((r = dalloc(c, &c->d_boxes, 2 * (size_t)G)) != LSGG_OK) return bail(r);
    if (cudaMemset(c->d_boxes, 0, 2 * (size_t)G * sizeof(Box)) != cudaSuccess) return bail(CUDA_FAIL());
    if ((r = dalloc(c, &c->B.bounds, (size_t)G)) != LSGG_OK) return bail(r);
    if ((r = dalloc(c, &c->B.st, 1)) != LSGG_OK) return bail(r);
    if ((r = dalloc(c, &c->B.worklist, (size_t)kNumClasses * G)) != LSGG_OK) return bail(r);
    if ((r = dalloc(c, &c->B.bu_part, ((size_t)(G + kBuChunk - 1) / kBuChunk + 1) * kBuVals)) != LSGG_OK)
        return bail(r);
    if ((r = dalloc(c, &c->d_vol, (size_t)G)) != LSGG_OK) return bail(r);
    if ((r = dalloc(c, &c->d_packed_off, (size_t)G + 1)) != LSGG_OK) return bail(r);
    if ((r = dalloc(c, &c->B.T, 2 * (size_t)ncell)) != LSGG_OK) return bail(r);
    if ((r = dalloc(c, &d_labels, (size_t)ncell)) != LSGG_OK) return bail(r);
    if ((r = dalloc(c, &d_bits, (size_t)G * wpr)) != LSGG_OK) return bail(r);
    if ((r = dalloc(c, &d_bb, 6 * (size_t)G)) != LSGG_OK) return bail(r);
    if (!energy.empty()) {
        std::vector<float> ef(energy.begin(), energy.end());
        if ((r = dalloc(c, &c->d_energy, (size_t)G)) != LSGG_OK) return bail(r);
        if (cudaMemcpy(c->d_energy, ef.data(), ef.size() * 4, cudaMemcpyHostToDevice) != cudaSuccess) return bail(CUDA_FAIL());
    }
    if (cfg_in->physics == LSGG_PHYSICS_READ_SHOCKLEY) {
        if ((r = dalloc(c, &c->d_quats, quats.size())) != LSGG_OK) return bail(r);
        if ((r = dalloc(c, &c->d_nb_tab, (size_t)G * kNbCap)) != LSGG_OK) return bail(r);
        if ((r = dalloc(c, &c->d_nb_cnt, (size_t)G)) != LSGG_OK) return bail(r);
        if ((r = dalloc(c, &c->d_nb_w, (size_t)G * kNbCap)) != LSGG_OK) return bail(r);
        if ((r = dalloc(c, &c->d_nb_m, (size_t)G * kNbCap)) != LSGG_OK) return bail(r);
        if (cudaMemcpy(c->d_quats, quats.data(), quats.size() * 8, cudaMemcpyHostToDevice) != cudaSuccess ||
            cudaMemset(c->d_nb_cnt, 0, (size_t)G * 4) != cudaSuccess)
            return bail(CUDA_FAIL());
    }
    if (cudaMemcpy(c->d_seeds, seeds.data(), seeds.size() * 8, cudaMemcpyHostToDevice) != cudaSuccess) return bail(CUDA_FAIL());
    if (!weights.empty() && cudaMemcpy(c->d_weights, weights.data(), weights.size() * 8, cudaMemcpyHostToDevice) != cudaSuccess)
        return bail(CUDA_FAIL());
    if (cudaMemsetAsync(c->B.st, 0, sizeof(StepState), c->stream) != cudaSuccess) return bail(CUDA_FAIL());

    c->B.dom = D;
    c->B.n_boxes = G;
    c->B.prev = c->d_boxes;
    c->B.cur = c->d_boxes + G;
    c->B.use_passes = cfg_in->exec == LSGG_EXEC_BATCHED ? 1 : 0;
    c->B.bf16 = cfg_in->storage == LSGG_STORAGE_BF16 ? 1 : 0;
    c->B.redist = cfg_in->redist;
    c->B.wait_limit = kWaitIters;
    if (configure_step_kernels(c->B) != cudaSuccess) return bail(CUDA_FAIL());
    if (c->B.bf16)
        for (int k = 0; k < kNumClasses; ++k)
            if (c->B.mode[k] == 0) return bail(LSGG_ERR_UNSUPPORTED);   // register-ring kernels are FP32-only
    if (c->B.use_passes) {
        c->B.plane_item_cap = (long long)G * D.nz;
        if ((r = dalloc(c, &c->B.plane_items, (size_t)c->B.plane_item_cap)) != LSGG_OK) return bail(r);
        if ((r = dalloc(c, &c->B.item_base, (size_t)G)) != LSGG_OK) return bail(r);
        c->B.slab_item_cap = (long long)G * ((D.nz + kMinSlab - 1) / kMinSlab);
        if ((r = dalloc(c, &c->B.slab_items, (size_t)c->B.slab_item_cap)) != LSGG_OK) return bail(r);
        if ((r = dalloc(c, &c->B.tile_cnt, (size_t)c->B.n_tiles)) != LSGG_OK) return bail(r);
        if ((r = dalloc(c, &c->B.tile_list, (size_t)c->B.n_tiles * kTileCap)) != LSGG_OK) return bail(r);
    }
    {
        bool ok = cudaEventCreateWithFlags(&c->ss.fork, cudaEventDisableTiming) == cudaSuccess;
        for (int k = 0; k < kNumClasses && ok; ++k)
            ok = cudaStreamCreateWithFlags(&c->ss.side[k], cudaStreamNonBlocking) == cudaSuccess &&
                 cudaEventCreateWithFlags(&c->ss.join[k], cudaEventDisableTiming) == cudaSuccess;
        if (!ok) return bail(CUDA_FAIL());
        c->have_ss = true;
    }

    // seeds binned on a uniform grid of about one seed per bin (labelling search)
    SeedBins bins{};
    long long bin_bytes = 0;
    float4* d_bpts = nullptr;
    int *d_bids = nullptr, *d_bstart = nullptr;
    unsigned* d_occ = nullptr;                   // label field: per grain and axis the positions it holds
    const int occ_words = (std::max(D.nx, std::max(D.ny, D.nz)) + 31) / 32;
    if (!from_labels) {
        const int Ns[3] = {D.nx, D.ny, D.nz};
        const double spacing = std::pow((double)ncell / G, 1.0 / D.dim);
        for (int a = 0; a < 3; ++a) {
            int nb = Ns[a] == 1 ? 1 : (int)(Ns[a] / spacing);
            bins.nb[a] = std::max(1, std::min(Ns[a], nb));
            bins.size[a] = (float)Ns[a] / (float)bins.nb[a];
        }
        const long long n_bins = (long long)bins.nb[0] * bins.nb[1] * bins.nb[2];
        std::vector<int> bin_of(G), start(n_bins + 1, 0), ids(G);
        std::vector<float4> pts(G);
        float wmax = 0.0f;
        for (int i = 0; i < G; ++i) {
            int bc[3];
            float w[3];
            for (int a = 0; a < 3; ++a) {
                const double sw = seeds[3 * (size_t)i + a] - Ns[a] * std::floor(seeds[3 * (size_t)i + a] / Ns[a]);
                w[a] = std::min((float)sw, std::nextafter((float)Ns[a], 0.0f));
                bc[a] = std::min(bins.nb[a] - 1, (int)(w[a] / bins.size[a]));
            }
            const float wt = weights.empty() ? 0.0f : (float)weights[i];
            wmax = std::max(wmax, wt);
            pts[i] = make_float4(w[0], w[1], w[2], wt);
            bin_of[i] = (bc[2] * bins.nb[1] + bc[1]) * bins.nb[0] + bc[0];
            start[bin_of[i] + 1] += 1;
        }
        for (long long b = 0; b < n_bins; ++b) start[b + 1] += start[b];
        std::vector<int> fill(start.begin(), start.end() - 1);
        std::vector<float4> spts(G);
        for (int i = 0; i < G; ++i) {
            const int q = fill[bin_of[i]]++;
            spts[q] = pts[i];
            ids[q] = i;
        }
        bins.wmax = wmax;
        if ((r = dalloc(c, &d_bpts, (size_t)G)) != LSGG_OK) return bail(r);
        if ((r = dalloc(c, &d_bids, (size_t)G)) != LSGG_OK) return bail(r);
        if ((r = dalloc(c, &d_bstart, (size_t)n_bins + 1)) != LSGG_OK) return bail(r);
        if (cudaMemcpy(d_bpts, spts.data(), (size_t)G * sizeof(float4), cudaMemcpyHostToDevice) != cudaSuccess ||
            cudaMemcpy(d_bids, ids.data(), (size_t)G * 4, cudaMemcpyHostToDevice) != cudaSuccess ||
            cudaMemcpy(d_bstart, start.data(), (size_t)(n_bins + 1) * 4, cudaMemcpyHostToDevice) != cudaSuccess)
            return bail(CUDA_FAIL());
        bins.pts = d_bpts;
        bins.ids = d_bids;
        bins.start = d_bstart;
        bin_bytes = (long long)G * (sizeof(float4) + 4) + (n_bins + 1) * 4;
    }
    if (from_labels) {
        // the given labels, every grain's box from the arcs of its cells
        if (cudaMemcpy(d_labels, cfg_in->labels, (size_t)ncell * 4, cudaMemcpyHostToDevice) != cudaSuccess)
            return bail(CUDA_FAIL());
        if ((r = dalloc(c, &d_occ, (size_t)G * 3 * occ_words)) != LSGG_OK) return bail(r);
        if (launch_label_boxes(D, G, d_labels, d_occ, occ_words, c->B.cur, c->stream) != cudaSuccess)
            return bail(CUDA_FAIL());
    } else if (launch_init(D, G, bins, c->d_seeds, c->d_weights, d_labels, d_bits, wpr, d_bb, c->B.cur, c->stream) !=
               cudaSuccess) {
        return bail(CUDA_FAIL());
    }
    // size the arena from the initial boxes
    std::vector<Box> hb(G);
    if (cudaMemcpyAsync(hb.data(), c->B.cur, (size_t)G * sizeof(Box), cudaMemcpyDeviceToHost, c->stream) != cudaSuccess ||
        cudaStreamSynchronize(c->stream) != cudaSuccess)
        return bail(CUDA_FAIL());
    long long need = 0;
    for (const Box& b : hb) need += host_box_elems(b);
    long long cap = (long long)(need * cfg_in->arena_slack) + (1 << 16);
    cap = (cap + 31) & ~31LL;
    c->B.cap = cap;
    if ((r = dalloc(c, &c->B.X, (size_t)cap)) != LSGG_OK) return bail(r);
    if ((r = dalloc(c, &c->B.Y, (size_t)cap)) != LSGG_OK) return bail(r);
    if ((r = dalloc(c, &c->B.IDF, (size_t)cap)) != LSGG_OK) return bail(r);
    c->separate_z = c->B.use_passes && cfg_in->physics != LSGG_PHYSICS_IDEAL;
    if (c->separate_z && (r = dalloc(c, &c->B.Z, (size_t)cap)) != LSGG_OK) return bail(r);
    if (c->B.use_passes && !c->separate_z) c->B.Z = reinterpret_cast<float*>(c->B.IDF);
    if ((r = ensure_chunk_cap(c)) != LSGG_OK) return bail(r);
    if (cfg_in->gb_map_tube > 0.0) {
        // the map per cell (arena layout) and the map kernel's scratch: per CTA
        // the triangles of a box of up to 2^16 cubes (larger boxes rebuild theirs)
        c->B.gb_tube = (float)cfg_in->gb_map_tube;
        c->B.gb_grid = 2 * c->B.n_sm;
        c->B.gb_cap_cubes = 1 << 16;
        c->B.gb_cap_tris = 1 << 14;
        if ((r = dalloc(c, &c->B.gb_map, (size_t)cap)) != LSGG_OK) return bail(r);
        const size_t sb = gb_map_scratch_bytes(c->B.gb_grid, c->B.gb_cap_cubes, c->B.gb_cap_tris);
        unsigned char* sc = nullptr;
        if ((r = dalloc(c, &sc, sb)) != LSGG_OK) return bail(r);
        c->B.gb_scratch = sc;
    }
    c->B.scratch_per_cta = large_class_scratch_floats(D);
    {
        long long total = 0;
        for (int k = 0; k < kNumClasses; ++k) {
            c->B.scratch_class_off[k] = total;
            if (c->B.mode[k] == 2)
                total += c->B.scratch_per_cta * std::max(c->B.grid[0][k], c->B.grid[1][k]);
        }
        if ((r = dalloc(c, &c->B.scratch, (size_t)std::max(total, 32LL))) != LSGG_OK) return bail(r);
    }
    if ((r = relayout(c)) != LSGG_OK) return bail(r);
    c->phys.kind = cfg_in->physics;
    c->phys.energy = c->d_energy;
    c->phys.quats = c->d_quats;
    c->phys.nb_tab = c->d_nb_tab;
    c->phys.nb_cnt = c->d_nb_cnt;
    c->phys.nb_w = c->d_nb_w;
    c->phys.nb_m = c->d_nb_m;
    c->phys.theta_max = cfg_in->theta_max_deg * M_PI / 180.0;
    c->phys.mob_low = cfg_in->mob_low;
    c->phys.mob_law = cfg_in->mobility_law;
    c->phys.pair_map = c->B.gb_map;
    if (cfg_in->physics == LSGG_PHYSICS_READ_SHOCKLEY && c->B.use_passes && !c->B.gb_map) {
        // the pass path's neighbour-list pool: about 64 pairs per grain (a
        // box that finds no room looks its pairs up per cell)
        const long long cap = std::min(std::max(64LL * G, 4096LL), (long long)INT_MAX / 2);
        for (int k = 0; k < 2; ++k) {
            if ((r = dalloc(c, &c->phys.pool_ent[k], (size_t)cap)) != LSGG_OK) return bail(r);
            if ((r = dalloc(c, &c->phys.pool_box[k], (size_t)G)) != LSGG_OK) return bail(r);
            if (cudaMemset(c->phys.pool_box[k], 0, (size_t)G * sizeof(int2)) != cudaSuccess) return bail(CUDA_FAIL());
        }
        c->phys.pool_cap = (int)cap;
    }
    if (from_labels) {
        // +-1/2 by membership, then the step's re-initialisation and box
        // update (with physics the field pass of the result gives the
        // ID-field the first step reads)
        if (launch_label_phi(D, G, c->B.cur, d_labels, c->B.Z, c->stream) != cudaSuccess ||
            launch_reinit(c->B, make_taps(1.0, D.radius), c->phys, cfg_in->physics != LSGG_PHYSICS_IDEAL,
                          c->stream) != cudaSuccess)
            return bail(CUDA_FAIL());
    } else {
        if (launch_sdf(D, G, c->B.cur, c->d_seeds, c->d_weights, d_bits, wpr, c->B.bf16 ? c->B.Y : c->B.X,
                       c->B.IDF, &c->B.st->status, c->stream) != cudaSuccess)
            return bail(CUDA_FAIL());
        if (c->B.bf16 && launch_f32_to_state(c->B.Y, c->B.X, c->B.cap, c->stream) != cudaSuccess)
            return bail(CUDA_FAIL());
        if (cudaMemcpyAsync(c->B.prev, c->B.cur, (size_t)G * sizeof(Box), cudaMemcpyDeviceToDevice, c->stream) !=
            cudaSuccess)
            return bail(CUDA_FAIL());
    }
    if ((r = read_state(c)) != LSGG_OK) return bail(r);
    if (c->h_st->status != 0) return bail(c->h_st->status);
    if (d_occ) {
        dfree(c, d_occ);
        c->device_bytes -= (long long)G * 3 * occ_words * 4;
    }
    dfree(c, d_labels);
    dfree(c, d_bits);
    dfree(c, d_bb);
    dfree(c, d_bpts);
    dfree(c, d_bids);
    dfree(c, d_bstart);
    c->device_bytes -= (long long)ncell * 4 + (long long)G * wpr * 4 + 6LL * G * 4 + bin_bytes;
    *out = c;
    return LSGG_OK;
}

int lsgg_step(lsgg_ctx* c, int32_t n, double dt) {
    if (!c || n < 0 || !(dt > 0.0) || dt > 4.0) return LSGG_ERR_INVALID_ARG;
    if (n == 0) return LSGG_OK;
    if (cudaSetDevice(c->device) != cudaSuccess) return CUDA_FAIL();
    c->steps_target += n;
    c->last_dt = dt;
    c->field_valid = field_stored(c);
    return enqueue_steps(c, n, dt, nullptr);
}

int lsgg_sync(lsgg_ctx* c, int64_t timeout_ms) {
    if (!c) return LSGG_ERR_INVALID_ARG;
    if (cudaSetDevice(c->device) != cudaSuccess) return CUDA_FAIL();
    for (int round = 0; round < 64; ++round) {
        auto t0 = std::chrono::steady_clock::now();
        if (timeout_ms < 0) {
            // no limit: a blocking wait returns as soon as the stream drains
            if (cudaStreamSynchronize(c->stream) != cudaSuccess) return CUDA_FAIL();
        }
        for (;;) {
            cudaError_t q = cudaStreamQuery(c->stream);
            if (q == cudaSuccess) break;
            if (q != cudaErrorNotReady) return CUDA_FAIL();
            if (timeout_ms >= 0) {
                auto ms = std::chrono::duration_cast<std::chrono::milliseconds>(std::chrono::steady_clock::now() - t0).count();
                if (ms > timeout_ms) return LSGG_ERR_TIMEOUT;
            }
            std::this_thread::sleep_for(std::chrono::microseconds(50));
        }
        int r = read_state(c);
        if (r != LSGG_OK) return r;
        if (c->h_st->status == 0) return LSGG_OK;
        if (c->h_st->status != LSGG_ERR_CAPACITY) {
            // a device-side failure (an expired wait, a refused launch): report it
            // once, clear it and drop the steps that did not complete
            const int st = c->h_st->status;
            if (cudaMemsetAsync(&c->B.st->status, 0, 2 * sizeof(int), c->stream) != cudaSuccess ||
                cudaStreamSynchronize(c->stream) != cudaSuccess)
                return CUDA_FAIL();
            c->steps_target = c->h_st->steps_done;
            return st;
        }
        // arena overflow: grow, lay out the pending boxes, finish the remaining steps
        r = grow_arena(c, c->h_st->box_cells);
        if (r != LSGG_OK) return r;
        r = relayout(c);
        if (r != LSGG_OK) return r;
        long long remaining = c->steps_target - c->h_st->steps_done;
        if (remaining > 0) {
            r = enqueue_steps(c, remaining, c->last_dt, nullptr);
            if (r != LSGG_OK) return r;
        }
    }
    return LSGG_ERR_OUT_OF_MEMORY;
}

}  // extern "C"

static_assert(LSGG_MAX_GROUP == kMaxGroup, "group size of the library and of the ABI");

struct lsgg_group {
    std::vector<lsgg_ctx*> m;
    int device = 0;
    cudaStream_t stream = nullptr;
    StepStreams ss{};
    bool have_ss = false;
    StepBuffers* d_B = nullptr;          // members' StepBuffers (device copy)
    long long* d_lim = nullptr;          // members' step limits
    std::vector<unsigned char> h_B;      // the members' StepBuffers bytes last sent
    std::vector<long long> h_lim;
    cudaEvent_t done = nullptr;          // after the group's latest steps
    std::vector<cudaEvent_t> ready;      // per member: after its enqueued work
    cudaGraphExec_t graph = nullptr;
    double graph_dt = -1.0;
};

namespace {

void group_free(lsgg_group* g) {
    if (g->stream) cudaStreamSynchronize(g->stream);
    if (g->graph) cudaGraphExecDestroy(g->graph);
    if (g->have_ss) {
        for (int k = 0; k < kNumClasses; ++k) {
            cudaStreamDestroy(g->ss.side[k]);
            cudaEventDestroy(g->ss.join[k]);
        }
        cudaEventDestroy(g->ss.fork);
    }
    for (cudaEvent_t e : g->ready) cudaEventDestroy(e);
    if (g->done) cudaEventDestroy(g->done);
    if (g->d_B) cudaFree(g->d_B);
    if (g->d_lim) cudaFree(g->d_lim);
    if (g->stream) cudaStreamDestroy(g->stream);
    delete g;
}

// One group step captured as a graph on the group's stream (the kernels read
// the members' buffers from the device array, so the graph stays valid while
// only their contents change).
int group_graph(lsgg_group* g, double dt, bool stale) {
    if (g->graph && g->graph_dt == dt && !stale) return LSGG_OK;
    const Taps taps = make_taps(dt, kGroupRadius);
    const GroupRef grp{g->d_B, (int)g->m.size()};
    cudaGraph_t graph = nullptr;
    CK(cudaStreamBeginCapture(g->stream, cudaStreamCaptureModeThreadLocal));
    cudaError_t e = launch_group_step(g->m[0]->B, grp, taps, g->stream, &g->ss);
    cudaError_t e2 = cudaStreamEndCapture(g->stream, &graph);
    if (e != cudaSuccess || e2 != cudaSuccess) {
        if (graph) cudaGraphDestroy(graph);
        return fail_cuda(e != cudaSuccess ? e : e2);
    }
    // the same launches with other parameters (member count, taps, shapes):
    // update the executable graph in place, else instantiate anew
    if (g->graph) {
        cudaGraphExecUpdateResultInfo info{};
        if (cudaGraphExecUpdate(g->graph, graph, &info) != cudaSuccess) {
            cudaGetLastError();
            cudaGraphExecDestroy(g->graph);
            g->graph = nullptr;
        }
    }
    if (!g->graph) {
        e = cudaGraphInstantiate(&g->graph, graph, 0);
        if (e != cudaSuccess) { cudaGraphDestroy(graph); g->graph = nullptr; return fail_cuda(e); }
    }
    cudaGraphDestroy(graph);
    g->graph_dt = dt;
    return LSGG_OK;
}

}  // namespace

extern "C" {

// lsgg_group_create's rules for a member list.
static int check_members(lsgg_ctx* const* members, int32_t n) {
    if (!members || n < 1 || n > kMaxGroup) return LSGG_ERR_INVALID_ARG;
    for (int k = 0; k < n; ++k) {
        lsgg_ctx* c = members[k];
        if (!c) return LSGG_ERR_INVALID_ARG;
        for (int j = 0; j < k; ++j)
            if (members[j] == c) return LSGG_ERR_INVALID_ARG;
    }
    for (int k = 0; k < n; ++k) {
        lsgg_ctx* c = members[k];
        if (c->device != members[0]->device || !c->B.use_passes || c->dom.dim != 3 ||
            c->cfg.physics != LSGG_PHYSICS_IDEAL || c->B.redist != LSGG_REDIST_TAXICAB ||
            c->dom.radius != kGroupRadius || c->B.gb_map || c->profiling)
            return LSGG_ERR_UNSUPPORTED;
    }
    return LSGG_OK;
}

int lsgg_group_create(lsgg_ctx* const* members, int32_t n, lsgg_group** out) {
    if (!out) return LSGG_ERR_INVALID_ARG;
    *out = nullptr;
    const int chk = check_members(members, n);
    if (chk != LSGG_OK) return chk;
    lsgg_group* g = new (std::nothrow) lsgg_group();
    if (!g) return LSGG_ERR_OUT_OF_MEMORY;
    g->m.assign(members, members + n);
    g->device = members[0]->device;
    auto bail = [&](int code) { group_free(g); return code; };
    if (cudaSetDevice(g->device) != cudaSuccess) return bail(CUDA_FAIL());
    if (configure_group_kernels(members[0]->B.n_sm) != cudaSuccess) return bail(CUDA_FAIL());
    if (cudaStreamCreateWithFlags(&g->stream, cudaStreamNonBlocking) != cudaSuccess) return bail(CUDA_FAIL());
    bool ok = cudaEventCreateWithFlags(&g->ss.fork, cudaEventDisableTiming) == cudaSuccess;
    for (int k = 0; k < kNumClasses && ok; ++k)
        ok = cudaStreamCreateWithFlags(&g->ss.side[k], cudaStreamNonBlocking) == cudaSuccess &&
             cudaEventCreateWithFlags(&g->ss.join[k], cudaEventDisableTiming) == cudaSuccess;
    if (!ok) return bail(CUDA_FAIL());
    g->have_ss = true;
    if (cudaEventCreateWithFlags(&g->done, cudaEventDisableTiming) != cudaSuccess) return bail(CUDA_FAIL());
    g->ready.resize(kMaxGroup, nullptr);
    for (int k = 0; k < kMaxGroup; ++k)
        if (cudaEventCreateWithFlags(&g->ready[k], cudaEventDisableTiming) != cudaSuccess) return bail(CUDA_FAIL());
    if (cudaMalloc(&g->d_B, sizeof(StepBuffers) * kMaxGroup) != cudaSuccess ||
        cudaMalloc(&g->d_lim, sizeof(long long) * kMaxGroup) != cudaSuccess) {
        cudaGetLastError();
        return bail(LSGG_ERR_OUT_OF_MEMORY);
    }
    *out = g;
    return LSGG_OK;
}

int lsgg_group_step(lsgg_group* g, int32_t n, double dt, const int64_t* step_limits) {
    if (!g || n < 0 || !(dt > 0.0) || dt > 4.0) return LSGG_ERR_INVALID_ARG;
    if (n == 0) return LSGG_OK;
    if (cudaSetDevice(g->device) != cudaSuccess) return CUDA_FAIL();
    const int nm = (int)g->m.size();
    // the members' buffers as they are now (an arena may have grown since),
    // compared byte for byte with the copy on the device
    std::vector<unsigned char> now(sizeof(StepBuffers) * nm);
    for (int k = 0; k < nm; ++k) std::memcpy(now.data() + sizeof(StepBuffers) * k, &g->m[k]->B, sizeof(StepBuffers));
    const bool fresh = now != g->h_B;
    std::vector<long long> lim(nm);
    for (int k = 0; k < nm; ++k) lim[k] = step_limits ? (long long)step_limits[k] : LLONG_MAX;
    // every member's enqueued work first
    for (int k = 0; k < nm; ++k) {
        CK(cudaEventRecord(g->ready[k], g->m[k]->stream));
        CK(cudaStreamWaitEvent(g->stream, g->ready[k], 0));
    }
    if (fresh) {
        g->h_B.swap(now);
        CK(cudaMemcpyAsync(g->d_B, g->h_B.data(), sizeof(StepBuffers) * nm, cudaMemcpyHostToDevice, g->stream));
    }
    if (lim != g->h_lim) {
        g->h_lim = lim;
        CK(cudaMemcpyAsync(g->d_lim, g->h_lim.data(), sizeof(long long) * nm, cudaMemcpyHostToDevice, g->stream));
    }
    CK(launch_group_limits(GroupRef{g->d_B, nm}, g->d_lim, g->stream));
    int r = group_graph(g, dt, fresh);       // member count and launch shapes may have changed
    if (r != LSGG_OK) return r;
    for (int i = 0; i < n; ++i) CK(cudaGraphLaunch(g->graph, g->stream));
    CK(cudaEventRecord(g->done, g->stream));
    for (int k = 0; k < nm; ++k) {
        lsgg_ctx* c = g->m[k];
        CK(cudaStreamWaitEvent(c->stream, g->done, 0));
        long long target = c->steps_target + n;
        if (step_limits) target = std::min(target, std::max(c->steps_target, (long long)step_limits[k]));
        c->steps_target = target;
        c->last_dt = dt;
        c->field_valid = field_stored(c);
    }
    return LSGG_OK;
}

int lsgg_group_set_members(lsgg_group* g, lsgg_ctx* const* members, int32_t n) {
    if (!g) return LSGG_ERR_INVALID_ARG;
    const int chk = check_members(members, n);
    if (chk != LSGG_OK) return chk;
    if (members[0]->device != g->device) return LSGG_ERR_UNSUPPORTED;
    g->m.assign(members, members + n);
    return LSGG_OK;     // the next step sends the new buffers and updates the graph
}

int lsgg_group_destroy(lsgg_group* g) {
    if (!g) return LSGG_ERR_INVALID_ARG;
    cudaSetDevice(g->device);
    group_free(g);
    return LSGG_OK;
}

int lsgg_get_stats(lsgg_ctx* c, lsgg_stats* out) {
    if (!c || !out) return LSGG_ERR_INVALID_ARG;
    int r = lsgg_sync(c, -1);
    if (r != LSGG_OK) return r;
    std::memset(out, 0, sizeof(*out));
    out->steps_done = c->h_st->steps_done;
    out->cell_updates = c->h_st->cell_updates;
    out->alive = c->h_st->alive;
    out->box_cells = c->h_st->box_cells;
    out->arena_capacity = c->B.cap;
    out->superimposition = (double)c->h_st->box_cells / ((double)c->dom.nx * c->dom.ny * c->dom.nz);
    out->device_bytes = c->device_bytes;
    out->n_classes = kNumClasses;
    for (int k = 0; k < kNumClasses; ++k) out->class_count[k] = c->h_st->class_count[k];
    for (int t = 0; t < kTiers; ++t) out->pass_cells[t] = c->B.use_passes ? c->h_st->tier_cells[t] : 0;
    return LSGG_OK;
}

// The pass path's tunables: per tier and pass the CTAs per SM of its
// persistent grid (pgrid index 0 conv_xy, 1 / 2 conv_z ideal / physics, 3
// redist_xy, 4 redist_z) and the slab depth of p_redist_xy.  Re-lays the work
// items out for the slab; the step graph is captured anew.
static int apply_pass_tuning(lsgg_ctx* c, const int (&ctas)[kTiers][5], int slab) {
    for (int t = 0; t < kTiers; ++t)
        for (int k = 0; k < 5; ++k) c->B.pgrid[t][k] = c->B.n_sm * std::max(1, std::min(ctas[t][k], c->B.pocc[t][k]));
    c->B.slab = slab;
    if (c->graph) { cudaGraphExecDestroy(c->graph); c->graph = nullptr; }
    return relayout(c);
}

// Autotuner of the pass path: trials of steps_per_trial profiled steps each
// with (a) every grid at its resident maximum and the default slab, (b) every
// grid at half of it, (c, d) slabs of 4 and 16 planes; per tier and pass the
// faster grid of (a, b), and the slab with the least re-initialisation
// plane-pass time over the tiers.  All settings give bit-identical steps.
static int autotune_passes(lsgg_ctx* c, int32_t steps_per_trial, double dt) {
    int full[kTiers][5], half[kTiers][5];
    for (int t = 0; t < kTiers; ++t)
        for (int k = 0; k < 5; ++k) { full[t][k] = c->B.pocc[t][k]; half[t][k] = std::max(1, c->B.pocc[t][k] / 2); }
    const int slabs[4] = {kSlab, kSlab, kMinSlab, 2 * kSlab};
    double ms[4][kTiers * 4 + 2] = {};
    c->profiling = true;
    for (int trial = 0; trial < 4; ++trial) {
        int r = apply_pass_tuning(c, trial == 1 ? half : full, slabs[trial]);
        if (r == LSGG_OK) r = lsgg_step(c, steps_per_trial, dt);
        if (r == LSGG_OK) r = lsgg_pass_times(c, ms[trial], nullptr);
        if (r != LSGG_OK) { c->profiling = false; return r; }
    }
    c->profiling = false;
    // pass index of lsgg_pass_times (conv_xy, conv_z, redist_xy, redist_z) -> pgrid index
    const int pk[4][2] = {{0, 0}, {1, 2}, {3, 3}, {4, 4}};
    int best[kTiers][5];
    for (int t = 0; t < kTiers; ++t)
        for (int q = 0; q < 4; ++q)
            for (int j = 0; j < 2; ++j) {
                const int k = pk[q][j];
                best[t][k] = ms[1][t * 4 + q] < ms[0][t * 4 + q] ? half[t][k] : full[t][k];
            }
    int slab = kSlab;
    double slab_ms = 0.0;
    for (int trial : {0, 2, 3}) {
        double tot = 0.0;
        for (int t = 0; t < kTiers; ++t) tot += ms[trial][t * 4 + 2];
        if (trial == 0 || tot < slab_ms) { slab_ms = tot; slab = slabs[trial]; }
    }
    return apply_pass_tuning(c, best, slab);
}

int lsgg_pass_tuning(lsgg_ctx* c, int32_t* ctas_per_sm, int32_t* slab) {
    if (!c) return LSGG_ERR_INVALID_ARG;
    if (ctas_per_sm)
        for (int t = 0; t < kTiers; ++t) {
            const int k4[4] = {0, c->phys.kind != LSGG_PHYSICS_IDEAL ? 2 : 1, 3, 4};
            for (int q = 0; q < 4; ++q) ctas_per_sm[t * 4 + q] = c->B.use_passes ? c->B.pgrid[t][k4[q]] / c->B.n_sm : -1;
        }
    if (slab) *slab = c->B.use_passes ? c->B.slab : -1;
    return LSGG_OK;
}

int lsgg_autotune(lsgg_ctx* c, int32_t steps_per_trial, double dt, int32_t* chosen) {
    if (!c || steps_per_trial < 1 || !(dt > 0.0) || dt > 4.0) return LSGG_ERR_INVALID_ARG;
    int r = lsgg_sync(c, -1);
    if (r != LSGG_OK) return r;
    if (c->B.use_passes) {
        if (chosen)
            for (int k = 0; k < 2 * kNumClasses; ++k) chosen[k] = -1;
        r = autotune_passes(c, steps_per_trial, dt);
        c->field_valid = field_stored(c);
        c->last_dt = dt;
        return r;
    }
    if (cudaSetDevice(c->device) != cudaSuccess) return CUDA_FAIL();
    const int nv = StepBuffers::kVariants;
    const int ne = 4 * kNumClasses;
    std::vector<cudaEvent_t> ev((size_t)ne * steps_per_trial);
    for (auto& e : ev)
        if (cudaEventCreate(&e) != cudaSuccess) return CUDA_FAIL();
    double best_ms[2][kNumClasses];
    int best_v[2][kNumClasses];
    for (int w = 0; w < 2; ++w)
        for (int k = 0; k < kNumClasses; ++k) { best_ms[w][k] = 1e300; best_v[w][k] = c->B.variant[w][k]; }
    Taps taps = make_taps(dt, c->dom.radius);
    c->phys.dt = (float)dt;
    int status = LSGG_OK;
    for (int v = 0; v < nv && status == LSGG_OK; ++v) {
        for (int w = 0; w < 2; ++w)
            for (int k = 0; k < kNumClasses; ++k)
                if (c->B.mode[k] == 0 && configure_fast_variant(c->B, w, k, v) != cudaSuccess) status = LSGG_ERR_CUDA;
        if (status != LSGG_OK) break;
        for (int sidx = 0; sidx < steps_per_trial; ++sidx) {
            c->steps_target += 1;
            if (launch_step(c->B, taps, c->phys, nullptr, c->stream, nullptr, &c->ss, ev.data() + (size_t)sidx * ne) !=
                cudaSuccess) { status = LSGG_ERR_CUDA; break; }
        }
        if (status != LSGG_OK) break;
        status = lsgg_sync(c, -1);
        if (status != LSGG_OK) break;
        for (int w = 0; w < 2; ++w)
            for (int k = 0; k < kNumClasses; ++k) {
                if (c->B.mode[k] != 0) continue;
                double tot = 0.0;
                for (int sidx = 0; sidx < steps_per_trial; ++sidx) {
                    float ms = 0.0f;
                    cudaEvent_t* e = ev.data() + (size_t)sidx * ne + (w * kNumClasses + k) * 2;
                    if (cudaEventElapsedTime(&ms, e[0], e[1]) == cudaSuccess) tot += ms;
                }
                if (tot < best_ms[w][k]) { best_ms[w][k] = tot; best_v[w][k] = v; }
            }
    }
    for (auto& e : ev) cudaEventDestroy(e);
    for (int w = 0; w < 2; ++w)
        for (int k = 0; k < kNumClasses; ++k) {
            if (c->B.mode[k] == 0 && configure_fast_variant(c->B, w, k, best_v[w][k]) != cudaSuccess) status = LSGG_ERR_CUDA;
            if (chosen) chosen[w * kNumClasses + k] = c->B.mode[k] == 0 ? best_v[w][k] : -1;
        }
    if (c->graph) { cudaGraphExecDestroy(c->graph); c->graph = nullptr; }
    c->field_valid = field_stored(c);
    c->last_dt = dt;
    return status;
}

int lsgg_profile(lsgg_ctx* c, int32_t enable) {
    if (!c) return LSGG_ERR_INVALID_ARG;
    c->profiling = enable != 0;
    return LSGG_OK;
}

}  // extern "C"

namespace {

// Fold the events of the profiled steps into the per-group and per-pass sums.
int drain_profile_events(lsgg_ctx* c) {
    int n_other = 0;
    for (int k = 0; k < kNumClasses; ++k) n_other += c->B.mode[k] != 3;
    const bool plain = c->cfg.exec == LSGG_EXEC_PLAIN;
    const long long passes = c->B.use_passes ? kTiers : 0;
    const long long per_step[4] = {passes ? 1 : 0, plain ? kNumClasses : n_other + 2 * passes + (passes ? 1 : 0),
                                   plain ? kNumClasses : n_other + 2 * passes, 1};
    for (auto& v : c->ev_pending) {
        for (int g = 0; g < 4; ++g) {
            float ms = 0.0f;
            if (cudaEventElapsedTime(&ms, v[g], v[g + 1]) != cudaSuccess) return CUDA_FAIL();
            c->acc_ms[g] += ms;
            c->acc_cnt[g] += per_step[g];
        }
        if (v.size() == 5 + (size_t)kPassEvents) {
            const cudaEvent_t* pe = v.data() + 5;
            auto add = [&](int slot, int e0, int e1) -> bool {
                float ms = 0.0f;
                if (cudaEventElapsedTime(&ms, pe[e0], pe[e1]) != cudaSuccess) return false;
                c->acc_pass_ms[slot] += ms;
                c->acc_pass_cnt[slot] += 1;
                return true;
            };
            bool ok = true;
            for (int t = 0; t < kTiers; ++t) {
                const int seg[4][2] = {{0, 1}, {1, 2}, {3, 4}, {4, 5}};
                for (int k = 0; k < 4; ++k) ok = ok && add(t * 4 + k, t * 6 + seg[k][0], t * 6 + seg[k][1]);
            }
            ok = ok && add(kTiers * 4, 6 * kTiers, 6 * kTiers + 1) && add(kTiers * 4 + 1, 6 * kTiers + 2, 6 * kTiers + 3);
            if (!ok) return CUDA_FAIL();
        }
        for (cudaEvent_t e : v) c->ev_pool.push_back(e);
    }
    c->ev_pending.clear();
    return LSGG_OK;
}

}  // namespace

extern "C" {

int lsgg_kernel_times(lsgg_ctx* c, double* out_ms, int64_t* out_count) {
    if (!c) return LSGG_ERR_INVALID_ARG;
    int r = lsgg_sync(c, -1);
    if (r != LSGG_OK) return r;
    if ((r = drain_profile_events(c)) != LSGG_OK) return r;
    for (int g = 0; g < 4; ++g) {
        if (out_ms) out_ms[g] = c->acc_ms[g];
        if (out_count) out_count[g] = c->acc_cnt[g];
        c->acc_ms[g] = 0.0;
        c->acc_cnt[g] = 0;
    }
    return LSGG_OK;
}

int lsgg_pass_times(lsgg_ctx* c, double* out_ms, int64_t* out_count) {
    if (!c) return LSGG_ERR_INVALID_ARG;
    int r = lsgg_sync(c, -1);
    if (r != LSGG_OK) return r;
    if ((r = drain_profile_events(c)) != LSGG_OK) return r;
    for (int g = 0; g < kTiers * 4 + 2; ++g) {
        if (out_ms) out_ms[g] = c->acc_pass_ms[g];
        if (out_count) out_count[g] = c->acc_pass_cnt[g];
        c->acc_pass_ms[g] = 0.0;
        c->acc_pass_cnt[g] = 0;
    }
    return LSGG_OK;
}

int lsgg_debug_set_capacity(lsgg_ctx* c, int64_t capacity) {
    if (!c) return LSGG_ERR_INVALID_ARG;
    int r = lsgg_sync(c, -1);
    if (r != LSGG_OK) return r;
    std::vector<Box> hp(c->G), hc(c->G);
    CK(cudaMemcpy(hp.data(), c->B.prev, (size_t)c->G * sizeof(Box), cudaMemcpyDeviceToHost));
    CK(cudaMemcpy(hc.data(), c->B.cur, (size_t)c->G * sizeof(Box), cudaMemcpyDeviceToHost));
    long long need_prev = 0, need_cur = 0;
    for (int i = 0; i < c->G; ++i) {
        need_prev = std::max(need_prev, hp[i].nx > 0 ? hp[i].off + host_box_elems(hp[i]) : 0);
        need_cur += host_box_elems(hc[i]);
    }
    capacity = (capacity + 31) & ~31LL;
    if (capacity < need_prev || capacity < need_cur) return LSGG_ERR_INVALID_ARG;
    float *X2 = nullptr, *Y2 = nullptr;
    int* I2 = nullptr;
    if ((r = dalloc(c, &X2, (size_t)capacity)) != LSGG_OK) return r;
    if ((r = dalloc(c, &Y2, (size_t)capacity)) != LSGG_OK) return r;
    if ((r = dalloc(c, &I2, (size_t)capacity)) != LSGG_OK) return r;
    CK(cudaMemcpyAsync(X2, c->B.X, (size_t)need_prev * 4, cudaMemcpyDeviceToDevice, c->stream));
    CK(cudaMemcpyAsync(I2, c->B.IDF, (size_t)need_prev * 4, cudaMemcpyDeviceToDevice, c->stream));
    CK(cudaStreamSynchronize(c->stream));
    c->device_bytes -= 3 * c->B.cap * 4;
    dfree(c, c->B.X);
    dfree(c, c->B.Y);
    dfree(c, c->B.IDF);
    c->B.X = X2;
    c->B.Y = Y2;
    c->B.IDF = I2;
    if ((r = replace_z(c, capacity)) != LSGG_OK) return r;
    if ((r = replace_map(c, capacity)) != LSGG_OK) return r;
    c->B.cap = capacity;
    if ((r = ensure_chunk_cap(c)) != LSGG_OK) return r;
    if (c->graph) { cudaGraphExecDestroy(c->graph); c->graph = nullptr; }
    return relayout(c);
}

int lsgg_debug_set_wait_limit(lsgg_ctx* c, int32_t polls) {
    if (!c) return LSGG_ERR_INVALID_ARG;
    int r = lsgg_sync(c, -1);
    if (r != LSGG_OK) return r;
    c->B.wait_limit = polls < 0 ? kWaitIters : polls;
    if (c->graph) {                       // the captured step holds the buffers by value
        cudaGraphExecDestroy(c->graph);
        c->graph = nullptr;
    }
    return LSGG_OK;
}

int lsgg_keep_field(lsgg_ctx* c, int32_t on) {
    if (!c) return LSGG_ERR_INVALID_ARG;
    const int v = on ? 1 : 0;
    if (c->B.keep_field == v) return LSGG_OK;
    c->B.keep_field = v;
    if (c->graph) { cudaGraphExecDestroy(c->graph); c->graph = nullptr; }   // the field pass's parameters changed
    return LSGG_OK;
}

int lsgg_grain_neighbours(lsgg_ctx* c, int32_t* counts, int32_t* ids, int32_t cap_per_grain) {
    if (!c || !counts || !ids || cap_per_grain < 1) return LSGG_ERR_INVALID_ARG;
    int r = lsgg_sync(c, -1);
    if (r != LSGG_OK) return r;
    if (!c->field_valid) return LSGG_ERR_NOT_READY;
    int *dt = nullptr, *dc = nullptr;
    if ((r = dalloc(c, &dt, (size_t)c->G * cap_per_grain)) != LSGG_OK) return r;
    if ((r = dalloc(c, &dc, (size_t)c->G)) != LSGG_OK) { dfree(c, dt); return r; }
    // the boxes the last step ran on (its field covers them): the prev table
    cudaError_t e = launch_field_neighbours(c->B, c->B.prev, cap_per_grain, dt, dc, c->stream);
    if (e == cudaSuccess) e = cudaMemcpyAsync(counts, dc, (size_t)c->G * 4, cudaMemcpyDeviceToHost, c->stream);
    if (e == cudaSuccess)
        e = cudaMemcpyAsync(ids, dt, (size_t)c->G * cap_per_grain * 4, cudaMemcpyDeviceToHost, c->stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(c->stream);
    c->device_bytes -= (long long)c->G * (cap_per_grain + 1) * 4;
    dfree(c, dt);
    dfree(c, dc);
    return e == cudaSuccess ? LSGG_OK : LSGG_ERR_CUDA;
}

int lsgg_get_boxes(lsgg_ctx* c, int32_t* out, int64_t cap) {
    if (!c || !out || cap < 7LL * c->G) return LSGG_ERR_INVALID_ARG;
    int r = lsgg_sync(c, -1);
    if (r != LSGG_OK) return r;
    std::vector<Box> hb(c->G);
    CK(cudaMemcpy(hb.data(), c->B.cur, (size_t)c->G * sizeof(Box), cudaMemcpyDeviceToHost));
    for (int i = 0; i < c->G; ++i) {
        const Box& b = hb[i];
        int32_t* o = out + 7 * (size_t)i;
        o[0] = b.nx > 0;
        o[1] = b.ox; o[2] = b.oy; o[3] = b.oz;
        o[4] = b.nx; o[5] = b.ny; o[6] = b.nz;
    }
    return LSGG_OK;
}

static int packed_offsets(lsgg_ctx* c, const Box* table, std::vector<long long>& off) {
    std::vector<Box> hb(c->G);
    CK(cudaMemcpy(hb.data(), table, (size_t)c->G * sizeof(Box), cudaMemcpyDeviceToHost));
    off.assign(c->G + 1, 0);
    for (int i = 0; i < c->G; ++i)
        off[i + 1] = off[i] + (hb[i].nx > 0 ? (long long)hb[i].nx * hb[i].ny * hb[i].nz : 0);
    CK(cudaMemcpy(c->d_packed_off, off.data(), off.size() * 8, cudaMemcpyHostToDevice));
    return LSGG_OK;
}

int lsgg_get_phi(lsgg_ctx* c, float* out, int64_t cap, int64_t* n_out) {
    if (!c) return LSGG_ERR_INVALID_ARG;
    int r = lsgg_sync(c, -1);
    if (r != LSGG_OK) return r;
    std::vector<long long> off;
    if ((r = packed_offsets(c, c->B.cur, off)) != LSGG_OK) return r;
    if (n_out) *n_out = off[c->G];
    if (!out || cap < off[c->G]) return LSGG_ERR_CAPACITY;
    float* d = nullptr;
    if ((r = dalloc(c, &d, (size_t)off[c->G])) != LSGG_OK) return r;
    const float* x = nullptr;
    cudaError_t e = state_as_f32(c, &x);
    if (e == cudaSuccess) e = launch_pack_state(c->dom, c->G, c->B.cur, c->B.prev, x, c->d_packed_off, d, c->stream);
    if (e == cudaSuccess) e = cudaMemcpyAsync(out, d, (size_t)off[c->G] * 4, cudaMemcpyDeviceToHost, c->stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(c->stream);
    c->device_bytes -= off[c->G] * 4;
    dfree(c, d);
    return e == cudaSuccess ? LSGG_OK : LSGG_ERR_CUDA;
}

int lsgg_debug_pair_ids(lsgg_ctx* c, int32_t* idf_out, int32_t* map_out, int64_t cap) {
    if (!c || !idf_out || !map_out) return LSGG_ERR_INVALID_ARG;
    if (!c->B.gb_map) return LSGG_ERR_UNSUPPORTED;
    int r = lsgg_sync(c, -1);
    if (r != LSGG_OK) return r;
    std::vector<long long> off;
    if ((r = packed_offsets(c, c->B.cur, off)) != LSGG_OK) return r;
    if (cap < off[c->G]) return LSGG_ERR_CAPACITY;
    int* tmp = nullptr;
    if ((r = dalloc(c, &tmp, (size_t)off[c->G] + 1)) != LSGG_OK) return r;
    cudaError_t e = launch_gb_map_step(c->B, c->stream);
    const void* src[2] = {c->B.Z, c->B.gb_map};      // the resampled ID-field, the map
    int32_t* dst[2] = {idf_out, map_out};
    for (int k = 0; k < 2 && e == cudaSuccess; ++k) {
        e = launch_pack_cur(c->G, c->B.cur, src[k], c->d_packed_off, tmp, c->stream);
        if (e == cudaSuccess) e = cudaMemcpyAsync(dst[k], tmp, (size_t)off[c->G] * 4, cudaMemcpyDeviceToHost, c->stream);
        if (e == cudaSuccess) e = cudaStreamSynchronize(c->stream);
    }
    c->device_bytes -= (off[c->G] + 1) * 4;
    dfree(c, tmp);
    return e == cudaSuccess ? LSGG_OK : LSGG_ERR_CUDA;
}

int lsgg_set_state(lsgg_ctx* c, const int32_t* boxes, const float* phi, const int32_t* idf) {
    if (!c || !boxes || !phi) return LSGG_ERR_INVALID_ARG;
    int r = lsgg_sync(c, -1);
    if (r != LSGG_OK) return r;
    const Domain& D = c->dom;
    std::vector<Box> hb(c->G);
    std::vector<long long> off(c->G + 1, 0);
    long long need = 0;
    for (int i = 0; i < c->G; ++i) {
        const int32_t* b = boxes + 7 * (size_t)i;
        Box x{};
        if (b[0]) {
            if (b[4] < 1 || b[5] < 1 || b[6] < 1 || b[4] > D.nx || b[5] > D.ny || b[6] > D.nz) return LSGG_ERR_INVALID_ARG;
            if (b[1] < 0 || b[2] < 0 || b[3] < 0 || b[1] >= D.nx || b[2] >= D.ny || b[3] >= D.nz) return LSGG_ERR_INVALID_ARG;
            x.ox = b[1]; x.oy = b[2]; x.oz = b[3];
            x.nx = b[4]; x.ny = b[5]; x.nz = b[6];
        }
        hb[i] = x;
        off[i + 1] = off[i] + (x.nx > 0 ? (long long)x.nx * x.ny * x.nz : 0);
        need += host_box_elems(x);
    }
    if (need > c->B.cap && (r = grow_arena(c, need)) != LSGG_OK) return r;
    CK(cudaMemcpy(c->B.cur, hb.data(), (size_t)c->G * sizeof(Box), cudaMemcpyHostToDevice));
    // the state will live in this layout: `prev` equal to `cur` already for the
    // size classes the layout assigns (the same as any later relayout's)
    CK(cudaMemcpy(c->B.prev, hb.data(), (size_t)c->G * sizeof(Box), cudaMemcpyHostToDevice));
    if ((r = relayout(c)) != LSGG_OK) return r;
    float* dphi = nullptr;
    int* didf = nullptr;
    if ((r = dalloc(c, &dphi, (size_t)off[c->G])) != LSGG_OK) return r;
    if (idf && (r = dalloc(c, &didf, (size_t)off[c->G])) != LSGG_OK) return r;
    CK(cudaMemcpy(c->d_packed_off, off.data(), off.size() * 8, cudaMemcpyHostToDevice));
    CK(cudaMemcpy(dphi, phi, (size_t)off[c->G] * 4, cudaMemcpyHostToDevice));
    if (idf) CK(cudaMemcpy(didf, idf, (size_t)off[c->G] * 4, cudaMemcpyHostToDevice));
    CK(launch_unpack_state(c->G, c->B.cur, dphi, didf, c->d_packed_off, c->B.bf16 ? c->B.Y : c->B.X, c->B.IDF,
                           c->stream));
    if (c->B.bf16) CK(launch_f32_to_state(c->B.Y, c->B.X, c->B.cap, c->stream));
    CK(cudaMemcpyAsync(c->B.prev, c->B.cur, (size_t)c->G * sizeof(Box), cudaMemcpyDeviceToDevice, c->stream));
    CK(cudaStreamSynchronize(c->stream));
    c->field_valid = false;
    c->device_bytes -= off[c->G] * 4 * (idf ? 2 : 1);
    dfree(c, dphi);
    dfree(c, didf);
    return LSGG_OK;
}

int lsgg_debug_step(lsgg_ctx* c, double dt, float* phip, float* m, int32_t* idm, float* phic, float* phin) {
    if (!c || !(dt > 0.0) || dt > 4.0) return LSGG_ERR_INVALID_ARG;
    int r = lsgg_sync(c, -1);
    if (r != LSGG_OK) return r;
    DebugOut dbg{};
    float* base = nullptr;
    if ((r = dalloc(c, &base, (size_t)c->B.cap * 5)) != LSGG_OK) return r;
    dbg.phip = base;
    dbg.m = base + c->B.cap;
    dbg.idm = reinterpret_cast<int*>(base + 2 * c->B.cap);
    dbg.phic = base + 3 * c->B.cap;
    dbg.phin = base + 4 * c->B.cap;
    c->steps_target += 1;
    c->last_dt = dt;
    c->field_valid = field_stored(c);
    r = enqueue_steps(c, 1, dt, &dbg);
    if (r == LSGG_OK) r = lsgg_sync(c, -1);
    if (r == LSGG_OK) {
        std::vector<long long> off;
        r = packed_offsets(c, c->B.prev, off);
        float* tmp = nullptr;
        if (r == LSGG_OK) r = dalloc(c, &tmp, (size_t)off[c->G] + 1);
        void* dst[5] = {phip, m, idm, phic, phin};
        void* src[5] = {dbg.phip, dbg.m, dbg.idm, dbg.phic, dbg.phin};
        for (int k = 0; k < 5 && r == LSGG_OK; ++k) {
            if (!dst[k]) continue;
            if (launch_pack_cur(c->G, c->B.prev, src[k], c->d_packed_off, tmp, c->stream) != cudaSuccess ||
                cudaMemcpyAsync(dst[k], tmp, (size_t)off[c->G] * 4, cudaMemcpyDeviceToHost, c->stream) != cudaSuccess ||
                cudaStreamSynchronize(c->stream) != cudaSuccess)
                r = LSGG_ERR_CUDA;
        }
        if (tmp) { c->device_bytes -= (off[c->G] + 1) * 4; dfree(c, tmp); }
    }
    c->device_bytes -= c->B.cap * 5 * 4;
    dfree(c, base);
    return r;
}

int lsgg_grain_volumes(lsgg_ctx* c, double* out, int64_t cap, int64_t* n_out) {
    if (!c) return LSGG_ERR_INVALID_ARG;
    if (n_out) *n_out = c->G;
    if (!out || cap < c->G) return LSGG_ERR_CAPACITY;
    // enqueued behind the pending steps, read back with their status in one
    // wait; a step that stopped (arena overflow, error) goes through lsgg_sync
    // and the volumes are taken again
    for (int attempt = 0; attempt < 2; ++attempt) {
        if (attempt == 1) {
            int r = lsgg_sync(c, -1);
            if (r != LSGG_OK) return r;
        }
        const float* x = nullptr;
        CK(state_as_f32(c, &x));
        CK(launch_volumes(c->dom, c->G, c->B.cur, c->B.prev, x, c->d_vol, c->stream));
        CK(cudaMemcpyAsync(out, c->d_vol, (size_t)c->G * 8, cudaMemcpyDeviceToHost, c->stream));
        CK(cudaMemcpyAsync(c->h_st, c->B.st, sizeof(StepState), cudaMemcpyDeviceToHost, c->stream));
        CK(cudaStreamSynchronize(c->stream));
        if (c->h_st->status == 0 && !c->h_st->halt) return LSGG_OK;
    }
    return c->h_st->status ? c->h_st->status : LSGG_ERR_CUDA;
}

int lsgg_grain_statistics(lsgg_ctx* c, int32_t n_bins, double r_max_rel, lsgg_grain_stats* out, double* hist) {
    if (!c || !out || !hist || n_bins < 1 || n_bins > 4096 || !(r_max_rel > 0.0)) return LSGG_ERR_INVALID_ARG;
    int r = lsgg_sync(c, -1);
    if (r != LSGG_OK) return r;
    const float* x = nullptr;
    CK(state_as_f32(c, &x));
    CK(launch_volumes(c->dom, c->G, c->B.cur, c->B.prev, x, c->d_vol, c->stream));
    double* d = nullptr;
    constexpr int kHead = 8;
    if ((r = dalloc(c, &d, (size_t)n_bins + kHead)) != LSGG_OK) return r;
    cudaError_t e = launch_grain_stats(c->d_vol, c->G, c->dom.dim, n_bins, r_max_rel, d, d + kHead, c->stream);
    double h[kHead];
    if (e == cudaSuccess) e = cudaMemcpyAsync(h, d, kHead * 8, cudaMemcpyDeviceToHost, c->stream);
    if (e == cudaSuccess) e = cudaMemcpyAsync(hist, d + kHead, (size_t)n_bins * 8, cudaMemcpyDeviceToHost, c->stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(c->stream);
    c->device_bytes -= (long long)(n_bins + kHead) * 8;
    dfree(c, d);
    if (e != cudaSuccess) return LSGG_ERR_CUDA;
    out->alive = (int64_t)h[0];
    out->mean_volume = h[1];
    out->mean_radius = h[2];
    out->rms_radius = h[3];
    out->max_radius = h[4];
    out->overflow = h[5];
    out->rho = h[6];
    out->var_z = h[7];
    return LSGG_OK;
}

int lsgg_texture_shares(lsgg_ctx* c, const int32_t* grain_class, int32_t n_classes, double* out) {
    if (!c || !grain_class || !out || n_classes < 1 || n_classes > 4096) return LSGG_ERR_INVALID_ARG;
    int r = lsgg_sync(c, -1);
    if (r != LSGG_OK) return r;
    const float* x = nullptr;
    CK(state_as_f32(c, &x));
    CK(launch_volumes(c->dom, c->G, c->B.cur, c->B.prev, x, c->d_vol, c->stream));
    int* dc = nullptr;
    double* d = nullptr;
    if ((r = dalloc(c, &dc, (size_t)c->G)) != LSGG_OK) return r;
    if ((r = dalloc(c, &d, (size_t)n_classes + 1)) != LSGG_OK) {
        c->device_bytes -= (long long)c->G * 4;
        dfree(c, dc);
        return r;
    }
    cudaError_t e = cudaMemcpyAsync(dc, grain_class, (size_t)c->G * 4, cudaMemcpyHostToDevice, c->stream);
    if (e == cudaSuccess) e = launch_texture_shares(c->d_vol, dc, c->G, n_classes, d, c->stream);
    if (e == cudaSuccess) e = cudaMemcpyAsync(out, d, (size_t)n_classes * 8, cudaMemcpyDeviceToHost, c->stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(c->stream);
    c->device_bytes -= (long long)c->G * 4 + (long long)(n_classes + 1) * 8;
    dfree(c, dc);
    dfree(c, d);
    return e == cudaSuccess ? LSGG_OK : LSGG_ERR_CUDA;
}

// Coarse origin and extent of a fine box [o, o + n) on an axis coarsened
// from N to N2 cells: every coarse cell i' whose fine interpolation corners
// floor(u), floor(u) + 1 (u = i' N / N2) can meet the box, i.e. from
// floor((o - 1) N2 / N) to ceil((o + n) N2 / N).
static void coarse_box_axis(int o, int n, int N, int N2, int* o2, int* n2) {
    if (n >= N) {
        *o2 = (int)((long long)o * N2 / N);
        *n2 = N2;
        return;
    }
    auto floor_div = [](long long a, long long b) { return a >= 0 ? a / b : -((-a + b - 1) / b); };
    const long long lo = floor_div((long long)(o - 1) * N2, N);
    const long long hi = -floor_div(-(long long)(o + n) * N2, N);
    const long long ext = hi - lo + 1;
    *o2 = (int)(((lo % N2) + N2) % N2);
    *n2 = ext >= N2 ? N2 : (int)ext;
}

int lsgg_coarsen(lsgg_ctx* c, int32_t nx, int32_t ny, int32_t nz) {
    if (!c) return LSGG_ERR_INVALID_ARG;
    const Domain fine = c->dom;
    if (fine.dim != 3 || !c->B.use_passes) return LSGG_ERR_UNSUPPORTED;
    if (nx < 1 || ny < 1 || nz < 1 || nx > fine.nx || ny > fine.ny || nz > fine.nz) return LSGG_ERR_INVALID_ARG;
    if ((long long)nx * fine.ny != (long long)ny * fine.nx || (long long)nx * fine.nz != (long long)nz * fine.nx)
        return LSGG_ERR_INVALID_ARG;                                       // one spacing on every axis
    int r = lsgg_sync(c, -1);
    if (r != LSGG_OK) return r;
    if (c->graph) { cudaGraphExecDestroy(c->graph); c->graph = nullptr; }
    // the grains' boxes on the fine grid (`cur`: the functions the next step
    // would start from) -> candidate boxes on the coarse grid
    std::vector<Box> hp((size_t)c->G), hc((size_t)c->G);
    CK(cudaMemcpy(hp.data(), c->B.cur, (size_t)c->G * sizeof(Box), cudaMemcpyDeviceToHost));
    const int N[3] = {fine.nx, fine.ny, fine.nz}, N2[3] = {nx, ny, nz};
    for (int b = 0; b < c->G; ++b) {
        Box o = hp[b], q{};
        if (o.nx > 0) {
            const int oo[3] = {o.ox, o.oy, o.oz}, on[3] = {o.nx, o.ny, o.nz};
            int qo[3], qn[3];
            for (int a = 0; a < 3; ++a) coarse_box_axis(oo[a], on[a], N[a], N2[a], &qo[a], &qn[a]);
            q.ox = qo[0]; q.oy = qo[1]; q.oz = qo[2];
            q.nx = qn[0]; q.ny = qn[1]; q.nz = qn[2];
        }
        hc[b] = q;
    }
    // the coarse domain, its tiles, the candidate layout
    c->dom.nx = nx;
    c->dom.ny = ny;
    c->dom.nz = nz;
    c->B.dom = c->dom;
    CK(configure_passes(c->B));
    CK(cudaMemcpy(c->B.cur, hc.data(), (size_t)c->G * sizeof(Box), cudaMemcpyHostToDevice));
    Box* d_fine = nullptr;                               // the grains' fine boxes, for the projection
    if ((r = dalloc(c, &d_fine, (size_t)c->G)) != LSGG_OK) return r;
    r = cudaMemcpy(d_fine, hp.data(), (size_t)c->G * sizeof(Box), cudaMemcpyHostToDevice) == cudaSuccess ? LSGG_OK
                                                                                                     : LSGG_ERR_CUDA;
    if (r == LSGG_OK) r = relayout(c);
    // projection into Z, then the re-initialisation and box update of a step
    const float* x = nullptr;
    cudaError_t e = cudaSuccess;
    if (r == LSGG_OK) e = state_as_f32(c, &x);
    if (r == LSGG_OK && e == cudaSuccess) e = launch_coarsen(c->B, fine, d_fine, x, c->stream);
    if (r == LSGG_OK && e == cudaSuccess) e = launch_reinit(c->B, make_taps(1.0, c->dom.radius), c->phys,
                                                                c->phys.kind != LSGG_PHYSICS_IDEAL, c->stream);
    if (r == LSGG_OK && e == cudaSuccess) e = cudaStreamSynchronize(c->stream);
    c->device_bytes -= (long long)c->G * (long long)sizeof(Box);
    dfree(c, d_fine);
    c->field_valid = false;
    if (r != LSGG_OK) return r;
    if (e != cudaSuccess) return fail_cuda(e);
    return lsgg_sync(c, -1);
}

int lsgg_voxel_owner(lsgg_ctx* c, int32_t* out, int64_t n_cells) {
    if (!c || !out) return LSGG_ERR_INVALID_ARG;
    long long n = (long long)c->dom.nx * c->dom.ny * c->dom.nz;
    if (n_cells < n) return LSGG_ERR_CAPACITY;
    int r = lsgg_sync(c, -1);
    if (r != LSGG_OK) return r;
    int* d = nullptr;
    if ((r = dalloc(c, &d, (size_t)n)) != LSGG_OK) return r;
    const float* x = nullptr;
    cudaError_t e = state_as_f32(c, &x);
    if (e == cudaSuccess) e = launch_owner(c->dom, c->G, c->B.cur, c->B.prev, x, c->B.T, d, c->stream);
    c->field_valid = false;        // the owner map reused the field's memory
    if (e == cudaSuccess) e = cudaMemcpyAsync(out, d, (size_t)n * 4, cudaMemcpyDeviceToHost, c->stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(c->stream);
    c->device_bytes -= n * 4;
    dfree(c, d);
    return e == cudaSuccess ? LSGG_OK : LSGG_ERR_CUDA;
}

int lsgg_grain_volumes_device(lsgg_ctx* c, double* out_dev, int64_t cap, int32_t* status_dev, void* stream) {
    if (!c || !out_dev) return LSGG_ERR_INVALID_ARG;
    if (cap < c->G) return LSGG_ERR_CAPACITY;
    cudaStream_t s = stream ? (cudaStream_t)stream : c->stream;
    const float* x = nullptr;
    CK(join_caller_stream(c, s, false));
    CK(state_as_f32(c, &x, s));
    CK(launch_volumes(c->dom, c->G, c->B.cur, c->B.prev, x, out_dev, s));
    if (status_dev) CK(launch_step_status(c->B.st, status_dev, s));
    CK(join_caller_stream(c, s, true));
    return LSGG_OK;
}

int lsgg_voxel_owner_device(lsgg_ctx* c, int32_t* out_dev, int64_t n_cells, int32_t* status_dev, void* stream) {
    if (!c || !out_dev) return LSGG_ERR_INVALID_ARG;
    if (n_cells < (long long)c->dom.nx * c->dom.ny * c->dom.nz) return LSGG_ERR_CAPACITY;
    cudaStream_t s = stream ? (cudaStream_t)stream : c->stream;
    const float* x = nullptr;
    CK(join_caller_stream(c, s, false));
    CK(state_as_f32(c, &x, s));
    c->field_valid = false;        // the owner map takes the field's memory as its scratch
    CK(launch_owner(c->dom, c->G, c->B.cur, c->B.prev, x, c->B.T, out_dev, s));
    if (status_dev) CK(launch_step_status(c->B.st, status_dev, s));
    CK(join_caller_stream(c, s, true));
    return LSGG_OK;
}

}  // extern "C"

namespace {

int enqueue_steps(lsgg_ctx* c, long long n, double dt, const DebugOut* dbg) {
    Taps taps = make_taps(dt, c->dom.radius);
    c->phys.dt = (float)dt;
    if (c->cfg.exec == LSGG_EXEC_PLAIN && !dbg) {
        int r;
        const Domain& D = c->dom;
        if (!c->p_t1) {
            long long R2 = 2 * c->dom.radius;
            long long t = (long long)D.nx * (D.ny + R2) * (D.dim == 3 ? D.nz + R2 : 1);
            if ((r = dalloc(c, &c->p_t1, (size_t)t)) != LSGG_OK) return r;
            if ((r = dalloc(c, &c->p_t2, (size_t)t)) != LSGG_OK) return r;
        }
        if (c->p_cap != c->B.cap) {
            dfree(c, c->p_C); dfree(c, c->p_G); dfree(c, c->p_H);
            if ((r = dalloc(c, &c->p_C, (size_t)c->B.cap)) != LSGG_OK) return r;
            if ((r = dalloc(c, &c->p_G, (size_t)c->B.cap)) != LSGG_OK) return r;
            if ((r = dalloc(c, &c->p_H, (size_t)c->B.cap)) != LSGG_OK) return r;
            c->p_cap = c->B.cap;
        }
        std::vector<Box> hc(c->G), hp(c->G);
        for (long long i = 0; i < n; ++i) {
            // the host loop over grains needs this step's boxes
            if (cudaMemcpyAsync(hc.data(), c->B.cur, (size_t)c->G * sizeof(Box), cudaMemcpyDeviceToHost, c->stream) != cudaSuccess ||
                cudaMemcpyAsync(hp.data(), c->B.prev, (size_t)c->G * sizeof(Box), cudaMemcpyDeviceToHost, c->stream) != cudaSuccess ||
                cudaMemcpyAsync(c->h_st, c->B.st, sizeof(StepState), cudaMemcpyDeviceToHost, c->stream) != cudaSuccess ||
                cudaStreamSynchronize(c->stream) != cudaSuccess)
                return CUDA_FAIL();
            if (c->h_st->halt) return LSGG_OK;         // arena overflow: lsgg_sync resumes
            cudaEvent_t* ev = nullptr;
            if (c->profiling) {
                std::vector<cudaEvent_t> v(5);
                for (auto& e : v) {
                    if (!c->ev_pool.empty()) { e = c->ev_pool.back(); c->ev_pool.pop_back(); }
                    else if (cudaEventCreate(&e) != cudaSuccess) return CUDA_FAIL();
                }
                c->ev_pending.push_back(v);
                ev = c->ev_pending.back().data();
                cudaEventRecord(ev[0], c->stream);
                cudaEventRecord(ev[1], c->stream);
            }
            if (launch_plain_step_impl(c->B, taps, c->phys, hc.data(), hp.data(), c->p_t1, c->p_t2, c->p_C,
                                       c->p_G, c->p_H, c->stream) != cudaSuccess)
                return CUDA_FAIL();
            if (ev) {
                cudaEventRecord(ev[2], c->stream);
                cudaEventRecord(ev[3], c->stream);
                cudaEventRecord(ev[4], c->stream);
            }
        }
        return LSGG_OK;
    }
    if (!dbg && !c->profiling) {
        // CUDA graph of one step, captured once per dt and replayed n times
        if (!c->graph || c->graph_dt != dt) {
            if (c->graph) { cudaGraphExecDestroy(c->graph); c->graph = nullptr; }
            cudaGraph_t g = nullptr;
            if (cudaStreamBeginCapture(c->stream, cudaStreamCaptureModeThreadLocal) != cudaSuccess) return CUDA_FAIL();
            cudaError_t le = launch_step(c->B, taps, c->phys, nullptr, c->stream, nullptr, &c->ss);
            cudaError_t ce = cudaStreamEndCapture(c->stream, &g);
            if (le != cudaSuccess || ce != cudaSuccess) { if (g) cudaGraphDestroy(g); return CUDA_FAIL(); }
            cudaGraphInstantiateParams ip{};
            ip.flags = 0;
            cudaError_t ie = cudaGraphInstantiateWithParams(&c->graph, g, &ip);
            if (ie != cudaSuccess && trace_errors()) {
                cudaGraphNodeType nt = cudaGraphNodeTypeEmpty;
                if (ip.errNode_out) cudaGraphNodeGetType(ip.errNode_out, &nt);
                std::fprintf(stderr, "lsgg: graph instantiation: result %d, failing node type %d\n", (int)ip.result_out,
                             (int)nt);
            }
            cudaGraphDestroy(g);
            if (ie != cudaSuccess) { c->graph = nullptr; return CUDA_FAIL(); }
            c->graph_dt = dt;
        }
        for (long long i = 0; i < n; ++i)
            if (cudaGraphLaunch(c->graph, c->stream) != cudaSuccess) return CUDA_FAIL();
        return LSGG_OK;
    }
    for (long long i = 0; i < n; ++i) {
        cudaEvent_t* ev = nullptr;
        if (c->profiling) {
            std::vector<cudaEvent_t> v(c->B.use_passes ? 5 + kPassEvents : 5);
            for (auto& e : v) {
                if (!c->ev_pool.empty()) { e = c->ev_pool.back(); c->ev_pool.pop_back(); }
                else if (cudaEventCreate(&e) != cudaSuccess) return CUDA_FAIL();
            }
            c->ev_pending.push_back(v);
            ev = c->ev_pending.back().data();
        }
        // profiled steps run every kernel on the context's stream, one after
        // another, so that each kernel's event time is its own
        if (launch_step(c->B, taps, c->phys, dbg, c->stream, ev, ev ? nullptr : &c->ss, nullptr,
                        ev && c->B.use_passes ? ev + 5 : nullptr) != cudaSuccess)
            return CUDA_FAIL();
    }
    return LSGG_OK;
}

}  // namespace
