// Serving: continuous batching of independent simulations on one GPU.
//
// A server owns a scheduler thread.  Submitted requests (a configuration,
// a number of steps and dt) wait in a FIFO queue; the scheduler admits the
// head of the queue as soon as the sum of the HBM estimates of the active
// requests plus its own stays within the budget and a slot is free, and
// creates its microstructure (boxes resident on the device from then on).
// With shared launches, the active requests that a step group accepts are
// advanced by one group: every chunk of steps is one set of launches over all
// of their boxes, each request stopping at its own step count (the group's
// step limits); the group is rebuilt when a request joins or completes.  The
// other requests (and all of them in per-context mode) have their own
// streams fed with chunks of steps (CUDA-graph replays), so that work from
// different requests overlaps on the device.  A request that has run all its
// steps has its grain volumes copied out and its device memory released,
// which admits the next ones.  The paper has no serving layer; this is the
// request loop around Algorithm 1.
#include <algorithm>
#include <atomic>
#include <chrono>
#include <condition_variable>
#include <cstring>
#include <deque>
#include <map>
#include <memory>
#include <mutex>
#include <thread>
#include <vector>

#include <cuda_runtime.h>

#include "../../include/lsgg.h"

namespace {

using Clock = std::chrono::steady_clock;

struct Request {
    int64_t ticket = 0;
    lsgg_config cfg{};
    std::vector<double> seeds, weights, quats, energy;
    std::vector<int32_t> labels;
    int32_t n_steps = 0;
    double dt = 1.0;
    int64_t estimate = 0;
    bool grouped = false;             // advanced by the server's step group
    // progress
    int32_t state = 0;                // 0 queued, 1 running, 2 done, < 0 failed (status code)
    lsgg_ctx* ctx = nullptr;
    int32_t enqueued = 0;
    int64_t device_bytes = 0;
    int64_t cell_updates = 0;
    double t_submit = 0, t_admit = 0, t_done = 0;
    std::vector<double> volumes;
};

int64_t estimate_bytes(const lsgg_config& c) {
    // arena X, Y, ID-field (and the pass path's Z when the physics keeps an
    // ID-field) at ~12 box cells per domain cell with 1.5x slack, the 16-byte
    // neighbour-max field, init temporaries (labels, neighbour bits), the pass
    // path's work-item lists
    const int64_t ncell = (int64_t)c.nx * c.ny * c.nz;
    const int64_t g = c.n_grains;
    const int64_t arenas = (c.exec == LSGG_EXEC_BATCHED && c.physics != LSGG_PHYSICS_IDEAL) ? 4 : 3;
    const int64_t items = c.exec == LSGG_EXEC_BATCHED ? 8 * g * ((int64_t)c.nz + 16) : 0;
    return arenas * 4 * 18 * ncell + 16 * ncell + 4 * ncell + g * ((g + 31) / 32) * 4 + items + (64LL << 20);
}

double seconds_since(Clock::time_point t0) {
    return std::chrono::duration<double>(Clock::now() - t0).count();
}

}  // namespace

// The server's step group (created once, its membership replaced as
// requests join and complete), the requests it advances (in member order) and
// an event per chunk still in flight (recorded on a member's stream, which
// waits for the chunk).
struct ServeGroup {
    lsgg_group* g = nullptr;
    std::vector<Request*> members;
    std::vector<int64_t> tickets;            // the members' tickets (identify them; addresses get reused)
    std::deque<cudaEvent_t> chunks;
    double dt = 0.0;
};

// Requests of at most this many domain cells share the step group.  A larger
// one fills the GPU with its own launches and gains more from overlapping the
// others on its own stream: measured on GB300, one group made 48 members of
// 48^3 5.3x and 16 of 96^3 1.4x faster than their own streams, 6 of 160^3
// equal, and a 256^3 member 5 % slower.
constexpr long long kGroupMaxCells = 128LL * 128 * 128;

// A request the server's step group takes (lsgg_group_create's conditions
// and the size bound).
bool groupable(const lsgg_config& c) {
    return c.exec == LSGG_EXEC_BATCHED && c.nz > 1 && c.physics == LSGG_PHYSICS_IDEAL &&
           c.redist == LSGG_REDIST_TAXICAB && c.radius == 5 && !(c.gb_map_tube > 0.0) &&
           (long long)c.nx * c.ny * c.nz <= kGroupMaxCells;
}

struct lsgg_server {
    int64_t budget = 0;
    int32_t max_active = 0;
    int32_t steps_per_round = 0;
    int32_t device = 0;
    int32_t mode = LSGG_SERVE_SHARED;
    ServeGroup cur;                          // the step group of shared launches
    std::vector<cudaEvent_t> free_events;
    Clock::time_point t0;
    std::mutex mu;
    std::condition_variable cv_work, cv_done;
    std::deque<std::shared_ptr<Request>> queue;
    std::vector<std::shared_ptr<Request>> active;
    std::map<int64_t, std::shared_ptr<Request>> all;
    int64_t next_ticket = 1;
    int64_t used = 0;
    int64_t peak_used = 0;
    int64_t completed = 0;
    int64_t cell_updates = 0;
    bool stop = false;
    std::thread worker;

    void run();
    bool admit_one(std::unique_lock<std::mutex>& lk);
    bool feed_group();
    cudaEvent_t take_event();
};

cudaEvent_t lsgg_server::take_event() {
    cudaEvent_t e = nullptr;
    if (!free_events.empty()) { e = free_events.back(); free_events.pop_back(); return e; }
    if (cudaEventCreateWithFlags(&e, cudaEventDisableTiming) != cudaSuccess) { cudaGetLastError(); return nullptr; }
    return e;
}

// Shared launches: the group's members are the running groupable requests
// that still have steps to enqueue (those of the first one's dt, at most
// LSGG_MAX_GROUP); keep up to two chunks of steps in flight.
bool lsgg_server::feed_group() {
    bool progress = false;
    while (!cur.chunks.empty() && cudaEventQuery(cur.chunks.front()) == cudaSuccess) {
        free_events.push_back(cur.chunks.front());
        cur.chunks.pop_front();
    }
    std::vector<Request*> want;
    for (auto& r : active)
        if (r->grouped && r->state == 1 && r->enqueued < r->n_steps && (want.empty() || r->dt == want[0]->dt) &&
            (int)want.size() < LSGG_MAX_GROUP)
            want.push_back(r.get());
    std::vector<int64_t> tickets;
    for (Request* r : want) tickets.push_back(r->ticket);
    if (want.empty()) {
        cur.members.clear();
        cur.tickets.clear();
        return false;
    }
    if (tickets != cur.tickets) {
        std::vector<lsgg_ctx*> ctxs;
        for (Request* r : want) ctxs.push_back(r->ctx);
        const int st = cur.g ? lsgg_group_set_members(cur.g, ctxs.data(), (int32_t)ctxs.size())
                             : lsgg_group_create(ctxs.data(), (int32_t)ctxs.size(), &cur.g);
        if (st != LSGG_OK) {
            for (Request* r : want) r->grouped = false;   // their own streams from now on
            cur.members.clear();
            cur.tickets.clear();
            return true;
        }
        cur.members = want;
        cur.tickets = tickets;
        cur.dt = want[0]->dt;
        progress = true;
    }
    if (cur.chunks.size() < 2) {
        std::vector<int64_t> lim;
        for (Request* r : cur.members) lim.push_back(r->n_steps);
        const int st = lsgg_group_step(cur.g, steps_per_round, cur.dt, lim.data());
        if (st != LSGG_OK) {
            for (Request* r : cur.members) { r->grouped = false; r->state = st; }
            cur.members.clear();
            cur.tickets.clear();
            return true;
        }
        for (Request* r : cur.members) r->enqueued = std::min(r->n_steps, r->enqueued + steps_per_round);
        cudaEvent_t e = take_event();
        if (e && cudaEventRecord(e, (cudaStream_t)lsgg_get_stream(cur.members[0]->ctx)) == cudaSuccess)
            cur.chunks.push_back(e);
        else if (e) free_events.push_back(e);
        progress = true;
    }
    return progress;
}

bool lsgg_server::admit_one(std::unique_lock<std::mutex>& lk) {
    if (queue.empty() || (int32_t)active.size() >= max_active) return false;
    std::shared_ptr<Request> r = queue.front();
    if (r->estimate > budget) {               // can never fit
        queue.pop_front();
        r->state = LSGG_ERR_OVER_BUDGET;
        r->t_done = seconds_since(t0);
        cv_done.notify_all();
        return true;
    }
    if (used + r->estimate > budget) return false;
    queue.pop_front();
    used += r->estimate;
    peak_used = std::max(peak_used, used);
    lsgg_config cfg = r->cfg;
    cfg.seeds = r->seeds.empty() ? nullptr : r->seeds.data();
    cfg.weights = r->weights.empty() ? nullptr : r->weights.data();
    cfg.quats = r->quats.empty() ? nullptr : r->quats.data();
    cfg.energy = r->energy.empty() ? nullptr : r->energy.data();
    cfg.labels = r->labels.empty() ? nullptr : r->labels.data();
    cfg.device = device;
    lk.unlock();
    lsgg_ctx* ctx = nullptr;
    int st = lsgg_create_microstructure(&cfg, nullptr, &ctx);
    lk.lock();
    if (st != LSGG_OK) {
        used -= r->estimate;
        r->state = st;
        r->t_done = seconds_since(t0);
        cv_done.notify_all();
        return true;
    }
    r->ctx = ctx;
    r->state = 1;
    r->grouped = mode == LSGG_SERVE_SHARED && groupable(cfg);
    r->t_admit = seconds_since(t0);
    lsgg_stats s{};
    if (lsgg_get_stats(ctx, &s) == LSGG_OK) r->device_bytes = s.device_bytes;
    active.push_back(r);
    return true;
}

void lsgg_server::run() {
    cudaSetDevice(device);
    std::unique_lock<std::mutex> lk(mu);
    while (!stop) {
        bool progress = false;
        while (admit_one(lk)) progress = true;
        if (mode == LSGG_SERVE_SHARED && feed_group()) progress = true;
        // feed idle streams, retire finished requests
        for (size_t k = 0; k < active.size();) {
            std::shared_ptr<Request> r = active[k];
            cudaStream_t s = (cudaStream_t)lsgg_get_stream(r->ctx);
            cudaError_t q = cudaStreamQuery(s);
            if (q == cudaErrorNotReady) { ++k; continue; }
            if (q != cudaSuccess) cudaGetLastError();
            if (r->grouped && r->state == 1 && r->enqueued < r->n_steps) { ++k; continue; }   // the group feeds it
            if (r->enqueued < r->n_steps && r->state == 1) {
                const int32_t chunk = std::min(steps_per_round, r->n_steps - r->enqueued);
                int st = lsgg_step(r->ctx, chunk, r->dt);
                if (st == LSGG_OK) {
                    r->enqueued += chunk;
                    progress = true;
                    ++k;
                    continue;
                }
                r->state = st;
            }
            // all steps enqueued and the stream is idle: finish (grows the arena if a step overflowed it)
            lk.unlock();
            int st = r->state < 0 ? r->state : lsgg_sync(r->ctx, -1);
            std::vector<double> vol((size_t)r->cfg.n_grains);
            int64_t n = 0;
            lsgg_stats rs{};
            if (st == LSGG_OK) st = lsgg_get_stats(r->ctx, &rs);
            if (st == LSGG_OK && rs.steps_done < r->n_steps) {   // resumed after an arena overflow
                lk.lock();
                ++k;
                continue;
            }
            if (st == LSGG_OK) st = lsgg_grain_volumes(r->ctx, vol.data(), (int64_t)vol.size(), &n);
            lsgg_destroy(r->ctx);
            lk.lock();
            r->ctx = nullptr;
            r->volumes.swap(vol);
            r->cell_updates = rs.cell_updates;
            r->state = st == LSGG_OK ? 2 : st;
            r->t_done = seconds_since(t0);
            used -= r->estimate;
            ++completed;
            cell_updates += rs.cell_updates;
            active.erase(active.begin() + (long)k);
            cv_done.notify_all();
            progress = true;
        }
        if (!progress) cv_work.wait_for(lk, std::chrono::microseconds(200));
    }
    if (cur.g) lsgg_group_destroy(cur.g);     // waits for its chunks
    for (cudaEvent_t e : cur.chunks) cudaEventDestroy(e);
    cur = ServeGroup{};
    for (cudaEvent_t e : free_events) cudaEventDestroy(e);
    free_events.clear();
    for (auto& r : active) {
        lk.unlock();
        lsgg_destroy(r->ctx);
        lk.lock();
        r->ctx = nullptr;
        r->state = LSGG_ERR_NOT_READY;
    }
    active.clear();
}

extern "C" {

int lsgg_server_create(int64_t budget_bytes, int32_t max_active, int32_t steps_per_round, int32_t device,
                       lsgg_server** out) {
    return lsgg_server_create_mode(budget_bytes, max_active, steps_per_round, device, LSGG_SERVE_SHARED, out);
}

int lsgg_server_create_mode(int64_t budget_bytes, int32_t max_active, int32_t steps_per_round, int32_t device,
                            int32_t mode, lsgg_server** out) {
    if (!out || budget_bytes <= 0 || max_active < 1 || steps_per_round < 1) return LSGG_ERR_INVALID_ARG;
    if (mode != LSGG_SERVE_SHARED && mode != LSGG_SERVE_PER_CONTEXT) return LSGG_ERR_INVALID_ARG;
    int ndev = 0;
    if (cudaGetDeviceCount(&ndev) != cudaSuccess || device < 0 || device >= ndev) {
        cudaGetLastError();
        return LSGG_ERR_CUDA;
    }
    lsgg_server* s = new lsgg_server();
    s->budget = budget_bytes;
    s->max_active = max_active;
    s->steps_per_round = steps_per_round;
    s->device = device;
    s->mode = mode;
    s->t0 = Clock::now();
    s->worker = std::thread([s] { s->run(); });
    *out = s;
    return LSGG_OK;
}

int lsgg_server_submit(lsgg_server* s, const lsgg_config* cfg, int32_t n_steps, double dt, int64_t* ticket) {
    if (!s || !cfg || !ticket || n_steps < 0 || !(dt > 0.0) || dt > 4.0) return LSGG_ERR_INVALID_ARG;
    if (cfg->n_grains < 1 || cfg->nx < 1 || cfg->ny < 1 || cfg->nz < 1) return LSGG_ERR_INVALID_ARG;
    auto r = std::make_shared<Request>();
    r->cfg = *cfg;
    const size_t g = (size_t)cfg->n_grains;
    if (cfg->seeds) r->seeds.assign(cfg->seeds, cfg->seeds + 3 * g);
    if (cfg->weights) r->weights.assign(cfg->weights, cfg->weights + g);
    if (cfg->quats) r->quats.assign(cfg->quats, cfg->quats + 4 * g);
    if (cfg->energy) r->energy.assign(cfg->energy, cfg->energy + g);
    if (cfg->labels) r->labels.assign(cfg->labels, cfg->labels + (size_t)cfg->nx * cfg->ny * cfg->nz);
    r->n_steps = n_steps;
    r->dt = dt;
    r->estimate = estimate_bytes(*cfg);
    std::lock_guard<std::mutex> lk(s->mu);
    r->ticket = s->next_ticket++;
    r->t_submit = seconds_since(s->t0);
    s->queue.push_back(r);
    s->all[r->ticket] = r;
    *ticket = r->ticket;
    s->cv_work.notify_all();
    return LSGG_OK;
}

static void fill_info(const Request& r, lsgg_request_info* info) {
    if (!info) return;
    info->state = r.state;
    info->t_submit = r.t_submit;
    info->t_admit = r.t_admit;
    info->t_done = r.t_done;
    info->cell_updates = r.cell_updates;
    info->device_bytes = r.device_bytes;
    info->estimate_bytes = r.estimate;
}

int lsgg_server_wait(lsgg_server* s, int64_t ticket, int64_t timeout_ms, lsgg_request_info* info) {
    if (!s) return LSGG_ERR_INVALID_ARG;
    std::unique_lock<std::mutex> lk(s->mu);
    auto it = s->all.find(ticket);
    if (it == s->all.end()) return LSGG_ERR_INVALID_ARG;
    std::shared_ptr<Request> r = it->second;
    auto done = [&] { return r->state == 2 || r->state < 0; };
    if (timeout_ms < 0) s->cv_done.wait(lk, done);
    else if (!s->cv_done.wait_for(lk, std::chrono::milliseconds(timeout_ms), done)) {
        fill_info(*r, info);
        return LSGG_ERR_TIMEOUT;
    }
    fill_info(*r, info);
    return r->state < 0 ? r->state : LSGG_OK;
}

int lsgg_server_poll(lsgg_server* s, int64_t ticket, lsgg_request_info* info) {
    if (!s) return LSGG_ERR_INVALID_ARG;
    std::lock_guard<std::mutex> lk(s->mu);
    auto it = s->all.find(ticket);
    if (it == s->all.end()) return LSGG_ERR_INVALID_ARG;
    fill_info(*it->second, info);
    if (it->second->state < 0) return it->second->state;
    return it->second->state == 2 ? LSGG_OK : LSGG_ERR_NOT_READY;
}

int lsgg_server_volumes(lsgg_server* s, int64_t ticket, double* out, int64_t cap, int64_t* n_out) {
    if (!s) return LSGG_ERR_INVALID_ARG;
    std::lock_guard<std::mutex> lk(s->mu);
    auto it = s->all.find(ticket);
    if (it == s->all.end()) return LSGG_ERR_INVALID_ARG;
    const Request& r = *it->second;
    if (r.state != 2) return r.state < 0 ? r.state : LSGG_ERR_NOT_READY;
    if (n_out) *n_out = (int64_t)r.volumes.size();
    if (!out || cap < (int64_t)r.volumes.size()) return LSGG_ERR_CAPACITY;
    std::memcpy(out, r.volumes.data(), r.volumes.size() * sizeof(double));
    return LSGG_OK;
}

int lsgg_server_release(lsgg_server* s, int64_t ticket) {
    if (!s) return LSGG_ERR_INVALID_ARG;
    std::lock_guard<std::mutex> lk(s->mu);
    auto it = s->all.find(ticket);
    if (it == s->all.end()) return LSGG_ERR_INVALID_ARG;
    if (it->second->state == 0 || it->second->state == 1) return LSGG_ERR_NOT_READY;
    s->all.erase(it);
    return LSGG_OK;
}

int lsgg_server_get_stats(lsgg_server* s, lsgg_server_stats* out) {
    if (!s || !out) return LSGG_ERR_INVALID_ARG;
    std::lock_guard<std::mutex> lk(s->mu);
    out->queued = (int64_t)s->queue.size();
    out->active = (int64_t)s->active.size();
    out->completed = s->completed;
    out->used_bytes = s->used;
    out->peak_bytes = s->peak_used;
    out->cell_updates = s->cell_updates;
    return LSGG_OK;
}

int lsgg_server_destroy(lsgg_server* s) {
    if (!s) return LSGG_ERR_INVALID_ARG;
    {
        std::lock_guard<std::mutex> lk(s->mu);
        s->stop = true;
        s->cv_work.notify_all();
    }
    if (s->worker.joinable()) s->worker.join();
    delete s;
    return LSGG_OK;
}

}  // extern "C"
