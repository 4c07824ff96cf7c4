// Serving: continuous batching of AIR reconstruction requests.
//
// One worker thread owns a CUDA stream.  Requests wait in a FIFO until the
// device bytes of all resident requests, plus theirs, fit the HBM budget and
// a slot is free; they are then admitted at the next step boundary, their
// sinogram copied in once and their state (plan tables, X, b, CG vectors,
// sinogram temporaries) kept on the device until they finish.  Every step
// advances each resident request by one phase of its split-Bregman program:
// one grouped launch per op present over the tiles of all requests in that
// op (plus the tensor-core filter of each BF16X3 request), so requests of
// different sizes and views, at different points of their solves, overlap on
// the device.  A finished request's image is copied out once and its device
// state returned to a per-geometry pool, so a warm server allocates nothing.
// A ring of pinned task tables with one event per entry bounds how many steps
// the host may run ahead of the GPU.
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

#include "host_common.h"
#include "ramp_tc.h"
#include "tiles.cuh"

using namespace air;

namespace {

enum ReqState { QUEUED = 0, ACTIVE = 1, FINISHING = 2, DONE = 3, FAILED = 4 };

struct Request {
    uint64_t id = 0;
    air_geometry geom{};
    float lam = 0.f, mu = 1.f;
    int n_outer = 0, n_cg = 0;
    float *y_pinned = nullptr, *x_pinned = nullptr;
    size_t bytes = 0;
    air_plan *plan = nullptr;
    std::vector<Phase> prog;
    size_t pc = 0;
    int slot = -1;
    std::atomic<int> state{QUEUED};   // read by API threads, advanced by the worker
    air_status status = AIR_OK;
    double t[3] = {0, 0, 0};     // submit, admitted, finished (s since creation)
    cudaEvent_t done_ev = nullptr;
};

bool same_geom(const air_geometry &a, const air_geometry &b) { return std::memcmp(&a, &b, sizeof(a)) == 0; }

constexpr int RING = 8;

}  // namespace

struct air_server {
    size_t budget = 0, used = 0, pooled = 0;
    int max_slots = 0;
    int device = 0;
    std::mutex mu;
    std::condition_variable cv_work, cv_done;
    std::atomic<int> waiters{0};     // API calls waiting for `mu` (the worker lets them in)
    std::deque<Request *> queue;
    std::vector<Request *> active;
    std::map<uint64_t, std::unique_ptr<Request>> all;
    std::vector<std::pair<air_geometry, air_plan *>> pool;   // idle plans, reused by geometry
    std::vector<std::pair<air_geometry, size_t>> plan_bytes; // device bytes of a plan, by geometry, once built
    std::thread worker;
    bool stop = false;
    uint64_t next_id = 1;
    std::chrono::steady_clock::time_point t0;
    cudaStream_t stream = nullptr;
    SliceDesc *d_slices = nullptr;       // [max_slots]
    SliceDesc *h_slices = nullptr;       // pinned staging, one per slot
    Task *d_tasks = nullptr;             // [RING][max_slots]
    Task *h_tasks = nullptr;             // pinned [RING][max_slots]
    cudaEvent_t ring_ev[RING] = {};
    int ring_pos = 0;
    // side streams the independent launches of a step fork onto, joined
    // back by events before the step's ring event
    static constexpr int TC_SIDE = 8;
    cudaStream_t side[TC_SIDE] = {};
    cudaEvent_t fork = nullptr, join[TC_SIDE] = {};
    // pinned host staging buffers of finished requests, by size, reused by
    // later submissions (pinning memory costs milliseconds per call)
    std::mutex pin_mu;
    std::multimap<size_t, float *> pin_pool;
    size_t pin_pooled = 0;
    std::vector<cudaEvent_t> ev_pool;    // completion events of finished requests (also under pin_mu)
    static constexpr size_t PIN_POOL_MAX = size_t(2) << 30;
    std::vector<int> free_slots;

    double now() const {
        return std::chrono::duration<double>(std::chrono::steady_clock::now() - t0).count();
    }
};

namespace {

// Takes the server lock for an API call, counted so that the worker, which
// retakes the lock after every step, yields to it instead of starving it.
struct ApiLock {
    air_server *S;
    std::unique_lock<std::mutex> lock;
    explicit ApiLock(air_server *s) : S(s) {
        S->waiters.fetch_add(1);
        lock = std::unique_lock<std::mutex>(S->mu);
        S->waiters.fetch_sub(1);
    }
};

// A pinned host buffer of `bytes` from the pool, or a new one.
cudaError_t pin_take(air_server *S, size_t bytes, float **out) {
    {
        std::lock_guard<std::mutex> lock(S->pin_mu);
        auto it = S->pin_pool.find(bytes);
        if (it != S->pin_pool.end()) {
            *out = it->second;
            S->pin_pooled -= bytes;
            S->pin_pool.erase(it);
            return cudaSuccess;
        }
    }
    return cudaMallocHost((void **)out, bytes);
}

// Returns a pinned buffer to the pool (freed instead when the pool is full).
void pin_give(air_server *S, size_t bytes, float *p) {
    if (!p) return;
    {
        std::lock_guard<std::mutex> lock(S->pin_mu);
        if (S->pin_pooled + bytes <= air_server::PIN_POOL_MAX) {
            S->pin_pool.emplace(bytes, p);
            S->pin_pooled += bytes;
            return;
        }
    }
    cudaFreeHost(p);
}

// Takes an idle plan of this geometry from the pool, or creates one.
air_status get_plan(air_server *S, const air_geometry &g, air_plan **out) {
    for (size_t i = 0; i < S->pool.size(); ++i)
        if (same_geom(S->pool[i].first, g)) {
            *out = S->pool[i].second;
            S->pooled -= air_plan_bytes(*out);
            S->pool.erase(S->pool.begin() + i);
            return AIR_OK;
        }
    return air_plan_create(&g, out);
}

void put_plan(air_server *S, air_plan *p) {
    S->pool.push_back({p->geom, p});
    S->pooled += air_plan_bytes(p);
}

// Frees idle pooled plans until `need` more bytes fit the budget.
void trim_pool(air_server *S, size_t need) {
    while (!S->pool.empty() && S->used + S->pooled + need > S->budget) {
        air_plan *p = S->pool.front().second;
        S->pooled -= air_plan_bytes(p);
        S->pool.erase(S->pool.begin());
        air_plan_destroy(p);
    }
}

void finish(air_server *S, Request *r, air_status st) {
    r->status = st;
    r->state = st == AIR_OK ? DONE : FAILED;
    r->t[2] = S->now();
    if (r->plan) {
        S->used -= r->bytes;
        put_plan(S, r->plan);
        r->plan = nullptr;
    }
    if (r->slot >= 0) S->free_slots.push_back(r->slot);
    r->slot = -1;
    S->cv_done.notify_all();
}

// Device bytes of a plan of this geometry: measured once a plan of it has
// been built, the estimate before.
size_t request_bytes(const air_server *S, const air_geometry &g) {
    for (const auto &kv : S->plan_bytes)
        if (same_geom(kv.first, g)) return kv.second;
    return plan_bytes_estimate(g);
}

// Admission at a step boundary (called with the lock held).  A request is
// charged the bytes of the plan it is given, which are known exactly once
// the plan exists: a request whose estimate fitted but whose plan does not
// waits with the plan pooled, and one whose plan alone exceeds the budget
// fails with AIR_ERR_BUDGET.
void admit(air_server *S) {
    while (!S->queue.empty() && !S->free_slots.empty()) {
        Request *r = S->queue.front();
        r->bytes = request_bytes(S, r->geom);
        if (S->used + r->bytes > S->budget) break;       // FIFO: wait for memory
        trim_pool(S, r->bytes);
        air_plan *plan = nullptr;
        air_status st = get_plan(S, r->geom, &plan);
        if (st != AIR_OK) {
            S->queue.pop_front();
            finish(S, r, st);
            continue;
        }
        const size_t actual = air_plan_bytes(plan);
        if (!std::any_of(S->plan_bytes.begin(), S->plan_bytes.end(),
                         [&](const auto &kv) { return same_geom(kv.first, r->geom); }))
            S->plan_bytes.push_back({r->geom, actual});
        if (S->used + actual > S->budget) {
            r->bytes = actual;
            if (actual > S->budget) {                     // can never fit
                air_plan_destroy(plan);
                S->queue.pop_front();
                finish(S, r, fail(AIR_ERR_BUDGET, "the request's plan needs more device bytes than the budget"));
                continue;
            }
            put_plan(S, plan);                             // wait for memory with the plan pooled
            break;
        }
        S->queue.pop_front();
        if (!r->done_ev) {
            {
                std::lock_guard<std::mutex> lock(S->pin_mu);
                if (!S->ev_pool.empty()) {
                    r->done_ev = S->ev_pool.back();
                    S->ev_pool.pop_back();
                }
            }
            if (!r->done_ev) {
                const cudaError_t ee = cudaEventCreateWithFlags(&r->done_ev, cudaEventDisableTiming);
                if (ee != cudaSuccess) {
                    r->done_ev = nullptr;
                    put_plan(S, plan);
                    finish(S, r, fail(AIR_ERR_CUDA, std::string("server event: ") + cudaGetErrorString(ee)));
                    continue;
                }
            }
        }
        r->plan = plan;
        r->bytes = actual;
        S->used += r->bytes;
        r->slot = S->free_slots.back();
        S->free_slots.pop_back();
        const bool tc = r->geom.precision == AIR_PREC_BF16X3 && r->geom.filter == AIR_FILTER_RAMLAK;
        r->prog = solve_program(r->n_outer, r->n_cg, tc);
        r->pc = 0;
        const size_t sino = (size_t)r->geom.n_views * r->geom.n_bins * 4;
        S->h_slices[r->slot] = solve_desc(plan, plan->ybuf, r->lam, r->mu, plan->xbuf, nullptr);
        cudaError_t e = cudaMemcpyAsync(plan->ybuf, r->y_pinned, sino, cudaMemcpyHostToDevice, S->stream);
        if (e == cudaSuccess)
            e = cudaMemcpyAsync(S->d_slices + r->slot, S->h_slices + r->slot, sizeof(SliceDesc),
                                cudaMemcpyHostToDevice, S->stream);
        if (e != cudaSuccess) {
            finish(S, r, fail(AIR_ERR_CUDA, std::string("server admission copy: ") + cudaGetErrorString(e)));
            continue;
        }
        r->state = ACTIVE;
        r->t[1] = S->now();
        S->active.push_back(r);
    }
}

// The end of a step: its ring event, then every active request advances
// one phase, and one past its last phase copies its image out.
air_status finish_step(air_server *S, int k) {
    cudaEventRecord(S->ring_ev[k], S->stream);
    for (Request *r : S->active) {
        if (r->state != ACTIVE) continue;
        if (++r->pc == r->prog.size()) {
            const size_t img = (size_t)r->geom.n * r->geom.n * 4;
            cudaError_t e = cudaMemcpyAsync(r->x_pinned, r->plan->xbuf, img, cudaMemcpyDeviceToHost, S->stream);
            if (e == cudaSuccess) e = cudaEventRecord(r->done_ev, S->stream);
            if (e != cudaSuccess) return fail(AIR_ERR_CUDA, std::string("server copy-out: ") + cudaGetErrorString(e));
            r->state = FINISHING;
        }
    }
    return AIR_OK;
}

// Enqueues one step: every active request advances one phase.
air_status enqueue_step(air_server *S) {
    const int k = S->ring_pos;
    S->ring_pos = (S->ring_pos + 1) % RING;
    cudaEventSynchronize(S->ring_ev[k]);              // this ring entry's previous step has run
    Task *ht = S->h_tasks + (size_t)k * S->max_slots;
    Task *dt = S->d_tasks + (size_t)k * S->max_slots;
    // group the active requests' current phases by op
    std::map<int, std::vector<Request *>> by_op;
    for (Request *r : S->active)
        if (r->state == ACTIVE && r->pc < r->prog.size()) by_op[r->prog[r->pc].op].push_back(r);
    struct L { int op, off, n, tiles; size_t smem; };
    std::vector<L> launches;
    int nt = 0;
    for (auto &kv : by_op) {
        if (kv.first == OP_NOP || kv.first == OP_RAMP_TC) continue;
        L l{kv.first, nt, 0, 0, 0};
        for (Request *r : kv.second) {
            const SliceDesc &sd = S->h_slices[r->slot];
            const int t = tiles_of(sd, kv.first);
            if (t <= 0) continue;
            ht[nt++] = Task{r->slot, kv.first, r->prog[r->pc].arg, l.tiles};
            l.tiles += t;
            l.smem = std::max(l.smem, tile_smem(sd, kv.first));
        }
        l.n = nt - l.off;
        if (l.n > 0) launches.push_back(l);
    }
    // The requests of a step are at different phases (they arrived at
    // different times), so a step is one grouped launch per op present, each
    // over few requests, plus a tensor-core filter per BF16X3 request in a
    // filter phase.  Every request is in exactly one of them, so they are
    // independent: they fork onto the side streams and run concurrently, and
    // the step's ring event follows the join.
    cudaError_t e = cudaSuccess;
    if (nt > 0) e = cudaMemcpyAsync(dt, ht, nt * sizeof(Task), cudaMemcpyHostToDevice, S->stream);
    auto it = by_op.find(OP_RAMP_TC);
    const size_t ntc = it != by_op.end() ? it->second.size() : 0;
    if (launches.size() + ntc == 1) {
        // one launch (every resident request in the same phase, not a
        // tensor-core filter): no other launch to overlap with, so it goes
        // on the server's stream without the fork and join
        if (e == cudaSuccess && !launches.empty()) {
            const L &l = launches[0];
            e = launch_group(l.op, S->d_slices, dt + l.off, l.n, l.tiles, l.smem, S->stream);
        }
        if (e != cudaSuccess) return fail(AIR_ERR_CUDA, std::string("server step: ") + cudaGetErrorString(e));
        air_status st1 = AIR_OK;
        if (ntc == 1) {
            Request *r = it->second[0];
            const SliceDesc &sd = S->h_slices[r->slot];
            const int arg = r->prog[r->pc].arg;
            st1 = ramp_tc_apply(r->plan, arg == RSRC_Y ? sd.y : sd.z, sd.zc, sd.cg, arg == RSRC_Z, S->stream);
        }
        if (st1 != AIR_OK) return st1;
        return finish_step(S, k);
    }
    const int nside = (int)std::min<size_t>(air_server::TC_SIDE, launches.size() + ntc);
    if (e == cudaSuccess) e = cudaEventRecord(S->fork, S->stream);
    for (int q = 0; q < nside && e == cudaSuccess; ++q) e = cudaStreamWaitEvent(S->side[q], S->fork, 0);
    if (e != cudaSuccess) return fail(AIR_ERR_CUDA, std::string("server step: ") + cudaGetErrorString(e));
    int q = 0;
    air_status st = AIR_OK;
    for (const L &l : launches) {
        e = launch_group(l.op, S->d_slices, dt + l.off, l.n, l.tiles, l.smem, S->side[q++ % nside]);
        if (e != cudaSuccess) {
            st = fail(AIR_ERR_CUDA, std::string("server step: ") + cudaGetErrorString(e));
            break;
        }
    }
    for (size_t i = 0; i < ntc && st == AIR_OK; ++i) {
        Request *r = it->second[i];
        const SliceDesc &sd = S->h_slices[r->slot];
        const int arg = r->prog[r->pc].arg;
        st = ramp_tc_apply(r->plan, arg == RSRC_Y ? sd.y : sd.z, sd.zc, sd.cg, arg == RSRC_Z, S->side[q++ % nside]);
    }
    for (int k2 = 0; k2 < nside; ++k2) {       // join even after a failure: the stream stays ordered
        cudaEventRecord(S->join[k2], S->side[k2]);
        cudaStreamWaitEvent(S->stream, S->join[k2], 0);
    }
    if (st != AIR_OK) return st;
    return finish_step(S, k);
}

void worker_main(air_server *S) {
    cudaSetDevice(S->device);
    std::unique_lock<std::mutex> lock(S->mu);
    for (;;) {
        // retire finished requests
        for (size_t i = 0; i < S->active.size();) {
            Request *r = S->active[i];
            if (r->state == FINISHING && cudaEventQuery(r->done_ev) == cudaSuccess) {
                air_status st = AIR_OK;
                if (r->plan->tc && ramp_tc_status(r->plan) != 0) st = AIR_ERR_TIMEOUT;
                finish(S, r, st);
                S->active.erase(S->active.begin() + i);
            } else {
                ++i;
            }
        }
        if (!S->stop) admit(S);
        bool any_active = false, any_running = false;
        for (Request *r : S->active) {
            any_active = true;
            any_running |= r->state == ACTIVE;
        }
        if (!any_active) {
            if (S->stop) break;
            if (S->queue.empty()) S->cv_work.wait_for(lock, std::chrono::milliseconds(20));
            continue;
        }
        if (!any_running) {        // only copies in flight: wait briefly for them
            lock.unlock();
            std::this_thread::sleep_for(std::chrono::microseconds(50));
            lock.lock();
            continue;
        }
        // the step is enqueued without the lock: only this thread touches
        // the active requests, and the wait on the task ring may block
        lock.unlock();
        air_status st = enqueue_step(S);
        for (int y = 0; y < 64 && S->waiters.load() > 0; ++y) std::this_thread::yield();
        lock.lock();
        if (st != AIR_OK) {
            cudaStreamSynchronize(S->stream);
            for (Request *r : S->active) finish(S, r, st);
            S->active.clear();
        }
    }
    cudaStreamSynchronize(S->stream);
}

}  // namespace

extern "C" air_status air_server_create(size_t hbm_budget_bytes, int max_slots, air_server **out) {
    if (!out) return fail(AIR_ERR_INVALID_ARG, "out is NULL");
    *out = nullptr;
    if (hbm_budget_bytes == 0) return fail(AIR_ERR_INVALID_ARG, "hbm_budget_bytes must be > 0");
    if (max_slots < 1 || max_slots > 4096) return fail(AIR_ERR_INVALID_ARG, "max_slots must be in 1..4096");
    auto S = std::make_unique<air_server>();
    S->budget = hbm_budget_bytes;
    S->max_slots = max_slots;
    S->t0 = std::chrono::steady_clock::now();
    cudaError_t e = cudaGetDevice(&S->device);
    if (e == cudaSuccess) e = cudaStreamCreateWithFlags(&S->stream, cudaStreamNonBlocking);
    if (e == cudaSuccess) e = cudaMalloc(&S->d_slices, sizeof(SliceDesc) * max_slots);
    if (e == cudaSuccess) e = cudaMalloc(&S->d_tasks, sizeof(Task) * max_slots * RING);
    if (e == cudaSuccess) e = cudaMallocHost(&S->h_slices, sizeof(SliceDesc) * max_slots);
    if (e == cudaSuccess) e = cudaMallocHost(&S->h_tasks, sizeof(Task) * max_slots * RING);
    for (int k = 0; k < RING && e == cudaSuccess; ++k) e = cudaEventCreateWithFlags(&S->ring_ev[k], cudaEventDisableTiming);
    if (e == cudaSuccess) e = cudaEventCreateWithFlags(&S->fork, cudaEventDisableTiming);
    for (int q = 0; q < air_server::TC_SIDE && e == cudaSuccess; ++q) {
        e = cudaStreamCreateWithFlags(&S->side[q], cudaStreamNonBlocking);
        if (e == cudaSuccess) e = cudaEventCreateWithFlags(&S->join[q], cudaEventDisableTiming);
    }
    if (e != cudaSuccess) {
        cudaGetLastError();
        return fail(AIR_ERR_CUDA, std::string("server creation: ") + cudaGetErrorString(e));
    }
    for (int i = max_slots - 1; i >= 0; --i) S->free_slots.push_back(i);
    air_server *raw = S.release();
    raw->worker = std::thread(worker_main, raw);
    *out = raw;
    return AIR_OK;
}

extern "C" air_status air_server_submit(air_server *S, const air_geometry *geom, const float *Y_host, float lambda,
                                        float mu, int n_outer, int n_cg, uint64_t *request_id) {
    if (!S || !request_id || !Y_host) return fail(AIR_ERR_INVALID_ARG, "NULL argument");
    air_status st = validate_geometry(geom);
    if (st != AIR_OK) return st;
    if (!(mu > 0.f) || !(lambda >= 0.f) || n_outer < 0 || n_cg < 0 || n_outer > 100000 || n_cg > 100000)
        return fail(AIR_ERR_INVALID_ARG, "lambda >= 0, mu > 0 and 0 <= n_outer, n_cg <= 100000 are required");
    auto r = std::make_unique<Request>();
    r->geom = *geom;
    r->lam = lambda;
    r->mu = mu;
    r->n_outer = n_outer;
    r->n_cg = n_cg;
    r->t[0] = S->now();              // arrival: when the caller submits
    r->bytes = plan_bytes_estimate(*geom);
    if (r->bytes > S->budget)
        return fail(AIR_ERR_BUDGET, "the request needs " + std::to_string(r->bytes) +
                                        " device bytes, more than the server's budget");
    const size_t sino = (size_t)geom->n_views * geom->n_bins * 4, img = (size_t)geom->n * geom->n * 4;
    // no CUDA call on this path when the pools hold buffers of these sizes:
    // the worker creates or reuses the completion event at admission
    cudaError_t e = pin_take(S, sino, &r->y_pinned);
    if (e == cudaSuccess) e = pin_take(S, img, &r->x_pinned);
    if (e != cudaSuccess) {
        pin_give(S, sino, r->y_pinned);
        pin_give(S, img, r->x_pinned);
        cudaGetLastError();
        return fail(AIR_ERR_OOM, std::string("pinned host buffers: ") + cudaGetErrorString(e));
    }
    std::memcpy(r->y_pinned, Y_host, sino);
    ApiLock lock(S);
    if (S->stop) return fail(AIR_ERR_INVALID_ARG, "the server is shutting down");
    r->id = S->next_id++;
    *request_id = r->id;
    S->queue.push_back(r.get());
    S->all[r->id] = std::move(r);
    S->cv_work.notify_all();
    return AIR_OK;
}

namespace {
air_status take_result(air_server *S, std::map<uint64_t, std::unique_ptr<Request>>::iterator it, float *X_host) {
    Request *r = it->second.get();
    const air_status st = r->status;
    if (st == AIR_OK && X_host) std::memcpy(X_host, r->x_pinned, (size_t)r->geom.n * r->geom.n * 4);
    pin_give(S, (size_t)r->geom.n_views * r->geom.n_bins * 4, r->y_pinned);
    pin_give(S, (size_t)r->geom.n * r->geom.n * 4, r->x_pinned);
    if (r->done_ev) {
        std::lock_guard<std::mutex> lock(S->pin_mu);
        S->ev_pool.push_back(r->done_ev);
    }
    S->all.erase(it);
    return st == AIR_OK ? AIR_OK : fail(st, "the request failed");
}
}  // namespace

extern "C" air_status air_server_poll(air_server *S, uint64_t id, float *X_host) {
    if (!S) return fail(AIR_ERR_INVALID_ARG, "server is NULL");
    ApiLock lock(S);
    auto it = S->all.find(id);
    if (it == S->all.end()) return fail(AIR_ERR_INVALID_ARG, "unknown request id");
    const int state = it->second->state;
    if (state != DONE && state != FAILED) return AIR_ERR_NOT_READY;
    return take_result(S, it, X_host);
}

extern "C" air_status air_server_wait(air_server *S, uint64_t id, float *X_host) {
    if (!S) return fail(AIR_ERR_INVALID_ARG, "server is NULL");
    ApiLock al(S);
    auto it = S->all.find(id);
    if (it == S->all.end()) return fail(AIR_ERR_INVALID_ARG, "unknown request id");
    Request *r = it->second.get();
    S->cv_done.wait(al.lock, [&] { return r->state == DONE || r->state == FAILED; });
    return take_result(S, S->all.find(id), X_host);
}

extern "C" air_status air_server_times(air_server *S, uint64_t id, double t[3]) {
    if (!S || !t) return fail(AIR_ERR_INVALID_ARG, "NULL argument");
    ApiLock lock(S);
    auto it = S->all.find(id);
    if (it == S->all.end()) return fail(AIR_ERR_INVALID_ARG, "unknown request id");
    const Request *r = it->second.get();
    if (r->state != DONE && r->state != FAILED) return AIR_ERR_NOT_READY;
    for (int i = 0; i < 3; ++i) t[i] = r->t[i];
    return AIR_OK;
}

extern "C" air_status air_server_destroy(air_server *S) {
    if (!S) return AIR_OK;
    {
        std::lock_guard<std::mutex> lock(S->mu);
        S->stop = true;
        // requests never admitted are dropped
        for (Request *r : S->queue) {
            r->state = FAILED;
            r->status = AIR_ERR_NOT_READY;
        }
        S->queue.clear();
        S->cv_work.notify_all();
        S->cv_done.notify_all();
    }
    if (S->worker.joinable()) S->worker.join();
    for (auto &pp : S->pool) air_plan_destroy(pp.second);
    for (auto &kv : S->all) {
        cudaFreeHost(kv.second->y_pinned);
        cudaFreeHost(kv.second->x_pinned);
        if (kv.second->done_ev) cudaEventDestroy(kv.second->done_ev);
    }
    for (auto &pp : S->pin_pool) cudaFreeHost(pp.second);
    for (cudaEvent_t ev : S->ev_pool) cudaEventDestroy(ev);
    for (int k = 0; k < RING; ++k)
        if (S->ring_ev[k]) cudaEventDestroy(S->ring_ev[k]);
    for (int q = 0; q < air_server::TC_SIDE; ++q) {
        if (S->side[q]) cudaStreamDestroy(S->side[q]);
        if (S->join[q]) cudaEventDestroy(S->join[q]);
    }
    if (S->fork) cudaEventDestroy(S->fork);
    cudaFree(S->d_slices);
    cudaFree(S->d_tasks);
    cudaFreeHost(S->h_slices);
    cudaFreeHost(S->h_tasks);
    cudaStreamDestroy(S->stream);
    delete S;
    return AIR_OK;
}
