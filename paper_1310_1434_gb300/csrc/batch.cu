// Batched solves of many independent slices of uneven geometry.
//
// air_solve_batch: the split-Bregman programs of all slices advance phase by
// phase; each phase is one grouped launch of that op's kernel over the tiles
// of every slice (plus the tensor-core filter of each BF16X3 slice), and the
// whole sequence is captured once per batch composition into a CUDA graph
// that later calls replay.
//
// air_solve_batch_persistent: the same programs in ONE persistent
// cooperative kernel (k_persistent) that runs every phase with a bounded grid
// barrier in between, also captured in a graph.  It has one register and
// shared-memory budget for every op, which costs occupancy on the projector
// pair; it is kept for callers that want a single launch.
#include <algorithm>
#include <cmath>
#include <climits>
#include <cstring>
#include <map>
#include <mutex>
#include <vector>

#include "host_common.h"
#include "ramp_tc.h"
#include "tiles.cuh"

using namespace air;

namespace {

// Side streams the tensor-core filters of one phase fork onto during capture
// (each slice's filter is a small GEMM that fills part of the GPU alone).
constexpr int TC_SIDE = 8;
// Independent chains a grouped batch may be captured as: slice i runs in
// chain i mod CHAINS, each chain its phases in order on a stream of its own,
// so that one chain's launches fill the partly empty last waves of the
// other's.  Whether that pays depends on the launches (chains of short
// launches gain, chains of long ones slow each other down), so the first
// call of a batch times the one-chain and the two-chain graph and keeps the
// faster.  A batch whose backprojector phase takes more than CHAIN_WAVES
// waves of the device is not tried in two chains.
constexpr int CHAINS = 2;
constexpr double CHAIN_WAVES = 64.0;

struct BatchGraph {
    std::vector<uintptr_t> key;
    cudaStream_t cap = nullptr;     // private stream the graph is captured on
    cudaStream_t chain[CHAINS] = {};   // chain 0 is cap
    cudaEvent_t start = nullptr, done[CHAINS] = {};
    cudaStream_t side[TC_SIDE] = {};
    cudaEvent_t fork = nullptr, join[TC_SIDE] = {};
    cudaGraphExec_t exec = nullptr;
    char *dmem = nullptr;
    BatchCtl *ctl = nullptr;
    std::vector<const air_plan *> tc_plans;   // plans whose status is checked after a run
    int chains = 1;                 // of the grouped graph in use
    long long kernels = 0;          // kernels one run of it launches
};

std::mutex g_batch_mu;
BatchGraph g_grouped, g_persistent;

void release(BatchGraph &b) {
    if (b.exec) cudaGraphExecDestroy(b.exec);
    if (b.dmem) cudaFree(b.dmem);
    BatchGraph keep;   // the capture streams and events outlive a graph
    keep.cap = b.cap;
    keep.fork = b.fork;
    keep.start = b.start;
    for (int c = 0; c < CHAINS; ++c) {
        keep.chain[c] = b.chain[c];
        keep.done[c] = b.done[c];
    }
    for (int i = 0; i < TC_SIDE; ++i) {
        keep.side[i] = b.side[i];
        keep.join[i] = b.join[i];
    }
    b = keep;
}

cudaError_t make_side_streams(BatchGraph &b) {
    cudaError_t e = cudaSuccess;
    if (!b.fork) e = cudaEventCreateWithFlags(&b.fork, cudaEventDisableTiming);
    if (e == cudaSuccess && !b.start) e = cudaEventCreateWithFlags(&b.start, cudaEventDisableTiming);
    for (int c = 1; c < CHAINS && e == cudaSuccess; ++c) {
        if (!b.chain[c]) e = cudaStreamCreateWithFlags(&b.chain[c], cudaStreamNonBlocking);
        if (e == cudaSuccess && !b.done[c]) e = cudaEventCreateWithFlags(&b.done[c], cudaEventDisableTiming);
    }
    for (int i = 0; i < TC_SIDE && e == cudaSuccess; ++i) {
        if (!b.side[i]) e = cudaStreamCreateWithFlags(&b.side[i], cudaStreamNonBlocking);
        if (e == cudaSuccess && !b.join[i]) e = cudaEventCreateWithFlags(&b.join[i], cudaEventDisableTiming);
    }
    return e;
}

struct Batch {
    std::vector<SliceDesc> slices;
    std::vector<std::vector<Phase>> progs;
    size_t nphases = 0;
    std::vector<uintptr_t> key;
};

air_status prepare(int n, air_plan *const *plans, const float *const *Y, const float *lambda, const float *mu,
                   const int *n_outer, const int *n_cg, float *const *X, cudaStream_t st, bool allow_tc, Batch *B) {
    if (n < 1 || n > 4096) return fail(AIR_ERR_INVALID_ARG, "n must be in 1..4096");
    if (!plans || !Y || !lambda || !mu || !n_outer || !n_cg || !X)
        return fail(AIR_ERR_INVALID_ARG, "NULL array argument");
    B->slices.resize(n);
    B->progs.resize(n);
    for (int i = 0; i < n; ++i) {
        air_status s = check_solve_args(plans[i], Y[i], lambda[i], mu[i], n_outer[i], n_cg[i], X[i]);
        if (s != AIR_OK) return s;
        if ((s = check_dev_ptr(Y[i], "Y[i]")) != AIR_OK) return s;
        if ((s = check_dev_ptr(X[i], "X[i]")) != AIR_OK) return s;
        for (int k = 0; k < i; ++k)
            if (plans[k] == plans[i]) return fail(AIR_ERR_INVALID_ARG, "plans of a batch must be distinct");
        const bool tc = plans[i]->geom.precision == AIR_PREC_BF16X3 && plans[i]->geom.filter == AIR_FILTER_RAMLAK;
        if (tc && !allow_tc)
            return fail(AIR_ERR_INVALID_ARG, "the persistent batch runs the FP32 filter; use FP32 plans");
        B->slices[i] = solve_desc(plans[i], Y[i], lambda[i], mu[i], X[i], nullptr);
        B->progs[i] = solve_program(n_outer[i], n_cg[i], tc);
        B->nphases = std::max(B->nphases, B->progs[i].size());
    }
    int dev = 0;
    cudaGetDevice(&dev);
    B->key.push_back((uintptr_t)dev);
    B->key.push_back((uintptr_t)st);
    for (int i = 0; i < n; ++i) {
        uint32_t lb, mb;
        std::memcpy(&lb, &lambda[i], 4);
        std::memcpy(&mb, &mu[i], 4);
        B->key.insert(B->key.end(), {(uintptr_t)plans[i], (uintptr_t)Y[i], (uintptr_t)X[i], (uintptr_t)lb,
                                     (uintptr_t)mb, (uintptr_t)n_outer[i], (uintptr_t)n_cg[i]});
    }
    return AIR_OK;
}

// After a run on st: waits for it, then reads the persistent kernel's barrier
// status and every tensor-core plan's status.
air_status finish_run(BatchGraph &G, cudaStream_t st) {
    cudaError_t e = cudaSuccess;
    BatchCtl ctl{};
    if (G.ctl) e = cudaMemcpyAsync(&ctl, G.ctl, sizeof(BatchCtl), cudaMemcpyDeviceToHost, st);
    if (e == cudaSuccess) e = cudaStreamSynchronize(st);
    if (e != cudaSuccess) return fail(AIR_ERR_CUDA, std::string("batch solve: ") + cudaGetErrorString(e));
    if (ctl.error != 0) return fail(AIR_ERR_TIMEOUT, "a grid barrier of the batch kernel timed out");
    // every tensor-core plan's status is read (which clears it), the first
    // failure reported
    air_status first = AIR_OK;
    for (const air_plan *p : G.tc_plans) {
        const air_status s = air_plan_status(p);
        if (first == AIR_OK && s != AIR_OK) first = s;
    }
    return first == AIR_OK ? AIR_OK : fail(first, "a bounded wait in a slice's tensor-core filter gave up");
}

air_status run_cached(BatchGraph &G, cudaStream_t st) {
    cudaError_t e = cudaGraphLaunch(G.exec, st);
    if (e != cudaSuccess) return fail(AIR_ERR_CUDA, std::string("batch graph launch: ") + cudaGetErrorString(e));
    return finish_run(G, st);
}

// One launch of the grouped form: an op over some slices' tiles, or one
// slice's tensor-core filter.
struct Launch { int op, off, ntasks, tiles; size_t smem; int slice, arg; };

// The launch lists of the batch split into nch chains (slice i in chain
// i mod nch), phase by phase one task list per op present; the tasks are
// appended to `tasks`.
void plan_chains(const Batch &B, int n, int nch, std::vector<Task> &tasks, std::vector<Launch> *launches) {
    for (int c = 0; c < nch; ++c) {
        for (size_t ph = 0; ph < B.nphases; ++ph) {
            std::map<int, std::vector<int>> by_op;   // op -> slices of the chain
            for (int i = c; i < n; i += nch)
                if (ph < B.progs[i].size()) by_op[B.progs[i][ph].op].push_back(i);
            for (auto &kv : by_op) {
                const int op = kv.first;
                if (op == OP_NOP) continue;
                if (op == OP_RAMP_TC) {   // the tensor-core filter, slice by slice
                    for (int i : kv.second) launches[c].push_back({op, 0, 0, 0, 0, i, B.progs[i][ph].arg});
                    continue;
                }
                Launch L{op, (int)tasks.size(), 0, 0, 0, -1, 0};
                for (int i : kv.second) {
                    const int t = tiles_of(B.slices[i], op);
                    if (t <= 0) continue;
                    tasks.push_back({i, op, B.progs[i][ph].arg, L.tiles});
                    L.tiles += t;
                    L.smem = std::max(L.smem, tile_smem(B.slices[i], op));
                }
                L.ntasks = (int)tasks.size() - L.off;
                if (L.ntasks > 0) launches[c].push_back(L);
            }
        }
    }
}

// Captures the chains' launch lists (each chain on a stream of its own with
// its share of the filter side streams, all joined at the end) and
// instantiates them into *exec.
air_status capture_chains(BatchGraph &G, const Batch &B, air_plan *const *plans, int nch,
                          const std::vector<Launch> *launches, const SliceDesc *d_slices, const Task *d_tasks,
                          cudaGraphExec_t *exec, long long *kernels) {
    *exec = nullptr;
    *kernels = 0;
    cudaError_t e = cudaStreamBeginCapture(G.cap, cudaStreamCaptureModeThreadLocal);
    if (e != cudaSuccess) return fail(AIR_ERR_CUDA, std::string("batch set-up: ") + cudaGetErrorString(e));
    const cudaStream_t cs = G.cap;
    G.chain[0] = cs;
    cudaError_t le = cudaEventRecord(G.start, cs);
    std::string tc_msg;
    for (int c = 0; c < nch && le == cudaSuccess && tc_msg.empty(); ++c) {
        const cudaStream_t ch = G.chain[c];
        if (c > 0) le = cudaStreamWaitEvent(ch, G.start, 0);
        const int s0 = c * TC_SIDE / nch, ns = (c + 1) * TC_SIDE / nch - s0;   // the chain's side streams
        const std::vector<Launch> &ls = launches[c];
        for (size_t li = 0; li < ls.size() && le == cudaSuccess && tc_msg.empty(); ++li) {
            const Launch &L = ls[li];
            if (L.op != OP_RAMP_TC) {
                le = launch_group(L.op, d_slices, d_tasks + L.off, L.ntasks, L.tiles, L.smem, ch);
                *kernels += 1;
                continue;
            }
            // a run of tensor-core filters (one phase, one per BF16X3 slice):
            // fork them onto the side streams and join them back
            size_t end = li;
            while (end < ls.size() && ls[end].op == OP_RAMP_TC && (end == li || ls[end].slice > ls[end - 1].slice))
                ++end;
            const int nside = (int)std::min<size_t>(ns, end - li);
            le = cudaEventRecord(G.fork, ch);
            for (int k = 0; k < nside && le == cudaSuccess; ++k) le = cudaStreamWaitEvent(G.side[s0 + k], G.fork, 0);
            for (size_t q = li; q < end && le == cudaSuccess && tc_msg.empty(); ++q) {
                const Launch &T = ls[q];
                const SliceDesc &sd = B.slices[T.slice];
                const float *src = T.arg == RSRC_Y ? sd.y : sd.z;
                if (ramp_tc_apply(plans[T.slice], src, sd.zc, sd.cg, T.arg == RSRC_Z,
                                  G.side[s0 + (int)((q - li) % nside)]) != AIR_OK)
                    tc_msg = air_last_error();
                *kernels += 2;   // the split and the tensor-core product
            }
            for (int k = 0; k < nside && le == cudaSuccess; ++k) {
                le = cudaEventRecord(G.join[s0 + k], G.side[s0 + k]);
                if (le == cudaSuccess) le = cudaStreamWaitEvent(ch, G.join[s0 + k], 0);
            }
            li = end - 1;
        }
    }
    for (int c = 1; c < nch; ++c) {   // the chains join the capture stream (also after a failure)
        cudaError_t je = cudaEventRecord(G.done[c], G.chain[c]);
        if (je == cudaSuccess) je = cudaStreamWaitEvent(cs, G.done[c], 0);
        if (le == cudaSuccess) le = je;
    }
    cudaGraph_t graph = nullptr;
    e = cudaStreamEndCapture(cs, &graph);
    if (le != cudaSuccess) e = le;
    if (e == cudaSuccess && tc_msg.empty()) e = cudaGraphInstantiate(exec, graph, 0);
    if (graph) cudaGraphDestroy(graph);
    if (!tc_msg.empty()) {
        cudaGetLastError();
        return fail(AIR_ERR_CUDA, "batch graph build: " + tc_msg);
    }
    if (e != cudaSuccess) {
        cudaGetLastError();
        return fail(AIR_ERR_CUDA, std::string("batch graph build: ") + cudaGetErrorString(e));
    }
    return AIR_OK;
}

air_status end_capture(BatchGraph &G, cudaStream_t cs, cudaError_t launch_err) {
    cudaGraph_t graph = nullptr;
    cudaError_t e = cudaStreamEndCapture(cs, &graph);
    if (launch_err != cudaSuccess) e = launch_err;
    if (e == cudaSuccess) e = cudaGraphInstantiate(&G.exec, graph, 0);
    if (graph) cudaGraphDestroy(graph);
    if (e != cudaSuccess) {
        release(G);
        cudaGetLastError();
        return fail(AIR_ERR_CUDA, std::string("batch graph build: ") + cudaGetErrorString(e));
    }
    return AIR_OK;
}

}  // namespace

extern "C" air_status air_solve_batch(int n, air_plan *const *plans, const float *const *Y, const float *lambda,
                                      const float *mu, const int *n_outer, const int *n_cg, float *const *X,
                                      air_stream stream) {
    const cudaStream_t st = (cudaStream_t)stream;
    Batch B;
    air_status s = prepare(n, plans, Y, lambda, mu, n_outer, n_cg, X, st, true, &B);
    if (s != AIR_OK) return s;
    std::lock_guard<std::mutex> lock(g_batch_mu);
    BatchGraph &G = g_grouped;
    if (G.key != B.key || !G.exec) {
        release(G);
        // one chain, and two chains where the batch is small enough for them
        // to pay (see CHAINS)
        int nch = std::min(CHAINS, n);
        {
            long long bwd_tiles = 0;
            size_t bwd_smem = 0;
            for (int i = 0; i < n; ++i) {
                bwd_tiles += tiles_of(B.slices[i], OP_BWD);
                bwd_smem = std::max(bwd_smem, tile_smem(B.slices[i], OP_BWD));
            }
            const int cap = group_bwd_capacity(bwd_smem);
            if (cap <= 0 || (double)bwd_tiles > CHAIN_WAVES * cap) nch = 1;
        }
        std::vector<Task> tasks;
        std::vector<Launch> one[1], many[CHAINS];
        plan_chains(B, n, 1, tasks, one);
        if (nch > 1) plan_chains(B, n, nch, tasks, many);
        const size_t b_slices = align_up(n * sizeof(SliceDesc), 256);
        const size_t b_tasks = align_up(std::max<size_t>(tasks.size(), 1) * sizeof(Task), 256);
        if (cudaMalloc(&G.dmem, b_slices + b_tasks) != cudaSuccess) {
            cudaGetLastError();
            G.dmem = nullptr;
            return fail(AIR_ERR_OOM, "batch table allocation failed");
        }
        SliceDesc *d_slices = (SliceDesc *)G.dmem;
        Task *d_tasks = (Task *)(G.dmem + b_slices);
        cudaError_t e = cudaMemcpy(d_slices, B.slices.data(), n * sizeof(SliceDesc), cudaMemcpyHostToDevice);
        if (e == cudaSuccess && !tasks.empty())
            e = cudaMemcpy(d_tasks, tasks.data(), tasks.size() * sizeof(Task), cudaMemcpyHostToDevice);
        // captured on a private stream (the caller's may be the legacy default
        // stream, which cannot be captured); launched on the caller's stream
        if (e == cudaSuccess && !G.cap) e = cudaStreamCreateWithFlags(&G.cap, cudaStreamNonBlocking);
        if (e == cudaSuccess) e = make_side_streams(G);
        if (e != cudaSuccess) {
            release(G);
            return fail(AIR_ERR_CUDA, std::string("batch set-up: ") + cudaGetErrorString(e));
        }
        cudaGraphExec_t x1 = nullptr, xn = nullptr;
        long long k1 = 0, kn = 0;
        s = capture_chains(G, B, plans, 1, one, d_slices, d_tasks, &x1, &k1);
        if (s == AIR_OK && nch > 1) s = capture_chains(G, B, plans, nch, many, d_slices, d_tasks, &xn, &kn);
        if (s != AIR_OK) {
            if (x1) cudaGraphExecDestroy(x1);
            release(G);
            return s;
        }
        G.key = B.key;
        for (int i = 0; i < n; ++i)
            if (plans[i]->tc) G.tc_plans.push_back(plans[i]);
        G.chains = 1;
        G.kernels = k1;
        if (!xn) {
            G.exec = x1;
        } else {
            // timed runs of both forms on the caller's stream (both uploaded
            // first, so neither run pays for it): one of each, and when they
            // are within 3 % one more of each in the other order; the faster
            // form is kept.  The forms compute the same results, so the last
            // run's output is this call's.
            cudaEvent_t ev[3] = {};
            for (int k = 0; k < 3 && e == cudaSuccess; ++k) e = cudaEventCreate(&ev[k]);
            if (e == cudaSuccess) e = cudaGraphUpload(x1, st);
            if (e == cudaSuccess) e = cudaGraphUpload(xn, st);
            float tn = 0.f, t1 = 0.f;
            auto pair = [&](cudaGraphExec_t a, float *ta, cudaGraphExec_t b, float *tb) {
                float da = 0.f, db = 0.f;
                if (e == cudaSuccess) e = cudaEventRecord(ev[0], st);
                if (e == cudaSuccess) e = cudaGraphLaunch(a, st);
                if (e == cudaSuccess) e = cudaEventRecord(ev[1], st);
                if (e == cudaSuccess) e = cudaGraphLaunch(b, st);
                if (e == cudaSuccess) e = cudaEventRecord(ev[2], st);
                if (e == cudaSuccess) e = cudaEventSynchronize(ev[2]);
                if (e == cudaSuccess) e = cudaEventElapsedTime(&da, ev[0], ev[1]);
                if (e == cudaSuccess) e = cudaEventElapsedTime(&db, ev[1], ev[2]);
                *ta += da;
                *tb += db;
            };
            pair(xn, &tn, x1, &t1);
            if (e == cudaSuccess && std::fabs(tn - t1) < 0.03f * std::min(tn, t1)) pair(x1, &t1, xn, &tn);
            for (int k = 0; k < 3; ++k)
                if (ev[k]) cudaEventDestroy(ev[k]);
            G.exec = (e == cudaSuccess && tn < t1) ? xn : x1;
            cudaGraphExecDestroy(G.exec == xn ? x1 : xn);
            if (G.exec == xn) {
                G.chains = nch;
                G.kernels = kn;
            }
            if (e != cudaSuccess) return fail(AIR_ERR_CUDA, std::string("batch solve: ") + cudaGetErrorString(e));
            return finish_run(G, st);
        }
    }
    return run_cached(G, st);
}

extern "C" air_status air_solve_batch_host(int n, air_plan *const *plans, const float *const *Y_host,
                                           const float *lambda, const float *mu, const int *n_outer,
                                           const int *n_cg, float *const *X_host, air_stream stream) {
    if (n < 1 || n > 4096) return fail(AIR_ERR_INVALID_ARG, "n must be in 1..4096");
    if (!plans || !Y_host || !X_host) return fail(AIR_ERR_INVALID_ARG, "NULL array argument");
    const cudaStream_t st = (cudaStream_t)stream;
    std::vector<const float *> Yd(n);
    std::vector<float *> Xd(n);
    for (int i = 0; i < n; ++i) {
        if (!plans[i]) return fail(AIR_ERR_INVALID_ARG, "plan is NULL");
        if (!Y_host[i] || !X_host[i]) return fail(AIR_ERR_INVALID_ARG, "Y_host[i] and X_host[i] must not be NULL");
        const size_t sino = (size_t)plans[i]->geom.n_views * plans[i]->geom.n_bins * 4;
        const cudaError_t e = cudaMemcpyAsync(plans[i]->ybuf, Y_host[i], sino, cudaMemcpyHostToDevice, st);
        if (e != cudaSuccess) return fail(AIR_ERR_CUDA, std::string("batch copy-in: ") + cudaGetErrorString(e));
        Yd[i] = plans[i]->ybuf;
        Xd[i] = plans[i]->xbuf;
    }
    air_status s = air_solve_batch(n, plans, Yd.data(), lambda, mu, n_outer, n_cg, Xd.data(), stream);
    if (s != AIR_OK) return s;
    for (int i = 0; i < n; ++i) {
        const size_t img = (size_t)plans[i]->geom.n * plans[i]->geom.n * 4;
        const cudaError_t e = cudaMemcpyAsync(X_host[i], plans[i]->xbuf, img, cudaMemcpyDeviceToHost, st);
        if (e != cudaSuccess) return fail(AIR_ERR_CUDA, std::string("batch copy-out: ") + cudaGetErrorString(e));
    }
    const cudaError_t e = cudaStreamSynchronize(st);
    if (e != cudaSuccess) return fail(AIR_ERR_CUDA, std::string("batch copy-out: ") + cudaGetErrorString(e));
    return AIR_OK;
}

extern "C" air_status air_solve_batch_persistent(int n, air_plan *const *plans, const float *const *Y,
                                                 const float *lambda, const float *mu, const int *n_outer,
                                                 const int *n_cg, float *const *X, air_stream stream) {
    const cudaStream_t st = (cudaStream_t)stream;
    Batch B;
    air_status s = prepare(n, plans, Y, lambda, mu, n_outer, n_cg, X, st, false, &B);
    if (s != AIR_OK) return s;
    size_t smem = 0;
    for (int i = 0; i < n; ++i)
        for (int op : {OP_RAMP, OP_SHRINK, OP_TRANSPOSE, OP_BWD}) smem = std::max(smem, tile_smem(B.slices[i], op));
    std::vector<Phase> prog(n * B.nphases, Phase{OP_NOP, 0});
    for (int i = 0; i < n; ++i)
        std::memcpy(&prog[i * B.nphases], B.progs[i].data(), B.progs[i].size() * sizeof(Phase));
    std::lock_guard<std::mutex> lock(g_batch_mu);
    BatchGraph &G = g_persistent;
    if (G.key != B.key || !G.exec) {
        release(G);
        const int grid = persistent_grid(smem);
        if (grid <= 0) return fail(AIR_ERR_CUDA, "batch set-up: no co-resident grid for the persistent kernel");
        // per phase: prefix sums of the slices' tile counts, and the phase's
        // first ticket (earlier phases' tiles plus one closing ticket per block)
        const size_t np = B.nphases;
        std::vector<int> tile_base(np * (n + 1));
        std::vector<unsigned long long> phase_base(np);
        unsigned long long tickets = 0;
        for (size_t ph = 0; ph < np; ++ph) {
            int *tb = &tile_base[ph * (n + 1)];
            long long sum = 0;
            tb[0] = 0;
            for (int i = 0; i < n; ++i) {
                sum += tiles_of(B.slices[i], prog[i * np + ph].op);
                if (sum > INT_MAX) return fail(AIR_ERR_INVALID_ARG, "batch too large for one persistent launch");
                tb[i + 1] = (int)sum;
            }
            phase_base[ph] = tickets;
            tickets += (unsigned long long)sum + (unsigned long long)grid;
        }
        const size_t b_slices = align_up(n * sizeof(SliceDesc), 256);
        const size_t b_prog = align_up(prog.size() * sizeof(Phase), 256);
        const size_t b_tb = align_up(tile_base.size() * sizeof(int), 256);
        const size_t b_pb = align_up(phase_base.size() * sizeof(unsigned long long), 256);
        if (cudaMalloc(&G.dmem, b_slices + b_prog + b_tb + b_pb + 256) != cudaSuccess) {
            cudaGetLastError();
            G.dmem = nullptr;
            return fail(AIR_ERR_OOM, "batch table allocation failed");
        }
        SliceDesc *d_slices = (SliceDesc *)G.dmem;
        Phase *d_prog = (Phase *)(G.dmem + b_slices);
        int *d_tb = (int *)(G.dmem + b_slices + b_prog);
        unsigned long long *d_pb = (unsigned long long *)(G.dmem + b_slices + b_prog + b_tb);
        G.ctl = (BatchCtl *)(G.dmem + b_slices + b_prog + b_tb + b_pb);
        cudaError_t e = cudaMemcpy(d_slices, B.slices.data(), n * sizeof(SliceDesc), cudaMemcpyHostToDevice);
        if (e == cudaSuccess) e = cudaMemcpy(d_prog, prog.data(), prog.size() * sizeof(Phase), cudaMemcpyHostToDevice);
        if (e == cudaSuccess)
            e = cudaMemcpy(d_tb, tile_base.data(), tile_base.size() * sizeof(int), cudaMemcpyHostToDevice);
        if (e == cudaSuccess)
            e = cudaMemcpy(d_pb, phase_base.data(), phase_base.size() * sizeof(unsigned long long),
                           cudaMemcpyHostToDevice);
        if (e == cudaSuccess && !G.cap) e = cudaStreamCreateWithFlags(&G.cap, cudaStreamNonBlocking);
        if (e == cudaSuccess) e = cudaStreamBeginCapture(G.cap, cudaStreamCaptureModeThreadLocal);
        if (e != cudaSuccess) {
            release(G);
            return fail(AIR_ERR_CUDA, std::string("batch set-up: ") + cudaGetErrorString(e));
        }
        cudaError_t le = cudaMemsetAsync(G.ctl, 0, sizeof(BatchCtl), G.cap);
        if (le == cudaSuccess)
            le = launch_persistent(d_slices, n, d_prog, (int)B.nphases, d_tb, d_pb, G.ctl, grid, smem, G.cap);
        if ((s = end_capture(G, G.cap, le)) != AIR_OK) return s;
        G.key = B.key;
    }
    return run_cached(G, st);
}

extern "C" air_status air_batch_graph_info(int *chains, int64_t *kernels) {
    if (!chains && !kernels) return fail(AIR_ERR_INVALID_ARG, "both outputs are NULL");
    std::lock_guard<std::mutex> lock(g_batch_mu);
    if (!g_grouped.exec) return fail(AIR_ERR_INVALID_ARG, "no batch graph has been built");
    if (chains) *chains = g_grouped.chains;
    if (kernels) *kernels = (int64_t)g_grouped.kernels;
    return AIR_OK;
}
