// air_solve_batch: many slices of uneven geometry solved by one persistent
// cooperative kernel (k_persistent) that runs every phase of every slice's
// split-Bregman program, separated by a bounded grid barrier.  The launch is
// captured once per batch composition into a CUDA graph and replayed.
#include <cstring>
#include <mutex>
#include <vector>

#include "host_common.h"
#include "tiles.cuh"

using namespace air;

namespace {

struct BatchGraph {
    std::vector<uintptr_t> key;
    cudaStream_t cap = nullptr;     // private stream the graph is captured on
    cudaGraphExec_t exec = nullptr;
    char *dmem = nullptr;
    BatchCtl *ctl = nullptr;
    int device = -1;
};

std::mutex g_batch_mu;
BatchGraph g_batch;

void release(BatchGraph &b) {
    if (b.exec) cudaGraphExecDestroy(b.exec);
    if (b.dmem) cudaFree(b.dmem);
    cudaStream_t cap = b.cap;
    b = BatchGraph();
    b.cap = cap;
}

}  // namespace

extern "C" air_status air_solve_batch(int n, air_plan *const *plans, const float *const *Y,
                                      const float *lambda, const float *mu, const int *n_outer,
                                      const int *n_cg, float *const *X, air_stream stream) {
    if (n < 1 || n > 4096) return fail(AIR_ERR_INVALID_ARG, "n must be in 1..4096");
    if (!plans || !Y || !lambda || !mu || !n_outer || !n_cg || !X)
        return fail(AIR_ERR_INVALID_ARG, "NULL array argument");
    const cudaStream_t st = (cudaStream_t)stream;
    std::vector<SliceDesc> slices(n);
    std::vector<std::vector<Phase>> progs(n);
    size_t nphases = 0, smem = 0;
    for (int i = 0; i < n; ++i) {
        air_status s = check_solve_args(plans[i], Y[i], lambda[i], mu[i], n_outer[i], n_cg[i], X[i]);
        if (s != AIR_OK) return s;
        if ((s = check_dev_ptr(Y[i], "Y[i]")) != AIR_OK) return s;
        if ((s = check_dev_ptr(X[i], "X[i]")) != AIR_OK) return s;
        for (int k = 0; k < i; ++k)
            if (plans[k] == plans[i]) return fail(AIR_ERR_INVALID_ARG, "plans of a batch must be distinct");
        if (plans[i]->geom.precision != AIR_PREC_FP32 && plans[i]->geom.filter == AIR_FILTER_RAMLAK)
            return fail(AIR_ERR_INVALID_ARG, "air_solve_batch runs the FP32 filter; use FP32 plans");
        slices[i] = solve_desc(plans[i], Y[i], lambda[i], mu[i], X[i], nullptr);
        progs[i] = solve_program(n_outer[i], n_cg[i], false);
        nphases = std::max(nphases, progs[i].size());
        for (int op : {OP_RAMP, OP_SHRINK, OP_TRANSPOSE, OP_BWD}) smem = std::max(smem, tile_smem(slices[i], op));
    }
    std::vector<Phase> prog(n * nphases, Phase{OP_NOP, 0});
    for (int i = 0; i < n; ++i) std::memcpy(&prog[i * nphases], progs[i].data(), progs[i].size() * sizeof(Phase));

    std::vector<uintptr_t> key;
    key.reserve(8 * n + 2);
    int dev = 0;
    cudaGetDevice(&dev);
    key.push_back((uintptr_t)dev);
    key.push_back((uintptr_t)st);
    for (int i = 0; i < n; ++i) {
        uint32_t lb, mb;
        std::memcpy(&lb, &lambda[i], 4);
        std::memcpy(&mb, &mu[i], 4);
        key.insert(key.end(), {(uintptr_t)plans[i], (uintptr_t)Y[i], (uintptr_t)X[i], (uintptr_t)lb,
                               (uintptr_t)mb, (uintptr_t)n_outer[i], (uintptr_t)n_cg[i]});
    }

    std::lock_guard<std::mutex> lock(g_batch_mu);
    if (g_batch.key != key || !g_batch.exec) {
        release(g_batch);
        const size_t b_slices = align_up(n * sizeof(SliceDesc), 256);
        const size_t b_prog = align_up(prog.size() * sizeof(Phase), 256);
        char *dmem = nullptr;
        if (cudaMalloc(&dmem, b_slices + b_prog + 256) != cudaSuccess) {
            cudaGetLastError();
            return fail(AIR_ERR_OOM, "batch table allocation failed");
        }
        g_batch.dmem = dmem;
        SliceDesc *d_slices = (SliceDesc *)dmem;
        Phase *d_prog = (Phase *)(dmem + b_slices);
        g_batch.ctl = (BatchCtl *)(dmem + b_slices + b_prog);
        cudaError_t e = cudaMemcpy(d_slices, slices.data(), n * sizeof(SliceDesc), cudaMemcpyHostToDevice);
        if (e == cudaSuccess) e = cudaMemcpy(d_prog, prog.data(), prog.size() * sizeof(Phase), cudaMemcpyHostToDevice);
        const int grid = persistent_grid(smem);
        if (e == cudaSuccess && grid <= 0) e = cudaErrorInvalidConfiguration;
        // captured on a private stream (the caller's may be the legacy default
        // stream, which cannot be captured); launched on the caller's stream
        if (e == cudaSuccess && !g_batch.cap) e = cudaStreamCreateWithFlags(&g_batch.cap, cudaStreamNonBlocking);
        const cudaStream_t cs = g_batch.cap;
        cudaGraph_t graph = nullptr;
        if (e == cudaSuccess) e = cudaStreamBeginCapture(cs, cudaStreamCaptureModeThreadLocal);
        if (e == cudaSuccess) {
            cudaError_t e1 = cudaMemsetAsync(g_batch.ctl, 0, sizeof(BatchCtl), cs);
            cudaError_t e2 = e1 == cudaSuccess
                                 ? launch_persistent(d_slices, n, d_prog, (int)nphases, g_batch.ctl, grid, smem, cs)
                                 : e1;
            e = cudaStreamEndCapture(cs, &graph);
            if (e2 != cudaSuccess) e = e2;
        }
        if (e == cudaSuccess) e = cudaGraphInstantiate(&g_batch.exec, graph, 0);
        if (graph) cudaGraphDestroy(graph);
        if (e != cudaSuccess) {
            release(g_batch);
            cudaGetLastError();
            return fail(AIR_ERR_CUDA, std::string("batch graph build: ") + cudaGetErrorString(e));
        }
        g_batch.key = key;
        g_batch.device = dev;
    }
    cudaError_t e = cudaGraphLaunch(g_batch.exec, st);
    if (e != cudaSuccess) return fail(AIR_ERR_CUDA, std::string("batch graph launch: ") + cudaGetErrorString(e));
    BatchCtl ctl{};
    e = cudaMemcpyAsync(&ctl, g_batch.ctl, sizeof(BatchCtl), cudaMemcpyDeviceToHost, st);
    if (e == cudaSuccess) e = cudaStreamSynchronize(st);
    if (e != cudaSuccess) return fail(AIR_ERR_CUDA, std::string("batch solve: ") + cudaGetErrorString(e));
    if (ctl.error != 0) return fail(AIR_ERR_TIMEOUT, "a grid barrier of the batch kernel timed out");
    return AIR_OK;
}
