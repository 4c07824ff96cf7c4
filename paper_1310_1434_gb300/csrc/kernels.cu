// Kernels of the AIR hot path (sm_103a): per-op kernels over one slice,
// grouped per-op kernels over the tiles of many slices, and the persistent
// batch kernel.
#include <atomic>

#include "launch.h"
#include "tiles.cuh"

namespace air {

// Opts a kernel in to more than 48 KB of dynamic shared memory once per
// device (the attribute belongs to the device's context): `done` holds one
// bit per device ordinal below 64; devices beyond that set it every time.
template <typename Kernel>
static cudaError_t opt_in_smem(Kernel kernel, std::atomic<unsigned long long> &done) {
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return e;
    const unsigned long long bit = dev >= 0 && dev < 64 ? 1ull << dev : 0ull;
    if (bit && (done.load(std::memory_order_acquire) & bit)) return cudaSuccess;
    e = cudaFuncSetAttribute(kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, 200 * 1024);
    if (e == cudaSuccess && bit) done.fetch_or(bit, std::memory_order_acq_rel);
    return e;
}

// ------------------------------------------------------------------------
// per-op kernels: one block per tile of one slice
// ------------------------------------------------------------------------
template <int OP>
__global__ void __launch_bounds__(AIR_THREADS) k_op(const SliceDesc s, int arg) {
    extern __shared__ __align__(16) float sm[];
    const int tile = blockIdx.x;
    if constexpr (OP == OP_FWD) {
        tile_fwd(s, arg, tile);
    } else if constexpr (OP == OP_RAMP) {
        tile_ramp(s, arg, tile, sm);
    } else if constexpr (OP == OP_BWD) {
        tile_bwd(s, arg, tile, sm);
    } else if constexpr (OP == OP_BWD_FIN) {
        tile_bwd_fin(s, arg, tile);
    } else if constexpr (OP == OP_CG_A) {
        tile_cg_a(s, tile);
    } else if constexpr (OP == OP_CG_B) {
        tile_cg_b(s, tile);
    } else if constexpr (OP == OP_ZERO) {
        tile_zero(s, tile);
    } else if constexpr (OP == OP_AXPY) {
        tile_axpy(s, tile);
    } else if constexpr (OP == OP_PROX) {
        tile_prox(s, tile, sm);
    } else if constexpr (OP == OP_FBP) {
        tile_fbp(s, tile);
    } else if constexpr (OP == OP_RESTART) {
        tile_restart(s, arg, tile);
    } else if constexpr (OP == OP_SHRINK) {
        if (arg < 2) {
            run_shrink(s, arg, tile, sm);
        } else {  // stand-alone call: X, b (read), scratch b', g from the ext operands
            ShrinkArgs a{s.ext_in, s.ext_out, s.b2, s.ext_out2, s.tau};
            tile_shrink(s, a, tile, true, s.ext_scalar, sm);
        }
    } else if constexpr (OP == OP_FRAMELET) {
        tile_framelet(s, arg, tile, sm);
    } else if constexpr (OP == OP_TRANSPOSE) {
        tile_transpose(s, arg, tile, sm);
    }
}

template <int OP>
static cudaError_t launch_one(const SliceDesc &s, int arg, cudaStream_t st) {
    const int tiles = tiles_of(s, OP == OP_FRAMELET && arg ? OP_FRAMELET_T : OP);
    if (tiles <= 0) return cudaSuccess;
    const size_t smem = tile_smem(s, OP);
    static std::atomic<unsigned long long> attr_done{0};
    if (cudaError_t e = opt_in_smem(k_op<OP>, attr_done); e != cudaSuccess) return e;
    k_op<OP><<<tiles, AIR_THREADS, smem, st>>>(s, arg);
    return cudaGetLastError();
}

cudaError_t launch_op(int op, const SliceDesc &s, int arg, cudaStream_t st) {
    switch (op) {
    case OP_FWD: return launch_one<OP_FWD>(s, arg, st);
    case OP_RAMP: return launch_one<OP_RAMP>(s, arg, st);
    case OP_BWD: return launch_one<OP_BWD>(s, arg, st);
    case OP_CG_A: return launch_one<OP_CG_A>(s, arg, st);
    case OP_CG_B: return launch_one<OP_CG_B>(s, arg, st);
    case OP_ZERO: return launch_one<OP_ZERO>(s, arg, st);
    case OP_SHRINK: return launch_one<OP_SHRINK>(s, arg, st);
    case OP_FRAMELET: return launch_one<OP_FRAMELET>(s, 0, st);
    case OP_FRAMELET_T: return launch_one<OP_FRAMELET>(s, 1, st);
    case OP_TRANSPOSE: return launch_one<OP_TRANSPOSE>(s, arg, st);
    case OP_BWD_FIN: return launch_one<OP_BWD_FIN>(s, arg, st);
    case OP_AXPY: return launch_one<OP_AXPY>(s, arg, st);
    case OP_PROX: return launch_one<OP_PROX>(s, arg, st);
    case OP_FBP: return launch_one<OP_FBP>(s, arg, st);
    case OP_RESTART: return launch_one<OP_RESTART>(s, arg, st);
    default: return cudaErrorInvalidValue;
    }
}

// ------------------------------------------------------------------------
// grouped kernels: block -> (task, tile) by binary search over tile0
// ------------------------------------------------------------------------
// The slice descriptor of the current tile is staged in shared memory: the
// tile functions read its fields inside their loops, which from global
// memory would cost a load each time.
__device__ __forceinline__ const SliceDesc &stage_desc(const SliceDesc *__restrict__ slices, int si,
                                                       SliceDesc *sd, int *staged) {
    if (*staged != si) {
        __syncthreads();
        const int words = (int)(sizeof(SliceDesc) / sizeof(int));
        const int *src = reinterpret_cast<const int *>(slices + si);
        int *dst = reinterpret_cast<int *>(sd);
        for (int i = threadIdx.x; i < words; i += AIR_THREADS) dst[i] = src[i];
        __syncthreads();
        *staged = si;
    }
    return *sd;
}

// Grouped form of one op: the tiles of many slices in one launch, the
// kernel specialised for the op (its own register budget).
template <int OP>
__global__ void __launch_bounds__(AIR_THREADS)
k_group(const SliceDesc *__restrict__ slices, const Task *__restrict__ tasks, int ntasks) {
    extern __shared__ __align__(16) float sm[];
    __shared__ __align__(16) SliceDesc sd;
    const int b = blockIdx.x;
    int lo = 0, hi = ntasks - 1;
    while (lo < hi) {
        const int mid = (lo + hi + 1) >> 1;
        if (tasks[mid].tile0 <= b) lo = mid;
        else hi = mid - 1;
    }
    const Task t = tasks[lo];
    int staged = -1;
    const SliceDesc &s = stage_desc(slices, t.slice, &sd, &staged);
    const int tile = b - t.tile0;
    if constexpr (OP == OP_FWD) tile_fwd(s, t.arg, tile);
    else if constexpr (OP == OP_RAMP) tile_ramp(s, t.arg, tile, sm);
    else if constexpr (OP == OP_BWD) tile_bwd(s, t.arg, tile, sm);
    else if constexpr (OP == OP_BWD_FIN) tile_bwd_fin(s, t.arg, tile);
    else if constexpr (OP == OP_CG_A) tile_cg_a(s, tile);
    else if constexpr (OP == OP_CG_B) tile_cg_b(s, tile);
    else if constexpr (OP == OP_ZERO) tile_zero(s, tile);
    else if constexpr (OP == OP_AXPY) tile_axpy(s, tile);
    else if constexpr (OP == OP_PROX) tile_prox(s, tile, sm);
    else if constexpr (OP == OP_TRANSPOSE) tile_transpose(s, t.arg, tile, sm);
    else if constexpr (OP == OP_SHRINK) run_shrink(s, t.arg, tile, sm);
    else if constexpr (OP == OP_RESTART) tile_restart(s, t.arg, tile);
}

template <int OP>
static cudaError_t launch_group_op(const SliceDesc *d_slices, const Task *d_tasks, int ntasks, int total_tiles,
                                   size_t smem, cudaStream_t st) {
    static std::atomic<unsigned long long> attr_done{0};
    if (cudaError_t e = opt_in_smem(k_group<OP>, attr_done); e != cudaSuccess) return e;
    k_group<OP><<<total_tiles, AIR_THREADS, smem, st>>>(d_slices, d_tasks, ntasks);
    return cudaGetLastError();
}

// Blocks of the grouped backprojector that the device holds at once (SMs x
// blocks per SM at the given shared memory), or 0 on failure.
int group_bwd_capacity(size_t smem) {
    int dev = 0, sms = 0, per = 0;
    if (cudaGetDevice(&dev) != cudaSuccess) return 0;
    if (cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess) return 0;
    static std::atomic<unsigned long long> attr_done{0};
    if (opt_in_smem(k_group<OP_BWD>, attr_done) != cudaSuccess) return 0;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per, k_group<OP_BWD>, AIR_THREADS, smem) != cudaSuccess)
        return 0;
    return sms * per;
}

cudaError_t launch_group(int op, const SliceDesc *d_slices, const Task *d_tasks, int ntasks, int total_tiles,
                         size_t smem, cudaStream_t st) {
    if (ntasks <= 0 || total_tiles <= 0) return cudaSuccess;
    switch (op) {
    case OP_FWD: return launch_group_op<OP_FWD>(d_slices, d_tasks, ntasks, total_tiles, smem, st);
    case OP_RAMP: return launch_group_op<OP_RAMP>(d_slices, d_tasks, ntasks, total_tiles, smem, st);
    case OP_BWD: return launch_group_op<OP_BWD>(d_slices, d_tasks, ntasks, total_tiles, smem, st);
    case OP_BWD_FIN: return launch_group_op<OP_BWD_FIN>(d_slices, d_tasks, ntasks, total_tiles, smem, st);
    case OP_CG_A: return launch_group_op<OP_CG_A>(d_slices, d_tasks, ntasks, total_tiles, smem, st);
    case OP_CG_B: return launch_group_op<OP_CG_B>(d_slices, d_tasks, ntasks, total_tiles, smem, st);
    case OP_ZERO: return launch_group_op<OP_ZERO>(d_slices, d_tasks, ntasks, total_tiles, smem, st);
    case OP_TRANSPOSE: return launch_group_op<OP_TRANSPOSE>(d_slices, d_tasks, ntasks, total_tiles, smem, st);
    case OP_SHRINK: return launch_group_op<OP_SHRINK>(d_slices, d_tasks, ntasks, total_tiles, smem, st);
    case OP_AXPY: return launch_group_op<OP_AXPY>(d_slices, d_tasks, ntasks, total_tiles, smem, st);
    case OP_PROX: return launch_group_op<OP_PROX>(d_slices, d_tasks, ntasks, total_tiles, smem, st);
    case OP_RESTART: return launch_group_op<OP_RESTART>(d_slices, d_tasks, ntasks, total_tiles, smem, st);
    default: return cudaErrorInvalidValue;
    }
}

// ------------------------------------------------------------------------
// persistent batch kernel with a bounded grid barrier
// ------------------------------------------------------------------------
// Spin budget of one barrier wait: 2^25 polls with a 128 ns back-off, a few
// seconds, far above any phase; on expiry the block records AIR_ERR_TIMEOUT
// and every block leaves at its next barrier.  g_barrier_budget replaces it
// when >= 0 (air_set_wait_budget; one copy per device).  A block that gives
// up has no asynchronous copy in flight, so it may leave at once.
constexpr long long BARRIER_POLLS = 1ll << 25;
__device__ long long g_barrier_budget = -1;

cudaError_t set_barrier_budget(long long polls) {
    return cudaMemcpyToSymbol(g_barrier_budget, &polls, sizeof(polls));
}

__device__ bool grid_barrier(BatchCtl *ctl) {
    __shared__ int ok;
    __syncthreads();
    if (threadIdx.x == 0) {
        volatile unsigned *vgen = &ctl->gen;
        volatile int *verr = &ctl->error;
        const unsigned gen = *vgen;
        __threadfence();
        const unsigned arrived = atomicAdd(&ctl->arrive, 1u);
        int good = 0;
        if (arrived == gridDim.x - 1) {
            atomicExch(&ctl->arrive, 0u);
            __threadfence();
            atomicAdd(&ctl->gen, 1u);
            good = *verr == 0;
        } else {
            const long long polls = g_barrier_budget < 0 ? BARRIER_POLLS : g_barrier_budget;
            for (long long it = 0; it < polls; ++it) {
                if (*vgen != gen) { good = 1; break; }
                if (*verr != 0) break;
                __nanosleep(128);
            }
            if (!good && *verr == 0) atomicCAS(&ctl->error, 0, (int)AIR_ERR_TIMEOUT);
            good = good && *verr == 0;
        }
        __threadfence();
        ok = good;
    }
    __syncthreads();
    return ok != 0;
}

// Tiles are handed out in each phase from one global ticket counter, so
// blocks that draw cheap tiles take more of them.  A block leaves a phase at
// its first ticket past the phase's last tile; the phase's first ticket
// (phase_base) counts those closing tickets, one per block, of every earlier
// phase, and the grid barrier keeps the phases' tickets apart.
__global__ void __launch_bounds__(AIR_THREADS, 5)
k_persistent(const SliceDesc *__restrict__ slices, int nslices, const Phase *__restrict__ prog,
             int nphases, const int *__restrict__ tile_base, const unsigned long long *__restrict__ phase_base,
             BatchCtl *ctl) {
    extern __shared__ __align__(16) float sm[];
    __shared__ __align__(16) SliceDesc sd;
    __shared__ long long drawn;
    int staged = -1;                  // slice whose descriptor sd holds
    for (int ph = 0; ph < nphases; ++ph) {
        const int *__restrict__ tb = tile_base + (size_t)ph * (nslices + 1);
        const long long ntiles = tb[nslices];
        int si = 0;
        for (;;) {
            if (threadIdx.x == 0) drawn = (long long)(atomicAdd(&ctl->ticket, 1ull) - phase_base[ph]);
            __syncthreads();
            const long long t = drawn;
            __syncthreads();
            if (t >= ntiles) break;
            while (t >= tb[si + 1]) ++si;       // a block's tickets increase
            const Phase P = prog[(size_t)si * nphases + ph];
            run_tile(stage_desc(slices, si, &sd, &staged), P.op, P.arg, (int)(t - tb[si]), sm);
        }
        if (!grid_barrier(ctl)) return;
    }
}

// Resident blocks per SM of the persistent kernel, and the shared-memory
// carveout it asks for.  Its shared memory is reserved through every phase
// (the backprojector's strips), and whatever the carveout leaves is L1, on
// which the projector phases' gathers depend: four blocks with the carveout
// sized for them leave about 60 KB of L1 where five leave about 28 KB, and
// measured 8 % faster on 8-slice 512^2 batches (three blocks lose more
// parallelism than the L1 gains).
constexpr int PERSISTENT_BLOCKS = 4;

int persistent_grid(size_t smem) {
    int dev = 0, sms = 0, per = 0, max_smem = 0;
    if (cudaGetDevice(&dev) != cudaSuccess) return 0;
    if (cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess) return 0;
    if (cudaDeviceGetAttribute(&max_smem, cudaDevAttrMaxSharedMemoryPerMultiprocessor, dev) != cudaSuccess)
        return 0;
    static std::atomic<unsigned long long> attr_done{0};
    if (opt_in_smem(k_persistent, attr_done) != cudaSuccess) return 0;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per, k_persistent, AIR_THREADS, smem) != cudaSuccess)
        return 0;
    const int blocks = per < PERSISTENT_BLOCKS ? per : PERSISTENT_BLOCKS;
    if (blocks < 1 || max_smem <= 0) return 0;
    // the blocks' dynamic and static shared memory plus the 1 KB the
    // hardware reserves per block, as a percentage of the SM's maximum
    // (the driver rounds up to a supported carveout)
    const double need = (double)blocks * ((double)smem + 2048.0);
    int pct = (int)(100.0 * need / max_smem) + 2;
    if (pct > 100) pct = 100;
    if (cudaFuncSetAttribute(k_persistent, cudaFuncAttributePreferredSharedMemoryCarveout, pct) != cudaSuccess)
        return 0;
    return sms * blocks;
}

cudaError_t launch_persistent(const SliceDesc *d_slices, int nslices, const Phase *d_prog,
                              int nphases, const int *d_tile_base, const unsigned long long *d_phase_base,
                              BatchCtl *d_ctl, int grid, size_t smem, cudaStream_t st) {
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3(grid);
    cfg.blockDim = dim3(AIR_THREADS);
    cfg.dynamicSmemBytes = smem;
    cfg.stream = st;
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeCooperative;
    attr[0].val.cooperative = 1;
    cfg.attrs = attr;
    cfg.numAttrs = 1;
    return cudaLaunchKernelEx(&cfg, k_persistent, d_slices, nslices, d_prog, nphases, d_tile_base, d_phase_base,
                              d_ctl);
}

}  // namespace air
