// Host-side launchers of the AIR kernels (defined in kernels.cu).
#pragma once

#include <cuda_runtime.h>

#include "air_internal.cuh"

namespace air {

// One op over all tiles of one slice.
cudaError_t launch_op(int op, const SliceDesc &s, int arg, cudaStream_t st);

// Blocks of the grouped backprojector resident on the current device at
// once, for the given dynamic shared memory (0 on failure).
int group_bwd_capacity(size_t smem);

// One op over the tiles of many slices in one launch (tasks all of that op).
cudaError_t launch_group(int op, const SliceDesc *d_slices, const Task *d_tasks, int ntasks, int total_tiles,
                         size_t smem, cudaStream_t st);

// Persistent batch solve: one cooperative launch runs every phase of every
// slice's program, with a bounded grid barrier between phases.
struct Phase {
    int op, arg;
};
struct BatchCtl {
    unsigned arrive;     // grid barrier: blocks arrived in this generation
    unsigned gen;        // grid barrier generation
    int error;           // AIR_ERR_TIMEOUT if a barrier wait gave up
    int pad;
    unsigned long long ticket;   // tiles handed out so far (see k_persistent)
};
// tile_base: [nphases][nslices + 1] prefix sums of the slices' tile counts in
// each phase; phase_base: [nphases] first ticket of each phase, the sum over
// earlier phases of their tiles plus one closing ticket per block.
cudaError_t launch_persistent(const SliceDesc *d_slices, int nslices, const Phase *d_prog,
                              int nphases, const int *d_tile_base, const unsigned long long *d_phase_base,
                              BatchCtl *d_ctl, int grid, size_t smem, cudaStream_t st);
// Largest co-resident grid of the persistent kernel for the given smem.
int persistent_grid(size_t smem);
// Poll budget of the persistent kernel's grid-barrier wait on the current
// device (negative: the default).  Synchronous.
cudaError_t set_barrier_budget(long long polls);

}  // namespace air
