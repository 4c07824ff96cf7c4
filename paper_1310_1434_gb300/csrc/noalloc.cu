// air_filtered_backproject_noalloc: the filtered adjoint X = A^T C Y for
// callers that must not allocate device memory at call time -- for example
// code running under a device-memory budget that forbids cudaMalloc after
// start-up, or a host thread that holds a lock another thread needs to
// allocate.  Its only scratch -- the filtered sinogram C Y and the
// backprojector's per-view-part images -- lives in the file-scope device
// array below instead of in plan or caller memory.
#include <mutex>
#include <string>

#include "host_common.h"

using namespace air;

namespace {

// Largest filtered sinogram the static scratch holds: n_views * n_bins.
constexpr size_t NOALLOC_MAX_SAMPLES = size_t(1) << 20;
// The whole array (16 MB of float): the filtered sinogram, then as many of
// the backprojector's view parts (n * n floats each) as fit, up to the plan's
// tuned split.
constexpr size_t NOALLOC_FLOATS = size_t(1) << 22;

// The array belongs to this file's module.  CUDA loads a module, and
// allocates its device arrays, when the module is first used on a device,
// so plan creation uses it (noalloc_prepare): every device on which a plan
// has been created holds the array until the process exits, and a later call
// of the entry point allocates nothing.  All calls on a device share it and
// it keeps the last call's contents; every element a call reads was written
// earlier by the same call (the filter writes all n_views * n_bins samples,
// each view part all n * n pixels), so nothing needs clearing.  Calls that
// overlap on the GPU race on it.
static __device__ __align__(256) float g_fbp_scratch[NOALLOC_FLOATS];

constexpr int MAX_DEVICES = 64;
std::mutex g_mu;
float *g_scratch_ptr[MAX_DEVICES] = {};

// Looks up the array's device address on the current device and records it.
// In host code g_fbp_scratch names a host-side stand-in, never a device
// address, so kernels only ever receive the address recorded here.
air_status lookup(int dev, float **out) {
    void *p = nullptr;
    const cudaError_t e = cudaGetSymbolAddress(&p, g_fbp_scratch);
    if (e != cudaSuccess)
        return fail(AIR_ERR_CUDA, std::string("cudaGetSymbolAddress of the static scratch: ") + cudaGetErrorString(e));
    g_scratch_ptr[dev] = static_cast<float *>(p);
    *out = g_scratch_ptr[dev];
    return AIR_OK;
}

air_status current_device(int *dev) {
    const cudaError_t e = cudaGetDevice(dev);
    if (e != cudaSuccess) return fail(AIR_ERR_CUDA, std::string("cudaGetDevice: ") + cudaGetErrorString(e));
    if (*dev < 0 || *dev >= MAX_DEVICES) return fail(AIR_ERR_CUDA, "device ordinal out of range");
    return AIR_OK;
}

// Device address of the scratch on the current device: the one plan creation
// recorded, or (a device on which no plan was created) looked up now.
air_status scratch_ptr(float **out) {
    int dev = 0;
    air_status st = current_device(&dev);
    if (st != AIR_OK) return st;
    std::lock_guard<std::mutex> lock(g_mu);
    if (g_scratch_ptr[dev]) {
        *out = g_scratch_ptr[dev];
        return AIR_OK;
    }
    return lookup(dev, out);
}

}  // namespace

// Every plan creation looks the address up again, so a plan created after a
// cudaDeviceReset (which unloads the module) records the new one.
air_status air::noalloc_prepare() {
    int dev = 0;
    air_status st = current_device(&dev);
    if (st != AIR_OK) return st;
    std::lock_guard<std::mutex> lock(g_mu);
    float *p = nullptr;
    return lookup(dev, &p);
}

extern "C" air_status air_filtered_backproject_noalloc(const air_plan *P, const float *Y, float *X,
                                                       air_stream stream) {
    if (!P) return fail(AIR_ERR_INVALID_ARG, "plan is NULL");
    const size_t samples = (size_t)P->geom.n_views * P->geom.n_bins;
    if (samples > NOALLOC_MAX_SAMPLES)
        return fail(AIR_ERR_INVALID_ARG, "n_views * n_bins = " + std::to_string(samples) +
                                             " exceeds the static scratch of this call (" +
                                             std::to_string(NOALLOC_MAX_SAMPLES) + " samples)");
    air_status st = check_dev_ptr(Y, "Y");
    if (st != AIR_OK) return st;
    if ((st = check_dev_ptr(X, "X")) != AIR_OK) return st;
    if (overlap(X, (size_t)P->geom.n * P->geom.n * 4, Y, samples * 4))
        return fail(AIR_ERR_INVALID_ARG, "X and Y overlap");
    float *scratch = nullptr;
    if ((st = scratch_ptr(&scratch)) != AIR_OK) return st;
    const cudaStream_t s = (cudaStream_t)stream;
    SliceDesc d = P->desc;
    d.ext_in = Y;            // C Y into the static scratch (FP32 filter)
    d.ext_out = scratch;
    cudaError_t e = launch_op(OP_RAMP, d, RSRC_EXT, s);
    if (e == cudaSuccess) {
        // X = A^T (C Y) over S view parts that fit beside C Y (one part is
        // written straight to X), their sum by the finish op
        const size_t nn = (size_t)P->geom.n * P->geom.n, off = align_up(samples, 64);
        int parts = P->desc.bwd_parts;
        while (parts > 1 && off + (size_t)parts * nn > NOALLOC_FLOATS) --parts;
        d.ext_in = scratch;
        d.ext_out = X;
        d.bwd_parts = parts;
        d.bwd_part = parts > 1 ? scratch + off : nullptr;
        e = launch_op(OP_BWD, d, BWD_PLAIN, s);
        if (e == cudaSuccess && parts > 1) e = launch_op(OP_BWD_FIN, d, BWD_PLAIN, s);
    }
    if (e != cudaSuccess) return fail(AIR_ERR_CUDA, std::string("filtered backprojection: ") + cudaGetErrorString(e));
    return AIR_OK;
}
