// Host-side shared declarations of the AIR library.
#pragma once

#include <string>
#include <vector>

#include "air_internal.cuh"
#include "launch.h"

// A plan: geometry tables + solver workspace of one slice geometry.
struct air_plan {
    air_geometry geom{};
    int device = 0;
    air::SliceDesc desc{};     // tables and workspace pointers
    char *mem = nullptr;       // the one allocation desc points into
    size_t bytes = 0;
    float *ybuf = nullptr;     // staging for the host-buffer solve
    float *xbuf = nullptr;
    void *tc = nullptr;        // tensor-core filter resources (AIR_PREC_BF16X3)
    size_t tc_bytes = 0;
    int bwd_parts_max = 1;     // view parts the backprojector's part buffer holds
};

namespace air {
air_status fail(air_status s, const std::string &msg);
air_status validate_geometry(const air_geometry *g);
air_status check_dev_ptr(const void *p, const char *what);
bool overlap(const void *a, size_t na, const void *b, size_t nb);
size_t align_up(size_t v, size_t a);
double fan_pitch(const air_geometry &g);
std::vector<Phase> solve_program(int n_outer, int n_cg, bool tc_ramp);
std::vector<Phase> l2_program(int n_cg, bool tc_ramp);
std::vector<Phase> fbs_program(int n_iter, bool tc_ramp);
air_status check_solve_args(const air_plan *P, const float *Y, float lambda, float mu, int n_outer,
                            int n_cg, const float *X);
SliceDesc solve_desc(const air_plan *P, const float *Y, float lambda, float mu, float *X, double *resid);
air_status run_program_single(const air_plan *P, const SliceDesc &s, const std::vector<Phase> &prog,
                              cudaStream_t st);
RayFx make_ray_fx(double px, double py, double ux, double uy, int n, unsigned *walk);
int choose_bwd_parts(const SliceDesc &s);
air_status autotune(air_plan *P);
size_t plan_bytes_estimate(const air_geometry &g);
air_status apply_filter(const air_plan *P, const SliceDesc &base, const float *src, float *dst,
                        cudaStream_t st);
// Loads the allocation-free filtered adjoint's static scratch on the current
// device (CUDA loads a module, and allocates its device arrays, on first
// use) and records its address; called by plan creation.
air_status noalloc_prepare();
}  // namespace air
