// Internal types and device helpers of the AIR library (sm_103a).
//
// Every operator of the hot path is written as a TILE function: one thread
// block of AIR_THREADS threads does one tile of one slice.  The same tile
// functions back three launch forms:
//   * per-op kernels over one slice            (air_project, air_solve, ...)
//   * grouped per-op kernels over the tiles of many slices, one launch per
//     phase (air_solve_batch, captured in a CUDA graph; the server's steps)
//   * a persistent kernel with a bounded grid barrier between phases
//     (air_solve_batch_persistent)
#pragma once

#include <cstdint>
#include <cuda_runtime.h>

#include "air.h"   // from include/ (nvcc -I)

#define AIR_THREADS 256

namespace air { constexpr int RAMP_MAX_BINS = 8192; }  // largest n_bins (filter row in shared memory)

namespace air {

// ---------------------------------------------------------------- ops ----
enum Op : int {
    OP_NOP = 0,
    OP_FWD,        // z = A src                      (src = x or p)
    OP_RAMP,       // zc = C src                     (src = y or z), FP32
    OP_RAMP_TC,    // zc = C z on tensor cores (split BF16) -- own kernel
    OP_BWD,        // A^T zc with a mode epilogue (see BwdMode)
    OP_CG_A,       // alpha; x += alpha p; r -= alpha q; rho' = r.r
    OP_CG_B,       // p = r + beta p
    OP_SHRINK,     // t = Wx + b; b' = t - d; g = W^T(d - b'); ||Wx - d||
    OP_ZERO,       // x = 0, b = 0, g = 0, cg.stop = 0
    OP_FRAMELET,   // out = W in            (API call)
    OP_FRAMELET_T, // out = W^T in          (API call)
    OP_TRANSPOSE,  // xp, xt = padded src, transpose(src)   (before every OP_FWD; arg = FwdSrc)
    OP_BWD_FIN,    // sum the backprojector's view parts, then the BwdMode epilogue
    OP_AXPY,       // q = x + step r            (forward step of Eq. 6, r = A'^T(Y - A x))
    OP_PROX,       // x = W^T S_tau(W q)        (framelet proximal step)
    OP_FBP,        // ext_out = fan-beam FBP weighted backprojection of zc
    OP_RESTART,    // CG restart of an outer step: r = rhs0 (arg -1) or r += mu (g_new - g_old); p = r; rho
    OP_COUNT
};

enum FwdSrc : int { SRC_X = 0, SRC_P = 1, SRC_EXT = 2 };
enum RampSrc : int { RSRC_Y = 0, RSRC_Z = 1, RSRC_EXT = 2 };
enum BwdMode : int {
    BWD_PLAIN = 0,   // out = dx * acc                      (air_backproject)
    BWD_RHS0 = 1,    // rhs0 = dx * acc
    BWD_RESID = 2,   // r = rhs0 + mu g - (dx acc + mu x); p = r; rho = r.r
    BWD_Q = 3        // q = dx acc + mu p; pq = p.q; stop if pq <= 0
};

// Device-resident CG / Bregman scalars of one slice.  FP64 where the paper's
// inner products and residual norms are formed.
struct CgState {
    double rho;        // r.r of the current CG iterate
    double pq;         // p.Mp
    double alpha, beta;
    double resid;      // ||W X - d||_2 of the last shrink
    int stop;          // CG of this outer step has stopped (rho == 0 or pq <= 0)
    int outer;         // outer iterations done (indexes the resid output)
    unsigned counter;  // blocks done in the current reducing phase
    int pad;
};

// One ray in fixed point (32 fractional bits, pixel units, origin at the
// image corner).  A ray with |ux| >= |uy| is walked column by column: in
// column k its y-span is [lo(k), lo(k) + Ma] with lo(k) = L0 + k*M; a ray
// with |uy| > |ux| is walked row by row with x and y exchanged.  The length
// inside pixel (k, row) is ov * c, ov the integer overlap of the span with
// [row, row + 1), c = sec/|M|.  Integer arithmetic is exact, so every kernel
// that evaluates a (ray, pixel) pair gets the same length, bit for bit.
// M (0 < |M| < 2^32) is stored as its low word Mlo, its high word given by
// the sign of cs = +-c; |M| = Mlo for M > 0 and 2^32 - Mlo for M < 0.  These
// 16 bytes are all the backprojector reads; the projector also reads the
// ray's walk word (ray_walk).
struct __align__(16) RayFx {
    long long L0;      // lower edge of the span in column (row) 0, 2^-32 px
    unsigned Mlo;      // low word of M = slope * 2^32
    float cs;          // c with the sign of M
};
__host__ __device__ inline long long ray_M(const RayFx &r) {
    return r.cs < 0.f ? (long long)r.Mlo - (1ll << 32) : (long long)r.Mlo;
}
__host__ __device__ inline unsigned ray_Ma(const RayFx &r) { return r.cs < 0.f ? 0u - r.Mlo : r.Mlo; }
// The walk word of a ray: columns (rows) [k0, k1) of the walk in bits 0-15
// and 16-30, bit 31 set when the ray walks columns (|ux| >= |uy|, reading
// the transposed image copy).
__host__ __device__ inline unsigned ray_walk(int k0, int k1, bool cols) {
    return (unsigned)k0 | ((unsigned)k1 << 16) | (cols ? 0x80000000u : 0u);
}
__host__ __device__ inline int walk_k0(unsigned w) { return (int)(w & 0xffffu); }
__host__ __device__ inline int walk_k1(unsigned w) { return (int)((w >> 16) & 0x7fffu); }
__host__ __device__ inline int walk_cols(unsigned w) { return (int)(w >> 31); }

// Per (view, backprojector pixel tile): the rays of the view that can meet
// the tile, [J0, J1), the orientation and slope sign of ray J0, and whether
// all rays of the range share both.
constexpr unsigned VT_MIXED = 1u << 29;   // the range holds both orientations or both signs of M
constexpr unsigned VT_NEG = 1u << 30;     // ray J0 has M < 0
__host__ __device__ inline unsigned vt_pack(int j0, int j1, int o, bool neg, bool mixed) {
    return (unsigned)j0 | ((unsigned)j1 << 14) | ((unsigned)o << 28) | (neg ? VT_NEG : 0u) |
           (mixed ? VT_MIXED : 0u);
}

// Everything a tile function needs to know about one slice.  Plain data:
// copied by value into kernel parameters or into a device task table.
struct SliceDesc {
    // geometry (pixel units: lengths divided by dx, image centre at 0)
    int n, V, nb;
    float half_n;        // n / 2
    float dx;            // mm per pixel
    int filter;          // AIR_FILTER_*
    // tables (plan-owned, read-only)
    const RayFx *ray;    // [V*nb] fixed-point rays
    const unsigned *walk;  // [V*nb] walk words (ray_walk)
    const unsigned *vt;  // [backprojector pixel tile][V] ray ranges (vt_pack)
    const float *taps;   // [nb] c0 * h[k], k = 0..nb-1 (h even)
    float ramp_diag;     // taps[0] + 2 sum_{odd m < nb} taps[m]
    const float *prew;   // [nb] weights applied to the filter's input, or nullptr (FBP: cos gamma_j)
    // fan-beam FBP (the analytic reconstruction): its filter runs the ramp
    // tile with taps = fbp_taps, ramp_diag = fbp_diag, prew = fbp_w
    const float2 *fview; // [V] central-ray direction of each view
    const float *fbp_w;  // [nb] cos gamma_j
    const float *fbp_taps;   // [nb] alpha D g(m alpha), the fan ramp
    float fbp_diag;      // fbp_taps[0] + 2 sum_{odd m < nb} fbp_taps[m]
    float dso_px;        // source-isocentre distance, pixels
    float inv_dg, inv_dg_lo, jmid;   // 1 / fan pitch (high and low parts), (nb - 1) / 2
    float fbp_scale;     // dbeta / dx^2
    // solver state (plan-owned workspace)
    float *x, *r, *p, *q, *rhs0, *g;   // n*n
    float *g2;                         // n*n: g of the previous outer step (g is double-buffered)
    float *xp, *xt;                    // n*(n+1) float2 each: pair copies {X[r], X[r+1]} of the projector's input and its transpose
    float *bwd_part;                   // bwd_parts * n*n: the backprojector's per-view-part sums
    int bwd_parts;                     // S: views split over S blocks per pixel tile (tuned)
    int fwd_vpb;                       // projector tile: views per block (1, 2, 4, 8; tuned)
    float *b, *b2;                     // 9*n*n each (Bregman variable, double-buffered)
    float *z, *zc;                     // V*nb
    const float *y;                    // V*nb measured sinogram
    float mu, tau;                     // mu, lambda/mu (forward-backward: 0, step * lambda)
    float step;                        // forward-backward step size (Eq. 6)
    CgState *cg;
    double *partial;                   // per-tile partial sums (>= max reducing tiles)
    double *resid_out;                 // n_outer doubles or nullptr
    // operands of the stand-alone API calls
    const float *ext_in;
    float *ext_out;
    float *ext_out2;
    double *ext_scalar;
};

struct Task {
    int slice;      // index into the SliceDesc table
    int op;         // Op
    int arg;        // FwdSrc / RampSrc / BwdMode
    int tile0;      // first global tile (block) index of this task
};

// ---------------------------------------------------- tile counts --------
// projector tile: fwd_vpb views x (AIR_THREADS / fwd_vpb) bins, one ray per thread
__host__ __device__ inline int tiles_fwd(const SliceDesc &s) {
    const int bpb = AIR_THREADS / s.fwd_vpb;
    return ((s.V + s.fwd_vpb - 1) / s.fwd_vpb) * ((s.nb + bpb - 1) / bpb);
}
__host__ __device__ inline int tiles_ramp(const SliceDesc &s) { return s.V; }
// backprojector tile: 32 x 32 pixels x one of bwd_parts view parts
constexpr int BWD_T = 32;
__host__ __device__ inline int tiles_bwd_xy(const SliceDesc &s) {
    return ((s.n + BWD_T - 1) / BWD_T) * ((s.n + BWD_T - 1) / BWD_T);
}
__host__ __device__ inline int tiles_bwd(const SliceDesc &s) { return tiles_bwd_xy(s) * s.bwd_parts; }
constexpr int VEC_PER_TILE = AIR_THREADS * 4;   // elementwise ops: 4 per thread
__host__ __device__ inline int tiles_vec(const SliceDesc &s) {
    return (s.n * s.n + VEC_PER_TILE - 1) / VEC_PER_TILE;
}
constexpr int SHR_T = 16;                      // shrink/framelet output tile
__host__ __device__ inline int tiles_shr(const SliceDesc &s) {
    return ((s.n + SHR_T - 1) / SHR_T) * ((s.n + SHR_T - 1) / SHR_T);
}
// pair-copy transpose tile: 32 x 32 pixels
__host__ __device__ inline int tiles_tr(const SliceDesc &s) {
    return ((s.n + 31) / 32) * ((s.n + 31) / 32);
}
__host__ __device__ inline int tiles_of(const SliceDesc &s, int op) {
    switch (op) {
    case OP_FWD: return tiles_fwd(s);
    case OP_RAMP: return tiles_ramp(s);
    case OP_BWD: return tiles_bwd(s);
    case OP_CG_A: case OP_CG_B: case OP_ZERO: case OP_BWD_FIN: case OP_AXPY: case OP_RESTART: return tiles_vec(s);
    case OP_TRANSPOSE: return tiles_tr(s);
    case OP_SHRINK: case OP_FRAMELET: case OP_FRAMELET_T: case OP_PROX: case OP_FBP:
        return tiles_shr(s);
    default: return 0;
    }
}
// largest number of tiles of any reducing op: sizes SliceDesc::partial
__host__ inline int max_reduce_tiles(const SliceDesc &s) {
    const int b = tiles_vec(s), c = tiles_shr(s);
    return b > c ? b : c;
}

// ------------------------------------------------ block reductions -------
__device__ __forceinline__ double warp_sum(double v) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    return v;
}
// Sum over the block, result valid in thread 0.  Fixed order: deterministic.
__device__ __forceinline__ double block_sum(double v, double *sh /* >= 8 */) {
    v = warp_sum(v);
    const int w = threadIdx.x >> 5, l = threadIdx.x & 31;
    __syncthreads();
    if (l == 0) sh[w] = v;
    __syncthreads();
    double t = 0.0;
    if (threadIdx.x == 0) {
        for (int i = 0; i < (AIR_THREADS >> 5); ++i) t += sh[i];
    }
    return t;
}

}  // namespace air
