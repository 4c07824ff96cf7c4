// Tile functions of the AIR hot path.  One call = one thread block of
// AIR_THREADS threads working on one tile of one slice.  See
// air_internal.cuh for the launch forms that share them.
#pragma once

#include "air_internal.cuh"

namespace air {

// ======================================================================
// Forward projector A (Eq. 1): Y_{v,j} = dx * sum_i l_ij X_i, l_ij the exact
// length of ray (v,j) inside pixel i.  Ray-driven, one thread per ray.  The
// ray is walked along its major axis one column (row) at a time; in column k
// its span [lo, lo + Ma] (fixed point, 2^-32 px) touches row r0 = lo >> 32
// and, when the low word lo32 + Ma wraps past 2^32, row r0 + 1 too.  The
// overlaps are ov1 = (lo32 + Ma) mod 2^32 with the next row (0 without a
// wrap) and ov0 = Ma - ov1 with row r0, and the lengths ov * c (see RayFx).
// The walk reads pair copies of the image: row k holds the n + 1 pairs
// {X[r], X[r + 1]} for r = -1 .. n-1 (X[-1] = X[n] = 0), so one aligned
// 8-byte load gives both rows a column step can touch; r0 lies in [-1, n-1]
// on the walk range, so the walk needs no bounds checks.  Rays walking
// columns read the transposed copy so that the rays of a warp read
// neighbouring addresses.  The per-ray factor c is taken out of the sum: a
// unit input still gives the entry ov * c exactly.
// ======================================================================
__host__ __device__ inline int pair_ld(int n) { return n + 1; }   // pairs per row of the pair copies

// One column of the walk: the overlaps of the span [lo, lo + Ma] with row r0
// and (when the span reaches past the next row boundary) row r0 + 1, times
// the pixel pair {X[r0], X[r0 + 1]} read with one 8-byte load.  The walk
// keeps nlo = ~lo: with f = lo mod 2^32 the span's first row takes
// min(Ma, 2^32 - f) = min(Ma - 1, ~f) + 1 of it (also for f = 0, a span
// starting on a row boundary) and the next row the rest, 0 when the span
// ends inside row r0; ~(lo >> 32) = -r0 - 1 turns the pair index off + r0 + 1
// into one subtraction.  The same integers as the wrap test of the
// backprojector, with fewer integer instructions on the walk's bound pipe;
// the image row is a 32-bit element offset into the copy.
__device__ __forceinline__ void fx_step(long long &nlo, const float2 *__restrict__ copy, unsigned &off, long long M,
                                        unsigned Ma1, unsigned Ma, int ld, float &a0, float &a1) {
    const unsigned nf = (unsigned)nlo;                    // ~(lo mod 2^32)
    const unsigned nr = (unsigned)(nlo >> 32);            // ~r0
    const unsigned ov0 = min(Ma1, nf) + 1u;
    const unsigned ov1 = Ma - ov0;
    const float2 xx = __ldg(copy + (off - nr));           // pair r0 + 1 of row k
    a0 = fmaf(__uint2float_rn(ov0), xx.x, a0);
    a1 = fmaf(__uint2float_rn(ov1), xx.y, a1);
    nlo -= M;
    off += (unsigned)ld;
}

// Sum over the walk of ov * X (without c), from the pair copies.
// Consecutive columns alternate between two accumulator pairs: four FP32
// accumulators of about a quarter of the terms each (two independent FMA
// chains), which keeps the ray sum's rounding error within the
// single-application bound for images up to 1024^2.
__device__ __forceinline__ float fx_ray(const float2 *__restrict__ XP, const float2 *__restrict__ XTP, int n,
                                        const RayFx &r, unsigned walk) {
    const int k0 = walk_k0(walk), k1 = walk_k1(walk);
    const int ld = pair_ld(n);
    const float2 *__restrict__ copy = walk_cols(walk) ? XTP : XP;
    unsigned off = (unsigned)k0 * (unsigned)ld;           // row k0 of the copy, pair {X[-1], X[0]}
    const long long M = ray_M(r);
    const unsigned Ma = ray_Ma(r);
    long long nlo = ~(r.L0 + (long long)k0 * M);
    float a0 = 0.f, a1 = 0.f, b0 = 0.f, b1 = 0.f;
    int k = k0;
    for (; k + 1 < k1; k += 2) {
        fx_step(nlo, copy, off, M, Ma - 1u, Ma, ld, a0, a1);
        fx_step(nlo, copy, off, M, Ma - 1u, Ma, ld, b0, b1);
    }
    if (k < k1) fx_step(nlo, copy, off, M, Ma - 1u, Ma, ld, a0, a1);
    return (a0 + a1) + (b0 + b1);
}

__device__ __forceinline__ void tile_fwd(const SliceDesc &s, int arg, int tile) {
    if (arg == SRC_P && s.cg->stop) return;
    float *dst = arg == SRC_EXT ? s.ext_out : s.z;
    // tile = (view group, bin range); a warp holds neighbouring bins of one
    // view, and the warps of a block neighbouring views, whose rays walk
    // neighbouring paths through the image
    const int bpb = AIR_THREADS / s.fwd_vpb;
    const int nbt = (s.nb + bpb - 1) / bpb;
    const int v = (tile / nbt) * s.fwd_vpb + threadIdx.x / bpb;
    const int j = (tile % nbt) * bpb + threadIdx.x % bpb;
    if (v >= s.V || j >= s.nb) return;
    const int idx = v * s.nb + j;
    const RayFx r = s.ray[idx];
    dst[idx] = s.dx * (fabsf(r.cs) * fx_ray(reinterpret_cast<const float2 *>(s.xp),
                                            reinterpret_cast<const float2 *>(s.xt), s.n, r, __ldg(s.walk + idx)));
}

// xp and xt: the pair copies of src and of its transpose (pair r + 1 of a
// row holds {X[r], X[r + 1]}, so each pixel is written as the first half of
// one pair and the second half of the one before), in 32 x 32 tiles through
// shared memory; runs before every projection.  The two ends that hold no
// pixel (X[-1] and X[n]) are zeroed once with the plan.
__device__ __forceinline__ void tile_transpose(const SliceDesc &s, int arg, int tile, float *sm) {
    if (arg == SRC_P && s.cg->stop) return;
    const float *src = arg == SRC_X ? s.x : (arg == SRC_P ? s.p : s.ext_in);
    const int n = s.n, tpr = (n + 31) / 32, ld = 2 * pair_ld(n);   // floats per row of pairs
    const int x0 = (tile % tpr) * 32, y0 = (tile / tpr) * 32;
    float(*t)[33] = reinterpret_cast<float(*)[33]>(sm);
    const int tx = threadIdx.x & 31, ty = threadIdx.x >> 5;
    for (int yy = ty; yy < 32; yy += AIR_THREADS / 32)
        if (y0 + yy < n && x0 + tx < n) {
            const float v = src[(size_t)(y0 + yy) * n + x0 + tx];
            t[yy][tx] = v;
            float *row = s.xp + (size_t)(y0 + yy) * ld;       // X[x] is pair x+1 .x and pair x .y
            row[2 * (x0 + tx + 1)] = v;
            row[2 * (x0 + tx) + 1] = v;
        }
    __syncthreads();
    for (int xx = ty; xx < 32; xx += AIR_THREADS / 32)
        if (x0 + xx < n && y0 + tx < n) {
            float *row = s.xt + (size_t)(x0 + xx) * ld;
            const float v = t[tx][xx];
            row[2 * (y0 + tx + 1)] = v;
            row[2 * (y0 + tx) + 1] = v;
        }
    __syncthreads();
}

// Sum `val` (valid in thread 0) of this tile into the slice's partials; the
// tile that completes the phase sums all partials in a fixed order and gets
// true with the total in *total (thread 0 only).
__device__ __forceinline__ bool reduce_tiles(const SliceDesc &s, int tile, int ntiles, double val,
                                             double *sh, double *total) {
    __shared__ int last;
    if (threadIdx.x == 0) {
        s.partial[tile] = val;
        __threadfence();
        const unsigned prev = atomicAdd(&s.cg->counter, 1u);
        last = prev == (unsigned)(ntiles - 1);
    }
    __syncthreads();
    if (!last) return false;
    __threadfence();
    double v = 0.0;
    for (int i = threadIdx.x; i < ntiles; i += AIR_THREADS) v += __ldcg(s.partial + i);
    v = block_sum(v, sh);
    if (threadIdx.x == 0) {
        *total = v;
        s.cg->counter = 0u;
    }
    return true;
}

// ======================================================================
// Backprojector A^T, the exact transpose of tile_fwd, without atomics.
// A tile is a 32 x 32 block of pixels and one of S parts of the views.  Warps
// 0-3 take the rays that walk columns, warps 4-7 the rays that walk rows, of
// the same views (warp w: views part + S (w mod 4) + 4 S k).  For each view a
// warp sweeps the rays of the view that meet the tile (a range the plan
// computes, see vt_pack) one ray per step: lane c takes the tile's column c
// (row c for rays walking rows); there the ray's span touches one or two
// pixels of the lane's strip, with the same integer overlaps the projector
// computes, and the lane adds ov * (c z) to its own shared-memory
// accumulator of that pixel.  Accumulators are laid out [strip row][lane], so
// the 32 lanes of a warp always hit 32 different banks, with one margin row
// on each side that catches spans just outside the tile and two spill rows
// that take every lane whose span misses the strip (all discarded): the
// update runs without a branch.  Each pixel's sum is formed in a fixed order
// by one lane of each warp; the warps are summed in a fixed order, and the S
// parts by OP_BWD_FIN.
// ======================================================================
static_assert(BWD_T == 32, "lane c of a warp owns column (row) c of a backprojector tile");
constexpr int BWD_WARPS = AIR_THREADS / 32;
constexpr int BWD_GROUP = BWD_WARPS / 2;            // warps per orientation
constexpr int BWD_ROWS = BWD_T + 2;                 // strip rows: pixel rows -1 .. 32
constexpr int BWD_SPILL = BWD_ROWS;                 // first spill row (a start row clamps to it)
constexpr int BWD_ACC = (BWD_ROWS + 2) * 32;        // one warp's accumulators: [row][lane]
constexpr int BWD_CHUNK = 32;                       // rays a warp stages at a time
// per warp: accumulators, then the staged rays (one float4 each) and their
// orientation / sign flags
constexpr int BWD_WARP_FLOATS = BWD_ACC + 4 * BWD_CHUNK + BWD_CHUNK;
constexpr int BWD_SMEM_FLOATS = BWD_WARPS * BWD_WARP_FLOATS;
static_assert(BWD_ACC >= BWD_T * (BWD_T + 1), "the final sum's staging fits in one warp's accumulators");

// A staged ray, relative to the tile and to the lane's walk index:
// {low and high word of L0'', |M|, c z}.  Lane c takes the tile's column
// (row) X0 + c; with kb = X0 for M > 0 and kb = X0 + 31 for M < 0, and the
// walk index kk = c or 31 - c to match, the span of that column starts at
// lo = L0 + (X0 + c) M = L0 + kb M + kk |M|.  Staging folds L0 + kb M,
// shifted by the strip's first row (base - 1) 2^32, into L0'', so that the
// lane forms lo as one 32 x 32 -> 64-bit product plus L0'' (the same 64-bit
// value the projector walks to) and its top word is the strip row.
__device__ __forceinline__ void bwd_ray(const float4 A, unsigned kk, float *a) {
    const unsigned long long L = ((unsigned long long)__float_as_uint(A.y) << 32) | __float_as_uint(A.x);
    const unsigned Ma = __float_as_uint(A.z);
    const unsigned long long p = (unsigned long long)kk * Ma + L;
    const unsigned row = (unsigned)(p >> 32);
    const unsigned t = (unsigned)p + Ma;
    const unsigned ov1 = t < Ma ? t : 0u;          // t < Ma iff the add wrapped: the span enters row i0 + 1
    const unsigned ov0 = Ma - ov1;
    // strip rows 0 .. BWD_T + 1 are pixel rows -1 .. 32; a span starting
    // anywhere else lands in the spill rows BWD_SPILL and BWD_SPILL + 1.
    // Without a wrap ov1 = 0 and the second update adds an exact zero.
    float *ap = a + min(row, (unsigned)BWD_SPILL) * 32;
    const float a0 = ap[0], a1 = ap[32];
    ap[0] = fmaf(__uint2float_rn(ov0), A.w, a0);
    ap[32] = fmaf(__uint2float_rn(ov1), A.w, a1);
}

// A staged ray, read as one 16-byte shared-memory load (every lane of the
// warp reads the same address).  A plain float4 read was issued as two load
// instructions (ncu: 4.1 instead of 3.1 shared loads per warp evaluation).
__device__ __forceinline__ float4 staged_ray(const float4 *p) {
    float4 q;
    asm("ld.shared.v4.f32 {%0, %1, %2, %3}, [%4];"
        : "=f"(q.x), "=f"(q.y), "=f"(q.z), "=f"(q.w)
        : "r"((unsigned)__cvta_generic_to_shared(p))
        : "memory");
    return q;
}

__device__ __forceinline__ void tile_bwd(const SliceDesc &s, int mode, int tile, float *sm) {
    if (mode == BWD_Q && s.cg->stop) return;
    const int n = s.n, nb = s.nb, V = s.V;
    const int ntxy = tiles_bwd_xy(s), part = tile / ntxy, txy = tile - part * ntxy;
    const int tpr = (n + BWD_T - 1) / BWD_T;
    const int X0 = (txy % tpr) * BWD_T, Y0 = (txy / tpr) * BWD_T;
    for (int i = threadIdx.x; i < BWD_SMEM_FLOATS; i += AIR_THREADS) sm[i] = 0.f;
    __syncthreads();
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const bool colw = warp < BWD_GROUP;             // this warp takes the rays that walk columns
    const unsigned myo = colw ? 1u : 0u;
    const float *__restrict__ Z = mode == BWD_PLAIN ? s.ext_in : s.zc;
    float *wsm = sm + warp * BWD_WARP_FLOATS;
    float *a = wsm + lane;                          // this lane's strip: row r at a + 32 r
    float4 *stA = reinterpret_cast<float4 *>(wsm + BWD_ACC);
    int *stF = reinterpret_cast<int *>(stA + BWD_CHUNK);        // bit 0: walks columns, bit 1: M < 0
    const int S = s.bwd_parts, dv = S * BWD_GROUP;
    const unsigned *__restrict__ vtt = s.vt + (size_t)txy * V;     // this tile's entries, by view

    // an entry this warp works on: a non-empty range holding rays of its orientation
    auto mine = [&](unsigned e) {
        return ((e >> 14) & 0x3fffu) > (e & 0x3fffu) && ((e & VT_MIXED) != 0u || ((e >> 28) & 1u) == myo);
    };
    // ray j of view v into registers (lane = position in the chunk)
    float4 rq = make_float4(0.f, 0.f, 0.f, 0.f);
    float rz = 0.f;
    int ro = 0;
    auto fetch = [&](unsigned e, int v, int j) {
        if (j < (int)((e >> 14) & 0x3fffu)) {
            const size_t ri = (size_t)v * nb + j;
            rq = __ldg(reinterpret_cast<const float4 *>(s.ray + ri));
            rz = __ldg(Z + ri);
            if (e & VT_MIXED) ro = walk_cols(__ldg(s.walk + ri));
        }
    };
    int v = part + S * (warp % BWD_GROUP);
    unsigned e = v < V ? __ldg(vtt + v) : 0u;
    unsigned en = v + dv < V ? __ldg(vtt + v + dv) : 0u;
    if (v < V && mine(e)) fetch(e, v, (int)(e & 0x3fffu) + lane);
#pragma unroll 1
    for (; v < V; v += dv) {
        const int vn = v + dv;
        const unsigned enn = vn + dv < V ? __ldg(vtt + vn + dv) : 0u;   // two views ahead
        if (!mine(e)) {                                                  // nothing here for this warp
            if (vn < V && mine(en)) fetch(en, vn, (int)(en & 0x3fffu) + lane);
            e = en;
            en = enn;
            continue;
        }
        const int j0 = e & 0x3fffu, j1 = (e >> 14) & 0x3fffu;
        const bool mixed = (e & VT_MIXED) != 0u;
#pragma unroll 1
        for (int c0 = j0; c0 < j1; c0 += BWD_CHUNK) {
            {   // stage this lane's ray, tile- and walk-index-relative (see bwd_ray)
                const bool col = mixed ? ro != 0 : colw;
                const unsigned Mlo = __float_as_uint(rq.z);
                const bool neg = __float_as_int(rq.w) < 0;          // the sign of c is the sign of M
                const unsigned kb = (unsigned)(col ? X0 : Y0) + (neg ? BWD_T - 1u : 0u);
                const unsigned hsub = (unsigned)((col ? Y0 : X0) - 1) + (neg ? kb : 0u);
                const unsigned long long L =
                    (unsigned long long)kb * Mlo +
                    (((unsigned long long)__float_as_uint(rq.y) << 32) | __float_as_uint(rq.x)) -
                    ((unsigned long long)hsub << 32);
                stA[lane] = make_float4(__uint_as_float((unsigned)L), __uint_as_float((unsigned)(L >> 32)),
                                        __uint_as_float(neg ? 0u - Mlo : Mlo), fabsf(rq.w) * rz);
                stF[lane] = (int)col | (neg ? 2 : 0);
            }
            __syncwarp();
            const int cnt = min(BWD_CHUNK, j1 - c0);
            // prefetch what is staged next while this chunk is swept: the
            // range's next chunk, else the next view's first
            if (c0 + BWD_CHUNK < j1) fetch(e, v, c0 + BWD_CHUNK + lane);
            else if (vn < V && mine(en)) fetch(en, vn, (int)(en & 0x3fffu) + lane);
            if (!mixed) {
                const unsigned kk = (e & VT_NEG) ? BWD_T - 1u - lane : (unsigned)lane;
#pragma unroll 8
                for (int i = 0; i < cnt; ++i) bwd_ray(staged_ray(stA + i), kk, a);
            } else {
#pragma unroll 1
                for (int i = 0; i < cnt; ++i) {
                    const int f = stF[i];
                    if ((unsigned)(f & 1) != myo) continue;               // the other orientation's ray
                    bwd_ray(staged_ray(stA + i), (f & 2) ? BWD_T - 1u - lane : (unsigned)lane, a);
                }
            }
            __syncwarp();
        }
        e = en;
        en = enn;
    }
    __syncthreads();
    // pixel (lx, ly) of the tile: the column-walking warps hold it at strip
    // row ly + 1, lane lx; the row-walking warps at strip row lx + 1, lane ly.
    // The row-walking sums are read with lanes along ly (no bank conflicts) and
    // handed over through a padded [ly][lx] table in warp BWD_GROUP's area.
    constexpr int PIX = BWD_T * BWD_T / AIR_THREADS;
    float vs[PIX];
#pragma unroll
    for (int q = 0; q < PIX; ++q) {
        const int p = threadIdx.x + q * AIR_THREADS, ly = p & 31, lx = p >> 5;
        float acc = 0.f;
#pragma unroll
        for (int w = BWD_GROUP; w < BWD_WARPS; ++w) acc += sm[w * BWD_WARP_FLOATS + (lx + 1) * 32 + ly];
        vs[q] = acc;
    }
    __syncthreads();
    float *hand = sm + BWD_GROUP * BWD_WARP_FLOATS;
#pragma unroll
    for (int q = 0; q < PIX; ++q) {
        const int p = threadIdx.x + q * AIR_THREADS, ly = p & 31, lx = p >> 5;
        hand[ly * 33 + lx] = vs[q];
    }
    __syncthreads();
#pragma unroll
    for (int q = 0; q < PIX; ++q) {
        const int p = threadIdx.x + q * AIR_THREADS, lx = p & 31, ly = p >> 5;
        float acc = 0.f;
#pragma unroll
        for (int w = 0; w < BWD_GROUP; ++w) acc += sm[w * BWD_WARP_FLOATS + (ly + 1) * 32 + lx];
        acc += hand[ly * 33 + lx];
        const int ix = X0 + lx, iy = Y0 + ly;
        if (ix < n && iy < n) {
            if (S == 1 && mode == BWD_PLAIN) s.ext_out[iy * n + ix] = s.dx * acc;
            else s.bwd_part[(size_t)part * n * n + iy * n + ix] = acc;
        }
    }
    __syncthreads();   // shared memory is reused by the next tile of a persistent block
}


// Sums the S view parts of the backprojection in a fixed order and applies
// the mode's epilogue (the CG and residual updates of the Eq. 5 system).
__device__ __forceinline__ void tile_bwd_fin(const SliceDesc &s, int mode, int tile) {
    __shared__ double sh[AIR_THREADS / 32];
    if (mode == BWD_Q && s.cg->stop) return;
    const int nn = s.n * s.n, S = s.bwd_parts;
    const int base = tile * VEC_PER_TILE;
    double part = 0.0;
#pragma unroll
    for (int k = 0; k < 4; ++k) {
        const int i = base + k * AIR_THREADS + threadIdx.x;
        if (i >= nn) continue;
        float a = 0.f;
        for (int p = 0; p < S; ++p) a += __ldcg(s.bwd_part + (size_t)p * nn + i);
        const float acc = s.dx * a;
        if (mode == BWD_PLAIN) {
            s.ext_out[i] = acc;
        } else if (mode == BWD_RHS0) {
            s.rhs0[i] = acc;
        } else if (mode == BWD_RESID) {
            const float mx = fmaf(s.mu, s.x[i], acc);
            const float rv = fmaf(s.mu, s.g[i], s.rhs0[i]) - mx;
            s.r[i] = rv;
            s.p[i] = rv;
            part += (double)rv * (double)rv;
        } else {  // BWD_Q
            const float pv = s.p[i];
            const float qv = fmaf(s.mu, pv, acc);
            s.q[i] = qv;
            part += (double)pv * (double)qv;
        }
    }
    if (mode == BWD_PLAIN || mode == BWD_RHS0) return;
    part = block_sum(part, sh);
    double tot;
    if (reduce_tiles(s, tile, tiles_vec(s), part, sh, &tot) && threadIdx.x == 0) {
        CgState *c = s.cg;
        if (mode == BWD_RESID) {
            c->rho = tot;
            c->stop = !(tot != 0.0);
        } else {
            c->pq = tot;
            if (!(tot > 0.0)) c->stop = 1;
            else c->alpha = c->rho / tot;
        }
    }
}

// ======================================================================
// Ramp filtration C (Eq. 2), FP32 on the CUDA cores.  Per view, with taps =
// c0 h (h[0] = 1/4, h[odd m] = -1/(pi m)^2) and samples outside the detector
// zero (a linear convolution):
//   Z[j] = taps[0] Y[j] + sum_{odd m} taps[m] (Y[j-m] + Y[j+m]).
// Evaluated in the algebraically equal DIFFERENCE form
//   Z[j] = diag Y[j] + sum_{odd m} taps[m] ((Y[j-m] - Y[j]) + (Y[j+m] - Y[j])),
//   diag = taps[0] + 2 sum_{odd m < n_b} taps[m],
// whose terms are differences of neighbouring samples instead of large
// values that cancel (the ramp is a high-pass filter): it keeps the FP32
// result within a few 1e-7 of the exact convolution where the direct form
// loses two digits.  One view per tile; each thread owns RAMP_R consecutive
// outputs and slides its left/right sample windows by two per tap.
// ======================================================================
constexpr int RAMP_R = 4;

__device__ __forceinline__ void tile_ramp(const SliceDesc &s, int arg, int tile, float *sm) {
    const float *src = arg == RSRC_Y ? s.y : (arg == RSRC_Z ? s.z : s.ext_in);
    float *dst = arg == RSRC_EXT ? s.ext_out : s.zc;
    const int nb = s.nb;
    const size_t off = (size_t)tile * nb;
    if (arg == RSRC_Z && s.cg->stop) return;
    if (!s.filter) {
        for (int j = threadIdx.x; j < nb; j += AIR_THREADS) dst[off + j] = src[off + j];
        return;
    }
    // P(PO + k) = Y[k] for 0 <= k < nb, zero elsewhere.  The windows reach
    // from j - (nb-1) - 2 (the prefetch after the last tap) to
    // j + RAMP_R + nb, so the padding is nb + 2 on the left and nb + R + 4 on
    // the right of any output j < nb.  P is stored de-interleaved by residue
    // mod 4, P(k) at (k & 3) * PQ + (k >> 2): a thread owns RAMP_R = 4
    // consecutive outputs, so in every load all threads of a warp share the
    // residue and read consecutive words (no bank conflicts).
    const int PO = nb + 2;
    const int plen = 3 * nb + 2 * RAMP_R + 4;
    const int PQ = (plen + 3) >> 2;
    float *P = sm, *tp = sm + 4 * PQ;
    const float *__restrict__ pw = s.prew;
    for (int k = threadIdx.x; k < plen; k += AIR_THREADS) {
        const int i = k - PO;
        P[(k & 3) * PQ + (k >> 2)] = (i >= 0 && i < nb) ? (pw ? src[off + i] * __ldg(pw + i) : src[off + i]) : 0.f;
    }
    for (int k = threadIdx.x; k < nb; k += AIR_THREADS) tp[k] = __ldg(s.taps + k);
    __syncthreads();
    const float diag = s.ramp_diag;
#pragma unroll 1
    for (int j0 = threadIdx.x * RAMP_R; j0 < nb; j0 += AIR_THREADS * RAMP_R) {
        // value at output offset o from j0: P(PO + j0 + o); j0 is a multiple of 4
        const int jq = j0 >> 2;
        auto at = [&](int o) { const int k = PO + o; return P[(k & 3) * PQ + (k >> 2) + jq]; };
        // taps from the outermost odd lag inward: the terms grow as the lag
        // shrinks (taps ~ 1/m^2), and summing the small ones first keeps the
        // FP32 sum within a few ulp even for long noisy rows
        const int mmax = (nb - 1) & 1 ? nb - 1 : nb - 2;   // largest odd lag < nb (-1: none)
        float ctr[RAMP_R], L[RAMP_R], R[RAMP_R], acc[RAMP_R];
#pragma unroll
        for (int i = 0; i < RAMP_R; ++i) {
            ctr[i] = at(i);
            L[i] = at(i - mmax);       // Y[j - m], m = mmax
            R[i] = at(i + mmax);       // Y[j + m], m = mmax
            acc[i] = 0.f;
        }
#pragma unroll 2
        for (int m = mmax; m >= 1; m -= 2) {
            const float h = tp[m];
#pragma unroll
            for (int i = 0; i < RAMP_R; ++i)
                acc[i] = fmaf(h, __fadd_rn(__fsub_rn(L[i], ctr[i]), __fsub_rn(R[i], ctr[i])), acc[i]);
            // slide to m - 2: the left window moves up by two, the right down by two
#pragma unroll
            for (int i = 0; i < RAMP_R - 2; ++i) L[i] = L[i + 2];
            L[RAMP_R - 2] = at(RAMP_R - 2 - m + 2);
            L[RAMP_R - 1] = at(RAMP_R - 1 - m + 2);
#pragma unroll
            for (int i = RAMP_R - 1; i >= 2; --i) R[i] = R[i - 2];
            R[1] = at(1 + m - 2);
            R[0] = at(m - 2);
        }
#pragma unroll
        for (int i = 0; i < RAMP_R; ++i)
            if (j0 + i < nb) dst[off + j0 + i] = fmaf(diag, ctr[i], acc[i]);
    }
    __syncthreads();
}

// ======================================================================
// Fan-beam FBP (the analytic reconstruction the Materials section compares
// AIR with; the textbook equiangular algorithm): after the filter
// Q_v(j) = sum_k fbp_taps[|j-k|] cos(gamma_k) Y_v(k), the weighted
// backprojection
//   f(x, y) = dbeta / dx^2 sum_v Q_v(gamma') / L^2
// with gamma' the fan angle of the pixel centre seen from the source of view
// v, L its distance from the source (pixels), and Q linearly interpolated
// between bins, zero beyond the detector.  With the central direction
// c = (cx, cy) of the view (the central ray passes through the centre), the
// source-relative products are L sin(gamma') = cx y - cy x and
// L cos(gamma') = D + cx x + cy y, which stay accurate in FP32.
// One thread per pixel, 16 x 16 pixels per block.
// ======================================================================
// arctan(u) for |u| <= 0.45 by its Maclaurin (Gregory) series through u^13;
// the alternating-series remainder is below 0.45^15/15 = 4.2e-7 rad.
__device__ __forceinline__ float atan_series(float u) {
    const float w = u * u;
    float p = 1.f / 13.f;
    p = fmaf(p, w, -1.f / 11.f);
    p = fmaf(p, w, 1.f / 9.f);
    p = fmaf(p, w, -1.f / 7.f);
    p = fmaf(p, w, 1.f / 5.f);
    p = fmaf(p, w, -1.f / 3.f);
    p = fmaf(p, w, 1.f);
    return u * p;
}

__device__ __forceinline__ void tile_fbp(const SliceDesc &s, int tile) {
    const int n = s.n, nb = s.nb, tpr = (n + SHR_T - 1) / SHR_T;
    const int ix = (tile % tpr) * SHR_T + (int)threadIdx.x % SHR_T;
    const int iy = (tile / tpr) * SHR_T + (int)threadIdx.x / SHR_T;
    if (ix >= n || iy >= n) return;
    const float x = (float)ix + 0.5f - s.half_n, y = (float)iy + 0.5f - s.half_n;
    const float *__restrict__ Q = s.zc;
    float acc = 0.f;
#pragma unroll 2
    for (int v = 0; v < s.V; ++v, Q += nb) {
        const float2 c = __ldg(s.fview + v);
        const float cr = fmaf(c.x, y, -c.y * x);                 // L sin(gamma')
        const float dt = fmaf(c.x, x, fmaf(c.y, y, s.dso_px));   // L cos(gamma') > 0
        const float u = cr / dt;
        const float gp = fabsf(u) <= 0.45f ? atan_series(u) : atan2f(cr, dt);
        // bin position t = gp / alpha + jmid: its integer part from a rounded
        // t, its fraction as an FMA residual against that integer with 1/alpha
        // in two parts, so neither t's magnitude (~n_b/2) nor 1/alpha's
        // rounding costs digits of the interpolation weight
        const float tr = floorf(fmaf(gp, s.inv_dg, s.jmid));
        float w = fmaf(gp, s.inv_dg, s.jmid - tr);
        w = fmaf(gp, s.inv_dg_lo, w);
        const int j0 = (int)tr + (w < 0.f ? -1 : (w >= 1.f ? 1 : 0));
        w = w < 0.f ? w + 1.f : (w >= 1.f ? w - 1.f : w);
        const float q0 = (unsigned)j0 < (unsigned)nb ? __ldg(Q + j0) : 0.f;
        const float q1 = (unsigned)(j0 + 1) < (unsigned)nb ? __ldg(Q + j0 + 1) : 0.f;
        acc += __fdividef(fmaf(w, q1 - q0, q0), fmaf(cr, cr, dt * dt));
    }
    s.ext_out[(size_t)iy * n + ix] = s.fbp_scale * acc;
}

// ======================================================================
// CG vector updates (Eq. 5 system) with FP64 inner products.
// ======================================================================
__device__ __forceinline__ void tile_cg_a(const SliceDesc &s, int tile) {
    __shared__ double sh[AIR_THREADS / 32];
    if (s.cg->stop) return;
    const float a = (float)s.cg->alpha;
    const int nn = s.n * s.n;
    const int base = tile * VEC_PER_TILE;
    double part = 0.0;
#pragma unroll
    for (int k = 0; k < 4; ++k) {
        const int i = base + k * AIR_THREADS + threadIdx.x;
        if (i < nn) {
            s.x[i] = fmaf(a, s.p[i], s.x[i]);
            const float rv = fmaf(-a, s.q[i], s.r[i]);
            s.r[i] = rv;
            part += (double)rv * (double)rv;
        }
    }
    part = block_sum(part, sh);
    double tot;
    if (reduce_tiles(s, tile, tiles_vec(s), part, sh, &tot) && threadIdx.x == 0) {
        CgState *c = s.cg;
        c->beta = tot / c->rho;
        c->rho = tot;
        if (!(tot != 0.0)) c->stop = 1;
    }
}

__device__ __forceinline__ void tile_cg_b(const SliceDesc &s, int tile) {
    if (s.cg->stop) return;
    const float bt = (float)s.cg->beta;
    const int nn = s.n * s.n;
    const int base = tile * VEC_PER_TILE;
#pragma unroll
    for (int k = 0; k < 4; ++k) {
        const int i = base + k * AIR_THREADS + threadIdx.x;
        if (i < nn) s.p[i] = fmaf(bt, s.p[i], s.r[i]);
    }
}

// The CG restart of an outer split-Bregman step.  CG keeps r = b - M x, so
// when the right-hand side b = A'^T Y + mu W^T(d - b') changes only by
// mu (g_new - g_old) between outer steps, the new residual is
// r + mu (g_new - g_old) with no operator application; at X = 0 it is
// A'^T Y.  arg = -1: r = rhs0; arg = parity of the outer step that just
// shrank (its g went to g2 if odd, g if even): r += mu (g_new - g_old).
// Then p = r and rho = r.r (FP64), and the CG restarts unless rho = 0.
__device__ __forceinline__ void tile_restart(const SliceDesc &s, int arg, int tile) {
    __shared__ double sh[AIR_THREADS / 32];
    const int nn = s.n * s.n;
    const int base = tile * VEC_PER_TILE;
    const float *gn = arg == 1 ? s.g2 : s.g, *go = arg == 1 ? s.g : s.g2;
    double part = 0.0;
#pragma unroll
    for (int k = 0; k < 4; ++k) {
        const int i = base + k * AIR_THREADS + threadIdx.x;
        if (i < nn) {
            const float rv = arg < 0 ? s.rhs0[i] : fmaf(s.mu, gn[i] - go[i], s.r[i]);
            s.r[i] = rv;
            s.p[i] = rv;
            part += (double)rv * (double)rv;
        }
    }
    part = block_sum(part, sh);
    double tot;
    if (reduce_tiles(s, tile, tiles_vec(s), part, sh, &tot) && threadIdx.x == 0) {
        CgState *c = s.cg;
        c->rho = tot;
        c->stop = !(tot != 0.0);
    }
}

// q = x + step r: the forward step of forward-backward splitting (Eq. 6),
// with r = A'^T (Y - A x) from the OP_BWD_FIN residual epilogue at mu = 0.
__device__ __forceinline__ void tile_axpy(const SliceDesc &s, int tile) {
    const int nn = s.n * s.n;
    const int base = tile * VEC_PER_TILE;
#pragma unroll
    for (int k = 0; k < 4; ++k) {
        const int i = base + k * AIR_THREADS + threadIdx.x;
        if (i < nn) s.q[i] = fmaf(s.step, s.r[i], s.x[i]);
    }
}

__device__ __forceinline__ void tile_zero(const SliceDesc &s, int tile) {
    const int nn = s.n * s.n;
    const int base = tile * VEC_PER_TILE;
#pragma unroll
    for (int k = 0; k < 4; ++k) {
        const int i = base + k * AIR_THREADS + threadIdx.x;
        if (i < nn) {
            s.x[i] = 0.f;
            s.g[i] = 0.f;
            s.g2[i] = 0.f;
#pragma unroll
            for (int band = 0; band < 9; ++band) s.b[(size_t)band * nn + i] = 0.f;
        }
    }
    if (tile == 0 && threadIdx.x == 0) {
        s.cg->stop = 0;
        s.cg->outer = 0;
        s.cg->counter = 0u;
    }
}

// ======================================================================
// Tensor framelet (piecewise-linear, one level, periodic) and the fused
// split-Bregman shrink.  Taps at offsets -1, 0, +1:
//   h0 = [1,2,1]/4, h1 = (sqrt2/4)[1,0,-1], h2 = [-1,2,-1]/4;
//   (W_ab X)[y][x] = sum_{p,q} h_a[p] h_b[q] X[y+p][x+q]   (indices mod n)
// ======================================================================
__device__ __forceinline__ float ftap(int a, int p) {
    const float s2 = 0.35355339059327373f;  // sqrt(2)/4
    return a == 0 ? (p == 0 ? 0.5f : 0.25f) : (a == 1 ? (p == 0 ? 0.f : (p < 0 ? s2 : -s2)) : (p == 0 ? 0.5f : -0.25f));
}

__device__ __forceinline__ int wrapi(int v, int n) {
    v %= n;
    return v < 0 ? v + n : v;
}

// W at one position from a 3x3 neighbourhood nb3[p+1][q+1] = X[y+p][x+q]
__device__ __forceinline__ void framelet9(const float nb3[3][3], float out[9]) {
    float rowf[3][3];  // rowf[b][p+1] = sum_q h_b[q] X[y+p][x+q]
#pragma unroll
    for (int p = 0; p < 3; ++p) {
        rowf[0][p] = 0.25f * (nb3[p][0] + nb3[p][2]) + 0.5f * nb3[p][1];
        rowf[1][p] = 0.35355339059327373f * (nb3[p][0] - nb3[p][2]);
        rowf[2][p] = 0.5f * nb3[p][1] - 0.25f * (nb3[p][0] + nb3[p][2]);
    }
#pragma unroll
    for (int b = 0; b < 3; ++b) {
        out[0 * 3 + b] = 0.25f * (rowf[b][0] + rowf[b][2]) + 0.5f * rowf[b][1];
        out[1 * 3 + b] = 0.35355339059327373f * (rowf[b][0] - rowf[b][2]);
        out[2 * 3 + b] = 0.5f * rowf[b][1] - 0.25f * (rowf[b][0] + rowf[b][2]);
    }
}

// W^T at one position of band c: sum_{p,q} h_a[p] h_b[q] C[y-p][x-q], with
// e3[p+1][q+1] = C[y+p][x+q] (so offset -p is index 1-p).
__device__ __forceinline__ float framelet_t1(int a, int b, const float e3[3][3]) {
    float acc = 0.f;
#pragma unroll
    for (int p = -1; p <= 1; ++p) {
        float rs = 0.f;
#pragma unroll
        for (int q = -1; q <= 1; ++q) rs = fmaf(ftap(b, q), e3[1 - p][1 - q], rs);
        acc = fmaf(ftap(a, p), rs, acc);
    }
    return acc;
}

// The Bregman variable is double-buffered: a tile reads b in its halo,
// which neighbouring tiles are updating, so the update reads b_in and writes
// b_out (the solver alternates the two buffers between outer steps).
struct ShrinkArgs {
    const float *X;
    const float *b_in;
    float *b_out;
    float *g;
    float tau;
};

constexpr int SHR_H = SHR_T + 2;   // coefficient tile incl. halo 1
constexpr int SHR_X = SHR_T + 4;   // image tile incl. halo 2

// Shared-memory layout of the shrink tile (floats): X tile, then E[9][SHR_H^2]
constexpr int SHR_SMEM_FLOATS = SHR_X * SHR_X + 9 * SHR_H * SHR_H;

__device__ __forceinline__ void tile_shrink(const SliceDesc &s, const ShrinkArgs &A, int tile,
                                            bool reduce, double *resid_dst, float *sm) {
    __shared__ double sh[AIR_THREADS / 32];
    const int n = s.n, nn = n * n;
    const int tpr = (n + SHR_T - 1) / SHR_T;
    const int x0 = (tile % tpr) * SHR_T, y0 = (tile / tpr) * SHR_T;
    float *Xs = sm;                      // [SHR_X][SHR_X], origin (y0-2, x0-2)
    float *E = sm + SHR_X * SHR_X;       // [9][SHR_H][SHR_H], origin (y0-1, x0-1)
    for (int k = threadIdx.x; k < SHR_X * SHR_X; k += AIR_THREADS) {
        const int ly = k / SHR_X, lx = k % SHR_X;
        Xs[k] = A.X[wrapi(y0 - 2 + ly, n) * n + wrapi(x0 - 2 + lx, n)];
    }
    __syncthreads();
    double part = 0.0;
    for (int k = threadIdx.x; k < SHR_H * SHR_H; k += AIR_THREADS) {
        const int cy = k / SHR_H, cx = k % SHR_H;
        const int gy = wrapi(y0 - 1 + cy, n), gx = wrapi(x0 - 1 + cx, n);
        const bool interior = cy >= 1 && cy <= SHR_T && cx >= 1 && cx <= SHR_T &&
                              y0 - 1 + cy < n && x0 - 1 + cx < n;
        float nb3[3][3];
#pragma unroll
        for (int p = 0; p < 3; ++p)
#pragma unroll
            for (int q = 0; q < 3; ++q) nb3[p][q] = Xs[(cy + p) * SHR_X + cx + q];
        float wx[9];
        framelet9(nb3, wx);
        const size_t gi = (size_t)gy * n + gx;
#pragma unroll
        for (int band = 0; band < 9; ++band) {
            const float bo = A.b_in[(size_t)band * nn + gi];
            const float t = wx[band] + bo;
            float d = t;
            if (band > 0) {
                const float m = fabsf(t) - A.tau;
                d = m > 0.f ? copysignf(m, t) : 0.f;
            }
            const float bn = t - d;
            E[band * SHR_H * SHR_H + k] = d - bn;
            if (interior) {
                A.b_out[(size_t)band * nn + gi] = bn;
                const double e = (double)wx[band] - (double)d;
                part += e * e;
            }
        }
    }
    __syncthreads();
    for (int k = threadIdx.x; k < SHR_T * SHR_T; k += AIR_THREADS) {
        const int ly = k / SHR_T, lx = k % SHR_T;
        if (y0 + ly >= n || x0 + lx >= n) continue;
        float acc = 0.f;
#pragma unroll
        for (int band = 0; band < 9; ++band) {
            float e3[3][3];
            const float *Eb = E + band * SHR_H * SHR_H;
#pragma unroll
            for (int p = 0; p < 3; ++p)
#pragma unroll
                for (int q = 0; q < 3; ++q) e3[p][q] = Eb[(ly + p) * SHR_H + lx + q];
            acc += framelet_t1(band / 3, band % 3, e3);
        }
        A.g[(size_t)(y0 + ly) * n + x0 + lx] = acc;
    }
    if (!reduce) {
        __syncthreads();
        return;
    }
    part = block_sum(part, sh);
    double tot;
    if (reduce_tiles(s, tile, tiles_shr(s), part, sh, &tot) && threadIdx.x == 0) {
        const double rn = sqrt(tot);
        CgState *c = s.cg;
        c->resid = rn;
        if (resid_dst) *resid_dst = rn;
        if (s.resid_out) s.resid_out[c->outer] = rn;
        c->outer += 1;
    }
    __syncthreads();
}

// The proximal step of forward-backward splitting for R = ||W X||_1 with the
// tight frame W (W^T W = I): x = W^T S_tau(W q), the high-pass bands
// soft-thresholded by tau = step * lambda and the low-pass band kept.  Reads q
// (with a 2-pixel periodic halo) and writes x, so tiles never read what
// another tile writes.
__device__ __forceinline__ void tile_prox(const SliceDesc &s, int tile, float *sm) {
    const int n = s.n;
    const int tpr = (n + SHR_T - 1) / SHR_T;
    const int x0 = (tile % tpr) * SHR_T, y0 = (tile / tpr) * SHR_T;
    float *Xs = sm;                      // [SHR_X][SHR_X], origin (y0-2, x0-2)
    float *E = sm + SHR_X * SHR_X;       // [9][SHR_H][SHR_H], origin (y0-1, x0-1)
    for (int k = threadIdx.x; k < SHR_X * SHR_X; k += AIR_THREADS) {
        const int ly = k / SHR_X, lx = k % SHR_X;
        Xs[k] = s.q[wrapi(y0 - 2 + ly, n) * n + wrapi(x0 - 2 + lx, n)];
    }
    __syncthreads();
    for (int k = threadIdx.x; k < SHR_H * SHR_H; k += AIR_THREADS) {
        const int cy = k / SHR_H, cx = k % SHR_H;
        float nb3[3][3];
#pragma unroll
        for (int p = 0; p < 3; ++p)
#pragma unroll
            for (int q = 0; q < 3; ++q) nb3[p][q] = Xs[(cy + p) * SHR_X + cx + q];
        float wx[9];
        framelet9(nb3, wx);
#pragma unroll
        for (int band = 0; band < 9; ++band) {
            float d = wx[band];
            if (band > 0) {
                const float m = fabsf(d) - s.tau;
                d = m > 0.f ? copysignf(m, d) : 0.f;
            }
            E[band * SHR_H * SHR_H + k] = d;
        }
    }
    __syncthreads();
    for (int k = threadIdx.x; k < SHR_T * SHR_T; k += AIR_THREADS) {
        const int ly = k / SHR_T, lx = k % SHR_T;
        if (y0 + ly >= n || x0 + lx >= n) continue;
        float acc = 0.f;
#pragma unroll
        for (int band = 0; band < 9; ++band) {
            float e3[3][3];
            const float *Eb = E + band * SHR_H * SHR_H;
#pragma unroll
            for (int p = 0; p < 3; ++p)
#pragma unroll
                for (int q = 0; q < 3; ++q) e3[p][q] = Eb[(ly + p) * SHR_H + lx + q];
            acc += framelet_t1(band / 3, band % 3, e3);
        }
        s.x[(size_t)(y0 + ly) * n + x0 + lx] = acc;
    }
    __syncthreads();
}

// out = W in (adjoint = 0) or W^T in (adjoint = 1), for the API call.
__device__ __forceinline__ void tile_framelet(const SliceDesc &s, int adjoint, int tile, float *sm) {
    const int n = s.n, nn = n * n;
    const int tpr = (n + SHR_T - 1) / SHR_T;
    const int x0 = (tile % tpr) * SHR_T, y0 = (tile / tpr) * SHR_T;
    const float *in = s.ext_in;
    float *out = s.ext_out;
    const int bands = adjoint ? 9 : 1;
    for (int k = threadIdx.x; k < bands * SHR_H * SHR_H; k += AIR_THREADS) {
        const int band = k / (SHR_H * SHR_H), rem = k % (SHR_H * SHR_H);
        const int ly = rem / SHR_H, lx = rem % SHR_H;
        sm[k] = in[(size_t)band * nn + wrapi(y0 - 1 + ly, n) * n + wrapi(x0 - 1 + lx, n)];
    }
    __syncthreads();
    for (int k = threadIdx.x; k < SHR_T * SHR_T; k += AIR_THREADS) {
        const int ly = k / SHR_T, lx = k % SHR_T;
        if (y0 + ly >= n || x0 + lx >= n) continue;
        const size_t gi = (size_t)(y0 + ly) * n + x0 + lx;
        if (!adjoint) {
            float nb3[3][3], wx[9];
#pragma unroll
            for (int p = 0; p < 3; ++p)
#pragma unroll
                for (int q = 0; q < 3; ++q) nb3[p][q] = sm[(ly + p) * SHR_H + lx + q];
            framelet9(nb3, wx);
#pragma unroll
            for (int band = 0; band < 9; ++band) out[(size_t)band * nn + gi] = wx[band];
        } else {
            float acc = 0.f;
#pragma unroll
            for (int band = 0; band < 9; ++band) {
                float e3[3][3];
#pragma unroll
                for (int p = 0; p < 3; ++p)
#pragma unroll
                    for (int q = 0; q < 3; ++q) e3[p][q] = sm[band * SHR_H * SHR_H + (ly + p) * SHR_H + lx + q];
                acc += framelet_t1(band / 3, band % 3, e3);
            }
            out[gi] = acc;
        }
    }
    __syncthreads();
}

// Dynamic shared memory (bytes) a tile of `op` needs for a slice.
__host__ inline size_t tile_smem(const SliceDesc &s, int op) {
    switch (op) {
    case OP_RAMP: return sizeof(float) * (4 * (size_t)((3 * s.nb + 2 * RAMP_R + 4 + 3) / 4) + (size_t)s.nb);
    case OP_SHRINK: case OP_PROX: return sizeof(float) * SHR_SMEM_FLOATS;
    case OP_FRAMELET: case OP_FRAMELET_T: return sizeof(float) * 9 * SHR_H * SHR_H;
    case OP_TRANSPOSE: return sizeof(float) * 32 * 33;
    case OP_BWD: return sizeof(float) * BWD_SMEM_FLOATS;
    default: return 0;
    }
}

// The shrink of outer step k of the solver, arg = k & 1: the Bregman
// variable goes b -> b2 on even steps and b2 -> b on odd ones, and g to g on
// even steps and to g2 on odd ones (the restart needs the previous g).
__device__ __forceinline__ void run_shrink(const SliceDesc &s, int arg, int tile, float *sm) {
    ShrinkArgs a{s.x, arg ? s.b2 : s.b, arg ? s.b : s.b2, arg ? s.g2 : s.g, s.tau};
    tile_shrink(s, a, tile, true, nullptr, sm);
}

// One tile of any op (used by the persistent kernel).
__device__ __forceinline__ void run_tile(const SliceDesc &s, int op, int arg, int tile, float *sm) {
    switch (op) {
    case OP_FWD: tile_fwd(s, arg, tile); break;
    case OP_TRANSPOSE: tile_transpose(s, arg, tile, sm); break;
    case OP_RAMP: tile_ramp(s, arg, tile, sm); break;
    case OP_BWD: tile_bwd(s, arg, tile, sm); break;
    case OP_BWD_FIN: tile_bwd_fin(s, arg, tile); break;
    case OP_CG_A: tile_cg_a(s, tile); break;
    case OP_CG_B: tile_cg_b(s, tile); break;
    case OP_ZERO: tile_zero(s, tile); break;
    case OP_AXPY: tile_axpy(s, tile); break;
    case OP_PROX: tile_prox(s, tile, sm); break;
    case OP_FBP: tile_fbp(s, tile); break;
    case OP_SHRINK: run_shrink(s, arg, tile, sm); break;
    case OP_RESTART: tile_restart(s, arg, tile); break;
    default: break;
    }
}

}  // namespace air
