// Ramp filtration C (Eq. 2) on the 5th-generation tensor cores (tcgen05),
// AIR_PREC_BF16X3.
//
// Z = c0 Y T with T the symmetric Toeplitz matrix of the Ram-Lak taps.  T is
// split by lag:
//   near band |j - k| < NEAR: FP32 on the CUDA cores in the cancellation-free
//     difference form (the same algebra as the FP32 filter), fused with the
//     split of Y below (k_split_near);
//   far band: a dense GEMM  Z_far = Y T_far  on tensor cores with operands in
//     split BF16: Y = Yh + Ym + Yl and T_far = Th + Tm + Tl, each piece BF16
//     (24 significant bits in all), and the six products of order >= 2^-16,
//     Yh Th + Yh Tm + Ym Th + Ym Tm + Yh Tl + Yl Th, accumulated in FP32 in
//     tensor memory (k_ramp_gemm).  The far taps are below c0/(pi^2 NEAR^2), so
//     the split's rounding reaches Z only at the 1e-7 level.  The ramp's even
//     lags are zero, so even output bins take only odd input bins and odd
//     outputs only even inputs: the GEMM runs as two half-size products, one
//     per output parity, with Y's columns ordered odd bins first, then even.
//   The products are kept in four TMEM accumulators by magnitude -- Yh Th
//   over the first and over the second half of K, the 2^-9-scale pair, and
//   the 2^-18-scale triple -- and summed small to large in the epilogue, so
//   that small terms are never added into a large running sum inside the
//   tensor core, whose accumulation error then stays at the 1e-7 level too.
//
// k_ramp_gemm: one CTA per 128 views x 64 bins of one parity of Z, 128 threads.  Thread 0
// streams 64-bin K chunks of the six operand pieces (3 of Y, 3 of T_far) with
// TMA into a 3-stage ring of 128-byte-swizzled shared-memory tiles and issues
// tcgen05.mma (M = 128, N = 64, K = 16) into a TMEM accumulator; the four
// warps then read it back with tcgen05.ld and add it to the near-band part.
// Every wait on an mbarrier is bounded: on expiry the kernel records an error
// in the plan's status word, waits (bounded) for its own copies and MMAs and
// frees its TMEM before returning.
#include <cuda.h>
#include <cuda_bf16.h>
#include <cudaTypedefs.h>

#include <cmath>
#include <cstring>
#include <string>
#include <vector>

#include "ramp_tc.h"

namespace air {

namespace {

constexpr int NEAR = 64;          // lags |m| < NEAR stay in FP32
constexpr int TM = 128, TN = 64, TK = 64;
constexpr int STAGES = 3;
constexpr int NACC = 4;                         // TMEM accumulators of TN columns each
constexpr uint32_t TMEM_COLS = NACC * TN;       // 256
constexpr int A_TILE = TM * TK * 2;             // bytes of one Y piece tile
constexpr int B_TILE = TN * TK * 2;             // bytes of one T piece tile
constexpr int STAGE_BYTES = 3 * A_TILE + 3 * B_TILE;
constexpr int GEMM_SMEM = STAGES * STAGE_BYTES + 1024 + 256;
constexpr long long WAIT_POLLS = 1ll << 24;     // bounded waits (~seconds with back-off)
static_assert(TM * (TN + 1) * 4 <= STAGES * STAGE_BYTES, "the epilogue's table fits in the stage ring");

// padded K (= N = bins): a multiple of 2 TK, so each parity's half is whole K chunks
constexpr int KPAD = 2 * TK;
static_assert(TN == TK, "both parities' halves of N are whole tiles");
// column of input bin k within one split piece of Y: odd bins, then even bins
__host__ __device__ inline int a_col(int k, int kh) { return (k & 1) ? (k >> 1) : kh + (k >> 1); }

struct TcRes {
    int kp = 0, np = 0;           // padded K (= bins) and N; kh = kp / 2 per parity
    __nv_bfloat16 *a = nullptr;   // [V][3 kp]: Yh | Ym | Yl per view, each [odd bins | even bins]
    __nv_bfloat16 *b = nullptr;   // [2 parities][3 pieces][np / 2][kp / 2]: T_far[2i + h][input bin of column l]
    float *near_taps = nullptr;   // [NEAR] c0 h[m], m < NEAR
    int *err = nullptr;           // device status word (0 = ok)
    char *mem = nullptr;
    CUtensorMap map_a, map_b;
    float near_diag = 0.f;        // taps[0] + 2 sum_{odd m < NEAR} taps[m]
};

// ------------------------------------------------------------ PTX wrappers
__device__ __forceinline__ uint32_t smem_u32(const void *p) {
    return (uint32_t)__cvta_generic_to_shared(p);
}
__device__ __forceinline__ void mbar_init(uint64_t *bar, uint32_t count) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(bar)), "r"(count) : "memory");
}
__device__ __forceinline__ void mbar_expect_tx(uint64_t *bar, uint32_t bytes) {
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_u32(bar)), "r"(bytes)
                 : "memory");
}
__device__ __forceinline__ bool mbar_test(uint64_t *bar, uint32_t parity) {
    uint32_t ok;
    asm volatile(
        "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n selp.u32 %0, 1, 0, p;\n}"
        : "=r"(ok)
        : "r"(smem_u32(bar)), "r"(parity)
        : "memory");
    return ok != 0;
}
// Poll budget of the K loop's waits for a stage's operands when >= 0 (see
// air_set_wait_budget; one copy per device); the waits that drain a CTA's
// own copies and MMAs before it leaves always keep WAIT_POLLS, so a CTA
// that gives up never exits with a copy or an MMA in flight.
__device__ long long g_tc_wait_budget = -1;

// Bounded wait for the completion of the phase with the given parity.
__device__ __forceinline__ bool mbar_wait(uint64_t *bar, uint32_t parity, long long polls = WAIT_POLLS) {
    for (long long i = 0; i < polls; ++i) {
        if (mbar_test(bar, parity)) return true;
        if (i > 32) __nanosleep(128);
    }
    return false;
}
__device__ __forceinline__ void tma_load_2d(void *dst, const CUtensorMap *map, uint64_t *bar, int x, int y) {
    asm volatile(
        "cp.async.bulk.tensor.2d.shared::cluster.global.tile.mbarrier::complete_tx::bytes [%0], [%1, {%2, %3}], "
        "[%4];" ::"r"(smem_u32(dst)),
        "l"(reinterpret_cast<uint64_t>(map)), "r"(x), "r"(y), "r"(smem_u32(bar))
        : "memory");
}
// 64-bit shared-memory matrix descriptor of a K-major tile with 128-byte
// swizzle: rows of 128 bytes, 8-row groups 1024 bytes apart.
__device__ __forceinline__ uint64_t sw128_desc(const void *tile) {
    const uint64_t addr = smem_u32(tile);
    uint64_t d = (addr >> 4) & 0x3FFFull;          // start address
    d |= 1ull << 16;                              // leading byte offset (unused for this layout)
    d |= (uint64_t)(1024 >> 4) << 32;             // stride byte offset: 8 rows x 128 B
    d |= 1ull << 46;                              // descriptor version
    d |= 2ull << 61;                              // 128-byte swizzle
    return d;
}
// Instruction descriptor: D F32, A and B BF16, both K-major, N = TN, M = TM.
constexpr uint32_t IDESC = (1u << 4) | (1u << 7) | (1u << 10) | ((uint32_t)(TN >> 3) << 17) |
                           ((uint32_t)(TM >> 4) << 24);

__device__ __forceinline__ void umma(uint32_t d_tmem, uint64_t a, uint64_t b, uint32_t accumulate) {
    asm volatile(
        "{\n .reg .pred p;\n setp.ne.b32 p, %4, 0;\n tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n}" ::"r"(
            d_tmem),
        "l"(a), "l"(b), "r"(IDESC), "r"(accumulate)
        : "memory");
}
__device__ __forceinline__ void umma_commit(uint64_t *bar) {
    asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(smem_u32(bar))
                 : "memory");
}
__device__ __forceinline__ void tc_fence_before() { asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory"); }
__device__ __forceinline__ void tc_fence_after() { asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory"); }

__device__ __forceinline__ void tmem_ld16(uint32_t taddr, float *out) {
    uint32_t r[16];
    asm volatile(
        "tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0, %1, %2, %3, %4, %5, %6, %7, %8, %9, %10, %11, %12, %13, %14, "
        "%15}, [%16];"
        : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]),
          "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]), "=r"(r[15])
        : "r"(taddr));
    asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
#pragma unroll
    for (int i = 0; i < 16; ++i) out[i] = __uint_as_float(r[i]);
}

// ------------------------------------------------------------ kernels
// One view per block: split the row into three BF16 pieces (GEMM operand A)
// and write the near-band part of Z.
__global__ void __launch_bounds__(256) k_split_near(const float *__restrict__ Y, float *__restrict__ Z,
                                                    __nv_bfloat16 *__restrict__ A, const float *__restrict__ taps,
                                                    float near_diag, int nb, int kp, const CgState *cg,
                                                    int respect_stop) {
    extern __shared__ __align__(16) float P[];    // [NEAR + nb + NEAR], zero padded
    if (respect_stop && cg->stop) return;
    const int v = blockIdx.x;
    const float *y = Y + (size_t)v * nb;
    for (int k = threadIdx.x; k < nb + 2 * NEAR; k += blockDim.x) {
        const int i = k - NEAR;
        P[k] = (i >= 0 && i < nb) ? y[i] : 0.f;
    }
    __syncthreads();
    __nv_bfloat16 *a = A + (size_t)v * 3 * kp;
    for (int k = threadIdx.x; k < kp; k += blockDim.x) {
        const float x = k < nb ? P[NEAR + k] : 0.f;
        const __nv_bfloat16 h = __float2bfloat16_rn(x);
        const float r1 = x - __bfloat162float(h);           // exact
        const __nv_bfloat16 m = __float2bfloat16_rn(r1);
        const float r2 = r1 - __bfloat162float(m);          // exact
        const int col = a_col(k, kp / 2);
        a[col] = h;
        a[kp + col] = m;
        a[2 * kp + col] = __float2bfloat16_rn(r2);
    }
    float *z = Z + (size_t)v * nb;
    float t[NEAR / 2];                                  // the odd-lag taps, in registers
#pragma unroll
    for (int q = 0; q < NEAR / 2; ++q) t[q] = __ldg(taps + 2 * q + 1);
    for (int j = threadIdx.x; j < nb; j += blockDim.x) {
        const float c = P[NEAR + j];
        float acc = 0.f;
#pragma unroll
        for (int q = 0; q < NEAR / 2; ++q) {
            const int m = 2 * q + 1;
            acc = fmaf(t[q], __fadd_rn(__fsub_rn(P[NEAR + j - m], c), __fsub_rn(P[NEAR + j + m], c)), acc);
        }
        z[j] = fmaf(near_diag, c, acc);
    }
}

__global__ void __launch_bounds__(128, 1)
k_ramp_gemm(const __grid_constant__ CUtensorMap map_a, const __grid_constant__ CUtensorMap map_b,
            float *__restrict__ Z, int V, int nb, int kp, int np, const CgState *cg, int respect_stop,
            int *err) {
    extern __shared__ __align__(16) uint8_t raw[];
    if (respect_stop && cg->stop) return;
    // 1024-byte aligned stage ring, then the barriers and the TMEM address
    uint8_t *base = (uint8_t *)(((uintptr_t)raw + 1023) & ~(uintptr_t)1023);
    uint64_t *full = reinterpret_cast<uint64_t *>(base + STAGES * STAGE_BYTES);
    uint64_t *empty = full + STAGES;
    uint64_t *done = empty + STAGES;
    uint32_t *tmem_slot = reinterpret_cast<uint32_t *>(done + 1);
    __shared__ int abort_flag, mma_any;
    const int warp = threadIdx.x >> 5;
    // output parity h: bins 2 i + h, i in [n0, n0 + TN); its input bins are
    // the other parity's, Y columns [a0, a0 + kh) of each piece
    const int kh = kp / 2, nh = np / 2, tiles_h = nh / TN;
    const int par = blockIdx.y / tiles_h;
    const int m0 = blockIdx.x * TM, n0 = (blockIdx.y - par * tiles_h) * TN;
    const int a0 = par == 0 ? 0 : kh;
    const int nk = kh / TK;

    if (threadIdx.x == 0) {
        for (int s = 0; s < STAGES; ++s) {
            mbar_init(&full[s], 1);
            mbar_init(&empty[s], 1);
        }
        mbar_init(done, 1);
        abort_flag = 0;
        mma_any = 0;
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
        asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
    }
    if (warp == 0) {   // the whole warp allocates TMEM_COLS columns
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(tmem_slot)),
                     "r"(TMEM_COLS)
                     : "memory");
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
    }
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    const uint32_t tmem = *tmem_slot;

    auto stage_a = [&](int s, int piece) { return base + s * STAGE_BYTES + piece * A_TILE; };
    auto stage_b = [&](int s, int piece) { return base + s * STAGE_BYTES + 3 * A_TILE + piece * B_TILE; };

    if (threadIdx.x == 0) {
        // producer + MMA issuer
        const long long first_polls = g_tc_wait_budget < 0 ? WAIT_POLLS : g_tc_wait_budget;
        bool ok = true;
        int issued = 0;                      // chunks whose loads were issued
        auto load = [&](int kc) {
            const int s = kc % STAGES;
            mbar_expect_tx(&full[s], STAGE_BYTES);
            for (int p = 0; p < 3; ++p) {
                tma_load_2d(stage_a(s, p), &map_a, &full[s], p * kp + a0 + kc * TK, m0);
                tma_load_2d(stage_b(s, p), &map_b, &full[s], kc * TK, (par * 3 + p) * nh + n0);
            }
        };
        for (; issued < nk && issued < STAGES; ++issued) load(issued);
        // the six products (A piece, B piece): h.h, h.m, m.h, m.m, h.l, l.h,
        // and the accumulator each goes to (h.h: 0 or 1 by half of K)
        const int pa[6] = {0, 0, 1, 1, 0, 2}, pb[6] = {0, 1, 0, 1, 2, 0};
        const int acc_of[6] = {0, 2, 2, 3, 3, 3};
        const int first_q[NACC] = {0, 0, 1, 3};   // first product of each accumulator
        const int half = (nk + 1) / 2;
        int mma_done_through = -1;           // chunks whose MMAs are known complete
        for (int kc = 0; kc < nk && ok; ++kc) {
            const int s = kc % STAGES;
            if (!mbar_wait(&full[s], (kc / STAGES) & 1, first_polls)) { ok = false; break; }
            tc_fence_after();
#pragma unroll
            for (int q = 0; q < 6; ++q) {
                const int acc = q == 0 ? (kc < half ? 0 : 1) : acc_of[q];
                const int kfirst = acc == 1 ? half : 0;
                const uint64_t da = sw128_desc(stage_a(s, pa[q])), db = sw128_desc(stage_b(s, pb[q]));
#pragma unroll
                for (int ks = 0; ks < TK / 16; ++ks) {
                    const bool first = kc == kfirst && q == first_q[acc] && ks == 0;
                    umma(tmem + (uint32_t)(acc * TN), da + 2 * ks, db + 2 * ks, first ? 0u : 1u);
                }
            }
            mma_any = 1;
            umma_commit(&empty[s]);
            // refill the stage of chunk kc-1 (its MMAs precede kc's) with chunk kc-1+STAGES
            const int prev = kc - 1;
            if (prev >= 0 && issued < nk) {
                const int sp = prev % STAGES;
                if (!mbar_wait(&empty[sp], (prev / STAGES) & 1)) { ok = false; break; }
                mma_done_through = prev;
                load(issued++);
            }
        }
        // every issued MMA signals `done` when complete (a CTA that gave up
        // before its first MMA has none to wait for)
        if (mma_any) umma_commit(done);
        if (!ok) {
            abort_flag = 1;
            atomicExch(err, (int)AIR_ERR_TIMEOUT);
            // wait (bounded) for the loads still in flight before leaving
            for (int kc = mma_done_through + 1; kc < issued; ++kc) mbar_wait(&full[kc % STAGES], (kc / STAGES) & 1);
        }
    }
    // everyone waits for the producer, then for the accumulator; the outcome
    // is made block-uniform because the TMEM loads below are warp-collective
    __syncthreads();
    const int have = __syncthreads_and(mma_any ? (mbar_wait(done, 0) ? 1 : 0) : 1);
    tc_fence_after();
    if (have && !abort_flag) {
        // lane l of warp w holds row 32 w + l of the tile: it sums the four
        // accumulators into a padded [row][TN + 1] table in the (now idle)
        // stage ring, and the warp then adds its 32 rows to Z with lanes along
        // the bins (coalesced)
        const int lane = threadIdx.x & 31;
        const uint32_t lane_base = tmem + ((uint32_t)(warp * 32) << 16);
        const bool two_halves = nk > (nk + 1) / 2;   // accumulator 1 holds the second half of K
        float *tile = reinterpret_cast<float *>(base) + (size_t)warp * 32 * (TN + 1);
        float a0[16], a1[16], a2[16], a3[16];
#pragma unroll 1
        for (int c0 = 0; c0 < TN; c0 += 16) {
            tmem_ld16(lane_base + 0 * TN + c0, a0);
            tmem_ld16(lane_base + 1 * TN + c0, a1);
            tmem_ld16(lane_base + 2 * TN + c0, a2);
            tmem_ld16(lane_base + 3 * TN + c0, a3);
#pragma unroll
            for (int i = 0; i < 16; ++i)
                tile[lane * (TN + 1) + c0 + i] = ((a3[i] + a2[i]) + (two_halves ? a1[i] : 0.f)) + a0[i];
        }
        __syncwarp();
        // all of the warp's loads of Z first (one memory latency), then the stores
        constexpr int PER = 32 * TN / 32;              // elements per lane
        float zv[PER];
#pragma unroll
        for (int q = 0; q < PER; ++q) {
            const int r = q / (TN / 32), c = lane + 32 * (q % (TN / 32));
            const int row = m0 + warp * 32 + r, j = 2 * (n0 + c) + par;
            zv[q] = (row < V && j < nb) ? Z[(size_t)row * nb + j] : 0.f;
        }
#pragma unroll
        for (int q = 0; q < PER; ++q) {
            const int r = q / (TN / 32), c = lane + 32 * (q % (TN / 32));
            const int row = m0 + warp * 32 + r, j = 2 * (n0 + c) + par;
            if (row < V && j < nb) Z[(size_t)row * nb + j] = zv[q] + tile[r * (TN + 1) + c];
        }
    } else if (threadIdx.x == 0 && !have) {
        atomicExch(err, (int)AIR_ERR_TIMEOUT);
    }
    tc_fence_before();
    __syncthreads();
    if (warp == 0)
        asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(TMEM_COLS)
                     : "memory");
}

// ------------------------------------------------------------ host side
uint16_t bf16_rn(float x) {   // round-to-nearest-even to BF16 (finite inputs)
    uint32_t u;
    std::memcpy(&u, &x, 4);
    const uint32_t lsb = (u >> 16) & 1u;
    u += 0x7FFFu + lsb;
    return (uint16_t)(u >> 16);
}
float bf16_f(uint16_t h) {
    const uint32_t u = (uint32_t)h << 16;
    float x;
    std::memcpy(&x, &u, 4);
    return x;
}

PFN_cuTensorMapEncodeTiled_v12000 encode_fn() {
    static PFN_cuTensorMapEncodeTiled_v12000 fn = nullptr;
    if (!fn) {
        void *p = nullptr;
        cudaDriverEntryPointQueryResult q;
        if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &p, 12000, cudaEnableDefault, &q) ==
                cudaSuccess &&
            q == cudaDriverEntryPointSuccess)
            fn = reinterpret_cast<PFN_cuTensorMapEncodeTiled_v12000>(p);
    }
    return fn;
}

bool make_map(CUtensorMap *m, void *gptr, uint64_t inner, uint64_t outer, uint32_t box_inner, uint32_t box_outer) {
    auto fn = encode_fn();
    if (!fn) return false;
    const cuuint64_t dims[2] = {inner, outer};
    const cuuint64_t strides[1] = {inner * 2};
    const cuuint32_t box[2] = {box_inner, box_outer};
    const cuuint32_t estr[2] = {1, 1};
    return fn(m, CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, 2, gptr, dims, strides, box, estr, CU_TENSOR_MAP_INTERLEAVE_NONE,
              CU_TENSOR_MAP_SWIZZLE_128B, CU_TENSOR_MAP_L2_PROMOTION_L2_128B,
              CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) == CUDA_SUCCESS;
}

}  // namespace

air_status ramp_tc_create(air_plan *P) {
    const int V = P->geom.n_views, nb = P->geom.n_bins;
    TcRes *R = new (std::nothrow) TcRes();
    if (!R) return fail(AIR_ERR_OOM, "host allocation failed");
    R->kp = (nb + KPAD - 1) / KPAD * KPAD;
    R->np = R->kp;
    const int kh = R->kp / 2, nh = R->np / 2;
    const size_t ba = (size_t)V * 3 * R->kp * 2, bb = (size_t)2 * 3 * nh * kh * 2;
    const size_t total = align_up(ba, 256) + align_up(bb, 256) + 256 + 256;
    if (cudaMalloc(&R->mem, total) != cudaSuccess) {
        cudaGetLastError();
        delete R;
        return fail(AIR_ERR_OOM, "cudaMalloc of the tensor-core filter buffers failed");
    }
    R->a = reinterpret_cast<__nv_bfloat16 *>(R->mem);
    R->b = reinterpret_cast<__nv_bfloat16 *>(R->mem + align_up(ba, 256));
    R->near_taps = reinterpret_cast<float *>(R->mem + align_up(ba, 256) + align_up(bb, 256));
    R->err = reinterpret_cast<int *>(R->mem + align_up(ba, 256) + align_up(bb, 256) + 256);
    // far band of c0 T split into three BF16 pieces (from FP64), near taps in FP32
    const double c0 = M_PI / ((double)V * P->geom.pixel_mm * P->geom.pixel_mm);
    auto h = [](int k) { return k == 0 ? 0.25 : (k % 2 ? -1.0 / (M_PI * M_PI * (double)k * (double)k) : 0.0); };
    // B[(h 3 + p) nh + i][l]: piece p of c0 T_far[n][k] for output bin n = 2 i + h
    // and the input bin k of column l among the other parity's bins
    std::vector<uint16_t> hb((size_t)2 * 3 * nh * kh, 0);
    for (int n = 0; n < nb; ++n)
        for (int k = 0; k < nb; ++k) {
            const int lag = n > k ? n - k : k - n;
            if (lag < NEAR || lag % 2 == 0) continue;      // the near band, and the zero even lags
            const double t = c0 * h(lag);
            const uint16_t p0 = bf16_rn((float)t);
            const double r1 = t - (double)bf16_f(p0);
            const uint16_t p1 = bf16_rn((float)r1);
            const double r2 = r1 - (double)bf16_f(p1);
            const uint16_t p2 = bf16_rn((float)r2);
            const int par = n & 1, i = n >> 1, l = a_col(k, kh) - (par == 0 ? 0 : kh);
            const uint16_t pc[3] = {p0, p1, p2};
            for (int p = 0; p < 3; ++p) hb[((size_t)(par * 3 + p) * nh + i) * kh + l] = pc[p];
        }
    float nt[NEAR];
    double diag = 0.0;
    for (int m = NEAR - 1; m >= 0; --m) {
        nt[m] = (float)(c0 * h(m));
        diag += m == 0 ? h(m) : 2.0 * h(m);   // every odd lag the near loop visits
    }
    R->near_diag = (float)(c0 * diag);
    cudaError_t e = cudaMemcpy(R->b, hb.data(), bb, cudaMemcpyHostToDevice);
    if (e == cudaSuccess) e = cudaMemcpy(R->near_taps, nt, sizeof(nt), cudaMemcpyHostToDevice);
    if (e == cudaSuccess) e = cudaMemset(R->err, 0, sizeof(int));
    if (e == cudaSuccess) e = cudaMemset(R->a, 0, ba);
    const bool maps = e == cudaSuccess && make_map(&R->map_a, R->a, 3 * (uint64_t)R->kp, V, TK, TM) &&
                      make_map(&R->map_b, R->b, kh, 2 * 3 * (uint64_t)nh, TK, TN);
    if (e == cudaSuccess) {
        e = cudaFuncSetAttribute(k_ramp_gemm, cudaFuncAttributeMaxDynamicSharedMemorySize, GEMM_SMEM);
        if (e == cudaSuccess)   // the largest any plan needs: the limit is per kernel, not per plan
            e = cudaFuncSetAttribute(k_split_near, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                     (int)((RAMP_MAX_BINS + 2 * NEAR) * sizeof(float)));
    }
    if (e != cudaSuccess || !maps) {
        cudaFree(R->mem);
        delete R;
        cudaGetLastError();
        return fail(AIR_ERR_CUDA, std::string("tensor-core filter set-up failed: ") +
                                      (e != cudaSuccess ? cudaGetErrorString(e) : "cuTensorMapEncodeTiled"));
    }
    P->tc = R;
    P->tc_bytes = total;
    return AIR_OK;
}

void ramp_tc_destroy(air_plan *P) {
    TcRes *R = static_cast<TcRes *>(P->tc);
    if (!R) return;
    cudaFree(R->mem);
    delete R;
    P->tc = nullptr;
    P->tc_bytes = 0;
}

air_status ramp_tc_apply(const air_plan *P, const float *src, float *dst, const CgState *cg, int respect_stop,
                         cudaStream_t st) {
    const TcRes *R = static_cast<const TcRes *>(P->tc);
    if (!R) return fail(AIR_ERR_INVALID_ARG, "plan has no tensor-core filter");
    const int V = P->geom.n_views, nb = P->geom.n_bins;
    k_split_near<<<V, 256, (nb + 2 * NEAR) * sizeof(float), st>>>(src, dst, R->a, R->near_taps, R->near_diag, nb,
                                                                   R->kp, cg, respect_stop);
    cudaError_t e = cudaGetLastError();
    if (e == cudaSuccess) {
        dim3 grid((V + TM - 1) / TM, R->np / TN);   // both parities: 2 x (np / 2) / TN
        k_ramp_gemm<<<grid, 128, GEMM_SMEM, st>>>(R->map_a, R->map_b, dst, V, nb, R->kp, R->np, cg, respect_stop,
                                                  R->err);
        e = cudaGetLastError();
    }
    if (e != cudaSuccess) return fail(AIR_ERR_CUDA, std::string("tensor-core filter launch: ") + cudaGetErrorString(e));
    return AIR_OK;
}

int ramp_tc_status(const air_plan *P) {
    const TcRes *R = static_cast<const TcRes *>(P->tc);
    if (!R) return 0;
    int v = 0;
    if (cudaMemcpy(&v, R->err, sizeof(int), cudaMemcpyDeviceToHost) != cudaSuccess) return (int)AIR_ERR_CUDA;
    if (v != 0 && cudaMemset(R->err, 0, sizeof(int)) != cudaSuccess) return (int)AIR_ERR_CUDA;
    return v;
}

cudaError_t ramp_tc_set_wait_budget(long long polls) {
    return cudaMemcpyToSymbol(g_tc_wait_budget, &polls, sizeof(polls));
}

}  // namespace air
