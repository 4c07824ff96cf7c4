// Host side of the AIR library: plans (geometry tables + workspace), argument
// checking, the stand-alone operator calls and the solver programs.
#include <cmath>
#include <algorithm>
#include <cstring>
#include <map>
#include <memory>
#include <mutex>
#include <string>
#include <vector>

#include "host_common.h"
#include "launch.h"
#include "ramp_tc.h"

using namespace air;

namespace air {

thread_local std::string g_err;

air_status fail(air_status s, const std::string &msg) {
    g_err = msg;
    return s;
}

double fan_pitch(const air_geometry &g) {
    if (g.dgamma > 0.0) return g.dgamma;
    return 2.0 * std::asin(g.n * g.pixel_mm / std::sqrt(2.0) / g.dso_mm) / g.n_bins;
}

air_status validate_geometry(const air_geometry *g) {
    if (!g) return fail(AIR_ERR_INVALID_ARG, "geometry is NULL");
    if (g->n < 1 || g->n > 4096) return fail(AIR_ERR_INVALID_ARG, "n must be in 1..4096");
    if (!(g->pixel_mm > 0.0) || !std::isfinite(g->pixel_mm))
        return fail(AIR_ERR_INVALID_ARG, "pixel_mm must be > 0");
    if (g->n_views < 1 || g->n_views > 65536) return fail(AIR_ERR_INVALID_ARG, "n_views must be in 1..65536");
    if (g->n_bins < 1 || g->n_bins > RAMP_MAX_BINS) return fail(AIR_ERR_INVALID_ARG, "n_bins must be in 1..8192");
    if ((long long)g->n_views * g->n_bins > (1ll << 26))
        return fail(AIR_ERR_INVALID_ARG, "n_views * n_bins must be <= 2^26");
    const double rc = g->n * g->pixel_mm / std::sqrt(2.0);
    if (!(g->dso_mm >= rc + 8.0 * g->pixel_mm) || !std::isfinite(g->dso_mm))
        return fail(AIR_ERR_INVALID_ARG,
                    "dso_mm must exceed the image's circumscribed radius n*dx/sqrt(2) by 8 pixels");
    if (!(g->dgamma >= 0.0) || !std::isfinite(g->dgamma)) return fail(AIR_ERR_INVALID_ARG, "dgamma must be >= 0");
    if (!std::isfinite(g->beta0) || !std::isfinite(g->arc) || g->arc == 0.0)
        return fail(AIR_ERR_INVALID_ARG, "beta0 must be finite and arc finite and nonzero");
    if (g->filter != AIR_FILTER_NONE && g->filter != AIR_FILTER_RAMLAK)
        return fail(AIR_ERR_INVALID_ARG, "filter must be AIR_FILTER_NONE or AIR_FILTER_RAMLAK");
    if (g->precision != AIR_PREC_FP32 && g->precision != AIR_PREC_BF16X3)
        return fail(AIR_ERR_INVALID_ARG, "precision must be AIR_PREC_FP32 or AIR_PREC_BF16X3");
    return AIR_OK;
}

// Device pointer check: non-NULL, 16-byte aligned, and device accessible
// (a host pointer handed to a kernel would fault the GPU).
air_status check_dev_ptr(const void *p, const char *what) {
    if (!p) return fail(AIR_ERR_INVALID_ARG, std::string(what) + " is NULL");
    if (reinterpret_cast<uintptr_t>(p) & 15u)
        return fail(AIR_ERR_INVALID_ARG, std::string(what) + " is not 16-byte aligned");
    cudaPointerAttributes a;
    cudaError_t e = cudaPointerGetAttributes(&a, p);
    if (e != cudaSuccess) {
        cudaGetLastError();
        return fail(AIR_ERR_INVALID_ARG, std::string(what) + " is not a CUDA pointer");
    }
    if (a.type != cudaMemoryTypeDevice && a.type != cudaMemoryTypeManaged)
        return fail(AIR_ERR_INVALID_ARG, std::string(what) + " is not device memory");
    return AIR_OK;
}

bool overlap(const void *a, size_t na, const void *b, size_t nb) {
    const char *pa = (const char *)a, *pb = (const char *)b;
    return pa < pb + nb && pb < pa + na;
}

size_t align_up(size_t v, size_t a) { return (v + a - 1) / a * a; }

}  // namespace air

// -------------------------------------------------------------------- plan
namespace air {
// Backprojector view parts of a slice: enough (pixel tile, part) blocks for
// about 12 per SM (2.4 waves at 5 resident blocks), at most one part per
// view.  The autotuner starts from this and tries up to twice as many.
int choose_bwd_parts(const SliceDesc &s) {
    int sms = 148, dev = 0;
    if (cudaGetDevice(&dev) == cudaSuccess) cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    cudaGetLastError();
    const int txy = tiles_bwd_xy(s), target = 2 * 6 * sms;
    const int S = (target + txy - 1) / txy;
    return S < 1 ? 1 : (S > s.V ? s.V : S);
}

// Device bytes a plan of this geometry will hold (the pieces of plan_build
// and, for BF16X3, the tensor-core filter buffers), to within alignment.
size_t plan_bytes_estimate(const air_geometry &g) {
    SliceDesc s{};
    s.n = g.n;
    s.V = g.n_views;
    s.nb = g.n_bins;
    const size_t nn = (size_t)g.n * g.n, rays = (size_t)g.n_views * g.n_bins;
    // the part buffer holds the autotuner's largest split, as plan_build sizes it
    const size_t parts = (size_t)std::min(g.n_views, 2 * choose_bwd_parts(s));
    size_t b = rays * (sizeof(RayFx) + 4) + (size_t)g.n_views * tiles_bwd_xy(s) * 4 + (size_t)g.n_bins * 4;
    b += nn * 4 * (7 + parts + 18 + 1);          // x r p q rhs0 g g', parts, b b2, xbuf
    b += (size_t)g.n * (g.n + 1) * 8 * 2;        // xp xt (pairs)
    b += (size_t)g.n_views * 8 + (size_t)g.n_bins * 8;   // FBP tables
    b += rays * 4 * 3;                           // z zc ybuf
    b += sizeof(CgState) + ((size_t)max_reduce_tiles(s) + 64) * 8 + 24 * 256;
    if (g.precision == AIR_PREC_BF16X3) {
        const size_t kp = ((size_t)g.n_bins + 127) / 128 * 128;   // split Y; both parities' T_far pieces
        b += (size_t)g.n_views * 3 * kp * 2 + 3 * kp * kp + 1024;
    }
    return b;
}
}  // namespace air

namespace {
long long floor_div(long long a, long long b) {   // b > 0
    long long q = a / b;
    return (a % b != 0 && a < 0) ? q - 1 : q;
}
long long ceil_div(long long a, long long b) {    // b > 0
    return -floor_div(-a, b);
}
}  // namespace

// The fixed-point form of the line through (px, py) with unit direction
// (ux, uy), pixel units with the origin at the image corner (see RayFx), and
// its walk word.
RayFx air::make_ray_fx(double px, double py, double ux, double uy, int n, unsigned *walk) {
    const double two32 = 4294967296.0;
    const bool cols = std::fabs(ux) >= std::fabs(uy);       // walk columns
    const double a = cols ? px : py, b = cols ? py : px;    // along / across the walk
    const double ua = cols ? ux : uy, ub = cols ? uy : ux;
    const double m = ub / ua;                               // |m| <= 1
    const double y0 = b - a * m;                            // across-coordinate at walk-coordinate 0
    long long M = std::llround(m * two32);
    const long long mmax = (1ll << 32) - 1;
    if (M > mmax) M = mmax;
    if (M < -mmax) M = -mmax;
    if (M == 0) M = 1;        // an exactly axis-parallel ray, tilted by 2^-32
    const long long Y0 = std::llround(y0 * two32);
    RayFx r{};
    r.Mlo = (unsigned)(M & 0xffffffffll);
    r.L0 = Y0 + (M < 0 ? M : 0);
    const unsigned Ma = (unsigned)(M < 0 ? -M : M);
    const float c = (float)((1.0 / std::fabs(ua)) / (double)Ma);
    r.cs = M < 0 ? -c : c;
    // walk range: columns k in [0, n) whose span [lo, lo + Ma] meets rows [0, n)
    const long long N2 = (long long)n << 32;
    long long ks, ke;
    if (M > 0) {
        ks = floor_div(-r.L0 - (long long)Ma, M) + 1;       // hi(k) > 0
        ke = ceil_div(N2 - r.L0, M);                        // lo(k) < N2
    } else {
        const long long Mp = -M;
        ks = floor_div(r.L0 - N2, Mp) + 1;                  // lo(k) < N2
        ke = ceil_div(r.L0 + (long long)Ma, Mp);            // hi(k) > 0
    }
    // clamp to [0, n] before packing: a ray that misses the image can give a
    // start column far outside it (the walk word holds 16 and 15 bits)
    ks = std::min<long long>(std::max<long long>(ks, 0), n);
    ke = std::min<long long>(std::max<long long>(ke, ks), n);
    auto meets = [&](long long k) {
        const long long lo = r.L0 + k * M;
        return lo + (long long)Ma > 0 && lo < N2;
    };
    while (ks < ke && !meets(ks)) ++ks;
    while (ke > ks && !meets(ke - 1)) --ke;
    *walk = ray_walk((int)ks, (int)ke, cols);
    return r;
}

// ------------------------------------------------------------ autotuner
// The projector's tile shape (views per block) and the backprojector's view
// split are timed on the plan's own workspace (the kernels' work does not
// depend on the data) and the fastest kept; results are cached per geometry
// for the life of the process, so every plan of a geometry uses the same
// configuration.
namespace {
struct TuneKey {
    int n, V, nb;
    double dx, dso, dg, beta0, arc;
    bool operator<(const TuneKey &o) const {
        return std::memcmp(this, &o, sizeof(TuneKey)) < 0;
    }
};
std::mutex g_tune_mu;
std::map<TuneKey, std::pair<int, int>> g_tune_cache;
}  // namespace

namespace air {
air_status autotune(air_plan *P) {
    SliceDesc &s = P->desc;
    TuneKey key;
    std::memset(&key, 0, sizeof(key));
    key.n = s.n;
    key.V = s.V;
    key.nb = s.nb;
    key.dx = P->geom.pixel_mm;
    key.dso = P->geom.dso_mm;
    key.dg = fan_pitch(P->geom);
    key.beta0 = P->geom.beta0;
    key.arc = P->geom.arc;
    {
        std::lock_guard<std::mutex> lock(g_tune_mu);
        auto it = g_tune_cache.find(key);
        if (it != g_tune_cache.end()) {
            s.fwd_vpb = it->second.first;
            s.bwd_parts = std::min(it->second.second, P->bwd_parts_max);
            return AIR_OK;
        }
    }
    cudaStream_t st = nullptr;
    cudaEvent_t e0 = nullptr, e1 = nullptr;
    cudaError_t e = cudaStreamCreateWithFlags(&st, cudaStreamNonBlocking);
    if (e == cudaSuccess) e = cudaEventCreate(&e0);
    if (e == cudaSuccess) e = cudaEventCreate(&e1);
    if (e == cudaSuccess) e = cudaMemsetAsync(s.x, 0, (size_t)s.n * s.n * 4, st);
    if (e == cudaSuccess) e = cudaMemsetAsync(s.z, 0, (size_t)s.V * s.nb * 4, st);
    auto timed = [&](auto &&launch) -> float {
        if (e != cudaSuccess) return 1e30f;
        launch();                                   // warm-up
        cudaEventRecord(e0, st);
        for (int r = 0; r < 3; ++r) launch();
        cudaEventRecord(e1, st);
        e = cudaEventSynchronize(e1);
        float ms = 1e30f;
        if (e == cudaSuccess) cudaEventElapsedTime(&ms, e0, e1);
        return ms;
    };
    // projector: views per block, from the most down; a smaller tile is
    // kept only if it is 2 % faster (within that, grouped batches run the
    // taller tiles a little faster)
    SliceDesc t = s;
    t.ext_in = s.x;
    t.ext_out = s.z;
    int best_vpb = 1;
    float best = 1e30f;
    for (int vpb : {8, 4, 2, 1}) {
        if (vpb > s.V) continue;
        t.fwd_vpb = vpb;
        const float ms = timed([&] {
            if (e == cudaSuccess) e = launch_op(OP_TRANSPOSE, t, SRC_EXT, st);
            if (e == cudaSuccess) e = launch_op(OP_FWD, t, SRC_EXT, st);
        });
        if (ms < best * 0.98f) {
            best = ms;
            best_vpb = vpb;
        }
    }
    // backprojector: view splits up to the part buffer's size, timed as the
    // solver runs them (the parts, then their sum, OP_BWD_FIN, which the CG
    // epilogue needs at any split); the heuristic's choice is tried first
    // and kept unless another is 2 % faster
    t = s;
    if (e == cudaSuccess) e = cudaMemsetAsync(s.zc, 0, (size_t)s.V * s.nb * 4, st);
    const int S0 = s.bwd_parts;
    int best_S = S0;
    best = 1e30f;
    for (int S : {S0, 1, 2, 3, 4, 6, 8, 12, 16}) {
        if (S > P->bwd_parts_max || (S == S0 && best < 1e30f)) continue;
        t.bwd_parts = S;
        const float ms = timed([&] {
            if (e == cudaSuccess) e = launch_op(OP_BWD, t, BWD_RHS0, st);
            if (e == cudaSuccess) e = launch_op(OP_BWD_FIN, t, BWD_RHS0, st);
        });
        if (ms < best * 0.98f) {
            best = ms;
            best_S = S;
        }
    }
    if (e0) cudaEventDestroy(e0);
    if (e1) cudaEventDestroy(e1);
    if (st) cudaStreamDestroy(st);
    if (e != cudaSuccess) return fail(AIR_ERR_CUDA, std::string("autotuning: ") + cudaGetErrorString(e));
    s.fwd_vpb = best_vpb;
    s.bwd_parts = best_S;
    std::lock_guard<std::mutex> lock(g_tune_mu);
    g_tune_cache[key] = {best_vpb, best_S};
    return AIR_OK;
}
}  // namespace air

// ------------------------------------------------------------ geometry tables
// The host-side tables of a geometry (FP64 arithmetic, stored as the device
// formats), cached per geometry for the process: plans of one geometry (a
// batch, the server's pool) share one computation.
namespace {
struct HostTables {
    std::vector<RayFx> ray;
    std::vector<unsigned> walk;
    std::vector<unsigned> vt;
    std::vector<float> taps, fbw, fbt;
    std::vector<float2> fview;
    float ramp_diag = 0.f, fbp_diag = 0.f;
};

air_status build_tables(const air_geometry &g, double dg, int ntxy, HostTables &T) {
    const int n = g.n, V = g.n_views, nb = g.n_bins;
    const size_t rays = (size_t)V * nb;
    // geometry tables, computed in FP64: per view the source (pixel units,
    // centred) and the central-ray direction; per ray the fixed-point line
    std::vector<RayFx> &hray = T.ray;
    std::vector<unsigned> &hwalk = T.walk;
    hray.resize(rays);
    hwalk.resize(rays);
    struct ViewSrc { double x, y, z, w; };   // source (pixel units, centred), central direction
    std::vector<ViewSrc> hsrc(V);
    std::vector<float> &htaps = T.taps;
    htaps.resize(nb);
    const double inv_dx = 1.0 / g.pixel_mm;
    for (int v = 0; v < V; ++v) {
        const double beta = g.beta0 + g.arc * (double)v / (double)V;
        const double cb = std::cos(beta), sb = std::sin(beta);
        const double Sx = g.dso_mm * cb, Sy = g.dso_mm * sb;
        hsrc[v] = ViewSrc{Sx * inv_dx, Sy * inv_dx, -cb, -sb};
        for (int j = 0; j < nb; ++j) {
            const double gamma = ((double)j - 0.5 * (nb - 1)) * dg;
            const double th = beta + M_PI + gamma;
            const double ux = std::cos(th), uy = std::sin(th);
            const double su = Sx * ux + Sy * uy;
            // closest point to the image centre, pixel units, origin at the image corner
            const double px = (Sx - su * ux) * inv_dx + 0.5 * n, py = (Sy - su * uy) * inv_dx + 0.5 * n;
            hray[(size_t)v * nb + j] = make_ray_fx(px, py, ux, uy, n, &hwalk[(size_t)v * nb + j]);
        }
    }
    // the projector walks [k0, k1) without bounds checks (the image copies
    // it reads are padded by one entry per row end): every walked column must
    // lie in the image and its span start in rows [-1, n-1]
    for (size_t i = 0; i < rays; ++i) {
        const RayFx &r = hray[i];
        const int k0 = walk_k0(hwalk[i]), k1 = walk_k1(hwalk[i]);
        bool ok = 0 <= k0 && k0 <= k1 && k1 <= n;
        for (int k : {k0, k1 - 1}) {
            if (!ok || k0 == k1) break;
            const long long r0 = (r.L0 + (long long)k * ray_M(r)) >> 32;
            ok = r0 >= -1 && r0 <= n - 1;
        }
        if (!ok) return fail(AIR_ERR_INTERNAL, "ray table: a walk range leaves the image");
    }
    // backprojector ray ranges: per view and 32 x 32 pixel tile, the rays
    // whose fan angle lies between the extreme fan angles of the tile's
    // corners (the tile is convex and the source outside it, so exactly
    // these rays can meet it), widened by 0.02 bin; and whether they all walk
    // the same way with slopes of one sign.  Fan angles at the corner grid
    // are shared by neighbouring tiles.
    const int tpr = (n + BWD_T - 1) / BWD_T;
    std::vector<unsigned> &hvt = T.vt;
    hvt.assign((size_t)V * ntxy, 0u);
    {
        std::vector<double> gam((size_t)(tpr + 1) * (tpr + 1));
        std::vector<int> chg(nb);   // number of changes of orientation or slope sign among rays 0..j
        const double jm = 0.5 * (nb - 1);
        for (int v = 0; v < V; ++v) {
            const ViewSrc w = hsrc[v];
            for (int iy = 0; iy <= tpr; ++iy)
                for (int ix = 0; ix <= tpr; ++ix) {
                    const double px = std::min(ix * BWD_T, n) - 0.5 * n, py = std::min(iy * BWD_T, n) - 0.5 * n;
                    const double dxs = px - w.x, dys = py - w.y;
                    gam[(size_t)iy * (tpr + 1) + ix] = std::atan2(w.z * dys - w.w * dxs, w.z * dxs + w.w * dys);
                }
            const RayFx *rv = hray.data() + (size_t)v * nb;
            const unsigned *wv = hwalk.data() + (size_t)v * nb;
            chg[0] = 0;
            for (int j = 1; j < nb; ++j)
                chg[j] = chg[j - 1] +
                         (walk_cols(wv[j]) != walk_cols(wv[j - 1]) || (rv[j].cs < 0.f) != (rv[j - 1].cs < 0.f));
            for (int ty = 0; ty < tpr; ++ty)
                for (int tx = 0; tx < tpr; ++tx) {
                    double gmin = 1e30, gmax = -1e30;
                    for (int cy = 0; cy < 2; ++cy)
                        for (int cx = 0; cx < 2; ++cx) {
                            const double gc = gam[(size_t)(ty + cy) * (tpr + 1) + tx + cx];
                            gmin = std::min(gmin, gc);
                            gmax = std::max(gmax, gc);
                        }
                    const double f0 = std::ceil(gmin / dg + jm - 0.02), f1 = std::floor(gmax / dg + jm + 0.02);
                    const int j0 = (int)std::max(0.0, std::min(f0, (double)nb));
                    const int j1 = (int)std::max(-1.0, std::min(f1, (double)nb - 1));   // inclusive
                    unsigned ent = vt_pack(0, 0, 0, false, false);
                    if (j1 >= j0)
                        ent = vt_pack(j0, j1 + 1, walk_cols(wv[j0]), rv[j0].cs < 0.f, chg[j1] != chg[j0]);
                    hvt[(size_t)(ty * tpr + tx) * V + v] = ent;
                }
        }
    }
    const double c0 = M_PI / ((double)V * g.pixel_mm * g.pixel_mm);
    double diag = 0.0;   // h[0] + 2 sum_{odd m < nb} h[m]: the difference form's centre weight
    for (int k = nb - 1; k >= 0; --k) {
        const double h = k == 0 ? 0.25 : (k % 2 ? -1.0 / (M_PI * M_PI * (double)k * (double)k) : 0.0);
        htaps[k] = (float)(c0 * h);
        diag += k == 0 ? h : 2.0 * h;
    }
    T.ramp_diag = (float)(c0 * diag);
    // fan-beam FBP (full scans): per view the central direction; per bin the
    // pre-weight cos gamma_j and the fan ramp alpha D g(m alpha), g(0) =
    // 1/(8 alpha^2), g(odd m) = -1/(2 pi^2 sin^2(m alpha)), g(even m) = 0
    std::vector<float2> &hfview = T.fview;
    std::vector<float> &hfbw = T.fbw, &hfbt = T.fbt;
    hfview.resize(V);
    hfbw.resize(nb);
    hfbt.resize(nb);
    for (int v = 0; v < V; ++v) {
        const double beta = g.beta0 + g.arc * (double)v / (double)V;
        hfview[v] = make_float2((float)(-std::cos(beta)), (float)(-std::sin(beta)));
    }
    double fdiag = 0.0;
    for (int k = nb - 1; k >= 0; --k) {
        const double gm = k == 0 ? 1.0 / (8.0 * dg * dg)
                                 : (k % 2 ? -1.0 / (2.0 * M_PI * M_PI * std::sin(k * dg) * std::sin(k * dg)) : 0.0);
        const double t = dg * g.dso_mm * gm;
        hfbt[k] = (float)t;
        fdiag += k == 0 ? t : 2.0 * t;
        hfbw[k] = (float)std::cos(((double)k - 0.5 * (nb - 1)) * dg);
    }
    T.fbp_diag = (float)fdiag;
    return AIR_OK;
}

struct GeomKey {
    int n, V, nb;
    double dx, dso, dg, beta0, arc;
    bool operator<(const GeomKey &o) const { return std::memcmp(this, &o, sizeof(GeomKey)) < 0; }
};
std::mutex g_tables_mu;
std::map<GeomKey, std::shared_ptr<const HostTables>> g_tables;
constexpr size_t TABLE_CACHE_MAX = 16;

air_status geometry_tables(const air_geometry &g, double dg, int ntxy, std::shared_ptr<const HostTables> *out) {
    GeomKey key;
    std::memset(&key, 0, sizeof(key));
    key.n = g.n;
    key.V = g.n_views;
    key.nb = g.n_bins;
    key.dx = g.pixel_mm;
    key.dso = g.dso_mm;
    key.dg = dg;
    key.beta0 = g.beta0;
    key.arc = g.arc;
    {
        std::lock_guard<std::mutex> lock(g_tables_mu);
        auto it = g_tables.find(key);
        if (it != g_tables.end()) {
            *out = it->second;
            return AIR_OK;
        }
    }
    auto T = std::make_shared<HostTables>();
    air_status st = build_tables(g, dg, ntxy, *T);
    if (st != AIR_OK) return st;
    std::lock_guard<std::mutex> lock(g_tables_mu);
    if (g_tables.size() >= TABLE_CACHE_MAX) g_tables.erase(g_tables.begin());
    g_tables[key] = T;
    *out = T;
    return AIR_OK;
}
}  // namespace

air_status plan_build(const air_geometry *geom, air_plan *P) {
    const air_geometry &g = *geom;
    const int n = g.n, V = g.n_views, nb = g.n_bins;
    const size_t nn = (size_t)n * n, rays = (size_t)V * nb;
    SliceDesc s{};
    s.n = n;
    s.V = V;
    s.nb = nb;
    s.half_n = 0.5f * n;
    s.dx = (float)g.pixel_mm;
    const double dg = fan_pitch(g);
    s.filter = g.filter;

    s.fwd_vpb = 1;
    s.bwd_parts = choose_bwd_parts(s);
    // the autotuner may pick up to twice the heuristic's view split
    const int parts_max = std::min(V, 2 * s.bwd_parts);
    // carve one allocation
    struct Piece { void **dst; size_t bytes; };
    float *x, *r, *p, *q, *rhs0, *gg, *gg2, *b, *b2, *z, *zc, *ybuf, *xbuf, *xp, *xt, *bpart;
    const size_t npad = (size_t)n * (n + 1) * 2;   // pair copies of the projector's input (floats)
    RayFx *ray;
    unsigned *walk;
    unsigned *vt;
    float2 *fview;
    float *fbw, *fbt;
    const int ntxy = tiles_bwd_xy(s);
    float *taps;
    CgState *cg;
    double *partial;
    const size_t npart = (size_t)max_reduce_tiles(s) + 64;
    std::vector<Piece> pieces = {
        {(void **)&ray, rays * sizeof(RayFx)}, {(void **)&walk, rays * sizeof(unsigned)},
        {(void **)&vt, (size_t)V * ntxy * sizeof(unsigned)},
        {(void **)&xp, npad * 4}, {(void **)&xt, npad * 4}, {(void **)&bpart, (size_t)parts_max * nn * 4},
        {(void **)&taps, (size_t)nb * sizeof(float)}, {(void **)&fview, (size_t)V * sizeof(float2)},
        {(void **)&fbw, (size_t)nb * sizeof(float)}, {(void **)&fbt, (size_t)nb * sizeof(float)},
        {(void **)&x, nn * 4}, {(void **)&r, nn * 4}, {(void **)&p, nn * 4}, {(void **)&q, nn * 4},
        {(void **)&rhs0, nn * 4}, {(void **)&gg, nn * 4}, {(void **)&gg2, nn * 4}, {(void **)&b, 9 * nn * 4}, {(void **)&b2, 9 * nn * 4},
        {(void **)&z, rays * 4}, {(void **)&zc, rays * 4}, {(void **)&ybuf, rays * 4}, {(void **)&xbuf, nn * 4},
        {(void **)&cg, sizeof(CgState)}, {(void **)&partial, npart * sizeof(double)}};
    size_t total = 0;
    for (auto &pc : pieces) total = align_up(total, 256) + pc.bytes;
    total = align_up(total, 256);
    char *mem = nullptr;
    if (cudaMalloc(&mem, total) != cudaSuccess) {
        cudaGetLastError();
        return fail(AIR_ERR_OOM, "cudaMalloc of the plan workspace failed (" + std::to_string(total) + " bytes)");
    }
    size_t off = 0;
    for (auto &pc : pieces) {
        off = align_up(off, 256);
        *pc.dst = mem + off;
        off += pc.bytes;
    }

    std::shared_ptr<const HostTables> T;
    if (air_status st = geometry_tables(g, dg, ntxy, &T); st != AIR_OK) {
        cudaFree(mem);
        return st;
    }
    const std::vector<RayFx> &hray = T->ray;
    const std::vector<unsigned> &hwalk = T->walk;
    const std::vector<unsigned> &hvt = T->vt;
    const std::vector<float> &htaps = T->taps, &hfbw = T->fbw, &hfbt = T->fbt;
    const std::vector<float2> &hfview = T->fview;
    s.ramp_diag = T->ramp_diag;
    s.fbp_diag = T->fbp_diag;
    s.dso_px = (float)(g.dso_mm / g.pixel_mm);
    s.inv_dg = (float)(1.0 / dg);
    s.inv_dg_lo = (float)(1.0 / dg - (double)s.inv_dg);
    s.jmid = 0.5f * (nb - 1);
    s.fbp_scale = (float)(g.arc / (double)V / (g.pixel_mm * g.pixel_mm));
    cudaError_t e = cudaMemcpy(ray, hray.data(), rays * sizeof(RayFx), cudaMemcpyHostToDevice);
    if (e == cudaSuccess) e = cudaMemcpy(walk, hwalk.data(), rays * sizeof(unsigned), cudaMemcpyHostToDevice);
    if (e == cudaSuccess) e = cudaMemcpy(vt, hvt.data(), hvt.size() * sizeof(unsigned), cudaMemcpyHostToDevice);
    if (e == cudaSuccess) e = cudaMemcpy(taps, htaps.data(), nb * sizeof(float), cudaMemcpyHostToDevice);
    if (e == cudaSuccess) e = cudaMemcpy(fview, hfview.data(), V * sizeof(float2), cudaMemcpyHostToDevice);
    if (e == cudaSuccess) e = cudaMemcpy(fbw, hfbw.data(), nb * sizeof(float), cudaMemcpyHostToDevice);
    if (e == cudaSuccess) e = cudaMemcpy(fbt, hfbt.data(), nb * sizeof(float), cudaMemcpyHostToDevice);
    if (e == cudaSuccess) e = cudaMemset(cg, 0, sizeof(CgState));
    if (e == cudaSuccess) e = cudaMemset(xp, 0, npad * 4);   // the pads stay zero
    if (e == cudaSuccess) e = cudaMemset(xt, 0, npad * 4);
    if (e != cudaSuccess) {
        cudaFree(mem);
        return fail(AIR_ERR_CUDA, std::string("plan table upload: ") + cudaGetErrorString(e));
    }
    s.ray = ray;
    s.walk = walk;
    s.vt = vt;
    s.fview = fview;
    s.fbp_w = fbw;
    s.fbp_taps = fbt;
    s.taps = taps;
    s.x = x; s.r = r; s.p = p; s.q = q; s.rhs0 = rhs0; s.g = gg; s.g2 = gg2; s.b = b; s.b2 = b2; s.xp = xp; s.xt = xt;
    s.bwd_part = bpart;
    s.z = z; s.zc = zc; s.y = ybuf;
    s.cg = cg;
    s.partial = partial;
    s.mu = 1.f;
    s.tau = 0.f;
    P->geom = g;
    P->desc = s;
    P->mem = mem;
    P->bytes = total;
    P->bwd_parts_max = parts_max;
    P->ybuf = ybuf;
    P->xbuf = xbuf;
    cudaGetDevice(&P->device);
    if (g.precision == AIR_PREC_BF16X3) {
        air_status st = ramp_tc_create(P);
        if (st != AIR_OK) {
            cudaFree(mem);
            return st;
        }
    }
    air_status st = autotune(P);
    if (st == AIR_OK) st = noalloc_prepare();
    if (st != AIR_OK) {
        ramp_tc_destroy(P);
        cudaFree(mem);
        return st;
    }
    return AIR_OK;
}

extern "C" const char *air_last_error(void) { return g_err.c_str(); }

extern "C" air_status air_plan_create(const air_geometry *geom, air_plan **out) {
    if (!out) return fail(AIR_ERR_INVALID_ARG, "out is NULL");
    *out = nullptr;
    air_status st = validate_geometry(geom);
    if (st != AIR_OK) return st;
    air_plan *P = new (std::nothrow) air_plan();
    if (!P) return fail(AIR_ERR_OOM, "host allocation failed");
    st = plan_build(geom, P);
    if (st != AIR_OK) {
        delete P;
        return st;
    }
    *out = P;
    return AIR_OK;
}

extern "C" air_status air_plan_destroy(air_plan *P) {
    if (!P) return AIR_OK;
    ramp_tc_destroy(P);
    if (P->mem) cudaFree(P->mem);
    delete P;
    return AIR_OK;
}

extern "C" size_t air_plan_bytes(const air_plan *P) { return P ? P->bytes + P->tc_bytes : 0; }

extern "C" air_status air_plan_tune(air_plan *P, int fwd_views_per_block, int bwd_view_parts) {
    if (!P) return fail(AIR_ERR_INVALID_ARG, "plan is NULL");
    const int v = fwd_views_per_block;
    if (v != 1 && v != 2 && v != 4 && v != 8) return fail(AIR_ERR_INVALID_ARG, "fwd_views_per_block must be 1, 2, 4 or 8");
    if (bwd_view_parts < 1 || bwd_view_parts > P->bwd_parts_max)
        return fail(AIR_ERR_INVALID_ARG, "bwd_view_parts must be in 1.." + std::to_string(P->bwd_parts_max));
    P->desc.fwd_vpb = v;
    P->desc.bwd_parts = bwd_view_parts;
    return AIR_OK;
}

extern "C" air_status air_plan_config(const air_plan *P, int *fwd_views_per_block, int *bwd_view_parts,
                                      int *bwd_view_parts_max) {
    if (!P) return fail(AIR_ERR_INVALID_ARG, "plan is NULL");
    if (fwd_views_per_block) *fwd_views_per_block = P->desc.fwd_vpb;
    if (bwd_view_parts) *bwd_view_parts = P->desc.bwd_parts;
    if (bwd_view_parts_max) *bwd_view_parts_max = P->bwd_parts_max;
    return AIR_OK;
}

extern "C" air_status air_set_wait_budget(int64_t polls) {
    const long long v = polls < 0 ? -1ll : (long long)polls;
    cudaError_t e = set_barrier_budget(v);
    if (e == cudaSuccess) e = ramp_tc_set_wait_budget(v);
    if (e != cudaSuccess) {
        cudaGetLastError();
        return fail(AIR_ERR_CUDA, std::string("setting the wait budget: ") + cudaGetErrorString(e));
    }
    return AIR_OK;
}

extern "C" air_status air_plan_status(const air_plan *P) {
    if (!P) return fail(AIR_ERR_INVALID_ARG, "plan is NULL");
    const int st = ramp_tc_status(P);
    if (st == (int)AIR_ERR_TIMEOUT) return fail(AIR_ERR_TIMEOUT, "a bounded wait in the tensor-core filter gave up");
    if (st != 0) return fail(AIR_ERR_CUDA, "reading the plan status failed");
    return AIR_OK;
}

// ------------------------------------------------------- stand-alone ops
#define TRY(expr)                                   \
    do {                                            \
        air_status st_ = (expr);                    \
        if (st_ != AIR_OK) return st_;              \
    } while (0)
#define CUDA_TRY(expr)                                                                           \
    do {                                                                                         \
        cudaError_t e_ = (expr);                                                                 \
        if (e_ != cudaSuccess) return fail(AIR_ERR_CUDA, std::string(#expr) + ": " + cudaGetErrorString(e_)); \
    } while (0)

static size_t img_bytes(const air_plan *P) { return (size_t)P->geom.n * P->geom.n * 4; }
static size_t sino_bytes(const air_plan *P) { return (size_t)P->geom.n_views * P->geom.n_bins * 4; }

namespace air {
// Z = C Y into dst (plan precision), from src (device).
air_status apply_filter(const air_plan *P, const SliceDesc &base, const float *src, float *dst,
                        cudaStream_t st) {
    if (P->geom.precision == AIR_PREC_BF16X3 && P->geom.filter == AIR_FILTER_RAMLAK)
        return ramp_tc_apply(P, src, dst, base.cg, 0, st);
    SliceDesc s = base;
    s.ext_in = src;
    s.ext_out = dst;
    CUDA_TRY(launch_op(OP_RAMP, s, RSRC_EXT, st));
    return AIR_OK;
}
}  // namespace air

extern "C" air_status air_project(const air_plan *P, const float *X, float *Y, air_stream stream) {
    if (!P) return fail(AIR_ERR_INVALID_ARG, "plan is NULL");
    TRY(check_dev_ptr(X, "X"));
    TRY(check_dev_ptr(Y, "Y"));
    if (overlap(X, img_bytes(P), Y, sino_bytes(P))) return fail(AIR_ERR_INVALID_ARG, "X and Y overlap");
    SliceDesc s = P->desc;
    s.ext_in = X;
    s.ext_out = Y;
    CUDA_TRY(launch_op(OP_TRANSPOSE, s, SRC_EXT, (cudaStream_t)stream));
    CUDA_TRY(launch_op(OP_FWD, s, SRC_EXT, (cudaStream_t)stream));
    return AIR_OK;
}

extern "C" air_status air_filter(const air_plan *P, const float *Y, float *Z, air_stream stream) {
    if (!P) return fail(AIR_ERR_INVALID_ARG, "plan is NULL");
    TRY(check_dev_ptr(Y, "Y"));
    TRY(check_dev_ptr(Z, "Z"));
    if (overlap(Y, sino_bytes(P), Z, sino_bytes(P))) return fail(AIR_ERR_INVALID_ARG, "Y and Z overlap");
    return apply_filter(P, P->desc, Y, Z, (cudaStream_t)stream);
}

extern "C" air_status air_backproject(const air_plan *P, const float *Y, float *X, air_stream stream) {
    if (!P) return fail(AIR_ERR_INVALID_ARG, "plan is NULL");
    TRY(check_dev_ptr(Y, "Y"));
    TRY(check_dev_ptr(X, "X"));
    if (overlap(X, img_bytes(P), Y, sino_bytes(P))) return fail(AIR_ERR_INVALID_ARG, "X and Y overlap");
    SliceDesc s = P->desc;
    s.ext_in = Y;
    s.ext_out = X;
    CUDA_TRY(launch_op(OP_BWD, s, BWD_PLAIN, (cudaStream_t)stream));
    if (s.bwd_parts > 1) CUDA_TRY(launch_op(OP_BWD_FIN, s, BWD_PLAIN, (cudaStream_t)stream));
    return AIR_OK;
}

extern "C" air_status air_filtered_backproject(const air_plan *P, const float *Y, float *X,
                                               air_stream stream) {
    if (!P) return fail(AIR_ERR_INVALID_ARG, "plan is NULL");
    TRY(check_dev_ptr(Y, "Y"));
    TRY(check_dev_ptr(X, "X"));
    if (overlap(X, img_bytes(P), Y, sino_bytes(P))) return fail(AIR_ERR_INVALID_ARG, "X and Y overlap");
    const cudaStream_t st = (cudaStream_t)stream;
    TRY(apply_filter(P, P->desc, Y, P->desc.zc, st));
    SliceDesc s = P->desc;
    s.ext_in = P->desc.zc;
    s.ext_out = X;
    CUDA_TRY(launch_op(OP_BWD, s, BWD_PLAIN, st));
    if (s.bwd_parts > 1) CUDA_TRY(launch_op(OP_BWD_FIN, s, BWD_PLAIN, st));
    return AIR_OK;
}

extern "C" air_status air_framelet(const air_plan *P, const float *in, float *out, int adjoint,
                                   air_stream stream) {
    if (!P) return fail(AIR_ERR_INVALID_ARG, "plan is NULL");
    TRY(check_dev_ptr(in, "in"));
    TRY(check_dev_ptr(out, "out"));
    const size_t bi = adjoint ? 9 * img_bytes(P) : img_bytes(P);
    const size_t bo = adjoint ? img_bytes(P) : 9 * img_bytes(P);
    if (overlap(in, bi, out, bo)) return fail(AIR_ERR_INVALID_ARG, "in and out overlap");
    SliceDesc s = P->desc;
    s.ext_in = in;
    s.ext_out = out;
    CUDA_TRY(launch_op(adjoint ? OP_FRAMELET_T : OP_FRAMELET, s, 0, (cudaStream_t)stream));
    return AIR_OK;
}

extern "C" air_status air_shrink(const air_plan *P, const float *X, float *b, float *g, float thresh,
                                 double *resid, air_stream stream) {
    if (!P) return fail(AIR_ERR_INVALID_ARG, "plan is NULL");
    TRY(check_dev_ptr(X, "X"));
    TRY(check_dev_ptr(b, "b"));
    TRY(check_dev_ptr(g, "g"));
    if (resid) TRY(check_dev_ptr(resid, "resid"));
    if (!(thresh >= 0.f) || !std::isfinite(thresh)) return fail(AIR_ERR_INVALID_ARG, "thresh must be >= 0");
    const size_t ib = img_bytes(P);
    if (overlap(X, ib, b, 9 * ib) || overlap(X, ib, g, ib) || overlap(b, 9 * ib, g, ib))
        return fail(AIR_ERR_INVALID_ARG, "X, b and g must not overlap");
    const cudaStream_t st = (cudaStream_t)stream;
    SliceDesc s = P->desc;
    s.ext_in = X;
    s.ext_out = b;
    s.ext_out2 = g;
    s.tau = thresh;
    s.ext_scalar = resid;
    s.resid_out = nullptr;
    CUDA_TRY(launch_op(OP_SHRINK, s, 2, st));
    CUDA_TRY(cudaMemcpyAsync(b, P->desc.b2, 9 * ib, cudaMemcpyDeviceToDevice, st));
    return AIR_OK;
}

// ------------------------------------------------------------------ solve
namespace air {

// The split-Bregman program of one slice as a list of phases.
// The split-Bregman program of one slice (Methods, Eq. 5 and ref. [24]).
// Each outer step's CG restarts from the residual the previous CG left,
// corrected for the change of the right-hand side (OP_RESTART): CG keeps
// r = b - M X, and b changes between outer steps only by mu (g_new - g_old).
std::vector<Phase> solve_program(int n_outer, int n_cg, bool tc_ramp) {
    std::vector<Phase> prog;
    const int ramp = tc_ramp ? OP_RAMP_TC : OP_RAMP;
    prog.push_back({ramp, RSRC_Y});        // zc = C y
    prog.push_back({OP_BWD, BWD_RHS0});   // rhs0 = A^T zc
    prog.push_back({OP_BWD_FIN, BWD_RHS0});
    prog.push_back({OP_ZERO, 0});         // X = 0, b = 0, g = g' = 0
    prog.push_back({OP_RESTART, -1});     // r = p = rhs0 (X = 0, g = 0)
    for (int k = 0; k < n_outer; ++k) {
        for (int i = 0; i < n_cg; ++i) {
            prog.push_back({OP_TRANSPOSE, SRC_P});    // q = M p
            prog.push_back({OP_FWD, SRC_P});
            prog.push_back({ramp, RSRC_Z});
            prog.push_back({OP_BWD, BWD_Q});
            prog.push_back({OP_BWD_FIN, BWD_Q});
            prog.push_back({OP_CG_A, 0});
            prog.push_back({OP_CG_B, 0});
        }
        prog.push_back({OP_SHRINK, k & 1});
        if (k + 1 < n_outer) prog.push_back({OP_RESTART, k & 1});   // r += mu (g_k - g_{k-1})
    }
    return prog;
}

// L2-regularised AIR, Eq. (5): (A'^T A + lambda I) X = A'^T Y by n_cg CG steps
// from X = 0 (the first L2 step of the split-Bregman program with g = 0 and
// mu = lambda, without the shrink).
std::vector<Phase> l2_program(int n_cg, bool tc_ramp) {
    std::vector<Phase> prog = solve_program(1, n_cg, tc_ramp);
    prog.pop_back();   // the SHRINK of the outer step
    return prog;
}

// Forward-backward splitting AIR: per iteration the forward step of Eq. (6),
// X + step A'^T (Y - A X) (the residual epilogue at mu = 0 gives
// r = A'^T Y - A'^T A X), then the framelet proximal step.
std::vector<Phase> fbs_program(int n_iter, bool tc_ramp) {
    std::vector<Phase> prog;
    const int ramp = tc_ramp ? OP_RAMP_TC : OP_RAMP;
    prog.push_back({ramp, RSRC_Y});
    prog.push_back({OP_BWD, BWD_RHS0});
    prog.push_back({OP_BWD_FIN, BWD_RHS0});
    prog.push_back({OP_ZERO, 0});
    for (int k = 0; k < n_iter; ++k) {
        prog.push_back({OP_TRANSPOSE, SRC_X});
        prog.push_back({OP_FWD, SRC_X});
        prog.push_back({ramp, RSRC_Z});
        prog.push_back({OP_BWD, BWD_RESID});
        prog.push_back({OP_BWD_FIN, BWD_RESID});
        prog.push_back({OP_AXPY, 0});
        prog.push_back({OP_PROX, 0});
    }
    return prog;
}

air_status run_program_single(const air_plan *P, const SliceDesc &s, const std::vector<Phase> &prog,
                              cudaStream_t st) {
    for (const Phase &ph : prog) {
        if (ph.op == OP_RAMP_TC) {
            const float *src = ph.arg == RSRC_Y ? s.y : s.z;
            TRY(ramp_tc_apply(P, src, s.zc, s.cg, ph.arg == RSRC_Z, st));
        } else {
            CUDA_TRY(launch_op(ph.op, s, ph.arg, st));
        }
    }
    return AIR_OK;
}

air_status check_solve_args(const air_plan *P, const float *Y, float lambda, float mu, int n_outer,
                            int n_cg, const float *X) {
    if (!P) return fail(AIR_ERR_INVALID_ARG, "plan is NULL");
    if (!(mu > 0.f) || !std::isfinite(mu)) return fail(AIR_ERR_INVALID_ARG, "mu must be > 0");
    if (!(lambda >= 0.f) || !std::isfinite(lambda)) return fail(AIR_ERR_INVALID_ARG, "lambda must be >= 0");
    if (n_outer < 0 || n_cg < 0 || n_outer > 100000 || n_cg > 100000)
        return fail(AIR_ERR_INVALID_ARG, "n_outer and n_cg must be in 0..100000");
    if (Y && X && overlap(X, img_bytes(P), Y, sino_bytes(P)))
        return fail(AIR_ERR_INVALID_ARG, "X and Y overlap");
    return AIR_OK;
}

SliceDesc solve_desc(const air_plan *P, const float *Y, float lambda, float mu, float *X, double *resid) {
    SliceDesc s = P->desc;
    s.y = Y;
    s.x = X;
    s.mu = mu;
    s.tau = lambda / mu;
    s.resid_out = resid;
    return s;
}

}  // namespace air

extern "C" air_status air_solve(const air_plan *P, const float *Y, float lambda, float mu, int n_outer,
                                int n_cg, float *X, double *resid, air_stream stream) {
    TRY(check_solve_args(P, Y, lambda, mu, n_outer, n_cg, X));
    TRY(check_dev_ptr(Y, "Y"));
    TRY(check_dev_ptr(X, "X"));
    if (resid) TRY(check_dev_ptr(resid, "resid"));
    const bool tc = P->geom.precision == AIR_PREC_BF16X3 && P->geom.filter == AIR_FILTER_RAMLAK;
    SliceDesc s = solve_desc(P, Y, lambda, mu, X, resid);
    return run_program_single(P, s, solve_program(n_outer, n_cg, tc), (cudaStream_t)stream);
}

extern "C" air_status air_solve_l2(const air_plan *P, const float *Y, float lambda, int n_cg, float *X,
                                   air_stream stream) {
    if (!(lambda > 0.f) || !std::isfinite(lambda)) return fail(AIR_ERR_INVALID_ARG, "lambda must be > 0");
    TRY(check_solve_args(P, Y, 0.f, lambda, 0, n_cg, X));
    TRY(check_dev_ptr(Y, "Y"));
    TRY(check_dev_ptr(X, "X"));
    const bool tc = P->geom.precision == AIR_PREC_BF16X3 && P->geom.filter == AIR_FILTER_RAMLAK;
    SliceDesc s = solve_desc(P, Y, 0.f, lambda, X, nullptr);
    return run_program_single(P, s, l2_program(n_cg, tc), (cudaStream_t)stream);
}

extern "C" air_status air_solve_fbs(const air_plan *P, const float *Y, float lambda, float step, int n_iter,
                                    float *X, air_stream stream) {
    if (!(step > 0.f) || !std::isfinite(step)) return fail(AIR_ERR_INVALID_ARG, "step must be > 0");
    TRY(check_solve_args(P, Y, lambda, 1.f, n_iter, 0, X));
    TRY(check_dev_ptr(Y, "Y"));
    TRY(check_dev_ptr(X, "X"));
    const bool tc = P->geom.precision == AIR_PREC_BF16X3 && P->geom.filter == AIR_FILTER_RAMLAK;
    SliceDesc s = solve_desc(P, Y, 0.f, 1.f, X, nullptr);
    s.mu = 0.f;                 // the residual epilogue then gives A'^T (Y - A X)
    s.tau = step * lambda;      // the proximal threshold
    s.step = step;
    return run_program_single(P, s, fbs_program(n_iter, tc), (cudaStream_t)stream);
}

extern "C" air_status air_fbp(const air_plan *P, const float *Y, float *X, air_stream stream) {
    if (!P) return fail(AIR_ERR_INVALID_ARG, "plan is NULL");
    if (std::fabs(P->geom.arc - 2.0 * M_PI) > 1e-9 * 2.0 * M_PI)
        return fail(AIR_ERR_INVALID_ARG, "FBP needs a full 2 pi scan");
    TRY(check_dev_ptr(Y, "Y"));
    TRY(check_dev_ptr(X, "X"));
    if (overlap(X, img_bytes(P), Y, sino_bytes(P))) return fail(AIR_ERR_INVALID_ARG, "X and Y overlap");
    const cudaStream_t st = (cudaStream_t)stream;
    SliceDesc f = P->desc;        // the filter: the ramp tile with the fan ramp and pre-weight
    f.filter = AIR_FILTER_RAMLAK;
    f.taps = f.fbp_taps;
    f.ramp_diag = f.fbp_diag;
    f.prew = f.fbp_w;
    f.ext_in = Y;
    f.ext_out = P->desc.zc;
    CUDA_TRY(launch_op(OP_RAMP, f, RSRC_EXT, st));
    SliceDesc b = P->desc;
    b.ext_out = X;
    CUDA_TRY(launch_op(OP_FBP, b, 0, st));
    return AIR_OK;
}

extern "C" air_status air_solve_host(const air_plan *P, const float *Y_host, float lambda, float mu,
                                     int n_outer, int n_cg, float *X_host, air_stream stream) {
    TRY(check_solve_args(P, nullptr, lambda, mu, n_outer, n_cg, nullptr));
    if (!Y_host || !X_host) return fail(AIR_ERR_INVALID_ARG, "Y_host and X_host must not be NULL");
    const cudaStream_t st = (cudaStream_t)stream;
    CUDA_TRY(cudaMemcpyAsync(P->ybuf, Y_host, sino_bytes(P), cudaMemcpyHostToDevice, st));
    const bool tc = P->geom.precision == AIR_PREC_BF16X3 && P->geom.filter == AIR_FILTER_RAMLAK;
    SliceDesc s = solve_desc(P, P->ybuf, lambda, mu, P->xbuf, nullptr);
    TRY(run_program_single(P, s, solve_program(n_outer, n_cg, tc), st));
    CUDA_TRY(cudaMemcpyAsync(X_host, P->xbuf, img_bytes(P), cudaMemcpyDeviceToHost, st));
    CUDA_TRY(cudaStreamSynchronize(st));
    return tc ? air_plan_status(P) : AIR_OK;
}
