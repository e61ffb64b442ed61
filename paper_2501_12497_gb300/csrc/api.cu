// C ABI entry points of libmof (include/mof.h): problem lifetime, argument
// validation, precision dispatch and error text. Numerical work happens in
// the kernels of ops_*.cu, krylov.cu, small.cu and solver.cu.
#include "common.cuh"
#include "solver.cuh"

#include <cmath>
#include <cstdarg>
#include <cstring>
#include <algorithm>
#include <atomic>
#include <mutex>
#include <new>

namespace mof {

static thread_local char g_err[512] = "";
static std::atomic<long long> g_launches{0};

void count_launch() { g_launches.fetch_add(1, std::memory_order_relaxed); }
void count_launches_add(long long k) { g_launches.fetch_add(k, std::memory_order_relaxed); }
long long launches_so_far() { return g_launches.load(std::memory_order_relaxed); }

void set_error(const char *fmt, ...) {
    va_list ap;
    va_start(ap, fmt);
    vsnprintf(g_err, sizeof(g_err), fmt, ap);
    va_end(ap);
}

mof_status fail(mof_status st, const char *fmt, ...) {
    va_list ap;
    va_start(ap, fmt);
    vsnprintf(g_err, sizeof(g_err), fmt, ap);
    va_end(ap);
    return st;
}

mof_status cuda_fail(cudaError_t e, const char *what, const char *file, int line) {
    set_error("CUDA error %d (%s) in %s at %s:%d", (int)e, cudaGetErrorString(e), what, file, line);
    return e == cudaErrorMemoryAllocation ? MOF_ENOMEM : MOF_ECUDA;
}

// Round v to 12 significant bits (head) and keep the remainder (tail).
static void split12(double v, float &hi, float &lo) {
    if (v == 0.0 || !std::isfinite(v)) {
        hi = (float)v;
        lo = 0.0f;
        return;
    }
    int e;
    std::frexp(v, &e);
    const double sc = std::ldexp(1.0, 12 - e);
    const double h = std::nearbyint(v * sc) / sc;
    hi = (float)h;
    lo = (float)(v - h);
}

static AngleParams angle_params(double theta, int frame, int nx, int ny, int nb, double h, double db) {
    AngleParams P{};
    const double c = std::cos(theta), s = std::sin(theta);
    P.c = c;
    P.s = s;
    P.frame = frame;
    const int rows = std::fabs(c) >= std::fabs(s);
    P.rows = rows;
    const double cc = rows ? c : s, ss = rows ? s : c;
    const int nfast = rows ? nx : ny, nstep = rows ? ny : nx;
    // f(k, j) = sigma_k / (cc h) + (nfast-1)/2 + ((nstep-1)/2 - j) (ss/cc)
    P.f0_k = db / (cc * h);
    P.f0_c = -0.5 * (nb - 1) * db / (cc * h) + 0.5 * (nfast - 1) + 0.5 * (nstep - 1) * (ss / cc);
    P.df = -ss / cc;
    split12(P.df, P.df_hi, P.df_lo);
    P.wstep_d = h / std::fabs(cc);
    P.wstep = (float)P.wstep_d;
    // t(i, j) = (x_i c + y_j s)/db + (nb-1)/2
    P.tA = h * c / db;
    P.tB = h * s / db;
    P.t0 = 0.5 * (nb - 1) - 0.5 * (nx - 1) * P.tA - 0.5 * (ny - 1) * P.tB;
    split12(P.tA, P.tA_hi, P.tA_lo);
    split12(P.tB, P.tB_hi, P.tB_lo);
    const double mu = std::fmax(std::fabs(c), std::fabs(s));
    P.rfoot_d = mu * h / db;
    P.wfoot_d = h / mu;
    P.rfoot = (float)P.rfoot_d;
    P.wfoot = (float)P.wfoot_d;
    P.inv_rfoot = (float)(1.0 / P.rfoot_d);
    const double fci = std::floor(P.f0_c);
    P.f0c_i = (int)std::fmax(std::fmin(fci, 1e9), -1e9);
    P.f0c_f = (float)(P.f0_c - fci);
    split12(P.f0_k, P.f0k_hi, P.f0k_lo);
    P.df_f = (float)P.df;
    return P;
}

// Fan-beam ray tables. Bin k sits at sigma_k on the detector; its ray leaves the
// source at the angle gamma_k = atan(sigma_k / (rs + rd)) from the central ray, so
// in the normal form {x cos(phi) + y sin(phi) = p} of the parallel rays it has
// phi = theta - gamma_k and p = rs sin(gamma_k) (the source lies on it). From there
// the Joseph march is set up as for a parallel ray of that angle and offset.
template <typename real>
static void fan_ray(double theta, double gamma, double poff, int nx, int ny, double h, FanRay<real> &R) {
    const double phi = theta - gamma, c = std::cos(phi), s = std::sin(phi);
    const int rows = std::fabs(c) >= std::fabs(s);
    const double cc = rows ? c : s, ss = rows ? s : c;
    const int nfast = rows ? nx : ny, nstep = rows ? ny : nx;
    const double f0 = poff / (cc * h) + 0.5 * (nfast - 1) + 0.5 * (nstep - 1) * (ss / cc);
    const double df = -ss / cc;
    // steps whose crossing can lie in (-1, nfast), two steps of margin each side
    int jlo = 0, jhi = nstep - 1;
    if (df != 0.0) {
        const double ja = (-1.0 - f0) / df, jb = ((double)nfast - f0) / df;
        const double lo = std::fmax(std::fmin(ja, jb), -1.0), hi = std::fmin(std::fmax(ja, jb), (double)nstep);
        if (hi < lo) {
            jhi = -1;
        } else {
            jlo = std::max(0, (int)std::floor(lo) - 2);
            jhi = std::min(nstep - 1, (int)std::ceil(hi) + 2);
        }
    } else if (!(f0 > -1.0 && f0 < (double)nfast)) {
        jhi = -1;
    }
    if constexpr (sizeof(real) == 4) {
        (void)jlo;
        (void)jhi;
        const double fl = std::floor(f0);
        R.ibr = 2 * (int)std::fmax(std::fmin(fl, 5e8), -5e8) + rows;
        R.fb = (float)(f0 - fl);
        split12(df, R.df_hi, R.df_lo);
    } else {
        R.rows = rows;
        R.jlo = jlo;
        R.jhi = jhi;
        R.f0 = f0;
        R.df = df;
        R.wstep = h / std::fabs(cc);
        R.pad_ = 0;
    }
}

template <typename real>
static cudaError_t upload_fan_rays(mof_problem *p, const double *angles) {
    const int nb = p->nb;
    std::vector<double> gam(nb), poff(nb);
    for (int k = 0; k < nb; ++k) {
        const double sig = (k - 0.5 * (nb - 1)) * p->db;
        gam[k] = std::atan2(sig, p->rs + p->rd);
        poff[k] = p->rs * std::sin(gam[k]);
    }
    std::vector<FanRay<real>> rays((size_t)p->A * nb);
    for (int a = 0; a < p->A; ++a)
        for (int k = 0; k < nb; ++k) fan_ray<real>(angles[a], gam[k], poff[k], p->nx, p->ny, p->h, rays[(size_t)a * nb + k]);
    cudaError_t e = cudaMalloc(&p->d_fanray, sizeof(FanRay<real>) * rays.size());
    if (e == cudaSuccess) e = cudaMemcpy(p->d_fanray, rays.data(), sizeof(FanRay<real>) * rays.size(), cudaMemcpyHostToDevice);
    return e;
}

static mof_status check_problem(const mof_problem *p) {
    if (!p) return fail(MOF_EINVAL, "null problem");
    return MOF_OK;
}

static cudaStream_t S(void *stream) { return reinterpret_cast<cudaStream_t>(stream); }

}  // namespace mof

using namespace mof;

extern "C" {

const char *mof_last_error(void) { return g_err; }

long long mof_kernel_launches(void) { return g_launches.load(std::memory_order_relaxed); }

void mof_default_params(mof_solver_params *p) {
    if (!p) return;
    p->ell = 10;
    p->tau = 1;
    p->of_iters = 20;
    p->of_ell = 10;
    p->of_dr = 1;
    p->image_rule = MOF_RULE_DP;
    p->eps = 1e-3;
    p->eta = 1.01;
    p->noise_norm = -1.0;
    p->lam_fixed = 0.0;
    p->breakdown_tol = 0.0;
    p->of_streams = 0;
    p->of_scale = 1;
    p->temporal_tv = 0;
    p->of_pq = 2;
    p->plain = 0;
}

mof_status mof_problem_create(const mof_geometry *g, int precision, mof_problem **out) {
    g_err[0] = 0;
    if (!g || !out) return fail(MOF_EINVAL, "null geometry or output pointer");
    *out = nullptr;
    if (g->nx < 2 || g->ny < 2 || g->nt < 2 || g->nb < 1)
        return fail(MOF_EINVAL, "need nx, ny, nt >= 2 and nb >= 1 (got %d %d %d %d)", g->nx, g->ny, g->nt, g->nb);
    if (g->nx > 4096 || g->ny > 4096) return fail(MOF_EUNSUPPORTED, "frames wider than 4096 pixels are not supported");
    if (!g->na || !g->angles) return fail(MOF_EINVAL, "null angle tables");
    if (!(g->pixel_size > 0) || !(g->bin_size > 0)) return fail(MOF_EINVAL, "pixel_size and bin_size must be > 0");
    if (precision != MOF_FP32 && precision != MOF_FP64) return fail(MOF_EINVAL, "unknown precision %d", precision);
    long long A = 0;
    for (int t = 0; t < g->nt; ++t) {
        if (g->na[t] < 1) return fail(MOF_EINVAL, "frame %d has %d angles", t, g->na[t]);
        A += g->na[t];
    }
    if ((long long)g->nx * g->ny * g->nt >= (1LL << 31) / 2 || A * g->nb >= (1LL << 31))
        return fail(MOF_EUNSUPPORTED, "problem too large for 32-bit pixel indexing");
    for (long long a = 0; a < A; ++a)
        if (!std::isfinite(g->angles[a])) return fail(MOF_EINVAL, "angle %lld is not finite", a);

    mof_problem *p = new (std::nothrow) mof_problem();
    if (!p) return fail(MOF_ENOMEM, "host allocation failed");
    p->nx = g->nx; p->ny = g->ny; p->nt = g->nt; p->nb = g->nb;
    p->precision = precision;
    p->h = g->pixel_size; p->db = g->bin_size;
    p->ns = (long long)g->nx * g->ny;
    p->n = p->ns * g->nt;
    p->m = A * g->nb;
    p->nv = (long long)(g->nt - 1) * 2 * p->ns;
    p->A = (int)A;
    p->na.assign(g->na, g->na + g->nt);
    p->aoff.resize(g->nt + 1);
    p->aoff[0] = 0;
    for (int t = 0; t < g->nt; ++t) p->aoff[t + 1] = p->aoff[t] + g->na[t];
    std::vector<AngleParams> tab(A);
    for (int t = 0; t < g->nt; ++t)
        for (int a = p->aoff[t]; a < p->aoff[t + 1]; ++a)
            tab[a] = angle_params(g->angles[a], t, g->nx, g->ny, g->nb, g->pixel_size, g->bin_size);
    cudaError_t e = cudaGetDevice(&p->device);
    if (e == cudaSuccess) e = cudaMalloc(&p->d_ang, sizeof(AngleParams) * A);
    if (e == cudaSuccess) e = cudaMalloc(&p->d_aoff, sizeof(int) * (g->nt + 1));
    if (e == cudaSuccess) e = cudaMemcpy(p->d_ang, tab.data(), sizeof(AngleParams) * A, cudaMemcpyHostToDevice);
    if (e == cudaSuccess) e = cudaMemcpy(p->d_aoff, p->aoff.data(), sizeof(int) * (g->nt + 1), cudaMemcpyHostToDevice);
    if (e != cudaSuccess) {
        mof_status st = cuda_fail(e, "mof_problem_create", __FILE__, __LINE__);
        mof_problem_destroy(p);
        return st;
    }
    *out = p;
    return MOF_OK;
}

mof_status mof_problem_create_fan(const mof_geometry *g, double source_distance, double detector_distance,
                                  int precision, mof_problem **out) {
    if (!g || !out) return fail(MOF_EINVAL, "null geometry or output pointer");
    *out = nullptr;
    const double half_diag = 0.5 * std::hypot((double)g->nx, (double)g->ny) * g->pixel_size;
    if (!(source_distance > half_diag + 2.0 * g->pixel_size) || !std::isfinite(source_distance))
        return fail(MOF_EINVAL, "source_distance %g must exceed half the frame diagonal plus two pixels (%g)",
                    source_distance, half_diag + 2.0 * g->pixel_size);
    if (!(detector_distance >= 0.0) || !std::isfinite(detector_distance))
        return fail(MOF_EINVAL, "detector_distance must be finite and >= 0");
    // The transpose finds a pixel's bins from the central projections t = (q . f) / (q . e) of
    // its segments' end points (q the point seen from the source), scaled by (rs + rd) / bin_size,
    // in FP32 with a margin of FAN_PAD_BINS. Each of about a dozen roundings (the stored source
    // offset and directions, the pixel position, the two dot products, the approximate
    // division) contributes at most the unit roundoff u = 2^-24 relative to
    // |q| / (q . e) <= 1 + |t|, which the division scales by 1 + |t| again; |t| is at most the
    // detector's half width over rs + rd, and the bin coordinate's own roundings add 2 u nb. A
    // geometry whose bound exceeds half the margin is rejected.
    const double fan_u = std::ldexp(1.0, -24), fan_scale = (source_distance + detector_distance) / g->bin_size;
    const double fan_tmax = (0.5 * g->nb + 1.0) / fan_scale;
    const double fan_bound = 12.0 * fan_u * (1.0 + fan_tmax) * (1.0 + fan_tmax) * fan_scale + 2.0 * fan_u * g->nb;
    if (!(fan_bound <= 0.5 * FAN_PAD_BINS))
        return fail(MOF_EUNSUPPORTED,
                    "fan geometry: the FP32 bin search's rounding bound %.3g bins (from (source_distance + "
                    "detector_distance) / bin_size = %g) exceeds half its margin of %g bins",
                    fan_bound, fan_scale, FAN_PAD_BINS);
    mof_problem *p = nullptr;
    MOF_TRY(mof_problem_create(g, precision, &p));
    p->fan = 1;
    p->rs = source_distance;
    p->rd = detector_distance;
    p->fan_scale = (float)((source_distance + detector_distance) / g->bin_size);
    std::vector<FanView> views(p->A);
    const double cx = 0.5 * (g->nx - 1) * g->pixel_size, cy = 0.5 * (g->ny - 1) * g->pixel_size;
    for (int a = 0; a < p->A; ++a) {
        const double th = g->angles[a], ex = -std::sin(th), ey = std::cos(th);
        // q = p - S, S = -rs e, p = (x h - cx, y h - cy)
        views[a] = FanView{(float)(-cx + source_distance * ex), (float)(-cy + source_distance * ey), (float)ex, (float)ey,
                           (float)std::cos(th), (float)std::sin(th)};
    }
    cudaError_t e = precision == MOF_FP64 ? upload_fan_rays<double>(p, g->angles) : upload_fan_rays<float>(p, g->angles);
    if (e == cudaSuccess) e = cudaMalloc(&p->d_fanview, sizeof(FanView) * p->A);
    if (e == cudaSuccess) e = cudaMemcpy(p->d_fanview, views.data(), sizeof(FanView) * p->A, cudaMemcpyHostToDevice);
    if (e != cudaSuccess) {
        mof_status st = cuda_fail(e, "mof_problem_create_fan", __FILE__, __LINE__);
        mof_problem_destroy(p);
        return st;
    }
    *out = p;
    return MOF_OK;
}

void mof_problem_destroy(mof_problem *p) {
    if (!p) return;
    free_workspace(p);
    if (p->d_fanray) cudaFree(p->d_fanray);
    if (p->d_fanview) cudaFree(p->d_fanview);
    if (p->d_ang) cudaFree(p->d_ang);
    if (p->d_aoff) cudaFree(p->d_aoff);
    delete p;
}

mof_status mof_problem_sizes(const mof_problem *p, long long *n, long long *m, long long *nv) {
    MOF_TRY(check_problem(p));
    if (n) *n = p->n;
    if (m) *m = p->m;
    if (nv) *nv = p->nv;
    return MOF_OK;
}

#define DISPATCH(p, call_f, call_d) ((p)->precision == MOF_FP64 ? (call_d) : (call_f))
#define F(x) ((float *)(x))
#define CF(x) ((const float *)(x))
#define D(x) ((double *)(x))
#define CD(x) ((const double *)(x))

mof_status mof_apply_A(mof_problem *p, const void *u, void *b, void *stream) {
    g_err[0] = 0;
    MOF_TRY(check_problem(p));
    if (!u || !b) return fail(MOF_EINVAL, "null array");
    void *uT = nullptr;
    MOF_TRY(apply_scratch(p, SCR_IMAGE, &uT));
    return DISPATCH(p, launch_project<float>(p, CF(u), F(uT), F(b), S(stream)),
                    launch_project<double>(p, CD(u), D(uT), D(b), S(stream)));
}

mof_status mof_apply_AT(mof_problem *p, const void *b, void *u, void *stream) {
    g_err[0] = 0;
    MOF_TRY(check_problem(p));
    if (!u || !b) return fail(MOF_EINVAL, "null array");
    return DISPATCH(p, launch_backproject<float>(p, CF(b), F(u), S(stream)),
                    launch_backproject<double>(p, CD(b), D(u), S(stream)));
}

mof_status mof_apply_grad(mof_problem *p, const void *u, void *g, void *stream) {
    g_err[0] = 0;
    MOF_TRY(check_problem(p));
    if (!u || !g) return fail(MOF_EINVAL, "null array");
    return DISPATCH(p, launch_grad<float>(p, p->nt, CF(u), F(g), S(stream)),
                    launch_grad<double>(p, p->nt, CD(u), D(g), S(stream)));
}

mof_status mof_apply_gradT(mof_problem *p, const void *g, void *u, void *stream) {
    g_err[0] = 0;
    MOF_TRY(check_problem(p));
    if (!u || !g) return fail(MOF_EINVAL, "null array");
    return DISPATCH(p, launch_gradT<float>(p, p->nt, CF(g), F(u), S(stream)),
                    launch_gradT<double>(p, p->nt, CD(g), D(u), S(stream)));
}

mof_status mof_set_warp(mof_problem *p, int mode) {
    MOF_TRY(check_problem(p));
    if (mode != 0 && mode != 1) return fail(MOF_EINVAL, "unknown warp mode %d (0 bilinear, 1 rounding)", mode);
    p->warp_mode = mode;
    return MOF_OK;
}

mof_status mof_apply_flow(mof_problem *p, const void *u, const void *s, const void *sr, void *r, void *stream) {
    g_err[0] = 0;
    MOF_TRY(check_problem(p));
    if (!u || !s || !sr || !r) return fail(MOF_EINVAL, "null array");
    return DISPATCH(p, launch_flow<float>(p, CF(u), CF(s), CF(sr), F(r), S(stream)),
                    launch_flow<double>(p, CD(u), CD(s), CD(sr), D(r), S(stream)));
}

mof_status mof_apply_flowT(mof_problem *p, const void *r, const void *s, const void *sr, void *u, void *stream) {
    g_err[0] = 0;
    MOF_TRY(check_problem(p));
    if (!u || !s || !sr || !r) return fail(MOF_EINVAL, "null array");
    void *rad = nullptr;
    MOF_TRY(apply_scratch(p, SCR_RADIUS, &rad));
    int *rs = (int *)rad, *rr = rs + (long long)(p->nt - 1) * tile_bound_ints(p);
    if (p->precision == MOF_FP64) {
        MOF_TRY(launch_tile_bounds<double>(p, CD(s), CD(sr), rs, rr, S(stream)));
        return launch_flowT<double>(p, CD(r), CD(s), CD(sr), rs, rr, D(u), S(stream));
    }
    MOF_TRY(launch_tile_bounds<float>(p, CF(s), CF(sr), rs, rr, S(stream)));
    return launch_flowT<float>(p, CF(r), CF(s), CF(sr), rs, rr, F(u), S(stream));
}

mof_status mof_apply_flow_ds(mof_problem *p, const void *u, const void *s, const void *sr, const void *gr, void *gs,
                             void *gsr, void *stream) {
    g_err[0] = 0;
    MOF_TRY(check_problem(p));
    if (!u || !s || !sr || !gr || !gs || !gsr) return fail(MOF_EINVAL, "null array");
    return DISPATCH(p, launch_flow_ds<float>(p, CF(u), CF(s), CF(sr), CF(gr), F(gs), F(gsr), S(stream)),
                    launch_flow_ds<double>(p, CD(u), CD(s), CD(sr), CD(gr), D(gs), D(gsr), S(stream)));
}

// Allocation-free Mhat^T: the per-tile displacement bounds of the gathers live
// in a fixed device array instead of the problem's lazily allocated workspace
// (include/mof.h states the size limit, the one-time set-up and the
// concurrency rule).
static __device__ __align__(256) int g_flowT_noalloc_bounds[MOF_FLOWT_NOALLOC_MAX_INTS];

static mof_status flowT_noalloc_scratch(const mof_problem *p, int **out) {
    constexpr int MAX_DEVICES = 64;
    static std::mutex mu;
    static int *addr[MAX_DEVICES] = {};
    if (p->device < 0 || p->device >= MAX_DEVICES)
        return fail(MOF_EUNSUPPORTED, "device ordinal %d is outside the supported range", p->device);
    // every call runs with the problem's device current: the kernels are launched on the
    // current device, and the cached address belongs to the problem's device
    int cur = -1;
    MOF_CUDA(cudaGetDevice(&cur));
    if (cur != p->device)
        return fail(MOF_EINVAL, "problem on device %d, called with device %d current", p->device, cur);
    std::lock_guard<std::mutex> lock(mu);
    if (!addr[p->device]) {  // one-time set-up on this device
        void *a = nullptr;
        MOF_CUDA(cudaGetSymbolAddress(&a, g_flowT_noalloc_bounds));
        addr[p->device] = static_cast<int *>(a);
    }
    *out = addr[p->device];
    return MOF_OK;
}

mof_status mof_apply_flowT_noalloc(mof_problem *p, const void *r, const void *s, const void *sr, void *u, void *stream) {
    g_err[0] = 0;
    MOF_TRY(check_problem(p));
    if (!u || !s || !sr || !r) return fail(MOF_EINVAL, "null array");
    const long long need = 2LL * (p->nt - 1) * tile_bound_ints(p);
    if (need > MOF_FLOWT_NOALLOC_MAX_INTS)
        return fail(MOF_EUNSUPPORTED,
                    "mof_apply_flowT_noalloc: the problem needs %lld ints of tile bounds, more than the fixed %d "
                    "(use mof_apply_flowT)",
                    need, MOF_FLOWT_NOALLOC_MAX_INTS);
    int *rad = nullptr;
    MOF_TRY(flowT_noalloc_scratch(p, &rad));
    int *rs = rad, *rr = rad + (long long)(p->nt - 1) * tile_bound_ints(p);
    if (p->precision == MOF_FP64) {
        MOF_TRY(launch_tile_bounds<double>(p, CD(s), CD(sr), rs, rr, S(stream)));
        return launch_flowT<double>(p, CD(r), CD(s), CD(sr), rs, rr, D(u), S(stream));
    }
    MOF_TRY(launch_tile_bounds<float>(p, CF(s), CF(sr), rs, rr, S(stream)));
    return launch_flowT<float>(p, CF(r), CF(s), CF(sr), rs, rr, F(u), S(stream));
}

mof_status mof_of_fields(mof_problem *p, const void *u, int dr, void *ux, void *uy, void *ut, void *stream) {
    g_err[0] = 0;
    MOF_TRY(check_problem(p));
    if (!u || !ux || !uy || !ut) return fail(MOF_EINVAL, "null array");
    if (dr < 1 || dr > 64) return fail(MOF_EINVAL, "dr must be in [1, 64] (got %d)", dr);
    return DISPATCH(p, launch_of_fields<float>(p, CF(u), dr, F(ux), F(uy), F(ut), S(stream)),
                    launch_of_fields<double>(p, CD(u), dr, D(ux), D(uy), D(ut), S(stream)));
}

mof_status mof_downsample(mof_problem *p, int a, const void *u, void *uc, void *stream) {
    g_err[0] = 0;
    MOF_TRY(check_problem(p));
    if (!u || !uc) return fail(MOF_EINVAL, "null array");
    if (a < 1 || p->nx % a || p->ny % a)
        return fail(MOF_EINVAL, "the factor must be >= 1 and divide nx and ny (got %d for %d x %d)", a, p->nx, p->ny);
    return DISPATCH(p, launch_downsample<float>(p, a, CF(u), F(uc), S(stream)),
                    launch_downsample<double>(p, a, CD(u), D(uc), S(stream)));
}

mof_status mof_upsample_velocity(mof_problem *p, int a, const void *sc, void *s, void *stream) {
    g_err[0] = 0;
    MOF_TRY(check_problem(p));
    if (!sc || !s) return fail(MOF_EINVAL, "null array");
    if (a < 1 || p->nx % a || p->ny % a)
        return fail(MOF_EINVAL, "the factor must be >= 1 and divide nx and ny (got %d for %d x %d)", a, p->nx, p->ny);
    return DISPATCH(p, launch_upsample_velocity<float>(p, a, CF(sc), F(s), S(stream)),
                    launch_upsample_velocity<double>(p, a, CD(sc), D(s), S(stream)));
}

mof_status mof_apply_flow_lin(mof_problem *p, const void *ux, const void *uy, const void *ut, const void *s, void *r,
                              void *stream) {
    g_err[0] = 0;
    MOF_TRY(check_problem(p));
    if (!ux || !uy || !ut || !s || !r) return fail(MOF_EINVAL, "null array");
    return DISPATCH(p, launch_flow_lin<float>(p, CF(ux), CF(uy), CF(ut), CF(s), F(r), S(stream)),
                    launch_flow_lin<double>(p, CD(ux), CD(uy), CD(ut), CD(s), D(r), S(stream)));
}

mof_status mof_apply_flow_linT(mof_problem *p, const void *ux, const void *uy, const void *r, void *gs, void *stream) {
    g_err[0] = 0;
    MOF_TRY(check_problem(p));
    if (!ux || !uy || !r || !gs) return fail(MOF_EINVAL, "null array");
    return DISPATCH(p, launch_flow_linT<float>(p, CF(ux), CF(uy), CF(r), F(gs), S(stream)),
                    launch_flow_linT<double>(p, CD(ux), CD(uy), CD(r), D(gs), S(stream)));
}

mof_status mof_apply_vgrad(mof_problem *p, const void *s, void *gs, void *stream) {
    g_err[0] = 0;
    MOF_TRY(check_problem(p));
    if (!s || !gs) return fail(MOF_EINVAL, "null array");
    const int nf = 2 * (p->nt - 1);
    return DISPATCH(p, launch_grad<float>(p, nf, CF(s), F(gs), S(stream)),
                    launch_grad<double>(p, nf, CD(s), D(gs), S(stream)));
}

mof_status mof_apply_vgradT(mof_problem *p, const void *gs, void *s, void *stream) {
    g_err[0] = 0;
    MOF_TRY(check_problem(p));
    if (!s || !gs) return fail(MOF_EINVAL, "null array");
    const int nf = 2 * (p->nt - 1);
    return DISPATCH(p, launch_gradT<float>(p, nf, CF(gs), F(s), S(stream)),
                    launch_gradT<double>(p, nf, CD(gs), D(s), S(stream)));
}

mof_status mof_reverse_flow(mof_problem *p, const void *s, void *sr, void *stream) {
    g_err[0] = 0;
    MOF_TRY(check_problem(p));
    if (!s || !sr) return fail(MOF_EINVAL, "null array");
    void *rad = nullptr, *dest = nullptr;
    MOF_TRY(apply_scratch(p, SCR_RADIUS, &rad));
    MOF_TRY(apply_scratch(p, SCR_DEST, &dest));
    if (p->precision == MOF_FP64) return launch_reverse_flow<double>(p, CD(s), (int *)rad, (int *)dest, D(sr), S(stream));
    return launch_reverse_flow<float>(p, CF(s), (int *)rad, (int *)dest, F(sr), S(stream));
}

mof_status mof_apply_reg_normal(mof_problem *p, const void *x, const void *uk, const void *s, const void *sr, double eps,
                                void *y, void *stream) {
    g_err[0] = 0;
    MOF_TRY(check_problem(p));
    if (!x || !uk || !s || !sr || !y) return fail(MOF_EINVAL, "null array");
    if (!(eps > 0) || !std::isfinite(eps)) return fail(MOF_EINVAL, "eps must be finite and > 0");
    void *rad = nullptr, *q = nullptr;
    MOF_TRY(apply_scratch(p, SCR_RADIUS, &rad));
    MOF_TRY(apply_scratch(p, SCR_FLOWROWS, &q));
    int *rs = (int *)rad, *rr = rs + (long long)(p->nt - 1) * tile_bound_ints(p);
    if (p->precision == MOF_FP64) {
        MOF_TRY(launch_tile_bounds<double>(p, CD(s), CD(sr), rs, rr, S(stream)));
        return launch_reg_normal<double>(p, 0, CD(x), CD(uk), CD(s), CD(sr), rs, rr, eps, 1.0, nullptr, nullptr, D(q), D(y),
                                         S(stream));
    }
    MOF_TRY(launch_tile_bounds<float>(p, CF(s), CF(sr), rs, rr, S(stream)));
    return launch_reg_normal<float>(p, 0, CF(x), CF(uk), CF(s), CF(sr), rs, rr, eps, 1.0, nullptr, nullptr, F(q), F(y),
                                    S(stream));
}

mof_status mof_debug_set_wait_limit(long long polls) {
    g_err[0] = 0;
    return set_wait_polls(polls);
}

mof_status mof_set_timing(mof_problem *p, int enable) {
    MOF_TRY(check_problem(p));
    p->timing = enable ? 1 : 0;
    return MOF_OK;
}

}  // extern "C"
