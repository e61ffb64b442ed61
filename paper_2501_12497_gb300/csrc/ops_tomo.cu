// K1 ray-driven Joseph projector b = H u and K2 pixel-driven exact transpose
// u = H^T b (Sec. 2.1: H = blockdiag(H^1..H^nt), 2D parallel beam).
//
// Both evaluate the same matrix entry
//     a(theta, k; i, j) = (h/mu) * max(0, 1 - |sigma_k - p_ij| / (mu h)),
//     p_ij = x_i cos(theta) + y_j sin(theta),  mu = max(|cos|, |sin|),
// K1 from the ray side (march over the axis the ray is least inclined to,
// two linear-interpolation taps per step, weight h/mu), K2 from the pixel
// side (the <= 2 bins within mu*h of p_ij), so <H u, b> = <u, H^T b> holds to
// rounding.
//
// Fan beam (flat detector, the geometry of the paper's experiments, Sec. 5.1):
// every ray is the line from the source through its bin, integrated by the
// same Joseph rule with its own direction (k_project_fan); the transpose
// (k_backproject_fan) visits, per pixel and view, the bins whose rays can
// cross the pixel's two Joseph segments and re-evaluates the forward entry.
#include "common.cuh"

namespace mof {

// --------------------------------------------------------------- transpose
// uT[t][x][y] = u[t][y][x], 32x32 tiles through shared memory.
template <typename real>
__global__ void k_transpose(const real *__restrict__ u, real *__restrict__ uT, int nx, int ny) {
    __shared__ real tile[32][33];
    const long long off = (long long)blockIdx.z * nx * ny;
    const int x0 = blockIdx.x * 32, y0 = blockIdx.y * 32;
    for (int dy = threadIdx.y; dy < 32; dy += blockDim.y) {
        const int x = x0 + threadIdx.x, y = y0 + dy;
        if (x < nx && y < ny) tile[dy][threadIdx.x] = u[off + (long long)y * nx + x];
    }
    __syncthreads();
    for (int dx = threadIdx.y; dx < 32; dx += blockDim.y) {
        const int y = y0 + threadIdx.x, x = x0 + dx;
        if (x < nx && y < ny) uT[off + (long long)x * ny + y] = tile[threadIdx.x][dx];
    }
}

// -------------------------------------------------------------- K1 project
// One thread per ray (angle a = blockIdx.y, bin k). Rays of one warp are 32
// adjacent bins of one angle, so at each step they read adjacent pixels of
// one image row (of the transposed frame for steep angles): coalesced. In FP32
// the ray sum is compensated (Kahan, per step of two taps): its rounding stays
// at a few units of FP32 however long the ray.
template <typename real>
__global__ void __launch_bounds__(128) k_project(const real *__restrict__ u, const real *__restrict__ uT,
                                                 real *__restrict__ b, const AngleParams *__restrict__ ang,
                                                 int nx, int ny, int nb) {
    const int a = blockIdx.y;
    const int k = blockIdx.x * blockDim.x + threadIdx.x;
    if (k >= nb) return;
    const AngleParams &P = ang[a];
    const long long ns = (long long)nx * ny;
    const int rows = P.rows;
    const real *img = rows ? u + P.frame * ns : uT + P.frame * ns;
    const int nfast = rows ? nx : ny, nstep = rows ? ny : nx;
    real acc = 0;
    if constexpr (sizeof(real) == 4) {
        // f(k, j) = f0(k) + j df, in FP32 with split steps (the base in FP64 when nb >= 4096):
        // the base f0(k) = f0c_i + f0c_f + k (f0k_hi + f0k_lo) and each step j df are
        // evaluated as an integer part plus a fraction accurate to ~1e-7
        int ib;
        float fb;
        if (nb < 4096) {
            affine_frac(P.f0c_i, P.f0c_f, P.f0k_hi, P.f0k_lo, k, ib, fb);
        } else {  // k * f0k_hi would not be exact: the base in FP64
            const double f0d = (double)k * P.f0_k + P.f0_c, fl0 = floor(f0d);
            ib = (int)fmax(fmin(fl0, 1e9), -1e9);
            fb = (float)(f0d - fl0);
        }
        // steps whose crossing can lie in (-1, nfast), with two steps of margin each side
        // (the taps are bounds-checked, so extra steps add nothing)
        int jlo = 0, jhi = nstep - 1;
        const float f0 = (float)ib + fb;
        if (P.df_f != 0.0f) {
            const float ja = (-1.0f - f0) / P.df_f, jb = ((float)nfast - f0) / P.df_f;
            const float lo = fmaxf(fminf(ja, jb), -1.0f), hi = fminf(fmaxf(ja, jb), (float)nstep);
            jlo = max(0, (int)floorf(lo) - 2);
            jhi = min(nstep - 1, (int)ceilf(hi) + 2);
        } else if (!(f0 > -1.0f && f0 < (float)nfast)) {
            jhi = -1;
        }
        float cmp = 0.f;  // Kahan compensation of the ray sum (a ray adds up to 2 nx taps)
#pragma unroll 4
        for (int j = jlo; j <= jhi; ++j) {
            int i0;
            float w1;
            affine_frac(ib, fb, P.df_hi, P.df_lo, j, i0, w1);
            const real *row = img + (long long)j * nfast;
            float tap = 0.f;
            if (i0 >= 0 && i0 < nfast) tap = (1.0f - w1) * ldg(row + i0);
            if (i0 + 1 >= 0 && i0 + 1 < nfast) tap = fmaf(w1, ldg(row + i0 + 1), tap);
            const float y = __fsub_rn(tap, cmp), t = __fadd_rn(acc, y);
            cmp = __fsub_rn(__fsub_rn(t, acc), y);
            acc = t;
        }
        b[(long long)a * nb + k] = acc * P.wstep;
    } else {
        const double f0 = (double)k * P.f0_k + P.f0_c;  // fractional fast index at step 0
        int jlo = 0, jhi = nstep - 1;
        if (P.df != 0.0) {
            double ja = (-1.0 - f0) / P.df, jb = ((double)nfast - f0) / P.df;
            double lo = fmin(ja, jb), hi = fmax(ja, jb);
            lo = fmax(lo, -1.0);
            hi = fmin(hi, (double)nstep);
            jlo = max(0, (int)floor(lo) - 1);
            jhi = min(nstep - 1, (int)ceil(hi) + 1);
        } else if (!(f0 > -1.0 && f0 < (double)nfast)) {
            jhi = -1;
        }
        for (int j = jlo; j <= jhi; ++j) {
            const double f = fma((double)j, P.df, f0);
            const double fl = floor(f);
            const int i0 = (int)fl;
            const double w1 = f - fl;
            const real *row = img + (long long)j * nfast;
            if (i0 >= 0 && i0 < nfast) acc = fma(1.0 - w1, ldg(row + i0), acc);
            if (i0 + 1 >= 0 && i0 + 1 < nfast) acc = fma(w1, ldg(row + i0 + 1), acc);
        }
        b[(long long)a * nb + k] = acc * (real)P.wstep_d;
    }
}

// ---------------------------------------------------------- K1 fan beam
// One thread per ray (view a = blockIdx.y, bin k); the march of the parallel
// kernel with the ray's own start and step from the ray table.
template <typename real>
__global__ void __launch_bounds__(128) k_project_fan(const real *__restrict__ u, const real *__restrict__ uT,
                                                     real *__restrict__ b, const FanRay<real> *__restrict__ rays,
                                                     const AngleParams *__restrict__ ang, int nx, int ny, int nb, real h) {
    const int a = blockIdx.y;
    const int k = blockIdx.x * blockDim.x + threadIdx.x;
    if (k >= nb) return;
    const long long ns = (long long)nx * ny;
    const FanRay<real> R = rays[(long long)a * nb + k];
    const int frame = ang[a].frame;
    real acc = 0, wstep;
    if constexpr (sizeof(real) == 4) {
        const int rows = R.ibr & 1, ib = R.ibr >> 1;
        const float *img = rows ? u + frame * ns : uT + frame * ns;
        const int nfast = rows ? nx : ny, nstep = rows ? ny : nx;
        const float df = R.df_hi + R.df_lo;
        wstep = h * sqrtf(fmaf(df, df, 1.0f));
        // steps whose crossing can lie in (-1, nfast), two steps of margin each side
        int jlo = 0, jhi = nstep - 1;
        const float f0 = (float)ib + R.fb;
        if (df != 0.0f) {
            const float ja = (-1.0f - f0) / df, jb = ((float)nfast - f0) / df;
            const float lo = fmaxf(fminf(ja, jb), -1.0f), hi = fminf(fmaxf(ja, jb), (float)nstep);
            jlo = max(0, (int)floorf(lo) - 2);
            jhi = min(nstep - 1, (int)ceilf(hi) + 2);
        } else if (!(f0 > -1.0f && f0 < (float)nfast)) {
            jhi = -1;
        }
#pragma unroll 4
        for (int j = jlo; j <= jhi; ++j) {
            int i0;
            float w1;
            affine_frac(ib, R.fb, R.df_hi, R.df_lo, j, i0, w1);
            const float *row = img + (long long)j * nfast;
            if (i0 >= 0 && i0 < nfast) acc = fmaf(1.0f - w1, ldg(row + i0), acc);
            if (i0 + 1 >= 0 && i0 + 1 < nfast) acc = fmaf(w1, ldg(row + i0 + 1), acc);
        }
    } else {
        const double *img = R.rows ? u + frame * ns : uT + frame * ns;
        const int nfast = R.rows ? nx : ny;
        wstep = R.wstep;
        for (int j = R.jlo; j <= R.jhi; ++j) {
            const double f = fma((double)j, R.df, R.f0), fl = floor(f);
            const int i0 = (int)fl;
            const double w1 = f - fl;
            const double *row = img + (long long)j * nfast;
            if (i0 >= 0 && i0 < nfast) acc = fma(1.0 - w1, ldg(row + i0), acc);
            if (i0 + 1 >= 0 && i0 + 1 < nfast) acc = fma(w1, ldg(row + i0 + 1), acc);
        }
    }
    b[(long long)a * nb + k] = acc * wstep;
}

template <typename real>
mof_status launch_project(const mof_problem *p, const real *u, real *uT, real *b, cudaStream_t st, bool per_frame) {
    dim3 tb(32, 8), tg((p->nx + 31) / 32, (p->ny + 31) / 32, p->nt);
    if (per_frame && !p->fan) {  // the plain form: frame by frame (the angles' tables hold their frame)
        const long long ns = (long long)p->nx * p->ny;
        for (int t = 0; t < p->nt; ++t) {
            dim3 tg1((p->nx + 31) / 32, (p->ny + 31) / 32, 1);
            ::mof::count_launch(), k_transpose<real><<<tg1, tb, 0, st>>>(u + t * ns, uT + t * ns, p->nx, p->ny);
            const int a0 = p->aoff[t], na = p->aoff[t + 1] - a0;
            ::mof::count_launch(), k_project<real><<<dim3((p->nb + 127) / 128, na), 128, 0, st>>>(u, uT, b + (long long)a0 * p->nb,
                                                                                             p->d_ang + a0, p->nx, p->ny, p->nb);
        }
        MOF_LAUNCH_CHECK();
        return MOF_OK;
    }
    ::mof::count_launch(), k_transpose<real><<<tg, tb, 0, st>>>(u, uT, p->nx, p->ny);
    MOF_LAUNCH_CHECK();
    if (p->fan) {
        dim3 grid((p->nb + 127) / 128, p->A);
        ::mof::count_launch(), k_project_fan<real><<<grid, 128, 0, st>>>(u, uT, b, static_cast<const FanRay<real> *>(p->d_fanray),
                                                                        p->d_ang, p->nx, p->ny, p->nb, (real)p->h);
        MOF_LAUNCH_CHECK();
        return MOF_OK;
    }
    dim3 grid((p->nb + 127) / 128, p->A);
    ::mof::count_launch(), k_project<real><<<grid, 128, 0, st>>>(u, uT, b, p->d_ang, p->nx, p->ny, p->nb);
    MOF_LAUNCH_CHECK();
    return MOF_OK;
}

// ---------------------------------------------------------- K2 backproject
// One thread per pixel (tile 32 x 8 per block), looping over the angles of
// its frame. Per angle the block's base bin coordinate at the tile origin is
// computed once in FP64 (shared memory); each pixel adds its small in-tile
// offset with the split-step evaluation, keeping the footprint weight
// accurate to ~1e-7 at any grid size.
constexpr int BP_TX = 32, BP_TY = 8, BP_CHUNK = 64;

template <typename real>
__global__ void __launch_bounds__(BP_TX *BP_TY) k_backproject(const real *__restrict__ b, real *__restrict__ u,
                                                              const AngleParams *__restrict__ ang,
                                                              const int *__restrict__ aoff, int nx, int ny, int nb, int t0) {
    // per angle of the chunk: the bin coordinate at the tile origin (integer + fraction,
    // from FP64) and the constants of the footprint, shared by the block's pixels
    __shared__ int s_ib[BP_CHUNK];
    __shared__ float s_fb[BP_CHUNK], s_tAh[BP_CHUNK], s_tAl[BP_CHUNK], s_tBh[BP_CHUNK], s_tBl[BP_CHUNK];
    __shared__ float s_r[BP_CHUNK], s_ir[BP_CHUNK], s_wf[BP_CHUNK];
    __shared__ double s_tb[BP_CHUNK];
    const int t = t0 + blockIdx.z;
    const int x0 = blockIdx.x * BP_TX, y0 = blockIdx.y * BP_TY;
    const int di = threadIdx.x, dj = threadIdx.y;
    const int x = x0 + di, y = y0 + dj;
    const int tid = threadIdx.y * BP_TX + threadIdx.x;
    const int a_begin = aoff[t], a_end = aoff[t + 1];
    real acc = 0;
    for (int ac = a_begin; ac < a_end; ac += BP_CHUNK) {
        const int cn = min(BP_CHUNK, a_end - ac);
        __syncthreads();
        if (tid < cn) {
            const AngleParams &P = ang[ac + tid];
            const double tb = P.t0 + (double)x0 * P.tA + (double)y0 * P.tB;
            const double fl = floor(tb);
            s_ib[tid] = (int)fmax(fmin(fl, 1e9), -1e9);
            s_fb[tid] = (float)(tb - fl);
            s_tb[tid] = tb;
            s_tAh[tid] = P.tA_hi;
            s_tAl[tid] = P.tA_lo;
            s_tBh[tid] = P.tB_hi;
            s_tBl[tid] = P.tB_lo;
            s_r[tid] = P.rfoot;
            s_ir[tid] = P.inv_rfoot;
            s_wf[tid] = P.wfoot;
        }
        __syncthreads();
        if (x < nx && y < ny) {
            for (int q = 0; q < cn; ++q) {
                const real *row = b + (long long)(ac + q) * nb;
                if constexpr (sizeof(real) == 4) {
                    // bin coordinate t = ib + fr of this pixel (split-step, exact products)
                    const float pa = (float)di * s_tAh[q], pb = (float)dj * s_tBh[q];
                    const float pfa = floorf(pa), pfb = floorf(pb);
                    float fr = s_fb[q] + (pa - pfa) + (pb - pfb) + fmaf((float)di, s_tAl[q], (float)dj * s_tBl[q]);
                    const float ff = floorf(fr);
                    const int ib = s_ib[q] + (int)pfa + (int)pfb + (int)ff;
                    fr -= ff;
                    const float r = s_r[q], ir = s_ir[q], wf = s_wf[q];
                    if (r <= 1.0f) {  // at most the two bins around t
                        const float d1 = 1.0f - fr;
                        if (fr < r && ib >= 0 && ib < nb) acc = fmaf(wf * (1.0f - fr * ir), ldg(row + ib), acc);
                        if (d1 < r && ib + 1 >= 0 && ib + 1 < nb) acc = fmaf(wf * (1.0f - d1 * ir), ldg(row + ib + 1), acc);
                    } else {
                        // bins k with |k - t| < r: k = ib - m (distance fr + m) and ib + 1 + m (1 - fr + m)
                        for (int m = 0; (float)m < r; ++m) {
                            const float d0 = fr + (float)m, d1 = 1.0f - fr + (float)m;
                            const int k0 = ib - m, k1 = ib + 1 + m;
                            if (d0 < r && k0 >= 0 && k0 < nb) acc = fmaf(wf * (1.0f - d0 * ir), ldg(row + k0), acc);
                            if (d1 < r && k1 >= 0 && k1 < nb) acc = fmaf(wf * (1.0f - d1 * ir), ldg(row + k1), acc);
                        }
                    }
                } else {
                    const AngleParams &P = ang[ac + q];
                    const double tt = s_tb[q] + (double)di * P.tA + (double)dj * P.tB;
                    const double ff = floor(tt);
                    const int ib = (int)ff;
                    const double fr = tt - ff;
                    const double rd = P.rfoot_d, wf = P.wfoot_d;
                    for (int m = 0; (double)m < rd; ++m) {
                        const double d0 = fr + m, d1 = 1.0 - fr + m;
                        const int k0 = ib - m, k1 = ib + 1 + m;
                        if (d0 < rd && k0 >= 0 && k0 < nb) acc = fma(wf * (1.0 - d0 / rd), ldg(row + k0), acc);
                        if (d1 < rd && k1 >= 0 && k1 < nb) acc = fma(wf * (1.0 - d1 / rd), ldg(row + k1), acc);
                    }
                }
            }
        }
    }
    if (x < nx && y < ny) u[(long long)t * nx * ny + (long long)y * nx + x] = acc;
}

// FP32 form with BP_PX pixels per thread (x = x0 + di + 32 e, e < BP_PX: a 128 x 8 tile
// per CTA): the per-angle constants come from shared memory as two 16-byte records
// and are reused for the thread's pixels, and the tile origin's FP64 set-up is shared
// by four times as many pixels. Each pixel's bin coordinate and weights are those of
// k_backproject (the same split products); a pixel's sum over the angles is compensated
// (Kahan), so its rounding does not grow with the number of angles.
constexpr int BP_PX = 4;
struct __align__(16) BpAngle {
    float fb, tAh, tAl, tBh;
    float tBl, r, ir, wf;
};

__global__ void __launch_bounds__(BP_TX *BP_TY) k_backproject4(const float *__restrict__ b, float *__restrict__ u,
                                                               const AngleParams *__restrict__ ang,
                                                               const int *__restrict__ aoff, int nx, int ny, int nb, int t0) {
    __shared__ BpAngle s_a[BP_CHUNK];
    __shared__ int s_ib[BP_CHUNK];
    const int t = t0 + blockIdx.z;
    const int x0 = blockIdx.x * BP_TX * BP_PX, y0 = blockIdx.y * BP_TY;
    const int di = threadIdx.x, dj = threadIdx.y;
    const int y = y0 + dj;
    const int tid = threadIdx.y * BP_TX + threadIdx.x;
    const int a_begin = aoff[t], a_end = aoff[t + 1];
    float acc[BP_PX];
#pragma unroll
    for (int e = 0; e < BP_PX; ++e) acc[e] = 0.f;
    float cmp[BP_PX];
#pragma unroll
    for (int e = 0; e < BP_PX; ++e) cmp[e] = 0.f;
    for (int ac = a_begin; ac < a_end; ac += BP_CHUNK) {
        const int cn = min(BP_CHUNK, a_end - ac);
        __syncthreads();
        if (tid < cn) {
            const AngleParams &P = ang[ac + tid];
            const double tb = P.t0 + (double)x0 * P.tA + (double)y0 * P.tB;
            const double fl = floor(tb);
            s_ib[tid] = (int)fmax(fmin(fl, 1e9), -1e9);
            s_a[tid] = BpAngle{(float)(tb - fl), P.tA_hi, P.tA_lo, P.tB_hi, P.tB_lo, P.rfoot, P.inv_rfoot, P.wfoot};
        }
        __syncthreads();
        if (y < ny) {
            for (int q = 0; q < cn; ++q) {
                const float *row = b + (long long)(ac + q) * nb;
                const BpAngle A = s_a[q];
                const int ib0 = s_ib[q];
                const float pb = (float)dj * A.tBh, pfb = floorf(pb);
                const float bl = (float)dj * A.tBl;
#pragma unroll
                for (int e = 0; e < BP_PX; ++e) {
                    const int dx = di + BP_TX * e;
                    if (x0 + dx >= nx) break;
                    const float pa = (float)dx * A.tAh, pfa = floorf(pa);
                    float fr = A.fb + (pa - pfa) + (pb - pfb) + fmaf((float)dx, A.tAl, bl);
                    const float ff = floorf(fr);
                    const int ib = ib0 + (int)pfa + (int)pfb + (int)ff;
                    fr -= ff;
                    if (A.r <= 1.0f) {  // at most the two bins around t
                        const float d1 = 1.0f - fr;
                        float tap = 0.f;
                        if (fr < A.r && ib >= 0 && ib < nb) tap = A.wf * (1.0f - fr * A.ir) * ldg(row + ib);
                        if (d1 < A.r && ib + 1 >= 0 && ib + 1 < nb) tap = fmaf(A.wf * (1.0f - d1 * A.ir), ldg(row + ib + 1), tap);
                        const float y = __fsub_rn(tap, cmp[e]), tt = __fadd_rn(acc[e], y);
                        cmp[e] = __fsub_rn(__fsub_rn(tt, acc[e]), y);
                        acc[e] = tt;
                    } else {
                        for (int m = 0; (float)m < A.r; ++m) {
                            const float d0 = fr + (float)m, d1 = 1.0f - fr + (float)m;
                            const int k0 = ib - m, k1 = ib + 1 + m;
                            if (d0 < A.r && k0 >= 0 && k0 < nb) acc[e] = fmaf(A.wf * (1.0f - d0 * A.ir), ldg(row + k0), acc[e]);
                            if (d1 < A.r && k1 >= 0 && k1 < nb) acc[e] = fmaf(A.wf * (1.0f - d1 * A.ir), ldg(row + k1), acc[e]);
                        }
                    }
                }
            }
        }
    }
    if (y < ny) {
#pragma unroll
        for (int e = 0; e < BP_PX; ++e) {
            const int x = x0 + di + BP_TX * e;
            if (x < nx) u[(long long)t * nx * ny + (long long)y * nx + x] = acc[e];
        }
    }
}

// ---------------------------------------------------------- K2 fan beam
// One thread per pixel. A ray steps over rows (or columns) and gives the pixel
// a weight only at the step of the pixel's row (column), when its crossing
// there is less than one pixel away; so the rays that reach the pixel are
// those crossing the open segments of half-length h through its centre along
// x and along y. Seen from the source, those segments cover the bins between
// the central projections of their four end points (widened by FAN_PAD bins
// for the FP32 evaluation of the bounds); for each such bin the forward entry
// is re-evaluated with the forward's own arithmetic. Steps the forward march
// skips have crossings more than a pixel outside the frame, so they cannot
// reach a pixel and need no test here.
constexpr float FAN_PAD = (float)FAN_PAD_BINS;

template <typename real>
__global__ void __launch_bounds__(BP_TX *BP_TY) k_backproject_fan(const real *__restrict__ b, real *__restrict__ u,
                                                                  const FanRay<real> *__restrict__ rays,
                                                                  const FanView *__restrict__ views,
                                                                  const int *__restrict__ aoff, int nx, int ny, int nb,
                                                                  float h, float scale) {
    const int t = blockIdx.z;
    const int x = blockIdx.x * BP_TX + threadIdx.x, y = blockIdx.y * BP_TY + threadIdx.y;
    if (x >= nx || y >= ny) return;
    const float toff = 0.5f * (float)(nb - 1);
    real acc = 0;
    for (int a = aoff[t]; a < aoff[t + 1]; ++a) {
        const FanView V = views[a];
        const float qx = fmaf((float)x, h, V.qx0), qy = fmaf((float)y, h, V.qy0);
        const float num = qx * V.fx + qy * V.fy, den = qx * V.ex + qy * V.ey;
        const float nxp = h * V.fx, dxp = h * V.ex, nyp = h * V.fy, dyp = h * V.ey;
        const float t0 = __fdividef(num + nxp, den + dxp), t1 = __fdividef(num - nxp, den - dxp);
        const float t2 = __fdividef(num + nyp, den + dyp), t3 = __fdividef(num - nyp, den - dyp);
        const float tlo = fminf(fminf(t0, t1), fminf(t2, t3)), thi = fmaxf(fmaxf(t0, t1), fmaxf(t2, t3));
        // clamped in floating point before the conversion (a non-finite bound gives no bins)
        const int klo = (int)fminf(fmaxf(ceilf(fmaf(tlo, scale, toff - FAN_PAD)), 0.0f), (float)nb);
        const int khi = (int)fminf(fmaxf(floorf(fmaf(thi, scale, toff + FAN_PAD)), -1.0f), (float)(nb - 1));
        const FanRay<real> *ra = rays + (long long)a * nb;
        const real *row = b + (long long)a * nb;
        for (int k = klo; k <= khi; ++k) {
            const FanRay<real> R = ra[k];
            int i0, fast;
            real w1, wstep;
            if constexpr (sizeof(real) == 4) {
                const int rows = R.ibr & 1;
                const int j = rows ? y : x;
                fast = rows ? x : y;
                affine_frac(R.ibr >> 1, R.fb, R.df_hi, R.df_lo, j, i0, w1);
                const float df = R.df_hi + R.df_lo;
                wstep = h * sqrtf(fmaf(df, df, 1.0f));
            } else {
                const int j = R.rows ? y : x;
                fast = R.rows ? x : y;
                const double f = fma((double)j, R.df, R.f0), fl = floor(f);
                i0 = (int)fl;
                w1 = f - fl;
                wstep = R.wstep;
            }
            const real w = i0 == fast ? (real)1 - w1 : (i0 + 1 == fast ? w1 : (real)0);
            if (w != (real)0) acc = fma(w * wstep, ldg(row + k), acc);
        }
    }
    u[(long long)t * nx * ny + (long long)y * nx + x] = acc;
}

template <typename real>
mof_status launch_backproject(const mof_problem *p, const real *b, real *u, cudaStream_t st, bool per_frame) {
    dim3 grid((p->nx + BP_TX - 1) / BP_TX, (p->ny + BP_TY - 1) / BP_TY, p->nt);
    if (p->fan) {
        ::mof::count_launch(), k_backproject_fan<real><<<grid, dim3(BP_TX, BP_TY), 0, st>>>(
            b, u, static_cast<const FanRay<real> *>(p->d_fanray), p->d_fanview, p->d_aoff, p->nx, p->ny, p->nb,
            (float)p->h, p->fan_scale);
        MOF_LAUNCH_CHECK();
        return MOF_OK;
    }
    // the plain form launches one frame at a time (t0 = t, one z slice), else all frames
    const int nlaunch = per_frame ? p->nt : 1, nz = per_frame ? 1 : p->nt;
    for (int t0 = 0; t0 < nlaunch; ++t0) {
        if (sizeof(real) == 4) {
            dim3 g4((p->nx + BP_TX * BP_PX - 1) / (BP_TX * BP_PX), (p->ny + BP_TY - 1) / BP_TY, nz);
            ::mof::count_launch(), k_backproject4<<<g4, dim3(BP_TX, BP_TY), 0, st>>>((const float *)b, (float *)u, p->d_ang,
                                                                                     p->d_aoff, p->nx, p->ny, p->nb, t0);
        } else {
            dim3 g1(grid.x, grid.y, nz);
            ::mof::count_launch(), k_backproject<real><<<g1, dim3(BP_TX, BP_TY), 0, st>>>(b, u, p->d_ang, p->d_aoff, p->nx, p->ny,
                                                                                         p->nb, t0);
        }
    }
    MOF_LAUNCH_CHECK();
    return MOF_OK;
}

template mof_status launch_project<float>(const mof_problem *, const float *, float *, float *, cudaStream_t, bool);
template mof_status launch_project<double>(const mof_problem *, const double *, double *, double *, cudaStream_t, bool);
template mof_status launch_backproject<float>(const mof_problem *, const float *, float *, cudaStream_t, bool);
template mof_status launch_backproject<double>(const mof_problem *, const double *, double *, cudaStream_t, bool);

}  // namespace mof
