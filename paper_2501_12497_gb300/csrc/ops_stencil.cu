// Stencil and flow operators of MMGKS-OF:
//   K3  Psi / Psi^T            forward differences of every frame (eq. (L))
//   K4  Mhat / Mhat^T          bilinear temporal warp rows (Sec. 3, Sec. 4)
//   K5  Theta^T W Theta        IRLS-weighted regulariser normal operator (Alg. 1)
//   K6  reverse flow           s' from s (remark of Sec. 3)
//   K7  App. C derivative fields u_x, u_y, u_t
//   K8  Upsilon s + u_t, Upsilon^T r (Sec. 2.2)
//
// The transposes of the warp (and the reverse flow) are computed per output tile
// from the sources that can reach it: every velocity field carries, per source tile,
// the bounds of its pixels' integer displacements and, for the whole field, the
// largest reach, so a destination tile visits only the rows and columns of the
// neighbouring source tiles whose footprints can fall into it (the only global
// atomics: one integer maximum per source tile for the field's reach). Mhat^T and
// Theta^T W Theta scatter the sources' weighted values into
// the tile in exact 64-bit fixed point (order independent, so repeated runs are
// bit-identical); the reverse flow averages the arrivals of each pixel in row-major
// source order.
#include "common.cuh"

#include <algorithm>

#include <cfloat>
#include <climits>

namespace mof {

namespace {

constexpr int TX = 32, TY = 8;

inline dim3 grid2d(int nx, int ny, int nz) { return dim3((nx + TX - 1) / TX, (ny + TY - 1) / TY, nz); }

// Sample coordinate of M(s) along one axis (Sec. 3). wm = 0, bilinear: X =
// clamp(x + v, 0, n - 1), i0 = floor(X), i1 = min(i0 + 1, n - 1), w = X - i0;
// the fraction is taken from v itself (v - floor(v) is exact), so the weights
// do not lose bits to the magnitude of x. wm = 1, rounding and clipping: i0 =
// clamp(x + round(v), 0, n - 1) with halves rounded away from zero, w = 0.
template <typename real>
__device__ __forceinline__ void warp_axis(int x, real v, int n, int &i0, int &i1, real &w, int wm) {
    const real vc = v > (real)16777216 ? (real)16777216 : (v < (real)-16777216 ? (real)-16777216 : v);
    const real fv = floor(vc);
    const int I = x + (int)fv;
    if (wm) {
        i0 = min(max(x + (int)round(vc), 0), n - 1); w = 0;
    } else if (I < 0) {
        i0 = 0; w = 0;
    } else if (I >= n - 1) {
        i0 = n - 1; w = 0;
    } else {
        i0 = I; w = vc - fv;
    }
    if (!(v == v)) { i0 = x; w = 0; }  // NaN velocity: identity sample (flagged elsewhere)
    i1 = min(i0 + 1, n - 1);
}

template <typename real>
__device__ __forceinline__ real bilinear(const real *__restrict__ f, int nx, int ny, int x, int y, real vx, real vy, int wm) {
    int x0, x1, y0, y1;
    real wx, wy;
    warp_axis(x, vx, nx, x0, x1, wx, wm);
    warp_axis(y, vy, ny, y0, y1, wy, wm);
    const real a = ldg(f + (long long)y0 * nx + x0), b = ldg(f + (long long)y0 * nx + x1);
    const real c = ldg(f + (long long)y1 * nx + x0), d = ldg(f + (long long)y1 * nx + x1);
    const real top = (1 - wx) * a + wx * b, bot = (1 - wx) * c + wx * d;
    return (1 - wy) * top + wy * bot;
}

// Destination of a source pixel under the reverse flow (remark of Sec. 3), one axis:
// round half away from zero of x + v, clipped. With v = fv + fr (fv = floor(v), fr in
// [0,1) exact) and I = x + fv: for I >= 0 the position is >= 0 and rounds up iff
// fr >= 1/2; for I < 0 it is negative and rounds up (towards zero) iff fr > 1/2. This
// takes the decision exactly, as an FP64 evaluation of x + v would.
template <typename real>
__device__ __forceinline__ int round_axis(int x, real v, int n) {
    const real vc = v > (real)16777216 ? (real)16777216 : (v < (real)-16777216 ? (real)-16777216 : v);
    const real fv = floor(vc);
    const real fr = vc - fv;
    int I = x + (int)fv;
    if (I >= 0) I += (fr >= (real)0.5) ? 1 : 0;
    else I += (fr > (real)0.5) ? 1 : 0;
    if (!(v == v)) I = x;
    return I < 0 ? 0 : (I > n - 1 ? n - 1 : I);
}

// ---------------------------------------------------------------- tiles of the transposes
// The warp transposes (Mhat^T, the flow part of Theta^T W Theta) and the reverse flow
// work on BW x BH pixel tiles, one CTA of BT threads per tile (BPT pixels per thread).
// For every velocity field the source tiles carry the bounds of the integer
// displacements of their pixels (x0(p) - px, y0(p) - py: the first pixel of the
// footprint, or the destination), and the field carries its reach: the largest
// distance between a source and any pixel of its footprint. A destination tile then
// finds every source that can reach it among the source tiles within the reach, each
// restricted to the rows and columns its own bounds allow.
constexpr int BW = 64, BH = 16, BT = 256, BPT = BW * BH / BT;

// Exact fixed-point accumulation of the terms of one output pixel: every term is scaled
// by 2^E, chosen per tile so that the sum of all terms of a pixel stays below 2^62 in
// magnitude, rounded to an integer and added into a 64-bit integer. Integer addition is
// associative, so the result is independent of the order in which the terms arrive
// (deterministic); the roundings are the terms' own (at 2^-E, far below the precision
// of the inputs) and the final conversion. An FP32 term is rounded with the FP32 adder
// (the 1.5 * 2^23 magic constant) in three exact 22-bit pieces: conversions between
// 64-bit integers and floating point run on the FP64 pipe, which this GPU runs at a
// small fraction of its FP32 rate.
__device__ __forceinline__ long long fx_term(float x) {  // round(x) for |x| < 2^62
    const float MAG = 12582912.0f;                      // 1.5 * 2^23
    const float h2 = (x * 5.684341886080802e-14f + MAG) - MAG;  // round(x / 2^44), |.| < 2^18
    const float r1 = fmaf(-h2, 17592186044416.0f, x);           // exact, |.| <= 2^43
    const float h1 = (r1 * 2.384185791015625e-07f + MAG) - MAG; // round(r1 / 2^22), |.| <= 2^21
    const float r0 = fmaf(-h1, 4194304.0f, r1);                 // exact, |.| <= 2^21
    const long long a = __float_as_int(h2 + MAG) - 0x4B400000, b = __float_as_int(h1 + MAG) - 0x4B400000;
    const long long c = __float_as_int(r0 + MAG) - 0x4B400000;
    return (a << 44) + (b << 22) + c;
}
__device__ __forceinline__ long long fx_term(double x) { return __double2ll_rn(x); }
// 2^E as the element type (E within the normal range of the type)
__device__ __forceinline__ void fx_pow2(int E, float &sc) { sc = __int_as_float((E + 127) << 23); }
__device__ __forceinline__ void fx_pow2(int E, double &sc) { sc = __longlong_as_double((long long)(E + 1023) << 52); }
// tot * 2^-E * f. FP32: the integer in three 22-bit pieces, each turned into a float by the
// magic constant (exact), combined by two FMAs (within an ulp), then two exact power-of-two
// factors and f; FP64 directly.
__device__ __forceinline__ float fx_out(long long tot, int E, float f) {
    const unsigned long long u = (unsigned long long)tot;
    const int c = (int)(u & 0x3fffffull), b = (int)((u >> 22) & 0x3fffffull);
    const int a = (int)(tot >> 44);  // signed, |a| < 2^19
    const float MAG = 12582912.0f;
    const float fc = __int_as_float(0x4B400000 + c) - MAG, fb = __int_as_float(0x4B400000 + b) - MAG;
    const float fa = __int_as_float(0x4B400000 + a) - MAG;
    const float v = fmaf(fa, 17592186044416.0f, fmaf(fb, 4194304.0f, fc));
    const int e1 = E / 2, e2 = E - E / 2;
    return v * __int_as_float((127 - e1) << 23) * __int_as_float((127 - e2) << 23) * f;
}
__device__ __forceinline__ double fx_out(long long tot, int E, double f) {
    return (double)tot * __longlong_as_double((long long)(1023 - E) << 52) * f;
}
// scale exponent E of a tile whose largest term is below 2^ex and whose pixels receive at
// most cb terms each
template <typename real>
__device__ __forceinline__ int fx_exponent(int ex, long long cb) { return 62 - (64 - __clzll(cb - 1)) - ex; }
// bit pattern of |v| (ordered like the magnitudes; non-finite values above every finite one)
__device__ __forceinline__ unsigned long long abs_bits(float v) { return (unsigned long long)(__float_as_uint(v) & 0x7fffffffu); }
__device__ __forceinline__ unsigned long long abs_bits(double v) {
    return (unsigned long long)__double_as_longlong(v) & 0x7fffffffffffffffull;
}
__device__ __forceinline__ bool bits_finite(unsigned long long b, float) { return b < 0x7f800000ull; }
__device__ __forceinline__ bool bits_finite(unsigned long long b, double) { return b < 0x7ff0000000000000ull; }
// exponent ex with |v| < 2^ex for the magnitude whose bits are b (b > 0, finite)
__device__ __forceinline__ int bits_exp(unsigned long long b, float) {
    int ex = 0;
    frexpf(__uint_as_float((unsigned)b), &ex);
    return ex;
}
__device__ __forceinline__ int bits_exp(unsigned long long b, double) {
    int ex = 0;
    frexp(__longlong_as_double((long long)b), &ex);
    return ex;
}
template <typename real> struct FxLimits;
template <> struct FxLimits<float> { static constexpr int EMAX = 126, EMIN = -126; };
template <> struct FxLimits<double> { static constexpr int EMAX = 1000, EMIN = -1000; };

// A rectangle of candidate source pixels of one destination tile: w columns from x0,
// rows from y0, its pixels numbered from `start` in the tile's flat candidate list;
// magic = ceil(2^64 / w) turns a pixel's number into its row with one multiply-high.
struct SrcRect {
    int x0, y0, w, start;
    unsigned long long magic;
    int term, pad_;
};
constexpr int MAXR = 64;  // rectangles per round of a destination tile

}  // namespace

// =================================================================== K3 Psi
template <typename real>
__global__ void k_grad(const real *__restrict__ u, real *__restrict__ g, int nx, int ny) {
    const int x = blockIdx.x * TX + threadIdx.x, y = blockIdx.y * TY + threadIdx.y, t = blockIdx.z;
    if (x >= nx || y >= ny) return;
    const long long ns = (long long)nx * ny, i = (long long)y * nx + x;
    const real *f = u + t * ns;
    const real c = f[i];
    g[(2LL * t) * ns + i] = (x < nx - 1) ? f[i + 1] - c : (real)0;
    g[(2LL * t + 1) * ns + i] = (y < ny - 1) ? f[i + nx] - c : (real)0;
}

template <typename real>
__global__ void k_gradT(const real *__restrict__ g, real *__restrict__ u, int nx, int ny) {
    const int x = blockIdx.x * TX + threadIdx.x, y = blockIdx.y * TY + threadIdx.y, t = blockIdx.z;
    if (x >= nx || y >= ny) return;
    const long long ns = (long long)nx * ny, i = (long long)y * nx + x;
    const real *gx = g + (2LL * t) * ns, *gy = g + (2LL * t + 1) * ns;
    real v = 0;
    if (x > 0) v += gx[i - 1];
    if (x < nx - 1) v -= gx[i];
    if (y > 0) v += gy[i - nx];
    if (y < ny - 1) v -= gy[i];
    u[t * ns + i] = v;
}

// FP32 forms with four consecutive pixels per thread (16-byte loads and stores of rows
// whose length is a multiple of 4, buffers 16-byte aligned): the same subtractions in the
// same order per pixel as k_grad / k_gradT, so the results are identical.
constexpr int V4X = 64, V4Y = 4;  // threads per block: 64 x 4 (256 pixels of a row per warp pair)
__device__ __forceinline__ float4 ld4(const float *p) { return *reinterpret_cast<const float4 *>(p); }
__device__ __forceinline__ void st4(float *p, float4 v) { *reinterpret_cast<float4 *>(p) = v; }
__device__ __forceinline__ float4 ldcs4(const float *p) { return __ldcs(reinterpret_cast<const float4 *>(p)); }
__device__ __forceinline__ void stcs4(float *p, float4 v) { __stcs(reinterpret_cast<float4 *>(p), v); }
inline dim3 grid4(int nx, int ny, int nz) { return dim3((nx / 4 + V4X - 1) / V4X, (ny + V4Y - 1) / V4Y, nz); }
inline bool al16(const void *p) { return (reinterpret_cast<uintptr_t>(p) & 15) == 0; }

__global__ void __launch_bounds__(V4X *V4Y) k_grad4(const float *__restrict__ u, float *__restrict__ g, int nx, int ny) {
    const int x = 4 * (blockIdx.x * V4X + threadIdx.x), y = blockIdx.y * V4Y + threadIdx.y, t = blockIdx.z;
    if (x >= nx || y >= ny) return;
    const long long ns = (long long)nx * ny, i = (long long)y * nx + x;
    const float *f = u + t * ns;
    const float4 c = ld4(f + i);
    const float e = (x + 4 < nx) ? f[i + 4] : 0.f;
    float4 gx, gy;
    gx.x = c.y - c.x;
    gx.y = c.z - c.y;
    gx.z = c.w - c.z;
    gx.w = (x + 4 < nx) ? e - c.w : 0.f;
    if (y < ny - 1) {
        const float4 d = ld4(f + i + nx);
        gy = make_float4(d.x - c.x, d.y - c.y, d.z - c.z, d.w - c.w);
    } else {
        gy = make_float4(0.f, 0.f, 0.f, 0.f);
    }
    stcs4(g + (2LL * t) * ns + i, gx);
    stcs4(g + (2LL * t + 1) * ns + i, gy);
}

__global__ void __launch_bounds__(V4X *V4Y) k_gradT4(const float *__restrict__ g, float *__restrict__ u, int nx, int ny) {
    const int x = 4 * (blockIdx.x * V4X + threadIdx.x), y = blockIdx.y * V4Y + threadIdx.y, t = blockIdx.z;
    if (x >= nx || y >= ny) return;
    const long long ns = (long long)nx * ny, i = (long long)y * nx + x;
    const float *gx = g + (2LL * t) * ns, *gy = g + (2LL * t + 1) * ns;
    const float4 a = ld4(gx + i), c = ld4(gy + i);
    const float al = x > 0 ? gx[i - 1] : 0.f;
    const float4 cu = y > 0 ? ld4(gy + i - nx) : make_float4(0.f, 0.f, 0.f, 0.f);
    const float gxa[4] = {a.x, a.y, a.z, a.w}, gya[4] = {c.x, c.y, c.z, c.w}, gyu[4] = {cu.x, cu.y, cu.z, cu.w};
    float o[4];
#pragma unroll
    for (int k = 0; k < 4; ++k) {
        float v = 0.f;
        if (x + k > 0) v += k == 0 ? al : gxa[k - 1];
        if (x + k < nx - 1) v -= gxa[k];
        if (y > 0) v += gyu[k];
        if (y < ny - 1) v -= gya[k];
        o[k] = v;
    }
    stcs4(u + t * ns + i, make_float4(o[0], o[1], o[2], o[3]));
}

template <typename real>
mof_status launch_grad(const mof_problem *p, int nf, const real *u, real *g, cudaStream_t st) {
    if (sizeof(real) == 4 && p->nx % 4 == 0 && al16(u) && al16(g))
        ::mof::count_launch(), k_grad4<<<grid4(p->nx, p->ny, nf), dim3(V4X, V4Y), 0, st>>>((const float *)u, (float *)g, p->nx, p->ny);
    else
        ::mof::count_launch(), k_grad<real><<<grid2d(p->nx, p->ny, nf), dim3(TX, TY), 0, st>>>(u, g, p->nx, p->ny);
    MOF_LAUNCH_CHECK();
    return MOF_OK;
}
template <typename real>
mof_status launch_gradT(const mof_problem *p, int nf, const real *g, real *u, cudaStream_t st) {
    if (sizeof(real) == 4 && p->nx % 4 == 0 && al16(u) && al16(g))
        ::mof::count_launch(), k_gradT4<<<grid4(p->nx, p->ny, nf), dim3(V4X, V4Y), 0, st>>>((const float *)g, (float *)u, p->nx, p->ny);
    else
        ::mof::count_launch(), k_gradT<real><<<grid2d(p->nx, p->ny, nf), dim3(TX, TY), 0, st>>>(g, u, p->nx, p->ny);
    MOF_LAUNCH_CHECK();
    return MOF_OK;
}

// ================================================================= K4 Mhat
template <typename real>
__global__ void k_flow(const real *__restrict__ u, const real *__restrict__ s, const real *__restrict__ sr,
                       real *__restrict__ r, int nx, int ny, int np, int wm) {
    const int x = blockIdx.x * TX + threadIdx.x, y = blockIdx.y * TY + threadIdx.y, p = blockIdx.z;
    if (x >= nx || y >= ny) return;
    const long long ns = (long long)nx * ny, i = (long long)y * nx + x;
    const real *u0 = u + p * ns, *u1 = u0 + ns;
    const real *sp = s + 2LL * p * ns, *srp = sr + 2LL * p * ns;
    r[p * ns + i] = u0[i] - bilinear(u1, nx, ny, x, y, sp[i], sp[ns + i], wm);
    r[(np + p) * ns + i] = u1[i] - bilinear(u0, nx, ny, x, y, srp[i], srp[ns + i], wm);
}

// FP32 form of k_flow with four consecutive pixels per thread: the streamed arrays (u_t,
// u_{t+1}, s, s', both residual rows) move as 16-byte vectors, the bilinear samples are
// gathered per pixel with the same arithmetic (identical results).
__global__ void __launch_bounds__(V4X *V4Y) k_flow4(const float *__restrict__ u, const float *__restrict__ s,
                                                   const float *__restrict__ sr, float *__restrict__ r, int nx, int ny,
                                                   int np, int wm) {
    const int x = 4 * (blockIdx.x * V4X + threadIdx.x), y = blockIdx.y * V4Y + threadIdx.y, p = blockIdx.z;
    if (x >= nx || y >= ny) return;
    const long long ns = (long long)nx * ny, i = (long long)y * nx + x;
    const float *u0 = u + p * ns, *u1 = u0 + ns;
    const float *sp = s + 2LL * p * ns, *srp = sr + 2LL * p * ns;
    const float4 a0 = ld4(u0 + i), a1 = ld4(u1 + i);
    const float4 svx = ldcs4(sp + i), svy = ldcs4(sp + ns + i), rvx = ldcs4(srp + i), rvy = ldcs4(srp + ns + i);
    const float A0[4] = {a0.x, a0.y, a0.z, a0.w}, A1[4] = {a1.x, a1.y, a1.z, a1.w};
    const float SX[4] = {svx.x, svx.y, svx.z, svx.w}, SY[4] = {svy.x, svy.y, svy.z, svy.w};
    const float RX[4] = {rvx.x, rvx.y, rvx.z, rvx.w}, RY[4] = {rvy.x, rvy.y, rvy.z, rvy.w};
    float f[4], b[4];
#pragma unroll
    for (int k = 0; k < 4; ++k) {
        f[k] = A0[k] - bilinear(u1, nx, ny, x + k, y, SX[k], SY[k], wm);
        b[k] = A1[k] - bilinear(u0, nx, ny, x + k, y, RX[k], RY[k], wm);
    }
    stcs4(r + p * ns + i, make_float4(f[0], f[1], f[2], f[3]));
    stcs4(r + (np + p) * ns + i, make_float4(b[0], b[1], b[2], b[3]));
}

template <typename real>
mof_status launch_flow(const mof_problem *p, const real *u, const real *s, const real *sr, real *r, cudaStream_t st) {
    const int np = p->nt - 1;
    if (np <= 0) return MOF_OK;
    if (sizeof(real) == 4 && p->nx % 4 == 0 && al16(u) && al16(s) && al16(sr) && al16(r))
        ::mof::count_launch(), k_flow4<<<grid4(p->nx, p->ny, np), dim3(V4X, V4Y), 0, st>>>(
            (const float *)u, (const float *)s, (const float *)sr, (float *)r, p->nx, p->ny, np, p->warp_mode);
    else
        ::mof::count_launch(), k_flow<real><<<grid2d(p->nx, p->ny, np), dim3(TX, TY), 0, st>>>(u, s, sr, r, p->nx, p->ny, np, p->warp_mode);
    MOF_LAUNCH_CHECK();
    return MOF_OK;
}

// ------------------------------------------------------------ K4/K5/K6 source-tile bounds
int tiles_x(const mof_problem *p) { return (p->nx + BW - 1) / BW; }
int tiles_count(const mof_problem *p) { return tiles_x(p) * ((p->ny + BH - 1) / BH); }
// per velocity field: one int4 per source tile, then one int4 {Rx, Ry, 0, 0}, the reach
long long tile_bound_ints(const mof_problem *p) { return 4LL * (tiles_count(p) + 1); }

// reach of every field to zero (the bounds kernels raise it with integer maxima)
__global__ void k_zero_reach(int *__restrict__ bnd_a, int *__restrict__ bnd_b, int nf, int tiles) {
    const int f = blockIdx.x * blockDim.x + threadIdx.x;
    if (f >= 2 * nf) return;
    int *b = f < nf ? bnd_a : bnd_b;
    if (!b) return;
    reinterpret_cast<int4 *>(b)[(long long)(f % nf) * (tiles + 1) + tiles] = make_int4(0, 0, 0, 0);
}

// Bounds of one source tile of velocity field f (fields f < nf from va, the next nf
// from vb): {min, max} over its pixels p of x0(p) - px and y0(p) - py, with x0, y0 the
// first pixel of the bilinear footprint {x0, x0 or x0 + 1} of M(v) (MODE 0), or the
// reverse flow's destination (MODE 1, which also stores it in dest). The field's reach
// max(-min, max + 1) (MODE 0; max(-min, max) in MODE 1) is raised with one integer
// atomicMax per tile and axis (exact and order independent).
template <typename real, int MODE>
__global__ void __launch_bounds__(BT) k_src_bounds(const real *__restrict__ va, const real *__restrict__ vb, int nf, int nx,
                                                   int ny, int wm, int *__restrict__ bnd_a, int *__restrict__ bnd_b, int tiles_x,
                                                   int tiles, int *__restrict__ dest) {
    const int fz = blockIdx.z, f = fz % nf;
    const real *v = fz < nf ? va : vb;
    int *bnd = fz < nf ? bnd_a : bnd_b;
    const long long ns = (long long)nx * ny;
    const real *vx = v + 2LL * f * ns, *vy = vx + ns;
    int dxmin = INT_MAX, dxmax = INT_MIN, dymin = INT_MAX, dymax = INT_MIN;
#pragma unroll
    for (int k = 0; k < BPT; ++k) {
        const int l = threadIdx.x + k * BT;
        const int x = blockIdx.x * BW + (l % BW), y = blockIdx.y * BH + l / BW;
        if (x >= nx || y >= ny) continue;
        const long long i = (long long)y * nx + x;
        int dx, dy;
        if (MODE == 0) {
            int x0, x1, y0, y1;
            real wx, wy;
            warp_axis(x, vx[i], nx, x0, x1, wx, wm);
            warp_axis(y, vy[i], ny, y0, y1, wy, wm);
            dx = x0 - x;
            dy = y0 - y;
        } else {
            const int qx = round_axis(x, vx[i], nx), qy = round_axis(y, vy[i], ny);
            dest[(long long)f * ns + i] = qy * nx + qx;
            dx = qx - x;
            dy = qy - y;
        }
        dxmin = min(dxmin, dx);
        dxmax = max(dxmax, dx);
        dymin = min(dymin, dy);
        dymax = max(dymax, dy);
    }
    dxmin = __reduce_min_sync(0xffffffffu, dxmin);
    dxmax = __reduce_max_sync(0xffffffffu, dxmax);
    dymin = __reduce_min_sync(0xffffffffu, dymin);
    dymax = __reduce_max_sync(0xffffffffu, dymax);
    __shared__ int red[BT / 32][4];
    const int w = threadIdx.x >> 5;
    if ((threadIdx.x & 31) == 0) {
        red[w][0] = dxmin;
        red[w][1] = dxmax;
        red[w][2] = dymin;
        red[w][3] = dymax;
    }
    __syncthreads();
    if (threadIdx.x == 0) {
        for (int j = 1; j < BT / 32; ++j) {
            dxmin = min(dxmin, red[j][0]);
            dxmax = max(dxmax, red[j][1]);
            dymin = min(dymin, red[j][2]);
            dymax = max(dymax, red[j][3]);
        }
        const int tile = blockIdx.y * tiles_x + blockIdx.x;
        int4 *b4 = reinterpret_cast<int4 *>(bnd) + (long long)f * (tiles + 1);
        b4[tile] = make_int4(dxmin, dxmax, dymin, dymax);
        const int ext = MODE == 0 ? 1 : 0;
        int *reach = reinterpret_cast<int *>(b4 + tiles);
        atomicMax(reach, max(-dxmin, dxmax + ext));
        atomicMax(reach + 1, max(-dymin, dymax + ext));
    }
}

inline dim3 grid_tiles(const mof_problem *p, int nz) { return dim3(tiles_x(p), (p->ny + BH - 1) / BH, nz); }

template <typename real>
mof_status launch_tile_bounds(const mof_problem *p, const real *s, const real *sr, int *bnd_s, int *bnd_sr, cudaStream_t st) {
    const int np = p->nt - 1, tiles = tiles_count(p);
    if (np <= 0) return MOF_OK;
    ::mof::count_launch(), k_zero_reach<<<(2 * np + 127) / 128, 128, 0, st>>>(bnd_s, sr ? bnd_sr : nullptr, np, tiles);
    MOF_LAUNCH_CHECK();
    ::mof::count_launch(), k_src_bounds<real, 0><<<grid_tiles(p, sr ? 2 * np : np), BT, 0, st>>>(
        s, sr, np, p->nx, p->ny, p->warp_mode, bnd_s, bnd_sr, tiles_x(p), tiles, nullptr);
    MOF_LAUNCH_CHECK();
    return MOF_OK;
}

// Warp 0 of a destination tile [X0, X1] x [Y0, Y1] appends to rect[] the candidate
// rectangles of the velocity fields' source tiles, numbered c in [cursor, nc0 + nc1)
// (the candidate tiles of term 0, then of term 1), until the list is full or the tiles
// are exhausted; MODE 0 (bilinear footprints) or MODE 1 (single destinations). Writes the
// number of rectangles and of their pixels and the next cursor to sh[0..2].
struct TermTiles {
    const int4 *bnd;  // the field's source-tile bounds (its reach after them)
    int txa, tya, ntx, nc;
};

__device__ __forceinline__ TermTiles term_tiles(const int *bnd_f, int tiles, int tiles_xn, int tiles_yn, int X0, int X1, int Y0,
                                                int Y1, int nx, int ny) {
    TermTiles T;
    T.bnd = reinterpret_cast<const int4 *>(bnd_f);
    const int4 R = __ldg(T.bnd + tiles);
    const int txa = max(0, X0 - R.x) / BW, txb = min(nx - 1, X1 + R.x) / BW;
    const int tya = max(0, Y0 - R.y) / BH, tyb = min(ny - 1, Y1 + R.y) / BH;
    T.txa = txa;
    T.tya = tya;
    T.ntx = min(txb, tiles_xn - 1) - txa + 1;
    T.nc = T.ntx * (min(tyb, tiles_yn - 1) - tya + 1);
    return T;
}

template <int MODE>
__device__ void build_rects(const TermTiles &T0, const TermTiles &T1, int cursor, int X0, int X1, int Y0, int Y1, int nx,
                            int ny, SrcRect *rect, int *sh) {
    const int lane = threadIdx.x & 31;
    const int total = T0.nc + T1.nc, ext = MODE == 0 ? 1 : 0;
    int cnt = 0, npx = 0;
    while (cursor < total && cnt <= MAXR - 32) {
        const int c = cursor + lane;
        bool valid = false;
        int rx0 = 0, ry0 = 0, w = 0, h = 0, term = 0;
        if (c < total) {
            term = c < T0.nc ? 0 : 1;
            const TermTiles &T = term ? T1 : T0;
            const int j = term ? c - T0.nc : c;
            const int tx = T.txa + j % T.ntx, ty = T.tya + j / T.ntx;
            const int4 b = __ldg(T.bnd + ty * ((nx + BW - 1) / BW) + tx);
            const int S0 = tx * BW, S1 = min(S0 + BW - 1, nx - 1), R0 = ty * BH, R1 = min(R0 + BH - 1, ny - 1);
            rx0 = max(S0, X0 - ext - b.y);
            const int rx1 = min(S1, X1 - b.x);
            ry0 = max(R0, Y0 - ext - b.w);
            const int ry1 = min(R1, Y1 - b.z);
            w = rx1 - rx0 + 1;
            h = ry1 - ry0 + 1;
            valid = w > 0 && h > 0;
        }
        const unsigned m = __ballot_sync(0xffffffffu, valid);
        const int mine = valid ? w * h : 0;
        int incl = mine;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            const int t = __shfl_up_sync(0xffffffffu, incl, o);
            if (lane >= o) incl += t;
        }
        if (valid) {
            SrcRect &R = rect[cnt + __popc(m & ((1u << lane) - 1u))];
            R.x0 = rx0;
            R.y0 = ry0;
            R.w = w;
            R.start = npx + incl - mine;
            R.magic = w > 1 ? (~0ull) / (unsigned long long)w + 1ull : 0ull;
            R.term = term;
        }
        cnt += __popc(m);
        npx += __shfl_sync(0xffffffffu, incl, 31);
        cursor += 32;
    }
    if (lane == 0) {
        sh[0] = cnt;
        sh[1] = npx;
        sh[2] = cursor;
    }
}

// pixel number k of the current round -> (term, px, py); r is the caller's running rectangle
// index (k only grows within a thread, so the search resumes where it stopped)
__device__ __forceinline__ void rect_pixel(const SrcRect *rect, int nrect, int k, int &r, int &term, int &px, int &py) {
    while (r + 1 < nrect && rect[r + 1].start <= k) ++r;
    const SrcRect &R = rect[r];
    const unsigned long long loc = (unsigned long long)(k - R.start);
    const int row = R.magic ? (int)__umul64hi(loc, R.magic) : (int)loc;
    px = R.x0 + (int)loc - row * R.w;
    py = R.y0 + row;
    term = R.term;
}

// ------------------------------------------------------------ K4 Mhat^T, K5 Theta^T W Theta
// One CTA per BW x BH tile D of frame t computes
//   out_t = [t<P] r0_t + [t>0] r1_{t-1} - [t<P] M(sr_t)^T r1_t - [t>0] M(s_{t-1})^T r0_{t-1}
// (REGN: r holds the weighted flow rows, plus the weighted differences Psi^T w Psi x and,
// with `temporal`, L_t^T w_t L_t x, all times scale * lam, plus y_add) as a scatter into
// the tile: every source p whose bilinear footprint can touch D (the candidate rectangles
// of the two velocity fields) adds w * r(p) to the pixels of its footprint inside D. The
// terms are summed exactly in 64-bit fixed point (shared-memory integer atomics), so the
// result does not depend on the order of the additions. Pass 0 finds the largest term
// magnitude of the tile (it sets the fixed-point scale), pass 1 scatters. A non-finite
// term makes the tile's outputs NaN.
template <typename real, bool REGN>
__global__ void __launch_bounds__(BT) k_warpT_tile(const real *__restrict__ r, const real *__restrict__ s,
                                                   const real *__restrict__ sr, const int *__restrict__ bnd_s,
                                                   const int *__restrict__ bnd_sr, int tiles, int nx, int ny, int np, int wm,
                                                   const real *__restrict__ x, const real *__restrict__ uk, real eps2,
                                                   double scale, const double *__restrict__ lam, const real *__restrict__ y_add,
                                                   int temporal, real *__restrict__ out) {
    __shared__ long long acc[BW * BH];
    __shared__ SrcRect rect[MAXR];
    __shared__ int sh[3];
    __shared__ unsigned long long s_max;
    __shared__ long long s_total;
    __shared__ real s_sc;  // scale * lam, once per block (FP64 kept out of the threads)
    const int t = blockIdx.z, tid = threadIdx.x;
    const int X0 = blockIdx.x * BW, Y0 = blockIdx.y * BH;
    const int X1 = min(X0 + BW - 1, nx - 1), Y1 = min(Y0 + BH - 1, ny - 1);
    const long long ns = (long long)nx * ny;
    const int txn = (nx + BW - 1) / BW, tyn = (ny + BH - 1) / BH;
    // term 0: rows r1 of pair t (sources on frame t+1, velocity sr_t); term 1: rows r0 of
    // pair t-1 (sources on frame t-1, velocity s_{t-1})
    TermTiles T0{nullptr, 0, 0, 1, 0}, T1{nullptr, 0, 0, 1, 0};
    if (t < np) T0 = term_tiles(bnd_sr + 4LL * t * (tiles + 1), tiles, txn, tyn, X0, X1, Y0, Y1, nx, ny);
    if (t > 0) T1 = term_tiles(bnd_s + 4LL * (t - 1) * (tiles + 1), tiles, txn, tyn, X0, X1, Y0, Y1, nx, ny);
    const real *val0 = r + (np + t) * ns, *val1 = r + (long long)(t - 1) * ns;
    const real *v0 = sr + 2LL * t * ns, *v1 = s + 2LL * (t - 1) * ns;
    for (int l = tid; l < BW * BH; l += BT) acc[l] = 0;
    if (tid == 0) {
        s_max = 0;
        s_total = 0;
        s_sc = REGN ? (real)(lam ? scale * *lam : scale) : (real)1;
    }

    // the pixel's own terms: the identity parts of Mhat^T and (REGN) the weighted differences
    constexpr int NOWN = REGN ? 8 : 2;
    real own[BPT][NOWN];
    unsigned long long mb = 0;
#pragma unroll
    for (int k = 0; k < BPT; ++k) {
        const int l = tid + k * BT, xx = X0 + (l % BW), yy = Y0 + l / BW;
#pragma unroll
        for (int e = 0; e < NOWN; ++e) own[k][e] = 0;
        if (xx > X1 || yy > Y1) continue;
        const long long i = (long long)yy * nx + xx;
        if (t < np) own[k][0] = r[t * ns + i];
        if (t > 0) own[k][1] = r[(np + t - 1) * ns + i];
        if (REGN) {
            const real *f = x + t * ns, *kk = uk + t * ns;
            auto wd = [&](const real *fa, const real *ka, long long j, long long step) -> real {
                const real g = fa[j + step] - fa[j], gk = ka[j + step] - ka[j];
                return g / sqrt(gk * gk + eps2);
            };
            if (xx > 0) own[k][2] = wd(f, kk, i - 1, 1);
            if (xx < nx - 1) own[k][3] = -wd(f, kk, i, 1);
            if (yy > 0) own[k][4] = wd(f, kk, i - nx, nx);
            if (yy < ny - 1) own[k][5] = -wd(f, kk, i, nx);
            if (temporal) {
                if (t > 0) own[k][6] = wd(f - ns, kk - ns, i, ns);
                if (t < np) own[k][7] = -wd(f, kk, i, ns);
            }
        }
#pragma unroll
        for (int e = 0; e < NOWN; ++e) mb = max(mb, abs_bits(own[k][e]));
    }

    real sc = 0;
    int E = 0;
    bool finite = true;
    for (int pass = 0; pass < 2; ++pass) {
        int cursor = 0;
        do {
            __syncthreads();  // the previous round's rectangles are consumed
            if (tid < 32) build_rects<0>(T0, T1, cursor, X0, X1, Y0, Y1, nx, ny, rect, sh);
            __syncthreads();
            const int nrect = sh[0], npx = sh[1];
            cursor = sh[2];
            if (pass == 0 && tid == 0) s_total += npx;
            int ri = 0;
            for (int k = tid; k < npx; k += BT) {
                int term, px, py;
                rect_pixel(rect, nrect, k, ri, term, px, py);
                const long long i = (long long)py * nx + px;
                const real val = term ? val1[i] : val0[i];
                if (pass == 0) {
                    mb = max(mb, abs_bits(val));
                    continue;
                }
                const real *vv = term ? v1 : v0;
                int x0, x1, y0, y1;
                real wx, wy;
                warp_axis(px, vv[i], nx, x0, x1, wx, wm);
                warp_axis(py, vv[ns + i], ny, y0, y1, wy, wm);
                // footprint corners with their axis weights (x1 == x0 only where the sample sits
                // on the last column, with wx = 0: one corner of weight (1 - wx) + wx); the
                // scaled value times the y weight, then times the x weight
                const bool xs = x1 == x0, ys = y1 == y0;
                const real ax0 = xs ? (1 - wx) + wx : 1 - wx, ay0 = ys ? (1 - wy) + wy : 1 - wy;
                const real vs = -(val * sc);
#pragma unroll
                for (int cy = 0; cy < 2; ++cy) {
                    const int yc = cy ? y1 : y0;
                    const real ay = cy ? wy : ay0;
                    if ((cy && ys) || yc < Y0 || yc > Y1 || ay == (real)0) continue;
                    const real vy = vs * ay;
#pragma unroll
                    for (int cx = 0; cx < 2; ++cx) {
                        const int xc = cx ? x1 : x0;
                        const real ax = cx ? wx : ax0;
                        if ((cx && xs) || xc < X0 || xc > X1 || ax == (real)0) continue;
                        atomicAdd(reinterpret_cast<unsigned long long *>(&acc[(yc - Y0) * BW + (xc - X0)]),
                                  (unsigned long long)fx_term(vy * ax));
                    }
                }
            }
        } while (cursor < T0.nc + T1.nc);
        if (pass == 0) {
            // the tile's largest magnitude (warp maximum of the 64-bit patterns in two 32-bit
            // halves, then the CTA maximum) and the fixed-point scale 2^E
            const unsigned hi = __reduce_max_sync(0xffffffffu, (unsigned)(mb >> 32));
            const unsigned lo = __reduce_max_sync(0xffffffffu, (unsigned)(mb >> 32) == hi ? (unsigned)mb : 0u);
            if ((tid & 31) == 0) atomicMax(&s_max, ((unsigned long long)hi << 32) | lo);
            __syncthreads();
            const unsigned long long M = s_max;
            finite = bits_finite(M, real(0));
            E = fx_exponent<real>(M ? bits_exp(M, real(0)) : 0, 4 * s_total + NOWN + 1);
            E = min(max(E, FxLimits<real>::EMIN), FxLimits<real>::EMAX);
            fx_pow2(E, sc);
            if (!finite) break;
        }
    }
    __syncthreads();
    const real f_out = s_sc;
#pragma unroll
    for (int k = 0; k < BPT; ++k) {
        const int l = tid + k * BT, xx = X0 + (l % BW), yy = Y0 + l / BW;
        if (xx > X1 || yy > Y1) continue;
        const long long o = t * ns + (long long)yy * nx + xx;
        long long tot = acc[l];
#pragma unroll
        for (int e = 0; e < NOWN; ++e) tot += fx_term(own[k][e] * sc);
        real res = fx_out(tot, E, f_out);
        if (!finite) res = (real)NAN;
        out[o] = (REGN && y_add) ? y_add[o] + res : res;
    }
}

template <typename real>
mof_status launch_flowT(const mof_problem *p, const real *r, const real *s, const real *sr, const int *bnd_s,
                        const int *bnd_sr, real *u, cudaStream_t st) {
    ::mof::count_launch(), k_warpT_tile<real, false><<<grid_tiles(p, p->nt), BT, 0, st>>>(
        r, s, sr, bnd_s, bnd_sr, tiles_count(p), p->nx, p->ny, p->nt - 1, p->warp_mode, nullptr, nullptr, (real)0, 1.0,
        nullptr, nullptr, 0, u);
    MOF_LAUNCH_CHECK();
    return MOF_OK;
}

// ============================================================ K12 velocity VJP of Mhat
// Derivative of the bilinear sample B(f; x + v) with respect to the displacement,
// on the cell the forward pass uses: dB/dvx = (1 - wy)(f01 - f00) + wy (f11 - f10),
// dB/dvy = (1 - wx)(f10 - f00) + wx (f11 - f01), and zero along an axis where
// the sample point is clipped (x + v < 0 or x + v >= n - 1: the sample does not
// move there). At an integer x + v this is the derivative from the right.
template <typename real>
__device__ __forceinline__ bool axis_moves(int x, real v, int n) {
    if (!(v == v)) return false;
    const real vc = v > (real)16777216 ? (real)16777216 : (v < (real)-16777216 ? (real)-16777216 : v);
    const int I = x + (int)floor(vc);
    return I >= 0 && I < n - 1;
}

template <typename real>
__device__ __forceinline__ void bilinear_grad(const real *__restrict__ f, int nx, int ny, int x, int y, real vx, real vy,
                                              real &gx, real &gy) {
    int x0, x1, y0, y1;
    real wx, wy;
    warp_axis(x, vx, nx, x0, x1, wx, 0);
    warp_axis(y, vy, ny, y0, y1, wy, 0);
    const real a = ldg(f + (long long)y0 * nx + x0), b = ldg(f + (long long)y0 * nx + x1);
    const real c = ldg(f + (long long)y1 * nx + x0), d = ldg(f + (long long)y1 * nx + x1);
    gx = axis_moves(x, vx, nx) ? (1 - wy) * (b - a) + wy * (d - c) : (real)0;
    gy = axis_moves(y, vy, ny) ? (1 - wx) * (c - a) + wx * (d - b) : (real)0;
}

// gs[t] = -gr[0][t] grad B(u_{t+1}; x + s_t), gsr[t] = -gr[1][t] grad B(u_t; x + sr_t):
// the vector-Jacobian product of r = Mhat(s, s') u with respect to s and s'.
// With the rounding-and-clipping M(s) (wm = 1) the rows are piecewise constant
// in s and the product is zero.
template <typename real>
__global__ void k_flow_ds(const real *__restrict__ u, const real *__restrict__ s, const real *__restrict__ sr,
                          const real *__restrict__ gr, real *__restrict__ gs, real *__restrict__ gsr, int nx, int ny, int np,
                          int wm) {
    const int x = blockIdx.x * TX + threadIdx.x, y = blockIdx.y * TY + threadIdx.y, t = blockIdx.z;
    if (x >= nx || y >= ny) return;
    const long long ns = (long long)nx * ny, i = (long long)y * nx + x;
    if (wm) {
        gs[2 * t * ns + i] = gs[(2 * t + 1) * ns + i] = 0;
        gsr[2 * t * ns + i] = gsr[(2 * t + 1) * ns + i] = 0;
        return;
    }
    const real g0 = gr[t * ns + i], g1 = gr[(np + t) * ns + i];
    real gx, gy;
    bilinear_grad(u + (t + 1) * ns, nx, ny, x, y, s[2 * t * ns + i], s[(2 * t + 1) * ns + i], gx, gy);
    gs[2 * t * ns + i] = -g0 * gx;
    gs[(2 * t + 1) * ns + i] = -g0 * gy;
    bilinear_grad(u + t * ns, nx, ny, x, y, sr[2 * t * ns + i], sr[(2 * t + 1) * ns + i], gx, gy);
    gsr[2 * t * ns + i] = -g1 * gx;
    gsr[(2 * t + 1) * ns + i] = -g1 * gy;
}

template <typename real>
mof_status launch_flow_ds(const mof_problem *p, const real *u, const real *s, const real *sr, const real *gr, real *gs,
                          real *gsr, cudaStream_t st) {
    ::mof::count_launch(), k_flow_ds<real><<<grid2d(p->nx, p->ny, p->nt - 1), dim3(TX, TY), 0, st>>>(u, s, sr, gr, gs, gsr, p->nx,
                                                                                                   p->ny, p->nt - 1, p->warp_mode);
    MOF_LAUNCH_CHECK();
    return MOF_OK;
}

// ============================================================ K6 reverse flow
// s'(q) = -(mean of s(p) over the sources p with dest(p) = q), dest(p) = round(p + s(p))
// clipped (k_src_bounds, MODE 1). One CTA per BW x BH destination tile: warp 0 takes the
// union of the displacement bounds of the source tiles whose destinations can fall into
// the tile; each pixel then scans the sources of its window in row-major order and sums
// their velocities in FP64 in that order, so the result is that of a sequential pass over
// the sources.
template <typename real>
__global__ void __launch_bounds__(BT) k_rev_gather(const real *__restrict__ s, const int *__restrict__ dest,
                                                   const int *__restrict__ bnd, real *__restrict__ sr, int nx, int ny,
                                                   int tiles) {
    __shared__ int4 ub;
    const int p = blockIdx.z, tid = threadIdx.x;
    const int X0 = blockIdx.x * BW, Y0 = blockIdx.y * BH;
    const int X1 = min(X0 + BW - 1, nx - 1), Y1 = min(Y0 + BH - 1, ny - 1);
    const int txn = (nx + BW - 1) / BW, tyn = (ny + BH - 1) / BH;
    if (tid < 32) {
        const TermTiles T = term_tiles(bnd + 4LL * p * (tiles + 1), tiles, txn, tyn, X0, X1, Y0, Y1, nx, ny);
        int dxmin = INT_MAX, dxmax = INT_MIN, dymin = INT_MAX, dymax = INT_MIN;
        for (int j = tid; j < T.nc; j += 32) {
            const int tx = T.txa + j % T.ntx, ty = T.tya + j / T.ntx;
            const int4 b = __ldg(T.bnd + ty * txn + tx);
            const int S0 = tx * BW, S1 = min(S0 + BW - 1, nx - 1), R0 = ty * BH, R1 = min(R0 + BH - 1, ny - 1);
            // destinations of this source tile lie in [S0 + b.x, S1 + b.y] x [R0 + b.z, R1 + b.w]
            if (S0 + b.x <= X1 && S1 + b.y >= X0 && R0 + b.z <= Y1 && R1 + b.w >= Y0) {
                dxmin = min(dxmin, b.x);
                dxmax = max(dxmax, b.y);
                dymin = min(dymin, b.z);
                dymax = max(dymax, b.w);
            }
        }
        dxmin = __reduce_min_sync(0xffffffffu, dxmin);
        dxmax = __reduce_max_sync(0xffffffffu, dxmax);
        dymin = __reduce_min_sync(0xffffffffu, dymin);
        dymax = __reduce_max_sync(0xffffffffu, dymax);
        if (tid == 0) ub = make_int4(dxmin, dxmax, dymin, dymax);
    }
    __syncthreads();
    const int4 bd = ub;
    const long long ns = (long long)nx * ny;
    const real *sx = s + 2LL * p * ns, *sy = sx + ns;
    const int *dp = dest + p * ns;
    real *rx = sr + 2LL * p * ns, *ry = rx + ns;
#pragma unroll
    for (int k = 0; k < BPT; ++k) {
        const int l = tid + k * BT, x = X0 + (l % BW), y = Y0 + l / BW;
        if (x > X1 || y > Y1) continue;
        const long long q = (long long)y * nx + x;
        // the first two arrivals in the element type, FP64 sums from the third: the mean of
        // one or two values (x, or (x0 + x1) / 2 with an exact halving) rounds as the FP64
        // mean does, so FP64 work is left to the pixels where three or more sources collide
        real a0 = 0, a1 = 0, b0 = 0, b1 = 0;
        double ax = 0.0, ay = 0.0;
        int cnt = 0;
        if (bd.x <= bd.y) {  // some source tile can reach this tile
            const int ylo = max(0, y - bd.w), yhi = min(ny - 1, y - bd.z);
            const int xlo = max(0, x - bd.y), xhi = min(nx - 1, x - bd.x);
            for (int py = ylo; py <= yhi; ++py)
                for (int px = xlo; px <= xhi; ++px) {
                    const long long i = (long long)py * nx + px;
                    if (ldg(dp + i) == (int)q) {
                        const real vx = ldg(sx + i), vy = ldg(sy + i);
                        if (cnt == 0) {
                            a0 = vx;
                            b0 = vy;
                        } else if (cnt == 1) {
                            a1 = vx;
                            b1 = vy;
                        } else {
                            if (cnt == 2) {  // in source order, as a sequential FP64 sum
                                ax = (double)a0 + (double)a1;
                                ay = (double)b0 + (double)b1;
                            }
                            ax += (double)vx;
                            ay += (double)vy;
                        }
                        ++cnt;
                    }
                }
        }
        real ox = 0, oy = 0;
        if (cnt == 1) {
            ox = -a0;
            oy = -b0;
        } else if (cnt == 2) {
            ox = -((a0 + a1) * (real)0.5);
            oy = -((b0 + b1) * (real)0.5);
        } else if (cnt > 2) {
            ox = (real)(-ax / cnt);
            oy = (real)(-ay / cnt);
        }
        rx[q] = ox;
        ry[q] = oy;
    }
}

template <typename real>
mof_status launch_reverse_flow(const mof_problem *p, const real *s, int *bnd, int *dest, real *sr, cudaStream_t st) {
    const int np = p->nt - 1, tiles = tiles_count(p);
    if (np <= 0) return MOF_OK;
    ::mof::count_launch(), k_zero_reach<<<(np + 127) / 128, 128, 0, st>>>(bnd, nullptr, np, tiles);
    MOF_LAUNCH_CHECK();
    ::mof::count_launch(), k_src_bounds<real, 1><<<grid_tiles(p, np), BT, 0, st>>>(s, s, np, p->nx, p->ny, 0, bnd, bnd,
                                                                                  tiles_x(p), tiles, dest);
    MOF_LAUNCH_CHECK();
    ::mof::count_launch(), k_rev_gather<real><<<grid_tiles(p, np), BT, 0, st>>>(s, dest, bnd, sr, p->nx, p->ny, tiles);
    MOF_LAUNCH_CHECK();
    return MOF_OK;
}

// ============================================================ K7 App. C fields
__device__ __forceinline__ int reflect_idx(int i, int n) {
    while (i < 0 || i >= n) {
        if (i < 0) i = -i - 1;
        if (i >= n) i = 2 * n - 1 - i;
    }
    return i;
}

template <typename real>
__global__ void k_of_fields(const real *__restrict__ u, int dr, real *__restrict__ ux, real *__restrict__ uy,
                            real *__restrict__ ut, int nx, int ny) {
    const int x = blockIdx.x * TX + threadIdx.x, y = blockIdx.y * TY + threadIdx.y, p = blockIdx.z;
    if (x >= nx || y >= ny) return;
    const long long ns = (long long)nx * ny;
    const real *a = u + p * ns, *b = a + ns;
    const real inv2 = (real)1 / (real)(2 * dr), box = (real)(2 * dr + 1);
    const int xp = reflect_idx(x + dr, nx), xm = reflect_idx(x - dr, nx);
    const int yp = reflect_idx(y + dr, ny), ym = reflect_idx(y - dr, ny);
    real sx = 0, sy = 0, st = 0;
    for (int k = -dr; k <= dr; ++k) {
        const int yk = reflect_idx(y + k, ny), xk = reflect_idx(x + k, nx);
        sx += (ldg(a + (long long)yk * nx + xp) - ldg(a + (long long)yk * nx + xm)) * inv2;
        sy += (ldg(a + (long long)yp * nx + xk) - ldg(a + (long long)ym * nx + xk)) * inv2;
        for (int j = -dr; j <= dr; ++j) {
            const long long q = (long long)yk * nx + reflect_idx(x + j, nx);
            st += ldg(b + q) - ldg(a + q);
        }
    }
    const long long i = p * ns + (long long)y * nx + x;
    ux[i] = sx / box;
    uy[i] = sy / box;
    ut[i] = st / (box * box);
}

// The same fields from shared-memory tiles: a CTA owns a 32 x 8 tile of every pair and
// walks the frames in order, so each frame's tile (with its reflected halo of DR pixels)
// is loaded once and serves as frame t + 1 of pair t and frame t of pair t + 1; the sums
// take the terms in the order of k_of_fields (identical results).
template <typename real, int DR>
__global__ void __launch_bounds__(TX *TY) k_of_fields_tiled(const real *__restrict__ u, real *__restrict__ ux,
                                                             real *__restrict__ uy, real *__restrict__ ut, int nx, int ny,
                                                             int np) {
    constexpr int W = TX + 2 * DR, H = TY + 2 * DR;
    __shared__ real tile[2][H][W];
    const int x0 = blockIdx.x * TX, y0 = blockIdx.y * TY;
    const int tid = threadIdx.y * TX + threadIdx.x;
    const int x = x0 + threadIdx.x, y = y0 + threadIdx.y;
    const long long ns = (long long)nx * ny;
    const real inv2 = (real)1 / (real)(2 * DR), box = (real)(2 * DR + 1);
    auto load = [&](int buf, int t) {
        const real *f = u + (long long)t * ns;
        for (int q = tid; q < W * H; q += TX * TY) {
            const int ly = q / W, lx = q - ly * W;
            const int gy = reflect_idx(y0 + ly - DR, ny), gx = reflect_idx(x0 + lx - DR, nx);
            tile[buf][ly][lx] = ldg(f + (long long)gy * nx + gx);
        }
    };
    load(0, 0);
    for (int p = 0; p < np; ++p) {
        const int ca = p & 1, cb = ca ^ 1;
        load(cb, p + 1);
        __syncthreads();
        if (x < nx && y < ny) {
            const int lx = threadIdx.x + DR, ly = threadIdx.y + DR;
            // the reflected neighbours of k_of_fields, as offsets in the halo tile
            real sx = 0, sy = 0, st = 0;
#pragma unroll
            for (int k = -DR; k <= DR; ++k) {
                sx += (tile[ca][ly + k][lx + DR] - tile[ca][ly + k][lx - DR]) * inv2;
                sy += (tile[ca][ly + DR][lx + k] - tile[ca][ly - DR][lx + k]) * inv2;
#pragma unroll
                for (int j = -DR; j <= DR; ++j) st += tile[cb][ly + k][lx + j] - tile[ca][ly + k][lx + j];
            }
            const long long i = p * ns + (long long)y * nx + x;
            ux[i] = sx / box;
            uy[i] = sy / box;
            ut[i] = st / (box * box);
        }
        __syncthreads();
    }
}

template <typename real>
mof_status launch_of_fields(const mof_problem *p, const real *u, int dr, real *ux, real *uy, real *ut, cudaStream_t st) {
    const int np = p->nt - 1;
    if (np <= 0) return MOF_OK;
    // each halo element is the reflected pixel of its own coordinate, as in k_of_fields
    if (dr == 1)
        ::mof::count_launch(), k_of_fields_tiled<real, 1><<<dim3((p->nx + TX - 1) / TX, (p->ny + TY - 1) / TY), dim3(TX, TY), 0, st>>>(
            u, ux, uy, ut, p->nx, p->ny, np);
    else if (dr == 2)
        ::mof::count_launch(), k_of_fields_tiled<real, 2><<<dim3((p->nx + TX - 1) / TX, (p->ny + TY - 1) / TY), dim3(TX, TY), 0, st>>>(
            u, ux, uy, ut, p->nx, p->ny, np);
    else
        ::mof::count_launch(), k_of_fields<real><<<grid2d(p->nx, p->ny, np), dim3(TX, TY), 0, st>>>(u, dr, ux, uy, ut, p->nx, p->ny);
    MOF_LAUNCH_CHECK();
    return MOF_OK;
}

// ================================================================ K8 Upsilon
template <typename real>
__global__ void k_flow_lin(const real *__restrict__ ux, const real *__restrict__ uy, const real *__restrict__ ut,
                           const real *__restrict__ s, real *__restrict__ r, long long ns, long long total) {
    for (long long q = blockIdx.x * (long long)blockDim.x + threadIdx.x; q < total; q += (long long)gridDim.x * blockDim.x) {
        const long long p = q / ns, i = q - p * ns;
        r[q] = ux[q] * s[2 * p * ns + i] + uy[q] * s[(2 * p + 1) * ns + i] + ut[q];
    }
}

template <typename real>
__global__ void k_flow_linT(const real *__restrict__ ux, const real *__restrict__ uy, const real *__restrict__ r,
                            real *__restrict__ gs, long long ns, long long total) {
    for (long long q = blockIdx.x * (long long)blockDim.x + threadIdx.x; q < total; q += (long long)gridDim.x * blockDim.x) {
        const long long p = q / ns, i = q - p * ns;
        gs[2 * p * ns + i] = ux[q] * r[q];
        gs[(2 * p + 1) * ns + i] = uy[q] * r[q];
    }
}

inline int flat_blocks(long long total) { return (int)std::min<long long>(152LL * 16, (total + 255) / 256); }

template <typename real>
mof_status launch_flow_lin(const mof_problem *p, const real *ux, const real *uy, const real *ut, const real *s, real *r,
                           cudaStream_t st) {
    const long long total = (long long)(p->nt - 1) * p->ns;
    ::mof::count_launch(), k_flow_lin<real><<<flat_blocks(total), 256, 0, st>>>(ux, uy, ut, s, r, p->ns, total);
    MOF_LAUNCH_CHECK();
    return MOF_OK;
}
template <typename real>
mof_status launch_flow_linT(const mof_problem *p, const real *ux, const real *uy, const real *r, real *gs, cudaStream_t st) {
    const long long total = (long long)(p->nt - 1) * p->ns;
    ::mof::count_launch(), k_flow_linT<real><<<flat_blocks(total), 256, 0, st>>>(ux, uy, r, gs, p->ns, total);
    MOF_LAUNCH_CHECK();
    return MOF_OK;
}

// ============================================================ K5 Theta^T W Theta
// Stage 1: q = W_M (Mhat x), W_M = ((Mhat uk)^2 + eps^2)^(-1/2), per flow row.
template <typename real>
__global__ void k_regn_flow_rows(const real *__restrict__ x, const real *__restrict__ uk, const real *__restrict__ s,
                                 const real *__restrict__ sr, real eps2, real *__restrict__ q, int nx, int ny, int np,
                                 int wm) {
    const int xx = blockIdx.x * TX + threadIdx.x, y = blockIdx.y * TY + threadIdx.y, p = blockIdx.z;
    if (xx >= nx || y >= ny) return;
    const long long ns = (long long)nx * ny, i = (long long)y * nx + xx;
    const real *sp = s + 2LL * p * ns, *srp = sr + 2LL * p * ns;
    const real svx = sp[i], svy = sp[ns + i], rvx = srp[i], rvy = srp[ns + i];
    const real *x0 = x + p * ns, *x1 = x0 + ns, *k0 = uk + p * ns, *k1 = k0 + ns;
    const real fx = x0[i] - bilinear(x1, nx, ny, xx, y, svx, svy, wm);
    const real fk = k0[i] - bilinear(k1, nx, ny, xx, y, svx, svy, wm);
    const real bx = x1[i] - bilinear(x0, nx, ny, xx, y, rvx, rvy, wm);
    const real bk = k1[i] - bilinear(k0, nx, ny, xx, y, rvx, rvy, wm);
    q[p * ns + i] = fx / sqrt(fk * fk + eps2);
    q[(np + p) * ns + i] = bx / sqrt(bk * bk + eps2);
}

// Stage 2: y = y_add + scale * lam * (Psi^T W_Psi Psi x [+ L_t^T W_t L_t x] + Mhat^T q), the
// transpose scatter of k_warpT_tile with the pixel's weighted differences as own terms.
template <typename real>
mof_status launch_reg_normal(const mof_problem *p, int temporal, const real *x, const real *uk, const real *s, const real *sr,
                             const int *bnd_s, const int *bnd_sr, double eps, double scale, const double *lam_dev,
                             const real *y_add, real *q, real *y, cudaStream_t st) {
    const int np = p->nt - 1;
    const real eps2 = (real)(eps * eps);
    if (np > 0) {
        ::mof::count_launch(), k_regn_flow_rows<real><<<grid2d(p->nx, p->ny, np), dim3(TX, TY), 0, st>>>(x, uk, s, sr, eps2, q, p->nx, p->ny, np, p->warp_mode);
        MOF_LAUNCH_CHECK();
    }
    ::mof::count_launch(), k_warpT_tile<real, true><<<grid_tiles(p, p->nt), BT, 0, st>>>(
        q, s, sr, bnd_s, bnd_sr, tiles_count(p), p->nx, p->ny, np, p->warp_mode, x, uk, eps2, scale, lam_dev, y_add,
        temporal, y);
    MOF_LAUNCH_CHECK();
    return MOF_OK;
}

#define MOF_INST(real)                                                                                                        \
    template mof_status launch_grad<real>(const mof_problem *, int, const real *, real *, cudaStream_t);                      \
    template mof_status launch_gradT<real>(const mof_problem *, int, const real *, real *, cudaStream_t);                     \
    template mof_status launch_flow<real>(const mof_problem *, const real *, const real *, const real *, real *, cudaStream_t); \
    template mof_status launch_tile_bounds<real>(const mof_problem *, const real *, const real *, int *, int *, cudaStream_t); \
    template mof_status launch_flow_ds<real>(const mof_problem *, const real *, const real *, const real *, const real *,      \
                                             real *, real *, cudaStream_t);                                                   \
    template mof_status launch_flowT<real>(const mof_problem *, const real *, const real *, const real *, const int *,         \
                                           const int *, real *, cudaStream_t);                                                \
    template mof_status launch_reverse_flow<real>(const mof_problem *, const real *, int *, int *, real *, cudaStream_t);     \
    template mof_status launch_of_fields<real>(const mof_problem *, const real *, int, real *, real *, real *, cudaStream_t);   \
    template mof_status launch_flow_lin<real>(const mof_problem *, const real *, const real *, const real *, const real *,     \
                                              real *, cudaStream_t);                                                          \
    template mof_status launch_flow_linT<real>(const mof_problem *, const real *, const real *, const real *, real *,          \
                                               cudaStream_t);                                                                 \
    template mof_status launch_reg_normal<real>(const mof_problem *, int, const real *, const real *, const real *, const real *,   \
                                                const int *, const int *, double, double, const double *, const real *,       \
                                                real *, real *, cudaStream_t);

MOF_INST(float)
MOF_INST(double)


// ------------------------------------------------------------ rescaling for Solve-OF
// Sec. 4.1.5 / Sec. 5: Solve-OF on frames downsampled by a factor a, the velocities
// upscaled to the full grid. Block means of a x a pixels (one thread per coarse pixel,
// summed row by row, scaled by 1/a^2); the velocity field interpolated bilinearly at
// the fine pixel centres, coarse coordinate (x + 1/2)/a - 1/2 clamped to the coarse
// grid, times a (one thread per fine value).
template <typename real>
__global__ void k_downsample(const real *__restrict__ u, real *__restrict__ uc, int nx, int ny, int nt, int a) {
    const int nxc = nx / a, nyc = ny / a;
    const long long nc = (long long)nt * nxc * nyc;
    const real inv = (real)1 / (real)(a * a);
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < nc; i += (long long)gridDim.x * blockDim.x) {
        const int X = (int)(i % nxc);
        const long long r = i / nxc;
        const int Y = (int)(r % nyc), t = (int)(r / nyc);
        const real *src = u + ((long long)t * ny + (long long)Y * a) * nx + (long long)X * a;
        real sum = 0;
        for (int dy = 0; dy < a; ++dy)
            for (int dx = 0; dx < a; ++dx) sum += src[(long long)dy * nx + dx];
        uc[i] = sum * inv;
    }
}

template <typename real>
__device__ __forceinline__ void up_axis(int x, int a, int nc, int &i0, int &i1, real &w) {
    real X = ((real)x + (real)0.5) / (real)a - (real)0.5;
    X = X < (real)0 ? (real)0 : (X > (real)(nc - 1) ? (real)(nc - 1) : X);
    i0 = (int)floor(X);
    i1 = min(i0 + 1, nc - 1);
    w = X - (real)i0;
}

template <typename real>
__global__ void k_upsample_vel(const real *__restrict__ sc, real *__restrict__ s, int nx, int ny, int nplanes, int a) {
    const int nxc = nx / a, nyc = ny / a;
    const long long nf = (long long)nplanes * nx * ny;
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < nf; i += (long long)gridDim.x * blockDim.x) {
        const int x = (int)(i % nx);
        const long long r = i / nx;
        const int y = (int)(r % ny), pl = (int)(r / ny);
        int x0, x1, y0, y1;
        real wx, wy;
        up_axis<real>(x, a, nxc, x0, x1, wx);
        up_axis<real>(y, a, nyc, y0, y1, wy);
        const real *c = sc + (long long)pl * nxc * nyc;
        const real v = c[y0 * nxc + x0] * ((real)1 - wx) * ((real)1 - wy) + c[y0 * nxc + x1] * wx * ((real)1 - wy) +
                       c[y1 * nxc + x0] * ((real)1 - wx) * wy + c[y1 * nxc + x1] * wx * wy;
        s[i] = (real)a * v;
    }
}

template <typename real>
mof_status launch_downsample(const mof_problem *p, int a, const real *u, real *uc, cudaStream_t st) {
    const long long nc = (long long)p->nt * (p->nx / a) * (p->ny / a);
    const int blocks = (int)std::min<long long>(152 * 16, (nc + 255) / 256);
    if (nc > 0) ::mof::count_launch(), k_downsample<real><<<blocks, 256, 0, st>>>(u, uc, p->nx, p->ny, p->nt, a);
    MOF_LAUNCH_CHECK();
    return MOF_OK;
}

template <typename real>
mof_status launch_upsample_velocity(const mof_problem *p, int a, const real *sc, real *s, cudaStream_t st) {
    const int nplanes = 2 * (p->nt - 1);
    const long long nf = (long long)nplanes * p->nx * p->ny;
    const int blocks = (int)std::min<long long>(152 * 16, (nf + 255) / 256);
    if (nf > 0) ::mof::count_launch(), k_upsample_vel<real><<<blocks, 256, 0, st>>>(sc, s, p->nx, p->ny, nplanes, a);
    MOF_LAUNCH_CHECK();
    return MOF_OK;
}

template mof_status launch_downsample<float>(const mof_problem *, int, const float *, float *, cudaStream_t);
template mof_status launch_downsample<double>(const mof_problem *, int, const double *, double *, cudaStream_t);
template mof_status launch_upsample_velocity<float>(const mof_problem *, int, const float *, float *, cudaStream_t);
template mof_status launch_upsample_velocity<double>(const mof_problem *, int, const double *, double *, cudaStream_t);

}  // namespace mof
