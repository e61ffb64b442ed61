// Stencil and flow operators of MMGKS-OF:
//   K3  Psi / Psi^T            forward differences of every frame (eq. (L))
//   K4  Mhat / Mhat^T          bilinear temporal warp rows (Sec. 3, Sec. 4)
//   K5  Theta^T W Theta        IRLS-weighted regulariser normal operator (Alg. 1)
//   K6  reverse flow           s' from s (remark of Sec. 3)
//   K7  App. C derivative fields u_x, u_y, u_t
//   K8  Upsilon s + u_t, Upsilon^T r (Sec. 2.2)
//
// The transposes of the warp (and the reverse flow) are computed as
// deterministic gathers: an output pixel q collects the contributions of the
// sources p within a window around q, in row-major source order, so repeated
// runs are bit-identical. The window is bounded per 32x8 output tile by the
// range of the integer displacements of the sources that reach it: every
// source p records, in each tile its footprint touches, its displacement
// (x0(p) - px, y0(p) - py) to the first corner of the footprint (integer
// atomic min and max), so a pixel scans only the sources whose displacement
// could bring them to it: 2 x 2 positions where the flow is locally constant
// at the integer level, one more row and column per unit of spread.
#include "common.cuh"

#include <algorithm>

#include <cfloat>

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

// Weight with which the source pixel (px, py), sampling at r + s(r), reaches
// the pixel (qx, qy): the transposed bilinear weight.
template <typename real>
__device__ __forceinline__ real warp_weight_to(int px, int py, real vx, real vy, int nx, int ny, int qx, int qy, int wm) {
    int x0, x1, y0, y1;
    real wx, wy;
    warp_axis(px, vx, nx, x0, x1, wx, wm);
    warp_axis(py, vy, ny, y0, y1, wy, wm);
    const real ax = (qx == x0 ? 1 - wx : (real)0) + (qx == x1 ? wx : (real)0);
    const real ay = (qy == y0 ? 1 - wy : (real)0) + (qy == y1 ? wy : (real)0);
    return ax * ay;
}

// Per-tile bounds of the integer displacements of the sources that reach a tile:
// {dxmin, dxmax, dymin, dymax}; an empty tile keeps (BND_EMPTY, -BND_EMPTY, ...),
// whose window is empty.
constexpr int BND_EMPTY = 1 << 29;

// Compensated sum of the terms of one output pixel of a transpose: in FP32 each term's
// rounding error is kept (DFAcc::add), so the result does not lose the digits that the
// cancellation between the terms of Mhat^T and Psi^T would otherwise cost; FP64 sums plainly.
template <typename real> struct CAcc;
template <> struct CAcc<float> {
    DFAcc a;
    __device__ __forceinline__ void add(float x) { a.add(x); }
    __device__ __forceinline__ double value() const { return a.value(); }
};
template <> struct CAcc<double> {
    double s = 0.0;
    __device__ __forceinline__ void add(double x) { s += x; }
    __device__ __forceinline__ double value() const { return s; }
};

// acc -= (M(v)^T r)(q), by a gather over the sources p whose footprint can contain q:
// px in [qx - 1 - dxmax, qx - dxmin] (x1(p) is x0(p) or x0(p) + 1), likewise py, in
// row-major source order.
template <typename real>
__device__ __forceinline__ void warpT_gather_sub(CAcc<real> &acc, const real *__restrict__ r, const real *__restrict__ vx,
                                                 const real *__restrict__ vy, int nx, int ny, int qx, int qy, int4 bd,
                                                 int wm) {
    const int ylo = max(0, qy - 1 - bd.w), yhi = min(ny - 1, qy - bd.z);
    const int xlo = max(0, qx - 1 - bd.y), xhi = min(nx - 1, qx - bd.x);
    for (int py = ylo; py <= yhi; ++py) {
        for (int px = xlo; px <= xhi; ++px) {
            const long long i = (long long)py * nx + px;
            const real w = warp_weight_to(px, py, ldg(vx + i), ldg(vy + i), nx, ny, qx, qy, wm);
            if (w != (real)0) acc.add(-(w * ldg(r + i)));
        }
    }
}

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

// Per-tile displacement bounds of M(v)^T for nf velocity fields v[f] (each [2][ny][nx]):
// bnd[f][tile] = {min, max} of x0(p) - px and of y0(p) - py over the sources p whose
// bilinear footprint {x0, x1} x {y0, y1} touches the tile (integer atomics: exact and
// order independent). Launched with the gather tiling; bounds of the block's own tile
// are reduced in shared memory first.
__device__ __forceinline__ void bnd_update(int *b, int dx, int dy) {
    atomicMin(b + 0, dx);
    atomicMax(b + 1, dx);
    atomicMin(b + 2, dy);
    atomicMax(b + 3, dy);
}

template <typename real>
__global__ void k_tile_bounds(const real *__restrict__ v, int nx, int ny, int *__restrict__ bnd, int tiles_x, int tiles, int wm) {
    __shared__ int own[4];
    const int x = blockIdx.x * TX + threadIdx.x, y = blockIdx.y * TY + threadIdx.y, f = blockIdx.z;
    const int tid = threadIdx.y * TX + threadIdx.x;
    if (tid == 0) {
        own[0] = BND_EMPTY; own[1] = -BND_EMPTY; own[2] = BND_EMPTY; own[3] = -BND_EMPTY;
    }
    __syncthreads();
    if (x < nx && y < ny) {
        const long long ns = (long long)nx * ny, i = (long long)y * nx + x;
        const real *vf = v + 2LL * f * ns;
        int x0, x1, y0, y1;
        real wx, wy;
        warp_axis(x, vf[i], nx, x0, x1, wx, wm);
        warp_axis(y, vf[ns + i], ny, y0, y1, wy, wm);
        const int dx = x0 - x, dy = y0 - y;
        const int tx0 = x0 / TX, tx1 = x1 / TX, ty0 = y0 / TY, ty1 = y1 / TY;
#pragma unroll
        for (int a = 0; a < 2; ++a) {
            if (a == 1 && tx1 == tx0) break;
            const int tx = a ? tx1 : tx0;
#pragma unroll
            for (int c = 0; c < 2; ++c) {
                if (c == 1 && ty1 == ty0) break;
                const int ty = c ? ty1 : ty0;
                if (tx == (int)blockIdx.x && ty == (int)blockIdx.y) bnd_update(own, dx, dy);
                else bnd_update(bnd + 4 * ((long long)f * tiles + ty * tiles_x + tx), dx, dy);
            }
        }
    }
    __syncthreads();
    if (tid == 0 && own[0] != BND_EMPTY) {
        int *b = bnd + 4 * ((long long)f * tiles + blockIdx.y * tiles_x + blockIdx.x);
        bnd_update(b, own[0], own[2]);
        bnd_update(b, own[1], own[3]);
    }
}

// every tile's bounds to the empty window
__global__ void k_bounds_empty(int *p, long long ntiles) {
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < ntiles; i += (long long)gridDim.x * blockDim.x)
        reinterpret_cast<int4 *>(p)[i] = make_int4(BND_EMPTY, -BND_EMPTY, BND_EMPTY, -BND_EMPTY);
}

__global__ void k_zero_ints(int *p, long long n) {
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x) p[i] = 0;
}

int tiles_x(const mof_problem *p) { return (p->nx + TX - 1) / TX; }
int tiles_count(const mof_problem *p) { return tiles_x(p) * ((p->ny + TY - 1) / TY); }
long long tile_bound_ints(const mof_problem *p) { return 4LL * tiles_count(p); }

static int bounds_blocks(long long ntiles) { return (int)std::min<long long>(152 * 4, (ntiles + 255) / 256); }

template <typename real>
mof_status launch_tile_bounds(const mof_problem *p, const real *s, const real *sr, int *bnd_s, int *bnd_sr, cudaStream_t st) {
    const int np = p->nt - 1, tiles = tiles_count(p);
    if (np <= 0) return MOF_OK;
    ::mof::count_launch(), k_bounds_empty<<<bounds_blocks((long long)np * tiles), 256, 0, st>>>(bnd_s, (long long)np * tiles);
    MOF_LAUNCH_CHECK();
    ::mof::count_launch(), k_tile_bounds<real><<<grid2d(p->nx, p->ny, np), dim3(TX, TY), 0, st>>>(s, p->nx, p->ny, bnd_s, tiles_x(p), tiles, p->warp_mode);
    MOF_LAUNCH_CHECK();
    if (sr) {
        ::mof::count_launch(), k_bounds_empty<<<bounds_blocks((long long)np * tiles), 256, 0, st>>>(bnd_sr, (long long)np * tiles);
        MOF_LAUNCH_CHECK();
        ::mof::count_launch(), k_tile_bounds<real><<<grid2d(p->nx, p->ny, np), dim3(TX, TY), 0, st>>>(sr, p->nx, p->ny, bnd_sr, tiles_x(p), tiles, p->warp_mode);
        MOF_LAUNCH_CHECK();
    }
    return MOF_OK;
}

// u = Mhat^T r (+ optional addend, times scale), one thread per pixel of a frame:
//   u_t = [t<P] r0_t + [t>0] r1_{t-1} - [t<P] M(sr_t)^T r1_t - [t>0] M(s_{t-1})^T r0_{t-1}
template <typename real>
__device__ __forceinline__ void flowT_at(CAcc<real> &v, const real *__restrict__ r, const real *__restrict__ s,
                                         const real *__restrict__ sr, int nx, int ny, int np, int t, int x, int y,
                                         const int *__restrict__ bnd_s, const int *__restrict__ bnd_sr, int tiles, int tile,
                                         int wm) {
    const long long ns = (long long)nx * ny, i = (long long)y * nx + x;
    if (t < np) {
        const real *r1 = r + (np + t) * ns;
        const real *srp = sr + 2LL * t * ns;
        v.add(r[t * ns + i]);
        const int4 bd = __ldg(reinterpret_cast<const int4 *>(bnd_sr) + (long long)t * tiles + tile);
        warpT_gather_sub(v, r1, srp, srp + ns, nx, ny, x, y, bd, wm);
    }
    if (t > 0) {
        const real *r0 = r + (long long)(t - 1) * ns;
        const real *sp = s + 2LL * (t - 1) * ns;
        v.add(r[(np + t - 1) * ns + i]);
        const int4 bd = __ldg(reinterpret_cast<const int4 *>(bnd_s) + (long long)(t - 1) * tiles + tile);
        warpT_gather_sub(v, r0, sp, sp + ns, nx, ny, x, y, bd, wm);
    }
}

template <typename real>
__global__ void k_flowT(const real *__restrict__ r, const real *__restrict__ s, const real *__restrict__ sr,
                        const int *__restrict__ bnd_s, const int *__restrict__ bnd_sr, real *__restrict__ u, int nx, int ny,
                        int np, int tiles, int wm) {
    const int x = blockIdx.x * TX + threadIdx.x, y = blockIdx.y * TY + threadIdx.y, t = blockIdx.z;
    if (x >= nx || y >= ny) return;
    const int tile = blockIdx.y * gridDim.x + blockIdx.x;
    CAcc<real> v;
    flowT_at(v, r, s, sr, nx, ny, np, t, x, y, bnd_s, bnd_sr, tiles, tile, wm);
    u[(long long)t * nx * ny + (long long)y * nx + x] = (real)v.value();
}

template <typename real>
mof_status launch_flowT(const mof_problem *p, const real *r, const real *s, const real *sr, const int *bnd_s,
                        const int *bnd_sr, real *u, cudaStream_t st) {
    ::mof::count_launch(), k_flowT<real><<<grid2d(p->nx, p->ny, p->nt), dim3(TX, TY), 0, st>>>(r, s, sr, bnd_s, bnd_sr, u, p->nx, p->ny, p->nt - 1,
                                                                      tiles_count(p), p->warp_mode);
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
// Destination of each source pixel, round half away from zero of r + s(r),
// clipped. With v = fv + fr (fv = floor(v), fr in [0,1) exact) and
// I = x + fv: for I >= 0 the position is >= 0 and rounds up iff fr >= 1/2;
// for I < 0 it is negative and rounds up (towards zero) iff fr > 1/2. This
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

template <typename real>
__global__ void k_rev_dest(const real *__restrict__ s, int *__restrict__ dest, int *__restrict__ bnd, int nx, int ny,
                           int tiles_x, int tiles) {
    __shared__ int own[4];
    const int x = blockIdx.x * TX + threadIdx.x, y = blockIdx.y * TY + threadIdx.y, p = blockIdx.z;
    const int tid = threadIdx.y * TX + threadIdx.x;
    if (tid == 0) {
        own[0] = BND_EMPTY; own[1] = -BND_EMPTY; own[2] = BND_EMPTY; own[3] = -BND_EMPTY;
    }
    __syncthreads();
    if (x < nx && y < ny) {
        const long long ns = (long long)nx * ny, i = (long long)y * nx + x;
        const real *sp = s + 2LL * p * ns;
        const int dx = round_axis(x, sp[i], nx), dy = round_axis(y, sp[ns + i], ny);
        dest[p * ns + i] = dy * nx + dx;
        const int tx = dx / TX, ty = dy / TY;
        if (tx == (int)blockIdx.x && ty == (int)blockIdx.y) bnd_update(own, dx - x, dy - y);
        else bnd_update(bnd + 4 * ((long long)p * tiles + ty * tiles_x + tx), dx - x, dy - y);
    }
    __syncthreads();
    if (tid == 0 && own[0] != BND_EMPTY) {
        int *b = bnd + 4 * ((long long)p * tiles + blockIdx.y * tiles_x + blockIdx.x);
        bnd_update(b, own[0], own[2]);
        bnd_update(b, own[1], own[3]);
    }
}

// s'(q) = -(mean of s(p) over the sources p with dest(p) = q), sources in row-major
// order within the window px in [qx - dxmax, qx - dxmin], py likewise (the tile's bounds)
template <typename real>
__global__ void k_rev_gather(const real *__restrict__ s, const int *__restrict__ dest, const int *__restrict__ bnd,
                             real *__restrict__ sr, int nx, int ny, int tiles) {
    const int x = blockIdx.x * TX + threadIdx.x, y = blockIdx.y * TY + threadIdx.y, p = blockIdx.z;
    if (x >= nx || y >= ny) return;
    const long long ns = (long long)nx * ny, q = (long long)y * nx + x;
    const real *sx = s + 2LL * p * ns, *sy = sx + ns;
    const int *dp = dest + p * ns;
    const int4 bd = __ldg(reinterpret_cast<const int4 *>(bnd) + (long long)p * tiles + blockIdx.y * gridDim.x + blockIdx.x);
    double ax = 0.0, ay = 0.0;
    int cnt = 0;
    // sources in row-major order, as the arrivals are accumulated in order of source
    const int ylo = max(0, y - bd.w), yhi = min(ny - 1, y - bd.z);
    const int xlo = max(0, x - bd.y), xhi = min(nx - 1, x - bd.x);
    for (int py = ylo; py <= yhi; ++py)
        for (int px = xlo; px <= xhi; ++px) {
            const long long i = (long long)py * nx + px;
            if (ldg(dp + i) == (int)q) {
                ax -= (double)ldg(sx + i);
                ay -= (double)ldg(sy + i);
                ++cnt;
            }
        }
    real *rx = sr + 2LL * p * ns, *ry = rx + ns;
    rx[q] = cnt ? (real)(ax / cnt) : (real)0;
    ry[q] = cnt ? (real)(ay / cnt) : (real)0;
}

template <typename real>
mof_status launch_reverse_flow(const mof_problem *p, const real *s, int *bnd, int *dest, real *sr, cudaStream_t st) {
    const int np = p->nt - 1, tiles = tiles_count(p);
    if (np <= 0) return MOF_OK;
    ::mof::count_launch(), k_bounds_empty<<<bounds_blocks((long long)np * tiles), 256, 0, st>>>(bnd, (long long)np * tiles);
    MOF_LAUNCH_CHECK();
    ::mof::count_launch(), k_rev_dest<real><<<grid2d(p->nx, p->ny, np), dim3(TX, TY), 0, st>>>(s, dest, bnd, p->nx, p->ny, tiles_x(p), tiles);
    MOF_LAUNCH_CHECK();
    ::mof::count_launch(), k_rev_gather<real><<<grid2d(p->nx, p->ny, np), dim3(TX, TY), 0, st>>>(s, dest, bnd, sr, p->nx, p->ny, tiles);
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

// Stage 2: y = y_add + scale * (Psi^T W_Psi Psi x + Mhat^T q).
template <typename real>
__global__ void k_regn_apply(const real *__restrict__ x, const real *__restrict__ uk, const real *__restrict__ s,
                             const real *__restrict__ sr, const real *__restrict__ q, const int *__restrict__ bnd_s,
                             const int *__restrict__ bnd_sr, int tiles, real eps2, double scale,
                             const double *__restrict__ lam, const real *__restrict__ y_add, real *__restrict__ y, int nx,
                             int ny, int np, int temporal, int wm) {
    const int xx = blockIdx.x * TX + threadIdx.x, yy = blockIdx.y * TY + threadIdx.y, t = blockIdx.z;
    __shared__ real s_sc;  // scale * lam once per block (FP64 kept out of the threads)
    if (threadIdx.x == 0 && threadIdx.y == 0) s_sc = (real)(lam ? scale * *lam : scale);
    __syncthreads();
    if (xx >= nx || yy >= ny) return;
    const long long ns = (long long)nx * ny, i = (long long)yy * nx + xx;
    const real *f = x + t * ns, *k = uk + t * ns;
    // weighted differences d(i) = w(i) * (f(i+e) - f(i)), w from uk
    auto wdx = [&](long long j) -> real {
        const real g = f[j + 1] - f[j], gk = k[j + 1] - k[j];
        return g / sqrt(gk * gk + eps2);
    };
    auto wdy = [&](long long j) -> real {
        const real g = f[j + nx] - f[j], gk = k[j + nx] - k[j];
        return g / sqrt(gk * gk + eps2);
    };
    CAcc<real> v;
    if (xx > 0) v.add(wdx(i - 1));
    if (xx < nx - 1) v.add(-wdx(i));
    if (yy > 0) v.add(wdy(i - nx));
    if (yy < ny - 1) v.add(-wdy(i));
    if (temporal) {  // L_t^T w_t L_t x: the weighted differences to the previous and next frame
        auto wdt = [&](const real *fa, const real *ka) -> real {
            const real g = fa[i + ns] - fa[i], gk = ka[i + ns] - ka[i];
            return g / sqrt(gk * gk + eps2);
        };
        if (t > 0) v.add(wdt(f - ns, k - ns));
        if (t < np) v.add(-wdt(f, k));
    }
    if (np > 0) flowT_at(v, q, s, sr, nx, ny, np, t, xx, yy, bnd_s, bnd_sr, tiles, blockIdx.y * gridDim.x + blockIdx.x, wm);
    const real out = (real)((double)s_sc * v.value());
    y[t * ns + i] = y_add ? y_add[t * ns + i] + out : out;
}

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
    ::mof::count_launch(), k_regn_apply<real><<<grid2d(p->nx, p->ny, p->nt), dim3(TX, TY), 0, st>>>(x, uk, s, sr, q, bnd_s, bnd_sr, tiles_count(p),
                                                                            eps2, scale, lam_dev, y_add, y, p->nx, p->ny, np, temporal,
                                                                            p->warp_mode);
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
