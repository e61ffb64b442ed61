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
// sources p within a square window around q, in a fixed order, so repeated
// runs are bit-identical. The window radius is per 32x8 output tile: every
// source records, in the tile of each pixel it reaches, the Chebyshev
// distance to that pixel (atomic max), so a tile scans only as far as its
// farthest actual arrival.
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

// (M(v)^T r)(q) by a gather over the window of radius R around q.
template <typename real>
__device__ __forceinline__ real warpT_gather(const real *__restrict__ r, const real *__restrict__ vx,
                                             const real *__restrict__ vy, int nx, int ny, int qx, int qy, int R, int wm) {
    real acc = 0;
    const int ylo = max(0, qy - R), yhi = min(ny - 1, qy + R);
    const int xlo = max(0, qx - R), xhi = min(nx - 1, qx + R);
    for (int py = ylo; py <= yhi; ++py) {
        for (int px = xlo; px <= xhi; ++px) {
            const long long i = (long long)py * nx + px;
            const real w = warp_weight_to(px, py, ldg(vx + i), ldg(vy + i), nx, ny, qx, qy, wm);
            if (w != (real)0) acc += w * ldg(r + i);
        }
    }
    return acc;
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

template <typename real>
mof_status launch_grad(const mof_problem *p, int nf, const real *u, real *g, cudaStream_t st) {
    ::mof::count_launch(), k_grad<real><<<grid2d(p->nx, p->ny, nf), dim3(TX, TY), 0, st>>>(u, g, p->nx, p->ny);
    MOF_LAUNCH_CHECK();
    return MOF_OK;
}
template <typename real>
mof_status launch_gradT(const mof_problem *p, int nf, const real *g, real *u, cudaStream_t st) {
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

template <typename real>
mof_status launch_flow(const mof_problem *p, const real *u, const real *s, const real *sr, real *r, cudaStream_t st) {
    const int np = p->nt - 1;
    ::mof::count_launch(), k_flow<real><<<grid2d(p->nx, p->ny, np), dim3(TX, TY), 0, st>>>(u, s, sr, r, p->nx, p->ny, np, p->warp_mode);
    MOF_LAUNCH_CHECK();
    return MOF_OK;
}

// Per-tile gather radii of M(v)^T for nf velocity fields v[f] (each [2][ny][nx]):
// rad[f][tile] = max over sources p and the pixels q of their bilinear
// footprint, q in the tile, of |p - q|_inf. Launched with the gather tiling.
template <typename real>
__global__ void k_tile_radius(const real *__restrict__ v, int nx, int ny, int *__restrict__ rad, int tiles_x, int tiles, int wm) {
    __shared__ int own;
    const int x = blockIdx.x * TX + threadIdx.x, y = blockIdx.y * TY + threadIdx.y, f = blockIdx.z;
    const int tid = threadIdx.y * TX + threadIdx.x;
    if (tid == 0) own = 0;
    __syncthreads();
    if (x < nx && y < ny) {
        const long long ns = (long long)nx * ny, i = (long long)y * nx + x;
        const real *vf = v + 2LL * f * ns;
        int x0, x1, y0, y1;
        real wx, wy;
        warp_axis(x, vf[i], nx, x0, x1, wx, wm);
        warp_axis(y, vf[ns + i], ny, y0, y1, wy, wm);
        const int qx[2] = {x0, x1}, qy[2] = {y0, y1};
#pragma unroll
        for (int a = 0; a < 2; ++a)
#pragma unroll
            for (int c = 0; c < 2; ++c) {
                const int d = max(abs(qx[a] - x), abs(qy[c] - y));
                const int tx = qx[a] / TX, ty = qy[c] / TY;
                if (tx == (int)blockIdx.x && ty == (int)blockIdx.y) atomicMax(&own, d);
                else atomicMax(&rad[(long long)f * tiles + ty * tiles_x + tx], d);
            }
    }
    __syncthreads();
    if (tid == 0) atomicMax(&rad[(long long)f * tiles + blockIdx.y * tiles_x + blockIdx.x], own);
}

__global__ void k_zero_ints(int *p, long long n) {
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x) p[i] = 0;
}

int tiles_x(const mof_problem *p) { return (p->nx + TX - 1) / TX; }
int tiles_count(const mof_problem *p) { return tiles_x(p) * ((p->ny + TY - 1) / TY); }

template <typename real>
mof_status launch_tile_radii(const mof_problem *p, const real *s, const real *sr, int *rad_s, int *rad_sr, cudaStream_t st) {
    const int np = p->nt - 1, tiles = tiles_count(p);
    ::mof::count_launch(), k_zero_ints<<<8, 256, 0, st>>>(rad_s, (long long)np * tiles);
    MOF_LAUNCH_CHECK();
    ::mof::count_launch(), k_tile_radius<real><<<grid2d(p->nx, p->ny, np), dim3(TX, TY), 0, st>>>(s, p->nx, p->ny, rad_s, tiles_x(p), tiles, p->warp_mode);
    MOF_LAUNCH_CHECK();
    if (sr) {
        ::mof::count_launch(), k_zero_ints<<<8, 256, 0, st>>>(rad_sr, (long long)np * tiles);
        MOF_LAUNCH_CHECK();
        ::mof::count_launch(), k_tile_radius<real><<<grid2d(p->nx, p->ny, np), dim3(TX, TY), 0, st>>>(sr, p->nx, p->ny, rad_sr, tiles_x(p), tiles, p->warp_mode);
        MOF_LAUNCH_CHECK();
    }
    return MOF_OK;
}

// u = Mhat^T r (+ optional addend, times scale), one thread per pixel of a frame:
//   u_t = [t<P] r0_t + [t>0] r1_{t-1} - [t<P] M(sr_t)^T r1_t - [t>0] M(s_{t-1})^T r0_{t-1}
template <typename real>
__device__ __forceinline__ real flowT_at(const real *__restrict__ r, const real *__restrict__ s, const real *__restrict__ sr,
                                         int nx, int ny, int np, int t, int x, int y, const int *__restrict__ rad_s,
                                         const int *__restrict__ rad_sr, int tiles, int tile, int wm) {
    const long long ns = (long long)nx * ny, i = (long long)y * nx + x;
    real v = 0;
    if (t < np) {
        const real *r1 = r + (np + t) * ns;
        const real *srp = sr + 2LL * t * ns;
        v += r[t * ns + i];
        v -= warpT_gather(r1, srp, srp + ns, nx, ny, x, y, rad_sr[(long long)t * tiles + tile], wm);
    }
    if (t > 0) {
        const real *r0 = r + (long long)(t - 1) * ns;
        const real *sp = s + 2LL * (t - 1) * ns;
        v += r[(np + t - 1) * ns + i];
        v -= warpT_gather(r0, sp, sp + ns, nx, ny, x, y, rad_s[(long long)(t - 1) * tiles + tile], wm);
    }
    return v;
}

template <typename real>
__global__ void k_flowT(const real *__restrict__ r, const real *__restrict__ s, const real *__restrict__ sr,
                        const int *__restrict__ rad_s, const int *__restrict__ rad_sr, real *__restrict__ u, int nx, int ny,
                        int np, int tiles, int wm) {
    const int x = blockIdx.x * TX + threadIdx.x, y = blockIdx.y * TY + threadIdx.y, t = blockIdx.z;
    if (x >= nx || y >= ny) return;
    const int tile = blockIdx.y * gridDim.x + blockIdx.x;
    u[(long long)t * nx * ny + (long long)y * nx + x] = flowT_at(r, s, sr, nx, ny, np, t, x, y, rad_s, rad_sr, tiles, tile, wm);
}

template <typename real>
mof_status launch_flowT(const mof_problem *p, const real *r, const real *s, const real *sr, const int *rad_s,
                        const int *rad_sr, real *u, cudaStream_t st) {
    ::mof::count_launch(), k_flowT<real><<<grid2d(p->nx, p->ny, p->nt), dim3(TX, TY), 0, st>>>(r, s, sr, rad_s, rad_sr, u, p->nx, p->ny, p->nt - 1,
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
__global__ void k_rev_dest(const real *__restrict__ s, int *__restrict__ dest, int *__restrict__ rad, int nx, int ny,
                           int tiles_x, int tiles) {
    __shared__ int own;
    const int x = blockIdx.x * TX + threadIdx.x, y = blockIdx.y * TY + threadIdx.y, p = blockIdx.z;
    const int tid = threadIdx.y * TX + threadIdx.x;
    if (tid == 0) own = 0;
    __syncthreads();
    if (x < nx && y < ny) {
        const long long ns = (long long)nx * ny, i = (long long)y * nx + x;
        const real *sp = s + 2LL * p * ns;
        const int dx = round_axis(x, sp[i], nx), dy = round_axis(y, sp[ns + i], ny);
        dest[p * ns + i] = dy * nx + dx;
        const int d = max(abs(dx - x), abs(dy - y));
        const int tx = dx / TX, ty = dy / TY;
        if (tx == (int)blockIdx.x && ty == (int)blockIdx.y) atomicMax(&own, d);
        else atomicMax(&rad[(long long)p * tiles + ty * tiles_x + tx], d);
    }
    __syncthreads();
    if (tid == 0) atomicMax(&rad[(long long)p * tiles + blockIdx.y * tiles_x + blockIdx.x], own);
}

template <typename real>
__global__ void k_rev_gather(const real *__restrict__ s, const int *__restrict__ dest, const int *__restrict__ rad,
                             real *__restrict__ sr, int nx, int ny, int tiles) {
    const int x = blockIdx.x * TX + threadIdx.x, y = blockIdx.y * TY + threadIdx.y, p = blockIdx.z;
    if (x >= nx || y >= ny) return;
    const long long ns = (long long)nx * ny, q = (long long)y * nx + x;
    const real *sx = s + 2LL * p * ns, *sy = sx + ns;
    const int *dp = dest + p * ns;
    const int R = rad[(long long)p * tiles + blockIdx.y * gridDim.x + blockIdx.x];
    double ax = 0.0, ay = 0.0;
    int cnt = 0;
    // sources in row-major order, as the arrivals are accumulated in order of source
    const int ylo = max(0, y - R), yhi = min(ny - 1, y + R);
    const int xlo = max(0, x - R), xhi = min(nx - 1, x + R);
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
mof_status launch_reverse_flow(const mof_problem *p, const real *s, int *rad, int *dest, real *sr, cudaStream_t st) {
    const int np = p->nt - 1, tiles = tiles_count(p);
    ::mof::count_launch(), k_zero_ints<<<8, 256, 0, st>>>(rad, (long long)np * tiles);
    MOF_LAUNCH_CHECK();
    ::mof::count_launch(), k_rev_dest<real><<<grid2d(p->nx, p->ny, np), dim3(TX, TY), 0, st>>>(s, dest, rad, p->nx, p->ny, tiles_x(p), tiles);
    MOF_LAUNCH_CHECK();
    ::mof::count_launch(), k_rev_gather<real><<<grid2d(p->nx, p->ny, np), dim3(TX, TY), 0, st>>>(s, dest, rad, sr, p->nx, p->ny, tiles);
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

template <typename real>
mof_status launch_of_fields(const mof_problem *p, const real *u, int dr, real *ux, real *uy, real *ut, cudaStream_t st) {
    ::mof::count_launch(), k_of_fields<real><<<grid2d(p->nx, p->ny, p->nt - 1), dim3(TX, TY), 0, st>>>(u, dr, ux, uy, ut, p->nx, p->ny);
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
                             const real *__restrict__ sr, const real *__restrict__ q, const int *__restrict__ rad_s,
                             const int *__restrict__ rad_sr, int tiles, real eps2, double scale,
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
    real v = 0;
    if (xx > 0) v += wdx(i - 1);
    if (xx < nx - 1) v -= wdx(i);
    if (yy > 0) v += wdy(i - nx);
    if (yy < ny - 1) v -= wdy(i);
    if (temporal) {  // L_t^T w_t L_t x: the weighted differences to the previous and next frame
        auto wdt = [&](const real *fa, const real *ka) -> real {
            const real g = fa[i + ns] - fa[i], gk = ka[i + ns] - ka[i];
            return g / sqrt(gk * gk + eps2);
        };
        if (t > 0) v += wdt(f - ns, k - ns);
        if (t < np) v -= wdt(f, k);
    }
    if (np > 0) v += flowT_at(q, s, sr, nx, ny, np, t, xx, yy, rad_s, rad_sr, tiles, blockIdx.y * gridDim.x + blockIdx.x, wm);
    const real out = s_sc * v;
    y[t * ns + i] = y_add ? y_add[t * ns + i] + out : out;
}

template <typename real>
mof_status launch_reg_normal(const mof_problem *p, int temporal, const real *x, const real *uk, const real *s, const real *sr,
                             const int *rad_s, const int *rad_sr, double eps, double scale, const double *lam_dev,
                             const real *y_add, real *q, real *y, cudaStream_t st) {
    const int np = p->nt - 1;
    const real eps2 = (real)(eps * eps);
    if (np > 0) {
        ::mof::count_launch(), k_regn_flow_rows<real><<<grid2d(p->nx, p->ny, np), dim3(TX, TY), 0, st>>>(x, uk, s, sr, eps2, q, p->nx, p->ny, np, p->warp_mode);
        MOF_LAUNCH_CHECK();
    }
    ::mof::count_launch(), k_regn_apply<real><<<grid2d(p->nx, p->ny, p->nt), dim3(TX, TY), 0, st>>>(x, uk, s, sr, q, rad_s, rad_sr, tiles_count(p),
                                                                            eps2, scale, lam_dev, y_add, y, p->nx, p->ny, np, temporal,
                                                                            p->warp_mode);
    MOF_LAUNCH_CHECK();
    return MOF_OK;
}

#define MOF_INST(real)                                                                                                        \
    template mof_status launch_grad<real>(const mof_problem *, int, const real *, real *, cudaStream_t);                      \
    template mof_status launch_gradT<real>(const mof_problem *, int, const real *, real *, cudaStream_t);                     \
    template mof_status launch_flow<real>(const mof_problem *, const real *, const real *, const real *, real *, cudaStream_t); \
    template mof_status launch_tile_radii<real>(const mof_problem *, const real *, const real *, int *, int *, cudaStream_t);  \
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
