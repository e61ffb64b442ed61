/*
 * FP64 CPU oracle: the linear operators of MMGKS-OF, written out plainly.
 *
 * TEST INFRASTRUCTURE ONLY. Nothing on the product path may call, link or
 * load this file; only the tests, the package smoke check and the bench's
 * CPU baseline use it. It shares no code, header or constant with the CUDA
 * library.
 *
 * Conventions (all arrays are caller-owned, FP64, row-major, x fastest):
 *   image sequence  u[t][y][x],  t < nt, y < ny, x < nx   (Sec. 2.1: column-stacked
 *                   frames; the paper's row index i = y*nx + x, Sec. 3 item 2)
 *   sinogram        b[t][a][k],  a < na[t] angles of frame t, k < nb bins
 *   velocities      s[p][c][y][x], p < nt-1 frame pairs, c = 0 (s_x) / 1 (s_y)
 *   reverse flow    sr[p] lives on frame p+1 (s'(t+1) of Sec. 3)
 *   gradient        g[t][d][y][x], d = 0: u(x+1)-u(x), d = 1: u(y+1)-u(y);
 *                   the last column (d=0) / last row (d=1) is identically 0,
 *                   which is the rectangular L_d of eq. (L) padded with zero rows.
 *
 * Geometry (2D parallel beam): pixel centres x_i = (i - (nx-1)/2) h,
 * y_j = (j - (ny-1)/2) h; bin centres sigma_k = (k - (nb-1)/2) db; the ray of
 * angle theta and bin k is { p : x cos(theta) + y sin(theta) = sigma_k }.
 * H is the Joseph line integral along each ray, blockdiag over frames
 * (Sec. 2.1, the block-diagonal H).
 *
 * Fan beam (orc_project_fan): the same Joseph rule along the lines from a point
 * source through the bins of a flat detector (fan_line below).
 *
 * Parity pins: tests/test_oracle_ops.py (adjoint identities, theta=0/90 column
 * and row sums, analytic disk chords (parallel and fan), the far-source limit,
 * the fan magnification, bilinear = scipy map_coordinates, exact
 * integer shifts, zero residual on constants and translated linear images,
 * box stencils = scipy correlate, hand-checked reverse-flow cases).
 */
#include <math.h>
#include <stdlib.h>
#include <string.h>

/* ---------------------------------------------------------------- projector */

/* One ray, Joseph's method: march over the axis along which the ray is least
 * inclined; at each step linearly interpolate between the two pixels that
 * straddle the crossing point; weight the step by its path length h/|cos|
 * (or h/|sin|). If `scatter` is set, the transposed entry is accumulated into
 * img instead (exact transpose of the same matrix entries). */
static double joseph_ray(int nx, int ny, double h, double theta, double sigma,
                         double *img, double bval, int scatter)
{
    const double c = cos(theta), s = sin(theta);
    double acc = 0.0;
    if (fabs(c) >= fabs(s)) {
        /* step over rows j; crossing x* = (sigma - y_j s)/c */
        const double wstep = h / fabs(c);
        for (int j = 0; j < ny; ++j) {
            const double yj = (j - 0.5 * (ny - 1)) * h;
            const double xs = (sigma - yj * s) / c;
            const double fi = xs / h + 0.5 * (nx - 1); /* fractional column index */
            const double i0d = floor(fi);
            const double f = fi - i0d;
            if (i0d < -1.0 || i0d > (double)nx) continue;
            const int i0 = (int)i0d;
            double *row = img + (size_t)j * nx;
            if (i0 >= 0 && i0 < nx) {
                if (scatter) row[i0] += (1.0 - f) * wstep * bval;
                else acc += (1.0 - f) * row[i0];
            }
            if (i0 + 1 >= 0 && i0 + 1 < nx) {
                if (scatter) row[i0 + 1] += f * wstep * bval;
                else acc += f * row[i0 + 1];
            }
        }
        return acc * wstep;
    } else {
        /* step over columns i; crossing y* = (sigma - x_i c)/s */
        const double wstep = h / fabs(s);
        for (int i = 0; i < nx; ++i) {
            const double xi = (i - 0.5 * (nx - 1)) * h;
            const double ys = (sigma - xi * c) / s;
            const double fj = ys / h + 0.5 * (ny - 1);
            const double j0d = floor(fj);
            const double f = fj - j0d;
            if (j0d < -1.0 || j0d > (double)ny) continue;
            const int j0 = (int)j0d;
            if (j0 >= 0 && j0 < ny) {
                if (scatter) img[(size_t)j0 * nx + i] += (1.0 - f) * wstep * bval;
                else acc += (1.0 - f) * img[(size_t)j0 * nx + i];
            }
            if (j0 + 1 >= 0 && j0 + 1 < ny) {
                if (scatter) img[(size_t)(j0 + 1) * nx + i] += f * wstep * bval;
                else acc += f * img[(size_t)(j0 + 1) * nx + i];
            }
        }
        return acc * wstep;
    }
}

/* b = H u (block-diagonal over frames). */
void orc_project(int nx, int ny, int nt, int nb, const int *na, const double *ang,
                 double h, double db, const double *u, double *b)
{
    size_t aoff = 0;
    size_t boff = 0;
    for (int t = 0; t < nt; ++t) {
        const double *ut = u + (size_t)t * nx * ny;
        for (int a = 0; a < na[t]; ++a) {
            for (int k = 0; k < nb; ++k) {
                const double sigma = (k - 0.5 * (nb - 1)) * db;
                b[boff + (size_t)a * nb + k] =
                    joseph_ray(nx, ny, h, ang[aoff + a], sigma, (double *)ut, 0.0, 0);
            }
        }
        aoff += na[t];
        boff += (size_t)na[t] * nb;
    }
}

/* u = H^T b: the same ray entries, scattered (the transpose by construction). */
void orc_backproject(int nx, int ny, int nt, int nb, const int *na, const double *ang,
                     double h, double db, const double *b, double *u)
{
    memset(u, 0, sizeof(double) * (size_t)nx * ny * nt);
    size_t aoff = 0;
    size_t boff = 0;
    for (int t = 0; t < nt; ++t) {
        double *ut = u + (size_t)t * nx * ny;
        for (int a = 0; a < na[t]; ++a) {
            for (int k = 0; k < nb; ++k) {
                const double sigma = (k - 0.5 * (nb - 1)) * db;
                joseph_ray(nx, ny, h, ang[aoff + a], sigma, ut, b[boff + (size_t)a * nb + k], 1);
            }
        }
        aoff += na[t];
        boff += (size_t)na[t] * nb;
    }
}

/* --------------------------------------------------------- fan-beam projector */

/* 2D fan beam with a flat detector (Sec. 5.1, the experiments' geometry). The
 * view at angle theta looks along e = (-sin theta, cos theta), the direction
 * of the parallel rays of the same angle: the source is the point S = -rs e,
 * the detector the line through rd e perpendicular to e, and bin k its point
 * D_k = rd e + sigma_k (cos theta, sin theta). The ray of bin k is the line
 * through S and D_k; with the unit normal n of D_k - S it is the set
 * {x n_x + y n_y = S . n}, which the parallel-beam Joseph rule integrates. */
static void fan_line(double theta, double sigma, double rs, double rd, double *phi, double *p)
{
    const double ex = -sin(theta), ey = cos(theta);
    const double sx = -rs * ex, sy = -rs * ey;
    const double dx = rd * ex + sigma * cos(theta), dy = rd * ey + sigma * sin(theta);
    const double vx = dx - sx, vy = dy - sy;
    const double len = hypot(vx, vy);
    const double nx = vy / len, ny = -vx / len;
    *phi = atan2(ny, nx);
    *p = sx * nx + sy * ny;
}

/* b = H u for the fan beam (block-diagonal over frames). */
void orc_project_fan(int nx, int ny, int nt, int nb, const int *na, const double *ang,
                     double h, double db, double rs, double rd, const double *u, double *b)
{
    size_t aoff = 0;
    size_t boff = 0;
    for (int t = 0; t < nt; ++t) {
        const double *ut = u + (size_t)t * nx * ny;
        for (int a = 0; a < na[t]; ++a) {
            for (int k = 0; k < nb; ++k) {
                double phi, p;
                fan_line(ang[aoff + a], (k - 0.5 * (nb - 1)) * db, rs, rd, &phi, &p);
                b[boff + (size_t)a * nb + k] = joseph_ray(nx, ny, h, phi, p, (double *)ut, 0.0, 0);
            }
        }
        aoff += na[t];
        boff += (size_t)na[t] * nb;
    }
}

/* u = H^T b for the fan beam: the same ray entries, scattered. */
void orc_backproject_fan(int nx, int ny, int nt, int nb, const int *na, const double *ang,
                         double h, double db, double rs, double rd, const double *b, double *u)
{
    memset(u, 0, sizeof(double) * (size_t)nx * ny * nt);
    size_t aoff = 0;
    size_t boff = 0;
    for (int t = 0; t < nt; ++t) {
        double *ut = u + (size_t)t * nx * ny;
        for (int a = 0; a < na[t]; ++a) {
            for (int k = 0; k < nb; ++k) {
                double phi, p;
                fan_line(ang[aoff + a], (k - 0.5 * (nb - 1)) * db, rs, rd, &phi, &p);
                joseph_ray(nx, ny, h, phi, p, ut, b[boff + (size_t)a * nb + k], 1);
            }
        }
        aoff += na[t];
        boff += (size_t)na[t] * nb;
    }
}

/* ------------------------------------------------------------ spatial Psi */

/* g = Psi u: forward differences along x and y for each of nf frames
 * (eq. (L), Psi = blockdiag(L, ..., L)). */
void orc_grad(int nx, int ny, int nf, const double *u, double *g)
{
    const size_t ns = (size_t)nx * ny;
    for (int t = 0; t < nf; ++t) {
        const double *f = u + t * ns;
        double *gx = g + (size_t)(2 * t) * ns;
        double *gy = g + (size_t)(2 * t + 1) * ns;
        for (int y = 0; y < ny; ++y)
            for (int x = 0; x < nx; ++x) {
                const size_t i = (size_t)y * nx + x;
                gx[i] = (x < nx - 1) ? f[i + 1] - f[i] : 0.0;
                gy[i] = (y < ny - 1) ? f[i + nx] - f[i] : 0.0;
            }
    }
}

/* u = Psi^T g, written as the scatter of each difference row. */
void orc_gradT(int nx, int ny, int nf, const double *g, double *u)
{
    const size_t ns = (size_t)nx * ny;
    memset(u, 0, sizeof(double) * ns * nf);
    for (int t = 0; t < nf; ++t) {
        double *f = u + t * ns;
        const double *gx = g + (size_t)(2 * t) * ns;
        const double *gy = g + (size_t)(2 * t + 1) * ns;
        for (int y = 0; y < ny; ++y)
            for (int x = 0; x < nx; ++x) {
                const size_t i = (size_t)y * nx + x;
                if (x < nx - 1) { f[i + 1] += gx[i]; f[i] -= gx[i]; }
                if (y < ny - 1) { f[i + nx] += gy[i]; f[i] -= gy[i]; }
            }
    }
}

/* --------------------------------------------------------- bilinear warp */

static double clampd(double v, double lo, double hi) { return v < lo ? lo : (v > hi ? hi : v); }

/* The four taps of row (x,y) of the bilinear warp M(s) (Sec. 3, item 2):
 * sample point r + s(r), clipped to the image, its four neighbours and their
 * bilinear weights. */
static void warp_taps(int nx, int ny, int x, int y, double sx, double sy,
                      size_t idx[4], double w[4])
{
    const double X = clampd(x + sx, 0.0, nx - 1.0);
    const double Y = clampd(y + sy, 0.0, ny - 1.0);
    const int x0 = (int)floor(X), y0 = (int)floor(Y);
    const int x1 = x0 + 1 < nx ? x0 + 1 : nx - 1;
    const int y1 = y0 + 1 < ny ? y0 + 1 : ny - 1;
    const double fx = X - x0, fy = Y - y0;
    idx[0] = (size_t)y0 * nx + x0; w[0] = (1 - fx) * (1 - fy);
    idx[1] = (size_t)y0 * nx + x1; w[1] = fx * (1 - fy);
    idx[2] = (size_t)y1 * nx + x0; w[2] = (1 - fx) * fy;
    idx[3] = (size_t)y1 * nx + x1; w[3] = fx * fy;
}

/* out = M(s) v for one frame. */
void orc_warp(int nx, int ny, const double *v, const double *sx, const double *sy, double *out)
{
    for (int y = 0; y < ny; ++y)
        for (int x = 0; x < nx; ++x) {
            const size_t i = (size_t)y * nx + x;
            size_t idx[4]; double w[4];
            warp_taps(nx, ny, x, y, sx[i], sy[i], idx, w);
            out[i] = w[0] * v[idx[0]] + w[1] * v[idx[1]] + w[2] * v[idx[2]] + w[3] * v[idx[3]];
        }
}

/* out += M(s)^T r for one frame (scatter of the same taps). */
static void warpT_add(int nx, int ny, const double *r, const double *sx, const double *sy,
                      double scale, double *out)
{
    for (int y = 0; y < ny; ++y)
        for (int x = 0; x < nx; ++x) {
            const size_t i = (size_t)y * nx + x;
            size_t idx[4]; double w[4];
            warp_taps(nx, ny, x, y, sx[i], sy[i], idx, w);
            for (int q = 0; q < 4; ++q) out[idx[q]] += scale * w[q] * r[i];
        }
}

void orc_warpT(int nx, int ny, const double *r, const double *sx, const double *sy, double *out)
{
    memset(out, 0, sizeof(double) * (size_t)nx * ny);
    warpT_add(nx, ny, r, sx, sy, 1.0, out);
}

/* r = Mhat(s, s') u (Sec. 3: the block rows of Mbar and Mbar', stacked as in
 * Sec. 4). Layout r[2][nt-1][ny][nx]:
 *   r[0][p] = u_p     - M(s_p)  u_{p+1}     (Mbar,  forward rows)
 *   r[1][p] = u_{p+1} - M(sr_p) u_p         (Mbar', reverse rows; sr_p = s'(p+1)) */
void orc_flow(int nx, int ny, int nt, const double *u, const double *s, const double *sr, double *r)
{
    const size_t ns = (size_t)nx * ny;
    const int np = nt - 1;
    double *tmp = (double *)malloc(sizeof(double) * ns);
    for (int p = 0; p < np; ++p) {
        const double *u0 = u + p * ns, *u1 = u + (p + 1) * ns;
        const double *sp = s + (size_t)(2 * p) * ns, *srp = sr + (size_t)(2 * p) * ns;
        double *rf = r + (size_t)p * ns, *rb = r + (size_t)(np + p) * ns;
        orc_warp(nx, ny, u1, sp, sp + ns, tmp);
        for (size_t i = 0; i < ns; ++i) rf[i] = u0[i] - tmp[i];
        orc_warp(nx, ny, u0, srp, srp + ns, tmp);
        for (size_t i = 0; i < ns; ++i) rb[i] = u1[i] - tmp[i];
    }
    free(tmp);
}

/* u = Mhat(s, s')^T r. */
void orc_flowT(int nx, int ny, int nt, const double *r, const double *s, const double *sr, double *u)
{
    const size_t ns = (size_t)nx * ny;
    const int np = nt - 1;
    memset(u, 0, sizeof(double) * ns * nt);
    for (int p = 0; p < np; ++p) {
        double *u0 = u + p * ns, *u1 = u + (p + 1) * ns;
        const double *sp = s + (size_t)(2 * p) * ns, *srp = sr + (size_t)(2 * p) * ns;
        const double *rf = r + (size_t)p * ns, *rb = r + (size_t)(np + p) * ns;
        for (size_t i = 0; i < ns; ++i) { u0[i] += rf[i]; u1[i] += rb[i]; }
        warpT_add(nx, ny, rf, sp, sp + ns, -1.0, u1);
        warpT_add(nx, ny, rb, srp, srp + ns, -1.0, u0);
    }
}

/* ------------------------------------------------ optical-flow derivatives */

/* Reflect an index into [0, n) by flipping the image about its edge
 * (App. C: "the image is flipped to complete the box"; edge sample repeated). */
static int reflect(int i, int n)
{
    while (i < 0 || i >= n) {
        if (i < 0) i = -i - 1;
        if (i >= n) i = 2 * n - 1 - i;
    }
    return i;
}

/* Box-averaged derivative fields of App. C for every pair p = (u_p, u_{p+1}):
 *   ux[p](x,y) = 1/(2dr+1) sum_k [u_p(x+dr, y+k) - u_p(x-dr, y+k)] / (2dr)
 *   uy[p](x,y) = 1/(2dr+1) sum_k [u_p(x+k, y+dr) - u_p(x+k, y-dr)] / (2dr)
 *   ut[p](x,y) = 1/(2dr+1)^2 sum_{j,k} [u_{p+1}(x+j, y+k) - u_p(x+j, y+k)]
 * with reflected boundary and unit time step. */
void orc_of_fields(int nx, int ny, int nt, int dr, const double *u,
                   double *ux, double *uy, double *ut)
{
    const size_t ns = (size_t)nx * ny;
    const double box = 2.0 * dr + 1.0;
    for (int p = 0; p < nt - 1; ++p) {
        const double *a = u + p * ns, *b = u + (p + 1) * ns;
        double *gx = ux + p * ns, *gy = uy + p * ns, *gt = ut + p * ns;
        for (int y = 0; y < ny; ++y)
            for (int x = 0; x < nx; ++x) {
                double sx = 0, sy = 0, st = 0;
                for (int k = -dr; k <= dr; ++k) {
                    const int yk = reflect(y + k, ny), xk = reflect(x + k, nx);
                    sx += (a[(size_t)yk * nx + reflect(x + dr, nx)] - a[(size_t)yk * nx + reflect(x - dr, nx)]) / (2.0 * dr);
                    sy += (a[(size_t)reflect(y + dr, ny) * nx + xk] - a[(size_t)reflect(y - dr, ny) * nx + xk]) / (2.0 * dr);
                    for (int j = -dr; j <= dr; ++j) {
                        const size_t q = (size_t)yk * nx + reflect(x + j, nx);
                        st += b[q] - a[q];
                    }
                }
                const size_t i = (size_t)y * nx + x;
                gx[i] = sx / box;
                gy[i] = sy / box;
                gt[i] = st / (box * box);
            }
    }
}

/* r = Upsilon s + u_t per pair (Sec. 2.2: the pointwise row [u_x u_y]). */
void orc_flow_lin(int nx, int ny, int np, const double *ux, const double *uy, const double *ut,
                  const double *s, double *r)
{
    const size_t ns = (size_t)nx * ny;
    for (int p = 0; p < np; ++p)
        for (size_t i = 0; i < ns; ++i) {
            const size_t q = p * ns + i;
            r[q] = ux[q] * s[(size_t)(2 * p) * ns + i] + uy[q] * s[(size_t)(2 * p + 1) * ns + i] + ut[q];
        }
}

/* gs = Upsilon^T r per pair. */
void orc_flow_linT(int nx, int ny, int np, const double *ux, const double *uy, const double *r,
                   double *gs)
{
    const size_t ns = (size_t)nx * ny;
    for (int p = 0; p < np; ++p)
        for (size_t i = 0; i < ns; ++i) {
            const size_t q = p * ns + i;
            gs[(size_t)(2 * p) * ns + i] = ux[q] * r[q];
            gs[(size_t)(2 * p + 1) * ns + i] = uy[q] * r[q];
        }
}

/* ------------------------------------------------------------ reverse flow */

/* s'(p+1) from s(p) by the Remark of Sec. 3: the pixel at r moves to
 * round(r + s(r)) (half away from zero, clipped to the image) and carries the
 * velocity -s(r) there. Several arrivals are averaged; pixels nothing arrives
 * at get 0. Sources are visited in row-major order. */
void orc_reverse_flow(int nx, int ny, int nt, const double *s, double *sr)
{
    const size_t ns = (size_t)nx * ny;
    double *cnt = (double *)malloc(sizeof(double) * ns);
    for (int p = 0; p < nt - 1; ++p) {
        const double *sx = s + (size_t)(2 * p) * ns, *sy = sx + ns;
        double *rx = sr + (size_t)(2 * p) * ns, *ry = rx + ns;
        memset(cnt, 0, sizeof(double) * ns);
        memset(rx, 0, sizeof(double) * ns);
        memset(ry, 0, sizeof(double) * ns);
        for (int y = 0; y < ny; ++y)
            for (int x = 0; x < nx; ++x) {
                const size_t i = (size_t)y * nx + x;
                const int dx = (int)clampd(round((double)x + sx[i]), 0.0, nx - 1.0);
                const int dy = (int)clampd(round((double)y + sy[i]), 0.0, ny - 1.0);
                const size_t d = (size_t)dy * nx + dx;
                rx[d] -= sx[i];
                ry[d] -= sy[i];
                cnt[d] += 1.0;
            }
        for (size_t i = 0; i < ns; ++i)
            if (cnt[i] > 0) { rx[i] /= cnt[i]; ry[i] /= cnt[i]; }
    }
    free(cnt);
}

/* Velocity derivative of the bilinear sample B(v; X, Y) at the clipped point
 * X = clamp(x + sx, 0, nx-1), Y = clamp(y + sy, 0, ny-1) of warp_taps: on the
 * cell (floor X, floor Y) the interpolant is bilinear, so
 *   dB/dsx = (1 - fy) (v01 - v00) + fy (v11 - v10),
 *   dB/dsy = (1 - fx) (v10 - v00) + fx (v11 - v01),
 * taken on the cell floor(X) (the right derivative where x + sx is an integer),
 * and zero along an axis where the clamp holds the sample point (x + sx < 0 or
 * x + sx >= nx - 1: there the sample does not move with sx). */
static void warp_grad(int nx, int ny, int x, int y, double sx, double sy, const double *v, double *gx, double *gy)
{
    const double Xu = x + sx, Yu = y + sy;
    const double X = clampd(Xu, 0.0, nx - 1.0), Y = clampd(Yu, 0.0, ny - 1.0);
    const int x0 = (int)floor(X), y0 = (int)floor(Y);
    const int x1 = x0 + 1 < nx ? x0 + 1 : nx - 1;
    const int y1 = y0 + 1 < ny ? y0 + 1 : ny - 1;
    const double fx = X - x0, fy = Y - y0;
    const double v00 = v[(size_t)y0 * nx + x0], v01 = v[(size_t)y0 * nx + x1];
    const double v10 = v[(size_t)y1 * nx + x0], v11 = v[(size_t)y1 * nx + x1];
    *gx = (Xu >= 0.0 && Xu < nx - 1.0) ? (1 - fy) * (v01 - v00) + fy * (v11 - v10) : 0.0;
    *gy = (Yu >= 0.0 && Yu < ny - 1.0) ? (1 - fx) * (v10 - v00) + fx * (v11 - v01) : 0.0;
}

/* Vector-Jacobian product of r = Mhat(s, s') u (orc_flow) with respect to the
 * velocities, for a cotangent gr[2][nt-1][ny][nx]: since
 * r[0][p] = u_p - B(u_{p+1}; x + s_p) and r[1][p] = u_{p+1} - B(u_p; x + sr_p),
 *   gs[p]  = -gr[0][p] * grad B(u_{p+1}; x + s_p)   (components x, y),
 *   gsr[p] = -gr[1][p] * grad B(u_p;     x + sr_p).
 * Layouts of s: gs, gsr [nt-1][2][ny][nx]. */
void orc_flow_ds(int nx, int ny, int nt, const double *u, const double *s, const double *sr, const double *gr,
                 double *gs, double *gsr)
{
    const size_t ns = (size_t)nx * ny;
    const int np = nt - 1;
    for (int p = 0; p < np; ++p) {
        const double *u0 = u + p * ns, *u1 = u + (p + 1) * ns;
        const double *sp = s + (size_t)(2 * p) * ns, *srp = sr + (size_t)(2 * p) * ns;
        const double *g0 = gr + (size_t)p * ns, *g1 = gr + (size_t)(np + p) * ns;
        double *os = gs + (size_t)(2 * p) * ns, *osr = gsr + (size_t)(2 * p) * ns;
        for (int y = 0; y < ny; ++y)
            for (int x = 0; x < nx; ++x) {
                const size_t i = (size_t)y * nx + x;
                double gx, gy;
                warp_grad(nx, ny, x, y, sp[i], sp[ns + i], u1, &gx, &gy);
                os[i] = -g0[i] * gx;
                os[ns + i] = -g0[i] * gy;
                warp_grad(nx, ny, x, y, srp[i], srp[ns + i], u0, &gx, &gy);
                osr[i] = -g1[i] * gx;
                osr[ns + i] = -g1[i] * gy;
            }
    }
}
