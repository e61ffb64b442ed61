"""Pins of the FP64 oracle operators against what the paper and mathematics fix.

Each test checks the oracle against something other than itself: closed forms
(parallel-beam chords of a disk, exact shifts, linear reproduction), library
routines (scipy.ndimage bilinear interpolation and correlation, numpy kron),
brute-force matrices, and invariants (adjoint identities, zero residuals).
"""
import numpy as np
import pytest
from scipy import ndimage

from oracle import ops
from paper_2501_12497_gb300 import synth


def rel(a, b):
    return np.linalg.norm(np.ravel(a) - np.ravel(b)) / max(np.linalg.norm(np.ravel(b)), 1e-300)


def geom(nx, ny, nt, nb, na, seed=0, h=1.0, db=1.0):
    rng = np.random.default_rng(seed)
    na_arr = np.full(nt, na, dtype=np.int32)
    ang = rng.uniform(0, 2 * np.pi, size=int(na_arr.sum()))
    return ops.Geometry(nx, ny, nt, nb, na_arr, ang, h, db)


# ------------------------------------------------------------------- H, H^T

def test_projector_adjoint_identity():
    """<H u, b> = <u, H^T b> (H^T is the transpose of the same entries)."""
    g = geom(13, 9, 3, 17, 5)
    rng = np.random.default_rng(1)
    u = rng.standard_normal((3, 9, 13))
    b = rng.standard_normal(g.m)
    lhs = np.dot(ops.project(g, u), b)
    rhs = np.dot(u.ravel(), ops.backproject(g, b).ravel())
    assert abs(lhs - rhs) <= 1e-13 * abs(lhs) + 1e-12


def test_projector_theta0_is_column_sums():
    """theta = 0 with bins on pixel centres: ray k integrates image column x = k."""
    n = 12
    g = ops.Geometry(n, 9, 1, n, [1], [0.0])
    u = np.random.default_rng(2).standard_normal((1, 9, n))
    np.testing.assert_allclose(ops.project(g, u), u[0].sum(axis=0), rtol=1e-13, atol=1e-13)


def test_projector_theta90_is_row_sums():
    """theta = 90 deg: ray k integrates image row y = k."""
    n = 10
    g = ops.Geometry(7, n, 1, n, [1], [np.pi / 2])
    u = np.random.default_rng(3).standard_normal((1, n, 7))
    np.testing.assert_allclose(ops.project(g, u), u[0].sum(axis=1), rtol=1e-12, atol=1e-12)


def test_projector_entries_match_pixel_footprint():
    """Every Joseph entry equals the pixel-side footprint (h/mu) max(0, 1 - |sigma - p|/(mu h)),
    p = x_i cos + y_j sin, mu = max(|cos|, |sin|): built column by column from H e_pixel."""
    nx, ny, nb = 6, 5, 11
    h, db = 1.3, 0.9
    ang = np.array([0.1, 0.7, 1.2, 2.0, 2.9, 3.9, 5.5, np.pi / 4])
    g = ops.Geometry(nx, ny, 1, nb, [len(ang)], ang, h, db)
    sig = (np.arange(nb) - 0.5 * (nb - 1)) * db
    for j in range(ny):
        for i in range(nx):
            e = np.zeros((1, ny, nx))
            e[0, j, i] = 1.0
            col = ops.project(g, e).reshape(len(ang), nb)
            x, y = (i - 0.5 * (nx - 1)) * h, (j - 0.5 * (ny - 1)) * h
            for a, th in enumerate(ang):
                c, s = np.cos(th), np.sin(th)
                mu = max(abs(c), abs(s))
                p = x * c + y * s
                want = (h / mu) * np.maximum(0.0, 1.0 - np.abs(sig - p) / (mu * h))
                np.testing.assert_allclose(col[a], want, rtol=1e-12, atol=1e-12)


def test_projector_converges_to_disk_chords():
    """H applied to the area-averaged raster of a disk tends to the analytic chord
    2 rho sqrt(r^2 - sigma'^2) as the grid is refined (textbook Radon transform)."""
    errs = []
    e = (1.3, -0.7, 10.0, 10.0, 0.0, 0.8)
    ang = np.deg2rad(np.array([0.0, 17.0, 45.0, 71.0, 123.0]))
    for h in (1.0, 0.5, 0.25):
        n = int(round(32 / h))
        g = ops.Geometry(n, n, 1, n, [len(ang)], ang, h, h)
        img = synth.raster([e], n, n, h)
        sig = (np.arange(n) - 0.5 * (n - 1)) * h
        exact = synth.ellipse_radon(e, ang[:, None], sig[None, :]).ravel()
        errs.append(rel(ops.project(g, img[None]), exact))
    assert errs[0] < 0.03 and errs[2] < 0.006
    assert errs[1] < 0.75 * errs[0] and errs[2] < 0.75 * errs[1]


# ------------------------------------------------------- fan-beam H, H^T
def _fan_source_and_bins(theta, nb, db, rs, rd):
    """Source S and detector points D_k of one view, written from the geometry: the view
    looks along e = (-sin, cos), S = -rs e, D_k = rd e + sigma_k (cos, sin)."""
    e = np.array([-np.sin(theta), np.cos(theta)])
    f = np.array([np.cos(theta), np.sin(theta)])
    sig = (np.arange(nb) - 0.5 * (nb - 1)) * db
    return -rs * e, rd * e[None, :] + sig[:, None] * f[None, :]


def test_fan_projector_adjoint_identity():
    g = geom(23, 19, 2, 41, 5, seed=11)
    g.fan = (40.0, 25.0)
    rng = np.random.default_rng(12)
    u = rng.standard_normal((2, 19, 23))
    b = rng.standard_normal(g.m)
    lhs = ops.project(g, u) @ b
    rhs = np.sum(u * ops.backproject(g, b))
    assert abs(lhs - rhs) <= 1e-12 * max(abs(lhs), 1.0)


def test_fan_projector_converges_to_disk_chords():
    """H (fan beam) applied to the raster of an off-centre disk tends to the exact chord
    2 rho sqrt(r^2 - d^2), d the distance of the disk centre from the line through the
    source and the bin (cross product), as the grid is refined. Views include fans that
    straddle 45 degrees (rays of one view stepping along both axes)."""
    cx, cy, r, rho = 4.1, -2.7, 8.0, 0.8
    e = (cx, cy, r, r, 0.0, rho)
    ang = np.deg2rad(np.array([0.0, 40.0, 45.0, 131.0, 222.0, 300.0]))
    rs, rd = 60.0, 30.0
    errs = []
    for h in (1.0, 0.5, 0.25):
        n = int(round(32 / h))
        nb = int(round(1.6 * n))
        db = 1.5 * h
        g = ops.Geometry(n, n, 1, nb, [len(ang)], ang, h, db, fan=(rs, rd))
        img = synth.raster([e], n, n, h)
        exact = []
        for th in ang:
            S, D = _fan_source_and_bins(th, nb, db, rs, rd)
            v = D - S
            w = np.array([cx, cy]) - S
            d = np.abs(v[:, 0] * w[1] - v[:, 1] * w[0]) / np.hypot(v[:, 0], v[:, 1])
            exact.append(np.where(d < r, 2 * rho * np.sqrt(np.maximum(r * r - d * d, 0.0)), 0.0))
        errs.append(rel(ops.project(g, img[None]), np.concatenate(exact)))
    assert errs[0] < 0.03 and errs[2] < 0.01, errs
    assert errs[1] < 0.75 * errs[0] and errs[2] < 0.75 * errs[1], errs


def test_fan_projector_far_source_is_parallel():
    """A source a million image widths away with the detector through the centre gives
    the parallel-beam projector of the same angles."""
    g = geom(21, 17, 2, 35, 4, seed=13)
    rng = np.random.default_rng(14)
    u = rng.standard_normal((2, 17, 21))
    par = ops.project(g, u)
    g.fan = (2e7, 0.0)
    assert rel(ops.project(g, u), par) < 1e-5


@pytest.mark.parametrize("pix", [(16, 16), (26, 9), (5, 27)])
def test_fan_projector_point_lands_at_its_magnified_position(pix):
    """A single pixel projects to a footprint centred on the detector coordinate of the
    ray through its centre: sigma = sdd ((p - S) . f) / ((p - S) . e) (central projection
    from the source onto the detector line)."""
    n, nb, db, rs, rd = 33, 121, 0.5, 50.0, 20.0
    ang = np.deg2rad(np.array([0.0, 33.0, 90.0, 160.0]))
    g = ops.Geometry(n, n, 1, nb, [len(ang)], ang, 1.0, db, fan=(rs, rd))
    u = np.zeros((1, n, n))
    i, j = pix
    u[0, j, i] = 1.0
    b = ops.project(g, u).reshape(len(ang), nb)
    p = np.array([i - 0.5 * (n - 1), j - 0.5 * (n - 1)])
    for a, th in enumerate(ang):
        e = np.array([-np.sin(th), np.cos(th)])
        f = np.array([np.cos(th), np.sin(th)])
        q = p + rs * e
        sigma = (rs + rd) * (q @ f) / (q @ e)
        t = sigma / db + 0.5 * (nb - 1)
        cen = np.sum(np.arange(nb) * b[a]) / np.sum(b[a])
        assert abs(cen - t) < 0.05, (a, cen, t)


# ---------------------------------------------------------------- Psi, Psi^T

def test_grad_zero_on_constants_and_constant_on_ramps():
    u = np.full((2, 6, 7), 3.25)
    assert np.all(ops.grad(u) == 0.0)
    yy, xx = np.meshgrid(np.arange(6), np.arange(7), indexing="ij")
    ramp = (0.5 * xx - 2.0 * yy + 1.0)[None]
    gr = ops.grad(ramp)
    np.testing.assert_allclose(gr[0, 0, :, :-1], 0.5, atol=1e-14)
    np.testing.assert_allclose(gr[0, 1, :-1, :], -2.0, atol=1e-14)
    assert np.all(gr[0, 0, :, -1] == 0) and np.all(gr[0, 1, -1, :] == 0)


def test_grad_equals_kronecker_form():
    """Psi for one frame equals the stacked Kronecker form of eq. (L)
    [I (x) D_x ; D_y (x) I] (x fastest), D the forward difference padded by a zero row."""
    nx, ny = 5, 4

    def D(n):
        d = np.zeros((n, n))
        for i in range(n - 1):
            d[i, i], d[i, i + 1] = -1.0, 1.0
        return d

    Psi = np.vstack([np.kron(np.eye(ny), D(nx)), np.kron(D(ny), np.eye(nx))])
    cols = []
    for q in range(nx * ny):
        e = np.zeros(nx * ny)
        e[q] = 1.0
        cols.append(ops.grad(e.reshape(1, ny, nx)).ravel())
    np.testing.assert_array_equal(np.array(cols).T, Psi)


def test_grad_adjoint_identity():
    rng = np.random.default_rng(4)
    u = rng.standard_normal((3, 7, 9))
    g = rng.standard_normal((3, 2, 7, 9))
    assert abs(np.vdot(ops.grad(u), g) - np.vdot(u, ops.gradT(g))) < 1e-12


# --------------------------------------------------------------- M(s), Mhat

def test_warp_zero_velocity_is_identity():
    v = np.random.default_rng(5).standard_normal((8, 9))
    z = np.zeros_like(v)
    np.testing.assert_array_equal(ops.warp(v, z, z), v)


def test_warp_integer_velocity_is_shift():
    """Integer s gives the exact shift of Sec. 3 eq. (m_matrix) away from the clipped border."""
    v = np.random.default_rng(6).standard_normal((10, 12))
    sx, sy = np.full_like(v, 2.0), np.full_like(v, -1.0)
    out = ops.warp(v, sx, sy)
    np.testing.assert_array_equal(out[1:, :-2], v[:-1, 2:])


def test_warp_matches_scipy_bilinear():
    """M(s) v equals scipy's order-1 map_coordinates with edge extension (clipped samples)."""
    rng = np.random.default_rng(7)
    v = rng.standard_normal((11, 14))
    sx = rng.uniform(-3.5, 3.5, v.shape)
    sy = rng.uniform(-3.5, 3.5, v.shape)
    yy, xx = np.meshgrid(np.arange(11), np.arange(14), indexing="ij")
    want = ndimage.map_coordinates(v, [yy + sy, xx + sx], order=1, mode="nearest")
    np.testing.assert_allclose(ops.warp(v, sx, sy), want, rtol=1e-12, atol=1e-12)


def test_warp_reproduces_translated_linear_image():
    """Bilinear interpolation is exact on linear functions: for u_{t+1}(r) = f(r - s) with f
    linear, M(s) u_{t+1} = u_t wherever r + s stays inside the grid."""
    ny, nx = 12, 13
    yy, xx = np.meshgrid(np.arange(ny), np.arange(nx), indexing="ij")
    f = lambda x, y: 0.3 * x - 0.7 * y + 2.0
    s = (0.37, -1.21)
    u0, u1 = f(xx, yy), f(xx - s[0], yy - s[1])
    out = ops.warp(u1, np.full_like(u0, s[0]), np.full_like(u0, s[1]))
    inside = (xx + s[0] >= 0) & (xx + s[0] <= nx - 1) & (yy + s[1] >= 0) & (yy + s[1] <= ny - 1)
    np.testing.assert_allclose(out[inside], u0[inside], atol=1e-13)


def test_warp_adjoint_identity():
    rng = np.random.default_rng(8)
    v, r = rng.standard_normal((2, 9, 10))
    sx, sy = rng.uniform(-2.5, 2.5, (2, 9, 10))
    assert abs(np.vdot(ops.warp(v, sx, sy), r) - np.vdot(v, ops.warpT(r, sx, sy))) < 1e-12


def test_flow_zero_on_constant_sequences():
    """Weights of every warp row sum to 1, so Mhat annihilates constant sequences for any s, s'."""
    nt, ny, nx = 4, 8, 9
    u = np.full((nt, ny, nx), -1.75)
    s = synth.random_velocities(nt - 1, ny, nx, 3.0, seed=9)
    sr = synth.random_velocities(nt - 1, ny, nx, 3.0, seed=10)
    assert np.max(np.abs(ops.flow(u, s, sr))) < 1e-14


def test_flow_block_rows():
    """Row blocks of Mbar and Mbar' (Sec. 3): r[0,p] = u_p - M(s_p) u_{p+1},
    r[1,p] = u_{p+1} - M(s'_{p+1}) u_p, checked against scipy's bilinear interpolation."""
    rng = np.random.default_rng(11)
    nt, ny, nx = 3, 7, 8
    u = rng.standard_normal((nt, ny, nx))
    s = rng.uniform(-2, 2, (nt - 1, 2, ny, nx))
    sr = rng.uniform(-2, 2, (nt - 1, 2, ny, nx))
    yy, xx = np.meshgrid(np.arange(ny), np.arange(nx), indexing="ij")
    bil = lambda img, v: ndimage.map_coordinates(img, [yy + v[1], xx + v[0]], order=1, mode="nearest")
    r = ops.flow(u, s, sr)
    for p in range(nt - 1):
        np.testing.assert_allclose(r[0, p], u[p] - bil(u[p + 1], s[p]), atol=1e-12)
        np.testing.assert_allclose(r[1, p], u[p + 1] - bil(u[p], sr[p]), atol=1e-12)


def test_flow_adjoint_identity():
    rng = np.random.default_rng(12)
    nt, ny, nx = 5, 9, 7
    u = rng.standard_normal((nt, ny, nx))
    r = rng.standard_normal((2, nt - 1, ny, nx))
    s = rng.uniform(-3, 3, (nt - 1, 2, ny, nx))
    sr = rng.uniform(-3, 3, (nt - 1, 2, ny, nx))
    lhs = np.vdot(ops.flow(u, s, sr), r)
    rhs = np.vdot(u, ops.flowT(r, s, sr))
    assert abs(lhs - rhs) <= 1e-12 * max(1.0, abs(lhs))


# ------------------------------------------------- App. C fields, Upsilon

def test_of_fields_match_scipy_correlate():
    """u_x, u_y, u_t equal correlations with the App. C box kernels under scipy's 'reflect'
    boundary (the image flipped about its edge)."""
    rng = np.random.default_rng(13)
    for dr in (1, 2):
        u = rng.standard_normal((2, 9, 11))
        ux, uy, ut = ops.of_fields(u, dr)
        w = 2 * dr + 1
        kx = np.zeros((w, w))
        kx[:, -1], kx[:, 0] = 1.0 / (2 * dr * w), -1.0 / (2 * dr * w)
        ky = kx.T.copy()
        kt = np.full((w, w), 1.0 / (w * w))
        np.testing.assert_allclose(ux[0], ndimage.correlate(u[0], kx, mode="reflect"), atol=1e-13)
        np.testing.assert_allclose(uy[0], ndimage.correlate(u[0], ky, mode="reflect"), atol=1e-13)
        np.testing.assert_allclose(ut[0], ndimage.correlate(u[1] - u[0], kt, mode="reflect"), atol=1e-13)


def test_of_fields_zero_on_constants():
    ux, uy, ut = ops.of_fields(np.full((3, 6, 5), 2.5), 1)
    assert np.max(np.abs(ux)) == 0 and np.max(np.abs(uy)) == 0 and np.max(np.abs(ut)) == 0


def test_flow_residual_exact_for_translated_linear_image():
    """A linear image translated by s has Upsilon s + u_t = 0 exactly away from the border
    (the OFC linearisation of Sec. 2.2 is exact and the stencils reproduce linear functions)."""
    ny, nx, dr = 14, 15, 1
    yy, xx = np.meshgrid(np.arange(ny), np.arange(nx), indexing="ij")
    f = lambda x, y: 1.1 * x + 0.4 * y - 3.0
    sx, sy = 0.63, -0.41
    u = np.stack([f(xx, yy), f(xx - sx, yy - sy)])
    ux, uy, ut = ops.of_fields(u, dr)
    s = np.stack([np.full((ny, nx), sx), np.full((ny, nx), sy)])[None]
    r = ops.flow_lin(ux, uy, ut, s)[0]
    np.testing.assert_allclose(r[dr:-dr, dr:-dr], 0.0, atol=1e-13)
    np.testing.assert_allclose(ux[0, dr:-dr, dr:-dr], 1.1, atol=1e-13)
    np.testing.assert_allclose(uy[0, dr:-dr, dr:-dr], 0.4, atol=1e-13)


def test_flow_residual_second_order_for_translating_blob():
    """Smooth blob moving with its true velocity: the interior residual of Upsilon s + u_t falls
    like h^2 as the grid is refined (central differences and the first-order Taylor step of
    Sec. 2.2 are both second order in the pixel size)."""
    errs, hs = [], [1.0, 0.5, 0.25]
    v = (0.8, -0.5)  # pixels per frame at every resolution: dt proportional to h
    for h in hs:
        n = int(round(40 / h))
        c = (np.arange(n) - 0.5 * (n - 1)) * h
        Y, X = np.meshgrid(c, c, indexing="ij")
        blob = lambda x, y: np.exp(-((x - 1.0) ** 2 + (y + 2.0) ** 2) / (2 * 5.0 ** 2))
        u = np.stack([blob(X, Y), blob(X - v[0] * h, Y - v[1] * h)])
        ux, uy, ut = ops.of_fields(u, 1)
        s = np.stack([np.full((n, n), v[0]), np.full((n, n), v[1])])[None]
        r = ops.flow_lin(ux, uy, ut, s)[0]
        k = n // 4
        errs.append(np.max(np.abs(r[k:-k, k:-k])))
    slopes = np.diff(np.log(errs)) / np.diff(np.log(hs))
    assert np.all(slopes > 1.8), (errs, slopes)


def test_flow_lin_adjoint_identity():
    rng = np.random.default_rng(14)
    ux, uy, ut = rng.standard_normal((3, 2, 6, 7))
    s = rng.standard_normal((2, 2, 6, 7))
    r = rng.standard_normal((2, 6, 7))
    lin = ops.flow_lin(ux, uy, np.zeros_like(ut), s)
    assert abs(np.vdot(lin, r) - np.vdot(s, ops.flow_linT(ux, uy, r))) < 1e-12
    np.testing.assert_allclose(ops.flow_lin(ux, uy, ut, s) - lin, ut, atol=1e-14)


def test_vgrad_is_gradient_of_each_component():
    rng = np.random.default_rng(15)
    s = rng.standard_normal((3, 2, 5, 6))
    gs = ops.vgrad(s)
    for p in range(3):
        for c in range(2):
            np.testing.assert_array_equal(gs[p, c], ops.grad(s[p, c][None])[0])
    g2 = rng.standard_normal(gs.shape)
    assert abs(np.vdot(gs, g2) - np.vdot(s, ops.vgradT(g2))) < 1e-12


# -------------------------------------------------------------- reverse flow

def test_reverse_flow_integer_shift():
    """s = (+1, 0): every pixel lands one column right; the last column receives two arrivals
    (clipped), the first column none (hole -> 0)."""
    ny, nx = 4, 6
    s = np.zeros((1, 2, ny, nx))
    s[0, 0] = 1.0
    sr = ops.reverse_flow(s)
    np.testing.assert_array_equal(sr[0, 0, :, 1:], -1.0)
    np.testing.assert_array_equal(sr[0, 0, :, 0], 0.0)
    np.testing.assert_array_equal(sr[0, 1], 0.0)


def test_reverse_flow_rounding_and_averaging():
    """Half-way positions round away from zero; arrivals at one pixel are averaged."""
    s = np.zeros((1, 2, 1, 5))
    s[0, 0, 0] = [0.5, -0.5, 0.4, 1.6, -0.5]
    # destinations: round(0.5)=1, round(0.5)=1, round(2.4)=2, round(4.6)=5->4, round(3.5)=4
    sr = ops.reverse_flow(s)
    np.testing.assert_allclose(sr[0, 0, 0], [0.0, -(0.5 - 0.5) / 2, -0.4, 0.0, -(1.6 - 0.5) / 2])
    s2 = np.zeros((1, 2, 1, 3))
    s2[0, 0, 0] = [-0.5, 0.0, 0.0]   # round(-0.5) = -1 -> clipped to 0
    np.testing.assert_allclose(ops.reverse_flow(s2)[0, 0, 0], [0.5, 0.0, 0.0])


def _smooth_velocities(npairs, ny, nx, seed, vmax=2.5):
    """Velocities whose sample points x + s keep 0.02 away from every integer and
    from the clamp, so a central difference of step 1e-6 never crosses a kink."""
    rng = np.random.default_rng(seed)
    s = rng.uniform(-vmax, vmax, size=(npairs, 2, ny, nx))
    frac = s - np.floor(s)
    s = np.where(frac < 0.02, s + 0.02, s)
    s = np.where(frac > 0.98, s - 0.02, s)
    return s


def test_flow_velocity_vjp_matches_central_differences():
    """The velocity VJP of Mhat(s, s')u against FP64 central differences of
    <gr, Mhat(s, s')u> along random directions (step 1e-6), sample points both
    inside the grid and clipped at its edges (zero derivative there)."""
    nt, ny, nx = 4, 13, 17
    u = synth.random_images(nt, ny, nx, seed=31)
    s = _smooth_velocities(nt - 1, ny, nx, seed=32)
    sr = _smooth_velocities(nt - 1, ny, nx, seed=33)
    rng = np.random.default_rng(34)
    gr = rng.standard_normal((2, nt - 1, ny, nx))
    gs, gsr = ops.flow_ds(u, s, sr, gr)
    loss = lambda s_, sr_: float(np.sum(gr * ops.flow(u, s_, sr_)))
    h = 1e-6
    for k in range(6):
        ds = rng.standard_normal(s.shape)
        dsr = rng.standard_normal(sr.shape)
        fd = (loss(s + h * ds, sr + h * dsr) - loss(s - h * ds, sr - h * dsr)) / (2 * h)
        an = float(np.sum(gs * ds) + np.sum(gsr * dsr))
        assert abs(fd - an) <= 1e-7 * max(1.0, abs(an)), (k, fd, an)


def test_flow_velocity_vjp_is_zero_where_the_sample_is_clipped():
    nt, ny, nx = 3, 8, 9
    u = synth.random_images(nt, ny, nx, seed=35)
    s = np.full((nt - 1, 2, ny, nx), 50.0)  # every sample point beyond the far edge
    sr = np.full((nt - 1, 2, ny, nx), -50.0)  # and beyond the near edge
    gr = np.ones((2, nt - 1, ny, nx))
    gs, gsr = ops.flow_ds(u, s, sr, gr)
    assert np.all(gs == 0) and np.all(gsr == 0)


def test_flow_velocity_vjp_of_a_linear_image_is_its_slope():
    """For u = a x + b y + c every interior bilinear sample moves with slope (a, b),
    so gs = -gr (a, b) wherever the sample point is not clipped."""
    nt, ny, nx = 2, 10, 12
    a, b = 0.7, -1.3
    yy, xx = np.mgrid[0:ny, 0:nx]
    u = np.stack([a * xx + b * yy + 0.5] * nt).astype(float)
    s = np.full((1, 2, ny, nx), 0.37)
    gr = np.ones((2, 1, ny, nx))
    gs, _ = ops.flow_ds(u, s, s, gr)
    inside = (xx + 0.37 < nx - 1) & (yy + 0.37 < ny - 1)
    np.testing.assert_allclose(gs[0, 0][inside], -a, atol=1e-12)
    np.testing.assert_allclose(gs[0, 1][inside], -b, atol=1e-12)


# ------------------------------------------------------------ rescaling for Solve-OF
@pytest.mark.parametrize("a", [2, 4])
def test_downsample_block_means_of_constants_and_ramps(a):
    """Block means: a constant stays constant; a linear ramp c0 + cx x + cy y goes to the
    ramp at the block centres, c0 + cx (a X + (a-1)/2) + cy (a Y + (a-1)/2); the total
    mass is kept (sum of the coarse frame times a^2)."""
    nt, ny, nx = 2, 4 * a, 3 * a
    assert np.allclose(ops.downsample(np.full((nt, ny, nx), 3.25), a), 3.25, rtol=0, atol=1e-15)
    y, x = np.mgrid[0:ny, 0:nx].astype(float)
    u = np.stack([1.5 + 0.25 * x - 0.75 * y, -2.0 + 1.0 * x + 0.5 * y])
    Y, X = np.mgrid[0:ny // a, 0:nx // a].astype(float)
    cx, cy = a * X + (a - 1) / 2, a * Y + (a - 1) / 2
    want = np.stack([1.5 + 0.25 * cx - 0.75 * cy, -2.0 + 1.0 * cx + 0.5 * cy])
    assert np.allclose(ops.downsample(u, a), want, rtol=0, atol=1e-13)
    r = np.random.default_rng(0).standard_normal((nt, ny, nx))
    assert np.allclose(ops.downsample(r, a).sum(axis=(1, 2)) * a * a, r.sum(axis=(1, 2)), rtol=1e-13, atol=1e-12)
    with pytest.raises(ValueError):
        ops.downsample(np.zeros((1, 4 * a + 1, 4 * a)), a)


@pytest.mark.parametrize("a", [2, 4])
def test_upsample_velocity_constants_ramps_and_clamping(a):
    """Velocities in coarse pixels become fine pixels (times a). A constant field c gives
    a c everywhere; the coarse ramp s_x = X gives a * clamp((x + 1/2)/a - 1/2, 0, nxc - 1)
    (bilinear interpolation is exact on linear fields, the clamp holds the border)."""
    npairs, nyc, nxc = 2, 3, 5
    c = np.zeros((npairs, 2, nyc, nxc))
    c[:, 0] = 0.7
    c[:, 1] = -1.3
    f = ops.upsample_velocity(c, a)
    assert f.shape == (npairs, 2, a * nyc, a * nxc)
    assert np.allclose(f[:, 0], a * 0.7, rtol=0, atol=1e-14) and np.allclose(f[:, 1], -a * 1.3, rtol=0, atol=1e-14)
    Yc, Xc = np.mgrid[0:nyc, 0:nxc].astype(float)
    ramp = np.zeros((1, 2, nyc, nxc))
    ramp[0, 0] = Xc
    ramp[0, 1] = 2.0 * Yc - Xc
    f = ops.upsample_velocity(ramp, a)
    xs = np.clip((np.arange(a * nxc) + 0.5) / a - 0.5, 0, nxc - 1)
    ys = np.clip((np.arange(a * nyc) + 0.5) / a - 0.5, 0, nyc - 1)
    assert np.allclose(f[0, 0], a * np.broadcast_to(xs[None, :], (a * nyc, a * nxc)), rtol=0, atol=1e-13)
    assert np.allclose(f[0, 1], a * (2.0 * ys[:, None] - xs[None, :]), rtol=0, atol=1e-13)


def test_rescaling_by_one_is_the_identity():
    r = np.random.default_rng(1).standard_normal((3, 6, 8))
    s = np.random.default_rng(2).standard_normal((2, 2, 6, 8))
    assert np.array_equal(ops.downsample(r, 1), r)
    assert np.allclose(ops.upsample_velocity(s, 1), s, rtol=0, atol=0)


# ------------------------------------------------------------ rounding-and-clipping M(s)
def test_round_warp_equals_bilinear_warp_on_integer_velocities():
    """Where every velocity is an integer the two encodings of M(s) (Sec. 3, items 1 and 2)
    are the same matrix: the rounding warp against the compiled bilinear oracle, including
    clipped samples."""
    rng = np.random.default_rng(4)
    ny, nx = 9, 13
    v = rng.standard_normal((ny, nx))
    sx = rng.integers(-4, 5, (ny, nx)).astype(float)
    sy = rng.integers(-4, 5, (ny, nx)).astype(float)
    assert np.allclose(ops.warp_round(v, sx, sy), ops.warp(v, sx, sy), rtol=0, atol=1e-15)
    r = rng.standard_normal((ny, nx))
    assert np.allclose(ops.warpT_round(r, sx, sy), ops.warpT(r, sx, sy), rtol=0, atol=1e-14)


def test_round_warp_halves_go_away_from_zero_and_rows_select_one_pixel():
    ny, nx = 5, 7
    v = np.arange(ny * nx, dtype=float).reshape(ny, nx)
    z = np.zeros((ny, nx))
    assert np.array_equal(ops.warp_round(v, z + 0.5, z), ops.warp_round(v, z + 1.0, z))
    assert np.array_equal(ops.warp_round(v, z - 0.5, z), ops.warp_round(v, z - 1.0, z))
    assert np.array_equal(ops.warp_round(v, z + 0.49, z - 0.49), v)
    out = ops.warp_round(v, z + 2.3, z - 1.7)  # every value is some pixel of v
    assert set(out.ravel()) <= set(v.ravel())


def test_round_flow_adjoint_identity():
    rng = np.random.default_rng(5)
    nt, ny, nx = 4, 8, 9
    s = synth.random_velocities(nt - 1, ny, nx, 2.5, seed=6)
    sr = ops.reverse_flow(s)
    u = rng.standard_normal((nt, ny, nx))
    r = rng.standard_normal((2, nt - 1, ny, nx))
    assert abs(np.sum(ops.flow_round(u, s, sr) * r) - np.sum(u * ops.flowT_round(r, s, sr))) < 1e-11
