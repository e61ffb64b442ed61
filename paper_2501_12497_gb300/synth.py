"""Seeded synthetic workloads: moving disk/ellipse phantoms, their exact
parallel-beam sinograms, and Gaussian noise.

This module holds none of the reconstruction method's arithmetic. It only
makes inputs: the phantoms are drawn from seeded random numbers, and the data
are the analytic Radon transform of the ellipses (chord length times
intensity), so the data are not produced by the discrete projector that the
method uses. Both the CUDA path and the oracle are fed from here.

Geometry convention shared by every workload: pixel centres
x_i = (i - (nx-1)/2) h, bin centres sigma_k = (k - (nb-1)/2) db, the ray of
angle theta and bin k is {x cos(theta) + y sin(theta) = sigma_k}; the angles
of frame t are theta_{t,a} = (a*180/na + t*180/(na*nt)) degrees, i.e. each
frame's fan of na equispaced angles is shifted by 180/(na*nt) degrees from the
previous frame's (the "shifted intervals" scheme of Sec. 5.1.1).

Fan-beam workloads (fan = (rs, rd)) put a point source at distance rs from the
centre, opposite a flat detector at distance rd, for the view of angle theta
on the line along (-sin theta, cos theta); the bins lie on the detector at
sigma_k along (cos theta, sin theta), and each ray is the line from the source
through its bin. Their data are the same analytic chords along those lines.
"""
from dataclasses import dataclass, field
import math

import numpy as np


@dataclass
class Ellipse:
    cx: float
    cy: float
    a: float        # semi-axis along the ellipse's own x axis
    b: float        # semi-axis along its own y axis
    phi: float      # orientation, radians
    rho: float      # intensity (added where ellipses overlap)
    vx: float = 0.0  # translation per frame (pixels)
    vy: float = 0.0
    omega: float = 0.0  # rotation per frame (radians)

    def at(self, t):
        """The ellipse at frame t (rigid motion: translate, rotate about its centre)."""
        return (self.cx + t * self.vx, self.cy + t * self.vy, self.a, self.b,
                self.phi + t * self.omega, self.rho)


@dataclass
class FlowField:
    """A smooth, divergence-free velocity field (pixels per frame) from a stream
    function that is a sum of Gaussians: psi(x) = sum_k c_k exp(-|x - m_k|^2 / (2 s_k^2)),
    v = (d psi/dy, -d psi/dx). Divergence-free, so the objects it carries keep their
    area while they shear and turn."""
    centres: np.ndarray  # (k, 2)
    sigmas: np.ndarray   # (k,)
    coefs: np.ndarray    # (k,)

    def velocity(self, x, y):
        vx = vy = 0.0
        for (mx, my), sg, c in zip(self.centres, self.sigmas, self.coefs):
            g = c * np.exp(-((x - mx) ** 2 + (y - my) ** 2) / (2 * sg * sg))
            vx = vx - g * (y - my) / (sg * sg)
            vy = vy + g * (x - mx) / (sg * sg)
        return vx, vy

    def jacobian(self, x, y):
        """d(vx, vy)/d(x, y) at one point, 2 x 2."""
        J = np.zeros((2, 2))
        for (mx, my), sg, c in zip(self.centres, self.sigmas, self.coefs):
            dx, dy, s2 = x - mx, y - my, sg * sg
            g = c * math.exp(-(dx * dx + dy * dy) / (2 * s2))
            # vx = -g dy / s2, vy = g dx / s2
            J[0, 0] += g * dx * dy / (s2 * s2)
            J[0, 1] += -g / s2 + g * dy * dy / (s2 * s2)
            J[1, 0] += g / s2 - g * dx * dx / (s2 * s2)
            J[1, 1] += -g * dx * dy / (s2 * s2)
        return J


def smooth_field(n, vmax, seed, count=3):
    """Seeded FlowField on an n x n frame (pixel units about the centre): `count` Gaussians
    with widths U(n/8, n/4), scaled so that the largest speed on the frame is vmax."""
    rng = np.random.default_rng(seed)
    R = 0.5 * (n - 1)
    f = FlowField(rng.uniform(-0.6 * R, 0.6 * R, (count, 2)), rng.uniform(n / 8.0, n / 4.0, count),
                  rng.uniform(-1.0, 1.0, count))
    g = np.linspace(-R, R, 65)
    X, Y = np.meshgrid(g, g)
    vx, vy = f.velocity(X, Y)
    f.coefs = f.coefs * (vmax / max(float(np.max(np.hypot(vx, vy))), 1e-30))
    return f


@dataclass
class TrackedEllipse:
    """An ellipse carried by a smooth field on top of its own rigid motion: per frame its
    centre moves by the rigid translation plus the field's velocity there, and its shape
    by the field's local linear map (I + grad v); an ellipse stays an ellipse, so its
    data remain exact line integrals. rho as in Ellipse."""
    track: list  # per frame (cx, cy, a, b, phi)
    rho: float

    def at(self, t):
        return tuple(self.track[t]) + (self.rho,)


def track_ellipse(e, field, nt):
    """Frames 0..nt-1 of Ellipse e (rigid translation and rotation per frame) with the
    field's motion added: centre c += (vx, vy) + v(c), shape matrix A <- R(omega)(I + J(c)) A."""
    c = np.array([e.cx, e.cy], dtype=np.float64)
    cp, sp = math.cos(e.phi), math.sin(e.phi)
    A = np.array([[cp, -sp], [sp, cp]]) @ np.diag([e.a, e.b])
    co, so = math.cos(e.omega), math.sin(e.omega)
    Rot = np.array([[co, -so], [so, co]])
    out = []
    for _ in range(nt):
        U, S, _ = np.linalg.svd(A)
        out.append((float(c[0]), float(c[1]), float(S[0]), float(S[1]), math.atan2(U[1, 0], U[0, 0])))
        vx, vy = (0.0, 0.0) if field is None else field.velocity(c[0], c[1])
        J = np.zeros((2, 2)) if field is None else field.jacobian(c[0], c[1])
        c = c + np.array([e.vx + vx, e.vy + vy])
        A = Rot @ (np.eye(2) + J) @ A
    return TrackedEllipse(out, e.rho)


@dataclass
class Paraboloid:
    """A static smooth background: rho (1 - |x|^2 / R^2) on the disk of radius R about the
    centre, zero outside. Line integral along {x cos + y sin = sigma} at distance |sigma| < R
    from the centre: (4/3) rho L^3 / R^2 with L = sqrt(R^2 - sigma^2)."""
    R: float
    rho: float

    def radon(self, sigma):
        L2 = np.maximum(self.R * self.R - sigma * sigma, 0.0)
        return (4.0 / 3.0) * self.rho * L2 * np.sqrt(L2) / (self.R * self.R)

    def sample(self, X, Y):
        return self.rho * np.maximum(1.0 - (X * X + Y * Y) / (self.R * self.R), 0.0)


@dataclass
class Workload:
    name: str
    nx: int
    ny: int
    nt: int
    nb: int
    na: np.ndarray          # angles per frame, int32 (nt,)
    angles: np.ndarray      # radians, float64 (sum na,)
    h: float
    db: float
    u_true: np.ndarray      # (nt, ny, nx) float64, area-averaged phantom
    b_clean: np.ndarray     # (m,) exact line integrals
    b: np.ndarray           # (m,) noisy data
    noise_norm: float       # delta = ||b - b_clean||
    ellipses: list = field(default_factory=list)
    fan: tuple = None       # (rs, rd) for a fan beam, None for parallel rays
    background: object = None  # static Paraboloid under the ellipses, or None
    field: object = None    # FlowField carrying the ellipses, or None (rigid motion only)

    @property
    def m(self):
        return int(self.na.sum()) * self.nb

    @property
    def n(self):
        return self.nx * self.ny * self.nt


def shifted_angles(nt, na):
    """Angles (radians) of every frame, concatenated: a*180/na + t*180/(na*nt) degrees."""
    na_arr = np.full(nt, na, dtype=np.int32) if np.isscalar(na) else np.asarray(na, np.int32)
    out = []
    for t in range(nt):
        k = int(na_arr[t])
        deg = np.arange(k) * 180.0 / k + t * 180.0 / (k * nt)
        out.append(np.deg2rad(deg))
    return na_arr, np.concatenate(out)


def ellipse_radon(e, theta, sigma):
    """Exact line integral of one ellipse (cx, cy, a, b, phi, rho) along the rays
    {x cos(theta) + y sin(theta) = sigma}: rho times the chord length."""
    cx, cy, a, b, phi, rho = e
    s = sigma - (cx * np.cos(theta) + cy * np.sin(theta))
    d = theta - phi
    a2 = (a * np.cos(d)) ** 2 + (b * np.sin(d)) ** 2
    q = a2 - s * s
    return np.where(q > 0, rho * 2.0 * a * b * np.sqrt(np.maximum(q, 0.0)) / a2, 0.0)


def fan_rays(theta, sigma, rs, rd):
    """Normal form (angle, offset) of the fan-beam rays: the line through the source
    -rs (-sin, cos) and the detector point rd (-sin, cos) + sigma (cos, sin)."""
    c, s = np.cos(theta), np.sin(theta)
    sx, sy = rs * s, -rs * c
    vx = -rd * s + sigma * c - sx
    vy = rd * c + sigma * s - sy
    ln = np.hypot(vx, vy)
    nx, ny = vy / ln, -vx / ln
    return np.arctan2(ny, nx), sx * nx + sy * ny


def raster(e_list, nx, ny, h=1.0, ss=4, background=None):
    """Area-averaged raster (ss x ss sub-samples per pixel) of a sum of ellipses (and of
    the background, when given)."""
    off = (np.arange(ss) + 0.5) / ss - 0.5
    xs = ((np.arange(nx) - 0.5 * (nx - 1))[:, None] + off[None, :]).ravel() * h
    ys = ((np.arange(ny) - 0.5 * (ny - 1))[:, None] + off[None, :]).ravel() * h
    X, Y = np.meshgrid(xs, ys)
    img = np.zeros_like(X) if background is None else background.sample(X, Y)
    for (cx, cy, a, b, phi, rho) in e_list:
        dx, dy = X - cx, Y - cy
        c, s = np.cos(phi), np.sin(phi)
        xr, yr = c * dx + s * dy, -s * dx + c * dy
        img += rho * ((xr / a) ** 2 + (yr / b) ** 2 <= 1.0)
    return img.reshape(ny, ss, nx, ss).mean(axis=(1, 3))


def _make(name, nx, ny, nt, na, nb, ellipses, noise_rel, seed, h=1.0, db=1.0, ss=4, fan=None, background=None,
          field=None):
    na_arr, angles = shifted_angles(nt, na)
    sig = (np.arange(nb) - 0.5 * (nb - 1)) * db
    u_true = np.empty((nt, ny, nx))
    b_clean = np.empty(int(na_arr.sum()) * nb)
    off = 0
    aoff = 0
    for t in range(nt):
        ets = [e.at(t) for e in ellipses]
        u_true[t] = raster(ets, nx, ny, h, ss, background)
        th = angles[aoff:aoff + na_arr[t]]
        blk = np.zeros((na_arr[t], nb))
        if fan is None:
            phi, off_ = th[:, None], sig[None, :]
        else:
            phi, off_ = fan_rays(th[:, None], sig[None, :], fan[0], fan[1])
        phi, off_ = np.broadcast_arrays(phi, off_)
        if background is not None:
            blk += background.radon(off_)
        for et in ets:
            blk += ellipse_radon(et, phi, off_)
        b_clean[off:off + blk.size] = blk.ravel()
        off += blk.size
        aoff += na_arr[t]
    rng = np.random.default_rng(seed + 7919)
    m = b_clean.size
    e = noise_rel * np.linalg.norm(b_clean) / math.sqrt(m) * rng.standard_normal(m)
    return Workload(name=name, nx=nx, ny=ny, nt=nt, nb=nb, na=na_arr, angles=angles, h=h, db=db,
                    u_true=u_true, b_clean=b_clean, b=b_clean + e,
                    noise_norm=float(np.linalg.norm(e)), ellipses=ellipses, fan=fan, background=background,
                    field=field)


def _inside(e, nt, R):
    """True if the ellipse stays inside the disk of radius R for frames 0..nt-1."""
    for t in range(nt):
        cx, cy, a, b, _, _ = e.at(t)
        if math.hypot(cx, cy) + max(a, b) > R:
            return False
    return True


def moving_disks(n=64, nt=8, na=16, nb=64, radii=(8.0, 12.0), rhos=(1.0, 0.6), speed=1.0,
                 noise=0.01, seed=0, name=None, db=1.0, fan=None):
    """Uniform disks translating `speed` px/frame in fixed seeded directions, kept
    inside the inscribed circle of the grid for every frame."""
    rng = np.random.default_rng(seed)
    R = 0.5 * (n - 1)
    ell = []
    for r, rho in zip(radii, rhos):
        for _ in range(10000):
            ang = rng.uniform(0, 2 * np.pi)
            vx, vy = speed * np.cos(ang), speed * np.sin(ang)
            rr = (R - r) * np.sqrt(rng.uniform(0, 1))
            pa = rng.uniform(0, 2 * np.pi)
            e = Ellipse(rr * np.cos(pa), rr * np.sin(pa), r, r, 0.0, rho, vx, vy, 0.0)
            if _inside(e, nt, R):
                ell.append(e)
                break
        else:
            raise RuntimeError("could not place disk")
    return _make(name or "disks%dx%dx%d" % (n, n, nt), n, n, nt, na, nb, ell, noise, seed, db=db, fan=fan)


def moving_ellipses(n=256, nt=32, na=30, nb=363, n_ell=6, axes=(8.0, 40.0), rho=(0.2, 1.0),
                    speed=(0.5, 2.0), rot_deg=2.0, noise=0.01, seed=0, name=None, ss=4, db=1.0, fan=None):
    """Seeded ellipses, each in rigid motion: translation of U(speed) px/frame and
    rotation of U(-rot_deg, rot_deg) degrees/frame about its own centre."""
    rng = np.random.default_rng(seed)
    R = 0.5 * (n - 1)
    ell = []
    scale = n / 256.0
    for _ in range(n_ell):
        for _ in range(10000):
            a = rng.uniform(*axes) * scale
            b = rng.uniform(*axes) * scale
            phi = rng.uniform(0, np.pi)
            sp = rng.uniform(*speed)
            ang = rng.uniform(0, 2 * np.pi)
            om = np.deg2rad(rng.uniform(-rot_deg, rot_deg))
            rr = (R - max(a, b)) * np.sqrt(rng.uniform(0, 1))
            pa = rng.uniform(0, 2 * np.pi)
            e = Ellipse(rr * np.cos(pa), rr * np.sin(pa), a, b, phi, rng.uniform(*rho),
                        sp * np.cos(ang), sp * np.sin(ang), om)
            if _inside(e, nt, R):
                ell.append(e)
                break
        else:
            raise RuntimeError("could not place ellipse")
    return _make(name or "ellipses%dx%dx%d" % (n, n, nt), n, n, nt, na, nb, ell, noise, seed, ss=ss, db=db, fan=fan)


def deforming_ellipses(n, nt, na, nb, n_ell, field_vmax, speed=(0.0, 0.0), rot_deg=0.0, axes=(8.0, 40.0),
                       rho=(0.2, 1.0), noise=0.01, seed=0, name=None, ss=1, background_rho=0.0, max_speed=None):
    """Seeded ellipses in smooth non-rigid motion: each has its own rigid translation of
    U(speed) px/frame and rotation of U(-rot_deg, rot_deg) deg/frame, and all are carried
    by one seeded divergence-free FlowField whose largest speed is field_vmax px/frame
    (track_ellipse). Every ellipse stays inside the inscribed circle for all frames, and
    its total displacement per frame stays within max_speed (default: the sum of the two
    maxima). background_rho > 0 adds a static Paraboloid of that height on the disk of
    radius 0.45 n. Data are exact line integrals (chord lengths), as for rigid motion."""
    rng = np.random.default_rng(seed)
    R = 0.5 * (n - 1)
    fld = smooth_field(n, field_vmax, seed + 104729) if field_vmax > 0 else None
    vcap = max_speed if max_speed is not None else speed[1] + field_vmax
    scale = n / 256.0
    ell = []
    for _ in range(n_ell):
        for _ in range(10000):
            a = rng.uniform(*axes) * scale
            b = rng.uniform(*axes) * scale
            phi = rng.uniform(0, np.pi)
            sp = rng.uniform(*speed)
            ang = rng.uniform(0, 2 * np.pi)
            om = np.deg2rad(rng.uniform(-rot_deg, rot_deg))
            rr = (R - max(a, b)) * np.sqrt(rng.uniform(0, 1))
            pa = rng.uniform(0, 2 * np.pi)
            e = Ellipse(rr * np.cos(pa), rr * np.sin(pa), a, b, phi, rng.uniform(*rho),
                        sp * np.cos(ang), sp * np.sin(ang), om)
            te = track_ellipse(e, fld, nt)
            ok = all(math.hypot(cx, cy) + max(aa, bb) <= R for cx, cy, aa, bb, _ in te.track)
            steps = np.diff(np.array([tr[:2] for tr in te.track]), axis=0)
            if ok and (steps.size == 0 or float(np.max(np.hypot(steps[:, 0], steps[:, 1]))) <= vcap + 1e-9):
                ell.append(te)
                break
        else:
            raise RuntimeError("could not place ellipse")
    bg = Paraboloid(0.45 * n, background_rho) if background_rho > 0 else None
    return _make(name or "deforming%dx%dx%d" % (n, n, nt), n, n, nt, na, nb, ell, noise, seed, ss=ss,
                 background=bg, field=fld)


# The workloads of the method's benchmark configurations.
def plain_fp64(seed=0):
    """64x64 frames, T=8, 16 angles/frame, 64 bins, two disks (r 8/12, rho 1.0/0.6)
    at 1 px/frame, 1% noise."""
    return moving_disks(64, 8, 16, 64, seed=seed, name="disks64x64x8")


def precision_form(seed=0):
    """256x256 frames, T=32, 30 angles/frame, 363 bins, six ellipses in rigid motion, 1% noise."""
    return moving_ellipses(256, 32, 30, 363, seed=seed, name="ellipses256x256x32")


def precision_form_small(seed=0):
    """A reduced instance of the same generator (96x96, T=6, 30 angles, 137 bins) that
    the FP64 oracle finishes in seconds; used for end-to-end parity."""
    return moving_ellipses(96, 6, 30, 137, seed=seed, name="ellipses96x96x6")


def differentiation_form(seed=0):
    """The two-disk generator at 256x256, T=32 (radii 32/48 px, 1 px/frame), 16 angles,
    256 bins."""
    return moving_disks(256, 32, 16, 256, radii=(32.0, 48.0), seed=seed, name="disks256x256x32")


def fan_form(seed=0):
    """The 256x256x32 moving-ellipse workload in a fan beam: source 512 px from the
    centre, flat detector 256 px beyond it (magnification 1.5), 363 bins of 1.6 px
    covering the magnified field of view, 30 views per frame over 180 degrees."""
    return moving_ellipses(256, 32, 30, 363, seed=seed, name="fan_ellipses256x256x32", db=1.6, fan=(512.0, 256.0))


def fan_form_small(seed=0):
    """The 64x64x8 two-disk workload in a fan beam (source 128 px, detector 64 px
    beyond the centre, 100 bins of 1.5 px, 16 views per frame): FP64 parity size."""
    return moving_disks(64, 8, 16, 100, seed=seed, name="fan_disks64x64x8", db=1.5, fan=(128.0, 64.0))


def batch_form(count=48, seed=0, sizes=(128, 192, 256, 384, 512), nt_range=(8, 40), na_range=(10, 45)):
    """Independent problems of uneven size: for each, seeded n from `sizes`, T and
    angles per frame uniform in the given ranges, ceil(sqrt(2) n) bins, and six ellipses
    carried by a seeded smooth field (a sum of three Gaussians, largest speed 2 px/frame;
    deforming_ellipses), 1% noise; the phantom raster at one sample per pixel."""
    rng = np.random.default_rng(seed)
    out = []
    for i in range(count):
        n = int(rng.choice(sizes))
        nt = int(rng.integers(nt_range[0], nt_range[1] + 1))
        na = int(rng.integers(na_range[0], na_range[1] + 1))
        nb = int(math.ceil(math.sqrt(2) * n))
        out.append(deforming_ellipses(n, nt, na, nb, 6, 2.0, seed=1000 * seed + i, ss=1,
                                      name="batch%d_%dx%dx%d" % (i, n, n, nt)))
    return out


def large_form(seed=0):
    """1024x1024 frames, T=64, 90 angles/frame, 1448 bins: 20 ellipses on a smooth static
    background (a paraboloid of height 0.1), each in rigid motion (0.5-2 px/frame, up to 2
    deg/frame) and all carried by a smooth non-rigid field (up to 1 px/frame), at most 3
    px/frame in total; 0.5% noise; the phantom raster at one sample per pixel."""
    return deforming_ellipses(1024, 64, 90, 1448, 20, 1.0, speed=(0.5, 2.0), rot_deg=2.0, noise=0.005, seed=seed,
                              name="ellipses1024x1024x64", ss=1, background_rho=0.1, max_speed=3.0)


# ------------------------------------------------------- generic random inputs

def random_images(nt, ny, nx, seed=0, smooth=2):
    """Seeded smooth random images (box-filtered white noise), float64."""
    rng = np.random.default_rng(seed)
    u = rng.standard_normal((nt, ny, nx))
    for _ in range(smooth):
        u = (u + np.roll(u, 1, -1) + np.roll(u, -1, -1)) / 3.0
        u = (u + np.roll(u, 1, -2) + np.roll(u, -1, -2)) / 3.0
    return u


def random_velocities(npairs, ny, nx, vmax=2.0, seed=0):
    """Seeded smooth velocity fields (npairs, 2, ny, nx) with |s| <= vmax, float64."""
    rng = np.random.default_rng(seed)
    yy, xx = np.meshgrid(np.arange(ny), np.arange(nx), indexing="ij")
    s = np.zeros((npairs, 2, ny, nx))
    for p in range(npairs):
        for c in range(2):
            f = np.zeros((ny, nx))
            for _ in range(3):
                cx, cy = rng.uniform(0, nx), rng.uniform(0, ny)
                sg = rng.uniform(0.1, 0.3) * max(nx, ny)
                f += rng.uniform(-1, 1) * np.exp(-((xx - cx) ** 2 + (yy - cy) ** 2) / (2 * sg * sg))
            s[p, c] = f
        mx = np.max(np.abs(s[p])) or 1.0
        s[p] *= vmax * rng.uniform(0.5, 1.0) / mx
    return s
