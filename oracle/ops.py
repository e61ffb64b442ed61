"""numpy bindings of the FP64 C oracle operators (oracle/ops.c).

TEST INFRASTRUCTURE ONLY: imported by tests/, the package smoke check and the
bench's CPU-baseline leg, never by the product path.

Every function takes and returns float64 numpy arrays in the layouts that
oracle/ops.c documents: images (nt, ny, nx), sinograms flat (sum_t na[t]*nb,),
velocities (nt-1, 2, ny, nx), gradients (nf, 2, ny, nx), flow residuals
(2, nt-1, ny, nx).
"""
import ctypes
from dataclasses import dataclass

import numpy as np

from .build import build_oracle

_lib = None
_D = ctypes.POINTER(ctypes.c_double)
_I = ctypes.POINTER(ctypes.c_int)


def _load():
    global _lib
    if _lib is None:
        lib = ctypes.CDLL(build_oracle())
        i, d = ctypes.c_int, ctypes.c_double
        lib.orc_project.argtypes = [i, i, i, i, _I, _D, d, d, _D, _D]
        lib.orc_backproject.argtypes = [i, i, i, i, _I, _D, d, d, _D, _D]
        lib.orc_project_fan.argtypes = [i, i, i, i, _I, _D, d, d, d, d, _D, _D]
        lib.orc_backproject_fan.argtypes = [i, i, i, i, _I, _D, d, d, d, d, _D, _D]
        lib.orc_grad.argtypes = [i, i, i, _D, _D]
        lib.orc_gradT.argtypes = [i, i, i, _D, _D]
        lib.orc_warp.argtypes = [i, i, _D, _D, _D, _D]
        lib.orc_warpT.argtypes = [i, i, _D, _D, _D, _D]
        lib.orc_flow.argtypes = [i, i, i, _D, _D, _D, _D]
        lib.orc_flowT.argtypes = [i, i, i, _D, _D, _D, _D]
        lib.orc_of_fields.argtypes = [i, i, i, i, _D, _D, _D, _D]
        lib.orc_flow_lin.argtypes = [i, i, i, _D, _D, _D, _D, _D]
        lib.orc_flow_linT.argtypes = [i, i, i, _D, _D, _D, _D]
        lib.orc_reverse_flow.argtypes = [i, i, i, _D, _D]
        lib.orc_flow_ds.argtypes = [i, i, i, _D, _D, _D, _D, _D, _D]
        for f in ("orc_project", "orc_backproject", "orc_project_fan", "orc_backproject_fan", "orc_grad", "orc_gradT", "orc_warp",
                  "orc_warpT", "orc_flow", "orc_flowT", "orc_of_fields", "orc_flow_lin",
                  "orc_flow_linT", "orc_reverse_flow", "orc_flow_ds"):
            getattr(lib, f).restype = None
        _lib = lib
    return _lib


def _d(a):
    return a.ctypes.data_as(_D)


def _c64(a):
    return np.ascontiguousarray(a, dtype=np.float64)


@dataclass
class Geometry:
    """2D parallel-beam or fan-beam geometry of an image sequence (Sec. 2.1:
    H = blockdiag(H^1..H^nt)).

    angles: radians, concatenated over frames (na[t] entries for frame t).
    fan: None for parallel beams, else (rs, rd): the source at distance rs from the
    centre of rotation and a flat detector at distance rd on the other side (Sec. 5.1).
    """
    nx: int
    ny: int
    nt: int
    nb: int
    na: np.ndarray
    angles: np.ndarray
    h: float = 1.0
    db: float = 1.0
    fan: tuple = None

    def __post_init__(self):
        self.na = np.ascontiguousarray(self.na, dtype=np.int32)
        self.angles = _c64(self.angles)
        assert self.na.shape == (self.nt,)
        assert self.angles.shape == (int(self.na.sum()),)

    @property
    def ns(self):
        return self.nx * self.ny

    @property
    def n(self):
        return self.ns * self.nt

    @property
    def m(self):
        return int(self.na.sum()) * self.nb


def project(g: Geometry, u):
    """b = H u (Joseph ray-driven line integrals)."""
    u = _c64(u).reshape(g.nt, g.ny, g.nx)
    b = np.empty(g.m)
    if g.fan is not None:
        _load().orc_project_fan(g.nx, g.ny, g.nt, g.nb, g.na.ctypes.data_as(_I), _d(g.angles), g.h, g.db,
                                float(g.fan[0]), float(g.fan[1]), _d(u), _d(b))
        return b
    _load().orc_project(g.nx, g.ny, g.nt, g.nb, g.na.ctypes.data_as(_I), _d(g.angles), g.h, g.db,
                        _d(u), _d(b))
    return b


def backproject(g: Geometry, b):
    """u = H^T b (scatter of the same ray entries)."""
    b = _c64(b).reshape(g.m)
    u = np.empty((g.nt, g.ny, g.nx))
    if g.fan is not None:
        _load().orc_backproject_fan(g.nx, g.ny, g.nt, g.nb, g.na.ctypes.data_as(_I), _d(g.angles), g.h,
                                    g.db, float(g.fan[0]), float(g.fan[1]), _d(b), _d(u))
        return u
    _load().orc_backproject(g.nx, g.ny, g.nt, g.nb, g.na.ctypes.data_as(_I), _d(g.angles), g.h,
                            g.db, _d(b), _d(u))
    return u


def grad(u):
    """Psi u for u of shape (nf, ny, nx) -> (nf, 2, ny, nx)."""
    u = _c64(u)
    nf, ny, nx = u.shape
    g = np.empty((nf, 2, ny, nx))
    _load().orc_grad(nx, ny, nf, _d(u), _d(g))
    return g


def gradT(g):
    """Psi^T g for g of shape (nf, 2, ny, nx) -> (nf, ny, nx)."""
    g = _c64(g)
    nf, two, ny, nx = g.shape
    assert two == 2
    u = np.empty((nf, ny, nx))
    _load().orc_gradT(nx, ny, nf, _d(g), _d(u))
    return u


def warp(v, sx, sy):
    """M(s) v for one frame (ny, nx)."""
    v, sx, sy = _c64(v), _c64(sx), _c64(sy)
    ny, nx = v.shape
    out = np.empty_like(v)
    _load().orc_warp(nx, ny, _d(v), _d(sx), _d(sy), _d(out))
    return out


def warpT(r, sx, sy):
    """M(s)^T r for one frame (ny, nx)."""
    r, sx, sy = _c64(r), _c64(sx), _c64(sy)
    ny, nx = r.shape
    out = np.empty_like(r)
    _load().orc_warpT(nx, ny, _d(r), _d(sx), _d(sy), _d(out))
    return out


def flow(u, s, sr):
    """Mhat(s, s') u: u (nt, ny, nx), s/sr (nt-1, 2, ny, nx) -> (2, nt-1, ny, nx)."""
    u, s, sr = _c64(u), _c64(s), _c64(sr)
    nt, ny, nx = u.shape
    assert s.shape == (nt - 1, 2, ny, nx) and sr.shape == s.shape
    r = np.empty((2, nt - 1, ny, nx))
    _load().orc_flow(nx, ny, nt, _d(u), _d(s), _d(sr), _d(r))
    return r


def flowT(r, s, sr):
    """Mhat(s, s')^T r -> (nt, ny, nx)."""
    r, s, sr = _c64(r), _c64(s), _c64(sr)
    _, npairs, ny, nx = r.shape
    u = np.empty((npairs + 1, ny, nx))
    _load().orc_flowT(nx, ny, npairs + 1, _d(r), _d(s), _d(sr), _d(u))
    return u


def flow_ds(u, s, sr, gr):
    """Velocity VJP of Mhat(s, s') u for the cotangent gr (2, nt-1, ny, nx):
    (gs, gsr), each (nt-1, 2, ny, nx)."""
    u, s, sr, gr = _c64(u), _c64(s), _c64(sr), _c64(gr)
    nt, ny, nx = u.shape
    gs = np.empty((nt - 1, 2, ny, nx))
    gsr = np.empty((nt - 1, 2, ny, nx))
    _load().orc_flow_ds(nx, ny, nt, _d(u), _d(s), _d(sr), _d(gr), _d(gs), _d(gsr))
    return gs, gsr


def of_fields(u, dr=1):
    """App. C derivative fields (u_x, u_y, u_t), each (nt-1, ny, nx)."""
    u = _c64(u)
    nt, ny, nx = u.shape
    if not (1 <= dr):
        raise ValueError("dr must be >= 1")
    ux = np.empty((nt - 1, ny, nx))
    uy = np.empty_like(ux)
    ut = np.empty_like(ux)
    _load().orc_of_fields(nx, ny, nt, dr, _d(u), _d(ux), _d(uy), _d(ut))
    return ux, uy, ut


def flow_lin(ux, uy, ut, s):
    """Upsilon s + u_t per pair -> (npairs, ny, nx)."""
    ux, uy, ut, s = _c64(ux), _c64(uy), _c64(ut), _c64(s)
    npairs, ny, nx = ux.shape
    r = np.empty_like(ux)
    _load().orc_flow_lin(nx, ny, npairs, _d(ux), _d(uy), _d(ut), _d(s), _d(r))
    return r


def flow_linT(ux, uy, r):
    """Upsilon^T r per pair -> (npairs, 2, ny, nx)."""
    ux, uy, r = _c64(ux), _c64(uy), _c64(r)
    npairs, ny, nx = ux.shape
    gs = np.empty((npairs, 2, ny, nx))
    _load().orc_flow_linT(nx, ny, npairs, _d(ux), _d(uy), _d(r), _d(gs))
    return gs


def vgrad(s):
    """(L (+) L) s: the gradient of each velocity component.
    s (npairs, 2, ny, nx) -> (npairs, 2 comps, 2 dirs, ny, nx)."""
    s = _c64(s)
    npairs, two, ny, nx = s.shape
    return grad(s.reshape(npairs * 2, ny, nx)).reshape(npairs, 2, 2, ny, nx)


def vgradT(gs):
    """(L (+) L)^T gs -> (npairs, 2, ny, nx)."""
    gs = _c64(gs)
    npairs, _, _, ny, nx = gs.shape
    return gradT(gs.reshape(npairs * 2, 2, ny, nx)).reshape(npairs, 2, ny, nx)


def reverse_flow(s):
    """s' from s by the reverse-flow remark of Sec. 3 -> same shape as s."""
    s = _c64(s)
    npairs, two, ny, nx = s.shape
    sr = np.empty_like(s)
    _load().orc_reverse_flow(nx, ny, npairs + 1, _d(s), _d(sr))
    return sr


# ------------------------------------------------------------ rescaling for Solve-OF
# Sec. 4.1.5 ("Rescaling Large Images for Optical Flow Computation") and Sec. 5 (frames
# downsampled by a factor of 2 or 4 before Solve-OF, velocities upscaled afterwards). The
# paper names neither operator; the readings: the frames are averaged over a x a blocks,
# and the coarse velocity field is interpolated bilinearly at the fine pixel centres
# (coarse coordinate (x + 1/2)/a - 1/2, clamped to the coarse grid) and multiplied by a,
# since a coarse pixel is a fine pixels wide.

def downsample(u, a):
    """Block mean over a x a pixels of every frame: (nt, ny, nx) -> (nt, ny/a, nx/a);
    ny and nx must be multiples of a."""
    u = np.asarray(u, dtype=np.float64)
    nt, ny, nx = u.shape
    if ny % a or nx % a:
        raise ValueError("frame size must be a multiple of the factor")
    return u.reshape(nt, ny // a, a, nx // a, a).mean(axis=(2, 4))


def upsample_velocity(sc, a):
    """Coarse velocities (npairs, 2, nyc, nxc) in coarse pixels -> fine velocities
    (npairs, 2, a nyc, a nxc) in fine pixels: bilinear interpolation at the fine pixel
    centres, clamped to the coarse grid, times a."""
    sc = np.asarray(sc, dtype=np.float64)
    npairs, two, nyc, nxc = sc.shape
    ny, nx = a * nyc, a * nxc

    def axis(n_fine, n_coarse):
        X = np.clip((np.arange(n_fine) + 0.5) / a - 0.5, 0.0, n_coarse - 1.0)
        i0 = np.floor(X).astype(int)
        i1 = np.minimum(i0 + 1, n_coarse - 1)
        return i0, i1, X - i0

    y0, y1, wy = axis(ny, nyc)
    x0, x1, wx = axis(nx, nxc)
    wy, wx = wy[:, None], wx[None, :]
    out = (sc[:, :, y0][:, :, :, x0] * (1 - wy) * (1 - wx) + sc[:, :, y0][:, :, :, x1] * (1 - wy) * wx
           + sc[:, :, y1][:, :, :, x0] * wy * (1 - wx) + sc[:, :, y1][:, :, :, x1] * wy * wx)
    return a * out


# ------------------------------------------------------------ rounding-and-clipping M(s)
# Sec. 3, item 1 (eq. (m_matrix)): the velocity components are rounded to the nearest
# integers and the source coordinates clipped to the image, so M(s) selects one pixel per
# row. Reading: halves round away from zero (the rule of the reverse-flow remark).

def _round_half_away(s):
    return np.sign(s) * np.floor(np.abs(s) + 0.5)


def warp_round(v, sx, sy):
    """M(s) v for one frame (ny, nx) with rounding and clipping."""
    v = np.asarray(v, dtype=np.float64)
    ny, nx = v.shape
    y, x = np.mgrid[0:ny, 0:nx]
    X = np.clip(x + _round_half_away(np.asarray(sx, dtype=np.float64)).astype(int), 0, nx - 1)
    Y = np.clip(y + _round_half_away(np.asarray(sy, dtype=np.float64)).astype(int), 0, ny - 1)
    return v[Y, X]


def warpT_round(r, sx, sy):
    """M(s)^T r for one frame with rounding and clipping (each row's entry scattered back)."""
    r = np.asarray(r, dtype=np.float64)
    ny, nx = r.shape
    y, x = np.mgrid[0:ny, 0:nx]
    X = np.clip(x + _round_half_away(np.asarray(sx, dtype=np.float64)).astype(int), 0, nx - 1)
    Y = np.clip(y + _round_half_away(np.asarray(sy, dtype=np.float64)).astype(int), 0, ny - 1)
    out = np.zeros((ny, nx))
    np.add.at(out, (Y, X), r)
    return out


def flow_round(u, s, sr):
    """Mhat(s, s') u with the rounding-and-clipping M: rows u_p - M(s_p) u_{p+1} and
    u_{p+1} - M(s'_p) u_p -> (2, nt-1, ny, nx)."""
    u = np.asarray(u, dtype=np.float64)
    nt = u.shape[0]
    r = np.empty((2, nt - 1) + u.shape[1:])
    for p in range(nt - 1):
        r[0, p] = u[p] - warp_round(u[p + 1], s[p, 0], s[p, 1])
        r[1, p] = u[p + 1] - warp_round(u[p], sr[p, 0], sr[p, 1])
    return r


def flowT_round(r, s, sr):
    """The transpose of flow_round -> (nt, ny, nx)."""
    npairs = r.shape[1]
    u = np.zeros((npairs + 1,) + r.shape[2:])
    for p in range(npairs):
        u[p] += r[0, p]
        u[p + 1] -= warpT_round(r[0, p], s[p, 0], s[p, 1])
        u[p + 1] += r[1, p]
        u[p] -= warpT_round(r[1, p], sr[p, 0], sr[p, 1])
    return u
