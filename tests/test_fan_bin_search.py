"""The fan-beam transpose finds a pixel's bins by central projection in FP32, with a margin of
0.02 bins (Sec. 5.1 geometry; reading 21 of the design notes). The host accepts a geometry only
if the rounding bound 12 u (1 + t)^2 S + 2 u nb (u = 2^-24, S = (rs + rd) / db, t the
detector's half width over rs + rd) is at most half the margin.

Here the transpose's FP32 arithmetic is emulated exactly (numpy float32 operations round as the
GPU's do; a fused multiply-add is formed in float64 and rounded once) for every pixel of a
frame and several views at geometries near that limit. Its bin coordinates are compared with
an FP64 evaluation of the same central projection, and the error must lie within the bound.
The emulation's division is correctly rounded; the GPU's approximate division adds at most 2
ulp of t, which the bound's constant covers. The host checks: a geometry just beyond the limit
gets MOF_EUNSUPPORTED and one just below does not.
"""
import math

import numpy as np
import pytest

from paper_2501_12497_gb300 import api

U = 2.0 ** -24
PAD = 0.02
f32 = np.float32


def bound(S, nb):
    t = (0.5 * nb + 1.0) / S
    return 12.0 * U * (1.0 + t) ** 2 * S + 2.0 * U * nb


def fma32(a, b, c):
    return (np.float64(a) * np.float64(b) + np.float64(c)).astype(np.float32)


def bins_fp32(nx, ny, h, nb, rs, rd, db, th):
    """The transpose's bin coordinates of the four segment end points of every pixel, FP32."""
    cx, cy = 0.5 * (nx - 1) * h, 0.5 * (ny - 1) * h
    ex, ey = -math.sin(th), math.cos(th)
    qx0, qy0 = f32(-cx + rs * ex), f32(-cy + rs * ey)
    exf, eyf, fxf, fyf = f32(ex), f32(ey), f32(math.cos(th)), f32(math.sin(th))
    hf = f32(h)
    scale = f32((rs + rd) / db)
    toff = f32(0.5 * (nb - 1))
    y, x = np.meshgrid(np.arange(ny, dtype=np.float32), np.arange(nx, dtype=np.float32), indexing="ij")
    qx, qy = fma32(x, hf, qx0), fma32(y, hf, qy0)
    num = (qx * fxf + qy * fyf).astype(np.float32)
    den = (qx * exf + qy * eyf).astype(np.float32)
    nxp, dxp, nyp, dyp = hf * fxf, hf * exf, hf * fyf, hf * eyf
    ts = [(num + nxp) / (den + dxp), (num - nxp) / (den - dxp), (num + nyp) / (den + dyp), (num - nyp) / (den - dyp)]
    return [fma32(t.astype(np.float32), scale, toff) for t in ts]


def bins_fp64(nx, ny, h, nb, rs, rd, db, th):
    cx, cy = 0.5 * (nx - 1) * h, 0.5 * (ny - 1) * h
    ex, ey, fx, fy = -math.sin(th), math.cos(th), math.cos(th), math.sin(th)
    y, x = np.meshgrid(np.arange(ny, dtype=np.float64), np.arange(nx, dtype=np.float64), indexing="ij")
    qx, qy = x * h - cx + rs * ex, y * h - cy + rs * ey
    num, den = qx * fx + qy * fy, qx * ex + qy * ey
    S = (rs + rd) / db
    ts = [(num + h * fx) / (den + h * ex), (num - h * fx) / (den - h * ex), (num + h * fy) / (den + h * ey),
          (num - h * fy) / (den - h * ey)]
    return [t * S + 0.5 * (nb - 1) for t in ts]


def largest_accepted_scale(nb):
    """The largest S = (rs + rd) / db the bound accepts for nb bins (bisection)."""
    lo, hi = 1.0, 1e7
    for _ in range(200):
        mid = math.sqrt(lo * hi)
        lo, hi = (mid, hi) if bound(mid, nb) <= 0.5 * PAD else (lo, mid)
    return lo


@pytest.mark.parametrize("nx,nb,frac", [(64, 96, 1.0), (96, 400, 0.999), (48, 64, 0.5)])
def test_fp32_bin_search_error_is_within_the_bound_near_the_limit(nx, nb, frac):
    h = 1.0
    S = frac * largest_accepted_scale(nb)
    # a detector wide enough for the magnified field: rd chosen so that nb bins of width db
    # cover the field seen from the source; rs a few field widths away
    rs = 4.0 * nx * h
    db = 1.5 * nx * h / nb
    rd = S * db - rs
    assert rd > 0
    worst = 0.0
    for th in np.linspace(0.0, 2.0 * math.pi, 13)[:-1] + 0.137:
        b32 = bins_fp32(nx, nx, h, nb, rs, rd, db, th)
        b64 = bins_fp64(nx, nx, h, nb, rs, rd, db, th)
        for a, b in zip(b32, b64):
            on = (b > -1.0) & (b < nb)  # central projections that land on the detector
            if on.any():
                worst = max(worst, float(np.max(np.abs(a[on].astype(np.float64) - b[on]))))
    assert worst <= bound(S, nb) <= 0.5 * PAD + 1e-15, (worst, bound(S, nb))
    assert worst > 0.0  # the emulation does round


def test_host_accepts_below_and_rejects_beyond_the_bound():
    try:
        api.load()
    except Exception as e:  # pragma: no cover - the library is built by the session fixture
        pytest.skip("libmof not built: %s" % e)
    nx, nb, db = 32, 64, 1.0
    S = largest_accepted_scale(nb)
    na, ang = [2, 2], [0.0, 1.0, 0.5, 1.5]
    with pytest.raises(api.MofError) as e:
        api.mof_problem_create(nx, nx, 2, nb, na, ang, bin_size=db, fan=(1.01 * S * db, 0.0))
    assert e.value.status == api.MOF_EUNSUPPORTED and "rounding bound" in str(e.value)
    # just below: the fan check passes (without a GPU the creation may still fail later, on the
    # device, but not with MOF_EUNSUPPORTED)
    try:
        p = api.mof_problem_create(nx, nx, 2, nb, na, ang, bin_size=db, fan=(0.99 * S * db, 0.0))
        p.close()
    except api.MofError as err:
        assert err.status != api.MOF_EUNSUPPORTED, str(err)
