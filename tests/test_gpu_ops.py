"""GPU parity of every operator of the hot path against the FP64 oracle.

Inputs are seeded; the oracle receives exactly the values the GPU received
(float32 inputs widened to float64). Bars, on the relative 2-norm error and on the
element-wise error (largest difference over the largest reference value) alike:
<= 1e-5 for the FP32 operators (the per-operator tolerance of the precision form),
<= 1e-12 for the FP64 build, bit-exact for the integer decisions (reverse-flow
destinations). Sizes span several tiles with ragged tails, the 64x64x8
workload and full 256x256 frames with 30 angles and 363 bins.
"""
import numpy as np
import pytest

torch = pytest.importorskip("torch")

from oracle import ops as O
from paper_2501_12497_gb300 import api, synth

pytestmark = pytest.mark.gpu

TOL = {api.MOF_FP32: 1e-5, api.MOF_FP64: 1e-12}
DT = {api.MOF_FP32: (np.float32, torch.float32), api.MOF_FP64: (np.float64, torch.float64)}

# (nx, ny, nt, na, nb): ragged tiles, the 64x64x8 workload, full-size frames
SHAPES = [(37, 29, 3, 7, 45), (64, 64, 8, 16, 64), (256, 256, 3, 30, 363)]


@pytest.fixture(scope="module", autouse=True)
def _build():
    import __graft_entry__
    __graft_entry__.build()


def rel(a, b):
    """The larger of the relative 2-norm error and the element-wise error (the largest
    difference over the largest reference value), so that every bar holds for both."""
    a, b = np.ravel(a), np.ravel(b)
    e_norm = np.linalg.norm(a - b) / max(np.linalg.norm(b), 1e-300)
    e_elem = np.max(np.abs(a - b)) / max(np.max(np.abs(b)), 1e-300) if b.size else 0.0
    print("  errors: norm-wise %.3g element-wise %.3g" % (e_norm, e_elem))
    return max(e_norm, e_elem)


def make(shape, prec, seed=0, h=1.0, db=1.0):
    nx, ny, nt, na, nb = shape
    na_arr, ang = synth.shifted_angles(nt, na)
    p = api.mof_problem_create(nx, ny, nt, nb, na_arr, ang, h, db, prec)
    g = O.Geometry(nx, ny, nt, nb, na_arr, ang, h, db)
    return p, g


def dev(a, prec):
    npdt, tdt = DT[prec]
    return torch.tensor(np.ascontiguousarray(a, dtype=npdt), device="cuda").reshape(-1)


def host(t):
    torch.cuda.synchronize()
    return t.detach().cpu().double().numpy()


def empty(n, prec):
    return torch.full((n,), float("nan"), dtype=DT[prec][1], device="cuda")


@pytest.mark.parametrize("prec", [api.MOF_FP32, api.MOF_FP64])
@pytest.mark.parametrize("shape", SHAPES)
def test_project_and_backproject(shape, prec):
    p, g = make(shape, prec)
    nx, ny, nt = shape[:3]
    u = synth.random_images(nt, ny, nx, seed=1)
    b = np.random.default_rng(2).standard_normal(g.m)
    ud, bd = dev(u, prec), dev(b, prec)
    out_b, out_u = empty(p.m, prec), empty(p.n, prec)
    api.mof_apply_A(p, ud, out_b)
    api.mof_apply_AT(p, bd, out_u)
    assert rel(host(out_b), O.project(g, host(ud))) <= TOL[prec]
    assert rel(host(out_u), O.backproject(g, host(bd))) <= TOL[prec]


def test_projector_general_pixel_and_bin_size():
    """h != db: footprints span more than two bins in the backprojector."""
    for prec in (api.MOF_FP32, api.MOF_FP64):
        p, g = make((40, 33, 2, 9, 101), prec, h=1.7, db=0.6)
        u = synth.random_images(2, 33, 40, seed=3)
        b = np.random.default_rng(4).standard_normal(g.m)
        ud, bd = dev(u, prec), dev(b, prec)
        ob, ou = empty(p.m, prec), empty(p.n, prec)
        api.mof_apply_A(p, ud, ob)
        api.mof_apply_AT(p, bd, ou)
        assert rel(host(ob), O.project(g, host(ud))) <= TOL[prec]
        assert rel(host(ou), O.backproject(g, host(bd))) <= TOL[prec]


def test_projector_adjoint_identity_fp32():
    p, g = make((256, 256, 2, 30, 363), api.MOF_FP32)
    u = dev(synth.random_images(2, 256, 256, seed=5), api.MOF_FP32)
    b = dev(np.random.default_rng(6).standard_normal(g.m), api.MOF_FP32)
    hb, hu = empty(p.m, api.MOF_FP32), empty(p.n, api.MOF_FP32)
    api.mof_apply_A(p, u, hb)
    api.mof_apply_AT(p, b, hu)
    lhs = np.dot(host(hb), host(b))
    rhs = np.dot(host(u), host(hu))
    assert abs(lhs - rhs) <= 1e-5 * np.linalg.norm(host(hb)) * np.linalg.norm(host(b))


# ------------------------------------------------------------ fan beam
# (nx, ny, nt, na, nb, db, rs, rd): ragged tiles with a wide fan and a detector through
# the centre, the 64x64x8 fan workload, full-size frames of the 256x256x32 fan workload
FAN = [(37, 29, 3, 7, 61, 1.1, 30.0, 0.0), (64, 64, 8, 16, 100, 1.5, 128.0, 64.0),
       (256, 256, 2, 30, 363, 1.6, 512.0, 256.0)]


def make_fan(case, prec, seed=0):
    nx, ny, nt, na, nb, db, rs, rd = case
    na_arr, ang = synth.shifted_angles(nt, na)
    ang = ang + np.deg2rad(7.0) * seed
    p = api.mof_problem_create(nx, ny, nt, nb, na_arr, ang, 1.0, db, prec, fan=(rs, rd))
    g = O.Geometry(nx, ny, nt, nb, na_arr, ang, 1.0, db, fan=(rs, rd))
    return p, g


@pytest.mark.parametrize("prec", [api.MOF_FP32, api.MOF_FP64])
@pytest.mark.parametrize("case", FAN)
def test_fan_project_and_backproject(case, prec):
    """Fan-beam H and H^T (flat detector, Sec. 5.1) against the oracle's rays through the
    source; the views include fans that straddle 45 degrees."""
    p, g = make_fan(case, prec)
    nx, ny, nt = case[:3]
    u = synth.random_images(nt, ny, nx, seed=31)
    b = np.random.default_rng(32).standard_normal(g.m)
    ud, bd = dev(u, prec), dev(b, prec)
    out_b, out_u = empty(p.m, prec), empty(p.n, prec)
    api.mof_apply_A(p, ud, out_b)
    api.mof_apply_AT(p, bd, out_u)
    assert rel(host(out_b), O.project(g, host(ud))) <= TOL[prec]
    assert rel(host(out_u), O.backproject(g, host(bd))) <= TOL[prec]


@pytest.mark.parametrize("prec,tol", [(api.MOF_FP32, 1e-5), (api.MOF_FP64, 1e-13)])
def test_fan_projector_adjoint_identity(prec, tol):
    p, g = make_fan(FAN[2], prec, seed=1)
    nx, ny, nt = FAN[2][:3]
    u = dev(synth.random_images(nt, ny, nx, seed=33), prec)
    b = dev(np.random.default_rng(34).standard_normal(g.m), prec)
    hb, hu = empty(p.m, prec), empty(p.n, prec)
    api.mof_apply_A(p, u, hb)
    api.mof_apply_AT(p, b, hu)
    lhs, rhs = np.dot(host(hb), host(b)), np.dot(host(u), host(hu))
    assert abs(lhs - rhs) <= tol * np.linalg.norm(host(hb)) * np.linalg.norm(host(b))


def test_fan_rejects_a_source_inside_the_field():
    na_arr, ang = synth.shifted_angles(2, 4)
    for rs, rd in ((20.0, 5.0), (60.0, -1.0), (float("inf"), 1.0)):
        with pytest.raises(api.MofError):
            api.mof_problem_create(32, 32, 2, 64, na_arr, ang, 1.0, 1.0, api.MOF_FP32, fan=(rs, rd))


@pytest.mark.parametrize("prec", [api.MOF_FP32, api.MOF_FP64])
@pytest.mark.parametrize("shape", SHAPES)
def test_grad_and_transpose(shape, prec):
    p, g = make(shape, prec)
    nx, ny, nt = shape[:3]
    u = dev(synth.random_images(nt, ny, nx, seed=7), prec)
    gg = dev(np.random.default_rng(8).standard_normal(2 * p.n), prec)
    og, ou = empty(2 * p.n, prec), empty(p.n, prec)
    api.mof_apply_grad(p, u, og)
    api.mof_apply_gradT(p, gg, ou)
    assert rel(host(og), O.grad(host(u).reshape(nt, ny, nx))) <= TOL[prec]
    assert rel(host(ou), O.gradT(host(gg).reshape(nt, 2, ny, nx))) <= TOL[prec]


@pytest.mark.parametrize("prec", [api.MOF_FP32, api.MOF_FP64])
@pytest.mark.parametrize("shape", SHAPES)
def test_flow_and_transpose(shape, prec):
    p, g = make(shape, prec)
    nx, ny, nt = shape[:3]
    u = dev(synth.random_images(nt, ny, nx, seed=9), prec)
    s = dev(synth.random_velocities(nt - 1, ny, nx, 2.5, seed=10), prec)
    sr = dev(synth.random_velocities(nt - 1, ny, nx, 3.5, seed=11), prec)
    r = dev(np.random.default_rng(12).standard_normal(2 * (nt - 1) * nx * ny), prec)
    orr, ou = empty(r.numel(), prec), empty(p.n, prec)
    api.mof_apply_flow(p, u, s, sr, orr)
    api.mof_apply_flowT(p, r, s, sr, ou)
    sh = (nt - 1, 2, ny, nx)
    hs, hsr = host(s).reshape(sh), host(sr).reshape(sh)
    assert rel(host(orr), O.flow(host(u).reshape(nt, ny, nx), hs, hsr)) <= TOL[prec]
    assert rel(host(ou), O.flowT(host(r).reshape(2, nt - 1, ny, nx), hs, hsr)) <= TOL[prec]


def test_flow_large_and_out_of_grid_velocities():
    """Velocities that push samples far outside the frame (clipping) and a wide window."""
    prec = api.MOF_FP32
    shape = (48, 40, 3, 4, 40)
    p, g = make(shape, prec)
    nx, ny, nt = shape[:3]
    rng = np.random.default_rng(13)
    u = dev(synth.random_images(nt, ny, nx, seed=14), prec)
    s = dev(rng.uniform(-9, 9, (nt - 1, 2, ny, nx)), prec)
    sr = dev(rng.uniform(-1, 1, (nt - 1, 2, ny, nx)), prec)
    r = dev(rng.standard_normal(2 * (nt - 1) * nx * ny), prec)
    orr, ou = empty(r.numel(), prec), empty(p.n, prec)
    api.mof_apply_flow(p, u, s, sr, orr)
    api.mof_apply_flowT(p, r, s, sr, ou)
    sh = (nt - 1, 2, ny, nx)
    assert rel(host(orr), O.flow(host(u).reshape(nt, ny, nx), host(s).reshape(sh), host(sr).reshape(sh))) <= 1e-5
    assert rel(host(ou), O.flowT(host(r).reshape(2, nt - 1, ny, nx), host(s).reshape(sh), host(sr).reshape(sh))) <= 1e-5


@pytest.mark.parametrize("prec", [api.MOF_FP32, api.MOF_FP64])
@pytest.mark.parametrize("shape", SHAPES)
def test_of_fields_flow_lin_and_vgrad(shape, prec):
    p, g = make(shape, prec)
    nx, ny, nt = shape[:3]
    P = nt - 1
    u = dev(synth.random_images(nt, ny, nx, seed=15), prec)
    for dr in (1, 2):
        ux, uy, ut = (empty(P * nx * ny, prec) for _ in range(3))
        api.mof_of_fields(p, u, dr, ux, uy, ut)
        rx, ry, rt = O.of_fields(host(u).reshape(nt, ny, nx), dr)
        assert rel(host(ux), rx) <= TOL[prec] and rel(host(uy), ry) <= TOL[prec] and rel(host(ut), rt) <= TOL[prec]
    s = dev(synth.random_velocities(P, ny, nx, 2.0, seed=16), prec)
    r = dev(np.random.default_rng(17).standard_normal(P * nx * ny), prec)
    lin, gs = empty(P * nx * ny, prec), empty(p.nv, prec)
    api.mof_apply_flow_lin(p, ux, uy, ut, s, lin)
    api.mof_apply_flow_linT(p, ux, uy, r, gs)
    sh = (P, ny, nx)
    hux, huy, hut = host(ux).reshape(sh), host(uy).reshape(sh), host(ut).reshape(sh)
    assert rel(host(lin), O.flow_lin(hux, huy, hut, host(s).reshape(P, 2, ny, nx))) <= TOL[prec]
    assert rel(host(gs), O.flow_linT(hux, huy, host(r).reshape(sh))) <= TOL[prec]
    vg, vt = empty(2 * p.nv, prec), empty(p.nv, prec)
    gsv = dev(np.random.default_rng(18).standard_normal(2 * p.nv), prec)
    api.mof_apply_vgrad(p, s, vg)
    api.mof_apply_vgradT(p, gsv, vt)
    assert rel(host(vg), O.vgrad(host(s).reshape(P, 2, ny, nx))) <= TOL[prec]
    assert rel(host(vt), O.vgradT(host(gsv).reshape(P, 2, 2, ny, nx))) <= TOL[prec]


@pytest.mark.parametrize("prec", [api.MOF_FP32, api.MOF_FP64])
def test_reverse_flow_bit_exact(prec):
    """Destinations are integer decisions: identical to the oracle's, so the averaged
    reverse velocities agree to rounding (FP32: the cast of an FP64 average)."""
    shape = (53, 47, 4, 4, 40)
    p, g = make(shape, prec)
    nx, ny, nt = shape[:3]
    rng = np.random.default_rng(19)
    sv = synth.random_velocities(nt - 1, ny, nx, 3.0, seed=20)
    # plant exact half-way positions and negative half-way positions
    sv[0, 0, :5, :5] = 0.5
    sv[0, 0, 5:10, :5] = -0.5
    sv[1, 1, :7, :] = -1.5
    s = dev(sv, prec)
    sr = empty(p.nv, prec)
    api.mof_reverse_flow(p, s, sr)
    want = O.reverse_flow(host(s).reshape(nt - 1, 2, ny, nx))
    got = host(sr).reshape(want.shape)
    if prec == api.MOF_FP64:
        np.testing.assert_array_equal(got, want)
    else:
        np.testing.assert_array_equal(got, want.astype(np.float32).astype(np.float64))


@pytest.mark.parametrize("prec", [api.MOF_FP32, api.MOF_FP64])
@pytest.mark.parametrize("shape", SHAPES[:2] + [(256, 256, 3, 30, 363)])
def test_reg_normal(shape, prec):
    """y = Theta^T W Theta x with W from uk (Alg. 1 weights), against the oracle's Theta."""
    from oracle import solver as OS
    p, g = make(shape, prec)
    nx, ny, nt = shape[:3]
    x = dev(synth.random_images(nt, ny, nx, seed=21), prec)
    uk = dev(synth.random_images(nt, ny, nx, seed=22), prec)
    s = dev(synth.random_velocities(nt - 1, ny, nx, 2.0, seed=23), prec)
    sr = dev(synth.random_velocities(nt - 1, ny, nx, 2.0, seed=24), prec)
    eps = 0.05
    y = empty(p.n, prec)
    api.mof_apply_reg_normal(p, x, uk, s, sr, eps, y)
    sh = (nt - 1, 2, ny, nx)
    th = OS.Theta((nt, ny, nx), host(s).reshape(sh), host(sr).reshape(sh))
    nu = th(host(uk))
    w = 1.0 / np.sqrt(nu * nu + eps * eps)
    want = th.T(w * th(host(x)))
    print("reg_normal %s rel %.3g" % (prec, rel(host(y), want)))
    assert rel(host(y), want) <= TOL[prec]


# ------------------------------------------------ rounding-and-clipping M(s)
def _round_velocities(nt, ny, nx, seed):
    """Velocities with planted exact halves (the tie rule), integers and far out-of-grid values."""
    rng = np.random.default_rng(seed)
    v = rng.uniform(-4.0, 4.0, (nt - 1, 2, ny, nx))
    v[0, 0, :3, :] = 0.5
    v[0, 1, 3:6, :] = -0.5
    v[-1, 0, :, :2] = 1.5
    v[-1, 1, :, 2:4] = -2.5
    v[0, :, -2:, :] = np.round(v[0, :, -2:, :])
    v[-1, 0, -1, :] = 40.0
    v[-1, 1, -2, :] = -40.0
    return v


@pytest.mark.parametrize("prec", [api.MOF_FP32, api.MOF_FP64])
@pytest.mark.parametrize("shape", SHAPES[:2] + [(256, 256, 3, 30, 363)])
def test_round_warp_flow_transpose_and_vjp(shape, prec):
    """Mhat with the rounding-and-clipping M(s) (Sec. 3): forward rows bit-exact against the
    oracle (one subtraction of a picked pixel), the transpose to rounding, the velocity VJP
    zero; setting the mode back restores the bilinear rows."""
    p, g = make(shape, prec)
    nx, ny, nt = shape[:3]
    u = dev(synth.random_images(nt, ny, nx, seed=41), prec)
    s = dev(_round_velocities(nt, ny, nx, 42), prec)
    sr = dev(_round_velocities(nt, ny, nx, 43), prec)
    r = dev(np.random.default_rng(44).standard_normal(2 * (nt - 1) * nx * ny), prec)
    sh = (nt - 1, 2, ny, nx)
    hs, hsr, hu = host(s).reshape(sh), host(sr).reshape(sh), host(u).reshape(nt, ny, nx)
    api.mof_set_warp(p, 1)
    orr, ou = empty(r.numel(), prec), empty(p.n, prec)
    api.mof_apply_flow(p, u, s, sr, orr)
    api.mof_apply_flowT(p, r, s, sr, ou)
    want = O.flow_round(hu, hs, hsr)
    if prec == api.MOF_FP64:
        np.testing.assert_array_equal(host(orr), want.ravel())
    else:
        np.testing.assert_array_equal(host(orr), want.astype(np.float32).astype(np.float64).ravel())
    assert rel(host(ou), O.flowT_round(host(r).reshape(2, nt - 1, ny, nx), hs, hsr)) <= TOL[prec]
    gs, gsr = empty(p.nv, prec), empty(p.nv, prec)
    api.mof_apply_flow_ds(p, u, s, sr, r, gs, gsr)
    assert not host(gs).any() and not host(gsr).any()
    api.mof_set_warp(p, 0)
    api.mof_apply_flow(p, u, s, sr, orr)
    assert rel(host(orr), O.flow(hu, hs, hsr)) <= TOL[prec]


@pytest.mark.parametrize("prec", [api.MOF_FP32, api.MOF_FP64])
def test_round_warp_reg_normal(prec):
    """Theta^T W Theta x with the rounding M(s) against the oracle's Theta(warp_round=True)."""
    from oracle import solver as OS
    shape = (64, 64, 8, 16, 64)
    p, g = make(shape, prec)
    nx, ny, nt = shape[:3]
    x = dev(synth.random_images(nt, ny, nx, seed=45), prec)
    uk = dev(synth.random_images(nt, ny, nx, seed=46), prec)
    s = dev(_round_velocities(nt, ny, nx, 47), prec)
    sr = dev(_round_velocities(nt, ny, nx, 48), prec)
    eps = 0.05
    y = empty(p.n, prec)
    api.mof_set_warp(p, 1)
    api.mof_apply_reg_normal(p, x, uk, s, sr, eps, y)
    sh = (nt - 1, 2, ny, nx)
    th = OS.Theta((nt, ny, nx), host(s).reshape(sh), host(sr).reshape(sh), warp_round=True)
    nu = th(host(uk))
    want = th.T(th(host(x)) / np.sqrt(nu * nu + eps * eps))
    print("reg_normal %s rel %.3g" % (prec, rel(host(y), want)))
    assert rel(host(y), want) <= TOL[prec]


def test_set_warp_rejects_unknown_modes():
    p, g = make(SHAPES[0], api.MOF_FP32)
    for mode in (-1, 2):
        with pytest.raises(api.MofError):
            api.mof_set_warp(p, mode)


# ------------------------------------------------------------ rescaling for Solve-OF
@pytest.mark.parametrize("prec,tol", [(api.MOF_FP32, 1e-6), (api.MOF_FP64, 1e-14)])
@pytest.mark.parametrize("a", [2, 4, 8])
def test_downsample_and_upsample_velocity_match_oracle(prec, tol, a):
    """Block means of the frames and the bilinear velocity upscaling (Sec. 4.1.5) against
    the oracle, on 96x56 frames (several thread blocks, a ragged last block)."""
    nx, ny, nt = 96, 56, 5
    p, g = make((nx, ny, nt, 3, 20), prec)
    u = synth.random_images(nt, ny, nx, seed=3)
    uc = empty(nt * (ny // a) * (nx // a), prec)
    api.mof_downsample(p, a, dev(u, prec), uc)
    assert rel(host(uc), O.downsample(u.astype(DT[prec][0]), a)) <= tol
    sc = synth.random_velocities(nt - 1, ny // a, nx // a, vmax=2.0, seed=4)
    s = empty(p.nv, prec)
    api.mof_upsample_velocity(p, a, dev(sc, prec), s)
    assert rel(host(s), O.upsample_velocity(sc.astype(DT[prec][0]), a)) <= tol


def test_rescaling_rejects_factors_that_do_not_divide_the_frame():
    p, _ = make((48, 40, 3, 3, 20), api.MOF_FP32)
    u = torch.zeros(p.n, device="cuda")
    with pytest.raises(api.MofError) as e:
        api.mof_downsample(p, 3, u, torch.zeros(p.nt * 13 * 16, device="cuda"))
    assert e.value.status == api.MOF_EINVAL
