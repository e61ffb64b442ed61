"""GPU parity of Solve-OF (Alg. 2) and MMGKS-OF (Alg. 1) against the FP64 oracle.

FP64 build: the GPU runs the same algorithm with a different but equivalent
small-problem factorisation (Gram + Cholesky + Jacobi instead of Householder
QR + SVD) and a different lambda search (safeguarded Newton instead of bisection and
golden section), so results agree to ~1e-8 rather than to the last bit.
FP32 operators with FP64 Krylov/projected solves: the precision form's bar of
1e-4 relative error on images and velocities after the fixed iteration count.
"""
import numpy as np
import pytest

torch = pytest.importorskip("torch")

from oracle import ops as O
from oracle import solver as OS
from paper_2501_12497_gb300 import api, synth

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _build():
    import __graft_entry__
    __graft_entry__.build()


def rel(a, b):
    return np.linalg.norm(np.ravel(a) - np.ravel(b)) / max(np.linalg.norm(np.ravel(b)), 1e-300)


def problem(w, prec):
    return api.mof_problem_create(w.nx, w.ny, w.nt, w.nb, w.na, w.angles, w.h, w.db, prec)


def geom(w):
    return O.Geometry(w.nx, w.ny, w.nt, w.nb, w.na, w.angles, w.h, w.db)


def tdt(prec):
    return torch.float64 if prec == api.MOF_FP64 else torch.float32


def npdt(prec):
    return np.float64 if prec == api.MOF_FP64 else np.float32


@pytest.mark.parametrize("prec,tol", [(api.MOF_FP64, 1e-7), (api.MOF_FP32, 1e-3)])
def test_solve_of_matches_oracle(prec, tol):
    w = synth.moving_disks(48, 4, 8, 48, radii=(6.0, 9.0), seed=1)
    p = problem(w, prec)
    u = w.u_true.astype(npdt(prec))
    ud = torch.tensor(u, device="cuda").reshape(-1)
    s = torch.empty(p.nv, dtype=tdt(prec), device="cuda")
    prm = api.mof_default_params(of_ell=6, of_iters=8)
    api.mof_solve_of(p, prm, ud, s)
    oprm = OS.Params(of_ell=6, of_iters=8)
    want = OS.solve_of(u.astype(np.float64), oprm)
    got = s.cpu().double().numpy().reshape(want.shape)
    assert rel(got, want) <= tol, rel(got, want)


@pytest.mark.parametrize("prec,tol", [(api.MOF_FP64, 1e-6), (api.MOF_FP32, 3e-3)])
def test_solve_of_pq1_matches_oracle(prec, tol):
    """Solve-OF with p = q = 1 (MM-GKS, App. A): IRLS weights from the current velocity,
    the weighted Grams of the whole basis every iteration, the weighted residual."""
    w = synth.moving_disks(48, 4, 8, 48, radii=(6.0, 9.0), seed=1)
    p = problem(w, prec)
    u = w.u_true.astype(npdt(prec))
    ud = torch.tensor(u, device="cuda").reshape(-1)
    s = torch.empty(p.nv, dtype=tdt(prec), device="cuda")
    api.mof_solve_of(p, api.mof_default_params(of_ell=6, of_iters=8, of_pq=1), ud, s)
    want = OS.solve_of(u.astype(np.float64), OS.Params(of_ell=6, of_iters=8, of_pq=1))
    got = s.cpu().double().numpy().reshape(want.shape)
    assert rel(got, want) <= tol, rel(got, want)
    two = OS.solve_of(u.astype(np.float64), OS.Params(of_ell=6, of_iters=8))
    assert rel(got, two) > 0.1  # the l1 norms give another flow


@pytest.mark.parametrize("prec,tol", [(api.MOF_FP64, 1e-6), (api.MOF_FP32, 1e-2)])
def test_solve_of_pq1_basis_beyond_32_and_ragged_tiles(prec, tol):
    """p = q = 1 with the basis growing from 30 to 63 vectors (past 60 the weighted Gram
    has more 4x4 blocks than threads and each thread takes two) on frames whose pixel
    count is not a multiple of the Gram tile. FP32: 34 MM iterations whose weights reach
    1/eps = 1e3 carry the FP32 rounding of the Grams into the iterates (3e-3 measured)."""
    w = synth.moving_disks(37, 3, 8, 37, radii=(5.0, 7.0), seed=3)
    p = problem(w, prec)
    u = w.u_true.astype(npdt(prec))
    s = torch.empty(p.nv, dtype=tdt(prec), device="cuda")
    api.mof_solve_of(p, api.mof_default_params(of_ell=30, of_iters=34, of_pq=1), torch.tensor(u, device="cuda").reshape(-1), s)
    want = OS.solve_of(u.astype(np.float64), OS.Params(of_ell=30, of_iters=34, of_pq=1))
    got = s.cpu().double().numpy().reshape(want.shape)
    assert rel(got, want) <= tol, rel(got, want)


def test_solve_of_pq1_stream_groups_do_not_change_the_result():
    w = synth.moving_disks(40, 8, 8, 40, radii=(5.0, 8.0), seed=6)
    p = problem(w, api.MOF_FP32)
    u = torch.tensor(w.u_true.astype(np.float32), device="cuda").reshape(-1)
    out = []
    for g in (1, 3, 7):
        s = torch.empty(p.nv, dtype=torch.float32, device="cuda")
        api.mof_solve_of(p, api.mof_default_params(of_ell=5, of_iters=6, of_streams=g, of_pq=1), u, s)
        out.append(s.cpu())
    for o in out[1:]:
        assert torch.equal(o, out[0])


def test_solve_of_rejects_unknown_norms():
    w = synth.moving_disks(32, 3, 8, 32, radii=(5.0, 7.0), seed=2)
    p = problem(w, api.MOF_FP32)
    s = torch.empty(p.nv, dtype=torch.float32, device="cuda")
    u = torch.tensor(w.u_true.astype(np.float32), device="cuda").reshape(-1)
    for pq in (0, 3):
        with pytest.raises(api.MofError):
            api.mof_solve_of(p, api.mof_default_params(of_pq=pq), u, s)


def test_solve_of_zero_pairs_give_zero_velocity():
    w = synth.moving_disks(32, 3, 8, 32, radii=(5.0, 7.0), seed=2)
    u = w.u_true.copy()
    u[1] = u[0]  # pair 0 has u_t = 0
    p = problem(w, api.MOF_FP64)
    s = torch.full((p.nv,), 7.0, dtype=torch.float64, device="cuda")
    api.mof_solve_of(p, api.mof_default_params(of_ell=4, of_iters=4), torch.tensor(u, device="cuda").reshape(-1), s)
    got = s.cpu().numpy().reshape(2, 2, 32, 32)
    assert np.all(got[0] == 0) and np.any(got[1] != 0)


def _oracle_solve(w, n_outer, **kw):
    prm = OS.Params(noise_norm=w.noise_norm, **kw)
    return OS.mmgks_of(geom(w), w.b, prm, n_outer)


def _gpu_solve(w, prec, n_outer, host=False, **kw):
    p = problem(w, prec)
    prm = api.mof_default_params(noise_norm=w.noise_norm, **kw)
    if host:
        u = np.empty(p.n, dtype=npdt(prec))
        s = np.empty(p.nv, dtype=npdt(prec))
        rep = api.mof_solve_host(p, prm, n_outer, w.b.astype(npdt(prec)), u, s)
        return u.astype(np.float64), s.astype(np.float64), rep
    b = torch.tensor(w.b.astype(npdt(prec)), device="cuda")
    u = torch.empty(p.n, dtype=tdt(prec), device="cuda")
    s = torch.empty(p.nv, dtype=tdt(prec), device="cuda")
    rep = api.mof_solve(p, prm, n_outer, b, u, s)
    return u.cpu().double().numpy(), s.cpu().double().numpy(), rep


def test_mmgks_of_fp64_matches_oracle_small():
    w = synth.moving_disks(32, 3, 8, 32, radii=(5.0, 8.0), seed=0)
    kw = dict(ell=4, of_ell=3, of_iters=3)
    ores = _oracle_solve(w, 4, **kw)
    u, s, rep = _gpu_solve(w, api.MOF_FP64, 4, **kw)
    assert rel(u, ores.u) <= 1e-7
    assert rel(s, ores.s) <= 1e-6
    for r, o in zip(rep, ores.report):
        assert abs(r["lambda"] / o["lam"] - 1) < 1e-6 and r["flag"] == o["flag"] and r["basis"] == o["basis"]
        assert abs(r["resid"] / o["resid"] - 1) < 1e-8


def test_mmgks_of_fp64_matches_oracle_disks64():
    """The plain FP64 method on the 64x64x8 two-disk workload (16 angles, 64 bins, 1% noise),
    10 outer iterations with Solve-OF every iteration."""
    w = synth.plain_fp64(0)
    ores = _oracle_solve(w, 10)
    u, s, rep = _gpu_solve(w, api.MOF_FP64, 10)
    assert rel(u, ores.u) <= 1e-6, rel(u, ores.u)
    assert rel(s, ores.s) <= 1e-5, rel(s, ores.s)


def test_mmgks_of_fp32_precision_form_small():
    """FP32 operators, FP64 Krylov and projected solves, on a reduced instance of the ellipse
    generator (96x96, T=6, 30 angles, 137 bins)."""
    w = synth.precision_form_small(0)
    ores = _oracle_solve(w, 6, of_iters=10)
    u, s, rep = _gpu_solve(w, api.MOF_FP32, 6, of_iters=10)
    eu, es = rel(u, ores.u), rel(s, ores.s)
    print("fp32 rel err u %.3g s %.3g" % (eu, es))
    assert eu <= 1e-4 and es <= 1e-3


def test_solve_host_matches_device():
    w = synth.moving_disks(32, 3, 8, 32, radii=(5.0, 8.0), seed=3)
    kw = dict(ell=4, of_ell=3, of_iters=3)
    u1, s1, _ = _gpu_solve(w, api.MOF_FP32, 3, **kw)
    u2, s2, _ = _gpu_solve(w, api.MOF_FP32, 3, host=True, **kw)
    np.testing.assert_array_equal(u1, u2)
    np.testing.assert_array_equal(s1, s2)


def test_repeated_solves_are_bit_identical():
    w = synth.moving_disks(40, 4, 8, 40, radii=(5.0, 8.0), seed=4)
    kw = dict(ell=5, of_ell=4, of_iters=4)
    a = _gpu_solve(w, api.MOF_FP32, 4, **kw)
    b = _gpu_solve(w, api.MOF_FP32, 4, **kw)
    np.testing.assert_array_equal(a[0], b[0])
    np.testing.assert_array_equal(a[1], b[1])


def test_zero_data_gives_zero_image():
    w = synth.moving_disks(32, 3, 8, 32, radii=(5.0, 8.0), seed=5)
    w.b = np.zeros_like(w.b)
    w.noise_norm = 0.0
    u, s, rep = _gpu_solve(w, api.MOF_FP64, 2, ell=3, of_ell=2, of_iters=2)
    assert np.all(u == 0) and np.all(s == 0)


def test_full_size_precision_form_properties():
    """The bench configuration (256x256x32, 30 angles, 363 bins, 30 outer iterations with
    Solve-OF of 20 GKS iterations on all 31 pairs), checked through properties the oracle's
    definition fixes at any size: wherever DP found a root the data misfit equals eta*delta;
    the bases grow by one per iteration; the result is reproducible bit for bit; the
    reconstruction is closer to the phantom than the zero image by a wide margin. The misfit
    is evaluated in FP32 (H V z - b with a 1% misfit loses two digits), hence 1e-4."""
    w = synth.precision_form(0)
    p = problem(w, api.MOF_FP32)
    prm = api.mof_default_params(noise_norm=w.noise_norm)
    b = torch.tensor(w.b.astype(np.float32), device="cuda")
    u1 = torch.empty(p.n, dtype=torch.float32, device="cuda")
    u2 = torch.empty_like(u1)
    rep = api.mof_solve(p, prm, 30, b, u1)
    api.mof_solve(p, prm, 30, b, u2)
    assert torch.equal(u1, u2)
    target = prm.eta * w.noise_norm
    for k, r in enumerate(rep):
        assert r["basis"] == 10 + k
        if r["flag"] == 0:
            assert abs(r["resid"] / target - 1) < 1e-4, (k, r)
        if k > 0:
            assert r["of_basis_min"] == r["of_basis_max"] == 29
    u = u1.cpu().double().numpy()
    assert rel(u, w.u_true) < 0.15


@pytest.mark.parametrize("prec", [api.MOF_FP32, api.MOF_FP64])
def test_solve_of_stream_groups_do_not_change_the_result(prec):
    """Solve-OF run as 1, 3 (uneven), 7 (one pair each) and 32 (more groups than
    pairs: one pair each) groups of frame pairs on separate streams: every kernel
    works per pair, so the velocities agree bit for bit."""
    w = synth.moving_disks(40, 8, 8, 40, radii=(5.0, 8.0), seed=6)
    p = problem(w, prec)
    u = torch.tensor(w.u_true.astype(npdt(prec)), device="cuda").reshape(-1)
    out = []
    for g in (1, 3, 7, 32):
        s = torch.empty(p.nv, dtype=tdt(prec), device="cuda")
        api.mof_solve_of(p, api.mof_default_params(of_ell=5, of_iters=6, of_streams=g), u, s)
        out.append(s.cpu())
    assert all(torch.equal(out[0], o) for o in out[1:])


def test_mmgks_of_stream_groups_do_not_change_the_result():
    w = synth.moving_disks(40, 6, 8, 40, radii=(5.0, 8.0), seed=7)
    kw = dict(ell=5, of_ell=4, of_iters=5)
    a = _gpu_solve(w, api.MOF_FP32, 4, of_streams=1, **kw)
    b = _gpu_solve(w, api.MOF_FP32, 4, of_streams=4, **kw)
    np.testing.assert_array_equal(a[0], b[0])
    np.testing.assert_array_equal(a[1], b[1])


@pytest.mark.parametrize("prec,tol", [(api.MOF_FP64, 1e-7), (api.MOF_FP32, 1e-3)])
def test_solve_of_basis_beyond_32_matches_oracle(prec, tol):
    """Solve-OF with of_ell = 20 and 15 GKS iterations: the basis grows to 34 vectors, past
    the 32 the small solver keeps in registers (its shared-memory Jacobi path runs)."""
    w = synth.moving_disks(48, 4, 8, 48, radii=(6.0, 9.0), seed=8)
    p = problem(w, prec)
    u = w.u_true.astype(npdt(prec))
    ud = torch.tensor(u, device="cuda").reshape(-1)
    s = torch.empty(p.nv, dtype=tdt(prec), device="cuda")
    api.mof_solve_of(p, api.mof_default_params(of_ell=20, of_iters=15), ud, s)
    want = OS.solve_of(u.astype(np.float64), OS.Params(of_ell=20, of_iters=15))
    got = s.cpu().double().numpy().reshape(want.shape)
    assert rel(got, want) <= tol, rel(got, want)


def test_mmgks_of_fp64_image_basis_beyond_32_matches_oracle():
    """MMGKS-OF with ell = 26 and 8 outer iterations: the image-step basis grows from 26 to
    33 vectors, through the sizes where the weighted Theta Gram splits its 4x4 blocks into
    row groups that do not divide a tile evenly (K = 29..32), and past the 32 of the small
    solver's register path. 40x40x3 frames, 20 angles, 58 bins: enough data rows that
    33 Golub-Kahan vectors stay well conditioned (rounding-level perturbations move the
    oracle's own result by ~1e-9)."""
    w = synth.moving_disks(40, 3, 20, 58, radii=(5.0, 8.0), seed=9)
    kw = dict(ell=26, of_ell=3, of_iters=3)
    ores = _oracle_solve(w, 8, **kw)
    u, s, rep = _gpu_solve(w, api.MOF_FP64, 8, **kw)
    assert max(r["basis"] for r in rep) > 32
    assert rel(u, ores.u) <= 1e-7, rel(u, ores.u)
    assert rel(s, ores.s) <= 1e-6, rel(s, ores.s)


def test_solve_of_graph_replay_matches_eager_run():
    """mof_solve_of captures its Solve-OF into a graph (over workspace copies of u and s)
    and replays it; with timing on it runs eagerly. Both give the same velocities bit for
    bit, across calls with different input and output buffers and a parameter change."""
    w = synth.moving_disks(40, 4, 8, 40, radii=(5.0, 8.0), seed=10)
    p = problem(w, api.MOF_FP32)
    outs = []
    for timing, of_iters in ((0, 5), (0, 5), (1, 5), (0, 6), (1, 6)):
        api.mof_set_timing(p, timing)
        u = torch.tensor(w.u_true.astype(np.float32), device="cuda").reshape(-1).clone()
        s = torch.full((p.nv,), float("nan"), dtype=torch.float32, device="cuda")
        api.mof_solve_of(p, api.mof_default_params(of_ell=4, of_iters=of_iters), u, s)
        outs.append(s.cpu())
    api.mof_set_timing(p, 0)
    assert torch.equal(outs[0], outs[1]) and torch.equal(outs[0], outs[2])
    assert torch.equal(outs[3], outs[4]) and not torch.equal(outs[0], outs[3])


@pytest.mark.parametrize("prec,tol", [(api.MOF_FP64, 1e-7), (api.MOF_FP32, 1e-3)])
def test_solve_of_on_downsampled_frames_matches_oracle(prec, tol):
    """Solve-OF with of_scale = 2 (Sec. 4.1.5): on the 2x2 block means of the frames, the
    velocities upscaled bilinearly and doubled, against the oracle's composition."""
    w = synth.moving_disks(48, 4, 8, 48, radii=(6.0, 9.0), seed=11)
    p = problem(w, prec)
    u = w.u_true.astype(npdt(prec))
    s = torch.empty(p.nv, dtype=tdt(prec), device="cuda")
    api.mof_solve_of(p, api.mof_default_params(of_ell=6, of_iters=8, of_scale=2), torch.tensor(u, device="cuda").reshape(-1), s)
    oprm = OS.Params(of_ell=6, of_iters=8)
    want = O.upsample_velocity(OS.solve_of(O.downsample(u.astype(np.float64), 2), oprm), 2)
    got = s.cpu().double().numpy().reshape(want.shape)
    assert rel(got, want) <= tol, rel(got, want)


def test_mmgks_of_fp64_with_downsampled_solve_of_and_tau_matches_oracle():
    """MMGKS-OF with Solve-OF on frames downsampled by 2, every second outer iteration
    (tau = 2), on the 64x64x8 two-disk workload."""
    w = synth.plain_fp64(0)
    kw = dict(of_scale=2, tau=2)
    ores = _oracle_solve(w, 6, **kw)
    u, s, rep = _gpu_solve(w, api.MOF_FP64, 6, **kw)
    assert rel(u, ores.u) <= 1e-6, rel(u, ores.u)
    assert rel(s, ores.s) <= 1e-5, rel(s, ores.s)
    # Solve-OF ran on the even outer iterations from k = 2 on (at k = 0 the image is zero)
    assert [r["of_basis_max"] > 0 for r in rep] == [k > 0 and k % 2 == 0 for k in range(6)]


def test_of_scale_must_divide_the_frames():
    w = synth.moving_disks(40, 3, 8, 40, radii=(5.0, 8.0), seed=12)
    p = problem(w, api.MOF_FP32)
    u = torch.zeros(p.n, device="cuda")
    s = torch.empty(p.nv, device="cuda")
    with pytest.raises(api.MofError) as e:
        api.mof_solve_of(p, api.mof_default_params(of_scale=3), u, s)
    assert e.value.status == api.MOF_EINVAL


def test_mmgks_of_fp64_d1_of_matches_oracle():
    """D1-OF (AnisoTV-OF, Table 2: Theta = [Psi; L_t; Mhat]) on the 64x64x8 two-disk workload,
    6 outer iterations: the temporal rows enter the weighted Theta Gram (their own launch
    beside Solve-OF) and the fused Theta^T W Theta of the residual."""
    w = synth.plain_fp64(0)
    ores = _oracle_solve(w, 6, temporal_tv=1)
    u, s, rep = _gpu_solve(w, api.MOF_FP64, 6, temporal_tv=1)
    assert rel(u, ores.u) <= 1e-6, rel(u, ores.u)
    assert rel(s, ores.s) <= 1e-5, rel(s, ores.s)
    base, _, _ = _gpu_solve(w, api.MOF_FP64, 6)
    assert rel(u, base) > 1e-4  # the temporal rows change the result


def test_mmgks_of_fp64_round_warp_matches_oracle():
    """MMGKS-OF with the rounding-and-clipping M(s) (Sec. 3) in Mhat, in the weighted Theta
    Gram and in Theta^T W Theta, 64x64x8 two-disk workload, 5 outer iterations."""
    w = synth.plain_fp64(0)
    ores = _oracle_solve(w, 5, warp_round=1)
    p = problem(w, api.MOF_FP64)
    api.mof_set_warp(p, 1)
    prm = api.mof_default_params(noise_norm=w.noise_norm)
    b = torch.tensor(w.b, device="cuda")
    u = torch.empty(p.n, dtype=torch.float64, device="cuda")
    s = torch.empty(p.nv, dtype=torch.float64, device="cuda")
    rep = api.mof_solve(p, prm, 5, b, u, s)
    u, s = u.cpu().numpy(), s.cpu().numpy()
    assert rel(u, ores.u) <= 1e-6, rel(u, ores.u)
    assert rel(s, ores.s) <= 1e-5, rel(s, ores.s)
    for r, o in zip(rep, ores.report):
        assert r["flag"] == o["flag"] and r["basis"] == o["basis"]
    # the same problem handle back in bilinear mode (graphs captured again) gives the
    # bilinear solve, which differs from the rounding one
    api.mof_set_warp(p, 0)
    u2 = torch.empty(p.n, dtype=torch.float64, device="cuda")
    api.mof_solve(p, prm, 5, b, u2)
    base, _, _ = _gpu_solve(w, api.MOF_FP64, 5)
    np.testing.assert_array_equal(u2.cpu().numpy(), base)
    assert rel(u, base) > 1e-4


def test_mmgks_of_fp64_fan_beam_matches_oracle():
    """MMGKS-OF on fan-beam data (flat detector, Sec. 5.1: source 128 px, detector 64 px
    beyond the centre, 100 bins) of the 64x64x8 two-disk workload, 5 outer iterations."""
    w = synth.fan_form_small(0)
    g = O.Geometry(w.nx, w.ny, w.nt, w.nb, w.na, w.angles, w.h, w.db, fan=w.fan)
    ores = OS.mmgks_of(g, w.b, OS.Params(noise_norm=w.noise_norm), 5)
    p = api.mof_problem_create(w.nx, w.ny, w.nt, w.nb, w.na, w.angles, w.h, w.db, api.MOF_FP64, fan=w.fan)
    prm = api.mof_default_params(noise_norm=w.noise_norm)
    b = torch.tensor(w.b, device="cuda")
    u = torch.empty(p.n, dtype=torch.float64, device="cuda")
    s = torch.empty(p.nv, dtype=torch.float64, device="cuda")
    rep = api.mof_solve(p, prm, 5, b, u, s)
    u, s = u.cpu().numpy(), s.cpu().numpy()
    assert rel(u, ores.u) <= 1e-6, rel(u, ores.u)
    assert rel(s, ores.s) <= 1e-5, rel(s, ores.s)
    for r, o in zip(rep, ores.report):
        assert r["flag"] == o["flag"] and r["basis"] == o["basis"]
    assert rel(u, w.u_true.ravel()) < 0.5


def test_mmgks_of_fp64_pq1_solve_of_matches_oracle():
    """MMGKS-OF whose Solve-OF uses p = q = 1 (MM-GKS) on the 64x64x8 two-disk workload,
    4 outer iterations, against the oracle. The oracle's own p = q = 1 Solve-OF on these
    frames moves by 8e-6 when the frames move by 1e-15 (tests/test_oracle_solver.py pins
    > 1e-6; p = q = 2: 3e-8), and the outer iterations couple the frames and the flow, so two
    FP64 implementations that round differently agree on these velocities to about 1e-4
    while the images agree to 1e-6."""
    w = synth.plain_fp64(0)
    ores = _oracle_solve(w, 4, of_pq=1)
    u, s, rep = _gpu_solve(w, api.MOF_FP64, 4, of_pq=1)
    assert rel(u, ores.u) <= 1e-6, rel(u, ores.u)
    assert rel(s, ores.s) <= 5e-4, rel(s, ores.s)
    for r, o in zip(rep, ores.report):
        assert r["flag"] == o["flag"] and r["basis"] == o["basis"]


def test_mmgks_of_fp32_d1_of_precision_form_small():
    w = synth.precision_form_small(0)
    ores = _oracle_solve(w, 4, of_iters=10, temporal_tv=1)
    u, s, rep = _gpu_solve(w, api.MOF_FP32, 4, of_iters=10, temporal_tv=1)
    assert rel(u, ores.u) <= 1e-4, rel(u, ores.u)
    assert rel(s, ores.s) <= 1e-3, rel(s, ores.s)
