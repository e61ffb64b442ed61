"""Batched solves of independent problems of uneven size (mof_solve_batch) and the
of_streams autotuner: every problem's result in a batch equals its own mof_solve
bit for bit, argument errors are caught before anything runs, and tuning changes
speed only."""
import numpy as np
import pytest

torch = pytest.importorskip("torch")

from paper_2501_12497_gb300 import api, synth

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _build():
    import __graft_entry__
    __graft_entry__.build()


def _setup(ws, precs):
    probs, params, bs = [], [], []
    for w, prec in zip(ws, precs):
        dt = torch.float64 if prec == api.MOF_FP64 else torch.float32
        p = api.mof_problem_create(w.nx, w.ny, w.nt, w.nb, w.na, w.angles, w.h, w.db, prec)
        probs.append(p)
        params.append(api.mof_default_params(noise_norm=w.noise_norm, ell=5, of_ell=4, of_iters=5))
        bs.append(torch.tensor(w.b, dtype=dt, device="cuda"))
    return probs, params, bs


def _uneven(seed):
    return synth.batch_form(count=5, seed=seed, sizes=(32, 40, 48), nt_range=(3, 6), na_range=(6, 12))


def test_batch_equals_individual_solves():
    ws = _uneven(0)
    precs = [api.MOF_FP32, api.MOF_FP64, api.MOF_FP32, api.MOF_FP32, api.MOF_FP64]
    probs, params, bs = _setup(ws, precs)
    n_outer = 4
    us = [torch.empty(p.n, dtype=b.dtype, device="cuda") for p, b in zip(probs, bs)]
    ss = [torch.empty(p.nv, dtype=b.dtype, device="cuda") for p, b in zip(probs, bs)]
    reps = api.mof_solve_batch(probs, params, n_outer, bs, us, ss)
    for p, prm, b, u, s, rep in zip(probs, params, bs, us, ss, reps):
        u1, s1 = torch.empty_like(u), torch.empty_like(s)
        rep1 = api.mof_solve(p, prm, n_outer, b, u1, s1)
        assert torch.equal(u, u1) and torch.equal(s, s1)
        assert [r["basis"] for r in rep] == [r["basis"] for r in rep1]
        assert [r["lambda"] for r in rep] == [r["lambda"] for r in rep1]


def test_batch_mixes_geometries_warps_and_solver_variants():
    """One batch holding a fan-beam problem, a rounding-warp problem, a p = q = 1 Solve-OF,
    a D1-OF problem and a rescaled Solve-OF: each result is its own mof_solve's, bit for bit."""
    ws = [synth.fan_form_small(0), synth.moving_disks(40, 4, 8, 40, radii=(5.0, 8.0), seed=11),
          synth.moving_disks(48, 4, 8, 48, radii=(6.0, 9.0), seed=12),
          synth.moving_disks(40, 5, 8, 40, radii=(5.0, 8.0), seed=13),
          synth.moving_disks(64, 4, 8, 64, radii=(8.0, 12.0), seed=14)]
    extra = [{}, {}, {"of_pq": 1}, {"temporal_tv": 1}, {"of_scale": 2, "tau": 2}]
    probs, params, bs = [], [], []
    for i, (w, ex) in enumerate(zip(ws, extra)):
        p = api.mof_problem_create(w.nx, w.ny, w.nt, w.nb, w.na, w.angles, w.h, w.db, api.MOF_FP32, fan=w.fan)
        if i == 1:
            api.mof_set_warp(p, 1)
        probs.append(p)
        params.append(api.mof_default_params(noise_norm=w.noise_norm, ell=5, of_ell=4, of_iters=5, **ex))
        bs.append(torch.tensor(w.b, dtype=torch.float32, device="cuda"))
    n_outer = 4
    us = [torch.empty(p.n, dtype=torch.float32, device="cuda") for p in probs]
    ss = [torch.empty(p.nv, dtype=torch.float32, device="cuda") for p in probs]
    reps = api.mof_solve_batch(probs, params, n_outer, bs, us, ss)
    for p, prm, b, u, s, rep in zip(probs, params, bs, us, ss, reps):
        u1, s1 = torch.empty_like(u), torch.empty_like(s)
        rep1 = api.mof_solve(p, prm, n_outer, b, u1, s1)
        assert torch.equal(u, u1) and torch.equal(s, s1)
        assert [r["basis"] for r in rep] == [r["basis"] for r in rep1]


def test_batch_rejects_bad_arguments_before_running():
    ws = _uneven(1)[:2]
    probs, params, bs = _setup(ws, [api.MOF_FP32, api.MOF_FP32])
    us = [torch.empty(p.n, dtype=torch.float32, device="cuda") for p in probs]
    with pytest.raises(api.MofError) as e:
        api.mof_solve_batch([probs[0], probs[0]], [params[0], params[0]], 2, [bs[0], bs[0]], [us[0], us[0]])
    assert e.value.status == api.MOF_EINVAL
    bad = api.mof_default_params(noise_norm=-1.0)  # DP without a noise level
    with pytest.raises(api.MofError) as e:
        api.mof_solve_batch(probs, [params[0], bad], 2, bs, us)
    assert e.value.status == api.MOF_EINVAL


def test_autotune_picks_a_candidate_and_leaves_results_unchanged():
    ws = _uneven(2)[:3]
    probs, params, bs = _setup(ws, [api.MOF_FP32] * 3)
    us = [torch.empty(p.n, dtype=torch.float32, device="cuda") for p in probs]
    g, ms = api.mof_autotune(probs, params, 2, bs, us)
    assert g in (1, 2, 4, 8, 16, 32, 64) and ms > 0 and all(prm.of_streams == g for prm in params)
    n_outer = 3
    out_t = [torch.empty_like(u) for u in us]
    api.mof_solve_batch(probs, params, n_outer, bs, out_t)
    ref = [api.mof_default_params(noise_norm=w.noise_norm, ell=5, of_ell=4, of_iters=5, of_streams=1) for w in ws]
    out_1 = [torch.empty_like(u) for u in us]
    api.mof_solve_batch(probs, ref, n_outer, bs, out_1)
    for a, b in zip(out_t, out_1):
        assert torch.equal(a, b)


def test_batch_form_reconstructs_every_problem():
    """A reduced instance of the uneven batch (8 problems, n in {64, 96, 128},
    T in [4, 10], 10-45 angles): every reconstruction is far closer to its phantom
    than the zero image, and wherever DP found a root the misfit is eta delta (to
    5e-4: the misfit H V z - b of a 1 % noise level is evaluated in FP32 on these
    small sinograms)."""
    ws = synth.batch_form(count=8, seed=3, sizes=(64, 96, 128), nt_range=(4, 10))
    probs, params, bs = _setup(ws, [api.MOF_FP32] * len(ws))
    params = [api.mof_default_params(noise_norm=w.noise_norm) for w in ws]
    n_outer = 8
    us = [torch.empty(p.n, dtype=torch.float32, device="cuda") for p in probs]
    reps = api.mof_solve_batch(probs, params, n_outer, bs, us)
    for w, u, rep, prm in zip(ws, us, reps, params):
        err = np.linalg.norm(u.cpu().double().numpy() - w.u_true.ravel()) / np.linalg.norm(w.u_true)
        assert err < 0.5, (w.name, err)
        for k, r in enumerate(rep):
            assert r["basis"] == prm.ell + k
            if r["flag"] == 0:
                assert abs(r["resid"] / (prm.eta * w.noise_norm) - 1) < 5e-4, (w.name, k, r)


@pytest.mark.parametrize("prec", [api.MOF_FP32, api.MOF_FP64])
def test_plain_per_frame_form_equals_the_batched_form(prec):
    """plain = 1 launches every kernel from the host (no graphs), runs Solve-OF one frame
    pair after another on one stream and the projector and its adjoint one frame per
    launch: the same kernels on the same data, so the result is the batched form's bit for
    bit (images, velocities, reports)."""
    w = synth.moving_disks(48, 5, 8, 48, radii=(6.0, 9.0), seed=31)
    dt = torch.float64 if prec == api.MOF_FP64 else torch.float32
    p = api.mof_problem_create(w.nx, w.ny, w.nt, w.nb, w.na, w.angles, w.h, w.db, prec)
    b = torch.tensor(w.b, dtype=dt, device="cuda")
    out = []
    for plain in (0, 1):
        prm = api.mof_default_params(noise_norm=w.noise_norm, ell=5, of_ell=4, of_iters=5, plain=plain)
        u = torch.empty(p.n, dtype=dt, device="cuda")
        s = torch.empty(p.nv, dtype=dt, device="cuda")
        rep = api.mof_solve(p, prm, 4, b, u, s)
        out.append((u, s, rep))
    assert torch.equal(out[0][0], out[1][0]) and torch.equal(out[0][1], out[1][1])
    assert [r["lambda"] for r in out[0][2]] == [r["lambda"] for r in out[1][2]]
    u = torch.tensor(w.u_true, dtype=dt, device="cuda").reshape(-1)
    s0, s1 = torch.empty(p.nv, dtype=dt, device="cuda"), torch.empty(p.nv, dtype=dt, device="cuda")
    api.mof_solve_of(p, api.mof_default_params(of_ell=4, of_iters=5), u, s0)
    api.mof_solve_of(p, api.mof_default_params(of_ell=4, of_iters=5, plain=1), u, s1)
    assert torch.equal(s0, s1)
