"""Backward kernels of the projector and of the flow residual (the differentiation
form): the velocity VJP against the FP64 oracle, torch.autograd.gradcheck of the
autograd functions in FP64, and FP64 central finite differences (step 1e-6) on
32 seeded random directions at the differentiation workload's size (two disks,
256x256, T = 32)."""
import numpy as np
import pytest

torch = pytest.importorskip("torch")

from oracle import ops as O
from paper_2501_12497_gb300 import api, synth
from paper_2501_12497_gb300 import autograd as AG

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _build():
    import __graft_entry__
    __graft_entry__.build()


def _problem(nx, ny, nt, prec, na=6, nb=None):
    nb = nb or int(np.ceil(np.sqrt(2) * max(nx, ny)))
    na_arr, angles = synth.shifted_angles(nt, na)
    return api.mof_problem_create(nx, ny, nt, nb, na_arr, angles, 1.0, 1.0, prec)


def _velocities(npairs, ny, nx, seed, vmax=2.5):
    """Velocities whose sample points keep 0.02 away from integers (no kink within a
    finite-difference step), some of them clipped at the grid's edges."""
    rng = np.random.default_rng(seed)
    s = rng.uniform(-vmax, vmax, size=(npairs, 2, ny, nx))
    frac = s - np.floor(s)
    s = np.where(frac < 0.02, s + 0.02, s)
    return np.where(frac > 0.98, s - 0.02, s)


def _rel(a, b):
    return np.linalg.norm(np.ravel(a) - np.ravel(b)) / max(np.linalg.norm(np.ravel(b)), 1e-300)


@pytest.mark.parametrize("prec,tol", [(api.MOF_FP64, 1e-13), (api.MOF_FP32, 1e-5)])
def test_flow_velocity_vjp_matches_oracle(prec, tol):
    nt, ny, nx = 5, 37, 45
    dt = torch.float64 if prec == api.MOF_FP64 else torch.float32
    npdt = np.float64 if prec == api.MOF_FP64 else np.float32
    p = _problem(nx, ny, nt, prec)
    u = synth.random_images(nt, ny, nx, seed=1).astype(npdt)
    s = _velocities(nt - 1, ny, nx, seed=2, vmax=4.0).astype(npdt)
    sr = _velocities(nt - 1, ny, nx, seed=3, vmax=4.0).astype(npdt)
    gr = np.random.default_rng(4).standard_normal((2, nt - 1, ny, nx)).astype(npdt)
    want_s, want_sr = O.flow_ds(u.astype(float), s.astype(float), sr.astype(float), gr.astype(float))
    T = lambda a: torch.tensor(a, dtype=dt, device="cuda").reshape(-1)
    gs, gsr = torch.empty(p.nv, dtype=dt, device="cuda"), torch.empty(p.nv, dtype=dt, device="cuda")
    api.mof_apply_flow_ds(p, T(u), T(s), T(sr), T(gr), gs, gsr)
    assert _rel(gs.cpu().numpy(), want_s) <= tol
    assert _rel(gsr.cpu().numpy(), want_sr) <= tol


def test_autograd_gradcheck_fp64():
    nt, ny, nx = 3, 9, 11
    p = _problem(nx, ny, nt, api.MOF_FP64, na=4, nb=16)
    dev = "cuda"
    u = torch.tensor(synth.random_images(nt, ny, nx, seed=5), device=dev).reshape(-1).requires_grad_()
    s = torch.tensor(_velocities(nt - 1, ny, nx, seed=6, vmax=2.0), device=dev).reshape(-1).requires_grad_()
    sr = torch.tensor(_velocities(nt - 1, ny, nx, seed=7, vmax=2.0), device=dev).reshape(-1).requires_grad_()
    assert torch.autograd.gradcheck(lambda a, b, c: AG.flow_residual(p, a, b, c), (u, s, sr), eps=1e-6, atol=1e-7,
                                    rtol=1e-5)
    assert torch.autograd.gradcheck(lambda a: AG.project(p, a), (u,), eps=1e-6, atol=1e-7, rtol=1e-5)


def test_differentiation_form_central_differences_on_32_directions():
    """At 256x256, T = 32 (two disks moving 1 px/frame, 16 angles, 256 bins): the loss
    L(u, s, s') = 0.5 ||H u - b||^2 + 0.5 ||Mhat(s, s') u||^2 through the autograd
    functions; its gradient against FP64 central differences of step 1e-6 along 32
    seeded random directions in (u, s, s') together. FP32 gradients agree with the FP64
    ones to 1e-4."""
    w = synth.differentiation_form(0)
    nt, ny, nx = w.nt, w.ny, w.nx
    p64 = api.mof_problem_create(nx, ny, nt, w.nb, w.na, w.angles, w.h, w.db, api.MOF_FP64)
    p32 = api.mof_problem_create(nx, ny, nt, w.nb, w.na, w.angles, w.h, w.db, api.MOF_FP32)
    dev = "cuda"
    b64 = torch.tensor(w.b, device=dev)
    u0 = torch.tensor(w.u_true, device=dev).reshape(-1) * 0.9
    s0 = torch.tensor(_velocities(nt - 1, ny, nx, seed=11, vmax=1.5), device=dev).reshape(-1)
    sr0 = torch.tensor(_velocities(nt - 1, ny, nx, seed=12, vmax=1.5), device=dev).reshape(-1)

    def loss(p, u, s, sr, b):
        return 0.5 * torch.sum((AG.project(p, u) - b) ** 2) + 0.5 * torch.sum(AG.flow_residual(p, u, s, sr) ** 2)

    u, s, sr = (t.clone().requires_grad_() for t in (u0, s0, sr0))
    L = loss(p64, u, s, sr, b64)
    gu, gs, gsr = torch.autograd.grad(L, (u, s, sr))
    gen = torch.Generator(device="cpu").manual_seed(13)
    h = 1e-6
    with torch.no_grad():
        for k in range(32):
            du, ds, dsr = (torch.randn(t.numel(), generator=gen, dtype=torch.float64).to(dev) for t in (u0, s0, sr0))
            # scale so each direction moves a sample point by at most ~1e-6 px
            ds /= ds.abs().max()
            dsr /= dsr.abs().max()
            fp = loss(p64, u0 + h * du, s0 + h * ds, sr0 + h * dsr, b64)
            fm = loss(p64, u0 - h * du, s0 - h * ds, sr0 - h * dsr, b64)
            fd = float((fp - fm) / (2 * h))
            an = float(torch.dot(gu, du) + torch.dot(gs, ds) + torch.dot(gsr, dsr))
            assert abs(fd - an) <= 1e-5 * max(1.0, abs(an)), (k, fd, an)
    u32, s32, sr32 = (t.float().clone().requires_grad_() for t in (u0, s0, sr0))
    L32 = loss(p32, u32, s32, sr32, b64.float())
    g32 = torch.autograd.grad(L32, (u32, s32, sr32))
    for a, bb in zip(g32, (gu, gs, gsr)):
        assert _rel(a.double().cpu().numpy(), bb.cpu().numpy()) <= 1e-4


def test_motion_step_by_gradient_descent_reduces_the_flow_residual():
    """A motion step driven by the backward kernels: gradient descent on
    0.5 ||Mbar(s) u||^2 from s = 0 for two disks translating 1 px per frame lowers
    the residual."""
    w = synth.moving_disks(64, 4, 8, 64, radii=(8.0, 12.0), seed=3)
    p = api.mof_problem_create(w.nx, w.ny, w.nt, w.nb, w.na, w.angles, w.h, w.db, api.MOF_FP64)
    u = torch.tensor(w.u_true, device="cuda").reshape(-1)
    s = torch.zeros(p.nv, dtype=torch.float64, device="cuda", requires_grad=True)
    sr = torch.zeros(p.nv, dtype=torch.float64, device="cuda")
    opt = torch.optim.SGD([s], lr=0.05)
    first = None
    for it in range(40):
        opt.zero_grad()
        r = AG.flow_residual(p, u, s, sr)
        loss = 0.5 * torch.sum(r[: r.numel() // 2] ** 2)
        if first is None:
            first = float(loss.detach())
        loss.backward()
        opt.step()
    assert float(loss.detach()) < 0.7 * first
