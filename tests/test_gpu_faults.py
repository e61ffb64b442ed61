"""Failure detection without a GPU fault: each failure is made on the host side of the
boundary or by a bounded device wait that is told to give up, and the library reports
it as a status code while the CUDA context stays usable.

- non-finite data: a NaN in the sinogram is found by the solver's data norm and
  returned as MOF_ENUMERIC at the solve's synchronising end (device and host entries);
- allocation failure: a problem whose workspace exceeds the device memory (a 4096x4096x63
  sequence with a 60-vector image basis and 64-vector Solve-OF bases, about 0.5 TB) makes
  the workspace allocation fail, returned as MOF_ENOMEM before any kernel runs;
- bounded waits: with the wait bound set to zero polls, every CTA of the fused
  reorthogonalisation pass gives up on its tile barrier at once, records the timeout,
  waits with the default bound for its own copies to land and returns; the solve returns
  MOF_ETIMEOUT, and with the default bound restored the same solve gives the result it
  gave before, bit for bit.
"""
import numpy as np
import pytest

torch = pytest.importorskip("torch")

from paper_2501_12497_gb300 import api, synth

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _build():
    import __graft_entry__
    __graft_entry__.build()


def _problem(w, prec=api.MOF_FP32):
    return api.mof_problem_create(w.nx, w.ny, w.nt, w.nb, w.na, w.angles, w.h, w.db, prec)


def test_nonfinite_data_returns_enumeric():
    w = synth.moving_disks(32, 3, 8, 32, radii=(5.0, 8.0), seed=21)
    p = _problem(w)
    prm = api.mof_default_params(noise_norm=w.noise_norm, ell=4, of_ell=3, of_iters=3)
    b = w.b.astype(np.float32)
    b[17] = np.nan
    u = torch.empty(p.n, dtype=torch.float32, device="cuda")
    with pytest.raises(api.MofError) as e:
        api.mof_solve(p, prm, 2, torch.tensor(b, device="cuda"), u)
    assert e.value.status == api.MOF_ENUMERIC and "non-finite" in str(e.value)
    uh = np.empty(p.n, dtype=np.float32)
    with pytest.raises(api.MofError) as e:
        api.mof_solve_host(p, prm, 2, b, uh)
    assert e.value.status == api.MOF_ENUMERIC
    # the problem and the context still work
    api.mof_solve(p, prm, 2, torch.tensor(w.b.astype(np.float32), device="cuda"), u)
    assert torch.isfinite(u).all()


def test_workspace_beyond_device_memory_returns_enomem():
    nx = ny = 4096
    nt = 63
    na, angles = synth.shifted_angles(nt, 1)
    p = api.mof_problem_create(nx, ny, nt, 8, na, angles, precision=api.MOF_FP32)
    total = torch.cuda.get_device_properties(0).total_memory
    need = 4 * p.n * (60 + 2 * 64)  # the image basis plus the Solve-OF bases alone
    assert need > 1.5 * total
    b = torch.ones(p.m, dtype=torch.float32, device="cuda")
    u = torch.empty(p.n, dtype=torch.float32, device="cuda")  # a full-size output all the same
    prm = api.mof_default_params(noise_norm=1.0, ell=10, of_ell=10, of_iters=54)
    with pytest.raises(api.MofError) as e:
        api.mof_solve(p, prm, 50, b, u)
    assert e.value.status == api.MOF_ENOMEM
    del b, u
    p.close()
    torch.cuda.synchronize()
    # a small solve in the same context afterwards
    w = synth.moving_disks(32, 3, 8, 32, radii=(5.0, 8.0), seed=22)
    q = _problem(w)
    uu = torch.empty(q.n, dtype=torch.float32, device="cuda")
    api.mof_solve(q, api.mof_default_params(noise_norm=w.noise_norm, ell=4, of_ell=3, of_iters=3), 2,
                  torch.tensor(w.b.astype(np.float32), device="cuda"), uu)
    assert torch.isfinite(uu).all()


def test_a_wait_that_gives_up_returns_etimeout():
    w = synth.moving_disks(64, 4, 8, 64, radii=(8.0, 12.0), seed=23)
    p = _problem(w)
    prm = api.mof_default_params(of_ell=6, of_iters=6)
    u = torch.tensor(w.u_true.astype(np.float32), device="cuda").reshape(-1)
    s0 = torch.empty(p.nv, dtype=torch.float32, device="cuda")
    api.mof_solve_of(p, prm, u, s0)
    s1 = torch.empty_like(s0)
    try:
        api.mof_debug_set_wait_limit(0)
        with pytest.raises(api.MofError) as e:
            api.mof_solve_of(p, prm, u, s1)
        assert e.value.status == api.MOF_ETIMEOUT
    finally:
        api.mof_debug_set_wait_limit(-1)
    s2 = torch.empty_like(s0)
    api.mof_solve_of(p, prm, u, s2)
    assert torch.equal(s2, s0)
