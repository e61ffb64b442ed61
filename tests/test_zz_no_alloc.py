"""The allocation-free Mhat^T entry point (mof_apply_flowT_noalloc) against
mof_apply_flowT: bit-identical results on two calls in a row with different
inputs, both precisions, and the size limit rejected on the host.

Kept in its own file, named to be collected last, so that it runs both alone
and after every other test in the same process."""
import ctypes

import numpy as np
import pytest

torch = pytest.importorskip("torch")

from paper_2501_12497_gb300 import api, synth

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _build():
    import __graft_entry__
    __graft_entry__.build()


def _problem(nx, ny, nt, prec):
    na, angles = synth.shifted_angles(nt, 3)
    return api.mof_problem_create(nx, ny, nt, 11, na, angles, 1.0, 1.0, prec)


@pytest.mark.parametrize("prec", [api.MOF_FP32, api.MOF_FP64])
def test_noalloc_flowT_matches_allocating_entry_on_two_calls(prec):
    nx, ny, nt = 70, 45, 5
    p = _problem(nx, ny, nt, prec)
    dt = torch.float64 if prec == api.MOF_FP64 else torch.float32
    for call, (seed, vmax) in enumerate([(0, 5.5), (1, 1.5)]):
        r = torch.tensor(synth.random_images(2 * (nt - 1), ny, nx, seed=seed), dtype=dt, device="cuda").reshape(-1)
        s = torch.tensor(synth.random_velocities(nt - 1, ny, nx, vmax=vmax, seed=seed + 10), dtype=dt,
                         device="cuda").reshape(-1)
        sr = torch.empty_like(s)
        api.mof_reverse_flow(p, s, sr)
        want = torch.empty(p.n, dtype=dt, device="cuda")
        got = torch.full((p.n,), float("nan"), dtype=dt, device="cuda")
        api.mof_apply_flowT(p, r, s, sr, want)
        api.mof_apply_flowT_noalloc(p, r, s, sr, got)
        torch.cuda.synchronize()
        assert torch.equal(got, want), "call %d differs" % call


def _compare_once(p, seed, vmax, dt):
    nx, ny, nt = p.nx, p.ny, p.nt
    r = torch.tensor(synth.random_images(2 * (nt - 1), ny, nx, seed=seed), dtype=dt, device="cuda").reshape(-1)
    s = torch.tensor(synth.random_velocities(nt - 1, ny, nx, vmax=vmax, seed=seed + 10), dtype=dt,
                     device="cuda").reshape(-1)
    sr = torch.empty_like(s)
    api.mof_reverse_flow(p, s, sr)
    want = torch.empty(p.n, dtype=dt, device="cuda")
    got = torch.full((p.n,), float("nan"), dtype=dt, device="cuda")
    api.mof_apply_flowT(p, r, s, sr, want)
    api.mof_apply_flowT_noalloc(p, r, s, sr, got)
    torch.cuda.synchronize()
    return torch.equal(got, want)


def test_noalloc_flowT_after_a_larger_problem_used_the_array():
    """A larger problem (another tile layout, large displacements) fills more of the shared
    array first; the smaller problem's call that follows must still equal the allocating
    entry point bit for bit."""
    big = _problem(160, 96, 6, api.MOF_FP32)
    small = _problem(70, 45, 5, api.MOF_FP32)
    assert _compare_once(big, 3, 9.0, torch.float32)
    assert _compare_once(small, 4, 0.7, torch.float32)
    assert _compare_once(small, 5, 2.5, torch.float32)


def test_noalloc_flowT_rejects_problems_beyond_its_fixed_scratch():
    # 4096 x 4096 frames, 40 of them: 64 x 256 tiles of 64 x 16 pixels,
    # 8 * 39 * (16384 + 1) ints of bounds > 2^22
    p = _problem(4096, 4096, 40, api.MOF_FP32)
    dummy = torch.zeros(16, dtype=torch.float32, device="cuda")
    ptr = ctypes.c_void_p(dummy.data_ptr())
    lib = api.load()
    st = lib.mof_apply_flowT_noalloc(p.handle, ptr, ptr, ptr, ptr, None)
    assert st == api.MOF_EUNSUPPORTED
    assert b"tile bounds" in lib.mof_last_error()
    torch.cuda.synchronize()
