"""Thin ctypes binding of libmof (include/mof.h), same entry-point names.

Argument marshalling only: every array is handed to the CUDA library as a raw
pointer and every numerical step runs in its kernels. Device arrays are torch
CUDA tensors (contiguous, float32 for an FP32 problem, float64 for FP64);
`mof_solve_host` takes host numpy arrays. There is no CPU fallback: if
libmof.so is missing or fails to load, every call raises.
"""
import ctypes
import os

import numpy as np

from . import build as _build

MOF_OK, MOF_EINVAL, MOF_ENOMEM, MOF_ECUDA, MOF_ENUMERIC, MOF_ETIMEOUT, MOF_EUNSUPPORTED = range(7)
MOF_FP32, MOF_FP64 = 0, 1
MOF_RULE_DP, MOF_RULE_GCV, MOF_RULE_FIXED = 0, 1, 2
STATUS_NAMES = {0: "MOF_OK", 1: "MOF_EINVAL", 2: "MOF_ENOMEM", 3: "MOF_ECUDA", 4: "MOF_ENUMERIC",
                5: "MOF_ETIMEOUT", 6: "MOF_EUNSUPPORTED"}


class MofError(RuntimeError):
    def __init__(self, status, text):
        super().__init__("%s: %s" % (STATUS_NAMES.get(status, status), text))
        self.status = status


class mof_geometry(ctypes.Structure):
    _fields_ = [("nx", ctypes.c_int), ("ny", ctypes.c_int), ("nt", ctypes.c_int), ("nb", ctypes.c_int),
                ("na", ctypes.POINTER(ctypes.c_int)), ("angles", ctypes.POINTER(ctypes.c_double)),
                ("pixel_size", ctypes.c_double), ("bin_size", ctypes.c_double)]


class mof_solver_params(ctypes.Structure):
    _fields_ = [("ell", ctypes.c_int), ("tau", ctypes.c_int), ("of_iters", ctypes.c_int),
                ("of_ell", ctypes.c_int), ("of_dr", ctypes.c_int), ("image_rule", ctypes.c_int),
                ("eps", ctypes.c_double), ("eta", ctypes.c_double), ("noise_norm", ctypes.c_double),
                ("lam_fixed", ctypes.c_double), ("breakdown_tol", ctypes.c_double), ("of_streams", ctypes.c_int),
                ("of_scale", ctypes.c_int), ("temporal_tv", ctypes.c_int), ("of_pq", ctypes.c_int),
                ("plain", ctypes.c_int)]


class mof_report(ctypes.Structure):
    _fields_ = [("lambda_", ctypes.c_double), ("resid", ctypes.c_double), ("rnorm", ctypes.c_double),
                ("basis", ctypes.c_int), ("flag", ctypes.c_int), ("of_basis_min", ctypes.c_int),
                ("of_basis_max", ctypes.c_int)]


_lib = None
LIB_PATH = _build.LIB_PATH

_SIGS = {
    "mof_default_params": (None, [ctypes.c_void_p]),
    "mof_problem_create": (ctypes.c_int, [ctypes.POINTER(mof_geometry), ctypes.c_int, ctypes.c_void_p]),
    "mof_problem_create_fan": (ctypes.c_int, [ctypes.POINTER(mof_geometry), ctypes.c_double, ctypes.c_double,
                                              ctypes.c_int, ctypes.c_void_p]),
    "mof_problem_destroy": (None, [ctypes.c_void_p]),
    "mof_problem_sizes": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p]),
    "mof_apply_A": (ctypes.c_int, [ctypes.c_void_p] * 4),
    "mof_apply_AT": (ctypes.c_int, [ctypes.c_void_p] * 4),
    "mof_apply_grad": (ctypes.c_int, [ctypes.c_void_p] * 4),
    "mof_apply_gradT": (ctypes.c_int, [ctypes.c_void_p] * 4),
    "mof_apply_flow": (ctypes.c_int, [ctypes.c_void_p] * 6),
    "mof_apply_flowT": (ctypes.c_int, [ctypes.c_void_p] * 6),
    "mof_apply_flowT_noalloc": (ctypes.c_int, [ctypes.c_void_p] * 6),
    "mof_apply_flow_ds": (ctypes.c_int, [ctypes.c_void_p] * 8),
    "mof_of_fields": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_void_p, ctypes.c_int] + [ctypes.c_void_p] * 4),
    "mof_downsample": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_int] + [ctypes.c_void_p] * 3),
    "mof_upsample_velocity": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_int] + [ctypes.c_void_p] * 3),
    "mof_apply_flow_lin": (ctypes.c_int, [ctypes.c_void_p] * 7),
    "mof_apply_flow_linT": (ctypes.c_int, [ctypes.c_void_p] * 6),
    "mof_apply_vgrad": (ctypes.c_int, [ctypes.c_void_p] * 4),
    "mof_apply_vgradT": (ctypes.c_int, [ctypes.c_void_p] * 4),
    "mof_reverse_flow": (ctypes.c_int, [ctypes.c_void_p] * 4),
    "mof_apply_reg_normal": (ctypes.c_int, [ctypes.c_void_p] * 5 + [ctypes.c_double] + [ctypes.c_void_p] * 2),
    "mof_solve_of": (ctypes.c_int, [ctypes.c_void_p] * 5),
    "mof_solve": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_void_p, ctypes.c_int] + [ctypes.c_void_p] * 6),
    "mof_solve_host": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_void_p, ctypes.c_int] + [ctypes.c_void_p] * 6),
    "mof_solve_batch": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_int, ctypes.c_void_p, ctypes.c_int] + [ctypes.c_void_p] * 5),
    "mof_autotune": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_int, ctypes.c_void_p, ctypes.c_int] + [ctypes.c_void_p] * 4),
    "mof_set_timing": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_int]),
    "mof_set_warp": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_int]),
    "mof_get_timing": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_int, ctypes.c_void_p, ctypes.c_void_p,
                                      ctypes.c_void_p, ctypes.c_void_p]),
    "mof_debug_set_wait_limit": (ctypes.c_int, [ctypes.c_longlong]),
    "mof_measure_fp32_peaks": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_void_p]),
    "mof_last_error": (ctypes.c_char_p, []),
    "mof_kernel_launches": (ctypes.c_longlong, []),
}


def load(path=None):
    """Load libmof.so (built by build.build()); raises if it is missing."""
    global _lib
    if _lib is not None:
        return _lib
    path = path or LIB_PATH
    if not os.path.exists(path):
        raise RuntimeError("libmof.so is not built (%s); run __graft_entry__.build()" % path)
    lib = ctypes.CDLL(path)
    for name, (res, args) in _SIGS.items():
        f = getattr(lib, name)
        f.restype = res
        f.argtypes = args
    _lib = lib
    return lib


def _check(st):
    if st != MOF_OK:
        raise MofError(st, _lib.mof_last_error().decode())


def _stream(stream):
    if stream is None:
        import torch
        return ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)
    if isinstance(stream, int):
        return ctypes.c_void_p(stream)
    return ctypes.c_void_p(stream.cuda_stream)


class Problem:
    """Owns one mof_problem*. Geometry arrays are copied at creation."""

    def __init__(self, handle, nx, ny, nt, nb, precision):
        self.handle = ctypes.c_void_p(handle)
        self.nx, self.ny, self.nt, self.nb, self.precision = nx, ny, nt, nb, precision
        n, m, nv = ctypes.c_longlong(), ctypes.c_longlong(), ctypes.c_longlong()
        _check(_lib.mof_problem_sizes(self.handle, ctypes.byref(n), ctypes.byref(m), ctypes.byref(nv)))
        self.n, self.m, self.nv = n.value, m.value, nv.value

    @property
    def dtype(self):
        import torch
        return torch.float64 if self.precision == MOF_FP64 else torch.float32

    def close(self):
        if self.handle and self.handle.value:
            _lib.mof_problem_destroy(self.handle)
            self.handle = ctypes.c_void_p(0)

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def mof_default_params(**over):
    load()
    p = mof_solver_params()
    _lib.mof_default_params(ctypes.byref(p))
    for k, v in over.items():
        setattr(p, k, v)
    return p


def mof_problem_create(nx, ny, nt, nb, na, angles, pixel_size=1.0, bin_size=1.0, precision=MOF_FP32, fan=None):
    """A parallel-beam problem, or with fan = (source_distance, detector_distance) a
    fan-beam problem (mof_problem_create_fan)."""
    load()
    na_arr = np.ascontiguousarray(na, dtype=np.int32)
    ang = np.ascontiguousarray(angles, dtype=np.float64)
    g = mof_geometry(nx, ny, nt, nb, na_arr.ctypes.data_as(ctypes.POINTER(ctypes.c_int)),
                     ang.ctypes.data_as(ctypes.POINTER(ctypes.c_double)), pixel_size, bin_size)
    h = ctypes.c_void_p()
    if fan is not None:
        _check(_lib.mof_problem_create_fan(ctypes.byref(g), float(fan[0]), float(fan[1]), precision, ctypes.byref(h)))
        return Problem(h.value, nx, ny, nt, nb, precision)
    _check(_lib.mof_problem_create(ctypes.byref(g), precision, ctypes.byref(h)))
    return Problem(h.value, nx, ny, nt, nb, precision)


def mof_problem_destroy(problem):
    problem.close()


def _ptr(problem, t, numel, name, allow_none=False):
    if t is None:
        if allow_none:
            return None
        raise ValueError("%s is required" % name)
    if not t.is_cuda:
        raise ValueError("%s must be a CUDA tensor" % name)
    if t.dtype != problem.dtype:
        raise ValueError("%s must be %s (got %s)" % (name, problem.dtype, t.dtype))
    if not t.is_contiguous():
        raise ValueError("%s must be contiguous" % name)
    if t.numel() != numel:
        raise ValueError("%s has %d elements, expected %d" % (name, t.numel(), numel))
    return ctypes.c_void_p(t.data_ptr())


def _sizes(p):
    ns = p.nx * p.ny
    return {"n": p.n, "m": p.m, "nv": p.nv, "pairs": (p.nt - 1) * ns, "flow": 2 * (p.nt - 1) * ns,
            "grad": 2 * p.n, "vgrad": 2 * p.nv}


def mof_apply_A(p, u, b, stream=None):
    s = _sizes(p)
    _check(_lib.mof_apply_A(p.handle, _ptr(p, u, s["n"], "u"), _ptr(p, b, s["m"], "b"), _stream(stream)))


def mof_apply_AT(p, b, u, stream=None):
    s = _sizes(p)
    _check(_lib.mof_apply_AT(p.handle, _ptr(p, b, s["m"], "b"), _ptr(p, u, s["n"], "u"), _stream(stream)))


def mof_apply_grad(p, u, g, stream=None):
    s = _sizes(p)
    _check(_lib.mof_apply_grad(p.handle, _ptr(p, u, s["n"], "u"), _ptr(p, g, s["grad"], "g"), _stream(stream)))


def mof_apply_gradT(p, g, u, stream=None):
    s = _sizes(p)
    _check(_lib.mof_apply_gradT(p.handle, _ptr(p, g, s["grad"], "g"), _ptr(p, u, s["n"], "u"), _stream(stream)))


def mof_apply_flow(p, u, sv, sr, r, stream=None):
    s = _sizes(p)
    _check(_lib.mof_apply_flow(p.handle, _ptr(p, u, s["n"], "u"), _ptr(p, sv, s["nv"], "s"),
                               _ptr(p, sr, s["nv"], "sr"), _ptr(p, r, s["flow"], "r"), _stream(stream)))


def mof_apply_flowT(p, r, sv, sr, u, stream=None):
    s = _sizes(p)
    _check(_lib.mof_apply_flowT(p.handle, _ptr(p, r, s["flow"], "r"), _ptr(p, sv, s["nv"], "s"),
                                _ptr(p, sr, s["nv"], "sr"), _ptr(p, u, s["n"], "u"), _stream(stream)))


def mof_apply_flowT_noalloc(p, r, sv, sr, u, stream=None):
    s = _sizes(p)
    _check(_lib.mof_apply_flowT_noalloc(p.handle, _ptr(p, r, s["flow"], "r"), _ptr(p, sv, s["nv"], "s"),
                                        _ptr(p, sr, s["nv"], "sr"), _ptr(p, u, s["n"], "u"), _stream(stream)))


def mof_apply_flow_ds(p, u, sv, sr, gr, gs, gsr, stream=None):
    s = _sizes(p)
    _check(_lib.mof_apply_flow_ds(p.handle, _ptr(p, u, s["n"], "u"), _ptr(p, sv, s["nv"], "s"), _ptr(p, sr, s["nv"], "sr"),
                                  _ptr(p, gr, s["flow"], "gr"), _ptr(p, gs, s["nv"], "gs"), _ptr(p, gsr, s["nv"], "gsr"),
                                  _stream(stream)))


def mof_of_fields(p, u, dr, ux, uy, ut, stream=None):
    s = _sizes(p)
    _check(_lib.mof_of_fields(p.handle, _ptr(p, u, s["n"], "u"), int(dr), _ptr(p, ux, s["pairs"], "ux"),
                              _ptr(p, uy, s["pairs"], "uy"), _ptr(p, ut, s["pairs"], "ut"), _stream(stream)))


def mof_downsample(p, a, u, uc, stream=None):
    """uc = a x a block means of the frames of u (uc has nt * (ny/a) * (nx/a) values)."""
    s = _sizes(p)
    a = int(a)
    nc = p.nt * (p.ny // a) * (p.nx // a) if a >= 1 else 0
    _check(_lib.mof_downsample(p.handle, a, _ptr(p, u, s["n"], "u"), _ptr(p, uc, nc, "uc"), _stream(stream)))


def mof_upsample_velocity(p, a, sc, sv, stream=None):
    """sv = a * bilinear interpolation of the coarse velocities sc at the fine pixel centres."""
    s = _sizes(p)
    a = int(a)
    nc = (p.nt - 1) * 2 * (p.ny // a) * (p.nx // a) if a >= 1 else 0
    _check(_lib.mof_upsample_velocity(p.handle, a, _ptr(p, sc, nc, "sc"), _ptr(p, sv, s["nv"], "s"), _stream(stream)))


def mof_apply_flow_lin(p, ux, uy, ut, sv, r, stream=None):
    s = _sizes(p)
    _check(_lib.mof_apply_flow_lin(p.handle, _ptr(p, ux, s["pairs"], "ux"), _ptr(p, uy, s["pairs"], "uy"),
                                   _ptr(p, ut, s["pairs"], "ut"), _ptr(p, sv, s["nv"], "s"),
                                   _ptr(p, r, s["pairs"], "r"), _stream(stream)))


def mof_apply_flow_linT(p, ux, uy, r, gs, stream=None):
    s = _sizes(p)
    _check(_lib.mof_apply_flow_linT(p.handle, _ptr(p, ux, s["pairs"], "ux"), _ptr(p, uy, s["pairs"], "uy"),
                                    _ptr(p, r, s["pairs"], "r"), _ptr(p, gs, s["nv"], "gs"), _stream(stream)))


def mof_apply_vgrad(p, sv, gs, stream=None):
    s = _sizes(p)
    _check(_lib.mof_apply_vgrad(p.handle, _ptr(p, sv, s["nv"], "s"), _ptr(p, gs, s["vgrad"], "gs"), _stream(stream)))


def mof_apply_vgradT(p, gs, sv, stream=None):
    s = _sizes(p)
    _check(_lib.mof_apply_vgradT(p.handle, _ptr(p, gs, s["vgrad"], "gs"), _ptr(p, sv, s["nv"], "s"), _stream(stream)))


def mof_reverse_flow(p, sv, sr, stream=None):
    s = _sizes(p)
    _check(_lib.mof_reverse_flow(p.handle, _ptr(p, sv, s["nv"], "s"), _ptr(p, sr, s["nv"], "sr"), _stream(stream)))


def mof_apply_reg_normal(p, x, uk, sv, sr, eps, y, stream=None):
    s = _sizes(p)
    _check(_lib.mof_apply_reg_normal(p.handle, _ptr(p, x, s["n"], "x"), _ptr(p, uk, s["n"], "uk"),
                                     _ptr(p, sv, s["nv"], "s"), _ptr(p, sr, s["nv"], "sr"), float(eps),
                                     _ptr(p, y, s["n"], "y"), _stream(stream)))


def mof_solve_of(p, params, u, sv, stream=None):
    s = _sizes(p)
    _check(_lib.mof_solve_of(p.handle, ctypes.byref(params), _ptr(p, u, s["n"], "u"), _ptr(p, sv, s["nv"], "s"),
                             _stream(stream)))


def _reports(rep):
    return [{"lambda": r.lambda_, "resid": r.resid, "rnorm": r.rnorm, "basis": r.basis, "flag": r.flag,
             "of_basis_min": r.of_basis_min, "of_basis_max": r.of_basis_max} for r in rep]


def mof_solve(p, params, n_outer, b, u_out, s_out=None, sr_out=None, stream=None):
    """MMGKS-OF (Alg. 1) on device arrays; returns the per-iteration report."""
    s = _sizes(p)
    rep = (mof_report * n_outer)()
    _check(_lib.mof_solve(p.handle, ctypes.byref(params), int(n_outer), _ptr(p, b, s["m"], "b"),
                          _ptr(p, u_out, s["n"], "u_out"), _ptr(p, s_out, s["nv"], "s_out", True),
                          _ptr(p, sr_out, s["nv"], "sr_out", True), rep, _stream(stream)))
    return _reports(rep)


def _host_ptr(p, a, numel, name, allow_none=False):
    if a is None:
        if allow_none:
            return None
        raise ValueError("%s is required" % name)
    want = np.float64 if p.precision == MOF_FP64 else np.float32
    if not isinstance(a, np.ndarray) or a.dtype != want or not a.flags.c_contiguous or a.size != numel:
        raise ValueError("%s must be a contiguous %s numpy array of %d elements" % (name, want.__name__, numel))
    return ctypes.c_void_p(a.ctypes.data)


def mof_solve_host(p, params, n_outer, b_host, u_host, s_host=None, sr_host=None, stream=None):
    """MMGKS-OF with host (numpy) input and outputs; copies in and out inside the call."""
    s = _sizes(p)
    rep = (mof_report * n_outer)()
    _check(_lib.mof_solve_host(p.handle, ctypes.byref(params), int(n_outer), _host_ptr(p, b_host, s["m"], "b"),
                               _host_ptr(p, u_host, s["n"], "u"), _host_ptr(p, s_host, s["nv"], "s", True),
                               _host_ptr(p, sr_host, s["nv"], "sr", True), rep, _stream(stream)))
    return _reports(rep)


def _ptr_array(items):
    arr = (ctypes.c_void_p * len(items))()
    for i, v in enumerate(items):
        arr[i] = v
    return arr


def mof_solve_batch(problems, params, n_outer, bs, us, ss=None, stream=None):
    """Batched solve: lists of problems, params (one each), device b and u (and
    optionally s) tensors. Returns one report list per problem."""
    count = len(problems)
    if not (len(params) == len(bs) == len(us) == count) or (ss is not None and len(ss) != count):
        raise ValueError("batch lists must have one entry per problem")
    sz = [_sizes(p) for p in problems]
    pa = (mof_solver_params * count)(*params)
    reps = [(mof_report * n_outer)() for _ in range(count)]
    rp = _ptr_array([ctypes.cast(r, ctypes.c_void_p).value for r in reps])
    handles = _ptr_array([p.handle.value for p in problems])
    bp = _ptr_array([_ptr(p, b, z["m"], "b").value for p, b, z in zip(problems, bs, sz)])
    up = _ptr_array([_ptr(p, u, z["n"], "u").value for p, u, z in zip(problems, us, sz)])
    sp = None if ss is None else _ptr_array([_ptr(p, s_, z["nv"], "s").value for p, s_, z in zip(problems, ss, sz)])
    _check(_lib.mof_solve_batch(handles, count, pa, int(n_outer), bp, up, sp, rp, _stream(stream)))
    return [[{"lambda": r.lambda_, "resid": r.resid, "rnorm": r.rnorm, "basis": r.basis, "flag": r.flag,
              "of_basis_min": r.of_basis_min, "of_basis_max": r.of_basis_max} for r in rep] for rep in reps]


def mof_autotune(problems, params, n_probe, bs, us, stream=None):
    """Tunes of_streams for the batch in place (params is a list of mof_solver_params);
    returns the chosen value and the probe time in ms."""
    count = len(problems)
    sz = [_sizes(p) for p in problems]
    pa = (mof_solver_params * count)(*params)
    handles = _ptr_array([p.handle.value for p in problems])
    bp = _ptr_array([_ptr(p, b, z["m"], "b").value for p, b, z in zip(problems, bs, sz)])
    up = _ptr_array([_ptr(p, u, z["n"], "u").value for p, u, z in zip(problems, us, sz)])
    ms = ctypes.c_double()
    _check(_lib.mof_autotune(handles, count, pa, int(n_probe), bp, up, ctypes.byref(ms), _stream(stream)))
    for i in range(count):
        params[i].of_streams = pa[i].of_streams
    return pa[0].of_streams, ms.value


def mof_set_timing(p, enable):
    _check(_lib.mof_set_timing(p.handle, 1 if enable else 0))


def mof_set_warp(p, mode):
    """M(s) encoding for every later operator and solve on p: 0 bilinear, 1 rounding and clipping."""
    _check(_lib.mof_set_warp(p.handle, int(mode)))


def mof_get_timing(p):
    """{kernel class: (milliseconds, launch groups)} of the last solve with timing on."""
    cap = 64
    names = (ctypes.c_char_p * cap)()
    ms = (ctypes.c_double * cap)()
    cnt = (ctypes.c_longlong * cap)()
    count = ctypes.c_int()
    _check(_lib.mof_get_timing(p.handle, cap, names, ms, cnt, ctypes.byref(count)))
    return {names[i].decode(): (ms[i], cnt[i]) for i in range(min(count.value, cap))}


def mof_debug_set_wait_limit(polls):
    """Bound of the device waits on tile copies (test hook of the timeout path; < 0: default)."""
    _check(load().mof_debug_set_wait_limit(int(polls)))


def mof_measure_fp32_peaks():
    """(FP32 FMA TFLOP/s, L1 4-byte loads in 1e9/s) measured on the current device."""
    a, b = ctypes.c_double(0.0), ctypes.c_double(0.0)
    _check(load().mof_measure_fp32_peaks(ctypes.byref(a), ctypes.byref(b)))
    return a.value, b.value


def mof_last_error():
    load()
    return _lib.mof_last_error().decode()


def mof_kernel_launches():
    """Kernels launched by libmof in this process so far."""
    return int(load().mof_kernel_launches())
