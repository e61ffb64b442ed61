"""The C-ABI library builds, loads and exports every entry point include/mof.h
declares; argument checks that happen on the host need no GPU."""
import ctypes
import os
import re

import numpy as np
import pytest

from paper_2501_12497_gb300 import api, build

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def declared_symbols():
    text = open(os.path.join(ROOT, "include", "mof.h")).read()
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    return sorted(set(re.findall(r"\b(mof_[A-Za-z0-9_]+)\s*\(", text)))


@pytest.fixture(scope="module")
def lib():
    build.build()
    return api.load()


def test_header_declares_the_boundary():
    names = declared_symbols()
    for required in ("mof_problem_create", "mof_problem_destroy", "mof_apply_A", "mof_apply_AT",
                     "mof_apply_grad", "mof_apply_gradT", "mof_apply_flow", "mof_apply_flowT",
                     "mof_apply_flow_lin", "mof_apply_flow_linT", "mof_solve", "mof_last_error"):
        assert required in names


def test_library_exports_every_declared_symbol(lib):
    missing = [n for n in declared_symbols() if not hasattr(lib, n)]
    assert not missing, missing


def test_default_params(lib):
    p = api.mof_default_params()
    assert (p.ell, p.tau, p.of_iters, p.of_ell, p.of_dr) == (10, 1, 20, 10, 1)
    assert p.image_rule == api.MOF_RULE_DP and p.eps == 1e-3 and p.eta == 1.01


def test_create_rejects_bad_geometry_on_the_host(lib):
    for nx, ny, nt, nb, na in ((1, 8, 3, 8, [2, 2, 2]), (8, 8, 1, 8, [2]), (8, 8, 3, 0, [2, 2, 2]),
                               (8, 8, 3, 8, [2, 0, 2])):
        with pytest.raises(api.MofError) as e:
            api.mof_problem_create(nx, ny, nt, nb, na, np.zeros(max(sum(na), 1)))
        assert e.value.status == api.MOF_EINVAL
    with pytest.raises(api.MofError) as e:
        api.mof_problem_create(8, 8, 2, 8, [1, 1], [0.0, np.nan])
    assert e.value.status == api.MOF_EINVAL
    with pytest.raises(api.MofError) as e:
        api.mof_problem_create(8, 8, 2, 8, [1, 1], [0.0, 1.0], pixel_size=0.0)
    assert e.value.status == api.MOF_EINVAL
    with pytest.raises(api.MofError) as e:
        api.mof_problem_create(5000, 8, 2, 8, [1, 1], [0.0, 1.0])
    assert e.value.status == api.MOF_EUNSUPPORTED


def test_null_arguments_are_rejected(lib):
    assert lib.mof_problem_create(None, 0, None) == api.MOF_EINVAL
    assert "null" in api.mof_last_error()
    assert lib.mof_apply_A(None, None, None, None) == api.MOF_EINVAL
    prm = api.mof_default_params()
    assert lib.mof_solve(None, ctypes.byref(prm), 3, None, None, None, None, None, None) == api.MOF_EINVAL
    assert lib.mof_solve_of(None, ctypes.byref(prm), None, None, None) == api.MOF_EINVAL


def _header_struct_fields(name):
    """(type, field) pairs of `typedef struct { ... } name;` in include/mof.h, in order."""
    text = open(os.path.join(ROOT, "include", "mof.h")).read()
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    body = re.search(r"typedef struct\s*\{([^}]*)\}\s*" + name + r"\s*;", text).group(1)
    out = []
    for decl in body.split(";"):
        decl = decl.strip()
        if not decl:
            continue
        m = re.match(r"(const\s+)?(\w+)\s+(.*)$", decl, flags=re.S)
        assert m, decl
        for item in m.group(3).split(","):  # "int nx, ny" declares several fields
            item = item.strip()
            ptr = item.startswith("*")
            out.append((m.group(2) + ("*" if ptr else ""), item.lstrip("*").strip()))
    return out


@pytest.mark.parametrize("name", ["mof_geometry", "mof_solver_params", "mof_report"])
def test_ctypes_structs_follow_the_header(name):
    """The binding's structures list the header's fields in the same order with the same
    scalar types, so the layouts agree on any platform."""
    ctype = {"int": ctypes.c_int, "double": ctypes.c_double}
    fields = getattr(api, name)._fields_
    hdr = _header_struct_fields(name)
    assert len(fields) == len(hdr), (fields, hdr)
    for (pyname, pytype), (ctyp, cname) in zip(fields, hdr):
        assert pyname.rstrip("_") == cname, (pyname, cname)
        if ctyp in ctype:
            assert pytype is ctype[ctyp], (cname, pytype, ctyp)
        else:
            assert ctyp.endswith("*") and issubclass(pytype, ctypes._Pointer), (cname, pytype, ctyp)


def test_defaults_of_the_widened_options(lib):
    p = api.mof_default_params()
    assert (p.of_scale, p.temporal_tv, p.of_pq, p.of_streams) == (1, 0, 2, 0)


def test_fan_problem_rejects_bad_distances_on_the_host(lib):
    na, ang = [2, 2], [0.0, 1.0, 0.5, 1.5]
    # half the diagonal of a 32 x 32 frame is 22.6 pixels: a source inside the field
    for rs, rd in ((20.0, 5.0), (24.0, 5.0), (60.0, -1.0), (float("inf"), 1.0), (60.0, float("nan"))):
        with pytest.raises(api.MofError) as e:
            api.mof_problem_create(32, 32, 2, 64, na, ang, fan=(rs, rd))
        assert e.value.status == api.MOF_EINVAL


def test_fan_problem_rejects_distances_beyond_the_fp32_bin_search(lib):
    with pytest.raises(api.MofError) as e:
        api.mof_problem_create(32, 32, 2, 64, [2, 2], [0.0, 1.0, 0.5, 1.5], bin_size=1.0, fan=(2e5, 0.0))
    assert e.value.status == api.MOF_EUNSUPPORTED


def test_set_warp_rejects_a_null_problem(lib):
    assert lib.mof_set_warp(None, 1) == api.MOF_EINVAL
