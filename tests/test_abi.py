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
