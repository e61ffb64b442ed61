"""The stored oracle result of the 64x64x8 configuration is the committed oracle's output:
Alg. 1 is run again here through the generating script's own function (it calls only the
oracle, on the seeded input generator's data) and compared with the stored file.

Bars: u and s element-wise to 1e-6 of their largest values, lambda to 1e-6 relative, the DP
flags and basis sizes exactly. The result is bit-identical when BLAS runs with the threading
it had when the file was written; a single-threaded BLAS sums in another order and moves the
30-iteration result by about 4e-8. (The 256x256x32 sample takes minutes to regenerate and is
left to the script.)
"""
import importlib.util
import os

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))


def _script():
    path = os.path.join(HERE, "golden", "make_oracle_results.py")
    spec = importlib.util.spec_from_file_location("make_oracle_results", path)
    mod = importlib.util.module_from_spec(spec)
    spec.loader.exec_module(mod)
    return mod


def test_disks64x64x8_stored_result_is_the_oracles():
    m = _script()
    from paper_2501_12497_gb300 import synth
    w = synth.plain_fp64(0)
    res = m._run(w, w.b, None)
    rep = m._reports(res)
    g = np.load(os.path.join(HERE, "golden", "disks64x64x8_oracle_30x20.npz"))
    for name, got in (("u", res.u), ("s", res.s)):
        want = g[name]
        err = np.max(np.abs(got - want)) / np.max(np.abs(want))
        assert err <= 1e-6, (name, err)
    assert np.max(np.abs(rep["lam"] / g["lam"] - 1.0)) <= 1e-6
    assert np.array_equal(rep["flag"], g["flag"]) and np.array_equal(rep["basis"], g["basis"])
