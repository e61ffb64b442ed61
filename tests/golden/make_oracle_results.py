"""Write the FP64 oracle's end-to-end results that the GPU parity tests compare with.

Test infrastructure: this script calls only the oracle (oracle/) on inputs from the
seeded generators (paper_2501_12497_gb300/synth.py, which holds none of the method's
arithmetic); no value here comes from the CUDA path.

  python tests/golden/make_oracle_results.py [disks64x64x8] [ellipses256x256x32]

disks64x64x8: Alg. 1 on the 64x64x8 two-disk workload (16 angles, 64 bins, 1% noise),
  30 outer iterations, each with Solve-OF of 20 GKS iterations (Alg. 2) on the 7
  frame pairs; the whole image sequence and velocity field in FP64 and the per-iteration
  reports (lambda, DP flag, basis size, data misfit).
ellipses256x256x32: the same on the 256x256x32 six-ellipse workload (30 angles, 363
  bins, 1% noise) on the FP32-rounded data the FP32 path consumes; frames 0, 11, 22, 31
  of the image sequence and pairs 0, 10, 20, 30 of the velocity field, stored FP32
  (their rounding, 6e-8, is far below the 1e-4 the tests ask), the norms of the whole
  sequence and field, and the reports. The oracle takes several minutes here (a spawned
  process pool over the frame pairs).
"""
import os
import sys
import time

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(os.path.dirname(HERE))
sys.path.insert(0, ROOT)

from oracle import ops, solver  # noqa: E402
from paper_2501_12497_gb300 import synth  # noqa: E402

N_OUTER = 30
C2_FRAMES = (0, 11, 22, 31)
C2_PAIRS = (0, 10, 20, 30)


def _run(w, b, pool):
    g = ops.Geometry(w.nx, w.ny, w.nt, w.nb, w.na, w.angles, w.h, w.db)
    prm = solver.Params(noise_norm=w.noise_norm)
    return solver.mmgks_of(g, b, prm, N_OUTER, pool=pool)


def _reports(res):
    return dict(lam=np.array([r["lam"] for r in res.report]), flag=np.array([r["flag"] for r in res.report]),
                basis=np.array([r["basis"] for r in res.report]), resid=np.array([r["resid"] for r in res.report]))


def disks64(pool):
    w = synth.plain_fp64(0)
    res = _run(w, w.b, pool)
    np.savez_compressed(os.path.join(HERE, "disks64x64x8_oracle_30x20.npz"), u=res.u, s=res.s, **_reports(res))


def ellipses256(pool):
    w = synth.precision_form(0)
    res = _run(w, w.b.astype(np.float32).astype(np.float64), pool)
    np.savez_compressed(os.path.join(HERE, "ellipses256x256x32_oracle_30x20_sample.npz"),
                        frames=np.array(C2_FRAMES), pairs=np.array(C2_PAIRS),
                        u=res.u[list(C2_FRAMES)].astype(np.float32), s=res.s[list(C2_PAIRS)].astype(np.float32),
                        u_norm=np.linalg.norm(res.u), s_norm=np.linalg.norm(res.s), **_reports(res))


if __name__ == "__main__":
    from multiprocessing import get_context
    which = sys.argv[1:] or ["disks64x64x8", "ellipses256x256x32"]
    os.environ["OPENBLAS_NUM_THREADS"] = "1"  # the pool's workers: one thread each
    with get_context("spawn").Pool(min(8, os.cpu_count() or 1)) as pool:
        for name in which:
            t = time.time()
            {"disks64x64x8": disks64, "ellipses256x256x32": ellipses256}[name](pool)
            print("%s: %.0f s" % (name, time.time() - t), flush=True)
