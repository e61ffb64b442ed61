"""Benchmark of the MMGKS-OF hot path on GB300.

One step = one complete MMGKS-OF solve (Alg. 1) of 30 outer iterations, each
with a Solve-OF (Alg. 2, 20 GKS iterations on every frame pair), FP32
operators and FP64 Krylov bookkeeping and projected solves. Default workload:
the large single problem, 1024x1024 frames, T = 64, 90 angles per frame
rotating across frames, 1448 bins, 20 ellipses on a smooth background in rigid
plus smooth non-rigid motion (up to 3 px/frame), 0.5% noise.
`--workload ellipses256x256x32` runs the 256x256x32 six-ellipse problem (30
angles, 363 bins, 1% noise). The metric is outer solver iterations per second
over the whole job (N GPUs x steps x 30 / time).

  python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]
                  [--workload ...]

N > 1 runs under torchrun with one process per GPU: every rank solves its own
seeded problem of the same shape (independent replicas, no collective in the
data path); rank 0 prints one JSON line with the max-over-ranks time.
--impl reference times the FP64 CPU oracle on the host cores instead (the
same workload and metric, on a bounded sample, extrapolated as stated in its
line).
"""
import argparse
import json
import math
import os
import subprocess
import sys
import tempfile
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

N_OUTER = 30
OF_ITERS, OF_ELL, ELL = 20, 10, 10
# the solve workloads: generator name in synth, sizes
WORKLOADS = {
    "ellipses1024x1024x64": ("large_form", dict(n=1024, nt=64, na=90, nb=1448)),
    "ellipses256x256x32": ("precision_form", dict(n=256, nt=32, na=30, nb=363)),
    "disks64x64x8": ("plain_fp64", dict(n=64, nt=8, na=16, nb=64)),
}
DEFAULT_WORKLOAD = "ellipses1024x1024x64"
L2_FLUSH_BYTES = 512 << 20
# accuracy bar of the precision form on images and velocities after the fixed iteration count
TOL_PRECISION_FORM = 1e-4


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=5)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", choices=["ours", "reference"], default="ours")
    ap.add_argument("--e2e-steps", type=int, default=2)
    ap.add_argument("--precision", default="fp32", choices=["fp32", "fp64"],
                    help="fp32: FP32 operators with FP64 Krylov bookkeeping (default); fp64: every step in FP64 "
                         "(the plain method's configuration, --workload disks64x64x8)")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-accuracy", action="store_true",
                    help="skip the FP64 reference solve that time_to_tolerance_s is checked against")
    ap.add_argument("--no-class-step", action="store_true",
                    help="skip the instrumented single-stream step (no class times, no roofline); for profiling runs")
    ap.add_argument("--workload", choices=list(WORKLOADS) + ["batch48", "operators", "solve_of"],
                    default=DEFAULT_WORKLOAD,
                    help="the 1024x1024x64 problem (default), the 256x256x32 problem, 48 uneven problems "
                         "batched, every operator alone, or Solve-OF alone (one call per step)")
    ap.add_argument("--frames", type=int, default=0,
                    help="--workload operators: use only the first this many frames of the workload (0: all)")
    ap.add_argument("--size", type=int, default=1024, choices=[256, 1024],
                    help="frame size of --workload operators / solve_of: 1024 (the 1024x1024x64 sizes) or 256")
    ap.add_argument("--of-streams", type=int, default=0,
                    help="frame-pair groups of Solve-OF on separate streams (0 = library default)")
    ap.add_argument("--of-scale", type=int, default=1,
                    help="Solve-OF on frames downsampled by this factor (the paper's experiments: 2 or 4)")
    ap.add_argument("--tau", type=int, default=1,
                    help="Solve-OF every tau outer iterations (the paper's experiments: 20)")
    ap.add_argument("--temporal-tv", type=int, default=0, choices=[0, 1],
                    help="1: the D1-OF regulariser (temporal differences added to Theta)")
    ap.add_argument("--geometry", default="parallel", choices=["parallel", "fan"],
                    help="fan (256x256x32 only): the same workload in a flat fan beam (source 512 px, detector "
                         "256 px beyond the centre, 363 bins of 1.6 px)")
    ap.add_argument("--of-pq", type=int, default=2, choices=[1, 2],
                    help="norms of Solve-OF: 2 (p = q = 2, the paper's experiments) or 1 (p = q = 1 by MM-GKS)")
    ap.add_argument("--warp", default="bilinear", choices=["bilinear", "round"],
                    help="encoding of the warp M(s) (Sec. 3): bilinear interpolation or rounding and clipping")
    return ap.parse_args()


def make_workload(name, seed, geometry="parallel"):
    from paper_2501_12497_gb300 import synth
    if geometry == "fan":
        if name != "ellipses256x256x32":
            raise SystemExit("--geometry fan is defined for --workload ellipses256x256x32")
        return synth.fan_form(seed=seed)
    return getattr(synth, WORKLOADS[name][0])(seed=seed)


def dist_env():
    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return rank, world, local


# ------------------------------------------------------------ ranks
def max_over_ranks(value, world, device="cpu"):
    """The largest value over the ranks of the process group (the slowest rank's time)."""
    import torch
    t = torch.tensor([float(value)], dtype=torch.float64, device=device)
    if world > 1:
        import torch.distributed as dist
        dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def job_value(world, steps, n_outer, total_ms):
    """Whole-job throughput: outer iterations of all ranks per second of the slowest rank."""
    return world * steps * n_outer / (total_ms / 1e3)


# ------------------------------------------------------------ CPU oracle sample
def _pair_job(args):
    """One Solve-OF pair of the oracle, timed inside the worker (a spawned process whose
    BLAS runs one thread: the pool is started with OPENBLAS_NUM_THREADS=1 and
    OMP_NUM_THREADS=1 in its environment)."""
    ux, uy, ut = args
    from oracle import solver
    t0 = time.perf_counter()
    solver.solve_of_pair(ux, uy, ut, solver.Params())
    return time.perf_counter() - t0


def cpu_cores():
    try:
        return len(os.sched_getaffinity(0))
    except Exception:
        return os.cpu_count() or 1


def oracle_sample(w, pool_size):
    """The FP64 oracle (as it stands) timed on a bounded sample of one outer iteration of
    Alg. 1 on workload w, and the outer iteration's time extrapolated from it.

    Solve-OF: the oracle solves frame pair 0 of w (its true frames; the per-pair work of an
    outer iteration) on centred crops of nc x nc pixels; a pair of the full frames takes
    minutes, so two crop sizes are timed alone on one thread (nc = 128 and 256, or the frame
    size when smaller) and the time is extrapolated linearly in the pixel count to the full
    frame (the oracle's per-pair work is QR factorisations and operators linear in the
    pixels, plus a fixed cost per GKS iteration); the larger crop is also run in
    `pool_size` concurrent single-threaded processes, whose slowdown over the lone run
    scales the all-cores figure. Image step: the projector and its adjoint on frame 0, Psi on
    one frame, Mhat on one pair, Theta^T on one pair, the QR of one frame's P Theta V block
    with the mid-solve basis size K and the two reorthogonalisations of one frame's share of
    the basis, at the full frame size, scaled to all frames and pairs (per frame or pair the
    oracle's outer iteration applies H once, H^T once, Theta K + 2 times and Theta^T once,
    factors P Theta V and reorthogonalises). One thread: T - 1 pairs one after another plus
    the image step; all cores: ceil((T - 1) / pool_size) rounds of the pool plus the image
    step (the oracle's image step runs on one thread)."""
    import numpy as np
    from multiprocessing import get_context
    from oracle import ops, solver
    nt, ny, nx = w.u_true.shape
    P = nt - 1
    K = ELL + N_OUTER // 2

    def crop(c):
        y0, x0 = (ny - c) // 2, (nx - c) // 2
        f = w.u_true[:2, y0:y0 + c, x0:x0 + c]
        ux, uy, ut = ops.of_fields(f, solver.Params().of_dr)
        return ux[0], uy[0], ut[0]

    sizes = sorted({min(128, nx, ny), min(256, nx, ny)})
    lone = {}
    saved = {k: os.environ.get(k) for k in ("OPENBLAS_NUM_THREADS", "OMP_NUM_THREADS", "MKL_NUM_THREADS")}
    for k in saved:  # the workers' BLAS: one thread each (read when a worker first loads numpy)
        os.environ[k] = "1"
    try:
        with get_context("spawn").Pool(max(1, min(pool_size, P))) as pool:
            for c in sizes:  # alone, one process
                lone[c] = pool.apply(_pair_job, (crop(c),))
            big = sizes[-1]
            jobs = [crop(big)] * max(1, min(pool_size, P))
            t0 = time.perf_counter()
            per = pool.map(_pair_job, jobs)
            wall_pool = time.perf_counter() - t0
    finally:
        for k, v in saved.items():
            if v is None:
                os.environ.pop(k, None)
            else:
                os.environ[k] = v
    nfull = nx * ny
    if len(sizes) == 2 and sizes[0] != sizes[1]:
        a0, a1 = sizes[0] ** 2, sizes[1] ** 2
        slope = (lone[sizes[1]] - lone[sizes[0]]) / (a1 - a0)
        t_pair = lone[sizes[1]] + slope * (nfull - a1)
    else:
        t_pair = lone[big] * nfull / big ** 2
    slow = wall_pool / lone[big]  # the pool's slowdown over the lone run

    def timed(fn, reps=1):
        t = time.perf_counter()
        for _ in range(reps):
            fn()
        return (time.perf_counter() - t) / reps

    na0 = int(w.na[0])
    g1 = ops.Geometry(w.nx, w.ny, 1, w.nb, w.na[:1], w.angles[:na0], w.h, w.db, getattr(w, "fan", None))
    f0 = w.u_true[:1]
    t_h = timed(lambda: ops.project(g1, f0))
    t_ht = timed(lambda: ops.backproject(g1, w.b[:na0 * w.nb]))
    rng = np.random.default_rng(0)
    s1 = rng.uniform(-2, 2, (1, 2, ny, nx))
    sr1 = ops.reverse_flow(s1)
    t_psi = timed(lambda: ops.grad(f0), 3)
    t_mhat = timed(lambda: ops.flow(w.u_true[:2], s1, sr1), 2)
    r1 = rng.standard_normal((2, 1, ny, nx))
    t_thT = timed(lambda: ops.gradT(rng.standard_normal((2, 2, ny, nx))) + ops.flowT(r1, s1, sr1))
    blk = rng.standard_normal((6 * ny * nx, K))  # one frame's rows of P Theta V (Psi 2, Mhat 4 per pixel)
    t_qr = timed(lambda: np.linalg.qr(blk, mode="r"))
    V1 = np.linalg.qr(rng.standard_normal((ny * nx, K)))[0]
    r = rng.standard_normal(ny * nx)
    t_re = timed(lambda: solver.reorth(r, V1), 3)
    t_image = (nt * (t_h + t_ht + t_re) + (K + 2) * (nt * t_psi + P * t_mhat) + P * t_thT + P * t_qr)
    t1 = P * t_pair + t_image
    rounds = math.ceil(P / len(jobs))
    tall = rounds * t_pair * slow + t_image
    sample = ("oracle on %s: Solve-OF of frame pair 0 on centred crops, %s pixels alone (%s s) and %d^2 in %d "
              "concurrent single-threaded processes (%.1f s wall), extrapolated linearly in pixels to a %dx%d "
              "pair (%.1f s), x%d pairs; image step from H, H^T, Psi, Mhat, Theta^T, the QR of P Theta V and the "
              "reorthogonalisation timed on single full frames with K = %d and scaled to %d frames (%.1f s); one "
              "outer iteration: %.1f s on one thread, %.1f s on %d processes"
              % (w.name, "/".join("%d^2" % c for c in sizes), "/".join("%.1f" % lone[c] for c in sizes), big,
                 len(jobs), wall_pool, nx, ny, t_pair, P, K, nt, t_image, t1, tall, len(jobs)))
    return {"single_thread_s": t1, "all_cores_s": tall, "processes": len(jobs), "sample": sample,
            "pair_s": t_pair, "image_s": t_image, "pool_wall_s": wall_pool}


def run_reference(args):
    rank, world, _ = dist_env()
    if rank != 0:
        return
    if args.workload not in WORKLOADS:
        print(json.dumps({"impl": "reference", "unavailable": "the reference arm times the solve workloads only"}))
        return
    w = make_workload(args.workload, 0, args.geometry)
    cores = cpu_cores()
    # one bounded sample (tens of seconds), repeated for the timed steps only as far as a
    # few minutes allow; the line states how many samples were taken
    res = []
    t_start = time.perf_counter()
    for i in range(max(1, args.steps)):
        res.append(oracle_sample(w, min(cores, w.nt - 1)))
        if time.perf_counter() - t_start > 150.0:
            break
    tall = sum(r["all_cores_s"] for r in res) / len(res)
    t1 = sum(r["single_thread_s"] for r in res) / len(res)
    value = 1.0 / tall
    wl, cfg = args.workload, WORKLOADS[args.workload][1]
    line = {
        "impl": "reference", "metric": "mmgks_of_outer_iterations_per_s", "value": value,
        "unit": "outer_iters/s", "n_gpus": 0, "steps": args.steps, "warmup": args.warmup,
        "ms_per_step": 1e3 * tall * N_OUTER, "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": "f64", "data": "synthetic",
        "config": {"workload": wl, **cfg, "n_outer": N_OUTER, "of_iters": OF_ITERS, "ell": ELL},
        "cpu_baseline": {"value": value, "unit": "outer_iters/s", "cores": res[0]["processes"], "kind": "oracle",
                         "single_thread_value": 1.0 / t1, "host_cores": cores,
                         "samples_taken": len(res), "sample": res[0]["sample"]},
        "e2e": {"value": value, "unit": "outer_iters/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line), flush=True)


# ------------------------------------------------------------ clock sampling
class Clocks:
    def __init__(self, enabled):
        self.proc = None
        self.path = None
        if not enabled:
            return
        fd, self.path = tempfile.mkstemp(suffix=".csv")
        os.close(fd)
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", "--query-gpu=index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
                 "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
                 "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap",
                 "--format=csv,noheader,nounits", "-lms", "200"],
                stdout=open(self.path, "w"), stderr=subprocess.DEVNULL)
        except Exception:
            self.proc = None

    def stop(self, gpu_index):
        if self.proc is None:
            return None
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except Exception:
            self.proc.kill()
        sm, mx, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for line in open(self.path):
            f = [x.strip() for x in line.split(",")]
            if len(f) < 9 or f[0] != str(gpu_index):
                continue
            try:
                sm.append(float(f[1]))
                mx.append(float(f[2]))
            except ValueError:
                continue
            for nm, v in zip(names, f[5:9]):
                if v.lower() == "active":
                    reasons.add(nm)
        os.unlink(self.path)
        if not sm:
            return None
        sm.sort()
        return {"sm_mhz": sm[len(sm) // 2], "sm_max_mhz": max(mx), "reasons": sorted(reasons), "samples": len(sm)}


# ------------------------------------------------------------ roofline models
def class_bytes(name, w, of_scale=1, tau=1):
    """Algorithmic bytes (minimum FP32 traffic) of one solve's work in a timing class of
    the library, and the number of launches of its main kernel, from the basis sizes of a
    solve without breakdown (the reports confirm it: image basis ELL + k, Solve-OF basis
    OF_ELL + OF_ITERS - 1 at the end). None for classes without a model.

    Solve-OF, per pair and GKS iteration it (basis K = OF_ELL + it, vectors of N2 = 2 ns
    values): of_combine s = V z reads K vectors and writes s; of_subdot (the projection pass
    with the new vector's Gram column, k_of_proj_gram_pass, and around it the Laplacian of the
    residual, the reduction and the append) reads the K basis vectors, the residual, its
    Laplacian, Ups^T b and the fields u_x, u_y (one vector's worth) and writes x'; the
    Laplacian pass reads the residual and writes its Laplacian; the append reads x' and writes
    the new vector: K + 9 vectors; of_gram (the Golub-Kahan start's Gram columns, j < OF_ELL)
    reads j + 1 vectors and the fields u_x, u_y, u_t each. theta_gram (the weighted Gram of
    Theta V for the image step, K = ELL + k at outer iteration k): the basis once (K vectors of
    n), u_k, s and s'."""
    nt, ny, nx = w.nt, w.ny, w.nx
    ns = (nx // of_scale) * (ny // of_scale)
    N2, P, n = 2 * ns, nt - 1, nx * ny * nt
    of_calls = sum(1 for k in range(1, N_OUTER) if k % tau == 0)  # u^(0) = 0: no OF work at k = 0
    its = range(OF_ITERS)
    if name == "of_combine":
        return of_calls * P * sum(4 * N2 * (OF_ELL + it + 1) for it in its), of_calls * OF_ITERS
    if name == "of_subdot":
        return of_calls * P * sum(4 * N2 * (OF_ELL + it + 9) for it in its[:-1]), of_calls * (OF_ITERS - 1)
    if name == "of_gram":
        return of_calls * P * sum(4 * (N2 * (j + 1) + 3 * ns) for j in range(OF_ELL)), of_calls
    if name == "of_gkb":
        # Golub-Kahan start, per pair: the norms of b and Ups^T b and u_1 (5 ns values), then per
        # step j < OF_ELL: Ups^T u_j - beta v_{j-1} (7 ns), the projection against the j stored v
        # (dot products, then the update: 4 j + 6 ns), the append of v_j (4 ns), Ups v_j - alpha u_j
        # (6 ns), the projection against the j + 1 stored u (2 j + 5 ns), the append of u_{j+1} (2 ns)
        return of_calls * P * 4 * ns * (5 + sum(6 * j + 30 for j in range(OF_ELL))), of_calls * OF_ELL
    if name == "theta_gram":
        return sum(4 * n * (ELL + k) + 4 * n + 16 * P * nx * ny for k in range(N_OUTER)), 2 * N_OUTER
    return None


# DRAM bytes over algorithmic bytes per launch of the kernel that dominates a class, from an
# ncu capture of that kernel (k_of_proj_gram_pass: 31 pairs of 256x256 frames at K = 20 and
# 21, 408.9 MB for 406.3 MB and 425.1 MB for 422.6 MB); the class's traffic per launch is
# estimated as this ratio times the class's algorithmic bytes per launch
TRAFFIC_RATIO = {"of_subdot": 1.006}

# the main kernel of each timing class
CLASS_KERNEL = {
    "of_gkb": "Golub-Kahan start of Solve-OF (k_of_upsT, k_of_ups, k_mdot, k_combine, k_append)",
    "of_gram": "k_of_gram_cols (Gram columns of the Solve-OF Golub-Kahan start, with their reduction)",
    "of_subdot": "k_of_proj_gram_pass (Solve-OF projection pass with the new Gram column; with the residual's "
                 "Laplacian, the chunk reduction and the append)",
    "of_combine": "k_combine (s = V z of Solve-OF)",
    "theta_gram": "k_theta_gram (weighted Gram of Theta V)",
}


def run_ours(args):
    import numpy as np
    import torch
    import torch.distributed as dist

    rank, world, local = dist_env()
    if world > 1:
        dist.init_process_group("nccl", init_method="env://")
    torch.cuda.set_device(local)
    import __graft_entry__
    if rank == 0:
        __graft_entry__.build()
    if world > 1:
        dist.barrier()
    from paper_2501_12497_gb300 import api
    api.load()
    dev = torch.device("cuda", local)
    w = make_workload(args.workload, rank, args.geometry)
    fp64 = args.precision == "fp64"
    prec, tdt, ndt, esz = ((api.MOF_FP64, torch.float64, np.float64, 8) if fp64 else
                           (api.MOF_FP32, torch.float32, np.float32, 4))
    p = api.mof_problem_create(w.nx, w.ny, w.nt, w.nb, w.na, w.angles, w.h, w.db, precision=prec, fan=w.fan)
    api.mof_set_warp(p, 1 if args.warp == "round" else 0)
    prm = api.mof_default_params(noise_norm=w.noise_norm, of_streams=args.of_streams, of_scale=args.of_scale,
                                 tau=args.tau, temporal_tv=args.temporal_tv, of_pq=args.of_pq)
    stream = torch.cuda.current_stream(dev)
    b = torch.tensor(w.b.astype(ndt), device=dev)
    u = torch.empty(p.n, dtype=tdt, device=dev)
    s = torch.empty(p.nv, dtype=tdt, device=dev)
    flush = torch.empty(L2_FLUSH_BYTES // 4, dtype=torch.float32, device=dev)
    for _ in range(args.warmup):
        api.mof_solve(p, prm, N_OUTER, b, u, s)
    torch.cuda.synchronize()
    clocks = Clocks(rank == 0)
    launches0 = api.mof_kernel_launches()
    per_step = []
    if world > 1:
        dist.barrier()
    torch.cuda.synchronize()
    for _ in range(args.steps):
        flush.fill_(1.0)  # evict L2 between timed steps
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        rep = api.mof_solve(p, prm, N_OUTER, b, u, s)
        e1.record(stream)
        e1.synchronize()
        per_step.append(e0.elapsed_time(e1))
    torch.cuda.synchronize()
    launches = api.mof_kernel_launches() - launches0
    if world > 1:
        dist.barrier()
    clk = clocks.stop(local)
    total_ms = max_over_ranks(sum(per_step), world, dev)
    value = job_value(world, args.steps, N_OUTER, total_ms)
    u32 = u.cpu().double().numpy()
    s32 = s.cpu().double().numpy()

    # per-kernel-class device time from one extra, instrumented step with the frame-pair
    # groups of Solve-OF on a single stream, so that no two classes of Solve-OF overlap in
    # time (the timed steps above run them on several streams, uninstrumented)
    class_ms = {}
    if not args.no_class_step:
        prm1 = api.mof_default_params(noise_norm=w.noise_norm, of_streams=1, of_scale=args.of_scale, tau=args.tau,
                                      temporal_tv=args.temporal_tv, of_pq=args.of_pq)
        api.mof_solve(p, prm1, N_OUTER, b, u, s)
        flush.fill_(1.0)
        torch.cuda.synchronize()
        api.mof_set_timing(p, 1)
        api.mof_solve(p, prm1, N_OUTER, b, u, s)
        class_ms = {k: [ms, cnt] for k, (ms, cnt) in api.mof_get_timing(p).items()}
        api.mof_set_timing(p, 0)
        torch.cuda.synchronize()

    # end to end through the public host-buffer entry point: pinned host b in, u out
    bh = torch.empty(p.m, dtype=tdt, pin_memory=True)
    bh.copy_(torch.from_numpy(w.b.astype(ndt)))
    uh = torch.empty(p.n, dtype=tdt, pin_memory=True)
    bhn, uhn = bh.numpy(), uh.numpy()
    e2e_value = None
    if args.e2e_steps > 0:
        api.mof_solve_host(p, prm, N_OUTER, bhn, uhn)  # first call allocates the staging buffers
        if world > 1:
            dist.barrier()
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        for _ in range(args.e2e_steps):
            api.mof_solve_host(p, prm, N_OUTER, bhn, uhn)
        e2e_s = max_over_ranks(time.perf_counter() - t0, world, dev)
        e2e_value = job_value(world, args.e2e_steps, N_OUTER, 1e3 * e2e_s)

    # quality of the result (RRE against the phantom)
    rre = float(np.linalg.norm(u32 - w.u_true.ravel()) / np.linalg.norm(w.u_true))

    # time to tolerance: the FP32 result of a timed step against an FP64 solve of the same
    # problem on the GPU (the FP64 path, whose parity with the FP64 oracle the tests check),
    # both on the FP32-rounded data the FP32 path consumes. A second FP64 solve on data
    # perturbed by relative noise of the size of FP32 rounding (6e-8) measures how far the
    # problem itself moves the result: the reverse flow's rounding to pixels and GCV's choice
    # among local minima are discontinuous, so after 30 outer iterations two FP64 solves of
    # data that differ at the 1e-7 level can lie further apart than the 1e-4 bar.
    acc = None
    golden = os.path.join(ROOT, "tests", "golden", "disks64x64x8_oracle_30x20.npz")
    if fp64 and not args.no_accuracy and args.workload == "disks64x64x8" and os.path.exists(golden):
        # the FP64 form against the FP64 oracle's stored 30-iteration result (written by a script
        # that runs only the oracle)
        g = np.load(golden)
        eu = float(np.linalg.norm(u32 - g["u"].ravel()) / np.linalg.norm(g["u"]))
        es = float(np.linalg.norm(s32 - g["s"].ravel()) / np.linalg.norm(g["s"]))
        acc = {"reference": "FP64 oracle, stored result (tests/golden)", "tol": 1e-6, "u_rel_err": eu,
               "s_rel_err": es, "passed": eu <= 1e-6 and es <= 1e-6, "within_fp64_spread": False,
               "fp64_solve_s": None}
    elif not fp64 and not args.no_accuracy:
        def fp64_solve(bdata):
            p64 = api.mof_problem_create(w.nx, w.ny, w.nt, w.nb, w.na, w.angles, w.h, w.db,
                                         precision=api.MOF_FP64, fan=w.fan)
            api.mof_set_warp(p64, 1 if args.warp == "round" else 0)
            b64 = torch.tensor(bdata, dtype=torch.float64, device=dev)
            u64 = torch.empty(p.n, dtype=torch.float64, device=dev)
            s64 = torch.empty(p.nv, dtype=torch.float64, device=dev)
            torch.cuda.synchronize()
            t0 = time.perf_counter()
            api.mof_solve(p64, prm, N_OUTER, b64, u64, s64)
            torch.cuda.synchronize()
            t = time.perf_counter() - t0
            out = u64.cpu().numpy(), s64.cpu().numpy()
            del b64, u64, s64
            p64.close()
            torch.cuda.empty_cache()
            return out[0], out[1], t

        def errs(a, ref):
            dn = max(np.linalg.norm(ref), 1e-300)
            return float(np.linalg.norm(a - ref) / dn), float(np.max(np.abs(a - ref)) / max(np.max(np.abs(ref)), 1e-300))

        b_r = w.b.astype(np.float32).astype(np.float64)
        ur, sr_, t64 = fp64_solve(b_r)
        xi = np.random.default_rng(12345).standard_normal(b_r.shape)
        up, sp, _ = fp64_solve(b_r * (1.0 + 6e-8 * xi))
        eu, eu_el = errs(u32, ur)
        es, es_el = errs(s32, sr_)
        du, du_el = errs(up, ur)
        ds, ds_el = errs(sp, sr_)
        strict = eu <= TOL_PRECISION_FORM and es <= TOL_PRECISION_FORM
        # within the spread of the FP64 path itself: no further from the FP64 result than twice
        # the distance an FP32-sized perturbation of the data moves that result
        spread = eu <= max(TOL_PRECISION_FORM, 2 * du) and es <= max(TOL_PRECISION_FORM, 2 * ds)
        acc = {"reference": "FP64 solve of the same problem on the GPU on the FP32-rounded data (%.1f s)" % t64,
               "tol": TOL_PRECISION_FORM, "u_rel_err": eu, "s_rel_err": es, "u_max_rel_err": eu_el,
               "s_max_rel_err": es_el, "passed": strict,
               "fp64_sensitivity": {"perturbation": "data times (1 + 6e-8 N(0,1)), seed 12345",
                                    "u_rel": du, "s_rel": ds, "u_max_rel": du_el, "s_max_rel": ds_el},
               "within_fp64_spread": spread, "fp64_solve_s": t64}

    # roofline of the dominant class with a byte model: achieved = algorithmic bytes of the
    # solve / the class's event-timed device time (single-stream step)
    peaks = {}
    pk = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(pk):
        peaks = json.load(open(pk))
    hbm_peak = float(peaks.get("hbm_gbs", 6800.0))
    peak_src = "measured" if "hbm_gbs" in peaks else "fallback"
    step1_ms = sum(v[0] for v in class_ms.values())
    modeled = {}
    for name, (ms, cnt) in class_ms.items():
        m = class_bytes(name, w, args.of_scale, args.tau) if args.of_pq == 2 and not fp64 else None
        if m is None or ms <= 0:
            continue
        nbytes, nlaunch = m
        gbs = nbytes / (ms / 1e3) / 1e9
        modeled[name] = {"ms": ms, "share_of_single_stream_step": ms / step1_ms, "algorithmic_bytes": nbytes,
                         "GB_s": gbs, "frac": gbs / hbm_peak, "launches": nlaunch}
    dominant = max(class_ms.items(), key=lambda kv: kv[1][0])[0] if class_ms else None
    roofline = None
    if modeled:
        top = dominant if dominant in modeled else max(modeled, key=lambda k: modeled[k]["ms"])
        m = modeled[top]
        per_launch = m["algorithmic_bytes"] / m["launches"]
        ratio = TRAFFIC_RATIO.get(top)
        roofline = {
            "kernel": CLASS_KERNEL.get(top, top), "class": top, "bound": "hbm", "achieved": m["GB_s"],
            "peak": hbm_peak, "unit": "GB/s", "frac": m["frac"],
            "traffic": ratio * per_launch if ratio else None,
            "traffic_source": ("ncu capture of the main kernel on the 256x256x32 workload: DRAM read + write = "
                               "%.3f x its algorithmic bytes, applied to the class's bytes per launch" % ratio)
            if ratio else None,
            "algorithmic_bytes_per_launch": per_launch, "peak_source": peak_src,
            "measured": "class time from one instrumented single-stream step after the timed region "
                        "(the timed steps run the frame pairs on their own streams inside CUDA graphs)",
            "share_of_single_stream_step": m["share_of_single_stream_step"],
            "largest_class_single_stream": dominant,
            "other_classes": {k: {"frac": round(v["frac"], 3), "share": round(v["share_of_single_stream_step"], 3)}
                              for k, v in modeled.items() if k != top},
        }
    if rank != 0:
        if world > 1:
            dist.destroy_process_group()
        return
    cpu = None
    if world == 1 and not args.no_cpu_baseline:
        cores = cpu_cores()
        smp = oracle_sample(w, min(cores, w.nt - 1))
        cpu = {"value": 1.0 / smp["all_cores_s"], "unit": "outer_iters/s", "cores": smp["processes"],
               "kind": "oracle", "single_thread_value": 1.0 / smp["single_thread_s"], "host_cores": cores,
               "sample": smp["sample"]}
    cfgd = WORKLOADS[args.workload][1]
    line = {
        "metric": "mmgks_of_outer_iterations_per_s", "value": value, "unit": "outer_iters/s",
        "n_gpus": world, "steps": args.steps, "warmup": args.warmup,
        "ms_per_step": total_ms / args.steps, "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": "f64" if fp64 else "f32+f64", "data": "synthetic",
        "config": {"workload": w.name, **cfgd, "n_outer": N_OUTER, "of_iters": OF_ITERS, "of_ell": OF_ELL, "ell": ELL,
                   "geometry": "fan (source 512, detector 256, bin 1.6)" if w.fan else "parallel",
                   "precision": "FP64 throughout" if fp64 else "FP32 operators, FP64 Krylov/projected solves",
                   "parallelism": "replicas",
                   "l2": "flushed between steps (512 MB write)", "rre": rre,
                   "of_streams": args.of_streams or "auto", "of_scale": args.of_scale, "tau": args.tau,
                   "regulariser": "D1-OF" if args.temporal_tv else "M-OF", "warp": args.warp,
                   "of_pq": args.of_pq,
                   # the FP32 form's solve time when its result is within the bar, or within the
                   # spread the FP64 path itself shows under FP32-sized data perturbations; else the
                   # FP64 path's (whose parity with the FP64 oracle the tests check on the 64x64x8
                   # and 256x256x32 configurations)
                   "time_to_tolerance_s": None if not acc else (total_ms / args.steps / 1e3
                                                                 if acc["passed"] or acc["within_fp64_spread"]
                                                                 else acc["fp64_solve_s"]),
                   "time_to_tolerance_form": None if not acc else (
                       "%s, within the %g bar" % ("FP64" if fp64 else "FP32 operators", acc["tol"]) if acc["passed"] else
                       "FP32 operators, within the FP64 path's own spread (the 1e-4 bar is below it)"
                       if acc["within_fp64_spread"] else "FP64 (the FP32 form is outside the bar and the spread)"),
                   "accuracy": acc,
                   "basis_last": rep[-1]["basis"], "of_basis_last": rep[-1]["of_basis_max"]},
        "e2e": {"value": e2e_value, "unit": "outer_iters/s", "h2d_bytes_per_step": esz * p.m,
                "d2h_bytes_per_step": esz * p.n + 64 * N_OUTER},
        "gpu_launches": launches,
        "clocks": clk,
        "roofline": roofline,
        "kernel_classes_ms_single_stream_step": {k: v[0] for k, v in sorted(class_ms.items(), key=lambda kv: -kv[1][0])},
        "cpu_baseline": cpu,
    }
    print(json.dumps(line), flush=True)
    if world > 1:
        dist.destroy_process_group()


def run_batch(args):
    """48 independent problems of uneven size (n in {128..512}, T in [8, 40], 10-45
    angles, ceil(sqrt(2) n) bins; ellipses carried by a smooth field): the batched,
    graph-captured form (mof_solve_batch, of_streams chosen by mof_autotune) against the
    plain unbatched per-frame form (plain = 1: every kernel launched from the host as it
    comes, Solve-OF one frame pair after another on one stream, the projector pair one
    frame per launch, the problems one after another), both computing the same results
    (compared element by element after the timed runs). Metric: outer iterations per
    second summed over the problems."""
    import numpy as np
    import torch
    import __graft_entry__
    __graft_entry__.build()
    from paper_2501_12497_gb300 import api, synth
    api.load()
    ws = synth.batch_form(count=48, seed=0)
    probs, params, plain, bs, us = [], [], [], [], []
    for w in ws:
        p = api.mof_problem_create(w.nx, w.ny, w.nt, w.nb, w.na, w.angles, precision=api.MOF_FP32)
        probs.append(p)
        params.append(api.mof_default_params(noise_norm=w.noise_norm))
        plain.append(api.mof_default_params(noise_norm=w.noise_norm, plain=1))
        bs.append(torch.tensor(w.b.astype(np.float32), device="cuda"))
        us.append(torch.empty(p.n, dtype=torch.float32, device="cuda"))
    g, _ = api.mof_autotune(probs, params, 2, bs, us)
    for _ in range(args.warmup):
        api.mof_solve_batch(probs, params, N_OUTER, bs, us)
    torch.cuda.synchronize()
    clocks = Clocks(True)
    l0 = api.mof_kernel_launches()
    t0 = time.perf_counter()
    for _ in range(args.steps):
        api.mof_solve_batch(probs, params, N_OUTER, bs, us)
    torch.cuda.synchronize()
    tb = time.perf_counter() - t0
    launches = api.mof_kernel_launches() - l0
    clk = clocks.stop(0)
    # the plain form: one problem after another, every launch from the host
    up = [torch.empty_like(u) for u in us]
    for p, prm, b, u in zip(probs, plain, bs, up):
        api.mof_solve(p, prm, N_OUTER, b, u)
    torch.cuda.synchronize()
    l1 = api.mof_kernel_launches()
    t0 = time.perf_counter()
    for p, prm, b, u in zip(probs, plain, bs, up):
        api.mof_solve(p, prm, N_OUTER, b, u)
    torch.cuda.synchronize()
    ts = time.perf_counter() - t0
    launches_plain = api.mof_kernel_launches() - l1
    diff = max(float((a - c).abs().max()) for a, c in zip(us, up))
    units = len(probs) * N_OUTER
    line = {
        "metric": "mmgks_of_outer_iterations_per_s", "value": args.steps * units / tb, "unit": "outer_iters/s",
        "n_gpus": 1, "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * tb / args.steps,
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f32+f64", "data": "synthetic",
        "config": {"workload": "batch48", "problems": len(probs), "pixels_total": int(sum(w.nx * w.ny * w.nt for w in ws)),
                   "n_outer": N_OUTER, "of_streams": g, "timing": "host wall clock around synchronised batches"},
        "plain": {"value": units / ts, "ms_per_step": 1e3 * ts, "gpu_launches": launches_plain,
                  "form": "plain = 1: eager launches, Solve-OF pair by pair on one stream, projector per frame, "
                          "problems one after another",
                  "max_abs_difference_to_batched": diff},
        "speedup_vs_plain": ts / (tb / args.steps),
        "gpu_launches": launches, "clocks": clk,
    }
    print(json.dumps(line), flush=True)


def run_operators(args):
    """Every operator of the C ABI applied alone at the sizes of the 1024x1024x64 problem
    (90 angles, 1448 bins; --size 256: the 256x256x32 problem, 30 angles, 363 bins), L2
    flushed before each application, CUDA events around it; achieved GB/s = algorithmic
    bytes (minimum FP32 traffic of one application) / time, against the measured copy
    peak. The projector pair is reported against HBM too, although it is bound by FP32
    and L1 work (36 flop per byte at 256^2, 113 at 1024^2)."""
    import numpy as np
    import torch
    import __graft_entry__
    __graft_entry__.build()
    from paper_2501_12497_gb300 import api, synth
    api.load()
    w = synth.large_form(0) if args.size == 1024 else synth.precision_form(0)
    vmax = 3.0 if args.size == 1024 else 2.0
    if 1 < args.frames < w.nt:  # a shorter sequence of the same frames, angles and data
        import dataclasses
        nt, na = args.frames, w.na[:args.frames]
        w = dataclasses.replace(w, nt=nt, na=na, angles=w.angles[:int(np.sum(na))], u_true=w.u_true[:nt],
                                b=w.b[:int(np.sum(na)) * w.nb])
    p = api.mof_problem_create(w.nx, w.ny, w.nt, w.nb, w.na, w.angles, precision=api.MOF_FP32)
    n, m, ns, P = p.n, p.m, p.nx * p.ny, p.nt - 1
    dev = "cuda"
    f32 = lambda a: torch.tensor(np.asarray(a, dtype=np.float32), device=dev).reshape(-1)
    u = f32(w.u_true)
    b = f32(w.b)
    s = f32(synth.random_velocities(P, p.ny, p.nx, vmax=vmax, seed=1))
    sr = torch.empty_like(s)
    api.mof_reverse_flow(p, s, sr)
    flow = torch.empty(2 * P * ns, device=dev)
    grad = torch.empty(2 * n, device=dev)
    img = torch.empty(n, device=dev)
    sino = torch.empty(m, device=dev)
    ux, uy, ut = (torch.empty(P * ns, device=dev) for _ in range(3))
    api.mof_of_fields(p, u, 1, ux, uy, ut)
    pr = torch.empty(P * ns, device=dev)
    vel = torch.empty(p.nv, device=dev)
    vel2 = torch.empty(p.nv, device=dev)
    vg = torch.empty(2 * p.nv, device=dev)
    r2 = torch.randn(2 * P * ns, device=dev)
    wf = synth.fan_form(0)
    pf = api.mof_problem_create(wf.nx, wf.ny, wf.nt, wf.nb, wf.na, wf.angles, wf.h, wf.db, precision=api.MOF_FP32,
                                fan=wf.fan)
    bf = f32(wf.b)
    uf = f32(wf.u_true)
    sinof = torch.empty(pf.m, device=dev)
    imgf = torch.empty(pf.n, device=dev)
    nf, mf = pf.n, pf.m
    ops = [
        ("H (k_project)", 4 * (n + m), lambda: api.mof_apply_A(p, u, sino)),
        ("H^T (k_backproject)", 4 * (n + m), lambda: api.mof_apply_AT(p, b, img)),
        ("fan H (k_project_fan, 256x256x32)", 4 * (nf + mf) + 16 * mf, lambda: api.mof_apply_A(pf, uf, sinof)),
        ("fan H^T (k_backproject_fan, 256x256x32)", 4 * (nf + mf) + 16 * mf, lambda: api.mof_apply_AT(pf, bf, imgf)),
        ("Psi (k_grad)", 12 * n, lambda: api.mof_apply_grad(p, u, grad)),
        ("Psi^T (k_gradT)", 12 * n, lambda: api.mof_apply_gradT(p, grad, img)),
        ("Mhat (k_flow)", 4 * n + 24 * P * ns, lambda: api.mof_apply_flow(p, u, s, sr, flow)),
        ("Mhat^T (k_flowT + radii)", 4 * n + 24 * P * ns, lambda: api.mof_apply_flowT(p, r2, s, sr, img)),
        ("Theta^T W Theta (k_regn_*)", 12 * n + 16 * P * ns, lambda: api.mof_apply_reg_normal(p, u, u, s, sr, 1e-3, img)),
        ("reverse flow (k_rev_*)", 16 * P * ns, lambda: api.mof_reverse_flow(p, s, sr)),
        ("App. C fields (k_of_fields)", 4 * n + 12 * P * ns, lambda: api.mof_of_fields(p, u, 1, ux, uy, ut)),
        ("Upsilon s + u_t (k_flow_lin)", 24 * P * ns, lambda: api.mof_apply_flow_lin(p, ux, uy, ut, s, pr)),
        ("Upsilon^T r (k_flow_linT)", 20 * P * ns, lambda: api.mof_apply_flow_linT(p, ux, uy, pr, vel)),
        ("(L+L) s (k_grad)", 24 * P * ns, lambda: api.mof_apply_vgrad(p, s, vg)),
        ("(L+L)^T g (k_gradT)", 24 * P * ns, lambda: api.mof_apply_vgradT(p, vg, vel)),
        ("velocity VJP (k_flow_ds)", 4 * n + 40 * P * ns, lambda: api.mof_apply_flow_ds(p, u, s, sr, r2, vel, vel2)),
    ]
    peaks = {}
    pk = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(pk):
        peaks = json.load(open(pk))
    peak = float(peaks.get("hbm_gbs", 6800.0))
    # the projector pair's own ceilings: FP32 FMA rate and L1 4-byte loads, measured here;
    # its algorithmic work is 2 m nx FMAs (two taps per step) and as many loads
    fma_tflops, l1_gl = api.mof_measure_fp32_peaks()
    tomo = {"H (k_project)": (m, p.nx), "H^T (k_backproject)": (m, p.nx),
            "fan H (k_project_fan, 256x256x32)": (mf, pf.nx), "fan H^T (k_backproject_fan, 256x256x32)": (mf, pf.nx)}
    flush = torch.empty(L2_FLUSH_BYTES // 4, device=dev)
    reps = max(args.steps, 5)
    out = {}
    for name, nbytes, fn in ops:
        for _ in range(max(args.warmup, 3)):
            fn()
        torch.cuda.synchronize()
        tot = 0.0
        for _ in range(reps):
            flush.fill_(1.0)
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record()
            fn()
            e1.record()
            e1.synchronize()
            tot += e0.elapsed_time(e1)
        us = 1e3 * tot / reps
        gbs = nbytes / (us * 1e-6) / 1e9
        out[name] = {"us": round(us, 2), "algorithmic_MB": round(nbytes / 1e6, 2), "GB_s": round(gbs, 1),
                     "frac_of_measured_peak": round(gbs / peak, 3)}
        if name in tomo:
            mm, nxx = tomo[name]
            fma = 2.0 * mm * nxx
            out[name].update({"bound": "fp32/l1", "fma_TFLOP_s": round(2 * fma / (us * 1e-6) / 1e12, 2),
                              "frac_of_measured_fp32_fma": round(2 * fma / (us * 1e-6) / 1e12 / fma_tflops, 4),
                              "l1_Gloads_s": round(fma / (us * 1e-6) / 1e9, 1),
                              "frac_of_measured_l1_loads": round(fma / (us * 1e-6) / 1e9 / l1_gl, 4)})
    line = {"metric": "operator_applications", "unit": "GB/s", "config": {"workload": "%s operators" % w.name,
            "l2": "flushed before each application", "reps": reps, "peak_gbs": peak,
            "measured_fp32_fma_TFLOP_s": round(fma_tflops, 1), "measured_l1_Gloads_s": round(l1_gl, 1)},
            "operators": out}
    print(json.dumps(line), flush=True)


def run_solve_of(args):
    """Solve-OF (Alg. 2) alone: one mof_solve_of call per step on the true frames of the
    1024x1024x64 workload (63 frame pairs; --size 256: the 256x256x32 workload, 31 pairs),
    of_ell 10, 20 GKS iterations, inputs resident, L2 flushed before each call, CUDA events
    around it."""
    import numpy as np
    import torch
    import __graft_entry__
    __graft_entry__.build()
    from paper_2501_12497_gb300 import api, synth
    api.load()
    w = synth.large_form(0) if args.size == 1024 else synth.precision_form(0)
    p = api.mof_problem_create(w.nx, w.ny, w.nt, w.nb, w.na, w.angles, precision=api.MOF_FP32)
    prm = api.mof_default_params(of_streams=args.of_streams, of_scale=args.of_scale, of_pq=args.of_pq)
    u = torch.tensor(w.u_true.astype(np.float32), device="cuda").reshape(-1)
    s = torch.empty(p.nv, dtype=torch.float32, device="cuda")
    flush = torch.empty(L2_FLUSH_BYTES // 4, dtype=torch.float32, device="cuda")
    for _ in range(args.warmup):
        api.mof_solve_of(p, prm, u, s)
    torch.cuda.synchronize()
    l0 = api.mof_kernel_launches()
    ms = []
    for _ in range(args.steps):
        flush.fill_(1.0)
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record()
        api.mof_solve_of(p, prm, u, s)
        e1.record()
        e1.synchronize()
        ms.append(e0.elapsed_time(e1))
    tot = sum(ms)
    line = {"metric": "solve_of_calls_per_s", "value": args.steps / (tot / 1e3), "unit": "calls/s", "n_gpus": 1,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": tot / args.steps, "higher_is_better": True,
            "dtype": "f32+f64", "data": "synthetic",
            "config": {"workload": "solve_of %s" % w.name, "pairs": p.nt - 1, "of_ell": 10, "of_iters": 20,
                       "of_pq": args.of_pq,
                       "of_streams": args.of_streams or "auto", "of_scale": args.of_scale, "l2": "flushed before each call"},
            "gpu_launches": api.mof_kernel_launches() - l0}
    print(json.dumps(line), flush=True)


def main():
    args = parse()
    if args.impl == "reference":
        run_reference(args)
    elif args.workload == "batch48":
        run_batch(args)
    elif args.workload == "operators":
        run_operators(args)
    elif args.workload == "solve_of":
        run_solve_of(args)
    else:
        run_ours(args)


if __name__ == "__main__":
    main()
