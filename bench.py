"""Benchmark of the MMGKS-OF hot path on GB300.

One step = one complete MMGKS-OF solve (Alg. 1) of 30 outer iterations, each
with a Solve-OF (Alg. 2, 20 GKS iterations on every one of the 31 frame
pairs), on the 256x256x32 moving-ellipse workload (30 angles per frame
rotating across frames, 363 bins, 1% noise): FP32 operators, FP64 Krylov
bookkeeping and projected solves. The metric is outer solver iterations per
second over the whole job (N GPUs x steps x 30 / time).

  python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]

N > 1 runs under torchrun with one process per GPU: every rank solves its own
seeded problem of the same shape (independent replicas, no collective in the
data path); rank 0 prints one JSON line with the max-over-ranks time.
--impl reference times the FP64 CPU oracle on the host cores instead (the
same workload and metric, a bounded sample per step, extrapolated).
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
WORKLOAD = "ellipses256x256x32"
CFG = dict(n=256, nt=32, na=30, nb=363)
L2_FLUSH_BYTES = 512 << 20


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=5)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", choices=["ours", "reference"], default="ours")
    ap.add_argument("--e2e-steps", type=int, default=2)
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-class-step", action="store_true",
                    help="skip the instrumented single-stream step (no class times, no roofline); for profiling runs")
    ap.add_argument("--workload", choices=["ellipses256x256x32", "batch48", "ellipses1024x1024x64", "operators",
                                           "solve_of"],
                    default="ellipses256x256x32",
                    help="the 256x256x32 ellipse problem (default), 48 uneven problems batched, "
                         "the 1024x1024x64 problem, every operator alone, or Solve-OF alone "
                         "(one call per step on the 256x256x32 frames)")
    ap.add_argument("--of-streams", type=int, default=0,
                    help="frame-pair groups of Solve-OF on separate streams (0 = library default)")
    ap.add_argument("--of-scale", type=int, default=1,
                    help="Solve-OF on frames downsampled by this factor (the paper's experiments: 2 or 4)")
    ap.add_argument("--tau", type=int, default=1,
                    help="Solve-OF every tau outer iterations (the paper's experiments: 20)")
    ap.add_argument("--temporal-tv", type=int, default=0, choices=[0, 1],
                    help="1: the D1-OF regulariser (temporal differences added to Theta)")
    ap.add_argument("--geometry", default="parallel", choices=["parallel", "fan"],
                    help="fan: the same workload in a flat fan beam (source 512 px, detector 256 px beyond "
                         "the centre, 363 bins of 1.6 px)")
    ap.add_argument("--of-pq", type=int, default=2, choices=[1, 2],
                    help="norms of Solve-OF: 2 (p = q = 2, the paper's experiments) or 1 (p = q = 1 by MM-GKS)")
    ap.add_argument("--warp", default="bilinear", choices=["bilinear", "round"],
                    help="encoding of the warp M(s) (Sec. 3): bilinear interpolation or rounding and clipping")
    return ap.parse_args()


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
def oracle_outer_iteration_seconds(w):
    """Time the oracle (as it stands) on a bounded sample of one outer iteration:
    Solve-OF of one frame pair (the step the paper names as the bottleneck) on the
    reconstruction's ground-truth frames, scaled by the number of pairs; the image
    step's own cost is left out, so the figure flatters the oracle."""
    import numpy as np
    from oracle import ops, solver
    prm = solver.Params(noise_norm=w.noise_norm)
    ux, uy, ut = ops.of_fields(w.u_true[:2], prm.of_dr)
    t0 = time.perf_counter()
    solver.solve_of_pair(ux[0], uy[0], ut[0], prm)
    dt = time.perf_counter() - t0
    return dt * (w.nt - 1), dt


def cpu_cores():
    try:
        return len(os.sched_getaffinity(0))
    except Exception:
        return os.cpu_count() or 1


def run_reference(args):
    rank, world, _ = dist_env()
    if rank != 0:
        return
    from paper_2501_12497_gb300 import synth
    w = synth.precision_form(0)
    for _ in range(args.warmup):
        oracle_outer_iteration_seconds(w)
    tot = 0.0
    sample = 0.0
    for _ in range(args.steps):
        est, dt = oracle_outer_iteration_seconds(w)
        tot += est
        sample += dt
    value = args.steps / tot
    line = {
        "impl": "reference", "metric": "mmgks_of_outer_iterations_per_s", "value": value,
        "unit": "outer_iters/s", "n_gpus": 0, "steps": args.steps, "warmup": args.warmup,
        "ms_per_step": 1e3 * tot / args.steps, "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": "f64", "data": "synthetic",
        "config": {"workload": WORKLOAD, **CFG, "n_outer": N_OUTER, "of_iters": 20, "ell": 10},
        "cpu_baseline": {"value": value, "unit": "outer_iters/s", "cores": cpu_cores(), "kind": "oracle",
                         "sample": "per step: Solve-OF of 1 of the 31 frame pairs (%.1f s measured), "
                                   "x31 = one outer iteration; image step not counted" % (sample / args.steps)},
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
def subdot_bytes(nvec_list, N, pairs, es=4):
    """Algorithmic bytes of the fused CGS pass (k_sub_dot) over a solve: x - V c1 and
    V^T (x - V c1) read the K basis vectors and x and write x once, K + 2 vectors of N
    values, K the basis size at each call, for every active pair."""
    return sum(pairs * es * N * (K + 2) for K in nvec_list)


# DRAM bytes over algorithmic bytes of one k_sub_dot launch (31 pairs, K = 22) in the
# committed ncu capture (profiles/k_sub_dot_and_k_of_gram_cols_ellipses256x256x32.md):
# 391.4 MB of traffic for 390.1 MB of algorithmic bytes
SUBDOT_TRAFFIC_RATIO = 391.4 / 390.1


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
    from paper_2501_12497_gb300 import api, synth
    api.load()
    dev = torch.device("cuda", local)
    w = synth.fan_form(seed=rank) if args.geometry == "fan" else synth.precision_form(seed=rank)
    p = api.mof_problem_create(w.nx, w.ny, w.nt, w.nb, w.na, w.angles, w.h, w.db, precision=api.MOF_FP32, fan=w.fan)
    api.mof_set_warp(p, 1 if args.warp == "round" else 0)
    prm = api.mof_default_params(noise_norm=w.noise_norm, of_streams=args.of_streams, of_scale=args.of_scale,
                                 tau=args.tau, temporal_tv=args.temporal_tv, of_pq=args.of_pq)
    stream = torch.cuda.current_stream(dev)
    b = torch.tensor(w.b.astype(np.float32), device=dev)
    u = torch.empty(p.n, dtype=torch.float32, device=dev)
    s = torch.empty(p.nv, dtype=torch.float32, device=dev)
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

    # per-kernel-class device time from one extra, instrumented step with the frame-pair
    # groups of Solve-OF on a single stream, so that no two classes overlap in time
    # (the timed steps above run them on several streams, uninstrumented)
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
    bh = torch.empty(p.m, dtype=torch.float32, pin_memory=True)
    bh.copy_(torch.from_numpy(w.b.astype(np.float32)))
    uh = torch.empty(p.n, dtype=torch.float32, pin_memory=True)
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

    # quality of the result (RRE against the phantom) and the DP residual
    rre = float(np.linalg.norm(u.cpu().numpy() - w.u_true.ravel()) / np.linalg.norm(w.u_true))

    # roofline of the dominant HBM-bound kernel: the fused CGS2 pass over the per-pair
    # Solve-OF bases (k_sub_dot)
    import json as _json
    peaks = {}
    pk = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(pk):
        peaks = _json.load(open(pk))
    hbm_peak = float(peaks.get("hbm_gbs", 6800.0))
    peak_src = "measured" if "hbm_gbs" in peaks else "fallback"
    N2 = 2 * (CFG["n"] // args.of_scale) ** 2
    pairs = CFG["nt"] - 1
    # OF runs on outer iterations k = 1..29 with k % tau == 0 (u^(0) = 0 gives u_t = 0 and no
    # work at k = 0); GKS iteration it reorthogonalises against of_ell + it vectors (it = 0..18)
    ks = [10 + it for it in range(19)] * sum(1 for k in range(1, N_OUTER) if k % args.tau == 0)
    bytes_total = subdot_bytes(ks, N2, pairs)
    sd_ms, sd_cnt = class_ms.get("of_subdot", [float("nan"), 0])
    achieved = bytes_total / (sd_ms / 1e3) / 1e9 if sd_ms == sd_ms and sd_ms > 0 else None
    step1_ms = sum(v[0] for v in class_ms.values())
    dominant = max(class_ms.items(), key=lambda kv: kv[1][0])[0] if class_ms else None
    n_subdot = len(ks)  # one launch per GKS iteration for all pairs in the single-stream step
    roofline = {
        "kernel": "k_sub_dot (fused CGS2 pass of the Solve-OF residuals, with its chunk reduction)",
        "bound": "hbm", "achieved": achieved, "peak": hbm_peak, "unit": "GB/s",
        "frac": (achieved / hbm_peak) if achieved else None,
        "traffic": SUBDOT_TRAFFIC_RATIO * bytes_total / n_subdot,
        "traffic_source": "ncu capture of one launch (31 pairs, K = 22): DRAM read + write = 1.003 x algorithmic; "
                          "scaled to the average launch by the vectors it streams",
        "algorithmic_bytes_per_launch": bytes_total / n_subdot,
        "peak_source": peak_src,
        "bytes_model": "K+2 vectors of 2*n*n FP32 per pair and GKS iteration",
        "measured": "class time from one instrumented single-stream step after the timed region "
                    "(the timed steps run every pair on its own stream inside CUDA graphs)",
        "share_of_single_stream_step": sd_ms / step1_ms if step1_ms else None,
        "largest_class_single_stream": dominant,
    }
    if rank != 0:
        if world > 1:
            dist.destroy_process_group()
        return
    cpu = None
    if world == 1 and not args.no_cpu_baseline:
        est, dt = oracle_outer_iteration_seconds(w)
        cpu = {"value": 1.0 / est, "unit": "outer_iters/s", "cores": cpu_cores(), "kind": "oracle",
               "sample": "Solve-OF of 1 of the 31 frame pairs (%.1f s), x31 = one outer iteration; "
                         "image step not counted" % dt}
    line = {
        "metric": "mmgks_of_outer_iterations_per_s", "value": value, "unit": "outer_iters/s",
        "n_gpus": world, "steps": args.steps, "warmup": args.warmup,
        "ms_per_step": total_ms / args.steps, "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": "f32+f64", "data": "synthetic",
        "config": {"workload": w.name, **CFG, "n_outer": N_OUTER, "of_iters": 20, "of_ell": 10, "ell": 10,
                   "geometry": "fan (source 512, detector 256, bin 1.6)" if w.fan else "parallel",
                   "precision": "FP32 operators, FP64 Krylov/projected solves", "parallelism": "replicas",
                   "l2": "flushed between steps (512 MB write)", "rre": rre,
                   "of_streams": args.of_streams or "auto", "of_scale": args.of_scale, "tau": args.tau,
                   "regulariser": "D1-OF" if args.temporal_tv else "M-OF", "warp": args.warp,
                   "of_pq": args.of_pq,
                   "time_to_tolerance_s": total_ms / args.steps / 1e3},
        "e2e": {"value": e2e_value, "unit": "outer_iters/s", "h2d_bytes_per_step": 4 * p.m,
                "d2h_bytes_per_step": 4 * p.n + 64 * N_OUTER},
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
    angles, ceil(sqrt(2) n) bins): the batched solve (mof_solve_batch, of_streams
    chosen by mof_autotune) against the same problems solved one after another with
    mof_solve. Metric: outer iterations per second summed over the problems."""
    import numpy as np
    import torch
    import __graft_entry__
    __graft_entry__.build()
    from paper_2501_12497_gb300 import api, synth
    api.load()
    ws = synth.batch_form(count=48, seed=0)
    probs, params, bs, us = [], [], [], []
    for w in ws:
        p = api.mof_problem_create(w.nx, w.ny, w.nt, w.nb, w.na, w.angles, precision=api.MOF_FP32)
        probs.append(p)
        params.append(api.mof_default_params(noise_norm=w.noise_norm))
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
    # the plain form: one problem after another
    for p, prm, b, u in zip(probs, params, bs, us):
        api.mof_solve(p, prm, N_OUTER, b, u)
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    for p, prm, b, u in zip(probs, params, bs, us):
        api.mof_solve(p, prm, N_OUTER, b, u)
    torch.cuda.synchronize()
    ts = time.perf_counter() - t0
    units = len(probs) * N_OUTER
    line = {
        "metric": "mmgks_of_outer_iterations_per_s", "value": args.steps * units / tb, "unit": "outer_iters/s",
        "n_gpus": 1, "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * tb / args.steps,
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f32+f64", "data": "synthetic",
        "config": {"workload": "batch48", "problems": len(probs), "pixels_total": int(sum(w.nx * w.ny * w.nt for w in ws)),
                   "n_outer": N_OUTER, "of_streams": g, "timing": "host wall clock around synchronised batches"},
        "sequential": {"value": units / ts, "ms_per_step": 1e3 * ts, "form": "mof_solve per problem, one after another"},
        "speedup_vs_sequential": ts / (tb / args.steps),
        "gpu_launches": launches, "clocks": clk,
    }
    print(json.dumps(line), flush=True)


def run_large(args):
    """The 1024x1024x64 problem (90 angles, 1448 bins, 20 ellipses, 0.5% noise), 30
    outer iterations; inputs resident, L2 flushed before each step."""
    import numpy as np
    import torch
    import __graft_entry__
    __graft_entry__.build()
    from paper_2501_12497_gb300 import api, synth
    api.load()
    w = synth.large_form(0)
    p = api.mof_problem_create(w.nx, w.ny, w.nt, w.nb, w.na, w.angles, precision=api.MOF_FP32)
    api.mof_set_warp(p, 1 if args.warp == "round" else 0)
    prm = api.mof_default_params(noise_norm=w.noise_norm, of_streams=args.of_streams, of_scale=args.of_scale,
                                 tau=args.tau, temporal_tv=args.temporal_tv, of_pq=args.of_pq)
    b = torch.tensor(w.b.astype(np.float32), device="cuda")
    u = torch.empty(p.n, dtype=torch.float32, device="cuda")
    flush = torch.empty(L2_FLUSH_BYTES // 4, dtype=torch.float32, device="cuda")
    for _ in range(args.warmup):
        api.mof_solve(p, prm, N_OUTER, b, u)
    torch.cuda.synchronize()
    clocks = Clocks(True)
    l0 = api.mof_kernel_launches()
    ms = []
    for _ in range(args.steps):
        flush.fill_(1.0)
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record()
        rep = api.mof_solve(p, prm, N_OUTER, b, u)
        e1.record()
        e1.synchronize()
        ms.append(e0.elapsed_time(e1))
    launches = api.mof_kernel_launches() - l0
    clk = clocks.stop(0)
    rre = float(np.linalg.norm(u.cpu().numpy() - w.u_true.ravel()) / np.linalg.norm(w.u_true))
    tot = sum(ms)
    line = {
        "metric": "mmgks_of_outer_iterations_per_s", "value": args.steps * N_OUTER / (tot / 1e3), "unit": "outer_iters/s",
        "n_gpus": 1, "steps": args.steps, "warmup": args.warmup, "ms_per_step": tot / args.steps,
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f32+f64", "data": "synthetic",
        "config": {"workload": "ellipses1024x1024x64", "n": 1024, "nt": 64, "na": 90, "nb": 1448, "n_outer": N_OUTER,
                   "rre": rre, "basis_last": rep[-1]["basis"], "l2": "flushed between steps (512 MB write)",
                   "warp": args.warp},
        "gpu_launches": launches, "clocks": clk,
    }
    print(json.dumps(line), flush=True)


def run_operators(args):
    """Every operator of the C ABI applied alone at the 256x256x32 sizes (30 angles, 363
    bins), L2 flushed before each application, CUDA events around it; achieved GB/s =
    algorithmic bytes (minimum FP32 traffic of one application) / time, against the
    measured copy peak. The projector pair is reported against HBM too, although it
    is bound by FP32 and L1 work (about 36 flop per byte)."""
    import numpy as np
    import torch
    import __graft_entry__
    __graft_entry__.build()
    from paper_2501_12497_gb300 import api, synth
    api.load()
    w = synth.precision_form(0)
    p = api.mof_problem_create(w.nx, w.ny, w.nt, w.nb, w.na, w.angles, precision=api.MOF_FP32)
    n, m, ns, P = p.n, p.m, p.nx * p.ny, p.nt - 1
    dev = "cuda"
    f32 = lambda a: torch.tensor(np.asarray(a, dtype=np.float32), device=dev).reshape(-1)
    u = f32(w.u_true)
    b = f32(w.b)
    s = f32(synth.random_velocities(P, p.ny, p.nx, vmax=2.0, seed=1))
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
    ops = [
        ("H (k_project)", 4 * (n + m), lambda: api.mof_apply_A(p, u, sino)),
        ("H^T (k_backproject)", 4 * (n + m), lambda: api.mof_apply_AT(p, b, img)),
        ("fan H (k_project_fan)", 4 * (n + m) + 16 * m, lambda: api.mof_apply_A(pf, u, sino)),
        ("fan H^T (k_backproject_fan)", 4 * (n + m) + 16 * m, lambda: api.mof_apply_AT(pf, bf, img)),
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
    line = {"metric": "operator_applications", "unit": "GB/s", "config": {"workload": "ellipses256x256x32 operators",
            "l2": "flushed before each application", "reps": reps, "peak_gbs": peak}, "operators": out}
    print(json.dumps(line), flush=True)


def run_solve_of(args):
    """Solve-OF (Alg. 2) alone: one mof_solve_of call per step on the true frames of the
    256x256x32 ellipse workload (31 frame pairs, of_ell 10, 20 GKS iterations), inputs
    resident, L2 flushed before each call, CUDA events around it."""
    import numpy as np
    import torch
    import __graft_entry__
    __graft_entry__.build()
    from paper_2501_12497_gb300 import api, synth
    api.load()
    w = synth.precision_form(0)
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
            "config": {"workload": "solve_of ellipses256x256x32", "pairs": p.nt - 1, "of_ell": 10, "of_iters": 20,
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
    elif args.workload == "ellipses1024x1024x64":
        run_large(args)
    elif args.workload == "operators":
        run_operators(args)
    elif args.workload == "solve_of":
        run_solve_of(args)
    else:
        run_ours(args)


if __name__ == "__main__":
    main()
