"""Benchmark of the DBIE hot path: one step = stage a magnetogram, solve lambda at every point
(on-device Downhill Simplex, every objective evaluation a full boundary quadrature), then the
backward pass (boundary adjoint dL/dB0 and dL/dlambda for L = sum |B|^2).

Workload: Low & Lou field (n=1, m=1, l=0.3, Phi=pi/4) on a 128 x 128 boundary, points on the
64 x 64 x 32 grid x, y in 32..95, z in 1..32 (131,072 points), mixed precision.

  python bench.py [--gpus N] [--steps K] [--warmup W] [--impl reference]

Prints one JSON line.  `value` is point x pixel pair evaluations per second over the K timed
steps with inputs resident on the device; `e2e` is the same through the C ABI with host buffers
(host<->device copies inside the timed region).  --impl reference times the FP64 CPU oracle on a
bounded sample of the same workload on the host cores.
"""
from __future__ import annotations

import argparse
import ctypes
import json
import os
import statistics
import subprocess
import sys
import tempfile
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = ("point×boundary pair evals/s and solve time at ≤1e-5 rel err vs FP64, "
          "fwd+bwd")
WORKLOAD = "ll128: Low&Lou n=1 m=1 l=0.3 Phi=pi/4, 128x128 boundary, 64x64x32 points (131072)"
SMS, MUFU_PER_SM_CLK, MAX_SM_MHZ = 152, 16, 2070.0
MUFU_PER_PAIR = 7           # objective variant, one lambda per component: rsqrt + 3 x (sin, cos)
FP32_PER_SM_CLK = 124       # measured FP32 FMA-pipe rate per SM and clock (of 128 lanes)
FF_FP32_PER_PAIR = 727      # float-float objective sums: FP32 operations per point-pixel pair
DIF_INST_PER_PAIR = 153     # difference sums: thread instructions per pair (ncu, all pipes)
ISSUE_PER_SM_CLK = 128      # thread instructions issued per SM and clock (4 schedulers x 32)
FP32_PER_PAIR = 44
# DRAM bytes (dram__bytes_read.sum + dram__bytes_write.sum) of one objective launch, the first
# simplex round of this workload (131,072 queries x 16,384 pixels), from one ncu capture of the
# current kernel: 6.679 MB read (queries and boundary tiles, each read once) + 4.378 MB written
# (partial sums).
OBJ_TRAFFIC_BYTES = 6.679296e6 + 4.377600e6
THROTTLE_BITS = {0x1: "gpu_idle", 0x2: "applications_clocks_setting", 0x4: "sw_power_cap",
                 0x8: "hw_slowdown", 0x10: "sync_boost", 0x20: "sw_thermal_slowdown",
                 0x40: "hw_thermal_slowdown", 0x80: "hw_power_brake_slowdown",
                 0x100: "display_clock_setting"}


def parse_args():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=5)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--cpu-seconds", type=float, default=12.0)
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-fp64-compare", action="store_true")
    ap.add_argument("--no-large", action="store_true",
                    help="skip the batch64, ar512 and ar1024 blocks of the default line")
    ap.add_argument("--fp64-points", type=int, default=8192)
    ap.add_argument("--workload", default="ll128", choices=["ll128", "batch64"])
    ap.add_argument("--max-points", type=int, default=200_000,
                    help="batch64: upper end of the per-problem point count")
    ap.add_argument("--case", default=None,
                    choices=["exact_near_field", "float_float", "difference", "implicit_adjoint"],
                    help="a single-kernel-family case for profiling instead of the step")
    return ap.parse_args()


def dist_env():
    return (int(os.environ.get("RANK", "0")), int(os.environ.get("WORLD_SIZE", "1")),
            int(os.environ.get("LOCAL_RANK", "0")))


def workload():
    from synth import workloads
    return workloads.ll128(with_truth=False)


# ----------------------------------------------------------------------------- clocks ----
class ClockSampler:
    def __init__(self, index):
        self.index = index
        self.proc = None
        self.path = None

    def __enter__(self):
        fd, self.path = tempfile.mkstemp(suffix=".csv")
        os.close(fd)
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.index),
                 "--query-gpu=clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active",
                 "--format=csv,noheader,nounits", "-lms", "200"],
                stdout=open(self.path, "w"), stderr=subprocess.DEVNULL)
        except (FileNotFoundError, OSError):
            self.proc = None
        time.sleep(0.3)
        return self

    def __exit__(self, *exc):
        if self.proc:
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except subprocess.TimeoutExpired:
                self.proc.kill()

    def summary(self):
        sm, mx, reasons = [], [], 0
        try:
            for line in open(self.path):
                parts = [p.strip() for p in line.split(",")]
                if len(parts) < 4:
                    continue
                try:
                    s, m = float(parts[0]), float(parts[1])
                    r = int(parts[3], 16)
                except ValueError:
                    continue
                if s > 0:
                    sm.append(s)
                    mx.append(m)
                    reasons |= r & ~0x1
        except OSError:
            pass
        if not sm:
            return None
        return {"sm_mhz": statistics.median(sm), "sm_max_mhz": max(mx), "samples": len(sm),
                "reasons": [n for b, n in THROTTLE_BITS.items() if reasons & b]}


# ----------------------------------------------------------------------- our arm (GPU) ----
def run_ours(args):
    import torch
    import torch.distributed as dist

    import paper_1306_1122_gb300 as dbie
    from paper_1306_1122_gb300 import _native as N

    rank, world, local = dist_env()
    if world > 1:
        dist.init_process_group("nccl", device_id=torch.device("cuda", local))
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    w = workload()
    m = w.mag
    npix = m.nx * m.ny
    n = len(w.points)
    B0_dev = [torch.from_numpy(c).to(dev) for c in (m.Bx, m.By, m.Bz)]
    xyz_dev = torch.from_numpy(w.points).to(dev)
    opt = dbie.Options()
    flush = torch.empty(256 * 1024 * 1024 // 4, dtype=torch.float32, device=dev)  # > L2 (129 MB)
    ptr = lambda t: ctypes.c_void_p(t.data_ptr())

    stream0 = ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)
    h = N.dbie_create(m.nx, m.ny, m.x0, m.y0, m.hx, m.hy, m.dA, *(ptr(c) for c in B0_dev),
                      N.DBIE_MEM_DEVICE, stream0)
    N.dbie_autotune(h, stream0)              # launch configuration per kernel (cached per device)
    tuned = N.dbie_get_config(h)
    N.dbie_set_profiling(h, 1)

    def step(stats_out):
        stream = ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)
        # a1: stage the boundary (B0 -> tile-blocked SoA, pre-scaled) on the device
        N.dbie_set_boundary(h, *(ptr(c) for c in B0_dev), N.DBIE_MEM_DEVICE, stream)
        r = dict(B=torch.empty((n, 3), dtype=torch.float64, device=dev),
                 lam=torch.empty((n, 3), dtype=torch.float64, device=dev),
                 iters=torch.empty(n, dtype=torch.int32, device=dev),
                 status=torch.empty(n, dtype=torch.int32, device=dev),
                 f=torch.empty(n, dtype=torch.float64, device=dev),
                 g=torch.empty(n, dtype=torch.float64, device=dev))
        so = N.dbie_solve_out()
        so.B, so.lambda_, so.iters, so.status, so.f, so.g = (
            ptr(r[k]) for k in ("B", "lam", "iters", "status", "f", "g"))
        N.dbie_solve(h, n, ptr(xyz_dev), opt.c(), None, N.DBIE_MEM_DEVICE, so, stream)
        gB = 2.0 * r["B"]
        gB0 = torch.empty((m.ny, m.nx, 3), dtype=torch.float64, device=dev)
        glam = torch.empty((n, 3), dtype=torch.float64, device=dev)
        N.dbie_vjp(h, n, ptr(xyz_dev), ptr(r["lam"]), ptr(gB), opt.c(), N.DBIE_MEM_DEVICE,
                   ptr(gB0), ptr(glam), 0, stream)
        st = N.dbie_get_stats(h, True)   # synchronises: pair-sum kernel event timings
        stats_out.append(dict(queries=st.queries, rounds=st.rounds, obj_ms=st.objective_ms,
                              launches=st.launches, obj_pairs=st.objective_pairs, ties=st.ties,
                              ff_pairs=st.refine_pairs, ff_ms=st.refine_ms, difs=st.difs,
                              dif_pairs=st.dif_pairs, dif_ms=st.dif_ms))
        return r

    P = lambda a: a.ctypes.data_as(ctypes.c_void_p)
    hh = N.dbie_create(m.nx, m.ny, m.x0, m.y0, m.hx, m.hy, m.dA, P(m.Bx), P(m.By), P(m.Bz),
                       N.DBIE_MEM_HOST, None)
    N.dbie_set_config(hh, tuned)

    def step_host(h2d, d2h):
        """Same step through the C ABI with host buffers (copies inside the calls)."""
        h = hh
        N.dbie_set_boundary(h, P(m.Bx), P(m.By), P(m.Bz), N.DBIE_MEM_HOST, None)
        out = dict(B=np.empty((n, 3)), lam=np.empty((n, 3)), iters=np.empty(n, np.int32),
                   status=np.empty(n, np.int32), f=np.empty(n), g=np.empty(n))
        so = N.dbie_solve_out()
        so.B, so.lambda_, so.iters, so.status, so.f, so.g = (
            P(out[k]) for k in ("B", "lam", "iters", "status", "f", "g"))
        N.dbie_solve(h, n, P(w.points), opt.c(), None, N.DBIE_MEM_HOST, so, None)
        gB = 2.0 * out["B"]
        gB0 = np.empty((m.ny, m.nx, 3))
        glam = np.empty((n, 3))
        N.dbie_vjp(h, n, P(w.points), P(out["lam"]), P(gB), opt.c(), N.DBIE_MEM_HOST,
                   P(gB0), P(glam), 0, None)
        # inputs: B0 (3 x float32 maps), points for solve and adjoint, lambda and gB for the adjoint
        h2d.append(3 * npix * 4 + n * 12 + n * 12 + n * 24 + n * 24)
        # outputs: B, lambda, iters, status, f, g; dL/dB0; dL/dlambda
        d2h.append(n * (24 + 24 + 4 + 4 + 8 + 8) + npix * 24 + n * 24)
        return out

    # warm-up
    for _ in range(args.warmup):
        step([])
    torch.cuda.synchronize()
    if world > 1:
        dist.barrier()

    # timed region: K steps, L2 flushed before each step (outside its events)
    stats, times = [], []
    ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True))
          for _ in range(args.steps)]
    with ClockSampler(local) as clk:
        if world > 1:
            dist.barrier()
        torch.cuda.synchronize()
        wall0 = time.perf_counter()
        for k in range(args.steps):
            flush.fill_(float(k))
            ev[k][0].record()
            step(stats)
            ev[k][1].record()
        torch.cuda.synchronize()
        wall = time.perf_counter() - wall0
        if world > 1:
            dist.barrier()
    times = [a.elapsed_time(b) for a, b in ev]
    step_ms = sum(times) / len(times)
    clocks = clk.summary()

    # pair evaluations of one step: simplex queries x pixels + adjoint + dB/dlambda pass (the
    # float-float re-evaluations of certified decisions are reported apart, not counted here)
    q = stats[-1]["queries"]
    pairs_step = q * npix + 2 * n * npix
    t_tot = sum(times) / 1e3
    local_pairs = pairs_step * args.steps
    if world > 1:
        t = torch.tensor([t_tot], device=dev, dtype=torch.float64)
        dist.all_reduce(t, op=dist.ReduceOp.MAX)
        t_tot = float(t.item())
        pr = torch.tensor([float(local_pairs)], device=dev, dtype=torch.float64)
        dist.all_reduce(pr, op=dist.ReduceOp.SUM)
        total_pairs = float(pr.item())
    else:
        total_pairs = float(local_pairs)
    value = total_pairs / t_tot

    # roofline of the dominant kernel (objective pair sums), live CUDA-event timing
    obj_pairs = sum(s["obj_pairs"] for s in stats)
    obj_ms = sum(s["obj_ms"] for s in stats)
    launches = sum(s["launches"] for s in stats)
    achieved = obj_pairs * MUFU_PER_PAIR / (obj_ms / 1e3) / 1e12 if obj_ms > 0 else None
    peak = SMS * MUFU_PER_SM_CLK * MAX_SM_MHZ * 1e6 / 1e12
    rounds = stats[-1]["rounds"]

    # e2e through the C ABI with host buffers
    h2d, d2h = [], []
    e2e_times = []
    step_host(h2d, d2h)   # warm
    for _ in range(max(1, min(args.steps, 3))):
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        step_host(h2d, d2h)
        e2e_times.append(time.perf_counter() - t0)
    e2e_value = pairs_step / statistics.mean(e2e_times) * (world if world > 1 else 1)
    N.dbie_destroy(hh)
    N.dbie_destroy(h)

    line = {
        "metric": METRIC, "value": value, "unit": "pair-evals/s", "n_gpus": world,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": step_ms,
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f32+f64",
        "data": "synthetic (seeded Low & Lou field, no observational data)",
        "config": {"workload": WORKLOAD, "points": n, "boundary": [m.ny, m.nx],
                   "precision": "mixed (FP32 pair terms, float-float sums, FP64 near field "
                                "z<=2px, FP64 objective and simplex; near-tied simplex "
                                "decisions re-evaluated in the float-float form, or as "
                                "differences from a float-float reference value)",
                   "fwd_bwd": "solve (Nelder-Mead, tol 1e-6, max 50 it) + adjoint + dL/dlambda",
                   "pairs_per_step": pairs_step, "simplex_rounds": rounds,
                   "objective_evals": q, "l2": "flushed before each step (256 MB write)",
                   "parallelism": f"replicas x{world} (points are independent)",
                   "launch_configs": tuned},
        "solve_ms": step_ms,
        "roofline_float_float": {
            "bound": "alu", "pipe": "FP32 (FMA)", "kernel": "g1_ff_kernel (float-float "
            "re-evaluation of near-tied simplex decisions)",
            "achieved": (stats[-1]["ff_pairs"] * FF_FP32_PER_PAIR /
                         (sum(s["ff_ms"] for s in stats) / args.steps / 1e3) / 1e12)
            if any(s["ff_ms"] for s in stats) else None,
            "peak": SMS * FP32_PER_SM_CLK * MAX_SM_MHZ * 1e6 / 1e12, "unit": "T FP32-op/s",
            "per_pair": {"fp32": FF_FP32_PER_PAIR, "mufu": 1},
            "peak_source": "152 SMs x 124 FP32 ops/clk/SM (measured per-clock rate) x 2070 MHz"},
        "roofline_difference": {
            "bound": "alu", "pipe": "instruction issue (FP32 FMA 68 %, MUFU 16 % of it)",
            "kernel": "g1_dif_kernel (difference sums of near-tied values from a float-float "
            "reference)",
            "achieved": (stats[-1]["dif_pairs"] * DIF_INST_PER_PAIR /
                         (sum(s["dif_ms"] for s in stats) / args.steps / 1e3) / 1e12)
            if any(s["dif_ms"] for s in stats) else None,
            "peak": SMS * ISSUE_PER_SM_CLK * MAX_SM_MHZ * 1e6 / 1e12, "unit": "T thread-inst/s",
            "per_pair": {"thread_instructions": DIF_INST_PER_PAIR, "mufu": 7},
            "peak_source": "152 SMs x 4 schedulers x 32 lanes x 2070 MHz"},
        "certified_decisions": {
            "near_ties_per_step": stats[-1]["ties"],
            "near_tie_frac_of_evals": stats[-1]["ties"] / max(1, q),
            "float_float_pairs_per_step": stats[-1]["ff_pairs"],
            "float_float_ms_per_step": sum(s["ff_ms"] for s in stats) / args.steps,
            "difference_values_per_step": stats[-1]["difs"],
            "difference_pairs_per_step": stats[-1]["dif_pairs"],
            "difference_ms_per_step": sum(s["dif_ms"] for s in stats) / args.steps,
            "difference_pairs_per_s": (stats[-1]["dif_pairs"] /
                                       (sum(s["dif_ms"] for s in stats) / args.steps / 1e3))
            if any(s["dif_ms"] for s in stats) else None,
            "band": 0.02, "band_difference": 0.02},
        "roofline": {"bound": "alu", "pipe": "MUFU (rsqrt, sin, cos)",
                     "kernel": "g1_kernel<float, objective, per-component lambda>",
                     "achieved": achieved, "peak": peak, "unit": "T MUFU-op/s",
                     "frac": (achieved / peak) if achieved else None,
                     "traffic": OBJ_TRAFFIC_BYTES if WORKLOAD.startswith("ll128") else None,
                     "traffic_launch": "first simplex round: 131072 queries x 16384 pixels",
                     "per_pair": {"mufu": MUFU_PER_PAIR, "fp32": FP32_PER_PAIR},
                     "kernel_ms_per_step": obj_ms / args.steps,
                     "kernel_launches_per_step": launches / args.steps,
                     "peak_source": "152 SMs x 16 MUFU ops/clk/SM (measured per-clock rate) x "
                                    "2070 MHz max SM clock"},
        "e2e": {"value": e2e_value, "unit": "pair-evals/s",
                "h2d_bytes_per_step": int(h2d[-1]), "d2h_bytes_per_step": int(d2h[-1])},
        # per step: staging 5 (checks, FP32/FP64 and float-float tiles), solve 4 + 9 per round
        # (plan, pair sums, near field, simplex step; float-float plan and pair sums, difference
        # plan and pair sums, simplex step), backward 9 (pack, plan, adjoint, finalize; pack,
        # plan, pair sums, near field, finalize)
        "gpu_launches": int(args.steps * (5 + 4 + 9 * rounds + 9)),
        "clocks": clocks,
        "wall_s": wall,
    }
    for key in ("roofline_float_float", "roofline_difference"):
        rf = line[key]
        rf["frac"] = rf["achieved"] / rf["peak"] if rf["achieved"] else None
    if rank == 0 and world == 1 and not args.no_fp64_compare:
        line["fp64_form"] = fp64_compare(w, args.fp64_points, dev)
        line["quasi_newton"] = method_compare(w, dev)
        line["backward_through_search"] = backward_compare(w, dev)
        line["quadrature_rules"] = quadrature_compare(w, dev)
        if not args.no_large:
            line["batch64"] = batch64_block(dev)
            line["ar512"] = ar512_block(dev)
            line["ar1024"] = ar1024_block(dev)
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        line["cpu_baseline"] = cpu_baseline(w, args.cpu_seconds)
    if world > 1:
        dist.destroy_process_group()
    if rank == 0:
        print(json.dumps(line))


def fp64_compare(w, npts, dev):
    """Time-to-solution of the mixed form, with certified decisions (the default) and without,
    against the plain FP64 GPU form on the same points (a seeded subsample), all running the full
    lambda search; the mixed results' accuracy against the FP64 one: B at the mixed lambda and,
    where both took the same simplex steps, lambda itself; the near ties that certification sent
    to float-float re-evaluation and their cost."""
    import torch

    import paper_1306_1122_gb300 as dbie
    idx = np.sort(np.random.default_rng(7).choice(len(w.points), min(npts, len(w.points)),
                                                  replace=False))
    pts = torch.from_numpy(w.points[idx]).to(dev)
    f = dbie.DBIEField.from_magnetogram(w.mag, device=dev)
    f.autotune()
    out = {}
    for name, prec, cert in (("mixed", 0, 0.02), ("mixed_uncertified", 0, 0.0), ("fp64", 1, 0.0)):
        opt = dbie.Options(precision=prec, certify=cert)
        f.solve(pts[:256], opt)                  # warm: graph capture, buffers
        torch.cuda.synchronize()
        f.set_profiling(True)
        f.stats(reset=True)
        t0 = time.perf_counter()
        r = f.solve(pts, opt, codes=50)
        torch.cuda.synchronize()
        out[name] = (time.perf_counter() - t0, r, f.stats(reset=True))
        f.set_profiling(False)
    td, rd, _ = out["fp64"]
    res = {"points": int(len(idx)), "fp64_s": td,
           "fp64_iters_mean": float(rd["iters"].float().mean())}
    for name in ("mixed", "mixed_uncertified"):
        tm, rm, st = out[name]
        same = (rm["codes"] == rd["codes"]).all(dim=1).cpu().numpy()
        lam_rel = ((rm["lam"] - rd["lam"]).abs() /
                   torch.clamp(rd["lam"].abs(), min=1.0 / (w.mag.nx * w.mag.hx))).max(dim=1).values
        lam_rel = lam_rel.cpu().numpy()
        res[name] = {
            "solve_s": tm, "speedup_vs_fp64": td / tm,
            "iters_mean": float(rm["iters"].float().mean()),
            "same_step_sequence_frac": float(same.mean()),
            "lambda_rel_err_where_same": ({
                "median": float(np.median(lam_rel[same])),
                "p99": float(np.percentile(lam_rel[same], 99)),
                "max": float(lam_rel[same].max()),
                "frac_le_1e-4": float((lam_rel[same] <= 1e-4).mean())} if same.any() else None),
            "near_ties": int(st["ties"]), "objective_evals": int(st["queries"]),
            "near_tie_frac_of_evals": st["ties"] / max(1, st["queries"]),
            "float_float_pairs": st["refine_pairs"], "float_float_ms": st["refine_ms"],
            "difference_values": st["difs"], "difference_ms": st["dif_ms"],
            "objective_ms": st["objective_ms"]}
    tm, rm, _ = out["mixed"]
    res["mixed"]["B_vs_fp64_at_mixed_lambda"] = b_error_stats(f, w.mag, w.points[idx],
                                                              rm["lam"].cpu().numpy(), dev)
    f.close()
    return res


def method_compare(w, dev):
    """The paper's Downhill Simplex against the gradient-based quasi-Newton search (not in the
    paper) on all points of the workload, mixed precision: solve time, objective evaluations and
    the final Phi = f + g."""
    import torch

    import paper_1306_1122_gb300 as dbie
    pts = torch.from_numpy(w.points).to(dev)
    f = dbie.DBIEField.from_magnetogram(w.mag, device=dev)
    f.autotune()
    out = {}
    for name, method in (("simplex", 0), ("quasi_newton", 1)):
        opt = dbie.Options(method=method)
        f.solve(pts[:256], opt)
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        r = f.solve(pts, opt)
        torch.cuda.synchronize()
        dt = time.perf_counter() - t0
        phi = (r["f"] + r["g"]).cpu().numpy()
        out[name] = {"solve_s": dt, "evals_mean": float(r["nfev"].float().mean()),
                     "phi_median": float(np.median(phi)), "phi_mean": float(phi.mean()),
                     "f_median": float(r["f"].median()), "g_median": float(r["g"].median())}
    f.close()
    out["speedup"] = out["simplex"]["solve_s"] / out["quasi_newton"]["solve_s"]
    return out


def backward_compare(w, dev):
    """Cost of the gradient through the lambda search (Hessian pass + seven-weight adjoint) next to
    the fixed-lambda adjoint, and of the noise variance, on all points of the workload at the
    simplex's lambda (mixed precision, tuned launch shapes, CUDA events, 3 repeats, minimum);
    both adjoints also with the exact near field."""
    import torch

    import paper_1306_1122_gb300 as dbie
    pts = torch.from_numpy(w.points).to(dev)
    f = dbie.DBIEField.from_magnetogram(w.mag, device=dev)
    f.autotune()
    r = f.solve(pts)
    gB = 2.0 * r["B"]
    n, npix = len(w.points), w.mag.nx * w.mag.ny

    def timed(fn):
        fn()
        best = 1e30
        for _ in range(3):
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record()
            fn()
            e1.record()
            torch.cuda.synchronize()
            best = min(best, e0.elapsed_time(e1))
        return best

    t_fixed = timed(lambda: f.vjp(pts, r["lam"], gB, glam=False))
    t_impl = timed(lambda: f.vjp_implicit(pts, r["lam"], gB))
    t_nv = timed(lambda: f.noise_var(pts, r["lam"], sigma0=10.0))
    _, _, fl = f.vjp_implicit(pts, r["lam"], gB)
    # the same two adjoints with the exact near field (its transpose for the points at z <= 2 px)
    f.set_quadrature(dbie.QUAD_PIXEL_EXACT)
    t_fixed_x = timed(lambda: f.vjp(pts, r["lam"], gB, glam=False))
    t_impl_x = timed(lambda: f.vjp_implicit(pts, r["lam"], gB))
    f.close()
    return {"points": n, "pixels": npix, "fixed_lambda_adjoint_ms": t_fixed,
            "implicit_adjoint_ms": t_impl, "noise_variance_ms": t_nv,
            "implicit_pair_evals_per_s": 2.0 * n * npix / (t_impl / 1e3),
            "points_without_positive_definite_hessian": int(fl.sum().item()),
            "exact_near_field": {"fixed_lambda_adjoint_ms": t_fixed_x,
                                 "implicit_adjoint_ms": t_impl_x}}


def quadrature_compare(w, dev):
    """The paper's pixel-centre rule (Eq. 16, 128 x 128 pixels) against the same rule with the
    exact near-field integration of the lambda = 0 kernel (points with z <= 2 px) and against
    Eq. 15's nine-node elements with 4 x 4 Gauss points (the same field on the 129 x 129 node grid
    at the same scale), each with the full simplex search on the same 131,072 physical points:
    solve time, pair evaluations per second and agreement with the analytic field (vector
    correlation C_vec and 1 - normalised vector error), over all points and over the two layers
    nearest the boundary (z <= 2 px, where the rules differ)."""
    import torch

    import paper_1306_1122_gb300 as dbie
    from synth import workloads

    def agreement(B, b):
        c_vec = float(np.sum(B * b) / np.sqrt(np.sum(B * B) * np.sum(b * b)))
        e_n = float(1.0 - np.sum(np.linalg.norm(B - b, axis=1)) / np.sum(np.linalg.norm(b, axis=1)))
        return c_vec, e_n

    out = {}
    lam_ref = None       # the pixel-centre search's lambda, to compare the rules at equal lambda
    ll128 = workloads.ll128(with_truth=True)
    for name, wk, order in (("pixel_centres", ll128, 0),
                            ("pixel_exact_near_field", ll128, dbie.QUAD_PIXEL_EXACT),
                            ("elements_g4", workloads.ll129_nodes(), 4)):
        f = dbie.DBIEField.from_magnetogram(wk.mag, device=dev)
        if order:
            f.set_quadrature(order)
        f.autotune()
        pts = torch.from_numpy(wk.points).to(dev)
        f.solve(pts[:256])
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        r = f.solve(pts)
        torch.cuda.synchronize()
        dt = time.perf_counter() - t0
        nq = wk.mag.npix if order <= 0 else ((wk.mag.nx - 1) // 2 * order) ** 2
        B = r["B"].cpu().numpy()
        c_vec, e_n = agreement(B, wk.truth)
        near = wk.points[:, 2] <= 2.0 * wk.mag.hx
        c_near, e_near = agreement(B[near], wk.truth[near])
        if lam_ref is None:
            lam_ref = r["lam"].to(torch.float32)
        Bq = f.eval(pts, lam_ref)["B"].cpu().numpy()
        _, e_same = agreement(Bq[near], wk.truth[near])
        out[name] = {"solve_s": dt, "quadrature_points": int(nq),
                     "pair_evals_per_s": float(r["nfev"].sum()) * nq / dt,
                     "C_vec": c_vec, "E_n": e_n, "C_vec_z_le_2": c_near, "E_n_z_le_2": e_near,
                     "E_n_z_le_2_at_pixel_centre_lambda": e_same}
        f.close()
    return out


# ------------------------------------------------------------- larger workloads ----
def abs_sum_scale(mag, pts, lam, dev, chunk=128):
    """S_i = | (sum_k |a_ik(lambda_p)| |B0_p,k|)_p |: the absolute-value sum of each point's
    quadrature (the scale below which B is dominated by cancellation); FP32 torch, measurement
    only."""
    import torch
    jj, ii = np.mgrid[0:mag.ny, 0:mag.nx]
    px = torch.from_numpy((mag.x0 + ii * mag.hx).ravel().astype(np.float32)).to(dev)
    py = torch.from_numpy((mag.y0 + jj * mag.hy).ravel().astype(np.float32)).to(dev)
    b = [torch.from_numpy(np.abs(c).ravel().astype(np.float32)).to(dev) * (mag.dA / (2 * np.pi))
         for c in (mag.Bx, mag.By, mag.Bz)]
    P = torch.as_tensor(pts, dtype=torch.float32).to(dev)
    L = torch.as_tensor(lam, dtype=torch.float32).to(dev).abs()
    out = torch.empty(len(P), 3, dtype=torch.float64, device=dev)
    for a in range(0, len(P), chunk):
        p = P[a:a + chunk]
        r = torch.sqrt((p[:, 0:1] - px) ** 2 + (p[:, 1:2] - py) ** 2 + p[:, 2:3] ** 2)
        for c in range(3):
            th = L[a:a + chunk, c:c + 1] * r
            u = (th * torch.sin(th) + torch.cos(th)).abs()
            out[a:a + chunk, c] = (p[:, 2:3] * u / r ** 3 * b[c]).sum(1).double()
    return out.norm(dim=1).cpu().numpy()


def b_error_stats(field, mag, pts, lam, dev):
    """Mixed B against the FP64 GPU form at the same lambda (float32) on a point sample: relative
    error distribution, the fraction above 1e-5, and that fraction split at S_i = 10 |B_i|
    (S_i the absolute-value sum: above it the sum is dominated by cancellation)."""
    import torch

    import paper_1306_1122_gb300 as dbie
    P = torch.as_tensor(pts).to(dev)
    Lm = torch.as_tensor(lam).to(dev, torch.float32)
    Bm = field.eval(P, Lm)["B"]
    Bd = field.eval(P, Lm, options=dbie.Options(precision=1))["B"]
    nB = Bd.norm(dim=1)
    rel = ((Bm - Bd).norm(dim=1) / nB).cpu().numpy()
    S = abs_sum_scale(mag, pts, lam, dev)
    canc = S > 10 * nB.cpu().numpy()
    big = rel > 1e-5
    return {"points": int(len(rel)), "median": float(np.median(rel)),
            "p99": float(np.percentile(rel, 99)), "max": float(rel.max()),
            "frac_gt_1e-5": float(big.mean()),
            "frac_cancellation_dominated": float(canc.mean()),
            "frac_gt_1e-5_where_S_le_10B": float(big[~canc].mean()) if (~canc).any() else 0.0,
            "max_where_S_le_10B": float(rel[~canc].max()) if (~canc).any() else 0.0,
            "max_err_over_S": float(((Bm - Bd).norm(dim=1).cpu().numpy() / S).max())}


def batch64_block(dev, sub_per_problem=128):
    """Config 4 in the default line: 64 magnetograms (sides 32..256), 1k..200k points each, one
    full mixed-precision simplex solve of all 6.35 M points through the batched persistent path
    (timed once after a warm-up solve of a subsample), the objective kernel's MUFU roofline from
    CUDA events inside the solve's graphs, the per-problem iteration histogram; then the batched
    mixed and batched FP64 forms on the same stated subsample (sub_per_problem points of every
    problem), and the mixed B error against the FP64 form on that subsample."""
    import torch

    import paper_1306_1122_gb300 as dbie
    from synth import workloads
    probs = workloads.batch64()
    fields = [dbie.DBIEField.from_magnetogram(w.mag, device=dev) for w in probs]
    fields[0].autotune()
    pts = [torch.from_numpy(w.points).to(dev) for w in probs]
    rng = np.random.default_rng(64)
    sub = [np.sort(rng.choice(len(w.points), min(sub_per_problem, len(w.points)), replace=False))
           for w in probs]
    sub_pts = [p[torch.from_numpy(i).to(dev)] for p, i in zip(pts, sub)]
    dbie.solve_batched(fields, sub_pts)                 # warm: kernels, buffers
    torch.cuda.synchronize()
    fields[0].set_profiling(True)
    fields[0].stats(reset=True)
    t0 = time.perf_counter()
    outs = dbie.solve_batched(fields, pts)
    torch.cuda.synchronize()
    t_full = time.perf_counter() - t0
    st = fields[0].stats(reset=True)
    fields[0].set_profiling(False)
    nfev = [int(o["nfev"].sum()) for o in outs]
    pairs = float(sum(nf * w.mag.npix for nf, w in zip(nfev, probs)))
    iters = torch.cat([o["iters"] for o in outs]).cpu().numpy()
    hist = np.bincount(np.minimum(iters, 50), minlength=51)
    mufu = st["objective_pairs"] * 7 / (st["objective_ms"] / 1e3) / 1e12 if st["objective_ms"] else None
    peak = SMS * MUFU_PER_SM_CLK * MAX_SM_MHZ * 1e6 / 1e12
    sub_t = {}
    for name, prec in (("mixed", 0), ("fp64", 1)):
        opt = dbie.Options(precision=prec)
        dbie.solve_batched(fields, [q[:8] for q in sub_pts], opt)
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        r = dbie.solve_batched(fields, sub_pts, opt)
        torch.cuda.synchronize()
        sub_t[name] = (time.perf_counter() - t0, r)
    errs = [b_error_stats(f, w.mag, w.points[i], o["lam"].cpu().numpy()[i], dev)
            for f, w, i, o in zip(fields[:8], probs[:8], sub, outs[:8])]
    for f in fields:
        f.close()
    n_sub = int(sum(len(i) for i in sub))
    return {"workload": "batch64: 64 magnetograms, sides U{32..256}, 1-4 patches, 1k..200k "
                        "points each, z in [1, 64] (seed 4)",
            "points": int(sum(len(w.points) for w in probs)),
            "solve_s": t_full, "pair_evals": pairs, "pair_evals_per_s": pairs / t_full,
            "roofline": {"bound": "alu", "kernel": "g1_kernel objective (batched)",
                         "achieved": mufu, "peak": peak, "unit": "T MUFU-op/s",
                         "frac": mufu / peak if mufu else None,
                         "kernel_s": st["objective_ms"] / 1e3},
            "iters_hist": hist.tolist(), "iters_mean": float(iters.mean()),
            "subsample": {"points": n_sub, "per_problem": sub_per_problem,
                          "mixed_s": sub_t["mixed"][0], "fp64_s": sub_t["fp64"][0],
                          "speedup_mixed_over_fp64": sub_t["fp64"][0] / sub_t["mixed"][0]},
            "B_vs_fp64_first8_problems": {
                k: (max(e[k] for e in errs) if k.startswith("max") else
                    float(np.mean([e[k] for e in errs]))) for k in errs[0]}}


def ar512_block(dev, max_iter=10, sub=8192):
    """Config 3: the 512 x 256 active region, 2,097,152 points (256 x 128 x 64 volume); a short
    simplex search (max_iter stated) over the whole volume, then the backward pass over the 32^3
    sub-volume at the searched lambda: dB/dlambda (fused pass) and dL/dB0, dL/dlambda for
    L = sum |B|^2 (fixed-lambda adjoint), and the gradient through the search (implicit adjoint);
    the mixed B error against the FP64 form on a point sample."""
    import torch

    import paper_1306_1122_gb300 as dbie
    from synth import workloads
    w = workloads.ar512()
    f = dbie.DBIEField.from_magnetogram(w.mag, device=dev)
    f.autotune()
    pts = torch.from_numpy(w.points).to(dev)
    opt = dbie.Options(max_iter=max_iter)
    f.solve(pts[:4096], opt)
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    r = f.solve(pts, opt)
    torch.cuda.synchronize()
    t_solve = time.perf_counter() - t0
    pairs = float(r["nfev"].sum()) * w.mag.npix
    sv = torch.from_numpy(workloads.ar512_backward_subvolume(w)).to(dev)
    xs, lam = pts[sv], r["lam"][sv]
    gB = 2.0 * r["B"][sv]

    def timed(fn):
        fn()
        torch.cuda.synchronize()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record()
        fn()
        e1.record()
        torch.cuda.synchronize()
        return e0.elapsed_time(e1)
    t_dl = timed(lambda: f.eval(xs, lam.float(), dlam=True))
    t_vjp = timed(lambda: f.vjp(xs, lam, gB))
    t_impl = timed(lambda: f.vjp_implicit(xs, lam, gB))
    idx = np.sort(np.random.default_rng(512).choice(len(w.points), sub, replace=False))
    err = b_error_stats(f, w.mag, w.points[idx], r["lam"].cpu().numpy()[idx], dev)
    f.close()
    nsv = len(sv)
    return {"workload": "ar512: 512x256 active region (seed 1306), 256x128x64 points (2097152); "
                        "backward over the 32^3 sub-volume",
            "search": {"max_iter": max_iter, "solve_s": t_solve, "pair_evals": pairs,
                       "pair_evals_per_s": pairs / t_solve,
                       "iters_mean": float(r["iters"].float().mean())},
            "backward_subvolume": {"points": nsv, "dBdlambda_ms": t_dl, "fixed_lambda_adjoint_ms": t_vjp,
                                   "implicit_adjoint_ms": t_impl,
                                   "adjoint_pair_evals_per_s": nsv * w.mag.npix / (t_vjp / 1e3)},
            "B_vs_fp64": err}


def ar1024_block(dev, sub=20000, oracle_points=48):
    """Config 5: 1024 x 512 active region (seed 5), 6,291,456 points (4,194,304 field-line samples
    + the 128^3 grid).  Forward (B and dB/dlambda, one fused pass) and the fixed-lambda adjoint
    dL/dB0 for L = sum |B|^2, at a seeded per-point lambda ~ U[0, 0.05]^3 (stated: no search at
    this size), with the value kernel's MUFU roofline from CUDA events; the mixed B error against
    the FP64 GPU form on a 20k-point sample, and against the FP64 CPU oracle on a smaller one."""
    import torch

    import oracle
    import paper_1306_1122_gb300 as dbie
    from synth import workloads
    w = workloads.ar1024()
    m = w.mag
    f = dbie.DBIEField.from_magnetogram(m, device=dev)
    f.autotune()
    n = len(w.points)
    pts = torch.from_numpy(w.points).to(dev)
    lam = torch.from_numpy(np.random.default_rng(1024).uniform(0, 0.05, (n, 3)).astype(np.float32)).to(dev)
    f.eval(pts[:65536], lam[:65536], dlam=True)
    torch.cuda.synchronize()
    f.set_profiling(True)
    f.stats(reset=True)
    e = [torch.cuda.Event(enable_timing=True) for _ in range(3)]
    e[0].record()
    r = f.eval(pts, lam, dlam=True)
    e[1].record()
    f.vjp(pts, lam.double(), 2.0 * r["B"], glam=False)
    e[2].record()
    torch.cuda.synchronize()
    st = f.stats(reset=True)
    f.set_profiling(False)
    t_fwd, t_bwd = e[0].elapsed_time(e[1]) / 1e3, e[1].elapsed_time(e[2]) / 1e3
    pairs = float(n) * m.npix
    mufu = st["pair_evals"] * 7 / (st["kernel_ms"] / 1e3) / 1e12 if st["kernel_ms"] else None
    peak = SMS * MUFU_PER_SM_CLK * MAX_SM_MHZ * 1e6 / 1e12
    rng = np.random.default_rng(5)
    idx = np.sort(rng.choice(n, sub, replace=False))
    lam_np = lam.cpu().numpy()
    err = b_error_stats(f, m, w.points[idx], lam_np[idx], dev)
    oi = idx[:oracle_points]
    bd = oracle.Boundary(oracle.Grid(m.nx, m.ny, m.x0, m.y0, m.hx, m.hy, m.dA), m.Bx, m.By, m.Bz)
    Bo, _, _ = oracle.field(bd, w.points[oi].astype(np.float64), lam_np[oi].astype(np.float64))
    Bg = r["B"][torch.from_numpy(oi).to(dev)].cpu().numpy()
    orel = np.linalg.norm(Bg - Bo, axis=1) / np.linalg.norm(Bo, axis=1)
    f.close()
    return {"workload": "ar1024: 1024x512 active region (seed 5), 4194304 field-line samples + "
                        "128^3 grid (6291456 points), lambda ~ U[0, 0.05]^3 seeded",
            "points": n, "pixels": int(m.npix), "pairs_per_pass": pairs,
            "forward_s": t_fwd, "forward_pair_evals_per_s": pairs / t_fwd,
            "adjoint_s": t_bwd, "adjoint_pair_evals_per_s": pairs / t_bwd,
            "roofline_forward_kernel": {"bound": "alu", "achieved": mufu, "peak": peak,
                                        "unit": "T MUFU-op/s", "frac": mufu / peak if mufu else None},
            "B_vs_fp64": err,
            "B_vs_oracle": {"points": int(len(oi)), "max_rel": float(orel.max()),
                            "median_rel": float(np.median(orel))}}


# --------------------------------------------------------------------- oracle (CPU) ----
def oracle_sample_step(w, npts, seed, nthreads):
    """One sample step of the oracle: lambda search at npts points of the workload plus the
    adjoint for those points.  Returns (pair evaluations, seconds)."""
    import oracle
    m = w.mag
    bd = oracle.Boundary(oracle.Grid(m.nx, m.ny, m.x0, m.y0, m.hx, m.hy, m.dA), m.Bx, m.By, m.Bz)
    idx = np.random.default_rng(seed).choice(len(w.points), npts, replace=False)
    pts = w.points[idx].astype(np.float64)
    t0 = time.perf_counter()
    r = oracle.solve(bd, pts, oracle.Options(), nthreads=nthreads)
    oracle.vjp(bd, pts, r["lam"], 2 * r["B"], nthreads=nthreads)
    oracle.field(bd, pts, r["lam"], nthreads=nthreads)
    dt = time.perf_counter() - t0
    npix = m.nx * m.ny
    pairs = (int(r["nfev"].sum()) + len(pts)) * npix + 2 * len(pts) * npix
    return pairs, dt


def cpu_baseline(w, seconds):
    import oracle
    oracle.build()
    cores = os.cpu_count() or 1
    p, dt = oracle_sample_step(w, max(cores, 16), 1, cores)
    npts = int(max(cores, min(len(w.points), max(cores, 16) * seconds / max(dt, 1e-3))))
    p, dt = oracle_sample_step(w, npts, 2, cores)
    return {"value": p / dt, "unit": "pair-evals/s", "cores": cores, "kind": "oracle",
            "sample": f"{npts} random points of the workload: full lambda search + adjoint + "
                      f"dB/dlambda pass, {dt:.1f} s on {cores} host threads"}


def run_reference(args):
    rank, world, _ = dist_env()
    if rank != 0:
        return
    import oracle
    oracle.build()
    w = workload()
    cores = os.cpu_count() or 1
    _, dt = oracle_sample_step(w, max(cores, 16), 0, cores)
    per_step = max(10.0, 150.0 / max(1, args.steps + args.warmup))
    npts = int(max(cores, min(len(w.points), max(cores, 16) * per_step / max(dt, 1e-3))))
    for k in range(args.warmup):
        oracle_sample_step(w, max(cores, 8), 100 + k, cores)
    tot_p, tot_t = 0, 0.0
    for k in range(args.steps):
        p, dt = oracle_sample_step(w, npts, 200 + k, cores)
        tot_p += p
        tot_t += dt
    value = tot_p / tot_t
    sample = (f"{npts} random points of the workload per step: full lambda search + adjoint + "
              f"dB/dlambda pass, FP64 oracle on {cores} host threads")
    print(json.dumps({
        "impl": "reference", "metric": METRIC, "value": value, "unit": "pair-evals/s",
        "n_gpus": world, "steps": args.steps, "warmup": args.warmup,
        "ms_per_step": tot_t / args.steps * 1e3, "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": "f64", "data": "synthetic (seeded Low & Lou field)",
        "config": {"workload": WORKLOAD, "sample_points_per_step": npts},
        "cpu_baseline": {"value": value, "unit": "pair-evals/s", "cores": cores,
                         "kind": "oracle", "sample": sample},
        "e2e": {"value": value, "unit": "pair-evals/s", "h2d_bytes_per_step": 0,
                "d2h_bytes_per_step": 0}}))


def run_batched(args):
    """64 magnetograms of uneven size (sides 32..256, 1-4 flux patches) each with 1k..max points,
    solved together: one persistent pair-sum launch per simplex round for all problems."""
    import torch

    import paper_1306_1122_gb300 as dbie
    from synth import workloads
    torch.cuda.set_device(0)
    probs = workloads.batch64(max_points=args.max_points)
    fields = [dbie.DBIEField.from_magnetogram(w.mag) for w in probs]
    fields[0].autotune()
    tuned = dbie._native.dbie_get_config(fields[0].handle)
    pts = [torch.from_numpy(w.points).cuda() for w in probs]
    opt = dbie.Options()
    for _ in range(args.warmup):
        dbie.solve_batched(fields, pts, opt)
    torch.cuda.synchronize()
    times, outs = [], None
    with ClockSampler(0) as clk:
        for _ in range(args.steps):
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record()
            outs = dbie.solve_batched(fields, pts, opt)
            e1.record()
            torch.cuda.synchronize()
            times.append(e0.elapsed_time(e1) / 1e3)
    nfev = [int(o["nfev"].sum()) for o in outs]
    pairs = sum(nf * w.mag.npix for nf, w in zip(nfev, probs))
    iters = [float(o["iters"].float().mean()) for o in outs]
    print(json.dumps({
        "metric": METRIC, "value": pairs / statistics.mean(times), "unit": "pair-evals/s",
        "n_gpus": 1, "steps": args.steps, "warmup": args.warmup,
        "ms_per_step": statistics.mean(times) * 1e3, "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "f32+f64",
        "data": "synthetic (seeded active regions, seed 4)",
        "config": {"workload": "batch64: 64 magnetograms, sides U{32..256}, 1-4 patches, "
                               f"1k..{args.max_points} points each, z in [1, 64]",
                   "points": int(sum(len(w.points) for w in probs)),
                   "pixels": [int(w.mag.npix) for w in probs], "launch_configs": tuned},
        "per_problem": {"points": [len(w.points) for w in probs], "iters_mean": iters,
                        "objective_evals": nfev},
        "clocks": clk.summary()}))
    for f in fields:
        f.close()


def run_case_exact_near_field():
    """Profiling case of the exact near field on the ll128 workload: field evaluation and the
    fixed-lambda adjoint of all 131,072 points at lambda_p = 0.02 with the correction (twice, to
    warm up) and once more of each on the pixel-centre rule; prints the CUDA-event times."""
    import torch

    import paper_1306_1122_gb300 as dbie
    from synth import workloads
    w = workloads.ll128()
    f = dbie.DBIEField.from_magnetogram(w.mag)
    pts = torch.from_numpy(w.points).cuda()
    lam = torch.full((len(w.points), 3), 0.02, device="cuda")
    gB = torch.ones((len(w.points), 3), dtype=torch.float64, device="cuda")
    out = {}
    for name, order in (("exact_near_field", dbie.QUAD_PIXEL_EXACT), ("pixel_centres", 0)):
        f.set_quadrature(order)
        for _ in range(2):
            f.eval(pts, lam)
            f.vjp(pts, lam.double(), gB, glam=False)
        ev = [torch.cuda.Event(enable_timing=True) for _ in range(3)]
        ev[0].record()
        f.eval(pts, lam)
        ev[1].record()
        f.vjp(pts, lam.double(), gB, glam=False)
        ev[2].record()
        torch.cuda.synchronize()
        out[name] = {"eval_ms": ev[0].elapsed_time(ev[1]), "vjp_ms": ev[1].elapsed_time(ev[2])}
    f.close()
    print(json.dumps({"case": "exact_near_field", "workload": "ll128 (131072 points, 128^2 pixels)",
                      **out}))


def run_case_float_float():
    """Profiling case of the float-float pair sums (the certified decisions' re-evaluation
    kernel): objective sums of 8,192 ll128 points at lambda_p = 0.02 in DBIE_PREC_FLOAT_FLOAT,
    twice to warm up and once timed; prints the CUDA-event time and pair rate."""
    import torch

    import paper_1306_1122_gb300 as dbie
    from synth import workloads
    w = workloads.ll128(with_truth=False)
    f = dbie.DBIEField.from_magnetogram(w.mag)
    pts = torch.from_numpy(w.points[::16].copy()).cuda()
    lam = torch.full((len(pts), 3), 0.02, device="cuda")
    opt = dbie.Options(precision=dbie._native.DBIE_PREC_FLOAT_FLOAT)
    for _ in range(2):
        f.eval(pts, lam, grad=True, options=opt)
    ev = [torch.cuda.Event(enable_timing=True) for _ in range(2)]
    ev[0].record()
    f.eval(pts, lam, grad=True, options=opt)
    ev[1].record()
    torch.cuda.synchronize()
    ms = ev[0].elapsed_time(ev[1])
    f.close()
    print(json.dumps({"case": "float_float", "workload": "ll128 objective sums, 8192 points x "
                      "16384 pixels, float-float form", "ms": ms,
                      "pairs_per_s": len(pts) * w.mag.npix / (ms / 1e3)}))


def run_case_difference():
    """Profiling case of the difference sums (the second level of the certified decisions):
    8,192 ll128 points x 16,384 pixels, reference lambda_p = 0.02, lambda a seeded step of up to
    1e-3 from it (the near-tie regime), with error bounds; twice to warm up and once timed;
    prints the CUDA-event time and pair rate."""
    import numpy as np
    import torch

    import paper_1306_1122_gb300 as dbie
    from synth import workloads
    w = workloads.ll128(with_truth=False)
    f = dbie.DBIEField.from_magnetogram(w.mag)
    pts = torch.from_numpy(w.points[::16].copy()).cuda()
    lam0 = torch.full((len(pts), 3), 0.02, dtype=torch.float64, device="cuda")
    step = np.random.default_rng(16).uniform(-1e-3, 1e-3, (len(pts), 3))
    lam = lam0 + torch.from_numpy(step).cuda()
    for _ in range(2):
        f.eval_difference(pts, lam, lam0)
    ev = [torch.cuda.Event(enable_timing=True) for _ in range(2)]
    ev[0].record()
    f.eval_difference(pts, lam, lam0)
    ev[1].record()
    torch.cuda.synchronize()
    ms = ev[0].elapsed_time(ev[1])
    f.close()
    print(json.dumps({"case": "difference", "workload": "ll128 difference sums, 8192 points x "
                      "16384 pixels, steps up to 1e-3 from lambda_p = 0.02", "ms": ms,
                      "pairs_per_s": len(pts) * w.mag.npix / (ms / 1e3)}))


def run_case_implicit_adjoint():
    """Profiling case of the gradient through the lambda search on the ll128 workload: tuned
    launch shapes, the simplex search of all 131,072 points, then dbie_vjp_implicit at its lambda
    (once to warm up, three times timed with CUDA events, minimum) and once more inside the NVTX
    range "implicit_adjoint" (for ncu --nvtx-include); prints the times and the chosen launch
    configurations."""
    import torch

    import paper_1306_1122_gb300 as dbie
    from synth import workloads
    w = workloads.ll128(with_truth=False)
    f = dbie.DBIEField.from_magnetogram(w.mag)
    cfg = f.autotune()
    pts = torch.from_numpy(w.points).cuda()
    r = f.solve(pts)
    gB = 2.0 * r["B"]

    def timed(fn):
        fn()
        best = 1e30
        for _ in range(3):
            ev = [torch.cuda.Event(enable_timing=True) for _ in range(2)]
            ev[0].record()
            fn()
            ev[1].record()
            torch.cuda.synchronize()
            best = min(best, ev[0].elapsed_time(ev[1]))
        return best

    out = {"implicit_adjoint_ms": timed(lambda: f.vjp_implicit(pts, r["lam"], gB)),
           "hessian_ms": timed(lambda: f.hessian(pts, r["lam"])),
           "fixed_lambda_adjoint_ms": timed(lambda: f.vjp(pts, r["lam"], gB, glam=False))}
    torch.cuda.nvtx.range_push("implicit_adjoint")
    f.vjp_implicit(pts, r["lam"], gB)
    torch.cuda.nvtx.range_pop()
    torch.cuda.synchronize()
    f.close()
    print(json.dumps({"case": "implicit_adjoint", "workload": "ll128 (131072 points, 128^2 "
                      "pixels), simplex lambda", "config": [int(x) for x in cfg], **out}))


def main():
    args = parse_args()
    if args.case == "exact_near_field":
        run_case_exact_near_field()
    elif args.case == "float_float":
        run_case_float_float()
    elif args.case == "difference":
        run_case_difference()
    elif args.case == "implicit_adjoint":
        run_case_implicit_adjoint()
    elif args.impl == "reference":
        run_reference(args)
    elif args.workload == "batch64":
        run_batched(args)
    else:
        run_ours(args)


if __name__ == "__main__":
    main()
