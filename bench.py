#!/usr/bin/env python
"""Throughput of the tangent-point energy + gradient on one GB300.

Default workload: icosphere level 7 (327,680 triangles, 163,842 vertices)
deformed by seeded spherical-harmonic modes l <= 12 with amplitudes
N(0, (0.05/l)^2), seed 2; q = 6, p = 12; direct all-pairs form, FP32 pair
terms with FP64 accumulation.  One step = one pass of the hot path: the
positions are re-uploaded (device to device), the per-triangle data is
recomputed, all admitted pairs are evaluated, the per-triangle derivatives
are pulled back to the vertices and the energy is reduced.

Metric: ordered pair interactions per second (nt (nt-1) minus the ordered
pairs of triangles sharing a vertex, per evaluation) and ms per evaluation.

``--impl reference`` times the FP64 CPU oracle on a bounded sample of the
same workload on the host cores.  Under torchrun every rank runs an
independent replica (the evaluation does not shard); ``value`` is the total
over ranks.
"""

from __future__ import annotations

import argparse
import json
import os
import statistics
import subprocess
import sys
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "TP energy+grad ms/eval & pair-interactions/s at 327k tris; rel err vs FP64"
UNIT = "pair-interactions/s"
# Algorithmic FP32 work per unordered admitted pair of the energy+gradient
# pair function (both orderings, shared subexpressions once), counted from
# its expression DAG with an FMA as 2 flops: 27 FMA + 22 FMUL/FADD = 76 flops
# in 49 operations (the hi/lo cancellation correction and the reduction
# overhead not counted).
FLOPS_PER_UNORDERED_PAIR = 76
# The same count for one (target, confining triangle) pair of the confinement
# energy+gradient (one ordering, target side only): 11 FMA + 14 FMUL/FADD = 36
# flops in 25 operations (the hi/lo cancellation correction, 6 FADD, not
# counted; the -p/q factor of Gx is applied once per item, not per pair).
FLOPS_PER_CONF_PAIR = 36
# The same count for one ordered (target, source) pair of the Barnes-Hut
# near-field kernel (target side of both orderings, the target weight applied
# to the sums): 17 FMA + 20 FMUL/FADD = 54 flops in 37 operations (the hi/lo
# correction of close clusters, 6 FADD, not counted).
FLOPS_PER_NEAR_PAIR = 54
FP32_LANES_PER_SM = 128
# DRAM bytes (read + write) per launch of the dominant kernel on the default
# workload, from the one-pass ncu capture summarised in
# profiles/k_pairs_grad_traffic_sh_l7.md (null it when that kernel changes).
NCU_TRAFFIC_BYTES = 60.61e6

# packaged learned far-field models (trained by paper_2509_22110_gb300.far_train), by the tree leaf size they were trained with
FAR_MODELS = {16: os.path.join(ROOT, "paper_2509_22110_gb300", "far_model_l7.bin"),
              32: os.path.join(ROOT, "paper_2509_22110_gb300", "far_model_l7_leaf32.bin")}

WORKLOADS = {
    "sh_l7": "icosphere level 7 (327,680 triangles) with seeded SH deformation l<=12, a_lm~N(0,(0.05/l)^2), seed 2",
    "dish_l5": "icosphere level 5 (20,480 triangles) mapped to a double-walled dish, gap 0.02, jitter N(0,0.002^2)",
    "sh_l6_s2": "icosphere level 6 (81,920 triangles) with seeded SH deformation l<=12, a_lm~N(0,(0.05/l)^2), seed 2",
    "folds_l8": "icosphere level 8 (1,310,720 triangles) with 40 seeded radial folds of depth 0.1",
    "conf_l7": "unit icosphere level 7 (327,680 triangles), radial jitter N(0,0.005^2), seed 13, inside the "
               "concentric icosphere level 7 of radius 1.1 (327,680 confining triangles)",
}


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=5)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--workload", default="sh_l7", choices=sorted(WORKLOADS))
    ap.add_argument("--mode", default="direct", choices=["direct", "bh", "learned", "dual", "conf"],
                    help="bh: inner integral clustered (Barnes-Hut); dual: both integrals clustered (cluster-cluster); "
                         "conf: the confinement energy (Eq. TPConf) of the conf_l7 workload")
    ap.add_argument("--far-model", default=None,
                    help="learned far-field model file (default: the packaged model trained with --leaf)")
    ap.add_argument("--theta", type=float, default=0.25)
    ap.add_argument("--leaf", type=int, default=16, help="cluster leaf size of the tree (1-32) in the clustered modes")
    ap.add_argument("--dual-theta", type=float, default=0.25, help="opening angle of the dual form in --inloop runs")
    ap.add_argument("--quad", type=int, default=1, choices=[1, 3, 6],
                    help="quadrature points per triangle for both integrals (tp_set_quadrature)")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-accuracy", action="store_true")
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--cpu-seconds", type=float, default=15.0)
    ap.add_argument("--inloop", type=int, default=0,
                    help="run N successive evaluations under a seeded smooth displacement (step 1e-3) with the "
                         "tree rebuilt every step, comparing direct, Barnes-Hut and learned forms")
    ap.add_argument("--inloop-thetas", type=float, nargs="+", default=None,
                    help="opening angles of the clustered forms in --inloop runs (default: --theta)")
    ap.add_argument("--inloop-ref-every", type=int, default=10,
                    help="in --inloop runs, evaluate the FP64 reference every N steps and on the last")
    args = ap.parse_args()
    if args.far_model is None:
        args.far_model = FAR_MODELS.get(args.leaf, "")
    return args


def job_throughput(local_ms, ws, steps, units_per_rank, device, tdist=None):
    """Whole-job time and throughput of replicas: the timed region of every rank
    ends at a barrier, the job takes the slowest rank's time, and the value is the
    units all ranks processed divided by it.  Returns (max_ms, units per second)."""
    import torch

    t = torch.tensor([float(local_ms)], dtype=torch.float64, device=device)
    if ws > 1:
        tdist.all_reduce(t, op=tdist.ReduceOp.MAX)
    max_ms = float(t.item())
    return max_ms, ws * steps * units_per_rank / (max_ms / 1e3)


def dist_info():
    ws = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return ws, rank, local


class ClockSampler:
    """nvidia-smi sampling of SM clocks and throttle reasons during the timed region."""

    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index):
        self.gpu = gpu_index
        self.proc = None
        self.path = os.path.join("/tmp", f"tp_clocks_{os.getpid()}.csv")

    def start(self):
        try:
            self.f = open(self.path, "w")
            self.proc = subprocess.Popen(["nvidia-smi", "-i", str(self.gpu), f"--query-gpu={self.FIELDS}",
                                          "--format=csv,noheader,nounits", "-lms", "200"], stdout=self.f,
                                         stderr=subprocess.DEVNULL)
        except (OSError, FileNotFoundError):
            self.proc = None

    def stop(self):
        if self.proc is None:
            return None
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except subprocess.TimeoutExpired:
            self.proc.kill()
        self.f.close()
        sm, mx, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        with open(self.path) as f:
            for line in f:
                parts = [p.strip() for p in line.split(",")]
                if len(parts) < 9:
                    continue
                try:
                    sm.append(float(parts[1]))
                    mx.append(float(parts[2]))
                except ValueError:
                    continue
                for nm, val in zip(names, parts[5:9]):
                    if val.lower() in ("active", "1", "yes"):
                        reasons.add(nm)
        os.unlink(self.path)
        if not sm:
            return None
        return {"sm_mhz": statistics.median(sm), "sm_max_mhz": max(mx), "samples": len(sm), "reasons": sorted(reasons)}


def measured_peaks():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            return json.load(f)
    except OSError:
        return {}


def run_cpu_baseline(V, F, seconds, quad=1):
    """The FP64 oracle as it stands, on a bounded sample of target elements (triangles,
    or quadrature points with quad > 1: the oracle's expanded point set)."""
    import oracle

    oracle.build()
    nth = oracle.nthreads_default()
    rng = np.random.default_rng(123)
    if quad == 1:
        x, nu, w = oracle.tri_data(V, F)
    else:
        x, nu, w, F = oracle.quad_points(V, F, quad)
    nt = F.shape[0]
    oracle.tri_accum(V, F, rng.choice(nt, nth, replace=False), soa=(x, nu, w), nthreads=nth)  # warm the pool
    cal = rng.choice(nt, 4 * nth, replace=False)
    t0 = time.perf_counter()
    oracle.tri_accum(V, F, cal, soa=(x, nu, w), nthreads=nth)
    dt = time.perf_counter() - t0
    per = dt / len(cal)
    m = int(max(len(cal), min(nt, seconds / max(per, 1e-9))))
    m = max(nth, (m // nth) * nth)
    tris = rng.choice(nt, m, replace=False)
    t0 = time.perf_counter()
    oracle.tri_accum(V, F, tris, soa=(x, nu, w), nthreads=nth)
    dt = time.perf_counter() - t0
    val = m * (nt - 1) / dt
    return {"value": val, "unit": UNIT, "cores": nth, "kind": "oracle",
            "sample": f"dPhi/d(w,nu,x) of {m} random target elements against all {nt - 1} others "
                      f"(both orderings, FP64, {quad} point(s) per triangle), {dt:.1f} s; rate = targets*(nt-1)/s"}


def reference_arm(args):
    ws, rank, _ = dist_info()
    if rank != 0:
        return 0
    from paper_2509_22110_gb300 import meshgen
    import oracle

    V, F = meshgen.workload(args.workload)
    nt = F.shape[0]
    oracle.build()
    nth = oracle.nthreads_default()
    rng = np.random.default_rng(7)
    x, nu, w = oracle.tri_data(V, F)
    # size one step at ~per-step seconds so warmup + steps stay within a few minutes
    per_step = max(2.0, min(20.0, 120.0 / max(1, args.steps + args.warmup)))
    cal = rng.choice(nt, nth, replace=False)
    t0 = time.perf_counter()
    oracle.tri_accum(V, F, cal, soa=(x, nu, w), nthreads=nth)
    per = (time.perf_counter() - t0) / nth
    m = max(nth, int(per_step / max(per, 1e-9)) // nth * nth)
    times = []
    for s in range(args.warmup + args.steps):
        tris = rng.choice(nt, m, replace=False)
        t0 = time.perf_counter()
        oracle.tri_accum(V, F, tris, soa=(x, nu, w), nthreads=nth)
        if s >= args.warmup:
            times.append(time.perf_counter() - t0)
    tot = sum(times)
    val = args.steps * m * (nt - 1) / tot
    full_ms = (nt / m) * (tot / args.steps) * 1e3
    line = {"metric": METRIC, "value": val, "unit": UNIT, "n_gpus": ws, "steps": args.steps, "warmup": args.warmup,
            "ms_per_step": full_ms, "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
            "data": "synthetic (seeded mesh)", "impl": "reference",
            "config": {"workload": WORKLOADS[args.workload], "mode": args.mode, "q": 6, "p": 12,
                       "step": f"{m} sampled targets per step; ms_per_step extrapolated to all {nt} targets"},
            "cpu_baseline": {"value": val, "unit": UNIT, "cores": nth, "kind": "oracle",
                             "sample": f"{m} random target triangles x {nt - 1} sources per step"},
            "e2e": {"value": val, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)
    return 0


def inloop(args):
    """Successive evaluations X <- X + 1e-3 u(X) (u a seeded smooth field, max |u| = 1)."""
    import torch

    import paper_2509_22110_gb300 as tp
    from paper_2509_22110_gb300 import _tp, build as _b, meshgen

    _b.build()
    V, F = meshgen.workload(args.workload)
    dev = torch.device("cuda", 0)
    stream = torch.cuda.Stream(dev)
    ctx = tp.tp_create(0, stream.cuda_stream)
    learned = bool(args.far_model) and os.path.exists(args.far_model)
    if learned:
        tp.tp_far_model_load(ctx, args.far_model)
    Vd = torch.tensor(V, device=dev)
    Fd = torch.tensor(F, device=dev)
    tp.tp_mesh_upload(ctx, Vd, Fd)
    X = V.copy()
    thetas = args.inloop_thetas or [args.theta]
    kinds = [("bh", tp.TP_BH, 0), ("dual", tp.TP_BH_DUAL, 0)]
    if learned:
        kinds += [("learned", tp.TP_LEARNED, 0), ("learned_energy", tp.TP_LEARNED, _tp.TP_LEARNED_ENERGY)]
    modes = [(f"{name}@{args.dual_theta if m == tp.TP_BH_DUAL else th:g}", m, fl,
              args.dual_theta if m == tp.TP_BH_DUAL else th)
             for th in thetas for name, m, fl in kinds]
    modes = list({mo[0]: mo for mo in modes}.values())  # the dual form once
    times = {"direct": []}
    times.update({mo[0]: [] for mo in modes})
    errs = []
    for k in range(args.inloop):
        Vd.copy_(torch.from_numpy(X))
        tp.tp_mesh_upload(ctx, Vd, None, flags=_tp.TP_POSITIONS_ONLY)
        t_up = tp.tp_get_stats(ctx)["ms_total"]
        ref = k % args.inloop_ref_every == 0 or k == args.inloop - 1
        if ref:
            # the FP64 direct sum (FP64 pair terms and sums, the form the tests hold to the
            # oracle) is the reference; the FP32-term direct sum is timed and compared too
            gd = torch.zeros_like(Vd)
            ed = tp.tp_gradient(ctx, gd, tp.tp_params_default(prec=tp.TP_F64))
            g32 = torch.zeros_like(Vd)
            e32 = tp.tp_gradient(ctx, g32, tp.tp_params_default())
            times["direct"].append(t_up + tp.tp_get_stats(ctx)["ms_total"])
        tp.tp_tree_build(ctx, args.leaf, 30)
        t_tree = tp.tp_get_stats(ctx)["ms_total"]
        row = {"step": k}
        if ref:
            row["direct"] = {"energy_err": abs(e32 - ed) / abs(ed),
                             "grad_err": float(torch.linalg.norm(g32 - gd) / torch.linalg.norm(gd))}
        for name, m, fl, th in modes:
            g = torch.zeros_like(Vd)
            e = tp.tp_gradient(ctx, g, tp.tp_params_default(mode=m, theta=th, flags=fl))
            times[name].append(t_up + t_tree + tp.tp_get_stats(ctx)["ms_total"])
            if ref:
                row[name] = {"energy_err": abs(e - ed) / abs(ed),
                             "grad_err": float(torch.linalg.norm(g - gd) / torch.linalg.norm(gd))}
        if ref:
            row["energy"] = ed
            errs.append(row)
        X = X + 1e-3 * meshgen.smooth_displacement(X, seed=4)
    tp.tp_destroy(ctx)
    out = {"metric": "in-loop TP energy+grad ms/eval", "workload": WORKLOADS[args.workload], "nt": int(F.shape[0]),
           "steps": args.inloop, "thetas": thetas, "dual_theta": args.dual_theta,
           "ms_per_eval_median": {k: (statistics.median(v) if v else None) for k, v in times.items()},
           "reference": "direct sum in FP64 (FP64 pair terms and sums; held to the oracle by the tests), evaluated "
                        f"on every {args.inloop_ref_every}th step and the last; errors are relative (energy) and "
                        "relative L2 (gradient)",
           "errors": errs}
    print(json.dumps(out), flush=True)
    return 0


def conf_bench(args):
    """Confinement energy + gradient of a sphere inside a confining sphere (one GPU)."""
    import torch

    import paper_2509_22110_gb300 as tp
    from paper_2509_22110_gb300 import _tp, build as _b, meshgen

    _b.build()
    V, F, Vc, Fc = meshgen.sphere_in_sphere(7, 1.1, 0.005, 13)
    dev = torch.device("cuda", 0)
    stream = torch.cuda.Stream(dev)
    ctx = tp.tp_create(0, stream.cuda_stream)
    with torch.cuda.stream(stream):
        Vd = torch.tensor(V, device=dev)
        Fd = torch.tensor(F, device=dev)
        gd = torch.zeros_like(Vd)
        flush = torch.empty(256 * 1024 * 1024 // 4, dtype=torch.float32, device=dev)
    stream.synchronize()
    tp.tp_mesh_upload(ctx, Vd, Fd)
    tp.tp_conf_upload(ctx, Vc, Fc)
    prm = tp.tp_params_default()
    launches, kern_ms = [0], []

    def step():
        tp.tp_mesh_upload(ctx, Vd, None, flags=_tp.TP_POSITIONS_ONLY)
        launches[0] += tp.tp_get_stats(ctx)["kernel_launches"]
        e = tp.tp_conf_gradient(ctx, gd, prm)
        st = tp.tp_get_stats(ctx)
        launches[0] += st["kernel_launches"]
        kern_ms.append(st["ms_kernel"])
        return e, st

    for _ in range(args.warmup):
        step()
    launches[0] = 0
    kern_ms.clear()
    starts = [torch.cuda.Event(enable_timing=True) for _ in range(args.steps)]
    ends = [torch.cuda.Event(enable_timing=True) for _ in range(args.steps)]
    clocks = ClockSampler(0)
    torch.cuda.synchronize(dev)
    clocks.start()
    for k in range(args.steps):
        with torch.cuda.stream(stream):
            flush.fill_(float(k))
        starts[k].record(stream)
        energy, st = step()
        ends[k].record(stream)
    torch.cuda.synchronize(dev)
    clk = clocks.stop()
    total_ms = sum(a.elapsed_time(b) for a, b in zip(starts, ends))
    pairs = st["pairs_exact"]
    sms = torch.cuda.get_device_properties(dev).multi_processor_count
    max_mhz = float(measured_peaks().get("sm_max_mhz", 2070.0))
    peak = sms * FP32_LANES_PER_SM * 2 * max_mhz * 1e6 / 1e12
    kms = statistics.mean(kern_ms)
    achieved = FLOPS_PER_CONF_PAIR * pairs / (kms / 1e3) / 1e12
    line = {"metric": "TP confinement energy+grad pair-interactions/s (Eq. TPConf)", "value": args.steps * pairs /
            (total_ms / 1e3), "unit": UNIT, "n_gpus": 1, "steps": args.steps, "warmup": args.warmup,
            "ms_per_step": total_ms / args.steps, "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
            "dtype": "f32", "data": "synthetic (seeded meshes)",
            "config": {"workload": WORKLOADS["conf_l7"], "nt": int(F.shape[0]), "nt_conf": int(Fc.shape[0]),
                       "q": 6, "p": 12, "accumulation": "f64",
                       "l2": "flushed (256 MB write) before every timed step", "parallelism": "single GPU"},
            "energy": energy, "gpu_launches": launches[0], "clocks": clk,
            "roofline": {"bound": "alu", "achieved": achieved, "peak": peak, "unit": "TFLOP/s",
                         "frac": achieved / peak, "traffic": None, "kernel": "k_conf_grad<6>", "kernel_ms": kms,
                         "flops_per_pair": FLOPS_PER_CONF_PAIR, "pairs_per_launch": pairs,
                         "peak_basis": f"{sms} SMs x {FP32_LANES_PER_SM} FP32 lanes x 2 x {max_mhz:.0f} MHz"}}
    if not args.no_accuracy:
        g64 = torch.zeros_like(Vd)
        e64 = tp.tp_conf_gradient(ctx, g64, tp.tp_params_default(prec=tp.TP_F64))
        line["accuracy"] = {"energy_rel_err_vs_f64": abs(energy - e64) / abs(e64),
                            "grad_rel_l2_vs_f64": float(torch.linalg.norm(gd - g64) / torch.linalg.norm(g64))}
    if not args.no_e2e:
        Vh = torch.tensor(V).pin_memory()
        gh = torch.zeros(V.shape, dtype=torch.float64).pin_memory()
        tp.tp_mesh_upload(ctx, Vh, None, flags=_tp.TP_POSITIONS_ONLY)
        tp.tp_conf_gradient(ctx, gh, prm)
        torch.cuda.synchronize(dev)
        t0 = time.perf_counter()
        for _ in range(args.steps):
            tp.tp_mesh_upload(ctx, Vh, None, flags=_tp.TP_POSITIONS_ONLY)
            tp.tp_conf_gradient(ctx, gh, prm)
        torch.cuda.synchronize(dev)
        line["e2e"] = {"value": args.steps * pairs / (time.perf_counter() - t0), "unit": UNIT,
                       "h2d_bytes_per_step": int(Vh.numel() * 8), "d2h_bytes_per_step": int(gh.numel() * 8 + 8)}
    tp.tp_destroy(ctx)
    print(json.dumps(line), flush=True)
    return 0


def main():
    args = parse()
    if args.impl == "reference":
        return reference_arm(args)
    if args.inloop:
        return inloop(args)
    if args.mode == "conf":
        return conf_bench(args)
    import torch
    import torch.distributed as tdist

    ws, rank, local = dist_info()
    if ws > 1:
        tdist.init_process_group("nccl", device_id=torch.device("cuda", local))
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)

    from paper_2509_22110_gb300 import build as _b

    if rank == 0:
        _b.build()
    if ws > 1:
        tdist.barrier()
    import paper_2509_22110_gb300 as tp
    from paper_2509_22110_gb300 import _tp, meshgen

    V, F = meshgen.workload(args.workload)
    nt, nv = F.shape[0], V.shape[0]
    stream = torch.cuda.Stream(dev)
    ctx = tp.tp_create(local, stream.cuda_stream)
    mode = {"direct": tp.TP_DIRECT, "bh": tp.TP_BH, "learned": tp.TP_LEARNED, "dual": tp.TP_BH_DUAL}[args.mode]
    if mode == tp.TP_LEARNED:
        if not args.far_model or not os.path.exists(args.far_model):
            raise SystemExit("--mode learned needs --far-model (python -m paper_2509_22110_gb300.far_train)")
        tp.tp_far_model_load(ctx, args.far_model)
    prm = tp.tp_params_default(mode=mode, theta=args.theta)
    with torch.cuda.stream(stream):
        Vd = torch.tensor(V, device=dev)
        Fd = torch.tensor(F, device=dev)
        gd = torch.zeros_like(Vd)
        flush = torch.empty(256 * 1024 * 1024 // 4, dtype=torch.float32, device=dev)  # > 129 MB L2
    stream.synchronize()
    if args.quad != 1:
        tp.tp_set_quadrature(ctx, args.quad)
    tp.tp_mesh_upload(ctx, Vd, Fd)
    up_stats = tp.tp_get_stats(ctx)

    launches = [0]
    kern_ms = []
    tree_ms = []

    def step():
        tp.tp_mesh_upload(ctx, Vd, None, flags=_tp.TP_POSITIONS_ONLY)
        launches[0] += tp.tp_get_stats(ctx)["kernel_launches"]
        if mode != tp.TP_DIRECT:
            tp.tp_tree_build(ctx, args.leaf, 30)
            tst = tp.tp_get_stats(ctx)
            launches[0] += tst["kernel_launches"]
            tree_ms.append(tst["ms_total"])
        e = tp.tp_gradient(ctx, gd, prm)
        st = tp.tp_get_stats(ctx)
        launches[0] += st["kernel_launches"]
        kern_ms.append(st["ms_kernel"])
        return e, st

    for _ in range(args.warmup):
        step()
    # admitted ordered pairs of the direct sum (the direct-equivalent work of any mode)
    e_direct = tp.tp_energy(ctx, tp.tp_params_default())
    direct_pairs = tp.tp_get_stats(ctx)["pairs_exact"]
    launches[0] = 0
    kern_ms.clear()
    tree_ms.clear()

    starts = [torch.cuda.Event(enable_timing=True) for _ in range(args.steps)]
    ends = [torch.cuda.Event(enable_timing=True) for _ in range(args.steps)]
    clocks = ClockSampler(local)
    if ws > 1:
        tdist.barrier()
    torch.cuda.synchronize(dev)
    clocks.start()
    stats = None
    energy = None
    for k in range(args.steps):
        with torch.cuda.stream(stream):
            flush.fill_(float(k))  # evict the previous step's working set from L2
        starts[k].record(stream)
        energy, stats = step()
        ends[k].record(stream)
    torch.cuda.synchronize(dev)
    if ws > 1:
        tdist.barrier()
    clk = clocks.stop()
    pairs = direct_pairs
    total_ms, value = job_throughput(sum(s.elapsed_time(e) for s, e in zip(starts, ends)), ws, args.steps, pairs,
                                     dev, tdist)
    ms_step = total_ms / args.steps

    # roofline of the dominant kernel (direct: the unmasked pair kernel; Barnes-Hut and
    # learned: the near-field kernel)
    roof = None
    if mode in (tp.TP_BH, tp.TP_LEARNED) and kern_ms and stats["kernel_pairs"] > 0:
        sms = torch.cuda.get_device_properties(dev).multi_processor_count
        max_mhz = float(measured_peaks().get("sm_max_mhz", 2070.0))
        peak_tflops = sms * FP32_LANES_PER_SM * 2 * max_mhz * 1e6 / 1e12
        opairs = stats["kernel_pairs"]  # ordered (target, source) pairs of the near-field launch
        kms = statistics.mean(kern_ms)
        achieved = FLOPS_PER_NEAR_PAIR * opairs / (kms / 1e3) / 1e12
        roof = {"bound": "alu", "achieved": achieved, "peak": peak_tflops, "unit": "TFLOP/s",
                "frac": achieved / peak_tflops, "traffic": None,
                "kernel": ("k_near_blk<6> (near clusters apart from the target leaf; one run per block)"
                           if args.leaf > 16 else "k_near<6> (near clusters apart from the target leaf)"),
                "kernel_ms": kms,
                "peak_basis": f"{sms} SMs x {FP32_LANES_PER_SM} FP32 lanes x 2 x {max_mhz:.0f} MHz (max SM clock)",
                "flops_per_ordered_pair": FLOPS_PER_NEAR_PAIR, "ordered_pairs_per_launch": opairs}
        if clk and clk.get("sm_mhz"):
            roof["frac_at_sampled_clock"] = achieved / (sms * FP32_LANES_PER_SM * 2 * clk["sm_mhz"] * 1e6 / 1e12)
    if mode == tp.TP_DIRECT:
        sms = torch.cuda.get_device_properties(dev).multi_processor_count
        pk = measured_peaks()
        max_mhz = float(pk.get("sm_max_mhz", 2070.0))
        peak_tflops = sms * FP32_LANES_PER_SM * 2 * max_mhz * 1e6 / 1e12
        upairs = stats["kernel_pairs"]  # unordered real pairs evaluated by the timed launch
        kms = statistics.mean(kern_ms) if kern_ms else float("nan")
        achieved = FLOPS_PER_UNORDERED_PAIR * upairs / (kms / 1e3) / 1e12
        roof = {"bound": "alu", "achieved": achieved, "peak": peak_tflops, "unit": "TFLOP/s",
                "frac": achieved / peak_tflops, "traffic": NCU_TRAFFIC_BYTES,
                "kernel": "k_pairs_grad<6,false> (PRECISE and FAST items)", "kernel_ms": kms,
                "peak_basis": f"{sms} SMs x {FP32_LANES_PER_SM} FP32 lanes x 2 x {max_mhz:.0f} MHz (max SM clock)",
                "flops_per_unordered_pair": FLOPS_PER_UNORDERED_PAIR, "unordered_pairs_per_launch": upairs}
        if clk and clk.get("sm_mhz"):
            roof["frac_at_sampled_clock"] = achieved / (sms * FP32_LANES_PER_SM * 2 * clk["sm_mhz"] * 1e6 / 1e12)
        # measured FP32 FMA throughput (after the timed region): full occupancy, and the pair
        # kernel's own occupancy (12 warps per SM) with 2 and 4 independent packed chains per thread
        probe = {}
        for key, packed, wps, ch in (("ffma2_64warps_8chains", 1, 64, 8), ("ffma_64warps_16chains", 0, 64, 16),
                                     ("ffma2_12warps_2chains", 1, 12, 2), ("ffma2_12warps_4chains", 1, 12, 4)):
            probe[key] = _tp.tp_measure_fp32_peak(local, stream.cuda_stream, packed, wps, ch)
        best = max(probe["ffma2_64warps_8chains"], probe["ffma_64warps_16chains"])
        roof["peak_measured"] = {"tflops": probe, "frac_of_best": achieved / best if best > 0 else None}

    line = {"metric": METRIC, "value": value, "unit": UNIT, "n_gpus": ws, "steps": args.steps, "warmup": args.warmup,
            "ms_per_step": ms_step, "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f32",
            "data": "synthetic (seeded mesh)",
            "config": {"workload": WORKLOADS[args.workload], "nt": nt, "nv": nv, "mode": args.mode,
                       "quadrature_points_per_triangle": args.quad,
                       "theta": args.theta if mode != tp.TP_DIRECT else None,
                       "leaf_size": args.leaf if mode != tp.TP_DIRECT else None, "q": 6, "p": 12,
                       "accumulation": "f64", "l2": "flushed (256 MB write) before every timed step",
                       "parallelism": "replicas" if ws > 1 else "single GPU"},
            "energy": energy, "gpu_launches": launches[0], "clocks": clk, "roofline": roof,
            "ordered_pairs_per_eval": pairs}
    if mode != tp.TP_DIRECT:
        line["bh"] = {"tree_build_ms": statistics.median(tree_ms) if tree_ms else None,
                      "near_pairs": stats["pairs_exact"], "far_terms": stats["far_terms"],
                      "far_pairs_represented": stats["far_pairs"], "learned_terms": stats["learned_terms"],
                      "energy_rel_err_vs_direct_f32": abs(energy - e_direct) / abs(e_direct),
                      "note": "value counts direct-equivalent pairs (the admitted ordered pairs of the full sum)"}

    if rank == 0 and not args.no_accuracy and mode == tp.TP_DIRECT:
        # FP64 reference on the GPU (the FP64 kernel is pinned to the oracle by the tests)
        g64 = torch.zeros_like(Vd)
        e64 = tp.tp_gradient(ctx, g64, tp.tp_params_default(prec=tp.TP_F64))
        line["accuracy"] = {"energy_rel_err_vs_f64": abs(energy - e64) / abs(e64),
                            "grad_rel_l2_vs_f64": float(torch.linalg.norm(gd - g64) / torch.linalg.norm(g64)),
                            "reference": "same mesh, FP64 pair terms and accumulation (TP_F64)"}

    if not args.no_e2e:
        # end to end through the public API with pinned host buffers
        Vh = torch.tensor(V).pin_memory()
        gh = torch.zeros(V.shape, dtype=torch.float64).pin_memory()
        for _ in range(2):
            tp.tp_mesh_upload(ctx, Vh, None, flags=_tp.TP_POSITIONS_ONLY)
            tp.tp_gradient(ctx, gh, prm)
        torch.cuda.synchronize(dev)
        t0 = time.perf_counter()
        for _ in range(args.steps):
            tp.tp_mesh_upload(ctx, Vh, None, flags=_tp.TP_POSITIONS_ONLY)
            if mode != tp.TP_DIRECT:
                tp.tp_tree_build(ctx, args.leaf, 30)
            tp.tp_gradient(ctx, gh, prm)
        torch.cuda.synchronize(dev)
        t_e2e = torch.tensor([time.perf_counter() - t0], dtype=torch.float64, device=dev)
        if ws > 1:
            tdist.all_reduce(t_e2e, op=tdist.ReduceOp.MAX)
        line["e2e"] = {"value": ws * args.steps * pairs / float(t_e2e.item()), "unit": UNIT,
                       "h2d_bytes_per_step": int(Vh.numel() * 8), "d2h_bytes_per_step": int(gh.numel() * 8 + 8)}

    tp.tp_destroy(ctx)
    if rank == 0 and ws == 1 and not args.no_cpu_baseline:
        line["cpu_baseline"] = run_cpu_baseline(V, F, args.cpu_seconds, args.quad)
    if rank == 0:
        print(json.dumps(line), flush=True)
    if ws > 1:
        tdist.barrier()
        tdist.destroy_process_group()
    return 0


if __name__ == "__main__":
    sys.exit(main())
