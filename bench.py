#!/usr/bin/env python3
"""Benchmark of the separable tensor-operator solve on one GB300 (or N replicas).

Workload (the paper's 4D spline reconstruction at its scale, Sec. 5): unknowns
160x160x160x8 (32.8M), cubic B-spline collocation factors on a 240^3 x 12
jittered sample grid, lambda = 1e-3 second-difference regulariser, synthetic
smooth ground truth plus N(0, 0.01^2) noise.  A step is one full solve of
(A^T A + lambda R) x = A^T b to a true relative residual of 1e-6 (A^T b, the
CG iterations and the FP64 true-residual check), with b resident in HBM.

Prints one JSON line (rank 0).  ``--impl reference`` times the CPU FP64 oracle
on the machine's host cores instead (bounded sample, extrapolated; see below).

``value`` times plain solves (one graph launch each: the CG passes loop on the
device).  The roofline's sweep time comes from a profiled solve run right after
each timed one: the same solve with every CG sweep bracketed by CUDA events on
the solve's stream (one graph pass per launch, the host reading the events).
``variants`` (after the plain timing, same workload unless stated):
  separable_pcg_s16 / _s32  the separable tensor-inverse preconditioner;
  separable_banded_pcg_*    the same with 7-band truncated factors (one fused sweep),
                            at s = 16, 32 and at the plan's corner-model default;
  tmg_pcg                   the two-grid tensor multigrid cycle (Sec. 4.2, Fig. 3),
                            every default, with its coarse CG steps and lambda_max;
  jacobi_pcg                point Jacobi, M = diag(K);
  bf16_ir                   the bfloat16 mixed-precision form (tensor-core sweep,
                            double-float refinement), autotuned, with its sweep's
                            roofline and, in the oracle leg, its error against the
                            FP64 oracle on the 40x40x40x8 instance of the generator;
  batched                   64 uneven instances in one graph launch (plain,
                            separable and Jacobi), against one solve after another;
  scattered                 the paper's own 4D problem at its size: a 128x128x128x16
                            grid (33.5M unknowns) with 9.06M random off-grid samples,
                            FP32 and FP64 CG through sample space;
  learned                   the network initial guess trained on solver pairs,
                            evaluated on held-out 160x160x160x8 instances.
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

METRIC = "time-to-solution at 1e-6 rel. residual, 33M-unknown 4D; mode-sweep HBM GB/s"
SHAPE = (160, 160, 160, 8)
SEED = 2
LAM = 1e-3
RTOL = 1e-6
# DRAM bytes (read + written) of one launch of the CG sweep kernel at this workload,
# counted by ncu (dram__bytes_read.sum + dram__bytes_write.sum) on the current kernel;
# to be re-measured (or set to None) whenever that kernel changes.
K2_TRAFFIC_BYTES = 510_850_000
SUBVOL = (40, 40, 40, 8)  # iteration-count probe for the oracle arm (same generator)
BF16_INNER = 3e-2  # inner relative tolerance of the bfloat16 refinement variant
WORKLOAD = ("bspline4d: unknowns 160x160x160x8 (32.8M) FP32, cubic B-spline factors on 240x240x240x12 "
            "jittered samples, lambda 1e-3, noise 0.01, CG to true rel. residual 1e-6")


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=5)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="tca", choices=["tca", "reference"])
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-learned", action="store_true", help="skip the learned-initial-guess variant (training)")
    ap.add_argument("--no-variants", action="store_true", help="plain solve only (launch lists under a profiler)")
    ap.add_argument("--small", action="store_true", help="quick 64x64x64x8 run (not a bench line)")
    ap.add_argument("--shape", default=None, help="sweep cases: tensor shape n1,n2,n3,n4 (profiling runs)")
    ap.add_argument("--train-instances", type=int, default=100, help="learned case: training instances (64^3 x 4)")
    ap.add_argument("--rhs-per-instance", type=int, default=20, help="learned case: right-hand sides per instance")
    ap.add_argument("--epochs", type=float, default=2.0, help="learned case: passes over the training pairs")
    ap.add_argument("--case", default=None, choices=["normal", "gram", "collocation", "cgsweep", "bf16sweep", "dense", "batched", "learned",
                             "netfwd", "scattered", "pcg", "tmg", "shear"],
                    help="time one sweep kernel alone on the full-size tensors (profiling runs; no bench line)")
    return ap.parse_args()


def run_case(args, local):
    """One kernel alone on the full-size tensors: small device footprint for profilers."""
    import torch

    from paper_1001_5460_gb300 import synth, tca

    device = torch.device("cuda", local)
    torch.cuda.set_device(device)
    if args.case == "dense":
        # Dense 96x96 Gram factor on mode 1 of a 96x96x96x24 tensor: tensor-core mode product.
        shape = (96, 96, 96, 24)
        rng = np.random.default_rng(SEED)
        facs = [synth.Factor("dense", int(1.5 * n), n, a=synth.dense_gaussian_factor(int(1.5 * n), n, rng))
                for n in shape]
        dplan = tca.Plan(shape, facs, lam=LAM, precision="f32")
        x = torch.randn(shape, dtype=torch.float32, device=device)
        y = torch.empty_like(x)
        fn = lambda: dplan.apply_mode(0, tca.OP_GRAM, shape, x, y)
        for _ in range(args.warmup):
            fn()
        torch.cuda.synchronize()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record()
        for _ in range(args.steps):
            fn()
        e1.record()
        torch.cuda.synchronize()
        ms = e0.elapsed_time(e1) / max(args.steps, 1)
        n = x.numel()
        print(json.dumps({"case": "dense", "ms": round(ms, 5), "gbs": round(2 * n * 4 / ms / 1e6, 1),
                          "useful_tflops": round(2 * n * 96 / ms / 1e9, 2),
                          "issued_tflops_3xtf32": round(3 * 2 * n * 96 / ms / 1e9, 2)}), flush=True)
        return
    if args.case == "batched":
        run_batched(args, device)
        return
    if args.case == "scattered":
        run_scattered(args, device)
        return
    if args.case == "learned":
        run_learned(args, device)
        return
    if args.case == "netfwd":
        # The network's forward pass alone on a full-size tensor (random weights and input).
        shape = (64, 64, 64, 8) if args.small else SHAPE
        net = tca.Net(synth.net_init_params(1))
        u = torch.randn(shape, dtype=torch.float32, device=device)
        y = torch.empty_like(u)
        for _ in range(args.warmup):
            net.forward(u, y)
        torch.cuda.synchronize()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record()
        for _ in range(args.steps):
            net.forward(u, y)
        e1.record()
        torch.cuda.synchronize()
        ms = e0.elapsed_time(e1) / max(args.steps, 1)
        flops = 2 * u.numel() * 27 * (32 + 32 * 32 * 2 + 32)
        print(json.dumps({"case": "netfwd", "shape": list(shape), "ms": round(ms, 4),
                          "tflops": round(flops / ms / 1e9, 2)}), flush=True)
        return
    shape = tuple(int(v) for v in args.shape.split(",")) if args.shape else SHAPE
    inst = synth.instance_bspline(shape, seed=SEED, lam=LAM, with_truth=False)
    plan = tca.plan_from_instance(inst, precision="f32")
    x = torch.randn(shape, dtype=torch.float32, device=device)
    N = x.numel()
    if args.case == "bf16sweep":
        # A few iterations of the bfloat16 inner CG: the tensor-core CG sweep in its solve context.
        bplan = tca.plan_from_instance(inst, precision="bf16_ir")
        b = torch.randn(inst.sample_shape, dtype=torch.float32, device=device)
        for _ in range(args.warmup + args.steps):
            st, info = bplan.solve(b, x, rtol=1e-30, inner_rtol=1e-30, max_iter=4, raise_on_error=False,
                                   profile=True)
        ms = info["sweep_ms"] / max(info["sweep_launches"], 1)
        print(json.dumps({"case": args.case, "ms": round(ms, 5), "gbs": round(4 * N * 2 / ms / 1e6, 1)}), flush=True)
        return
    if args.case == "pcg":
        # Profiled solves (one graph launch per pass, so profilers see every kernel) of the
        # bench workload preconditioned by the banded separable inverse at the default shift.
        inst_t, plan_t, b = make_problem(shape, SEED, device)
        xz = torch.zeros(shape, dtype=torch.float32, device=device)
        for _ in range(args.warmup + args.steps):
            st, info = plan_t.solve(b, xz, rtol=RTOL, precond="separable_banded", profile=True)
        torch.cuda.synchronize()
        print(json.dumps({"case": args.case, "status": int(st), "cg_iters": info["iters"],
                          "rel_res_true": info["rel_res_true"], "shift": plan_t.precond_default_shift()}), flush=True)
        return
    if args.case == "shear":
        # Shears of the 160^3 x 8 volume (FP32), each kernel alone (inputs larger than L2): along
        # mode 1 driven by mode 2 (linear and cubic), along mode 2 driven by mode 1, and along the
        # fastest mode driven by mode 1 (slope tan 15 degrees about the centre of mode 2).
        xs = torch.randn(shape, dtype=torch.float32, device=device)
        ys = torch.empty_like(xs)
        N = xs.numel()
        c = (shape[1] - 1) / 2.0
        for (ma, mb), kind in (((0, 1), "linear"), ((0, 1), "cubic"), ((1, 0), "cubic"), ((3, 0), "cubic")):
            for _ in range(3):
                tca.apply_shear(xs, ys, ma, mb, 0.2679, c, kind=kind)
            torch.cuda.synchronize()
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            reps = max(5, args.steps)
            e0.record()
            for _ in range(reps):
                tca.apply_shear(xs, ys, ma, mb, 0.2679, c, kind=kind)
            e1.record()
            torch.cuda.synchronize()
            ms = e0.elapsed_time(e1) / reps
            gbs = 8 * N / ms / 1e6
            peaks, _ = measured_peaks()
            print(json.dumps({"case": "shear", "modes": [ma, mb], "kind": kind, "ms": round(ms, 5),
                              "gbs": round(gbs, 1), "frac_of_measured_hbm": round(gbs / peaks["hbm_gbs"], 4)}),
                  flush=True)
        return
    if args.case == "tmg":
        # Solves of the bench workload preconditioned by the two-grid tensor multigrid cycle,
        # timed with CUDA events on the solve's stream: every default, then more smoothing
        # steps and a looser coarse solve.
        inst_t, plan_t, b = make_problem(shape, SEED, device)
        xz = torch.zeros(shape, dtype=torch.float32, device=device)
        for nu, crt in ((0, 0.0), (2, 0.1), (3, 0.5), (4, 0.3)):
            ms, info = timed_solve(plan_t, b, xz, max(1, args.steps), torch.cuda.current_stream(), precond="tmg",
                                   tmg_nu=nu, tmg_coarse_rtol=crt)
            st_t = plan_t.tmg_info()
            print(json.dumps({"case": args.case, "nu": nu or 3, "coarse_rtol": crt or 0.3, "ms": round(ms, 3),
                              "cg_iters": info["iters"], "rel_res_true": info["rel_res_true"],
                              "coarse_cg_iters": st_t["coarse_iters"], "lambda_max": st_t["lambda_max"]}),
                  flush=True)
            if args.steps <= 1:
                break
        return
    if args.case == "cgsweep":
        # A few CG iterations on random data: the CG-mode fused sweep in its solve context.
        b = torch.randn(inst.sample_shape, dtype=torch.float32, device=device)
        for _ in range(args.warmup + args.steps):
            st, info = plan.solve(b, x, rtol=1e-30, max_iter=4, raise_on_error=False, profile=True)
        ms = info["sweep_ms"] / max(info["sweep_launches"], 1)
        print(json.dumps({"case": args.case, "ms": round(ms, 5), "gbs": round(4 * N * 4 / ms / 1e6, 1)}), flush=True)
        return
    if args.case == "normal":
        y = torch.empty_like(x)
        fn, nbytes = (lambda: plan.apply_normal(x, y)), 2 * N * 4
    elif args.case == "gram":
        y = torch.empty_like(x)
        fn, nbytes = (lambda: plan.apply_mode(0, tca.OP_GRAM, shape, x, y)), 2 * N * 4
    else:
        y = torch.empty((inst.factors[0].m,) + shape[1:], dtype=torch.float32, device=device)
        fn, nbytes = (lambda: plan.apply_mode(0, tca.OP_FACTOR, shape, x, y)), (N + y.numel()) * 4
    for _ in range(args.warmup):
        fn()
    torch.cuda.synchronize()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record()
    for _ in range(args.steps):
        fn()
    e1.record()
    torch.cuda.synchronize()
    ms = e0.elapsed_time(e1) / max(args.steps, 1)
    print(json.dumps({"case": args.case, "ms": round(ms, 5), "gbs": round(nbytes / ms / 1e6, 1)}), flush=True)


BATCH = 64


def run_batched(args, device, emit=True):
    """64 uneven instances (3D/4D, n_k ~ U[24,96], n_4 in {1,4,8}, half dense, half B-spline,
    lambda log-uniform in [1e-4,1e-2]) solved to 1e-6 in one graph launch, against the same
    instances solved one after another with tca_solve."""
    import torch

    from paper_1001_5460_gb300 import synth, tca

    insts = [synth.instance_batched(i) for i in range(BATCH)]
    plans = [tca.plan_from_instance(inst, precision="f32") for inst in insts]
    bs, xs = [], []
    for inst, plan in zip(insts, plans):
        xt = torch.from_numpy(inst.x_true).to(device)
        b = torch.from_numpy(np.ascontiguousarray(inst.noise, dtype=np.float32)).to(device)
        ax = torch.empty_like(b)
        plan.apply(xt, ax)
        bs.append(ax + b)
        xs.append(torch.empty(inst.shape, dtype=torch.float32, device=device))
    torch.cuda.synchronize()
    unknowns = sum(int(np.prod(i.shape)) for i in insts)
    t0 = time.perf_counter()
    st, infos = tca.solve_batched(plans, bs, xs, rtol=RTOL, max_iter=20000)
    torch.cuda.synchronize()
    first_s = time.perf_counter() - t0  # graph capture + solve
    for _ in range(max(args.warmup - 1, 0)):
        tca.solve_batched(plans, bs, xs, rtol=RTOL, max_iter=20000)
    torch.cuda.synchronize()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    launches0 = tca.kernel_launches()
    e0.record()
    for _ in range(args.steps):
        st, infos = tca.solve_batched(plans, bs, xs, rtol=RTOL, max_iter=20000)
    e1.record()
    torch.cuda.synchronize()
    batched_ms = e0.elapsed_time(e1) / max(args.steps, 1)
    launches = (tca.kernel_launches() - launches0) // max(args.steps, 1)
    # The autotuner's SM share for this batch (each candidate solved twice), then the tuned batch.
    t0 = time.perf_counter()
    share = tca.autotune_batched(plans, bs, xs, rtol=RTOL, max_iter=20000)
    tune_s = time.perf_counter() - t0
    tca.solve_batched(plans, bs, xs, rtol=RTOL, max_iter=20000)
    torch.cuda.synchronize()
    e0.record()
    for _ in range(args.steps):
        st_t, t_infos = tca.solve_batched(plans, bs, xs, rtol=RTOL, max_iter=20000)
    e1.record()
    torch.cuda.synchronize()
    tuned_ms = e0.elapsed_time(e1) / max(args.steps, 1)
    # The same instances, one tca_solve each (each plan's own cached iteration graph).
    for plan, b, x in zip(plans, bs, xs):
        plan.solve(b, x, rtol=RTOL, max_iter=20000)
    torch.cuda.synchronize()
    e0.record()
    seq_infos = []
    for _ in range(args.steps):
        seq_infos = [plan.solve(b, x, rtol=RTOL, max_iter=20000)[1] for plan, b, x in zip(plans, bs, xs)]
    e1.record()
    torch.cuda.synchronize()
    seq_ms = e0.elapsed_time(e1) / max(args.steps, 1)
    # The same batch with the separable tensor-inverse preconditioner.
    tca.solve_batched(plans, bs, xs, rtol=RTOL, max_iter=20000, precond="separable")
    torch.cuda.synchronize()
    e0.record()
    for _ in range(args.steps):
        st_pc, pc_infos = tca.solve_batched(plans, bs, xs, rtol=RTOL, max_iter=20000, precond="separable")
    e1.record()
    torch.cuda.synchronize()
    pc_batched_ms = e0.elapsed_time(e1) / max(args.steps, 1)
    pc_iters = [i["iters"] for i in pc_infos]
    iters = [i["iters"] for i in infos]
    slowest = sorted(range(BATCH), key=lambda k: -seq_infos[k]["seconds"])[:4]
    # Per-instance rate of each solve alone: one CG iteration moves at least ten
    # FP32 vector passes (sweep: r, p_old in, p, q out; update: r, q in, r out;
    # x += alpha p: x, p in, x out), 40 B per unknown, times its iterations.
    inst_gbs = sorted(40.0 * float(np.prod(insts[k].shape)) * seq_infos[k]["iters"] / seq_infos[k]["seconds"] / 1e9
                      for k in range(BATCH))
    # The same batch with the point-Jacobi preconditioner.
    tca.solve_batched(plans, bs, xs, rtol=RTOL, max_iter=20000, precond="jacobi")
    torch.cuda.synchronize()
    e0.record()
    for _ in range(args.steps):
        st_j, j_infos = tca.solve_batched(plans, bs, xs, rtol=RTOL, max_iter=20000, precond="jacobi")
    e1.record()
    torch.cuda.synchronize()
    j_batched_ms = e0.elapsed_time(e1) / max(args.steps, 1)
    j_iters = [i["iters"] for i in j_infos]
    out = {
        "case": "batched", "instances": BATCH, "unknowns": unknowns, "status": int(st),
        "batched_ms": round(batched_ms, 3), "sequential_ms": round(seq_ms, 3),
        "autotuned": {"sm_share": f"1/{share}", "batched_ms": round(tuned_ms, 3), "status": int(st_t),
                      "tune_s": round(tune_s, 2),
                      "rel_res_true_max": max(i["rel_res_true"] for i in t_infos)},
        "speedup": round(seq_ms / batched_ms, 3), "first_call_s": round(first_s, 3),
        "iters_min": min(iters), "iters_median": int(statistics.median(iters)), "iters_max": max(iters),
        "iters_total": int(sum(iters)), "restarts": int(sum(i["refinements"] for i in infos)),
        "rel_res_true_max": max(i["rel_res_true"] for i in infos),
        "seq_iters_total": int(sum(i["iters"] for i in seq_infos)),
        "gpu_launches_lower_bound": int(launches),
        "separable_pcg": {"status": int(st_pc), "batched_ms": round(pc_batched_ms, 3),
                          "iters_median": int(statistics.median(pc_iters)), "iters_max": max(pc_iters),
                          "iters_total": int(sum(pc_iters)),
                          "rel_res_true_max": max(i["rel_res_true"] for i in pc_infos)},
        "jacobi_pcg": {"status": int(st_j), "batched_ms": round(j_batched_ms, 3),
                       "iters_median": int(statistics.median(j_iters)), "iters_max": max(j_iters),
                       "iters_total": int(sum(j_iters)),
                       "rel_res_true_max": max(i["rel_res_true"] for i in j_infos)},
        "per_instance_gbs_alone": {"min": round(inst_gbs[0], 1), "median": round(statistics.median(inst_gbs), 1),
                                   "max": round(inst_gbs[-1], 1), "bytes_per_unknown_iter": 40},
        "slowest_alone": [{"shape": list(insts[k].shape), "kind": insts[k].factors[0].kind,
                           "iters": seq_infos[k]["iters"], "ms": round(1e3 * seq_infos[k]["seconds"], 2)}
                          for k in slowest],
    }
    # Whole-batch rate in the same 40 B per unknown and iteration convention.
    out["batched_gbs"] = round(40.0 * sum(float(np.prod(i.shape)) * f["iters"] for i, f in zip(insts, infos))
                               / batched_ms / 1e6, 1)
    for pl in plans:
        pl.close()
    if emit:
        print(json.dumps(out), flush=True)
    return out


# The paper's 4D spline reconstruction (Sec. 5): a 128 x 128 x 128 x 16 grid and about 9M
# scattered measurements, solved there in under 60 minutes on a multicore PC (tolerance not stated).
SCATTER_SHAPE = (128, 128, 128, 16)
SCATTER_FRACTION = 0.27  # samples per unknown: 9.06M samples on that grid


def run_scattered(args, device, emit=True, shape=None, precisions=("f32", "f64")):
    """Scattered-sample reconstruction: samples at random off-grid positions (0.27 per unknown, as
    in the paper's 4D problem), cubic B-spline rows per mode, CG to 1e-6 through sample space
    (gather + scatter-add per iteration), for each precision (FP32: FP32 iterations with the
    FP64 operator for A^T b and the true residual; FP64 throughout)."""
    from paper_1001_5460_gb300 import synth

    shape = tuple(shape or SCATTER_SHAPE)
    m = int(SCATTER_FRACTION * int(np.prod(shape)))
    t0 = time.perf_counter()
    inst = synth.instance_scattered(shape, m, seed=SEED, lam=LAM)
    gen_s = time.perf_counter() - t0
    out = {"case": "scattered", "shape": list(shape), "samples": m, "generate_s": round(gen_s, 1),
           "paper_context": "Sec. 5: 128x128x128x16 unknowns, about 9M measurements, under 60 min on a "
                            "multicore PC with 2 GB (tolerance not stated)",
           "what": "rows = Kronecker products of per-sample cubic B-spline rows; K applied through sample "
                   "space (samples grouped by grid tile; gather of 4^d taps from a shared-memory image of "
                   "the tile's region, scatter-add into it with shared-memory atomics, one global atomic "
                   "per region cell) + separable regulariser"}
    b64 = None
    for prec in precisions:
        out[prec], b64 = _scattered_one(args, device, inst, shape, m, prec, b64)
    if emit:
        print(json.dumps(out), flush=True)
    return out


def _scattered_one(args, device, inst, shape, m, prec, b64):
    """One precision of the scattered case: the timed solves, then the normal operator, the
    gather and the scatter-add alone (CUDA events), on the solution."""
    import torch

    from paper_1001_5460_gb300 import tca

    dt = torch.float64 if prec == "f64" else torch.float32
    t0 = time.perf_counter()
    plan = tca.ScatteredPlan(inst.shape, inst.col0, inst.w, lam=inst.lam, precision=prec)
    plan_s = time.perf_counter() - t0
    if b64 is None:
        # b = A x_true + noise by the FP64 gather (a plan of its own when this one is FP32)
        gen = plan if prec == "f64" else tca.ScatteredPlan(inst.shape, inst.col0, inst.w, lam=inst.lam)
        b64 = torch.empty(m, dtype=torch.float64, device=device)
        gen.apply(torch.from_numpy(inst.x_true).to(device), b64)
        b64 += torch.from_numpy(inst.noise).to(device)
        if gen is not plan:
            gen.close()
    b = b64.to(dt)
    x = torch.zeros(shape, dtype=dt, device=device)
    s = torch.cuda.current_stream()
    ms, info = timed_solve(plan, b, x, max(1, min(args.steps, 3)), s, max_iter=20000)
    y = torch.empty_like(x)
    ys = torch.empty(m, dtype=dt, device=device)

    def timed(fn, reps=10):
        for _ in range(3):
            fn()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(s)
        for _ in range(reps):
            fn()
        e1.record(s)
        torch.cuda.synchronize()
        return e0.elapsed_time(e1) / reps

    k_ms = timed(lambda: plan.apply_normal(x, y))
    g_ms = timed(lambda: plan.apply(x, ys))
    t_ms = timed(lambda: plan.apply_T(ys, y))
    taps = m * 4 ** len(shape)
    plan.close()
    return {"precision": prec, "ms": round(ms, 3), "cg_iters": info["iters"], "restarts": info["refinements"],
            "rel_res_true": info["rel_res_true"], "plan_s": round(plan_s, 3),
            "normal_apply_ms": round(k_ms, 4), "gather_ms": round(g_ms, 4), "scatter_ms": round(t_ms, 4),
            "taps_per_s_G": round(2 * taps / k_ms / 1e6, 1)}, b64


TRAIN_SHAPE = (64, 64, 64, 4)


def run_learned(args, device, emit=True):
    """Learned initial guess: train the network on (A^T b, x) pairs that the plain solver produces on
    64x64x64x4 B-spline instances, then solve held-out 160x160x160x8 instances from x0 = s Net(A^T b / s)
    and compare with plain CG from zero at the same true relative residual (1e-6)."""
    import torch

    from paper_1001_5460_gb300 import synth, tca

    t_start = time.perf_counter()
    rng = np.random.default_rng(77)
    # Pool of smooth fields (unit RMS); each training right-hand side is A x + noise with a field
    # from the pool, flipped along random modes, so that every pair is distinct.
    pool = [torch.from_numpy(synth.smooth_random_field(TRAIN_SHAPE, 4.0, rng)).to(device) for _ in range(16)]
    us, ts = [], []
    gen_iters = 0
    for k in range(args.train_instances):
        inst = synth.instance_bspline(TRAIN_SHAPE, seed=5000 + k, with_truth=False)
        plan = tca.plan_from_instance(inst)
        b = torch.empty(inst.sample_shape, dtype=torch.float32, device=device)
        u = torch.empty(TRAIN_SHAPE, dtype=torch.float32, device=device)
        for j in range(args.rhs_per_instance):
            xt = pool[int(rng.integers(len(pool)))]
            dims = [d for d in range(3) if rng.random() < 0.5]
            if dims:
                xt = torch.flip(xt, dims)
            plan.apply(xt.contiguous(), b)
            b += 0.01 * torch.randn(b.shape, device=device)
            plan.apply_T(b, u)
            x = torch.empty_like(u)
            _, info = plan.solve(b, x, rtol=RTOL)
            gen_iters += info["iters"]
            s = torch.sqrt(torch.mean(u.double() ** 2)).float()
            us.append((u / s).contiguous())
            ts.append((x / s).contiguous())
        plan.close()
    torch.cuda.synchronize()
    t_gen = time.perf_counter() - t_start
    npairs = len(us)
    net = tca.Net(synth.net_init_params(7))
    steps = int(args.epochs * npairs)
    order = rng.permutation(npairs)
    losses = []
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    for step in range(steps):
        k = int(order[step % npairs])
        net.accumulate(us[k], ts[k])
        lr = 2e-3 * (0.5 * (1 + np.cos(np.pi * step / max(steps, 1))))  # cosine decay
        net.adam(lr)
        if step % 50 == 0 or step == steps - 1:
            losses.append((step, net.take_loss()))
    torch.cuda.synchronize()
    t_train = time.perf_counter() - t0
    del us, ts
    # Held-out evaluation at the full size.
    evals = []
    for seed in (9001, 9002):
        inst = synth.instance_bspline(SHAPE, seed=seed, lam=LAM)
        plan = tca.plan_from_instance(inst)
        xt = torch.from_numpy(inst.x_true).to(device)
        b = torch.empty(inst.sample_shape, dtype=torch.float32, device=device)
        plan.apply(xt, b)
        b += torch.from_numpy(inst.noise).to(device)
        x = torch.empty(SHAPE, dtype=torch.float32, device=device)
        for _ in range(2):  # warm-up: graphs, workspaces
            plan.solve(b, x, rtol=RTOL)
            net.solve(plan, b, x, rtol=RTOL)
            net.solve(plan, b, x, rtol=RTOL, net_every=16)
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        res = {}
        variants = (("plain", lambda: plan.solve(b, x, rtol=RTOL)),
                    ("net_x0", lambda: net.solve(plan, b, x, rtol=RTOL)),
                    ("net_x0_step16", lambda: net.solve(plan, b, x, rtol=RTOL, net_every=16)))
        for name, fn in variants:
            e0.record()
            for _ in range(args.steps):
                _, info = fn()
            e1.record()
            torch.cuda.synchronize()
            res[name] = {"ms": round(e0.elapsed_time(e1) / args.steps, 3), "iters": info["iters"],
                         "net_steps": info["refinements"] if name != "plain" else 0,
                         "rel_res_true": info["rel_res_true"]}
        # network forward alone at this size
        u = torch.empty(SHAPE, dtype=torch.float32, device=device)
        y = torch.empty_like(u)
        plan.apply_T(b, u)
        net.forward(u, y)
        e0.record()
        for _ in range(args.steps):
            net.forward(u, y)
        e1.record()
        torch.cuda.synchronize()
        res["net_forward_ms"] = round(e0.elapsed_time(e1) / args.steps, 3)
        evals.append({"seed": seed, **res})
        plan.close()
    out = {
        "case": "learned", "train_pairs": npairs, "train_shape": list(TRAIN_SHAPE), "gen_s": round(t_gen, 2),
        "gen_iters_mean": round(gen_iters / max(npairs, 1), 1), "train_steps": steps,
        "train_s": round(t_train, 2), "train_ms_per_step": round(1e3 * t_train / max(steps, 1), 3),
        "loss": losses[:3] + losses[-3:], "eval_shape": list(SHAPE), "eval": evals,
    }
    net.close()
    if emit:
        print(json.dumps(out), flush=True)
    return out


def dist_setup(n_gpus):
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    if world > 1:
        import torch
        import torch.distributed as dist

        backend = "nccl" if torch.cuda.is_available() else "gloo"
        if torch.cuda.is_available():
            torch.cuda.set_device(local)
        dist.init_process_group(backend=backend)
    return rank, world, local


def barrier(world):
    if world > 1:
        import torch.distributed as dist

        dist.barrier()


def max_over_ranks(v, world):
    if world == 1:
        return v
    import torch
    import torch.distributed as dist

    t = torch.tensor([v], dtype=torch.float64, device="cuda" if torch.cuda.is_available() else "cpu")
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def measured_peaks():
    path = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(path):
        with open(path) as f:
            return json.load(f), "measured"
    return {"hbm_gbs": 6800.0, "bf16_tflops": 1900.0}, "fallback"


class ClockSampler:
    """nvidia-smi clock / throttle sampling during the timed region."""

    def __init__(self, gpu_index: int):
        self.proc = None
        self.lines = []
        self.idx = gpu_index

    def __enter__(self):
        q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
             "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
             "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")
        try:
            self.proc = subprocess.Popen(["nvidia-smi", f"--id={self.idx}", f"--query-gpu={q}",
                                          "--format=csv,noheader,nounits", "-lms", "100"],
                                         stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
        except (FileNotFoundError, OSError):
            self.proc = None
        time.sleep(0.3)
        return self

    def __exit__(self, *exc):
        if self.proc is not None:
            self.proc.terminate()
            try:
                out, _ = self.proc.communicate(timeout=5)
            except subprocess.TimeoutExpired:
                self.proc.kill()
                out, _ = self.proc.communicate()
            self.lines = [l for l in out.splitlines() if l.strip()]

    def summary(self):
        sm, mx, reasons = [], None, set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for l in self.lines:
            f = [x.strip() for x in l.split(",")]
            if len(f) < 9:
                continue
            try:
                sm.append(float(f[1]))
                mx = float(f[2])
            except ValueError:
                continue
            for n, v in zip(names, f[5:9]):
                if v.lower().startswith("active"):
                    reasons.add(n)
        if not sm:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["unsampled"], "samples": 0}
        loaded = [v for v in sm if mx and v >= 0.5 * mx] or sm
        return {"sm_mhz": statistics.median(loaded), "sm_max_mhz": mx, "reasons": sorted(reasons),
                "samples": len(sm)}


def make_problem(shape, seed, device):
    import torch

    from paper_1001_5460_gb300 import synth, tca

    inst = synth.instance_bspline(shape, seed=seed, lam=LAM, dtype=np.float32)
    plan = tca.plan_from_instance(inst, precision="f32")
    xt = torch.from_numpy(inst.x_true).to(device)
    b = torch.empty(inst.sample_shape, dtype=torch.float32, device=device)
    plan.apply(xt, b)  # b = A x_true on the device, then the measurement noise
    b += torch.from_numpy(inst.noise).to(device)
    torch.cuda.synchronize()
    del xt
    return inst, plan, b


def timed_solve(plan, b, x, steps, stream, **kw):
    """Mean device time (CUDA events on the solve's stream) of `steps` solves after one warm-up."""
    import torch

    plan.solve(b, x, rtol=RTOL, **kw)
    torch.cuda.synchronize()
    times, info = [], None
    for _ in range(steps):
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        _, info = plan.solve(b, x, rtol=RTOL, **kw)
        e1.record(stream)
        torch.cuda.synchronize()
        times.append(e0.elapsed_time(e1))
    return statistics.mean(times), info


def bf16_subvolume_error():
    """The mixed-precision form's error against the FP64 oracle on the 40x40x40x8 instance of the
    workload's generator (60^3 x 12 samples): relative L2 distance between the GPU's bfloat16 /
    double-float solution and the oracle's CG solution (rtol 1e-12)."""
    import torch

    from oracle import tca_oracle as O
    from paper_1001_5460_gb300 import synth, tca

    inst = synth.instance_bspline(SUBVOL, seed=SEED, lam=LAM, dtype=np.float64)
    mats = [f.dense() for f in inst.factors]
    b = (O.apply(inst.x_true, mats) + inst.noise).astype(np.float32)
    plan = tca.plan_from_instance(inst, precision="bf16_ir")
    x = torch.zeros(SUBVOL, dtype=torch.float32, device="cuda")
    st, info = plan.solve(torch.from_numpy(b).cuda(), x, rtol=RTOL, inner_rtol=BF16_INNER)
    got = x.cpu().numpy().astype(np.float64)
    ref = O.solve(b.astype(np.float64), mats, inst.lam, rtol=1e-12).x
    plan.close()
    return {"shape": list(SUBVOL), "status": int(st),
            "rel_l2_error": float(np.linalg.norm(got - ref) / np.linalg.norm(ref)),
            "oracle_rel_residual": O.rel_residual(got, b.astype(np.float64), mats, inst.lam)}


def time_sweeps(plan, inst, device, reps=20):
    """Standalone sweep timings (CUDA events on the launching stream)."""
    import torch

    from paper_1001_5460_gb300 import tca

    N = int(np.prod(inst.shape))
    x = torch.randn(inst.shape, dtype=torch.float32, device=device)
    y = torch.empty_like(x)
    s = torch.cuda.current_stream()
    out = {}

    def timed(fn, nbytes):
        for _ in range(3):
            fn()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        torch.cuda.synchronize()
        e0.record(s)
        for _ in range(reps):
            fn()
        e1.record(s)
        torch.cuda.synchronize()
        ms = e0.elapsed_time(e1) / reps
        return {"ms": round(ms, 5), "gbs": round(nbytes / ms / 1e6, 1)}

    out["normal_fused"] = timed(lambda: plan.apply_normal(x, y), 2 * N * 4)
    for k in range(len(inst.shape)):
        out[f"gram_mode{k + 1}"] = timed(lambda k=k: plan.apply_mode(k, tca.OP_GRAM, inst.shape, x, y), 2 * N * 4)
    # collocation sweep on mode 1 (n -> 1.5 n): reads N, writes 1.5 N
    big = torch.empty((inst.factors[0].m,) + tuple(inst.shape[1:]), dtype=torch.float32, device=device)
    out["collocation_mode1"] = timed(lambda: plan.apply_mode(0, tca.OP_FACTOR, inst.shape, x, big),
                                     (N + big.numel()) * 4)
    del big, x, y
    return out


def oracle_sample(inst, b_host, iters, nthreads):
    """Bounded oracle sample on the full problem: A^T b once and one application of
    K (the long way); time-to-solution = t(A^T b) + (iters + 1) * t(K)."""
    from oracle import tca_oracle as O

    mats = [f.dense() for f in inst.factors]
    t0 = time.perf_counter()
    rhs = O.apply_T(b_host, mats)
    t1 = time.perf_counter()
    O.normal_apply(rhs, mats, inst.lam)
    t2 = time.perf_counter()
    t_rhs, t_k = t1 - t0, t2 - t1
    return {"value_ms": 1e3 * (t_rhs + (iters + 1) * t_k), "t_rhs_s": t_rhs, "t_k_s": t_k,
            "cores": nthreads}


def oracle_iterations(seed):
    """Iterations the oracle's CG needs on the 40x40x40x8 instance of the same generator."""
    from oracle import tca_oracle as O
    from paper_1001_5460_gb300 import synth

    inst = synth.instance_bspline(SUBVOL, seed=seed, lam=LAM, dtype=np.float64)
    mats = [f.dense() for f in inst.factors]
    b = O.apply(inst.x_true, mats) + inst.noise
    return O.solve(b, mats, inst.lam, rtol=RTOL).iters


def run_reference(args, rank, world):
    if rank != 0:
        return
    from paper_1001_5460_gb300 import synth
    from oracle import tca_oracle as O

    inst = synth.instance_bspline(SHAPE, seed=SEED, lam=LAM, dtype=np.float32)
    mats = [f.dense() for f in inst.factors]
    b = O.apply(inst.x_true, mats) + inst.noise.astype(np.float64)
    iters = oracle_iterations(SEED)
    nthreads = os.cpu_count()
    vals = []
    for i in range(args.warmup + args.steps):
        r = oracle_sample(inst, b, iters, nthreads)
        if i >= args.warmup:
            vals.append(r["value_ms"])
    v = statistics.mean(vals)
    sample = (f"per step: A^T b and one normal-operator application of the FP64 oracle on the full "
              f"160x160x160x8 problem, extrapolated as t(A^T b) + (iters+1) t(K) with iters={iters} "
              f"(oracle CG on the 40x40x40x8 instance of the same generator)")
    line = {"impl": "reference", "metric": METRIC, "value": round(v, 3), "unit": "ms", "n_gpus": args.gpus,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": round(v, 3), "higher_is_better": False,
            "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": {"workload": WORKLOAD},
            "cpu_baseline": {"value": round(v, 3), "unit": "ms", "cores": nthreads, "kind": "oracle",
                             "sample": sample},
            "e2e": {"value": round(v, 3), "unit": "ms", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


def run_variants(args, plan, inst, b, x, s, N, world, device, peaks, variants):
    """The variants of the bench line (see the module docstring), after the plain timing."""
    from paper_1001_5460_gb300 import tca

    # The same solve with the point-Jacobi preconditioner M = diag(K).
    j_ms, j_info = timed_solve(plan, b, x, args.steps, s, precond="jacobi")
    variants["jacobi_pcg"] = {
        "ms": round(max_over_ranks(j_ms, world), 3), "cg_iters": j_info["iters"], "restarts": j_info["refinements"],
        "rel_res_true": j_info["rel_res_true"],
        "what": "CG preconditioned by point Jacobi, M = diag(K) = prod_k diag(G_k) + lambda sum_k diag(L_k)"}

    # Mixed precision in bfloat16: the same problem, TCA_BF16_IR (bfloat16 inner CG on the
    # tensor-core sweep, double-float refinement), tuned by tca_autotune.
    try:
        bplan = tca.plan_from_instance(inst, precision="bf16_ir")
        t0 = time.perf_counter()
        bplan.autotune()
        tune_s = time.perf_counter() - t0
        bf_ms, bf_info = timed_solve(bplan, b, x, args.steps, s, inner_rtol=BF16_INNER)
        _, bf_prof = bplan.solve(b, x, rtol=RTOL, inner_rtol=BF16_INNER, profile=True)
        bf_sweep_ms = bf_prof["sweep_ms"] / max(bf_prof["sweep_launches"], 1)
        bf_gbs = 4 * N * 2 / bf_sweep_ms / 1e6  # CG sweep: r, p_old in; p, q out (bfloat16)
        variants["bf16_ir"] = {
            "ms": round(max_over_ranks(bf_ms, world), 3), "inner_iters": bf_info["iters"],
            "refinements": bf_info["refinements"], "rel_res_true": bf_info["rel_res_true"],
            "inner_rtol": BF16_INNER, "autotune_s": round(tune_s, 3),
            "autotuned": {"chunks": tca._lib.tca_autotuned_chunks(bplan.handle), "rows_per_thread": bplan.autotuned_rows()},
            "sweep": {"kernel": "bfloat16 tensor-core CG sweep (tcgen05 kind::f16, FP32 accumulation)",
                      "avg_launch_ms": round(bf_sweep_ms, 5), "launches": bf_prof["sweep_launches"],
                      "algorithmic_bytes": 4 * N * 2, "achieved_gbs": round(bf_gbs, 1),
                      "frac_of_measured_hbm": round(bf_gbs / peaks["hbm_gbs"], 4)},
            "what": "iterative refinement: outer FP64-accurate (double-float) residual, inner CG with r, p, q in "
                    "bfloat16 and the modes-3/4 contraction on the tensor cores (BF16 x BF16 -> FP32)"}
        bplan.close()
    except Exception as exc:  # reported, not fatal: the plain solve is the bench value
        variants["bf16_ir"] = {"error": repr(exc)[:300]}

    sub = argparse.Namespace(**vars(args))
    sub.steps = max(1, min(args.steps, 3))
    sub.warmup = 1
    if not args.small:
        try:
            variants["scattered"] = run_scattered(sub, device, emit=False)
        except Exception as exc:
            variants["scattered"] = {"error": repr(exc)[:300]}
        try:
            variants["batched"] = run_batched(sub, device, emit=False)
        except Exception as exc:
            variants["batched"] = {"error": repr(exc)[:300]}
        if not args.no_learned:
            try:
                variants["learned"] = run_learned(sub, device, emit=False)
            except Exception as exc:
                variants["learned"] = {"error": repr(exc)[:300]}



def run_tca(args, rank, world, local):
    import torch

    from paper_1001_5460_gb300 import tca

    device = torch.device("cuda", local)
    torch.cuda.set_device(device)
    shape = (64, 64, 64, 8) if args.small else SHAPE
    inst, plan, b = make_problem(shape, SEED + rank, device)
    N = int(np.prod(shape))
    M = int(np.prod(inst.sample_shape))
    x = torch.zeros(shape, dtype=torch.float32, device=device)
    s = torch.cuda.current_stream()

    for _ in range(max(args.warmup, 0)):
        st, info = plan.solve(b, x, rtol=RTOL)
        st, info = plan.solve(b, x, rtol=RTOL, profile=True)
    barrier(world)
    torch.cuda.synchronize()
    tca.kernel_launches(reset=True)
    times, sweep_ms, sweep_n, infos = [], 0.0, 0, []
    launches = 0
    with ClockSampler(local) as clk:
        for _ in range(args.steps):
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record(s)
            st, info = plan.solve(b, x, rtol=RTOL)
            e1.record(s)
            torch.cuda.synchronize()
            times.append(e0.elapsed_time(e1))
            infos.append(info)
            launches += tca.kernel_launches(reset=True)
            # The same solve with every CG sweep bracketed by CUDA events on the
            # solve's stream (one graph pass per launch): the sweep's live
            # launch time for the roofline, sampled right after each timed solve.
            st_p, info_p = plan.solve(b, x, rtol=RTOL, profile=True)
            sweep_ms += info_p["sweep_ms"]
            sweep_n += info_p["sweep_launches"]
            tca.kernel_launches(reset=True)
        torch.cuda.synchronize()
    barrier(world)
    ms = max_over_ranks(statistics.mean(times), world)

    # End to end through the public API with host (pinned) buffers.
    b_host = b.cpu().pin_memory()
    x_host = torch.zeros(shape, dtype=torch.float32).pin_memory()
    plan.solve(b_host, x_host, rtol=RTOL)
    e2e = []
    for _ in range(max(1, min(args.steps, 3))):
        t0 = time.perf_counter()
        plan.solve(b_host, x_host, rtol=RTOL)
        e2e.append(1e3 * (time.perf_counter() - t0))
    e2e_ms = max_over_ranks(statistics.mean(e2e), world)

    # Variants: the same solve preconditioned by the separable tensor inverse
    # (device buffers, same timing) at the default shift and at twice it;
    # `value` stays the plain CG of Fig. 2.
    variants = {}
    for kind, shift in (() if args.no_variants else (("separable", 16.0), ("separable", 32.0),
                                                      ("separable_banded", 16.0), ("separable_banded", 32.0),
                                                      ("separable_banded", 0.0))):
        plan.solve(b, x, rtol=RTOL, precond=kind, precond_shift=shift)
        torch.cuda.synchronize()
        pc_times, pc_info = [], None
        for _ in range(args.steps):
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record(s)
            st, pc_info = plan.solve(b, x, rtol=RTOL, precond=kind, precond_shift=shift)
            e1.record(s)
            torch.cuda.synchronize()
            pc_times.append(e0.elapsed_time(e1))
        pc_ms = max_over_ranks(statistics.mean(pc_times), world)
        how = ("dense TF32 mode products on the tensor cores" if kind == "separable" else
               "each factor cut to its 7 central diagonals, applied as one plain fused sweep")
        used = shift if shift > 0 else plan.precond_default_shift()
        name = f"{kind}_pcg_s{int(shift)}" if shift > 0 else f"{kind}_pcg_default_shift"
        variants[name] = {
            "ms": round(pc_ms, 3), "cg_iters": pc_info["iters"], "restarts": pc_info["refinements"],
            "rel_res_true": pc_info["rel_res_true"], "shift": used,
            "what": f"CG preconditioned by the separable tensor inverse (x)_k (G_k + s lambda L_k)^-1, s = {used:g}"
                    + (" (the plan's corner-model default)" if shift <= 0 else "")
                    + f" ({how}), same tolerance on the FP64 true residual"}

    if not args.no_variants:
        # The same solve preconditioned by the two-grid tensor multigrid cycle (Sec. 4.2,
        # Fig. 3) with every default: modes 1-3 coarsened, three Chebyshev steps, coarse CG to 0.3.
        try:
            tmg_ms, tmg_info = timed_solve(plan, b, x, max(1, min(args.steps, 5)), s, precond="tmg")
            st_t = plan.tmg_info()
            variants["tmg_pcg"] = {
                "ms": round(max_over_ranks(tmg_ms, world), 3), "cg_iters": tmg_info["iters"],
                "restarts": tmg_info["refinements"], "rel_res_true": tmg_info["rel_res_true"],
                "coarse_cg_iters": st_t["coarse_iters"], "lambda_max_DinvK": round(st_t["lambda_max"], 4),
                "what": "CG preconditioned by a two-grid tensor multigrid cycle: Chebyshev smoothing on "
                        "D^-1 K (3 steps before and after), separable linear-interpolation transfers on "
                        "modes 1-3, Galerkin coarse operator P^T K P solved by CG to 0.3 (host-steered)"}
        except Exception as exc:
            variants["tmg_pcg"] = {"error": repr(exc)[:300]}

    peaks, peak_src = measured_peaks()
    if not args.no_variants:
        run_variants(args, plan, inst, b, x, s, N, world, device, peaks, variants)
    sweeps = time_sweeps(plan, inst, device)
    if rank != 0:
        return
    k2_ms = sweep_ms / max(sweep_n, 1)
    k2_bytes = 4 * N * 4  # CG sweep: reads r and p_old, writes p_new and q (FP32)
    achieved = k2_bytes / k2_ms / 1e6
    last = infos[-1]
    line = {
        "metric": METRIC, "value": round(ms, 3), "unit": "ms", "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": round(ms, 3), "higher_is_better": False, "scaling": "weak",
        "vs_baseline": None, "dtype": "f32", "data": "synthetic",
        "config": {"workload": WORKLOAD if not args.small else "small 64x64x64x8 check run",
                   "precision": "plain FP32 CG, FP64 scalars and FP64 true residual",
                   "cg_iters": last["iters"], "restarts": last["refinements"],
                   "rel_res_true": last["rel_res_true"],
                   "l2": "inputs larger than L2 (b 664 MB, 5 FP32 vectors of 131 MB)",
                   "parallelism": "replicas" if world > 1 else "single GPU"},
        "roofline": {"kernel": "fused normal-operator CG sweep (p = r + beta p; q = K p; <p,q>)",
                     "bound": "hbm", "achieved": round(achieved, 1), "peak": peaks["hbm_gbs"],
                     "unit": "GB/s", "frac": round(achieved / peaks["hbm_gbs"], 4),
                     "traffic": K2_TRAFFIC_BYTES if not args.small else None,
                     "peak_source": peak_src, "avg_launch_ms": round(k2_ms, 5),
                     "algorithmic_bytes": k2_bytes, "launches": sweep_n},
        "sweeps": sweeps,
        "variants": variants,
        "e2e": {"value": round(e2e_ms, 3), "unit": "ms", "h2d_bytes_per_step": M * 4, "d2h_bytes_per_step": N * 4},
        "gpu_launches": int(launches),
        "clocks": clk.summary(),
    }
    if world == 1 and not args.no_cpu_baseline and not args.small:
        # Oracle leg (CPU): the FP64 reference for the bfloat16 variant's error, then the timed sample.
        if "error" not in variants.get("bf16_ir", {"error": 1}):
            try:
                line["variants"]["bf16_ir"]["err_vs_fp64_oracle"] = bf16_subvolume_error()
            except Exception as exc:
                line["variants"]["bf16_ir"]["err_vs_fp64_oracle"] = {"error": repr(exc)[:300]}
        r = oracle_sample(inst, b.cpu().numpy().astype(np.float64), last["iters"], os.cpu_count())
        line["cpu_baseline"] = {
            "value": round(r["value_ms"], 1), "unit": "ms", "cores": r["cores"], "kind": "oracle",
            "sample": (f"A^T b ({r['t_rhs_s']:.2f} s) and one normal-operator application "
                       f"({r['t_k_s']:.2f} s) of the FP64 oracle on the full problem, scaled to the GPU's "
                       f"{last['iters']} CG iterations + 1 residual check")}
    print(json.dumps(line), flush=True)


def main():
    args = parse()
    rank, world, local = dist_setup(args.gpus)
    if args.case:
        run_case(args, local)
    elif args.impl == "reference":
        run_reference(args, rank, world)
    else:
        run_tca(args, rank, world, local)
    if world > 1:
        import torch.distributed as dist

        dist.destroy_process_group()


if __name__ == "__main__":
    main()
