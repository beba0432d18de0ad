"""Benchmark: Parareal solves of the 256^2 mass-conserving Allen-Cahn workload.

One step = one complete Parareal solve (Algorithm 2) of 16 independent
problems: 256 x 256 periodic grid, eps = 0.01, S = 2, dt = 5e-5, 32 slices of
200 fine steps, zero-mean U(-0.9, 0.9) initial data, coarse propagator
1 -> 32 x 6 layers of 3x3 circular conv with GELU (bf16 operands, float32
accumulation; weights trained by paper_2510_07672_gb300/train.py, or the
N(0, 0.01^2) initialisation with --weights untrained), iterated until every
problem's relative L2 increment is below 1e-6 (or k = s, where Parareal is
exact).

value = delivered fine trajectory throughput of the solve,
        problems * slices * steps * n^2 / (device time of one solve)   [cell-steps/s]
The sequential float32 fine solve of the same problems (the same fine kernel,
slices one after another, all 16 problems per launch) is timed next to it.

Usage: python bench.py [--gpus N] [--steps K] [--warmup W] [--impl reference]
Under torchrun (N > 1) every rank solves its own 16 problems (replicas; the
path has no exchange between problems) and rank 0 prints the line.
"""
from __future__ import annotations

import argparse
import json
import os
import statistics
import subprocess
import sys
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

import numpy as np  # noqa: E402

import acpr_inputs as I  # noqa: E402

METRIC = "Parareal time-to-1e-6 vs sequential fine on GB300; fine cell-steps/s, %roofline"
TRAINED = os.path.join(ROOT, "paper_2510_07672_gb300", "weights", "mass256_c32l6_gelu.npz")
UNIT = "cell-steps/s"
WL = I.MASS_F32_256


def fine_flops_per_cell_step(n: int) -> float:
    """Algorithmic flops of one fine step per grid cell: a forward and an
    inverse real 2D FFT at 2.5 * M * log2(M) flops each (M = n^2), plus 10
    pointwise flops (right-hand side and symbol divide)."""
    return 5.0 * np.log2(n * n) + 10.0


def peak_fp32_tflops(sm_mhz: float) -> float:
    """FP32 CUDA-core peak: 152 SMs x 128 lanes x 2 flop (FMA) x clock."""
    return 152 * 128 * 2 * sm_mhz * 1e6 / 1e12


def conv_flops_per_cell(layers: int, C: int) -> float:
    return float(sum(2 * 9 * ci * co for ci, co in I.cnn_layer_dims(layers, C)))


def measured_peaks():
    path = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(path):
        with open(path) as f:
            return json.load(f), "measured"
    return {"hbm_gbs": 6800.0, "bf16_tflops": 1900.0, "bf16_tflops_sustained": 1700.0,
            "sm_max_mhz": 2070.0}, "fallback"


class ClockSampler:
    """nvidia-smi clock / throttle sampling during the timed region."""
    Q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
         "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
         "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index: int):
        self.gpu = gpu_index
        self.proc = None

    def __enter__(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", f"--id={self.gpu}", f"--query-gpu={self.Q}", "--format=csv,noheader,nounits",
                 "-lms", "200"], stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
        except OSError:
            self.proc = None
        return self

    def __exit__(self, *a):
        self.out = ""
        if self.proc is not None:
            self.proc.terminate()
            try:
                self.out, _ = self.proc.communicate(timeout=5)
            except subprocess.TimeoutExpired:
                self.proc.kill()
                self.out, _ = self.proc.communicate()

    def summary(self):
        sm, mx, reasons = [], None, set()
        for line in (self.out or "").splitlines():
            f = [x.strip() for x in line.split(",")]
            if len(f) < 9:
                continue
            try:
                sm.append(float(f[1]))
                mx = float(f[2])
            except ValueError:
                continue
            names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
            for nm, v in zip(names, f[5:9]):
                if v.lower().startswith("active"):
                    reasons.add(nm)
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": mx,
                "reasons": sorted(reasons), "samples": len(sm)}


def cpu_oracle_rate(n: int, steps: int, variant: int, seed: int = 0):
    """The float64 oracle's fine propagation of one field on one host core."""
    import oracle as O
    O.build()
    p = O.params(n, WL.eps, WL.S, WL.dt, variant)
    u = I.random_field(n, seed=seed, zero_mean=True)
    t0 = time.perf_counter()
    O.fine_propagate(p, steps, u)
    dt = time.perf_counter() - t0
    return steps * n * n / dt, dt


def _oracle_worker(seed: int):
    return cpu_oracle_rate(WL.n, 150, WL.variant, seed=seed)[1]


def cpu_oracle_rate_all_cores(n: int, steps: int, variant: int):
    """The oracle on every host core at once: one spawned process per core,
    each propagating its own field (independent fine solves, as the slices of
    one Parareal iteration are).  Returns (aggregate rate, wall seconds,
    processes)."""
    import multiprocessing as mp
    import oracle as O
    O.build()
    workers = os.cpu_count() or 1
    ctx = mp.get_context("spawn")
    with ctx.Pool(workers) as pool:
        pool.map(_oracle_worker, [0] * workers)  # start-up and first touch, untimed
        t0 = time.perf_counter()
        pool.map(_oracle_worker, list(range(workers)))
        wall = time.perf_counter() - t0
    return workers * steps * n * n / wall, wall, workers


def run_reference(args, rank: int, world: int):
    """The oracle, timed on the host cores, on the same workload and metric."""
    if rank != 0:
        return
    steps_per_sample = 40
    for _ in range(args.warmup):
        cpu_oracle_rate(WL.n, 4, WL.variant)
    rates, times = [], []
    for k in range(args.steps):
        r, t = cpu_oracle_rate(WL.n, steps_per_sample, WL.variant, seed=k)
        rates.append(r)
        times.append(t)
    value = float(np.median(rates))
    line = {
        "impl": "reference", "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": args.gpus,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * float(np.mean(times)),
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
        "data": "synthetic",
        "config": {"workload": WL.name, "n": WL.n, "problems": WL.problems, "slices": WL.slices,
                   "steps_per_slice": WL.steps},
        "cpu_baseline": {"value": value, "unit": UNIT, "cores": 1, "kind": "oracle",
                         "sample": f"{steps_per_sample} fine steps of one {WL.n}^2 field per step "
                                   "(float64 oracle, sequential fine throughput; upper bound of its "
                                   "Parareal delivered rate on one core)"},
        "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line), flush=True)


def run_uneven(args):
    """64 independent classic problems of uneven grid (128/256/512), slice count
    (16..64) and steps per slice (50..400), eps = 2.5 h: one handle per grid
    size, all solved together on three streams, each iteration a CUDA graph.
    Prints one JSON line (not the benchmark line)."""
    import torch
    import paper_2510_07672_gb300 as G
    probs = I.uneven_problems()
    classes = sorted({p["n"] for p in probs})
    Wc = I.cnn_weights(6, 32, seed=0)
    net = G.CoarseNet(6, 32, Wc[0].astype(np.float32), Wc[1].astype(np.float32), act=1, precision=G.AC_F32)
    handles, streams, groups = [], [], []
    tuned = {}
    for n in classes:
        grp = [p for p in probs if p["n"] == n]
        fp = G.FineParams(n, 2.5 / n, 2.0, 5e-5, variant=G.AC_CLASSIC, precision=G.AC_F32)
        u0 = torch.tensor(np.stack([I.random_field(n, seed=p["seed"]) for p in grp]), dtype=torch.float32,
                          device="cuda")
        # the tuners pick the fine launch shape (on a batch of the size a fine
        # phase launches) and the conv kernel shape (on the problems' fields) before
        # the handle exists, so no solve changes shape midway
        reps = max(1, 256 // len(grp))
        fb = u0.repeat(reps, 1, 1).contiguous()
        f_ms, f_idx = G.ac_fine_autotune(fp, 20, fb, torch.empty_like(fb))
        c_choice = None
        if G.cnn_conv_variants(n, 32):
            c_ms, c_idx = G.cnn_autotune(net, u0)
            c_choice = {"shape_ring_slots": list(G.cnn_conv_variants(n, 32)[c_idx]),
                        "ms": {str(k): v for k, v in c_ms.items()}}
        tuned[str(n)] = {"fine": G.ac_fine_variants(n, G.AC_F32)[f_idx], "fine_ms_per_20_steps": f_ms,
                         "conv": c_choice}
        h = G.Parareal(fp, net, u0, [p["slices"] for p in grp], [p["steps"] for p in grp])
        h.enable_graphs(not args.no_graphs)
        h.enable_timing(True)
        handles.append(h)
        streams.append(torch.cuda.Stream())
        groups.append((fp, grp, u0))

    def solve():
        for h, (fp, grp, u0) in zip(handles, groups):
            h.reset(u0)
        return G.parareal_solve_many(handles, streams, tol=1e-6, kmax=64)

    for _ in range(args.warmup):
        solve()
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    for _ in range(args.steps):
        out = solve()
    torch.cuda.synchronize()
    ms = (time.perf_counter() - t0) * 1e3 / args.steps
    cells = sum(p["slices"] * p["steps"] * p["n"] ** 2 for p in probs)
    # sequential fine solves of the same problems: per grid size and slice j, one
    # work-list launch advancing every problem with s_p > j by its c_p steps
    seqs = []
    for fp, grp, u0 in groups:
        S = max(p["slices"] for p in grp)
        traj = torch.zeros((len(grp), S + 1, fp.n, fp.n), dtype=torch.float32, device="cuda")
        traj[:, 0] = u0
        works = []
        for j in range(S):
            items = sorted(([i * (S + 1) + j, i * (S + 1) + j + 1, p["steps"], 0] for i, p in enumerate(grp)
                            if p["slices"] > j), key=lambda w: -w[2])
            works.append(torch.tensor(items, dtype=torch.int32, device="cuda"))
        seqs.append((fp, traj, works))

    def sequential():
        for (fp, traj, works), st in zip(seqs, streams):
            with torch.cuda.stream(st):
                for w in works:
                    G.ac_fine_propagate_work(fp, w, traj, traj, stream=st)

    sequential()
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    sequential()
    torch.cuda.synchronize()
    seq_ms = (time.perf_counter() - t0) * 1e3
    its = [i for o in out for i in o[0]]
    st = [h.stats() for h in handles]
    fine_ms = sum(x["fine_ms"] for x in st) / (args.steps + args.warmup)
    print(json.dumps({
        "metric": METRIC, "workload": "uneven-64-classic-f32", "value": cells / (ms * 1e-3), "unit": UNIT,
        "ms_per_solve": ms, "sequential_ms": seq_ms, "speedup_vs_sequential": seq_ms / ms,
        "iterations_mean": float(np.mean(its)), "problems": len(probs),
        "grid_classes": {str(n): sum(1 for p in probs if p["n"] == n) for n in classes},
        "fine_ms_per_solve_summed_over_streams": fine_ms, "steps": args.steps, "warmup": args.warmup,
        "coarse_weights": "untrained N(0, 0.01^2)", "cuda_graphs": not args.no_graphs, "autotuned": tuned}),
        flush=True)


def run_train(args):
    """The differentiation workload: training iterations of the 1 -> 64 x 8
    GELU bf16 coarse net on 256^2 fields -- a 4-step unrolled MSE against fine
    trajectories with 100 fine steps between snapshots, backward through the
    chain, Adam -- with batches of 16 windows drawn from 512 trajectories of
    the classic model (eps = 0.01, dt = 5e-5, S = 2) from seeded U(-0.9, 0.9)
    initial data.  Prints one JSON line (not the benchmark line)."""
    import torch
    import paper_2510_07672_gb300 as G
    from paper_2510_07672_gb300.train import make_trajectories, train_coarse
    n, C, L, unroll, batch, R, snaps = 256, 64, 8, 4, 16, 512, 6
    fp = G.FineParams(n, 0.01, 2.0, 5e-5, variant=G.AC_CLASSIC, precision=G.AC_F32)
    ics = torch.tensor(np.stack([I.random_field(n, seed=s) for s in range(R)]), dtype=torch.float32,
                       device="cuda")
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    traj = make_trajectories(fp, ics, snaps, 100)
    torch.cuda.synchronize()
    gen_s = time.perf_counter() - t0
    w, b = I.cnn_weights(L, C, seed=0)
    net = G.TrainableCoarseNet(L, C, w.astype(np.float32), b.astype(np.float32), act=G.AC_ACT_GELU)
    train_coarse(net, traj, max(args.warmup, 1), batch, unroll, 1e-3)
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    losses = train_coarse(net, traj, args.steps, batch, unroll, 1e-3, seed=1)
    torch.cuda.synchronize()
    ms = (time.perf_counter() - t0) * 1e3 / args.steps
    fwd = batch * unroll * n * n * 2 * 9 * (C + (L - 2) * C * C + C)
    print(json.dumps({
        "metric": "coarse-net training iteration (4-step unrolled MSE, backward, Adam)",
        "workload": "train-c64l8-gelu-bf16-256sq-b16-u4", "ms_per_iteration": ms,
        "windows_per_s": batch / (ms * 1e-3), "tflops_est": 3 * fwd / (ms * 1e-3) / 1e12,
        "flops_note": "3 x forward conv flops (forward, input and weight gradients)",
        "trajectories": R, "snapshots": snaps, "trajectory_generation_s": gen_s,
        "loss_first": losses[0], "loss_last": losses[-1], "steps": args.steps, "warmup": args.warmup,
        "timing": "wall clock per iteration, one host read of the loss per iteration included"}), flush=True)


def run_acnn(args):
    """The paper's light coarse network (Sec. 3.2: ResBlock mACNN, C = 4, two
    blocks, tanh, mass shift, limiter [-1, 1]) on the benchmark's problems
    (mass-conserving 256^2 fields, eps = 0.01, fine dt = 5e-5, slices of 200
    fine steps):
      1. Algorithm 1 with the scheme-residual loss (Eq. loss_ACN) at the slice
         step 200 dt: 32 seeded initial conditions disjoint from the
         benchmark's, subsets of q = 16, 8 coarse steps, 4 inner updates,
         `--acnn-epochs` epochs; time per update;
      2. one application of G to the 16 benchmark fields (the fused kernel),
         CUDA-event time over 200 launches (4 MB of input, L2-resident: the
         kernel is bound by FP32 issue), with its FP32 roofline;
      3. the benchmark's Parareal solve (16 problems, 32 slices x 200 steps,
         tol 1e-6, CUDA graphs) with this G, against the sequential fine solve.
    Prints one JSON line (not the benchmark line)."""
    import torch
    import paper_2510_07672_gb300 as G
    W = I.MASS_F32_256
    n, C, R, q, steps, b_inner = W.n, 4, 32, 16, 8, 4
    fp = G.FineParams(n, W.eps, W.S, W.dt, variant=W.variant, precision=G.AC_F32)
    coarse = G.FineParams(n, W.eps, 0.0, W.dt * W.steps, variant=W.variant, precision=G.AC_F32)
    w, b = I.acnn_weights(C, 2, seed=0)
    net = G.Acnn(C, 2, w, b, mass_fix=1, limiter=1, lo=-1.0, hi=1.0, precision=G.AC_F32)
    U0s = torch.tensor(np.stack([I.random_field(n, seed=5000 + i, zero_mean=True) for i in range(R)]),
                       dtype=torch.float32, device="cuda")
    rng = np.random.default_rng(0)
    epochs = args.acnn_epochs
    perm = np.stack([rng.permutation(R) for _ in range(epochs)])
    net.train_alg1(coarse, U0s, perm[:1], q, 1, 1, lr=1e-3)  # warm-up: one update
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    losses = net.train_alg1(coarse, U0s, perm, q, steps, b_inner, lr=1e-3).cpu().numpy()
    train_s = time.perf_counter() - t0
    updates = len(losses)

    u0 = torch.tensor(W.ics().astype(np.float32), device="cuda")
    out = torch.empty_like(u0)
    for _ in range(10):
        net(u0, out=out)
    stream = torch.cuda.current_stream()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    reps = 200
    e0.record(stream)
    for _ in range(reps):
        net(u0, out=out)
    e1.record(stream)
    torch.cuda.synchronize()
    g_us = e0.elapsed_time(e1) * 1e3 / reps
    px = W.problems * n * n
    flops = 2 * px * (9 * C + 4 * 9 * C * C + 9 * C)
    peaks, src = measured_peaks()
    sm_mhz = peaks.get("sm_max_mhz", 2070.0)
    peak = peak_fp32_tflops(sm_mhz)
    achieved = flops / (g_us * 1e-6) / 1e12

    pr = G.Parareal(fp, net, u0, W.slices, W.steps)
    pr.enable_timing(True)
    pr.enable_graphs(True)
    pr.solve(tol=W.tol, kmax=W.kmax)
    pr.reset(u0)
    pr.reset_stats()
    s0, s1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    s0.record(stream)
    its, l2 = pr.solve(tol=W.tol, kmax=W.kmax)
    s1.record(stream)
    torch.cuda.synchronize()
    para_ms = s0.elapsed_time(s1)
    st = pr.stats()
    a, bb = u0.clone(), torch.empty_like(u0)
    for _ in range(W.slices):
        G.ac_fine_propagate_slices(fp, W.steps, a, bb)
        a, bb = bb, a
    torch.cuda.synchronize()
    s0.record(stream)
    for _ in range(W.slices):
        G.ac_fine_propagate_slices(fp, W.steps, a, bb)
        a, bb = bb, a
    s1.record(stream)
    torch.cuda.synchronize()
    seq_ms = s0.elapsed_time(s1)
    print(json.dumps({
        "metric": "ResBlock mACNN coarse propagator (C = 4, 2 blocks): Algorithm 1 training, G time, Parareal",
        "workload": "acnn-c4b2-mass-256sq", "config": {"n": n, "eps": W.eps, "fine_dt": W.dt,
                                                      "coarse_dt": W.dt * W.steps, "channels": C, "blocks": 2},
        "train": {"R": R, "q": q, "steps": steps, "b_inner": b_inner, "epochs": epochs, "updates": updates,
                  "ms_per_update": train_s * 1e3 / updates, "loss_first": float(losses[0]),
                  "loss_last_mean8": float(losses[-8:].mean()), "timing": "host wall clock of one synchronous call"},
        "g": {"fields": W.problems, "us_per_application": g_us, "flops_per_application": flops,
              "roofline": {"bound": "alu", "kernel": "acnn_fused_kernel", "achieved": achieved, "peak": peak,
                           "unit": "TFLOP/s", "frac": achieved / peak,
                           "peak_source": f"FP32 lanes x 2 x sm_max_mhz {sm_mhz:.0f} from {src} peaks"},
              },
        "parareal": {"iterations": its, "final_rel_l2": l2, "ms": para_ms, "sequential_ms": seq_ms,
                     "coarse_ms": st["coarse_ms"], "fine_ms": st["fine_ms"], "coarse_calls": st["coarse_calls"]},
    }), flush=True)


def run_fine3d(args):
    """The fine step on the periodic cube (the 3D experiments of Sec. 4: eps =
    0.02, h = 1/128): 16 mass-conserving float32 fields of 128^3 (seeded
    U(-0.9, 0.9), zero mean), 20 steps of dt = 1e-4 per call, CUDA events over
    `--steps` calls after `--warmup`.  Prints one JSON line (not the benchmark
    line)."""
    import torch
    import paper_2510_07672_gb300 as G
    n, F, steps = 128, 16, 20
    u = torch.tensor(np.stack([(-0.9 + 1.8 * I.uniform01(7000 + f, I.STREAM_IC, n ** 3)).reshape(n, n, n)
                               for f in range(F)]), dtype=torch.float32, device="cuda")
    u -= u.mean(dim=(1, 2, 3), keepdim=True)
    fp = G.FineParams(n, 0.02, 2.0, 1e-4, variant=G.AC_MASS_CONSERVING, precision=G.AC_F32)
    out = torch.empty_like(u)
    work = torch.empty(G.load().ac_fine3d_work_bytes(n, F, G.AC_F32), dtype=torch.uint8, device="cuda")
    for _ in range(max(args.warmup, 1)):
        G.ac_fine3d_propagate(fp, steps, u, out, work=work)
    stream = torch.cuda.current_stream()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    l0 = G.ac_launch_count()
    e0.record(stream)
    for _ in range(args.steps):
        G.ac_fine3d_propagate(fp, steps, u, out, work=work)
    e1.record(stream)
    torch.cuda.synchronize()
    launches = G.ac_launch_count() - l0
    ms = e0.elapsed_time(e1) / args.steps
    cells = F * n ** 3 * steps
    peaks, src = measured_peaks()
    hbm = peaks.get("hbm_gbs", 6800.0)
    pass_bytes = 40.0 * cells  # five passes: 80 bytes per complex cell pair and step
    print(json.dumps({
        "metric": "3D fine propagation (periodic cube, 7-point Laplacian, FFT solve)",
        "workload": "fine3d-mass-f32-128cube-16f-20steps", "ms_per_call": ms, "cell_steps_per_s": cells / (ms * 1e-3),
        "us_per_step": ms * 1e3 / steps, "gpu_launches_per_call": launches / args.steps,
        "roofline": {"bound": "hbm", "achieved": pass_bytes / (ms * 1e-3) / 1e9, "peak": hbm, "unit": "GB/s",
                     "frac": pass_bytes / (ms * 1e-3) / 1e9 / hbm,
                     "traffic_model": "40 B per cell-step (5 passes, complex pairs); the one-read-one-write "
                                      "minimum is 8 B", "peak_source": src},
        "mass_drift": float((out.double().mean(dim=(1, 2, 3)) - u.double().mean(dim=(1, 2, 3))).abs().max().item()),
        "steps": args.steps, "warmup": args.warmup}), flush=True)


def run_adjoint(args):
    """The adjoint workload: dE_h(u^2000)/du^0 of one 256^2 classic field
    (eps = 0.01, dt = 5e-5, S = 2) by the checkpointed adjoint (a checkpoint
    every 32 steps), float32 and float64, against the 2000-step forward solve
    of the same field.  Prints one JSON line (not the benchmark line)."""
    import torch
    import paper_2510_07672_gb300 as G
    n, steps, every = 256, 2000, 32
    out = {"metric": "energy gradient through 2000 fine steps (checkpointed adjoint)",
           "workload": "adjoint-256sq-2000-steps-ckpt32", "steps": args.steps, "warmup": args.warmup}
    for prec, dt_, name in ((G.AC_F32, torch.float32, "f32"), (G.AC_F64, torch.float64, "f64")):
        fp = G.FineParams(n, 0.01, 2.0, 5e-5, variant=G.AC_CLASSIC, precision=prec)
        u0 = torch.tensor(I.random_field(n, seed=0)[None], dtype=dt_, device="cuda")
        fwd_out = torch.empty_like(u0)

        def timed(fn):
            for _ in range(max(args.warmup, 1)):
                fn()
            torch.cuda.synchronize()
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record()
            for _ in range(args.steps):
                fn()
            e1.record()
            torch.cuda.synchronize()
            return e0.elapsed_time(e1) / args.steps

        fwd_ms = timed(lambda: G.ac_fine_propagate_slices(fp, steps, u0, fwd_out))
        grad_ms = timed(lambda: G.ac_energy_gradient_ic(fp, steps, u0, checkpoint_every=every))
        out[name] = {"forward_ms": fwd_ms, "gradient_ms": grad_ms, "ratio": grad_ms / fwd_ms,
                     "forward_cell_steps_per_s": steps * n * n / (fwd_ms * 1e-3)}
    out["note"] = ("one field per call (the entry point's shape): one 8-CTA cluster of the GPU's 152 SMs "
                   "works; the gradient runs the forward pass, a recompute of each segment and the adjoint "
                   "steps, about 3x the forward work")
    print(json.dumps(out), flush=True)


def run_plain64(args):
    """The plain float64 configuration: classic Allen-Cahn on a 64^2 grid,
    eps = 0.025, S = 2, dt = 1e-4, 8 slices x 100 steps, conv 1-16-16-16-1
    tanh with N(0, 0.01^2) weights, iterated to a relative increment < 1e-10
    or k = 8.  Times the GPU Parareal solve and the GPU sequential float64
    fine solve (CUDA events, `--steps` repetitions after `--warmup`), and the
    oracle's Algorithm 2 on the same problem on one host core and on all host
    cores (its conv rows and independent fine solves split over threads).
    Prints one JSON line (not the benchmark line)."""
    import oracle as O
    W = I.PLAIN_F64_64
    O.build()
    u0 = W.ics()
    wt, bs = W.weights()
    spec = O.CnnSpec(W.layers, W.channels, wt, bs, act=W.act)
    p_o = O.params(W.n, W.eps, W.S, W.dt, W.variant)
    t0 = time.perf_counter()
    ref = O.parareal(p_o, spec, W.slices, W.steps, kmax=W.kmax, tol=W.tol, u0=u0[0])
    oracle_1 = time.perf_counter() - t0
    cores = os.cpu_count() or 1
    with O.threads(cores):
        t0 = time.perf_counter()
        O.parareal(p_o, spec, W.slices, W.steps, kmax=W.kmax, tol=W.tol, u0=u0[0])
        oracle_n = time.perf_counter() - t0
    import torch
    import paper_2510_07672_gb300 as G
    fp = G.FineParams(W.n, W.eps, W.S, W.dt, variant=W.variant, precision=G.AC_F64)
    net = G.CoarseNet(W.layers, W.channels, wt, bs, act=W.act, precision=G.AC_F64)
    u = torch.tensor(u0, device="cuda")
    pr = G.Parareal(fp, net, u, W.slices, W.steps)
    pr.enable_graphs(not args.no_graphs)
    stream = torch.cuda.current_stream()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)

    def solve():
        pr.reset(u)
        return pr.solve(tol=W.tol, kmax=W.kmax, allow_unconverged=True)

    for _ in range(max(args.warmup, 1)):
        its, l2 = solve()
    torch.cuda.synchronize()
    e0.record(stream)
    for _ in range(args.steps):
        its, l2 = solve()
    e1.record(stream)
    torch.cuda.synchronize()
    para_ms = e0.elapsed_time(e1) / args.steps
    err = float(np.abs(pr.trajectory()[0].cpu().numpy() - ref["U"]).max())
    a, b = u.clone(), torch.empty_like(u)
    for _ in range(W.slices):
        G.ac_fine_propagate_slices(fp, W.steps, a, b)
        a, b = b, a
    torch.cuda.synchronize()
    e0.record(stream)
    for _ in range(args.steps):
        for _ in range(W.slices):
            G.ac_fine_propagate_slices(fp, W.steps, a, b)
            a, b = b, a
    e1.record(stream)
    torch.cuda.synchronize()
    seq_ms = e0.elapsed_time(e1) / args.steps
    print(json.dumps({
        "metric": METRIC, "workload": W.name,
        "config": {"n": W.n, "eps": W.eps, "dt": W.dt, "slices": W.slices, "steps_per_slice": W.steps,
                   "conv": "1-16-16-16-1 tanh float64", "tol": W.tol, "kmax": W.kmax},
        "gpu_parareal_ms": para_ms, "gpu_sequential_ms": seq_ms, "iterations": its[0], "final_rel_l2": l2[0],
        "oracle_iterations": ref["iters"], "max_abs_vs_oracle": err,
        "oracle_parareal_s_1core": oracle_1, "oracle_parareal_s_all_cores": oracle_n, "host_cores": cores,
        "steps": args.steps, "warmup": args.warmup}), flush=True)


LARGE_WEIGHTS = os.path.join(ROOT, "paper_2510_07672_gb300", "weights", "large1024_c64l8_gelu.npz")


def run_large(args):
    """The large single problem: classic Allen-Cahn on a 1024^2 periodic grid,
    eps = 0.004, S = 2, dt = 2e-5, 128 slices x 500 fine steps (T = 1.28), one
    seeded U(-0.9, 0.9) initial field; float32 fine step (two-pass path
    through L2/HBM), float64 increments, coarse net 1 -> 64 x 8 GELU bf16
    (weights trained by train.py --workload large, or N(0, 0.01^2) with
    --weights untrained).  Times the sequential float32 fine solve (128 slices
    one after another, one field) and the Parareal solve to a relative L2
    increment < 1e-6 or `--large-kmax` iterations, both with CUDA events on
    the same GPU.  Prints one JSON line (not the benchmark line)."""
    W = I.LARGE_F32_1024
    n, s, c = W.n, W.slices, W.steps
    # the oracle's sequential fine rate at 1024^2 on one host core, from 10
    # float64 steps (before any GPU work in this process), extrapolated to
    # the 64,000-step solve
    import oracle as O
    O.build()
    p_o = O.params(n, W.eps, W.S, W.dt, W.variant)
    u_host = W.ics()[0]
    t0 = time.perf_counter()
    O.fine_propagate(p_o, 10, u_host)
    o_s = time.perf_counter() - t0
    cpu = {"value": 10 * n * n / o_s, "unit": "cell-steps/s", "cores": 1, "kind": "oracle",
           "sample": f"10 float64 fine steps of the 1024^2 field on one core ({o_s:.1f} s); the sequential "
                     f"64,000-step solve extrapolates to {o_s * s * c / 10:.0f} s"}
    import torch
    import paper_2510_07672_gb300 as G
    fp = G.FineParams(n, W.eps, W.S, W.dt, variant=W.variant, precision=G.AC_F32)
    wt, bs = W.weights()
    wsrc = "untrained N(0, 0.01^2)"
    wpath = LARGE_WEIGHTS if args.weights == "trained" else (None if args.weights == "untrained" else args.weights)
    if wpath:
        z = np.load(wpath)
        wt, bs = z["w"], z["b"]
        wsrc = (f"trained by paper_2510_07672_gb300/train.py --workload large ({int(z['iters'])} Adam steps, "
                f"{int(z['unroll'])}-step unrolled MSE on {int(z['crop'])}^2 crops, h = 1/1024): "
                f"{os.path.relpath(wpath, ROOT)}")
    net = G.CoarseNet(W.layers, W.channels, wt.astype(np.float32), bs.astype(np.float32), act=W.act,
                      precision=G.AC_F32)
    u0 = torch.tensor(W.ics().astype(np.float32), device="cuda")
    stream = torch.cuda.current_stream()
    ev = lambda: torch.cuda.Event(enable_timing=True)  # noqa: E731

    # sequential float32 fine solve: 128 slices of 500 steps, one field
    a, b = u0.clone(), torch.empty_like(u0)
    G.ac_fine_propagate_slices(fp, c, a, b)  # warm-up (workspace, tables)
    torch.cuda.synchronize()
    e0, e1 = ev(), ev()
    e0.record(stream)
    for _ in range(s):
        G.ac_fine_propagate_slices(fp, c, a, b)
        a, b = b, a
    e1.record(stream)
    torch.cuda.synchronize()
    seq_ms = e0.elapsed_time(e1)
    seq_final = a.clone()

    # one batched fine launch of all 128 slices (Parareal's fine phase at k = 1)
    batch_in = u0.expand(s, n, n).contiguous()
    batch_out = torch.empty_like(batch_in)
    G.ac_fine_propagate_slices(fp, 2, batch_in, batch_out)
    torch.cuda.synchronize()
    e0.record(stream)
    G.ac_fine_propagate_slices(fp, c, batch_in, batch_out)
    e1.record(stream)
    torch.cuda.synchronize()
    batch_ms = e0.elapsed_time(e1)

    # one application of G to one 1024^2 field
    g_out = torch.empty_like(u0)
    for _ in range(3):
        G.cnn_coarse_step(net, u0, g_out)
    torch.cuda.synchronize()
    reps = 20
    e0.record(stream)
    for _ in range(reps):  # each call ends with a status read (a sync of a few us)
        G.cnn_coarse_step(net, u0, g_out)
    e1.record(stream)
    torch.cuda.synchronize()
    g_ms = e0.elapsed_time(e1) / reps

    # Parareal, iteration by iteration (each a CUDA graph), until the
    # increment is below tol or k = --large-kmax; the clock runs from the
    # k = 0 coarse sweep to the last increment
    pr = G.Parareal(fp, net, u0, s, c)
    pr.enable_timing(True)
    pr.enable_graphs(not args.no_graphs)
    pr.iterate()  # k = 0 (records its graph)
    pr.reset(u0)
    pr.reset_stats()
    torch.cuda.synchronize()
    incs, its_ms = [], []
    e0.record(stream)
    pr.iterate()  # k = 0
    k = 0
    while k < args.large_kmax:
        t_it = time.perf_counter()
        l2_k, _ = pr.iterate()
        its_ms.append((time.perf_counter() - t_it) * 1e3)
        k += 1
        incs.append(l2_k[0])
        if l2_k[0] < W.tol:
            break
    e1.record(stream)
    torch.cuda.synchronize()
    para_ms = e0.elapsed_time(e1)
    its, l2 = [k], [incs[-1]]
    st = pr.stats()
    U = pr.trajectory()[0]
    err_vs_seq = float(((U[-1].double() - seq_final[0].double()).norm() / seq_final[0].double().norm()).item())
    peaks, src = measured_peaks()
    hbm = peaks.get("hbm_gbs", 6800.0)
    bf16 = peaks.get("bf16_tflops", 1900.0)
    cells_batch = s * c * n * n
    conv_fl = conv_flops_per_cell(W.layers, W.channels) * n * n
    pr.close()
    print(json.dumps({
        "metric": METRIC, "workload": W.name,
        "config": {"n": n, "eps": W.eps, "S": W.S, "dt": W.dt, "slices": s, "steps_per_slice": c,
                   "variant": "classic", "conv": "1-64x8-1 gelu bf16", "coarse_weights": wsrc, "tol": W.tol,
                   "kmax": args.large_kmax, "cuda_graphs": not args.no_graphs},
        "sequential_ms": seq_ms, "parareal_ms": para_ms, "speedup_vs_sequential": seq_ms / para_ms,
        "iterations": its[0], "final_rel_l2": l2[0], "tol_reached": bool(l2[0] < W.tol),
        "increments": incs, "iteration_wall_ms": its_ms,
        "breakeven_iterations": "Parareal beats the sequential solve only if it stops by the k where "
                                "k0 sweep + k x (fine phase + coarse sweep) < sequential_ms",
        "rel_l2_final_field_vs_sequential": err_vs_seq,
        "phase_ms": {"fine": st["fine_ms"], "coarse": st["coarse_ms"], "increment": st["increment_ms"]},
        "sequential_us_per_step": seq_ms * 1e3 / (s * c),
        "batched_fine": {"fields": s, "steps": c, "ms": batch_ms, "cell_steps_per_s": cells_batch / (batch_ms * 1e-3),
                         "roofline": {"bound": "hbm", "achieved": 16.0 * cells_batch / (batch_ms * 1e-3) / 1e9,
                                      "peak": hbm, "unit": "GB/s",
                                      "frac": 16.0 * cells_batch / (batch_ms * 1e-3) / 1e9 / hbm,
                                      "traffic_model": "16 B per cell-step (rows pass and columns pass, each "
                                                       "one float32 read and write per cell)", "peak_source": src}},
        "coarse_g": {"ms_per_application": g_ms, "tflops": conv_fl / (g_ms * 1e-3) / 1e12,
                     "frac_of_bf16_peak": conv_fl / (g_ms * 1e-3) / 1e12 / bf16},
        "cpu_baseline": cpu,
        "steps": 1, "warmup": 1}), flush=True)


# DRAM bytes (read + write) the fine kernel moved per field-slice in one ncu
# capture of the 256^2 launch shape (512 fields x 20 steps: 134.3 MB read,
# 87.7 MB written); a slice is read once and written once whatever its step
# count, so a launch's traffic scales with the field-slices it processes.
FINE_DRAM_BYTES_PER_FIELD_SLICE_256 = (134.330112e6 + 87.662080e6) / 512


def max_over_ranks(x: float, world: int, device) -> float:
    """The largest x over the ranks (a job's time is its slowest rank's); every
    rank gets it.  device: where the reduction tensor lives (cuda for NCCL,
    cpu for gloo)."""
    if world <= 1:
        return float(x)
    import torch
    import torch.distributed as dist
    t = torch.tensor([float(x)], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def job_rate(cells_per_rank: float, ms: float, world: int) -> float:
    """Whole-job throughput of `world` replicas that each deliver
    cells_per_rank in a step, over the slowest rank's step time (weak
    scaling: the work per GPU is fixed)."""
    return world * cells_per_rank / (ms * 1e-3)


def cost_model(st, seq_ms, its, steps, s=None, c=None, m=1):
    """The cost model of Sec. 3.4 with the measured unit costs: t_num = one
    fine step of one slice (all problems), from the sequential solve; t_nn =
    one application of G (all problems), from the solve's coarse phase.  The
    model puts every slice on its own device, so iteration k's fine sweep
    costs c t_num; with G composed m times per slice each coarse evaluation
    costs m t_nn, so T(k) = c k t_num + (2s - k)(k + 1)/2 m t_nn and
    S_k = s c t_num / T(k).  The measured single-GPU solve is parareal_ms."""
    s = WL.slices if s is None else s
    c = WL.steps if c is None else c
    calls = st.get("coarse_calls", 0) / max(steps, 1)
    if not calls:
        return None
    t_num = seq_ms / (s * c)
    t_nn = st["coarse_ms"] / max(steps, 1) / calls
    k = max(its) if its else s
    T = c * k * t_num + (2 * s - k) * (k + 1) / 2 * m * t_nn
    return {"t_num_ms": t_num, "t_nn_ms": t_nn, "k": k, "s": s, "c": c, "m": m, "coarse_calls_per_solve": calls,
            "T_k_ms": T, "S_k": s * c * t_num / T,
            "note": "Sec. 3.4 model, one slice per device; measured on one GPU: parareal_ms"}


def fine_traffic_per_launch(st, wl, steps=None):
    if wl.n != 256 or not st.get("fine_launches"):
        return None
    slices = st["fine_cell_steps"] / (wl.n * wl.n * (wl.steps if steps is None else steps))
    return FINE_DRAM_BYTES_PER_FIELD_SLICE_256 * slices / st["fine_launches"]


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=3)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--weights", default="trained", help="'trained' (the committed G), 'untrained', or a .npz path")
    ap.add_argument("--workload", default="mass256",
                    choices=["mass256", "uneven", "train", "adjoint", "acnn", "fine3d", "large", "plain64"],
                    help="mass256: the benchmark line; uneven: 64 classic problems of uneven size (batching); "
                         "train: coarse-net training iterations (C = 64, 8 layers); "
                         "adjoint: checkpointed energy gradient through 2000 steps; "
                         "acnn: the paper's ResBlock mACNN (Algorithm 1 training, G time, Parareal); "
                         "fine3d: the fine step on the 128^3 periodic cube; "
                         "large: the 1024^2 single problem, Parareal vs the sequential fine solve; "
                         "plain64: the 64^2 float64 problem, GPU and oracle")
    ap.add_argument("--large-kmax", type=int, default=8)
    ap.add_argument("--acnn-epochs", type=int, default=20)
    ap.add_argument("--no-graphs", action="store_true")
    ap.add_argument("--coarse-substeps", type=int, default=1,
                    help="mass256 only: M > 1 covers the same time span with slices of M x 200 fine steps "
                         "(32 / M slices) and composes G M times per slice")
    args = ap.parse_args()

    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local_rank = int(os.environ.get("LOCAL_RANK", "0"))
    if args.impl == "reference":
        run_reference(args, rank, world)
        return
    if args.workload == "uneven":
        run_uneven(args)
        return
    if args.workload == "train":
        run_train(args)
        return
    if args.workload == "adjoint":
        run_adjoint(args)
        return
    if args.workload == "acnn":
        run_acnn(args)
        return
    if args.workload == "fine3d":
        run_fine3d(args)
        return
    if args.workload == "large":
        run_large(args)
        return
    if args.workload == "plain64":
        run_plain64(args)
        return

    # host-side oracle sample first (before any GPU work in this process)
    cpu = None
    cpu1 = None
    if rank == 0 and not args.no_cpu_baseline:
        rate, secs = cpu_oracle_rate(WL.n, 150, WL.variant)
        cpu1 = {"value": rate, "unit": UNIT, "cores": 1, "kind": "oracle",
                "sample": f"150 fine steps of one {WL.n}^2 mass-conserving field on one core, float64 "
                          f"({secs:.1f} s)"}
        rate_all, wall, procs = cpu_oracle_rate_all_cores(WL.n, 150, WL.variant)
        cpu = {"value": rate_all, "unit": UNIT, "cores": procs, "kind": "oracle",
               "sample": f"150 fine steps of one {WL.n}^2 mass-conserving field per process, {procs} spawned "
                         f"processes on {procs} host cores at once, float64 ({wall:.1f} s wall); the oracle's "
                         f"fine rate bounds its Parareal rate"}

    import torch
    import torch.distributed as dist
    import paper_2510_07672_gb300 as G

    torch.cuda.set_device(local_rank)
    if world > 1:
        dist.init_process_group("nccl", device_id=torch.device("cuda", local_rank))
    dev = torch.device("cuda", local_rank)
    G.load()

    fp = G.FineParams(WL.n, WL.eps, WL.S, WL.dt, variant=WL.variant, precision=G.AC_F32)
    wt, bs = WL.weights()
    wsrc = "untrained N(0, 0.01^2)"
    wpath = TRAINED if args.weights == "trained" else (None if args.weights == "untrained" else args.weights)
    if wpath:
        z = np.load(wpath)
        wt, bs = z["w"], z["b"]
        wsrc = (f"trained by paper_2510_07672_gb300/train.py ({int(z['iters'])} Adam steps, {int(z['unroll'])}-step "
                f"unrolled MSE on fine trajectories from ICs disjoint from the bench's): {os.path.relpath(wpath, ROOT)}")
    net = G.CoarseNet(WL.layers, WL.channels, wt.astype(np.float32), bs.astype(np.float32),
                      act=WL.act, precision=G.AC_F32, mass_fix=WL.mass_fix, device=dev)
    ics = WL.ics().astype(np.float32)  # same 16 problems on every rank (weak scaling replicas)
    u0 = torch.tensor(ics, device=dev)
    M = args.coarse_substeps
    if M < 1 or WL.slices % M:
        raise SystemExit(f"--coarse-substeps must divide {WL.slices}")
    slices, steps = WL.slices // M, WL.steps * M
    pr = G.Parareal(fp, net, u0, slices, steps)
    pr.set_coarse_substeps(M)
    pr.enable_timing(True)
    pr.enable_graphs(not args.no_graphs)
    stream = torch.cuda.current_stream()

    def solve():
        pr.reset(u0)
        its, l2 = pr.solve(tol=WL.tol, kmax=WL.kmax)
        return its, l2

    def barrier():
        if world > 1:
            dist.barrier()
        torch.cuda.synchronize()

    for _ in range(args.warmup):
        its, l2 = solve()
    barrier()
    pr.reset_stats()
    n_launch0 = G.ac_launch_count()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    with ClockSampler(local_rank) as clk:
        barrier()
        e0.record(stream)
        for _ in range(args.steps):
            its, l2 = solve()
        e1.record(stream)
        barrier()
    launches = G.ac_launch_count() - n_launch0
    ms = max_over_ranks(e0.elapsed_time(e1) / args.steps, world, dev)
    st = pr.stats()
    clocks = clk.summary()

    cells = WL.problems * slices * steps * WL.n * WL.n  # delivered per solve per rank
    value = job_rate(cells, ms, world)

    # sequential float32 fine solve of the same problems, same kernel
    seq_in = u0.clone()
    seq_out = torch.empty_like(seq_in)

    def sequential():
        a, b = seq_in, seq_out
        for _ in range(slices):
            G.ac_fine_propagate_slices(fp, steps, a, b)
            a, b = b, a
        return a

    # the sequential reference runs the launch shape that is fastest for its
    # own batch (16 fields per launch), chosen by the library's tuner; the
    # default shape (the fastest on Parareal's large fine batches) is restored
    # afterwards
    default_shape = G.ac_fine_get_variant(WL.n, G.AC_F32)
    _, seq_shape = G.ac_fine_autotune(fp, steps, seq_in, seq_out)
    sequential()
    torch.cuda.synchronize()
    s0, s1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    s0.record(stream)
    sequential()
    s1.record(stream)
    torch.cuda.synchronize()
    seq_ms = s0.elapsed_time(s1)
    G.ac_fine_set_variant(WL.n, G.AC_F32, default_shape)
    seq_shape_name = G.ac_fine_variants(WL.n, G.AC_F32)[seq_shape]

    # end to end through the public API: pinned host ICs in, final fields out
    host_u0 = torch.tensor(ics).pin_memory()
    host_out = torch.empty((WL.problems, WL.n, WL.n), dtype=torch.float32).pin_memory()
    traj = torch.empty((WL.problems, slices + 1, WL.n, WL.n), dtype=torch.float32, device=dev)
    dev_u0 = torch.empty_like(u0)

    def e2e_step():
        dev_u0.copy_(host_u0, non_blocking=True)
        pr.reset(dev_u0)
        pr.solve(tol=WL.tol, kmax=WL.kmax)
        pr.trajectory(out=traj)
        host_out.copy_(traj[:, -1], non_blocking=True)
        torch.cuda.current_stream().synchronize()

    e2e_step()
    barrier()
    t0 = time.perf_counter()
    for _ in range(args.steps):
        e2e_step()
    barrier()
    e2e_ms = max_over_ranks((time.perf_counter() - t0) * 1e3 / args.steps, world, dev)

    if rank == 0:
        peaks, src = measured_peaks()
        sm_mhz = peaks.get("sm_max_mhz", 2070.0)
        fpc = fine_flops_per_cell_step(WL.n)
        fine_tflops = st["fine_cell_steps"] * fpc / (st["fine_ms"] * 1e-3) / 1e12 if st["fine_ms"] else 0.0
        peak = peak_fp32_tflops(sm_mhz)
        conv_tflops = (st["coarse_cells"] * conv_flops_per_cell(WL.layers, WL.channels) /
                       (st["coarse_ms"] * 1e-3) / 1e12) if st["coarse_ms"] else 0.0
        line = {
            "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": ms, "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "f32", "data": "synthetic",
            "config": {"workload": WL.name if M == 1 else f"{WL.name}, G composed {M}x per slice",
                       "n": WL.n, "problems": WL.problems, "slices": slices,
                       "steps_per_slice": steps, "coarse_substeps": M, "variant": "mass-conserving", "conv": "1-32x6-1 gelu bf16, mACNN mass shift",
                       "tol": WL.tol, "coarse_weights": wsrc,
                       "l2": "state larger than L2 (trajectories, stored G and F values: 0.54 GB)",
                       "parallelism": f"replicas x{world}", "cuda_graphs": not args.no_graphs},
            "iterations": its, "final_rel_l2": l2,
            "tol_reached": bool(all(r < WL.tol and k < slices for k, r in zip(its, l2))),
            "problems_stopped_at_k_eq_s": int(sum(1 for k in its if k >= slices)),
            "sequential_ms": seq_ms, "sequential_fine_shape": seq_shape_name, "parareal_ms": ms,
            "speedup_vs_sequential": seq_ms / ms,
            "phase_ms_per_solve": {"fine": st["fine_ms"] / args.steps, "coarse": st["coarse_ms"] / args.steps,
                                   "increment": st["increment_ms"] / args.steps},
            "fine_cell_steps_per_s": st["fine_cell_steps"] / (st["fine_ms"] * 1e-3) if st["fine_ms"] else None,
            "conv_tflops": conv_tflops,
            "roofline": {"bound": "alu", "kernel": "fine_field_kernel", "achieved": fine_tflops,
                         "peak": peak, "unit": "TFLOP/s", "frac": fine_tflops / peak,
                         # the counters were taken on the asynchronous-exchange launch shape (2 CTAs
                         # per SM); the default shape has changed since (no exchange buffer, 3 CTAs per
                         # SM) and was not captured again
                         "traffic": None,
                         "traffic_earlier_shape": fine_traffic_per_launch(st, WL, steps),
                         "traffic_unit": "bytes per launch (ncu DRAM bytes per field-slice x field-slices per launch)",
                         "traffic_note": "null: the DRAM counters (433.6 KB per field-slice, 512 KB algorithmic) "
                                         "are of the asynchronous-exchange launch shape, not of the current "
                                         "default (no exchange buffer, 3 CTAs per SM); traffic_earlier_shape "
                                         "scales them to this run's launches",
                         "peak_source": f"FP32 lanes x 2 x sm_max_mhz {sm_mhz:.0f} from {src} peaks",
                         "flops_per_cell_step": fpc},
            "cpu_baseline": cpu,
            "cpu_baseline_1core": cpu1,
            "cost_model": cost_model(st, seq_ms, its, args.steps, slices, steps, M),
            "e2e": {"value": job_rate(cells, e2e_ms, world), "unit": UNIT,
                    "h2d_bytes_per_step": int(host_u0.numel() * 4), "d2h_bytes_per_step": int(host_out.numel() * 4)},
            "gpu_launches": int(launches),
            "clocks": clocks,
        }
        print(json.dumps(line), flush=True)
    pr.close()
    if world > 1:
        dist.destroy_process_group()


if __name__ == "__main__":
    main()
