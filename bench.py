#!/usr/bin/env python
"""Benchmark: MASE solves/s on the 9241-bus, 32-area, 64-snapshot workload.

One step = one full multi-area Gauss-Newton solve of a batch of 64
snapshots (every GN iteration: templated evaluation, fused accumulation,
per-area Schur condensation, boundary assembly/solve, back-substitution)
through the library's C ABI.  value = snapshots solved per second, summed
over ranks.  Inputs are synthetic (seeded generator; z = h(x_true) + e with
h evaluated by the library's measurement kernel).

  python bench.py [--gpus N] [--steps K] [--warmup W] [--impl reference]

Rank 0 prints one JSON line.  Under torchrun every rank solves its own
replica of the workload (the path is replicated, not sharded).
"""
from __future__ import annotations

import argparse
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

METRIC = "MASE solves/s, 9241-bus x64 snapshots, vs plain FP64 GPU path at 1e-6 state err"
UNIT = "solves/s"
WORKLOAD = "grid9241_k32"
N_SNAP = 64
STATE_SEED, NOISE_SEED = 2002, 2003
TOL, MAX_ITER = 1e-8, 10
WORKLOAD_DESC = "9241-bus/16049-branch synthetic grid, 32 areas (150-450 buses), 64-snapshot random walk"


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=10)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--cpu-sample", type=int, default=4, help="snapshots in the oracle sample")
    ap.add_argument("--comparator-steps", type=int, default=3)
    ap.add_argument("--workload", default=WORKLOAD, help="grid shape (smaller ones for profiling)")
    ap.add_argument("--train-samples", type=int, default=32768,
                    help="estimator-solved snapshots for the warm-start networks (0: flat start)")
    ap.add_argument("--train-epochs", type=int, default=40)
    ap.add_argument("--snapshots", type=int, default=N_SNAP)
    ap.add_argument("--family", default="", choices=["", "Pf", "Qf", "Pt", "Qt", "Pinj", "Qinj", "Vm"],
                    help="drop one whole measurement family from every snapshot")
    ap.add_argument("--areas", type=int, default=0,
                    help="draw the workload's grid with this many areas instead (sweeps)")
    return ap.parse_args()


# ---------------------------------------------------------------------------
# distributed plumbing (barrier + max over ranks only; no data-path collective)
# ---------------------------------------------------------------------------
class Dist:
    def __init__(self, n):
        self.rank = int(os.environ.get("RANK", 0))
        self.world = int(os.environ.get("WORLD_SIZE", 1))
        self.local = int(os.environ.get("LOCAL_RANK", 0))
        self.pg = None
        if self.world > 1:
            import torch
            import torch.distributed as dist
            backend = "nccl" if torch.cuda.is_available() else "gloo"
            if backend == "nccl":
                torch.cuda.set_device(self.local)
            dist.init_process_group(backend)
            self.pg = dist

    def barrier(self):
        if self.pg:
            if self.pg.get_backend() == "nccl":
                import torch
                self.pg.barrier(device_ids=[torch.cuda.current_device()])
            else:
                self.pg.barrier()

    def max(self, v: float) -> float:
        if not self.pg:
            return v
        import torch
        dev = "cuda" if self.pg.get_backend() == "nccl" else "cpu"
        t = torch.tensor([v], dtype=torch.float64, device=dev)
        self.pg.all_reduce(t, op=self.pg.ReduceOp.MAX)
        return float(t.item())

    def close(self):
        if self.pg:
            self.pg.destroy_process_group()


# ---------------------------------------------------------------------------
# clocks during the timed region
# ---------------------------------------------------------------------------
class ClockSampler:
    Q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
         "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
         "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, device_index: int):
        self.dev = device_index
        self.proc = None
        self.path = None

    def start(self):
        try:
            fd, self.path = tempfile.mkstemp(suffix=".csv")
            os.close(fd)
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.dev), f"--query-gpu={self.Q}", "--format=csv,noheader,nounits",
                 "-lms", "200"], stdout=open(self.path, "w"), stderr=subprocess.DEVNULL)
        except Exception:
            self.proc = None

    def stop(self):
        if not self.proc:
            return None
        time.sleep(0.25)
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except Exception:
            self.proc.kill()
        rows = []
        for line in open(self.path):
            p = [x.strip() for x in line.split(",")]
            if len(p) < 9:
                continue
            try:
                rows.append((float(p[1]), float(p[2]), p[5], p[6], p[7], p[8]))
            except ValueError:
                continue
        os.unlink(self.path)
        if not rows:
            return None
        reasons = set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for r in rows:
            for n, v in zip(names, r[2:]):
                if v.lower().startswith("active"):
                    reasons.add(n)
        return {"sm_mhz": statistics.median(r[0] for r in rows), "sm_max_mhz": max(r[1] for r in rows),
                "samples": len(rows), "reasons": sorted(reasons)}


# ---------------------------------------------------------------------------
# workload
# ---------------------------------------------------------------------------
def workload_inputs(args):
    from paper_2604_23175_gb300 import synth
    if args.areas:
        # the workload's bus and branch counts drawn with another number of
        # areas, sizes scaled like the 32-area case (150-450 buses, mean 289)
        base = synth.SPECS[args.workload]
        mean = base.n_bus / args.areas
        spec = synth.GridSpec(f"{base.name}_k{args.areas}", base.n_bus, base.n_branch, args.areas,
                              max(8, round(0.52 * mean)), round(1.56 * mean), base.ties_lo,
                              base.ties_hi, base.extra_pairs, seed=base.seed)
        g = synth.make_grid(spec)
    else:
        g = synth.make_grid(args.workload)
    Vm, Va = synth.make_states(g, args.snapshots, STATE_SEED)
    e = synth.make_noise(g, args.snapshots, NOISE_SEED)
    sig = synth.sigma_vector(g.n_bus, g.n_branch)
    return g, Vm, Va, e, sig


def measured_peaks():
    try:
        return json.load(open(os.path.join(ROOT, "MEASURED_PEAKS.json")))
    except Exception:
        return {}


def gemm_rate(torch, dtype, n=4096, reps=5):
    """Measured dense GEMM rate (TFLOP/s) of cuBLAS in the given dtype."""
    a = torch.randn(n, n, device="cuda", dtype=dtype)
    b = torch.randn(n, n, device="cuda", dtype=dtype)
    torch.matmul(a, b)
    torch.cuda.synchronize()
    best = 1e30
    for _ in range(reps):
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record()
        torch.matmul(a, b)
        e1.record()
        torch.cuda.synchronize()
        best = min(best, e0.elapsed_time(e1))
    del a, b
    return 2.0 * n ** 3 / (best * 1e-3) / 1e12


def time_steps(torch, fn, steps, warmup, flush):
    for _ in range(warmup):
        fn()
    torch.cuda.synchronize()
    times = []
    for _ in range(steps):
        flush()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record()
        fn()
        e1.record()
        torch.cuda.synchronize()
        times.append(e0.elapsed_time(e1))
    return times


def kernel_op_counts(g, info):
    """Algorithmic work of one launch of the area kernel for one snapshot.

    FP64 operations per owned branch end (two per branch): flows (16),
    residuals and objective (6), partials (12), gradient weights and scatter
    (16), recomputed trigonometric combinations (16): 66; per bus: injection
    sums and residuals (12).  FP32 multiply-adds: the symbolic factor's count
    plus 2 per gain-matrix update.
    """
    ends = 2 * g.n_branch
    fp64 = 66 * ends + 12 * g.n_bus
    fp32_fma = info["local_flops"] + 2 * info["g_updates"]
    return fp64, fp32_fma


def run_ours(args, dist):
    import torch
    from paper_2604_23175_gb300 import mase

    if not torch.cuda.is_available():
        raise SystemExit("bench needs a CUDA device")
    import __graft_entry__
    __graft_entry__.build()
    dev = dist.local if dist.world > 1 else 0
    torch.cuda.set_device(dev)
    g, Vm, Va, e, sig = workload_inputs(args)
    N = g.n_bus
    N_SNAP = args.snapshots
    # measurements z = h(x_true) + e, h by the library's measurement kernel
    x_true = torch.tensor(np.concatenate([Vm, Va], axis=1), device="cuda")
    z_dev = torch.empty((N_SNAP, g.n_meas), dtype=torch.float64, device="cuda")
    stream = torch.cuda.current_stream().cuda_stream
    est = mase.Estimator(g, sig, N_SNAP, z=None, precision=mase.MIXED, schedule=mase.BATCHED,
                         use_graph=True, refine=1, device=dev, stream=stream, profile=True)
    est.measure(x_true, z_dev)
    z_dev += torch.tensor(e, device="cuda")
    z_host = z_dev.cpu().numpy().copy()
    mask_dev, mask_pin = None, None
    if args.family:
        from paper_2604_23175_gb300 import synth
        mh = synth.family_mask(g, args.family, N_SNAP)
        mask_dev = torch.tensor(mh, device="cuda")
        mask_pin = torch.from_numpy(mh).pin_memory()
    est.set_measurements(z_dev, mask_dev)
    info = est.info()
    x_dev = torch.zeros((N_SNAP, 2 * N), dtype=torch.float64, device="cuda")
    flush_buf = torch.empty(256 * 1024 * 1024 // 4, dtype=torch.float32, device="cuda")

    def flush():
        flush_buf.zero_()

    last = {}

    def step():
        est.set_measurements(z_dev, mask_dev)
        last["r"] = est.solve(tol=TOL, max_iter=MAX_ITER, x_out=x_dev)

    # ---- learned warm start (untimed set-up): train the per-area networks on
    # independent snapshots solved by the estimator itself (seeds disjoint from
    # the benchmark batch)
    warm = {"trained": False}
    if args.train_samples >= 256:
        t0 = time.perf_counter()
        from paper_2604_23175_gb300 import synth
        Zs, Xs = [], []
        nb = args.train_samples // N_SNAP
        for b in range(nb):
            Vt, At = synth.make_states(g, N_SNAP, 30000 + 7 * b, walk_len=1)
            et = synth.make_noise(g, N_SNAP, 30001 + 7 * b)
            zt = torch.empty((N_SNAP, g.n_meas), dtype=torch.float64, device="cuda")
            est.measure(torch.tensor(np.concatenate([Vt, At], 1), device="cuda"), zt)
            zt += torch.tensor(et, device="cuda")
            est.set_measurements(zt)
            xt = torch.zeros((N_SNAP, 2 * N), dtype=torch.float64, device="cuda")
            est.solve(tol=TOL, max_iter=MAX_ITER, x_out=xt)
            Zs.append(zt)
            Xs.append(xt)
        t1 = time.perf_counter()
        loss = est.warmstart_train(torch.cat(Zs), torch.cat(Xs), epochs=args.train_epochs, batch=256, lr=1e-3)
        torch.cuda.synchronize()
        t2 = time.perf_counter()
        del Zs, Xs
        warm = {"trained": True, "samples": nb * N_SNAP, "epochs": args.train_epochs,
                "final_loss": loss, "data_s": t1 - t0, "train_s": t2 - t1}
        est.set_measurements(z_dev, mask_dev)
        # iterations from the flat, previous-snapshot and learned starts
        rf = est.solve(tol=TOL, max_iter=MAX_ITER, x_out=x_dev)
        x_flat = x_dev.clone()
        x0 = x_flat.clone()
        x0[1:] = x_flat[:-1]
        x0[0, :N] = 1.0
        x0[0, N:] = 0.0
        rp = est.solve(x0=x0, tol=TOL, max_iter=MAX_ITER, x_out=x_dev)
        est.set_start_mode(mase.START_LEARNED)
        rl = est.solve(tol=TOL, max_iter=MAX_ITER, x_out=x_dev)
        warm.update({"iters_flat": float(rf.iters.mean()), "iters_prev": float(rp.iters.mean()),
                     "iters_learned": float(rl.iters.mean()),
                     "max_state_diff_learned_vs_flat": float((x_dev - x_flat).abs().max().item())})
        # value with the flat start, same timing rules, for comparison
        est.set_start_mode(mase.START_FLAT)
        tf = time_steps(torch, step, max(3, args.steps // 2), 2, flush)
        warm["value_flat_start"] = dist.world * N_SNAP / (dist.max(float(np.mean(tf))) * 1e-3)
        est.set_start_mode(mase.START_LEARNED)

    # ---- timed region (device-resident inputs)
    for _ in range(args.warmup):
        step()
    torch.cuda.synchronize()
    dist.barrier()
    torch.cuda.synchronize()
    clocks = ClockSampler(torch.cuda.current_device())
    clocks.start()
    times, stages, launches, iters, steps_run = [], np.zeros(4), 0, [], 0
    for _ in range(args.steps):
        flush()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record()
        step()
        e1.record()
        torch.cuda.synchronize()
        times.append(e0.elapsed_time(e1))
        r = last["r"]
        stages += np.array(r.stage_ms)
        launches += r.launches + 1            # + the measurement-layout gather
        iters.append(r.iters.copy())
        steps_run += r.steps
    dist.barrier()
    torch.cuda.synchronize()
    clk = clocks.stop()
    ms = float(np.mean(times))
    ms_max = dist.max(ms)
    value = dist.world * N_SNAP / (ms_max * 1e-3)
    res = last["r"]
    x_mixed = x_dev.cpu().numpy().copy()

    # ---- end to end through host buffers
    x_host = np.zeros((N_SNAP, 2 * N))
    pin_z = torch.from_numpy(z_host).pin_memory()
    pin_x = torch.zeros((N_SNAP, 2 * N), dtype=torch.float64).pin_memory()

    def step_e2e():
        est.set_measurements(pin_z, mask_pin)
        est.solve(tol=TOL, max_iter=MAX_ITER, x_out=pin_x)

    e2e_times = time_steps(torch, step_e2e, max(3, args.steps // 2), 2, flush)
    e2e_ms = dist.max(float(np.mean(e2e_times)))
    x_host[:] = pin_x.numpy()

    # ---- comparator: plain FP64 per-area pipeline, same GPU
    cmp = mase.Estimator(g, sig, N_SNAP, z=z_dev, precision=mase.FP64, schedule=mase.PER_AREA,
                         use_graph=False, device=dev, stream=stream)
    x_fp64 = torch.zeros_like(x_dev)
    cres = {}

    def step_cmp():
        cmp.set_measurements(z_dev, mask_dev)
        cres["r"] = cmp.solve(tol=TOL, max_iter=MAX_ITER, x_out=x_fp64)

    if args.comparator_steps > 0:
        cmp_times = time_steps(torch, step_cmp, args.comparator_steps, 1, flush)
        cmp_ms = dist.max(float(np.mean(cmp_times)))
    else:
        step_cmp()
        cmp_ms = float("nan")
    x_fp64_h = x_fp64.cpu().numpy()
    cmp.close()

    # ---- roofline of the dominant kernel (area kernel), timed in the region above
    n_local = steps_run                       # one batched launch per GN step
    local_ms = stages[0] / max(1, n_local)
    fp64_ops, fp32_fma = kernel_op_counts(g, info)
    active = np.mean([np.mean(it >= 1) for it in iters])
    fp64_per_launch = fp64_ops * N_SNAP
    fp64_rate = gemm_rate(torch, torch.float64, 4096, 3)
    torch.backends.cuda.matmul.allow_tf32 = False
    fp32_rate = gemm_rate(torch, torch.float32, 8192, 3)
    achieved = fp64_per_launch / (local_ms * 1e-3) / 1e12
    roof = {"kernel": "k_local (evaluation + fused accumulation + Schur condensation)",
            "bound": "alu", "unit": "TFLOP/s",
            "achieved": achieved, "peak": fp64_rate, "frac": achieved / fp64_rate,
            "peak_source": "measured cuBLAS DGEMM in this run (FP64 pipe)",
            "traffic": None,
            "avg_launch_ms": local_ms,
            "fp32_fma_per_launch": fp32_fma * N_SNAP,
            "fp32_tflops_achieved": 2 * fp32_fma * N_SNAP / (local_ms * 1e-3) / 1e12,
            "fp32_peak_tflops": fp32_rate, "fp64_ops_per_launch": fp64_per_launch}
    try:
        prof = json.load(open(os.path.join(ROOT, "profiles", "k_local_traffic.json")))
        if prof.get("kernel_hash") == kernel_hash():
            roof["traffic"] = prof["bytes_per_launch_full_size"]
    except Exception:
        pass

    # the headline workload, or a sweep / profiling variant of it
    variant = bool(args.workload != WORKLOAD or N_SNAP != 64 or args.areas or args.family)
    out = {
        "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": dist.world,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": ms_max,
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
        "dtype": "f32+f64", "data": "synthetic",
        "config": {"workload": WORKLOAD_DESC if not variant else
                   f"{g.name} x{N_SNAP} snapshots" + (f", {args.family} rows dropped" if args.family else ""),
                   "n_bus": g.n_bus, "n_branch": g.n_branch,
                   "n_area": g.n_area, "n_snap": N_SNAP, "precision": "mixed (FP32 gain/factor/Schur/solves, FP64 residual/gradient/boundary refinement/update)",
                   "schedule": "batched, CUDA graph per iteration",
                   "start": "learned (per-area MLP, judged against flat by J)" if warm["trained"] else "flat",
                   "tol": TOL, "max_iter": MAX_ITER, "l2": "flushed between steps (256 MB write)",
                   "parallelism": f"replicas x{dist.world}"},
        "comparator": {"impl": "plain FP64 per-area GPU pipeline (same library, one launch per area and stage)",
                       "value": dist.world * N_SNAP / (cmp_ms * 1e-3), "ms_per_step": cmp_ms,
                       "iters_mean": float(np.mean(cres["r"].iters)),
                       "speedup_of_value": (dist.world * N_SNAP / (ms_max * 1e-3)) / (dist.world * N_SNAP / (cmp_ms * 1e-3))},
        "iters": {"mean": float(np.mean(res.iters)), "max": int(res.iters.max())},
        "warm_start": warm,
        "accuracy": {"max_state_diff_vs_fp64_gpu": float(np.max(np.abs(x_mixed - x_fp64_h))),
                     "all_converged": bool(np.all(res.status == 0))},
        "stages_ms_per_step": {"area": stages[0] / args.steps, "boundary": stages[1] / args.steps,
                               "back": stages[2] / args.steps, "bookkeeping": stages[3] / args.steps},
        "roofline": roof,
        "e2e": {"value": dist.world * N_SNAP / (e2e_ms * 1e-3), "unit": UNIT,
                "h2d_bytes_per_step": int(z_host.nbytes) + (int(mask_pin.numel()) if mask_pin is not None else 0),
                "d2h_bytes_per_step": int(x_host.nbytes),
                "ms_per_step": e2e_ms},
        "gpu_launches": launches,
        "clocks": clk,
        "info": info,
    }
    est.close()
    return out, x_mixed, (Vm, Va, e, sig, g)


def oracle_sample(n: int, nthreads: int = 1):
    """Time the CPU oracle on the first n snapshots of the workload in a child
    process with single-threaded math libraries; returns (seconds, x[n,2N])."""
    code = r"""
import sys, time, json, numpy as np
sys.path.insert(0, %r)
from oracle import wls
from paper_2604_23175_gb300 import synth
g = synth.make_grid(%r)
Vm, Va = synth.make_states(g, %d, %d)
e = synth.make_noise(g, %d, %d)
sig = synth.sigma_vector(g.n_bus, g.n_branch)
net = wls.Net(g.n_bus, g.from_bus.astype(np.int64), g.to_bus.astype(np.int64), g.r, g.x, g.b_charge, g.slack)
n = %d
z = [wls.measure(net, Vm[s], Va[s]) + e[s] for s in range(n)]
w = wls.weights(sig)
t = time.perf_counter()
res = [wls.gauss_newton(net, z[s], w, tol=%r, max_iter=%d) for s in range(n)]
dt = time.perf_counter() - t
x = np.stack([np.concatenate([r.Vm, r.Va]) for r in res])
np.save(sys.argv[1], x)
print(json.dumps({"seconds": dt, "iters": [r.iters for r in res], "J": [r.J for r in res]}))
""" % (ROOT, WORKLOAD, N_SNAP, STATE_SEED, N_SNAP, NOISE_SEED, n, TOL, MAX_ITER)
    env = dict(os.environ)
    for k in ("OMP_NUM_THREADS", "OPENBLAS_NUM_THREADS", "MKL_NUM_THREADS"):
        env[k] = str(nthreads)
    fd, path = tempfile.mkstemp(suffix=".npy")
    os.close(fd)
    r = subprocess.run([sys.executable, "-c", code, path], capture_output=True, text=True, env=env,
                       timeout=1800)
    if r.returncode != 0:
        raise RuntimeError(r.stderr[-2000:])
    info = json.loads(r.stdout.strip().splitlines()[-1])
    x = np.load(path)
    os.unlink(path)
    return info, x


def kernel_hash() -> str:
    """Hash of the device code with comments and blank lines removed, so that
    recorded counters stay attached to the code they were taken on."""
    import hashlib
    import re
    h = hashlib.sha256()
    for f in ("kernels.cuh",):
        src = open(os.path.join(ROOT, "paper_2604_23175_gb300", "csrc", f)).read()
        src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
        lines = [ln.split("//", 1)[0].rstrip() for ln in src.splitlines()]
        h.update("\n".join(ln for ln in lines if ln.strip()).encode())
    return h.hexdigest()[:16]


def run_reference(args, dist):
    """The oracle as the reference arm: each step solves a bounded sample of
    the workload's snapshots on the host cores."""
    if dist.rank != 0:
        return None
    n = 2
    times = []
    for i in range(args.warmup + args.steps):
        info, _ = oracle_sample(n)
        if i >= args.warmup:
            times.append(info["seconds"])
    sec = float(np.mean(times))
    v = n / sec
    return {"impl": "reference", "metric": METRIC, "value": v, "unit": UNIT, "n_gpus": dist.world,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": sec * 1e3,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
            "data": "synthetic",
            "config": {"workload": WORKLOAD_DESC, "n_snap_per_step": n, "tol": TOL, "max_iter": MAX_ITER},
            "cpu_baseline": {"value": v, "unit": UNIT, "cores": 1, "kind": "oracle",
                             "sample": f"first {n} of the 64 snapshots per step, centralised FP64 Gauss-Newton (SciPy sparse LU), 1 thread"},
            "e2e": {"value": v, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}


def main():
    args = parse()
    dist = Dist(args.gpus)
    if args.impl == "reference":
        out = run_reference(args, dist)
        if dist.rank == 0:
            print(json.dumps(out))
        dist.close()
        return
    out, x_mixed, (Vm, Va, e, sig, g) = run_ours(args, dist)
    if dist.rank == 0:
        if not args.no_cpu_baseline:
            n = args.cpu_sample
            info, x_or = oracle_sample(n)
            N = g.n_bus
            err = float(np.max(np.abs(x_mixed[:n] - x_or)))
            out["cpu_baseline"] = {"value": n / info["seconds"], "unit": UNIT, "cores": 1,
                                   "kind": "oracle",
                                   "sample": f"first {n} of the 64 snapshots, centralised FP64 Gauss-Newton (SciPy sparse LU), 1 thread",
                                   "seconds": info["seconds"]}
            out["accuracy"]["max_state_err_vs_oracle_sample"] = err
            out["accuracy"]["oracle_iters"] = info["iters"]
        else:
            out["cpu_baseline"] = None
        print(json.dumps(out))
    dist.close()


if __name__ == "__main__":
    main()
