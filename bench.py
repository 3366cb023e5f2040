#!/usr/bin/env python
"""Benchmark: MASE solves/s on the 9241-bus, 32-area, 64-snapshot workload.

One step = one full multi-area Gauss-Newton solve of a batch of 64
snapshots (every GN iteration: templated evaluation, fused accumulation,
per-area Schur condensation, boundary assembly/solve, back-substitution)
through the library's C ABI, preceded by handing the step's measurements to
the library.  value = snapshots solved per second, summed over ranks.
Inputs are synthetic (seeded generator; z = h(x_true) + e with h evaluated by
the library's measurement kernel).

The timed legs - flat and learned start, each with device-resident inputs
and end to end through pinned host buffers - are interleaved over several
rounds with the clock sampler running across all of them; the headline is
the faster start, and every leg reports its median and spread.

  python bench.py [--gpus N] [--steps K] [--warmup W] [--impl reference]

Rank 0 prints one JSON line.  Under torchrun every rank solves its own
replica of the workload (the path is replicated, not sharded).
"""
from __future__ import annotations

import argparse
import json
import os
import platform
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
STATE_SEED, NOISE_SEED, MASK_SEED = 2002, 2003, 2004
TOL, MAX_ITER = 1e-8, 10
WORKLOAD_DESC = "9241-bus/16049-branch synthetic grid, 32 areas (150-450 buses), 64-snapshot random walk"
STAGES = ("area", "coordinator", "back", "bookkeeping", "learned_start", "start_finish", "loop_gaps")


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=10)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--repeats", type=int, default=3, help="rounds the timed legs are interleaved over")
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--cpu-sample", type=int, default=4, help="snapshots of the 1-thread oracle sample")
    ap.add_argument("--comparator-steps", type=int, default=3)
    ap.add_argument("--workload", default=WORKLOAD, help="grid shape (smaller ones for profiling)")
    ap.add_argument("--train-samples", type=int, default=32768,
                    help="estimator-solved snapshots for the warm-start networks (0: flat start)")
    ap.add_argument("--train-epochs", type=int, default=40)
    ap.add_argument("--snapshots", type=int, default=N_SNAP)
    ap.add_argument("--family", default="", choices=["", "Pf", "Qf", "Pt", "Qt", "Pinj", "Qinj", "Vm"],
                    help="drop one whole measurement family from every snapshot")
    ap.add_argument("--drop", type=float, default=0.0,
                    help="fraction of measurement rows dropped at random per snapshot")
    ap.add_argument("--areas", type=int, default=0,
                    help="split the workload's network into this many areas with the partitioner")
    ap.add_argument("--max-iter", type=int, default=MAX_ITER,
                    help="Gauss-Newton step cap per snapshot")
    ap.add_argument("--tensor-units", type=int, default=-1,
                    help="update units of panels at least this wide on the tensor cores (3xTF32); "
                         "0 = none, -1 = the library default")
    ap.add_argument("--inner-iters", type=int, default=0,
                    help="local Gauss-Newton steps per area with the boundary fixed before each condensed step")
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
def workload_grid(args):
    from paper_2604_23175_gb300 import synth
    g = synth.make_grid(args.workload)
    if args.areas:
        # the same network split into another number of areas
        g = synth.partition_network(g, args.areas)
    return g


def workload_inputs(args):
    from paper_2604_23175_gb300 import synth
    g = workload_grid(args)
    Vm, Va = synth.make_states(g, args.snapshots, STATE_SEED)
    e = synth.make_noise(g, args.snapshots, NOISE_SEED)
    sig = synth.sigma_vector(g.n_bus, g.n_branch)
    return g, Vm, Va, e, sig


def workload_desc(args, g, S):
    """Name of the workload a run times: the benchmark's own, or the variant
    the flags select."""
    variant = bool(args.workload != WORKLOAD or S != N_SNAP or args.areas or args.family or args.drop
                   or args.inner_iters or args.tensor_units >= 0)
    if not variant:
        return WORKLOAD_DESC
    return (f"{g.name} x{S} snapshots" + (f", {args.family} rows dropped" if args.family else "")
            + (f", {100 * args.drop:g}% rows dropped at random" if args.drop else "")
            + (f", {args.inner_iters} inner local steps" if args.inner_iters else "")
            + (f", tensor-core update units from panel width {args.tensor_units}"
               if args.tensor_units > 0 else ""))


def workload_mask(args, g):
    """Presence mask [S][m] of the workload's measurement rows, or None."""
    from paper_2604_23175_gb300 import synth
    if args.family:
        return synth.family_mask(g, args.family, args.snapshots)
    if args.drop > 0:
        return synth.make_mask(g, args.snapshots, args.drop, MASK_SEED)
    return None


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


def measured_hbm_peak():
    try:
        return float(json.load(open(os.path.join(ROOT, "MEASURED_PEAKS.json")))["hbm_gbs"]), "measured"
    except Exception:
        return 6800.0, "fallback"


N_SM = 152
FP64_FMA_PER_SM_CYCLE = 2   # 1.25 TFLOP/s nominal FP64 / (152 SMs x 2.07 GHz x 2 flops)


def fp64_alu_peak_tflops():
    """FP64 peak from unit counts and clocks: SMs x FP64 FMAs per SM cycle x
    2 flops x the maximum SM clock (the pool's measured value, else 2070 MHz).
    Returns (TFLOP/s, description)."""
    try:
        mhz = float(json.load(open(os.path.join(ROOT, "MEASURED_PEAKS.json")))["sm_max_mhz"])
    except Exception:
        mhz = 2070.0
    peak = N_SM * FP64_FMA_PER_SM_CYCLE * 2 * mhz * 1e6 / 1e12
    return peak, f"derived: {N_SM} SMs x {FP64_FMA_PER_SM_CYCLE} FP64 FMA/cycle x 2 flops x {mhz:g} MHz"


def headline_roofline(lo, alu_peak, alu_src, dgemm_rate, traffic):
    """The dominant kernel's roofline entry: the area kernel's algorithmic
    FP64 rate against the FP64 ALU peak, with the measured DGEMM beside it."""
    return {"kernel": "k_local (evaluation + fused accumulation + Schur condensation)",
            "bound": "alu", "unit": "TFLOP/s",
            "achieved": lo["fp64_tflops"], "peak": alu_peak, "frac": lo["fp64_tflops"] / alu_peak,
            "peak_source": alu_src,
            "peak_measured_dgemm": dgemm_rate, "frac_of_measured_dgemm": lo["fp64_tflops"] / dgemm_rate,
            "traffic": traffic, "avg_launch_ms": lo["avg_launch_ms"],
            "timing": "CUDA events around each launch on the library's stream (host-stepped profiling pass, flat start)"}


def stage_work(g, info, n_snap):
    """Algorithmic work of one launch of each stage kernel over n_snap
    active snapshots (bytes that must cross HBM once, and arithmetic).

    Area kernel: FP64 operations per owned branch end (two per branch): flows
    (16), residuals and objective (6), partials (12), gradient weights and
    scatter (16), recomputed trigonometric combinations (16): 66; per bus:
    injection sums and residuals (12).  FP32 multiply-adds: the symbolic
    factor's count plus 2 per gain-matrix update.  Bytes: z and the bus
    states read, the factor storage, the forward-solved interior rhs (FP32)
    and the condensed boundary rhs (FP64) written.
    Coordinator: the Schur blocks and condensed rhs read, the assembled
    system written once for the refinement, boundary step and state updated;
    FP32 multiply-adds of the boundary factor plus its two solves per sweep,
    FP64 residual of one refinement sweep.
    Back-substitution: the factor storage and interior rhs read, the state
    read and written; one FP32 multiply-add per stored factor entry.
    """
    S = n_snap
    n_int = info["n_state"] - info["n_gamma"]
    ends = 2 * g.n_branch
    local = {
        "bytes": S * (8 * g.n_meas + 16 * g.n_bus + 4 * info["factor_nnz"] + 4 * n_int
                      + 8 * info["coord_b_elems"]),
        "fp64_ops": S * (66 * ends + 12 * g.n_bus),
        "fp32_fma": S * (info["local_flops"] + 2 * info["g_updates"]),
    }
    bstore = info["boundary_store"]
    coord = {
        "bytes": S * (4 * info["coord_S_elems"] + 8 * info["coord_b_elems"] + 4 * bstore
                      + 8 * info["n_gamma"] * 3),
        "fp64_ops": S * 2 * (2 * bstore),
        "fp32_fma": S * (info["boundary_flops"] + 2 * 2 * bstore),
    }
    back = {
        "bytes": S * (4 * info["factor_nnz"] + 4 * n_int + 8 * info["n_gamma"] + 32 * g.n_bus),
        "fp64_ops": S * 2 * n_int,
        "fp32_fma": S * info["factor_nnz"],
    }
    return {"k_local": local, "k_boundary_cl": coord, "k_back": back}


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


def _split(k: int, r: int) -> list[int]:
    return [k // r + (1 if i < k % r else 0) for i in range(r)]


def run_ours(args, dist):
    import torch
    from paper_2604_23175_gb300 import mase, synth

    if not torch.cuda.is_available():
        raise SystemExit("bench needs a CUDA device")
    import __graft_entry__
    __graft_entry__.build()
    dev = dist.local if dist.world > 1 else 0
    torch.cuda.set_device(dev)
    g, Vm, Va, e, sig = workload_inputs(args)
    N = g.n_bus
    S = args.snapshots
    # measurements z = h(x_true) + e, h by the library's measurement kernel
    x_true = torch.tensor(np.concatenate([Vm, Va], axis=1), device="cuda")
    z_dev = torch.empty((S, g.n_meas), dtype=torch.float64, device="cuda")
    stream = torch.cuda.current_stream().cuda_stream
    est = mase.Estimator(g, sig, S, z=None, precision=mase.MIXED, schedule=mase.BATCHED,
                         use_graph=True, refine=1, device=dev, stream=stream, inner_iters=args.inner_iters,
                         tensor_units=args.tensor_units)
    est.measure(x_true, z_dev)
    z_dev += torch.tensor(e, device="cuda")
    z_host = z_dev.cpu().numpy().copy()
    mask_dev, mask_pin = None, None
    mask_h = workload_mask(args, g)
    if mask_h is not None:
        mask_dev = torch.tensor(mask_h, device="cuda")
        mask_pin = torch.from_numpy(mask_h).pin_memory()
    est.set_measurements(z_dev, mask_dev)
    info = est.info()
    x_dev = torch.zeros((S, 2 * N), dtype=torch.float64, device="cuda")
    flush_buf = torch.empty(256 * 1024 * 1024 // 4, dtype=torch.float32, device="cuda")

    def flush():
        flush_buf.zero_()

    # ---- learned warm start (untimed set-up): train the per-area networks on
    # independent snapshots solved by the estimator itself (seeds disjoint from
    # the benchmark batch)
    warm = {"trained": False}
    if args.train_samples >= 256:
        t0 = time.perf_counter()
        Zs, Xs = [], []
        nb = max(1, args.train_samples // S)
        # training snapshots see the benchmark's kind of drops: under random
        # drops each training batch draws its own masks (four batches of
        # masks, reused in turn), is solved under them and trains the
        # networks with them; a family mask is the same for every batch.
        # Snapshots that do not converge are left out of the training set.
        all_rows = torch.ones((S, g.n_meas), dtype=torch.uint8, device="cuda") if mask_dev is not None else None
        train_masks = []
        if mask_dev is not None and not args.family:
            train_masks = [torch.tensor(synth.make_mask(g, S, args.drop, 40000 + 7 * b), device="cuda")
                           for b in range(min(nb, 4))]
        elif mask_dev is not None:
            train_masks = [mask_dev]
        Ms = []
        left_out = 0
        for b in range(nb):
            Vt, At = synth.make_states(g, S, 30000 + 7 * b, walk_len=1)
            et = synth.make_noise(g, S, 30001 + 7 * b)
            zt = torch.empty((S, g.n_meas), dtype=torch.float64, device="cuda")
            est.measure(torch.tensor(np.concatenate([Vt, At], 1), device="cuda"), zt)
            zt += torch.tensor(et, device="cuda")
            mt = train_masks[b % len(train_masks)] if train_masks else all_rows
            est.set_measurements(zt, mt)
            xt = torch.zeros((S, 2 * N), dtype=torch.float64, device="cuda")
            rt = est.solve(tol=TOL, max_iter=MAX_ITER, x_out=xt, check=False)
            ok = torch.tensor(rt.status == 0, device="cuda")
            left_out += int(S - int(ok.sum().item()))
            Zs.append(zt[ok])
            Xs.append(xt[ok])
            if train_masks:
                Ms.append(mt[ok])
        t1 = time.perf_counter()
        loss = est.warmstart_train(torch.cat(Zs), torch.cat(Xs), epochs=args.train_epochs, batch=256, lr=1e-3,
                                   mask=torch.cat(Ms) if Ms else None)
        torch.cuda.synchronize()
        t2 = time.perf_counter()
        del Zs, Xs, Ms
        warm = {"trained": True, "samples": nb * S - left_out, "left_out": left_out, "epochs": args.train_epochs,
                "masked_training": bool(train_masks),
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
                     "iters_max_flat": int(rf.iters.max()), "iters_max_prev": int(rp.iters.max()),
                     "iters_max_learned": int(rl.iters.max()), "flat_fallbacks_learned": rl.restarted,
                     "max_state_diff_learned_vs_flat": float((x_dev - x_flat).abs().max().item())})

    # ---- the timed legs
    pin_z = torch.from_numpy(z_host).pin_memory()
    pin_x = torch.zeros((S, 2 * N), dtype=torch.float64).pin_memory()
    starts = [("flat", mase.START_FLAT)] + ([("learned", mase.START_LEARNED)] if warm["trained"] else [])
    legs = {}
    for sname, smode in starts:
        legs[f"device_{sname}"] = (smode, False)
        legs[f"e2e_{sname}"] = (smode, True)
    rec = {k: {"ms": [], "solve_ms": [], "stages": [], "launches": 0, "iters": [], "round": [], "restarted": 0}
           for k in legs}

    def run_leg(name, n, timed, rnd=0):
        smode, e2e = legs[name]
        est.set_start_mode(smode)
        r = rec[name]
        for _ in range(n):
            flush()
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record()
            if e2e:
                est.set_measurements(pin_z, mask_pin)
                res = est.solve(tol=TOL, max_iter=MAX_ITER, x_out=pin_x)
            else:
                est.set_measurements(z_dev, mask_dev)
                res = est.solve(tol=TOL, max_iter=MAX_ITER, x_out=x_dev)
            e1.record()
            torch.cuda.synchronize()
            if timed:
                r["ms"].append(e0.elapsed_time(e1))
                r["solve_ms"].append(res.solve_ms)
                r["stages"].append(res.stage_ms)
                # + the measurement gather (and the mask gather) in set_measurements
                r["launches"] += res.launches + 1 + (1 if mask_dev is not None else 0)
                r["iters"].append(res.iters.copy())
                r["round"].append(rnd)
                r["restarted"] += res.restarted
        return res

    for name in legs:
        run_leg(name, max(3, args.warmup), False)
    torch.cuda.synchronize()
    dist.barrier()
    torch.cuda.synchronize()
    clocks = ClockSampler(torch.cuda.current_device())
    clocks.start()
    t_wall0 = time.perf_counter()
    for rnd, k in enumerate(_split(args.steps, max(1, args.repeats))):
        for name in legs:
            run_leg(name, k, True, rnd)
    torch.cuda.synchronize()
    t_wall = time.perf_counter() - t_wall0
    dist.barrier()
    torch.cuda.synchronize()
    clk = clocks.stop()

    def summary(name):
        r = rec[name]
        ms = np.array(r["ms"])
        rounds = [float(np.mean(ms[np.array(r["round"]) == i])) for i in sorted(set(r["round"]))]
        st = np.mean(np.array(r["stages"]), axis=0)
        solve = float(np.mean(r["solve_ms"]))
        mean = dist.max(float(ms.mean()))
        stages = {k: float(v) for k, v in zip(STAGES, st)}
        stages["set_measurements_and_host"] = float(ms.mean()) - solve
        return {"value": dist.world * S / (mean * 1e-3), "ms_per_step": mean,
                "ms_median": float(np.median(ms)), "ms_min": float(ms.min()), "ms_max": float(ms.max()),
                "round_means_ms": rounds,
                "spread_pct": 100.0 * (max(rounds) - min(rounds)) / float(np.median(ms)),
                "iters_mean": float(np.mean(np.concatenate(r["iters"]))),
                "iters_max": int(np.max(np.concatenate(r["iters"]))),
                "stages_ms_per_step": stages,
                "stages_sum_ms": float(st.sum()) + stages["set_measurements_and_host"],
                "solve_ms": solve, "launches_per_step": r["launches"] / len(ms),
                "flat_fallbacks_per_step": r["restarted"] / len(ms)}

    sums = {name: summary(name) for name in legs}
    # headline: the faster start with device-resident inputs
    head = min(("device_" + s for s, _ in starts), key=lambda k: sums[k]["ms_per_step"])
    head_start = head.split("_", 1)[1]
    H = sums[head]
    E = sums["e2e_" + head_start]
    res = run_leg(head, 1, False)
    x_mixed = x_dev.cpu().numpy().copy()
    if warm["trained"]:
        warm["value_flat_start"] = sums["device_flat"]["value"]
        warm["value_learned_start"] = sums["device_learned"]["value"]
        warm["learned_over_flat"] = sums["device_learned"]["value"] / sums["device_flat"]["value"]

    # ---- per-stage kernel times with CUDA events (host-stepped, flat start:
    # every launch works on all snapshots, 6 steps), for the rooflines
    prof = mase.Estimator(g, sig, S, z=z_dev, mask=mask_dev, precision=mase.MIXED,
                          schedule=mase.BATCHED, refine=1, device=dev, stream=stream, profile=True,
                          inner_iters=args.inner_iters, tensor_units=args.tensor_units)
    pst, psteps, pact = np.zeros(7), 0, []
    for i in range(1 + 3):
        flush()
        rp_ = prof.solve(tol=TOL, max_iter=MAX_ITER, x_out=x_dev)
        if i:
            pst += np.array(rp_.stage_ms)
            psteps += rp_.steps
            pact.append(float(np.mean(rp_.iters)) / max(1, rp_.steps))
    prof.close()
    per_launch = {"k_local": pst[0] / psteps, "k_boundary_cl": pst[1] / psteps, "k_back": pst[2] / psteps}
    active_frac = float(np.mean(pact))          # mean share of snapshots active per launch
    work = stage_work(g, info, S)
    fp64_rate = gemm_rate(torch, torch.float64, 4096, 3)
    torch.backends.cuda.matmul.allow_tf32 = False
    fp32_rate = gemm_rate(torch, torch.float32, 8192, 3)
    hbm, hbm_src = measured_hbm_peak()
    stage_roof = {}
    for kname, w in work.items():
        t = per_launch[kname] * 1e-3
        scale = active_frac
        stage_roof[kname] = {
            "avg_launch_ms": per_launch[kname],
            "hbm_gbs": w["bytes"] * scale / t / 1e9, "hbm_frac": w["bytes"] * scale / t / 1e9 / hbm,
            "fp64_tflops": w["fp64_ops"] * scale / t / 1e12,
            "fp64_frac": w["fp64_ops"] * scale / t / 1e12 / fp64_rate,
            "fp32_tflops": 2 * w["fp32_fma"] * scale / t / 1e12,
            "fp32_frac": 2 * w["fp32_fma"] * scale / t / 1e12 / fp32_rate,
            "algorithmic_bytes_per_launch": w["bytes"] * scale,
        }
    traffic = None
    try:
        pj = json.load(open(os.path.join(ROOT, "profiles", "k_local_traffic.json")))
        if pj.get("kernel_hash") == kernel_hash():
            traffic = pj["bytes_per_launch_full_size"]
    except Exception:
        pass
    alu_peak, alu_src = fp64_alu_peak_tflops()
    roof = headline_roofline(stage_roof["k_local"], alu_peak, alu_src, fp64_rate, traffic)

    # ---- comparator: plain FP64 per-area pipeline, same GPU
    cmp = mase.Estimator(g, sig, S, z=z_dev, mask=mask_dev, precision=mase.FP64,
                         schedule=mase.PER_AREA, use_graph=False, device=dev, stream=stream)
    x_fp64 = torch.zeros_like(x_dev)
    cres = {}
    cmp_times = []
    for i in range(1 + max(1, args.comparator_steps)):
        flush()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record()
        cmp.set_measurements(z_dev, mask_dev)
        cres["r"] = cmp.solve(tol=TOL, max_iter=MAX_ITER, x_out=x_fp64)
        e1.record()
        torch.cuda.synchronize()
        if i:
            cmp_times.append(e0.elapsed_time(e1))
    cmp_ms = dist.max(float(np.mean(cmp_times)))
    x_fp64_h = x_fp64.cpu().numpy()
    cmp.close()

    desc = workload_desc(args, g, S)
    # every kernel of the library launched inside the timed region (all legs)
    launches = sum(r["launches"] for r in rec.values())
    out = {
        "metric": METRIC, "value": H["value"], "unit": UNIT, "n_gpus": dist.world,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": H["ms_per_step"],
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
        "dtype": "f32+f64", "data": "synthetic",
        "config": {"workload": desc, "n_bus": g.n_bus, "n_branch": g.n_branch,
                   "n_area": g.n_area, "n_snap": S,
                   "precision": "mixed (FP32 gain/factor/Schur/solves, FP64 residual/gradient/boundary refinement/update)",
                   "schedule": "batched, one CUDA graph per solve with a device-side Gauss-Newton loop",
                   "start": (f"{head_start} (the faster of flat and learned in this run; both reported)"
                             if warm["trained"] else "flat"),
                   "tol": TOL, "max_iter": MAX_ITER, "l2": "flushed between steps (256 MB write)",
                   "timed_legs": f"{len(legs)} legs interleaved over {args.repeats} rounds, "
                                 f"{args.steps} steps each",
                   "parallelism": f"replicas x{dist.world}"},
        "legs": sums,
        "comparator": {"impl": "plain FP64 per-area GPU pipeline (same library, one launch per area and stage)",
                       "value": dist.world * S / (cmp_ms * 1e-3), "ms_per_step": cmp_ms,
                       "iters_mean": float(np.mean(cres["r"].iters)),
                       "speedup_of_value": H["value"] / (dist.world * S / (cmp_ms * 1e-3))},
        "iters": {"mean": H["iters_mean"], "max": H["iters_max"]},
        "warm_start": warm,
        "accuracy": {"max_state_diff_vs_fp64_gpu": float(np.max(np.abs(x_mixed - x_fp64_h))),
                     "all_converged": bool(np.all(res.status == 0))},
        "stages_ms_per_step": H["stages_ms_per_step"],
        "stages_sum_ms": H["stages_sum_ms"],
        "roofline": roof,
        "roofline_stages": stage_roof,
        "peaks": {"fp64_alu_tflops": alu_peak, "fp64_dgemm_tflops": fp64_rate, "fp32_sgemm_tflops": fp32_rate,
                  "hbm_gbs": hbm,
                  "hbm_source": hbm_src},
        "e2e": {"value": E["value"], "unit": UNIT,
                "h2d_bytes_per_step": int(z_host.nbytes) + (int(mask_pin.numel()) if mask_pin is not None else 0),
                "d2h_bytes_per_step": int(pin_x.numel() * 8),
                "ms_per_step": E["ms_per_step"], "start": head_start},
        "gpu_launches": launches,
        "clocks": clk,
        "timed_wall_s": t_wall,
        "info": info,
    }
    est.close()
    return out, x_mixed, g


# ---------------------------------------------------------------------------
# CPU baselines: the oracle on the host cores
# ---------------------------------------------------------------------------
def host_info():
    model = platform.processor() or platform.machine()
    try:
        for line in open("/proc/cpuinfo"):
            if line.lower().startswith(("model name", "cpu part", "hardware")):
                model = line.split(":", 1)[1].strip()
                break
    except Exception:
        pass
    try:
        out = subprocess.run(["lscpu"], capture_output=True, text=True, timeout=10).stdout
        for line in out.splitlines():
            if line.startswith("Model name:"):
                model = line.split(":", 1)[1].strip()
    except Exception:
        pass
    return {"nproc": os.cpu_count(), "cpu_model": model, "machine": platform.machine()}


_ORACLE_CHILD = r"""
import sys, time, json, os, numpy as np
sys.path.insert(0, %(root)r)
from oracle import wls
from paper_2604_23175_gb300 import synth
import bench
args = bench.parse_from(%(argv)r)
g = bench.workload_grid(args)
Vm, Va = synth.make_states(g, args.snapshots, %(sseed)d)
e = synth.make_noise(g, args.snapshots, %(nseed)d)
sig = synth.sigma_vector(g.n_bus, g.n_branch)
net = wls.Net(g.n_bus, g.from_bus.astype(np.int64), g.to_bus.astype(np.int64), g.r, g.x, g.b_charge, g.slack)
snaps = %(snaps)r
mask = bench.workload_mask(args, g)
w = {s: wls.weights(sig, None if mask is None else mask[s]) for s in snaps}
z = {s: wls.measure(net, Vm[s], Va[s]) + e[s] for s in snaps}
part = wls.partition(net, g.area_of_bus, g.n_area) if %(multi)r else None
sys.stdout.write("ready\n"); sys.stdout.flush()
sys.stdin.readline()
t = time.perf_counter()
res = {}
for s in snaps:
    if part is None:
        r = wls.gauss_newton(net, z[s], w[s], tol=%(tol)r, max_iter=%(mi)d)
    else:
        r = wls.multi_area_gauss_newton(net, part, z[s], w[s], tol=%(tol)r, max_iter=%(mi)d)
    res[s] = r
dt = time.perf_counter() - t
np.save(sys.argv[1], np.stack([np.concatenate([res[s].Vm, res[s].Va]) for s in snaps]))
print(json.dumps({"seconds": dt, "iters": [res[s].iters for s in snaps]}))
"""


def parse_from(argv):
    old = sys.argv
    try:
        sys.argv = ["bench.py"] + list(argv)
        return parse()
    finally:
        sys.argv = old


def oracle_run(argv, snap_lists, multi=False):
    """Time the CPU oracle: one child process per list of snapshots, each with
    single-threaded math libraries; the children build their inputs first and
    start solving together, and the wall time covers the solves only.
    Returns (wall seconds, per-child results, x[n, 2N] in snapshot order)."""
    env = dict(os.environ)
    for k in ("OMP_NUM_THREADS", "OPENBLAS_NUM_THREADS", "MKL_NUM_THREADS"):
        env[k] = "1"
    procs, paths = [], []
    for snaps in snap_lists:
        fd, path = tempfile.mkstemp(suffix=".npy")
        os.close(fd)
        paths.append(path)
        code = _ORACLE_CHILD % {"root": ROOT, "argv": list(argv), "sseed": STATE_SEED, "nseed": NOISE_SEED,
                                "snaps": list(snaps), "multi": multi, "tol": TOL, "mi": MAX_ITER}
        procs.append(subprocess.Popen([sys.executable, "-c", code, path], stdin=subprocess.PIPE,
                                      stdout=subprocess.PIPE, stderr=subprocess.PIPE, text=True,
                                      env=env, cwd=ROOT))
    for p in procs:
        line = p.stdout.readline()
        if line.strip() != "ready":
            raise RuntimeError(p.stderr.read()[-2000:])
    t0 = time.perf_counter()
    for p in procs:
        p.stdin.write("go\n")
        p.stdin.flush()
    outs = []
    for p in procs:
        o, err = p.communicate(timeout=3600)
        if p.returncode != 0:
            raise RuntimeError(err[-2000:])
        outs.append(json.loads(o.strip().splitlines()[-1]))
    wall = time.perf_counter() - t0
    xs = [np.load(pth) for pth in paths]
    for pth in paths:
        os.unlink(pth)
    return wall, outs, np.concatenate(xs)


def cpu_baselines(args, argv):
    """Three oracle baselines on the host cores, in the paper's baseline
    layouts: centralised FP64 on one thread; centralised FP64 with one
    snapshot per worker process on every core; multi-area FP64 (Schur
    condensation) with the same worker layout."""
    hi = host_info()
    n1 = args.cpu_sample
    rows = []
    wall, outs, x1 = oracle_run(argv, [list(range(n1))])
    rows.append({"value": n1 / wall, "unit": UNIT, "cores": 1, "kind": "oracle",
                 "sample": f"first {n1} of the {args.snapshots} snapshots, centralised FP64 Gauss-Newton "
                           f"(SciPy sparse LU), 1 thread", "seconds": wall})
    P = max(1, min(hi["nproc"] or 1, args.snapshots))
    wall, outs, _ = oracle_run(argv, [[s] for s in range(P)])
    rows.append({"value": P / wall, "unit": UNIT, "cores": P, "kind": "oracle",
                 "sample": f"first {P} snapshots, centralised FP64 Gauss-Newton, one snapshot per worker "
                           f"process ({P} processes, 1 BLAS thread each)", "seconds": wall})
    wall, outs, _ = oracle_run(argv, [[s] for s in range(P)], multi=True)
    rows.append({"value": P / wall, "unit": UNIT, "cores": P, "kind": "oracle",
                 "sample": f"first {P} snapshots, multi-area FP64 Gauss-Newton (per-area Schur condensation, "
                           f"dense), one snapshot per worker process", "seconds": wall})
    return hi, rows, x1


def run_reference(args, dist):
    """The oracle as the reference arm: each step solves a bounded sample of
    the workload's snapshots, one per host core in worker processes."""
    if dist.rank != 0:
        return None
    hi = host_info()
    g = workload_grid(args)
    P = max(1, min(hi["nproc"] or 1, args.snapshots))
    argv = [a for a in sys.argv[1:]]
    times = []
    for i in range(args.warmup + args.steps):
        wall, _, _ = oracle_run(argv, [[s] for s in range(P)])
        if i >= args.warmup:
            times.append(wall)
    sec = float(np.mean(times))
    v = P / sec
    return {"impl": "reference", "metric": METRIC, "value": v, "unit": UNIT, "n_gpus": dist.world,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": sec * 1e3,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
            "data": "synthetic",
            "config": {"workload": workload_desc(args, g, args.snapshots), "n_bus": g.n_bus,
                       "n_branch": g.n_branch, "n_area": g.n_area, "n_snap": args.snapshots,
                       "precision": "fp64 (the oracle)", "tol": TOL, "max_iter": MAX_ITER,
                       "snapshots_solved_per_step": P, "parallelism": "one snapshot per host worker process"},
            "cpu_baseline": {"value": v, "unit": UNIT, "cores": P, "kind": "oracle",
                             "sample": f"first {P} of the {args.snapshots} snapshots per step, centralised FP64 Gauss-Newton "
                                       f"(SciPy sparse LU), one snapshot per worker process"},
            "host": hi,
            "e2e": {"value": v, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}


def main():
    global MAX_ITER
    args = parse()
    MAX_ITER = args.max_iter
    dist = Dist(args.gpus)
    if args.impl == "reference":
        out = run_reference(args, dist)
        if dist.rank == 0:
            print(json.dumps(out))
        dist.close()
        return
    out, x_mixed, g = run_ours(args, dist)
    if dist.rank == 0:
        if not args.no_cpu_baseline:
            hi, rows, x_or = cpu_baselines(args, sys.argv[1:])
            n = x_or.shape[0]
            out["cpu_baseline"] = rows[1]
            out["cpu_baselines"] = rows
            out["host"] = hi
            out["accuracy"]["max_state_err_vs_oracle_sample"] = float(np.max(np.abs(x_mixed[:n] - x_or)))
            out["accuracy"]["oracle_sample_snapshots"] = n
        else:
            out["cpu_baseline"] = None
        print(json.dumps(out))
    dist.close()


if __name__ == "__main__":
    main()
