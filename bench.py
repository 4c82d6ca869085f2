#!/usr/bin/env python3
"""Benchmark: cell updates/s per RK2 (Heun) step of the KT viscous-hydro step at 128^3.

Workload: the 128^3 Milne grid with the nonconformal EOS (c_s^2(T) = 1/3 - 0.2 exp(-((T-0.17)/0.05)^2)),
eta/s = 0.08, zeta/s = 0.1 exp(-((T-0.17)/0.03)^2), 50 Gaussian hotspots (seed 1), tau0 = 0.5 fm,
dtau = 0.005 fm.  The state (~1.1-1.7 GB) is far larger than L2, so no flush is needed between steps.

    python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference] [--mode mixed|fp64]

Under torchrun (N > 1) every rank advances its own event (different seed): replicas, weak scaling.
With --batch, one batch of events is partitioned across the ranks by cell count (strong scaling).
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

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "cell updates/s per RK2 step at 128^3, plain FP64 vs FP32+learned; % HBM peak"
UNIT = "cell updates/s"
# Algorithmic bytes per cell per RK2 step, every field read and written once per launch.
# FP64 (one fused kernel per stage): stage 1 reads q, u, u_prev, e, p (25 words) and writes q*, u*,
# e, p (21); stage 2 reads q*, q^n, u*, u^n, e, p (40) and writes 21: 107 words = 856 B.
# Mixed (per stage an FP32 right-hand-side kernel and an update kernel):
#   rhs 1:    qf 60 + u 16 + u_prev 16 + e, p 8 -> k1 60                         = 160
#   update 1: q (T, pi^{tau mu}, Pi) 72 + k1 60 + qf 60 + e 4 -> qsf 60 + u 16 + e, p 8
#             + regulated k1 (pi) 40                                            = 320
#   rhs 2:    qsf 60 + u 16 + u_prev 16 + e, p 8 -> k2 60                        = 160
#   update 2: q 120 + k1 60 + k2 60 + e 4 -> q 120 + qf 60 + u 16 + e, p 8       = 448
# = 1088 B (the learned start reads no previous e but, in both stages, the network's 4-byte
# output instead: also 1088 B; the network's own launch reads 9 components of the FP32 copy of q^n
# and writes z, 40 B per element of the padded arrays: 1128 B).
BYTES_PER_CELL = {"fp64": 856, "mixed": 1088, "learned": 1128}
# The algorithmic bytes of the method's step, independent of this design: per cell and RK2 step
# every field is read and written once by a fused kernel per stage (stage 1 reads q^n (15), u^n,
# u^{n-1} (4 + 4), e, p and writes q*, u*, e, p; stage 2 reads q*, u*, u^n, e, p, q^n and writes
# q^{n+1}, u^{n+1}, e, p: 107 words): FP64 856 B; mixed precision (q FP64; u, e, p FP32) 728 B.
# The roofline of the step is taken against these; BYTES_PER_CELL above is what this design's
# kernels move, and the recorded DRAM traffic shows the difference.
ALG_BYTES_PER_CELL = {"fp64": 856, "mixed": 728, "learned": 728}
# FP64 add/multiply/FMA instructions per cell and RK2 step of the FP64 mode (ncu counts of the two
# fused stage kernels), and GB300's FP64 rate: 2 FMA per SM and clock (152 SMs; 1.25 TFLOP/s at
# 2.07 GHz nominal), taken at the SM clock sampled during the timed steps
FP64_INST_PER_CELL_STEP = 1799 + 1828
FP64_FMA_PER_SM_CLK = 2
N_SM = 152
# per launch slot of kt_time_kernels (bytes per cell); FP64: the fused stage kernels
SLOT_BYTES = {
    "fp64": {"stage1_rhs": 368, "stage2_rhs": 488},
    "mixed": {"stage1_rhs": 160, "stage1_update": 320, "stage2_rhs": 160, "stage2_update": 448},
    "learned": {"learned_start": 40, "stage1_rhs": 160, "stage1_update": 320, "stage2_rhs": 160,
                "stage2_update": 448},
}
# The fused launch per stage: stage 1 reads qf 60,
# u 16, u_prev 16, e, p 8, q (T, pi^{tau mu}, Pi) 72, qf at the cell 60 and writes k1 60, qsf 60, u
# 16, e, p 8 = 376 (+ network output 4, learned); stage 2 reads qsf 60, u 16, u_prev 16, e, p 8,
# q 120, k1 60 and writes q 120, qf 60, u 16, e, p 8 = 484 (+ 4, learned): 868 B per step, k never
# leaves the SM within a stage (+ 40 for the network's launch, learned).
FUSED_SLOT_BYTES = {"learned_start": 40, "stage1_rhs": 380, "stage2_rhs": 488}
FUSED_FIRST_CANDIDATE = 24  # tuning candidates 24-35 are the fused launches (timed by the autotuner too)
SLOT_KERNEL = {"learned_start": "mlp_start_kernel", "stage1_rhs": "rhs_kernel", "stage2_rhs": "rhs_kernel",
               "stage1_update": "update_kernel", "stage2_update": "update_kernel", "tau_advance": "advance_tau_kernel"}
LAUNCHES_PER_STEP = {"fp64": 3, "mixed": 5}  # + the tau advance (+ 1 for the network, learned start)
# DRAM bytes per launch (dram__bytes_read.sum + dram__bytes_write.sum) of the current kernels: one-
# kernel ncu captures of the 96^3 learned workload, per cell times the 128^3 cells (average over
# the two stages of each kernel; the update and fused kernels captured on 32x2x2 tiles, one block
# per tile).  Only that mode (workload EOS) has a capture.
MEASURED_TRAFFIC = {("learned", 128): {"rhs_kernel": 311.2e6, "update_kernel": 756.7e6, "fused_kernel": 827.8e6,
                                        "mlp_start_kernel": 85.4e6}}
# Warp instructions per 32 cells of each launch slot (ncu smsp__inst_executed.sum over the warps of
# one-kernel captures of the 96^3 learned workload, current kernels), for each kernel's fraction of
# the SMs' issue rate: one warp instruction per scheduler and clock, 4 schedulers per SM.  The
# kernels are bound by instruction issue and latency rather than by HBM.
INST_PER_WARP = {"learned": {"learned_start": 259, "stage1_rhs": 2811, "stage2_rhs": 2811, "stage1_update": 1621,
                             "stage2_update": 1914}}
INST_PER_WARP_FUSED = {"learned": {"learned_start": 259, "stage1_rhs": 4319, "stage2_rhs": 4622}}  # fused launches
ISSUE_PER_SM_CLK = 4
REPEATS = 3  # timed runs of K steps per mode; the median is reported


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=30)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--mode", default="learned", choices=["learned", "mixed", "fp64"])
    ap.add_argument("--only-main", action="store_true", help="time only --mode")
    ap.add_argument("--train-samples", type=int, default=1_000_000)
    ap.add_argument("--epochs", type=int, default=20)
    ap.add_argument("--n", type=int, default=128)
    ap.add_argument("--tuning", type=int, default=None,
                    help="force autotuner candidate 12 v + 2 s + g of the timed mode (kt_set_tuning)")
    ap.add_argument("--large", action="store_true",
                    help="the large single event: 256x256x128, 100 hotspots, eta/s 0.2 (timing only)")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--iface", default="recon", choices=["recon", "invert"],
                    help="face velocities: extrapolated u (default) or root-finds of the face states")
    ap.add_argument("--batch", type=int, default=0,
                    help="instead of the 128^3 event: a batch of this many events with uneven grids "
                         "(64 = the batch workload), one launch per stage for all events")
    ap.add_argument("--eos", default="workload", choices=["workload", "lattice"],
                    help="workload: c_s^2(T) table, eta/s 0.08, gaussian zeta/s; lattice: the paper's "
                         "lattice EOS with its zeta/s parametrisation and eta/s 0.2")
    return ap.parse_args()


def measured_peaks():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            d = json.load(f)
        return float(d["hbm_gbs"]), "measured"
    except Exception:
        return 6800.0, "fallback"


class ClockSampler:
    """nvidia-smi clocks and throttle reasons sampled every 200 ms during the timed region."""

    def __init__(self, index):
        self.index = index
        self.proc = None
        self.path = None

    def __enter__(self):
        fd, self.path = tempfile.mkstemp(suffix=".csv")
        os.close(fd)
        q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
             "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
             "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")
        try:
            self.proc = subprocess.Popen(["nvidia-smi", f"--query-gpu={q}", "--format=csv,noheader,nounits",
                                          "-i", str(self.index), "-lms", "200"],
                                         stdout=open(self.path, "w"), stderr=subprocess.DEVNULL)
        except Exception:
            self.proc = None
        time.sleep(0.3)
        return self

    def __exit__(self, *a):
        if self.proc:
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except Exception:
                self.proc.kill()

    def summary(self):
        sm, smax, reasons = [], None, set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        try:
            for line in open(self.path):
                f = [x.strip() for x in line.split(",")]
                if len(f) < 9:
                    continue
                try:
                    sm.append(float(f[1]))
                    smax = float(f[2])
                except ValueError:
                    continue
                for nm, v in zip(names, f[5:9]):
                    if v.lower() == "active":
                        reasons.add(nm)
        except Exception:
            pass
        finally:
            try:
                os.unlink(self.path)
            except Exception:
                pass
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": smax, "reasons": sorted(reasons),
                "samples": len(sm)}


def dist_setup(args):
    """One process per GPU under torchrun; NCCL for our arm, gloo for the CPU reference arm."""
    from paper_1608_06577_gb300 import parallel
    return parallel.init("nccl" if args.impl == "ours" else "gloo")


def barrier(world):
    from paper_1608_06577_gb300 import parallel
    parallel.barrier(world)


def max_over_ranks(x, world):
    from paper_1608_06577_gb300 import parallel
    return parallel.max_over_ranks(x, world)


# ----------------------------------------------------------------------------- oracle timing
def oracle_rate(prob_full, nz_sample, nsteps, threads=None):
    """Time the CPU oracle on a slab of the workload (same grid spacing, nz_sample eta cells)."""
    import oracle
    from workload.problem import hotspot_problem
    p = hotspot_problem(nx=prob_full.nx, ny=prob_full.ny, neta=nz_sample)
    o = oracle.Oracle(p, threads=threads)
    cores = oracle.set_threads(threads or 0)
    t0 = time.perf_counter()
    o.step(nsteps)
    dt = time.perf_counter() - t0
    return (p.ncells * nsteps / dt, cores,
            f"{p.nx}x{p.ny}x{p.neta} slab of the {prob_full.nx}x{prob_full.ny}x{prob_full.neta} workload, {nsteps} steps")


def run_reference(args, world, rank):
    """The reference arm: the CPU oracle (the only other implementation of the method here)."""
    if rank != 0:
        return
    import oracle
    oracle.build()
    from workload.problem import hotspot_problem
    cores = os.cpu_count()
    prob = hotspot_problem(nx=args.n, ny=args.n, neta=args.n, nsteps=1)
    nz = 16  # 2,048 (eta, y) rows: the oracle's threads split rows, so every core has work
    p = hotspot_problem(nx=args.n, ny=args.n, neta=nz)
    o = oracle.Oracle(p, threads=cores)
    cores = oracle.set_threads(cores)
    o.step(args.warmup)
    t0 = time.perf_counter()
    o.step(args.steps)
    dt = time.perf_counter() - t0
    value = p.ncells * args.steps / dt
    line = {"impl": "reference", "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": args.gpus,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": dt / args.steps * 1e3,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": {"workload": f"hotspots {prob.nx}x{prob.ny}x{prob.neta} (sampled as a "
                                   f"{p.nx}x{p.ny}x{p.neta} slab per step)", "dx_fm": 0.1, "deta": 0.1,
                       "dtau_fm": 0.005, "eos": "tabulated c_s^2(T)", "l2": "inputs larger than L2"},
            "cpu_baseline": {"value": value, "unit": UNIT, "cores": cores, "kind": "oracle",
                             "sample": f"{p.nx}x{p.ny}x{p.neta} slab, {args.steps} steps after {args.warmup} warm-up"},
            "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


# ----------------------------------------------------------------------------- our arm
# (precision, inversion); "network_off" is the learned mode with all-zero weights, i.e. started
# from the conformal root alone: the ablation that shows what the trained network adds;
# "conformal" the same start without the network (KT_INV_CONFORMAL: e_conf, no inference), so
# that network_off - conformal is the inference's cost and network_off - learned its saving;
# "learned_pi32" the learned mode with the FP32 storage of pi and Pi (KT_STORE_PI_FP32: only the
# conserved T^{tau mu} kept and Heun-summed in FP64)
MODES = {"learned": (1, 1), "mixed": (1, 0), "fp64": (0, 0), "network_off": (1, 1), "conformal": (1, 2),
         "learned_pi32": (1, 1)}


def make_kt(prob, mode, weights, stream, tuning=None):
    import numpy as np
    import torch
    from paper_1608_06577_gb300 import KT
    prec, inv = MODES[mode]
    if mode == "network_off" and weights is not None:
        weights = np.zeros_like(weights)
    with torch.cuda.stream(stream):
        kt = KT(prob, precision=prec, inversion=inv, mlp_weights=weights if inv == 1 else None,
                pi_fp32=(mode == "learned_pi32"))
        if tuning is not None:
            kt.set_tuning(tuning)
        return kt


def time_mode(prob, mode, weights, steps, warmup, stream, world, profile_range=False, tuning=None):
    """Times REPEATS runs of exactly `steps` RK2 steps each (after `warmup` untimed steps) with CUDA
    events on the launching stream, each run bracketed by a barrier and a device synchronisation,
    max over ranks; returns the context and the per-run times in ms.  With profile_range the first
    timed run sits between cudaProfilerStart/Stop, so `ncu --profile-from-start off` lists exactly
    its launches."""
    import torch
    kt = make_kt(prob, mode, weights, stream, tuning)
    kt.set_problem_state()
    kt.step(warmup)
    torch.cuda.synchronize()
    ev0, ev1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    runs = []
    for r in range(REPEATS):
        barrier(world)
        torch.cuda.synchronize()
        if profile_range and r == 0:
            torch.cuda.profiler.start()
        ev0.record(stream)
        kt.step(steps)
        ev1.record(stream)
        ev1.synchronize()
        if profile_range and r == 0:
            torch.cuda.profiler.stop()
        runs.append(max_over_ranks(ev0.elapsed_time(ev1), world))
    return kt, runs


def run_ours(args, world, rank, local):
    import numpy as np
    import torch
    from workload.problem import hotspot_problem
    torch.cuda.set_device(local)
    stream = torch.cuda.Stream()
    n = args.n
    if args.eos == "lattice":
        from workload.eos import lattice_table
        prob = hotspot_problem(nx=n, ny=n, neta=n, seed=1 + rank, eta_over_s=0.2, zeta="paper",
                               eos_table=lattice_table())
    elif args.large:
        prob = hotspot_problem(nx=256, ny=256, neta=128, nhot=100, seed=7 + rank, eta_over_s=0.2)
    else:
        prob = hotspot_problem(nx=n, ny=n, neta=n, seed=1 + rank)
    prob.iface = args.iface
    cells = prob.ncells
    hbm_peak, peak_kind = measured_peaks()

    weights, train_info = None, None
    if args.mode == "learned" or not args.only_main:
        from paper_1608_06577_gb300 import learned
        t0 = time.perf_counter()
        with torch.cuda.stream(stream):
            params, losses, (X, Y) = learned.train_default(n=n, n_samples=args.train_samples, epochs=args.epochs)
            mx, rms = learned.evaluate(params, X, Y)
        torch.cuda.synchronize()
        weights = params.cpu().numpy()
        train_info = {"samples": int(X.shape[0]), "epochs": args.epochs, "final_loss": losses[-1], "rms_err_y": rms,
                      "max_err_y": mx, "rms_err_y_conformal": float(np.sqrt(np.mean(Y.cpu().numpy().astype(np.float64) ** 2))),
                      "seconds": time.perf_counter() - t0,
                      "data": f"hotspots {n}^3 seeds 2-11, every 10 steps of 100"}

    results = {}
    modes = [args.mode] + ([] if args.only_main else [m for m in MODES if m != args.mode])
    clocks = None
    for mode in modes:
        steps = args.steps  # every mode: the headline's step count, median of REPEATS runs
        barrier(world)
        torch.cuda.synchronize()
        if mode == args.mode:
            with ClockSampler(local) as cs:
                kt, runs = time_mode(prob, mode, weights, steps, args.warmup, stream, world, profile_range=True,
                                     tuning=args.tuning)
            clocks = cs.summary()
        else:
            kt, runs = time_mode(prob, mode, weights, steps, args.warmup, stream, world)
        torch.cuda.synchronize()
        barrier(world)
        ms = statistics.median(runs)
        st = kt.stats()
        results[mode] = {"ms_per_step": ms / steps, "value": cells * world * steps / (ms * 1e-3), "steps": steps,
                         "stats": st, "runs_ms_per_step": [r / steps for r in runs]}
        if mode == args.mode:  # per-launch durations (CUDA events between launches, after the timed steps)
            results[mode]["slots_ms"] = kt.time_kernels(max(3, min(steps, 10)))
            tu = kt.tuning()
            best = min(range(len(tu["candidate_ms"])), key=lambda i: tu["candidate_ms"][i] or float("inf"))
            if args.tuning is not None:
                best = args.tuning
            results[mode]["tuning"] = {"tile": list(tu["block"]), "grid_blocks": tu["grid_blocks"],
                                       "candidate": best, "one_block_per_tile": bool(best % 2),
                                       "layout": "fp64_stage" if mode == "fp64" else
                                       ("split", "split_update_staged_by_tma", "fused_stage")[best // 12]}
        del kt
        torch.cuda.empty_cache()

    # The other layouts of the mixed-precision stage on the autotuned tile shape and grid: split
    # launches with direct reads, the update's inputs staged in shared memory by TMA, one fused
    # launch per stage (the autotuner times the first and the last)
    variants = None
    if args.mode != "fp64" and not args.only_main:
        variants = {}
        picked = results[args.mode]["tuning"]["candidate"]
        base = picked % 12
        for name, v in (("split", 0), ("split_update_staged_by_tma", 1), ("fused_stage", 2)):
            if 12 * v + base == picked:
                continue
            kt = make_kt(prob, args.mode, weights, stream)
            kt.set_tuning(12 * v + base)
            kt.set_problem_state()
            kt.step(args.warmup)
            torch.cuda.synchronize()
            ev0, ev1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            runs = []
            for _ in range(REPEATS):
                barrier(world)
                torch.cuda.synchronize()
                ev0.record(stream)
                kt.step(args.steps)
                ev1.record(stream)
                ev1.synchronize()
                runs.append(max_over_ranks(ev0.elapsed_time(ev1), world) / args.steps)
            variants[name] = {"candidate": 12 * v + base, "ms_per_step": statistics.median(runs),
                              "runs_ms_per_step": runs, "slots_ms": kt.time_kernels(3)}
            del kt
            torch.cuda.empty_cache()

    main = results[args.mode]
    ms_step = main["ms_per_step"]
    fused = args.mode != "fp64" and main.get("tuning", {}).get("candidate", 0) >= FUSED_FIRST_CANDIDATE
    slot_bytes = FUSED_SLOT_BYTES if fused else SLOT_BYTES[args.mode]
    bpc = sum(b for slot, b in slot_bytes.items() if main["slots_ms"].get(slot, 0.0) > 0.0)
    alg = ALG_BYTES_PER_CELL[args.mode]
    # per kernel: launches per step, average launch time, algorithmic bytes per launch, GB/s
    kernels = {}
    for slot, t in main["slots_ms"].items():
        if t <= 0.0 or (fused and slot.endswith("update")):  # (fused: the update slots are empty)
            continue
        name = SLOT_KERNEL[slot]
        if slot.endswith("rhs") and (args.mode == "fp64" or fused):
            name = "stage_kernel" if args.mode == "fp64" else "fused_kernel"
        k = kernels.setdefault(name, {"launches_per_step": 0, "ms_per_step": 0.0, "bytes_per_step": 0.0})
        k["launches_per_step"] += 1
        k["ms_per_step"] += t
        k["bytes_per_step"] += cells * slot_bytes.get(slot, 8.0 / cells)
    inst = (INST_PER_WARP_FUSED if fused else INST_PER_WARP).get(args.mode)
    sm_hz_k = ((clocks or {}).get("sm_mhz") or 2070.0) * 1e6
    for slot, t in main["slots_ms"].items():
        if inst and slot in inst and t > 0.0:
            k = kernels["fused_kernel" if (fused and slot.endswith("rhs")) else SLOT_KERNEL[slot]]
            k.setdefault("warp_inst_per_step", 0.0)
            k["warp_inst_per_step"] += inst[slot] * cells / 32
    for k in kernels.values():
        k["avg_launch_ms"] = k["ms_per_step"] / k["launches_per_step"]
        if "warp_inst_per_step" in k:
            ach = k["warp_inst_per_step"] / (k["ms_per_step"] * 1e-3)
            peak = ISSUE_PER_SM_CLK * N_SM * sm_hz_k
            k["issue"] = {"bound": "issue", "achieved": ach, "peak": peak, "unit": "warp instructions/s",
                          "frac": ach / peak, "note": "ncu warp instructions per 32 cells (96^3 capture) x the "
                          "launches' warps / CUDA-event time; peak 4 per SM and clock at the sampled SM clock"}
        k["gbs"] = k["bytes_per_step"] / (k["ms_per_step"] * 1e-3) / 1e9
        k["frac_of_hbm"] = k["gbs"] / hbm_peak
        k["share"] = k["ms_per_step"] / sum(v["ms_per_step"] for v in kernels.values())
        k["share_of_step_bytes"] = k["bytes_per_step"] / (cells * bpc)
    dom = max(kernels, key=lambda n: kernels[n]["ms_per_step"])
    traffic_k = None if (args.large or args.eos != "workload") else MEASURED_TRAFFIC.get((args.mode, n))
    traffic = None
    if traffic_k and all(k in traffic_k for k in kernels if k != "advance_tau_kernel"):
        # DRAM bytes per step: every kernel's recorded traffic per launch times its launches
        traffic = sum(traffic_k[k] * v["launches_per_step"] for k, v in kernels.items() if k in traffic_k)
    achieved = cells * alg / (ms_step * 1e-3) / 1e9
    roofline = {"bound": "hbm", "achieved": achieved, "peak": hbm_peak, "unit": "GB/s",
                "frac": achieved / hbm_peak, "traffic": traffic, "peak_kind": peak_kind,
                "kernel": "the whole step (all launches)", "alg_bytes_per_cell_step": alg,
                "design_bytes_per_cell_step": bpc,
                "traffic_bytes_per_cell_step": None if traffic is None else traffic / cells,
                "design_gbs": cells * bpc / (ms_step * 1e-3) / 1e9, "dominant_kernel": dom,
                "note": "achieved = the method's algorithmic bytes per RK2 step (107 words per cell: 728 B "
                        "mixed, 856 B FP64) / the CUDA-event time per step; design_gbs counts the bytes "
                        "this design's kernels move; traffic = ncu DRAM bytes per step (null unless this "
                        "mode and size were captured with the current kernels); per-kernel rooflines "
                        "under `kernels`"}
    fp64_pipe = None
    if args.mode == "fp64" or "fp64" in results:
        r64 = results["fp64"]
        sm_hz = ((clocks or {}).get("sm_mhz") or 2070.0) * 1e6
        ach = FP64_INST_PER_CELL_STEP * cells * world / (r64["ms_per_step"] * 1e-3)
        peak = FP64_FMA_PER_SM_CLK * N_SM * sm_hz * world
        fp64_pipe = {"bound": "fp64 alu", "achieved": ach, "peak": peak, "unit": "FP64 instructions/s",
                     "frac": ach / peak, "inst_per_cell_step": FP64_INST_PER_CELL_STEP,
                     "note": "FP64 add/multiply/FMA instructions per cell-step from ncu; peak from the unit "
                             "count (2 FP64 FMA per SM and clock, 152 SMs) at the sampled SM clock"}

    e2e = None
    if not args.no_e2e:
        kt = make_kt(prob, args.mode, weights, stream)
        kt.set_problem_state()
        kt.step(args.warmup)  # tile autotuning and graph capture happen here, outside the timed region

        def pinned(a):
            t = torch.from_numpy(np.ascontiguousarray(a, dtype=np.float64)).pin_memory()
            keep.append(t)
            return t.numpy()
        keep = []
        e_h, u_h, pi_h, Pi_h = pinned(prob.e), pinned(prob.u), pinned(prob.pi), pinned(prob.Pi)
        out_h = {"e": pinned(np.empty(cells)), "u": pinned(np.empty((4, cells)))}
        times = []
        for _ in range(3):  # the median of three end-to-end runs (host copies vary from run to run)
            torch.cuda.synchronize()
            barrier(world)
            t0 = time.perf_counter()
            kt.set_state(prob.tau0, e_h, u_h, pi_h, Pi_h)  # host -> device from pinned memory
            kt.step(args.steps)
            kt.get_state(fields=("e", "u"), out=out_h)  # device -> host into pinned memory
            t1 = time.perf_counter()
            barrier(world)
            times.append(max_over_ranks(t1 - t0, world))
        dt = sorted(times)[1]
        h2d = (1 + 3 + 10 + 1) * cells * 8
        d2h = 5 * cells * 8
        e2e = {"value": cells * world * args.steps / dt, "unit": UNIT,
               "h2d_bytes_per_step": h2d / args.steps, "d2h_bytes_per_step": d2h / args.steps,
               "note": f"kt_set_state from pinned host memory, {args.steps} steps, kt_get_state(e, u) into "
                       f"pinned host memory, on a context tuned by {args.warmup} warm-up steps; median of 3"}
        del kt

    cpu = None
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        try:
            # about 10 s of host work each: a slab of ~1e6 cells of the same workload, 20 steps, on
            # all cores; a slab of ~1.3e5 cells, 8 steps, on one core
            nz = max(4, min(prob.neta, (1 << 20) // (prob.nx * prob.ny)))
            v, cores, sample = oracle_rate(prob, nz, 20, threads=os.cpu_count())
            nz1 = max(2, min(prob.neta, (1 << 17) // (prob.nx * prob.ny)))
            v1, _, sample1 = oracle_rate(prob, nz1, 8, threads=1)
            cpu = {"value": v, "unit": UNIT, "cores": cores, "kind": "oracle", "sample": sample,
                   "single_core": {"value": v1, "unit": UNIT, "sample": sample1}}
        except Exception as ex:  # the baseline never blocks the GPU line
            cpu = {"value": None, "unit": UNIT, "cores": None, "kind": "oracle", "sample": f"failed: {ex}"}

    if rank == 0:
        ncs = lambda r: cells * 2 * r["steps"]  # noqa: E731
        line = {"metric": METRIC, "value": main["value"], "unit": UNIT, "n_gpus": world, "steps": main["steps"],
                "warmup": args.warmup, "ms_per_step": ms_step, "higher_is_better": True, "scaling": "weak",
                "vs_baseline": None, "dtype": "f64" if args.mode == "fp64" else "f32+f64", "data": "synthetic",
                "config": {"workload": ("hotspots 256x256x128 Milne, 100 hotspots, nonconformal EOS, eta/s 0.2, "
                                        "zeta/s gaussian, dtau 0.005 fm") if args.large else
                                       (f"hotspots {n}x{n}x{n} Milne, nonconformal EOS, eta/s 0.08, "
                                        f"zeta/s gaussian, dtau 0.005 fm") if args.eos == "workload" else
                                       (f"hotspots {n}x{n}x{n} Milne, lattice EOS (Sec. 2.3), eta/s 0.2, "
                                        f"zeta/s of Eq. (zetas), dtau 0.005 fm"),
                           "global_batch": world, "seq_len": None,
                           "parallelism": f"replicas x{world}", "l2": "inputs larger than L2 (no flush)",
                           "mode": args.mode, "iface": args.iface, "eos": args.eos,
                           "tuning": main.get("tuning")},
                "modes": {m: {"value": r["value"], "ms_per_step": r["ms_per_step"], "steps": r["steps"],
                              "runs_ms_per_step": r["runs_ms_per_step"],
                              "hbm_frac_alg": cells * world * ALG_BYTES_PER_CELL[m if m in ALG_BYTES_PER_CELL
                                                                                 else "learned"]
                                              / (r["ms_per_step"] * 1e-3) / 1e9 / hbm_peak,
                              "newton_iters_per_cell_stage": r["stats"]["newton_iters"] / ncs(r),
                              "fallbacks_per_cell_stage": r["stats"]["fallbacks"] / ncs(r)}
                          for m, r in results.items()},
                "fp64_pipe": fp64_pipe, "layout_variants": variants,
                "learned_training": train_info,
                "roofline": roofline, "kernels": kernels, "cpu_baseline": cpu, "e2e": e2e, "clocks": clocks,
                "gpu_launches": ((3 if (args.mode == "fp64" or fused) else 5)
                                 + (1 if MODES[args.mode][1] == 1 else 0)) * main["steps"]}
        print(json.dumps(line), flush=True)


def run_batch(args, world, rank, local):
    """The batch workload: one batch of events with fluctuating hotspot initial states and uneven
    grids (nx = ny in 64..160, neta in 16..64, 20-100 hotspots, seeds 1000 + event), advanced by
    one launch per stage for all events of a context.  Under torchrun the batch is partitioned
    across the ranks by cell count (parallel.rank_share: largest event first onto the least-loaded
    rank); every rank advances only its share, with no data-path collective (strong scaling: the
    whole job's work is the one batch)."""
    import torch
    from paper_1608_06577_gb300 import KT, learned, parallel
    from workload.problem import batch_problems, batch_shapes
    torch.cuda.set_device(local)
    stream = torch.cuda.Stream()
    shapes = batch_shapes(args.batch, seed=1000)
    mine, total_cells = parallel.rank_share([n * n * nz for n, nz, _ in shapes], world, rank)
    probs = batch_problems(n_events=args.batch, seed=1000, events=mine)
    cells = sum(p.ncells for p in probs)
    prec, inv = MODES[args.mode]
    weights = None
    if inv:
        with torch.cuda.stream(stream):
            params, _, _ = learned.train_default(n=64, n_samples=args.train_samples, epochs=args.epochs)
        weights = params.cpu().numpy()
    with torch.cuda.stream(stream):
        kt = KT(probs, precision=prec, inversion=inv, mlp_weights=weights)
    kt.set_problem_state()
    kt.step(args.warmup)
    torch.cuda.synchronize()
    barrier(world)
    torch.cuda.synchronize()
    ev0, ev1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    ev0.record(stream)
    kt.step(args.steps)
    ev1.record(stream)
    ev1.synchronize()
    barrier(world)
    ms = max_over_ranks(ev0.elapsed_time(ev1), world)
    slots = kt.time_kernels(max(3, min(args.steps, 10)))
    tu = kt.tuning()
    cand = min(range(len(tu["candidate_ms"])), key=lambda i: tu["candidate_ms"][i] or float("inf"))
    fused = args.mode != "fp64" and cand >= FUSED_FIRST_CANDIDATE
    if rank == 0:
        line = {"metric": "cell updates/s per RK2 step, batch of events", "value": total_cells * args.steps / (ms * 1e-3),
                "unit": UNIT, "n_gpus": world, "steps": args.steps, "warmup": args.warmup,
                "ms_per_step": ms / args.steps, "higher_is_better": True, "scaling": "strong", "vs_baseline": None,
                "dtype": "f64" if args.mode == "fp64" else "f32+f64", "data": "synthetic",
                "config": {"workload": f"{args.batch} events, nx=ny in 64..160, neta in 16..64, 20-100 hotspots",
                           "cells_total": total_cells, "events_rank0": len(mine), "cells_rank0": cells,
                           "parallelism": f"events sharded over {world} ranks", "mode": args.mode,
                           "tile": tu["block"], "candidate": cand,
                           "layout": "fp64_stage" if args.mode == "fp64" else
                           ("split", "split_update_staged_by_tma", "fused_stage")[cand // 12]},
                "slots_ms": slots,
                "gpu_launches": (LAUNCHES_PER_STEP["fp64" if (args.mode == "fp64" or fused) else "mixed"]
                                 + (1 if MODES[args.mode][1] == 1 else 0)) * args.steps}
        print(json.dumps(line), flush=True)


def main():
    args = parse()
    world, rank, local = dist_setup(args)
    try:
        if args.impl == "reference":
            run_reference(args, world, rank)
        elif args.batch > 0:
            run_batch(args, world, rank, local)
        else:
            run_ours(args, world, rank, local)
    finally:
        if world > 1:
            import torch.distributed as dist
            dist.destroy_process_group()


if __name__ == "__main__":
    main()
