"""Benchmark: cell-updates/s of the PP-WCNS-IS fractional step on the
1024 x 512 three-species 2D shock-bubble workload (water, air, helium; SSP-RK3
with relaxation after every stage, CFL 0.4), FP64 plain, with the other forms
reported beside it at their relative L1 error against FP64: the FP32-bulk
form, and the FP32 and FP64 forms with the learned smoothness gate (trained
first, on the GPU, on stencils of the method's own runs), here and on the
2048 x 1024 shock-water-column workload.

    python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]

Prints one JSON line (rank 0). A step is one full SSP-RK3 step (three stages,
three relaxations, the CFL reduction) of the whole grid. With N > 1 (torchrun),
every rank advances its own replica of the workload (the instances are
independent; weak scaling) and the value is the total over ranks divided by the
slowest rank's time.
"""
from __future__ import annotations

import argparse
import json
import math
import os
import statistics
import subprocess
import sys
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

# DRAM traffic per launch of the dominant kernels, dram__bytes_read.sum + dram__bytes_write.sum from one
# ncu capture on this workload (profiles/k_face_fp64_shock_bubble_1024x512.md and
# profiles/k_face32_shock_bubble_1024x512.md); to be re-taken whenever those kernels change.
TRAFFIC_BYTES = {"k_face_fp64": 82.78e6, "k_face32": 73.09e6}
# FP64-pipe activity of the FP64 sweep in the same ncu capture (fraction of peak sustained)
FP64_PIPE_ACTIVE = {"k_face_fp64": 0.716}
METRIC = "cell-updates/s (FP64 plain vs FP32+learned) at stated L1 err; % of roofline"
UNIT = "cell-updates/s"
WORKLOAD = "2D three-species shock-bubble, 1024x512 cells, Mach 1.5 shock, water+air+helium, SSP-RK3, CFL 0.4"


def peaks():
    path = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(path):
        with open(path) as fh:
            return json.load(fh), "measured"
    return {"hbm_gbs": 6800.0, "bf16_tflops": 1900.0}, "fallback"


class Clocks:
    """nvidia-smi sampling of SM clocks and throttle reasons during the timed region."""

    Q = ("clocks.sm,clocks.max.sm,clocks_event_reasons.active,clocks_event_reasons.hw_slowdown,"
         "clocks_event_reasons.hw_thermal_slowdown,clocks_event_reasons.sw_thermal_slowdown,"
         "clocks_event_reasons.sw_power_cap")

    def __init__(self, index):
        self.index = index
        self.proc = None

    def __enter__(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.index), f"--query-gpu={self.Q}", "--format=csv,noheader,nounits",
                 "-lms", "200"], stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
        except OSError:
            self.proc = None
        return self

    def __exit__(self, *a):
        self.samples = []
        if self.proc is None:
            return
        self.proc.terminate()
        out, _ = self.proc.communicate(timeout=10)
        for line in out.strip().splitlines():
            parts = [x.strip() for x in line.split(",")]
            if len(parts) >= 7:
                self.samples.append(parts)

    def summary(self):
        if not getattr(self, "samples", None):
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["unsampled"]}
        sm = [float(p[0]) for p in self.samples if p[0].replace(".", "").isdigit()]
        mx = [float(p[1]) for p in self.samples if p[1].replace(".", "").isdigit()]
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = sorted({names[i] for p in self.samples for i in range(4) if p[3 + i].lower() == "active"})
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": max(mx) if mx else None,
                "reasons": reasons, "samples": len(self.samples)}


def dist_env():
    ws = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return ws, rank, local


def algorithmic_face_flops(problem, cfl, W=None):
    """Algorithmic flops per midpoint of each direction on the state W (default:
    the initial state), from the oracle's operation-counting build (add, mul,
    div, sqrt, tanh each one flop)."""
    import oracle
    f, g, W0 = oracle.setup(problem)
    W = W0 if W is None else np.ascontiguousarray(W, dtype=np.float64)
    dt, _ = oracle.dt(f, g, W, cfl)
    lam = oracle.lambdas(f, g, W, dt)
    out = []
    for d in range(problem.D):
        c, nf = oracle.faces_flops(f, oracle.make_params(), g, W, lam, d)
        out.append((sum(c.values()) / nf, nf, c))
    return out


def run_face_flops(problem, cfl, W_end):
    """Flops per midpoint of each direction over a run from the initial state to
    W_end: the mean of the counts on the two states. A uniform stencil (six
    bit-identical node states) costs only the node flux, and the share of such
    midpoints falls as the waves spread, so the initial state alone undercounts."""
    a = algorithmic_face_flops(problem, cfl)
    b = algorithmic_face_flops(problem, cfl, W_end)
    return [(0.5 * (x[0] + y[0]), x[1], {"first": round(x[0], 1), "last": round(y[0], 1)}) for x, y in zip(a, b)]


def first_order_face_flops(problem, cfl, d):
    """Flops per midpoint of the first-order HLLC flux alone (the scheme with
    only that flux, oracle counting build): part of the method as written at
    every midpoint, which the CUDA sweeps evaluate only where the flux limiter
    can act."""
    import oracle
    f, g, W = oracle.setup(problem)
    dt, _ = oracle.dt(f, g, W, cfl)
    lam = oracle.lambdas(f, g, W, dt)
    c, nf = oracle.faces_flops(f, oracle.make_params(scheme=1), g, W, lam, d)
    return sum(c.values()) / nf


def host_cpu():
    """CPU model and logical core count of this host."""
    model = None
    try:
        for line in open("/proc/cpuinfo"):
            key = line.split(":")[0].strip().lower()
            if key in ("model name", "cpu model", "hardware") and ":" in line:
                model = line.split(":", 1)[1].strip()
                break
    except OSError:
        pass
    if model is None:
        # Arm hosts list implementer and part codes instead of a model name
        try:
            fields = {}
            for line in open("/proc/cpuinfo"):
                if ":" in line:
                    k, v = line.split(":", 1)
                    fields.setdefault(k.strip(), v.strip())
            if "CPU implementer" in fields:
                model = f"implementer {fields['CPU implementer']} part {fields.get('CPU part')}"
        except OSError:
            pass
    import platform
    return {"model": model, "machine": platform.machine(), "nproc": os.cpu_count()}


def cpu_baseline(problem, seconds_budget=25.0):
    """The CPU oracle as it stands (FP64; the OpenMP build on all host cores
    where the compiler has OpenMP) on a bounded sample of the same workload:
    whole SSP-RK3 steps of the full grid."""
    import oracle
    f, g, W = oracle.setup(problem)
    dt, _ = oracle.dt(f, g, W, problem.cfl)
    p = oracle.make_params()
    omp = oracle.has_omp()
    threads = oracle.threads(omp)
    W = oracle.step(f, p, g, W, dt, 1, omp=omp)  # loads the library, touches the memory
    t0 = time.perf_counter()
    steps = 0
    while True:
        W = oracle.step(f, p, g, W, dt, 1, omp=omp)
        steps += 1
        el = time.perf_counter() - t0
        if el > seconds_budget * 0.5 or steps >= 40:
            break
    return {"value": problem.ncells * steps / el, "unit": UNIT, "cores": threads, "kind": "oracle",
            "host": host_cpu(),
            "sample": f"{steps} full SSP-RK3 step(s) of the {problem.n[0]}x{problem.n[1]} workload "
                      f"({el:.1f} s, FP64 C++ oracle, {'OpenMP over grid lines, ' if omp else ''}"
                      f"{threads} thread(s))"}


def cpu_serial_rates():
    """The serial oracle (one host core) on the benchmark configurations, per
    cell-update: the 400-cell tube to its final time, five steps of the
    1024x512 workload, two steps of a 64^3 box of the 3D configuration."""
    import oracle
    from paper_2208_04488_gb300 import problems
    out = {}
    for name, pr, nsteps in (("tube_400_full_run", problems.shock_tube_1d_baseline(400), None),
                             ("shock_bubble_1024x512_5_steps", problems.shock_bubble_2d(1024, 512), 5),
                             ("interface_3d_64^3_2_steps", problems.interface_3d(64), 2)):
        f, g, W = oracle.setup(pr)
        p = oracle.make_params()
        t0 = time.perf_counter()
        steps, t = 0, 0.0
        while (nsteps is None and t < pr.t_end * (1 - 1e-14)) or (nsteps is not None and steps < nsteps):
            dt, _ = oracle.dt(f, g, W, pr.cfl if pr.D < 3 else 0.4)
            if nsteps is None:
                dt = min(dt, pr.t_end - t)
            W = oracle.step(f, p, g, W, dt, 1)
            t += dt
            steps += 1
        el = time.perf_counter() - t0
        out[name] = {"value": pr.ncells * steps / el, "unit": UNIT, "steps": steps, "seconds": round(el, 2)}
    return {"cores": 1, "kind": "oracle (serial build)", "runs": out}


def run_reference(args):
    """--impl reference: the CPU oracle timed on the host cores (rank 0 only)."""
    ws, rank, _ = dist_env()
    if rank != 0:
        return
    from paper_2208_04488_gb300 import problems
    pr = problems.shock_bubble_2d(1024, 512)
    import oracle
    f, g, W = oracle.setup(pr)
    dt, _ = oracle.dt(f, g, W, pr.cfl)
    p = oracle.make_params()
    omp = oracle.has_omp()
    threads = oracle.threads(omp)
    for _ in range(args.warmup):
        W = oracle.step(f, p, g, W, dt, 1, omp=omp)
    t0 = time.perf_counter()
    for _ in range(args.steps):
        W = oracle.step(f, p, g, W, dt, 1, omp=omp)
    el = time.perf_counter() - t0
    value = pr.ncells * args.steps / el
    line = {"impl": "reference", "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": args.gpus,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * el / args.steps,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
            "data": "synthetic", "config": {"workload": WORKLOAD, "cells": pr.ncells},
            "cpu_baseline": {"value": value, "unit": UNIT, "cores": threads, "kind": "oracle",
                             "host": host_cpu(),
                             "sample": f"{args.steps} full SSP-RK3 steps of the 1024x512 workload, FP64 C++ "
                                       f"oracle, {threads} host thread(s)"},
            "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


def time_steps(torch, s, K, flush, ev_stream, dt=0.0):
    """K single steps, each bracketed by CUDA events on the library's stream,
    with an L2 flush (a write larger than L2) before each. The step graph
    carries an event pair around every kernel (hrm_set_profiling), read after
    each step; dt <= 0: the automatic CFL step. Returns (seconds,
    {kernel kind: (launches, seconds)})."""
    total = 0.0
    per = {}
    for _ in range(K):
        flush.fill_(1.0)
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record(ev_stream)
        s.step(dt, 1)
        e1.record(ev_stream)
        e1.synchronize()
        total += e0.elapsed_time(e1) * 1e-3
        for kind, ms in s.profile_read():
            n, t = per.get(kind, (0, 0.0))
            per[kind] = (n + 1, t + ms * 1e-3)
    return total, per


def measure_batched(torch, hrm, problems, stream, flush, args):
    """64 seeded 2D instances (128x128 .. 1024x512, 2-3 species, Mach 1.2-3)
    advanced together, one persistent launch per RK stage: the launch shape
    autotuned per form, then total-cells-weighted cell-updates/s of both
    forms."""
    ps = problems.batch_instances(64, seed=4242)
    out = {"instances": len(ps), "total_cells": int(sum(p.ncells for p in ps)),
           "species": sorted({p.N for p in ps}), "scaling": "n/a (one GPU)"}
    for name, prec in (("fp32", hrm.FP32), ("fp64", hrm.FP64)):
        b = hrm.BatchSolver(ps, params=hrm.params_default(cfl=0.4, check=0, precision=prec), stream=stream)
        t0 = time.perf_counter()
        shape = b.tune(1)
        tune_s = time.perf_counter() - t0
        K = max(8, args.steps // 2) if prec == hrm.FP64 else max(3, args.steps)
        b.step(1)
        torch.cuda.synchronize()
        l0 = b.kernel_launches()
        total = 0.0
        for _ in range(K):
            flush.fill_(1.0)
            e0 = torch.cuda.Event(enable_timing=True)
            e1 = torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            b.step(1)
            e1.record(stream)
            e1.synchronize()
            total += e0.elapsed_time(e1) * 1e-3
        out[name] = {"value": out["total_cells"] * K / total, "unit": UNIT, "ms_per_step": 1e3 * total / K,
                     "steps": K, "launches_per_step": (b.kernel_launches() - l0) / K,
                     "tuned_shape": {"cell_tile": shape["cell_tile"], "blocks_per_sm": shape["blocks_per_sm"]},
                     "tune_seconds": tune_s, "admissibility_after": b.admissibility()}
        del b
    return out


def measure_tube(torch, hrm, problems, stream):
    """The first configuration: the 400-cell water-air tube run to its final
    time (CFL steps from the device, one graph launch per step). 16 KB of state:
    the rate measures the step graph's latency, not the kernels' throughput."""
    pr = problems.shock_tube_1d_baseline(400)
    s = hrm.Solver.from_problem(pr, params=hrm.params_default(cfl=pr.cfl, check=0), stream=stream)
    s.step(0.0, 10)
    s.set_primitive(pr.prim)
    torch.cuda.synchronize()
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    n = 0
    e0.record(stream)
    t = 0.0
    while t < pr.t_end:
        s.step(0.0, 50)
        n += 50
        t, _ = s.time()
    e1.record(stream)
    e1.synchronize()
    el = e0.elapsed_time(e1) * 1e-3
    out = {"workload": "1D water-air shock tube, 400 cells, CFL 0.4, to t = 2.4e-4 s", "steps": n, "t": t,
           "value": pr.ncells * n / el, "unit": UNIT, "us_per_step": 1e6 * el / n,
           "admissibility_after": s.admissibility(), "note": "latency-bound (one graph launch per step)"}
    s.close()
    return out


def measure_3d(torch, hrm, problems, stream, flush, args):
    """The 3D configuration: the 256^3 perturbed liquid-gas interface hit by a
    Mach 1.5 shock (three species, periodic in y and z). Both forms advance the
    same fixed steps from the initial state (L2 flushed before each, CUDA events
    around each step); the precision form's relative L1 error against FP64."""
    from paper_2208_04488_gb300.metrics import rel_l1_state
    pr = problems.interface_3d(256)
    out = {"workload": "3D perturbed interface, 256^3 cells, Mach 1.5 shock, water + air + helium, SSP-RK3",
           "cells": pr.ncells}
    s64 = hrm.Solver.from_problem(pr, params=hrm.params_default(cfl=0.4, check=0), stream=stream)
    dt, _ = s64.dt(0.4)
    dt *= 0.8
    states = {}
    for name, prec, K in (("fp32", hrm.FP32, max(3, args.steps // 2)), ("fp64", hrm.FP64, 3)):
        s = s64 if prec == hrm.FP64 else hrm.Solver.from_problem(
            pr, params=hrm.params_default(cfl=0.4, check=0, precision=prec), stream=stream)
        total = 0.0
        for _ in range(K):
            flush.fill_(1.0)
            e0 = torch.cuda.Event(enable_timing=True)
            e1 = torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            s.step(dt, 1)
            e1.record(stream)
            e1.synchronize()
            total += e0.elapsed_time(e1) * 1e-3
        out[name] = {"value": pr.ncells * K / total, "unit": UNIT, "ms_per_step": 1e3 * total / K, "steps": K,
                     "admissibility_after": s.admissibility()}
        if prec == hrm.FP32:
            # the error run: three more steps from the initial state, as the FP64 run does
            s.set_primitive(pr.prim)
            s.step(dt, 3)
        states[name] = s.get(hrm.FIELD_W)
        s.close()
    out["fp32"]["rel_l1_vs_fp64"] = {"max_over_variables": float(max(rel_l1_state(states["fp32"], states["fp64"],
                                                                                 pr.N, pr.D))),
                                     "after_steps": 3, "dt": dt}
    return out


def measure_decomposed(torch, hrm, problems, dist, rank, ws, stream):
    """The 256^3 3D configuration split over the ranks (one GPU each) into
    slabs along z with 3 ghost layers per inner side: halo layers exchanged
    with NCCL before every RK stage, the CFL maxima max-reduced per step
    (paper_2208_04488_gb300.decomp). All ranks take part; the whole grid's
    cell-updates over the slowest rank's time (CUDA events on the library's
    stream, after a barrier)."""
    from paper_2208_04488_gb300 import decomp
    from paper_2208_04488_gb300.replicas import whole_job_rate
    pr = problems.interface_3d(256)
    slab = decomp.partition(pr.n[-1], ws, periodic=True)[rank]
    loc = decomp.local_problem(pr, slab)
    out = {"workload": "3D perturbed interface, 256^3 cells, Mach 1.5 shock, water + air + helium, SSP-RK3, "
                       f"split into {ws} slabs along z (periodic), 3 ghost layers per inner side",
           "cells": pr.ncells, "ranks": ws, "owned_layers": slab.count, "exchange": "NCCL send/recv per stage",
           "scaling": "strong"}
    for name, prec, K in (("fp32", hrm.FP32, 6), ("fp64", hrm.FP64, 2)):
        s = hrm.Solver.from_problem(loc, params=hrm.params_default(cfl=pr.cfl, check=0, precision=prec),
                                    stream=stream)
        run = decomp.Decomposed(s, slab, decomp.TorchComm(dist, device="cuda"), device_buffers=True)
        run.step(1)
        dist.barrier()
        torch.cuda.synchronize()
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        b0 = run.exchanged_bytes
        e0.record(stream)
        run.step(K)
        e1.record(stream)
        e1.synchronize()
        el = e0.elapsed_time(e1) * 1e-3
        rate, t_max = whole_job_rate(pr.ncells * K, el, dist, device="cuda")
        out[name] = {"value": rate, "unit": UNIT, "ms_per_step": 1e3 * t_max / K, "steps": K,
                     "halo_bytes_sent_per_step_per_rank": (run.exchanged_bytes - b0) / K}
        s.close()
    return out


def gated_face_flops(problem, cfl, W_end=None):
    """Algorithmic flops per midpoint with every midpoint gated to the linear
    WENO weights (oracle counting build), per direction; with W_end, the mean of
    the counts on the initial state and on W_end."""
    import oracle
    f, g, W0 = oracle.setup(problem)

    def count(W):
        dt, _ = oracle.dt(f, g, W, cfl)
        lam = oracle.lambdas(f, g, W, dt)
        out = []
        for d in range(problem.D):
            c, nf = oracle.faces_flops(f, oracle.make_params(), g, W, lam, d, gated=True)
            out.append(sum(c.values()) / nf)
        return out

    a = count(W0)
    if W_end is None:
        return a
    b = count(np.ascontiguousarray(W_end, dtype=np.float64))
    return [0.5 * (x + y) for x, y in zip(a, b)]


def train_detector(hrm, stream):
    """The learned smoothness gate, trained on the GPU on stencils of the
    method's own runs (1D shock tube, 2D shock-bubble 1024x512, 3D interface
    128^3); returns (detector, report dict)."""
    from paper_2208_04488_gb300 import learned
    det, rep = learned.build_detector(scale="full", steps=4000, stream=stream)
    ev = det.evaluate(0.5, bf16=True)
    n = max(1, ev["tp"] + ev["fp"] + ev["tn"] + ev["fn"])
    return det, {"samples": rep.samples, "rough_fraction": rep.rough / max(1, rep.samples),
                 "per_source": rep.per_source, "collect_s": rep.collect_s, "train_s": rep.train_s,
                 "adam_steps": rep.steps, "batch": 4096, "delta": 0.01,
                 "loss_first_last": [float(rep.losses[:20].mean()), float(rep.losses[-200:].mean())],
                 "train_accuracy_bf16": (ev["tp"] + ev["tn"]) / n,
                 "train_rough_as_smooth_rate": ev["fp"] / max(1, ev["fp"] + ev["tn"])}


def run_form(torch, hrm, pr, precision, det, dt, steps, warmup, flush, stream, threshold=0.5):
    """One form of the method on a problem: W warm-up steps, restart from the
    initial condition, then `steps` timed steps of size dt (L2 flushed before
    each). Returns timing, per-kernel times, gated share, final state."""
    prm = hrm.params_default(cfl=pr.cfl, check=0, precision=precision)
    s = hrm.Solver.from_problem(pr, params=prm, stream=stream)
    if det is not None:
        s.set_detector(det)
        s.set_params(hrm.params_default(cfl=pr.cfl, check=0, precision=precision, learned=hrm.LEARNED_GATE,
                                        learned_threshold=threshold))
    s.set_profiling(True)
    for _ in range(warmup):
        s.step(dt, 1)
    s.set_primitive(pr.prim)
    torch.cuda.synchronize()
    l0 = s.kernel_launches()
    t, per = time_steps(torch, s, steps, flush, stream, dt)
    out = {"t": t, "per": per, "launches": s.kernel_launches() - l0, "adm": s.admissibility(),
           "W": s.get(hrm.FIELD_W)}
    # gate bytes: 1 linear weights, 0 full WENO-IS, 2 (precision form) a
    # uniform stencil, which takes the exact node flux
    gb = np.concatenate([s.get_gate(d) for d in range(pr.D)]) if det is not None else np.zeros(1, np.uint8)
    out["gated"] = float(np.mean(gb != 0)) if det is not None else 0.0
    out["gated_uniform"] = float(np.mean(gb == 2)) if det is not None else 0.0
    s.close()
    return out


def final_time_errors(hrm, pr, det, stream, nsteps):
    """The workload's full run (its configuration's step count): FP64 with the
    CFL step of each step's start state, then the precision form, FP32 + learned
    and FP64 + learned with the same sequence of steps; each form's relative L1
    error against FP64 at the final time."""
    from paper_2208_04488_gb300.metrics import rel_l1_state
    prm = hrm.params_default(cfl=pr.cfl, check=0)
    s = hrm.Solver.from_problem(pr, params=prm, stream=stream)
    dts = []
    for _ in range(nsteps):
        dt, _ = s.dt(pr.cfl)
        dts.append(dt)
        s.step(dt, 1)
    ref = s.get(hrm.FIELD_W)
    t_final = s.time()[0]
    out = {"steps": nsteps, "t_final": t_final, "dt_source": "CFL step of the FP64 run, replayed by every form",
           "fp64_admissibility": s.admissibility()}
    s.close()
    forms = [("fp32", hrm.FP32, False), ("fp32_learned", hrm.FP32, True), ("fp64_learned", hrm.FP64, True)]
    for name, prec, gated in forms:
        if gated and det is None:
            continue
        s = hrm.Solver.from_problem(pr, params=hrm.params_default(cfl=pr.cfl, check=0, precision=prec),
                                    stream=stream)
        if gated:
            s.set_detector(det)
            s.set_params(hrm.params_default(cfl=pr.cfl, check=0, precision=prec, learned=hrm.LEARNED_GATE))
        for dt in dts:
            s.step(dt, 1)
        l1 = rel_l1_state(s.get(hrm.FIELD_W), ref, pr.N, pr.D).tolist()
        out[name] = {"rel_l1_vs_fp64": max(l1), "per_variable": l1, "admissibility": s.admissibility()}
        s.close()
    return out


def sweep_time(hrm, per, D):
    """(launches, seconds) of the per-midpoint sweeps: the D sweeps of a stage run
    concurrently (D > 1), so their time is the bracket around all of them
    (HRM_KERNEL_SWEEPS), shared by the launches; each sweep's own bracket
    overlaps the others'."""
    kinds = [hrm.KERNEL_FACE_X + d for d in range(D)]
    n = sum(per[k][0] for k in kinds if k in per)
    t = per[hrm.KERNEL_SWEEPS][1] if hrm.KERNEL_SWEEPS in per else sum(per[k][1] for k in kinds if k in per)
    return n, t


def time_shares(hrm, per, D):
    """Share of each non-overlapping bracket (the sweeps as one) in their sum."""
    skip = {hrm.KERNEL_FACE_X + d for d in range(D)} if hrm.KERNEL_SWEEPS in per else set()
    tot = sum(v[1] for k, v in per.items() if k not in skip)
    return {hrm.KERNEL_NAMES[k]: round(v[1] / tot, 4) for k, v in sorted(per.items()) if k not in skip}


def form_summary(hrm, pr, r, ref_W, steps, face_fl, face_fl_gated, peak, peak_name):
    """JSON block of one form: throughput, L1 error against plain FP64 after the
    same equal steps, and the per-midpoint kernel's achieved fraction of the
    pipe peak (algorithmic flops of the midpoints as gated)."""
    from paper_2208_04488_gb300.metrics import rel_l1_state
    n, tf = sweep_time(hrm, r["per"], pr.D)
    g = r["gated"]
    fl = sum((g * face_fl_gated[d] + (1 - g) * face_fl[d][0]) * face_fl[d][1] for d in range(pr.D)) / pr.D
    gate_t = r["per"].get(hrm.KERNEL_GATE, (0, 0.0))
    l1 = rel_l1_state(r["W"], ref_W, pr.N, pr.D).tolist() if ref_W is not None else None
    return {"value": pr.ncells * steps / r["t"], "unit": UNIT, "ms_per_step": 1e3 * r["t"] / steps,
            "gated_share": g, "gated_share_uniform": r.get("gated_uniform", 0.0),
            "rel_l1_vs_fp64": None if l1 is None else {"max_over_variables": max(l1), "per_variable": l1},
            "admissibility_after": r["adm"],
            "launches_per_step": r["launches"] / steps,
            "face_kernel": {"avg_launch_ms": 1e3 * tf / n, "achieved_tflops": fl / (tf / n) / 1e12,
                            "peak_tflops": peak / 1e12, "peak": peak_name, "frac": fl / (tf / n) / peak},
            "gate_kernel_ms_per_step": 1e3 * gate_t[1] / steps}


def measure_learned_workload(torch, hrm, problems, det, stream, flush, args, fp64_peak, fp32_peak):
    """The learned-detector workload: 2D shock-water column with an SF6 bubble,
    2048 x 1024 (Sec. 5.7 shape, paper fluids), a problem the detector was not
    trained on. Plain FP64, FP32, FP32+learned and FP64+learned, equal fixed
    steps from the initial condition; errors against plain FP64."""
    from paper_2208_04488_gb300 import learned
    pr = problems.shock_water_column_2d(2048, 1024)
    s0 = hrm.Solver.from_problem(pr, params=hrm.params_default(cfl=pr.cfl, check=0), stream=stream)
    dt0, _ = s0.dt(pr.cfl)
    s0.close()
    dt = 0.8 * dt0
    K = max(4, args.steps // 2)
    ref = run_form(torch, hrm, pr, hrm.FP64, None, dt, K, args.warmup, flush, stream)
    faces = run_face_flops(pr, pr.cfl, ref["W"])
    faces_g = gated_face_flops(pr, pr.cfl, ref["W"])
    out = {"workload": "2D shock-water column + SF6 bubble, 2048x1024, Mach 1.47, paper fluids, CFL 0.5 "
                       "(0.8 x the initial CFL step, fixed)", "cells": pr.ncells, "steps": K, "dt": dt,
           "validation_on_this_workload": learned.validation(det, problems.shock_water_column_2d(1024, 512), 100,
                                                             3, 0.5, stream=stream)}
    out["fp64"] = form_summary(hrm, pr, ref, None, K, faces, faces_g, fp64_peak, "fp64 fma probe")
    for name, prec, d in (("fp32", hrm.FP32, None), ("fp32_learned", hrm.FP32, det),
                          ("fp64_learned", hrm.FP64, det)):
        r = run_form(torch, hrm, pr, prec, d, dt, K, args.warmup, flush, stream)
        out[name] = form_summary(hrm, pr, r, ref["W"], K, faces, faces_g,
                                 fp64_peak if prec == hrm.FP64 else fp32_peak,
                                 "fp64 fma probe" if prec == hrm.FP64 else "fp32 fma probe")
    out["speedup_fp32_learned_vs_fp64"] = out["fp32_learned"]["value"] / out["fp64"]["value"]
    return out


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=20)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-batch", action="store_true")
    ap.add_argument("--no-learned", action="store_true")
    ap.add_argument("--no-3d", action="store_true")
    ap.add_argument("--final-steps", type=int, default=2000,
                    help="steps of the full-run error comparison (the configuration's 2000; 0: skip)")
    ap.add_argument("--nx", type=int, default=1024)
    ap.add_argument("--ny", type=int, default=512)
    args = ap.parse_args()
    if args.impl == "reference":
        return run_reference(args)

    import torch
    ws, rank, local = dist_env()
    torch.cuda.set_device(local)
    dist = None
    if ws > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl", device_id=torch.device("cuda", local))
    from paper_2208_04488_gb300 import build, hrm, problems
    if rank == 0:
        build.build()
    if dist is not None:
        dist.barrier()
    pr = problems.shock_bubble_2d(args.nx, args.ny)
    stream = torch.cuda.current_stream()

    def make(precision):
        prm = hrm.params_default(cfl=pr.cfl, check=0, precision=precision)
        return hrm.Solver.from_problem(pr, params=prm, stream=stream)

    flush = torch.empty(256 * 1024 * 1024 // 4, dtype=torch.float32, device="cuda")
    s = make(hrm.FP64)
    s.set_profiling(True)
    for _ in range(args.warmup):
        s.step(0.0, 1)
    torch.cuda.synchronize()
    s.set_primitive(pr.prim)  # timed run starts from the initial condition
    launches0 = s.kernel_launches()
    if dist is not None:
        dist.barrier()
    torch.cuda.synchronize()
    with Clocks(local) as clk:
        t_dev, per_kernel = time_steps(torch, s, args.steps, flush, stream)
    launches = s.kernel_launches() - launches0
    torch.cuda.synchronize()
    adm = s.admissibility()
    W_fp64 = s.get(hrm.FIELD_W)
    from paper_2208_04488_gb300.replicas import whole_job_rate
    value, t_max = whole_job_rate(pr.ncells * args.steps, t_dev, dist, device="cuda")

    # end-to-end through the public API with host buffers, on every rank: the
    # same steps from the initial condition, the state living in pinned host
    # memory; per step it is uploaded, advanced one step and read back into the
    # host state the next step uploads.
    s.set_primitive(pr.prim)
    Wh = torch.from_numpy(s.get(hrm.FIELD_W)).pin_memory()
    Wdev = torch.empty(Wh.shape, dtype=torch.float64, device="cuda")
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    K_e2e = args.steps
    if dist is not None:
        dist.barrier()
    torch.cuda.synchronize()
    e0.record(stream)
    for _ in range(K_e2e):
        Wdev.copy_(Wh, non_blocking=True)
        s.set(Wdev)
        s.step(0.0, 1)
        s.get(hrm.FIELD_W, out=Wdev)
        Wh.copy_(Wdev, non_blocking=True)
    e1.record(stream)
    e1.synchronize()
    t_e2e = e0.elapsed_time(e1) * 1e-3
    bytes_step = Wh.numel() * 8
    e2e_value, _ = whole_job_rate(pr.ncells * K_e2e, t_e2e, dist, device="cuda")
    s.set(W_fp64)  # back to the state after the timed steps (the fixed dt below comes from it)
    # more than one GPU: the 3D configuration decomposed over all of them
    decomposed = measure_decomposed(torch, hrm, problems, dist, rank, ws, stream) if dist is not None else None
    if dist is not None:
        # the other replicas are done: rank 0 measures the rest alone, with no
        # collective after this point
        dist.barrier()
        if rank != 0:
            dist.destroy_process_group()
            return
    # precision form on the same workload: timed the same way, and its relative
    # L1 error against FP64 after the same number of equal fixed-size steps
    s32 = make(hrm.FP32)
    s32.set_profiling(True)
    for _ in range(args.warmup):
        s32.step(0.0, 1)
    s32.set_primitive(pr.prim)
    torch.cuda.synchronize()
    t32, per32 = time_steps(torch, s32, args.steps, flush, stream)
    adm32 = s32.admissibility()
    dt0, _ = s.dt(pr.cfl)
    ea, eb = make(hrm.FP64), make(hrm.FP32)
    ea.step(dt0, args.steps)
    eb.step(dt0, args.steps)
    Wa, Wb = ea.get(hrm.FIELD_W), eb.get(hrm.FIELD_W)
    from paper_2208_04488_gb300.metrics import rel_l1_state
    l1_32 = rel_l1_state(Wb, Wa, pr.N, pr.D).tolist()
    del ea, eb, s32

    # learned smoothness gate (rank 0): trained on the GPU on the method's own
    # stencils, then the gated forms on this workload (same fixed steps as the
    # error runs above) and on the shock-water-column workload
    det = learned_runs = None
    if rank == 0 and not args.no_learned:
        det, train_rep = train_detector(hrm, stream)
        learned_runs = {name: run_form(torch, hrm, pr, prec, det, dt0, args.steps, args.warmup, flush, stream)
                        for name, prec in (("fp32_learned", hrm.FP32), ("fp64_learned", hrm.FP64))}

    # batched form: the 64 seeded uneven instances, one persistent launch per phase
    batched = measure_batched(torch, hrm, problems, stream, flush, args) if rank == 0 and not args.no_batch else None
    three_d = measure_3d(torch, hrm, problems, stream, flush, args) if rank == 0 and not args.no_3d else None
    tube = measure_tube(torch, hrm, problems, stream) if rank == 0 else None
    final = (final_time_errors(hrm, pr, det, stream, args.final_steps)
             if rank == 0 and args.final_steps > 0 else None)


    line = None
    if rank == 0:
        pk, pk_src = peaks()
        fp64_peak = hrm.probe_fma_peak(hrm.FP64)
        fp32_peak = hrm.probe_fma_peak(hrm.FP32)
        # flops of the method per midpoint over the timed steps (they start from
        # the initial state and end at W_fp64)
        faces = run_face_flops(pr, pr.cfl, W_fp64)
        # dominant kernels: the per-midpoint sweeps (one launch per direction and
        # stage); algorithmic flops per launch / average launch duration
        fl_launch = sum(faces[d][0] * faces[d][1] for d in range(pr.D)) / pr.D
        n_face, t_face = sweep_time(hrm, per_kernel, pr.D)
        achieved = fl_launch / (t_face / n_face)
        frac = achieved / fp64_peak
        share = time_shares(hrm, per_kernel, pr.D)
        n32, tf32 = sweep_time(hrm, per32, pr.D)
        ach32 = fl_launch / (tf32 / n32)
        share32 = time_shares(hrm, per32, pr.D)
        # the precision form's sweep finishes a uniform stencil exactly (the node
        # flux) without the method's arithmetic: the share of such midpoints, as
        # the learned form's sweep reports it in its gate bytes (byte 2) at the
        # end of the same steps, and the sweep's compulsory bytes per launch (the
        # FP32 planes of the cells read once, the FP64 flux planes written once)
        uni = (learned_runs["fp32_learned"].get("gated_uniform") if learned_runs is not None else None)
        nfx = (pr.n[0] + 1) * int(np.prod(pr.n[1:]))
        bytes32 = 4 * (pr.M + 4 + pr.D + pr.N - 1) * pr.ncells + 8 * (pr.M + pr.N - 1) * nfx
        learned_block = None
        if learned_runs is not None:
            faces_g = gated_face_flops(pr, pr.cfl, W_fp64)
            learned_block = {"detector": train_rep,
                             "threshold": 0.5,
                             "shock_water_column": measure_learned_workload(torch, hrm, problems, det, stream, flush,
                                                                            args, fp64_peak, fp32_peak)}
        line = {
            "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": ws, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": 1e3 * t_max / args.steps, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": {"workload": WORKLOAD, "cells": pr.ncells, "species": pr.N,
                       "l2": "working set ~190 MB > L2 and L2 flushed (256 MB write) before every timed step",
                       "parallelism": (f"{ws} independent replica(s); decomposed_3d: the 256^3 case split over {ws} GPUs"
                                       if ws > 1 else "single GPU")},
            "roofline": {"bound": "alu", "kernel": "k_face (per-midpoint, FP64)",
                         "achieved": achieved / 1e12, "peak": fp64_peak / 1e12, "unit": "TFLOP/s",
                         "frac": frac, "traffic": TRAFFIC_BYTES["k_face_fp64"],
                         "traffic_unit": "bytes per launch (ncu capture, y sweep)",
                         "fp64_pipe_active_ncu": FP64_PIPE_ACTIVE["k_face_fp64"],
                         "peak_source": "measured FP64 FMA-chain probe on this GPU (hrm_probe_fma_peak)",
                         "algorithmic_flops_per_face": [round(x[0], 1) for x in faces],
                         "flops_per_face_first_last_state": [x[2] for x in faces],
                         "first_order_flux_flops_per_nonuniform_midpoint": round(first_order_face_flops(pr, pr.cfl, 0), 1),
                         "flop_count": "the oracle's count of the method as written (add, mul, div, sqrt, "
                                       "tanh one flop each), the mean of its counts on the first and the last "
                                       "state of the timed steps; it includes the first-order HLLC flux at every "
                                       "non-uniform midpoint, which the sweep evaluates only where the flux "
                                       "limiter can act, and only the node flux at uniform stencils",
                         "avg_launch_ms": 1e3 * t_face / n_face, "launches_timed": n_face,
                         "launch_timing": "the x and y sweeps of a stage run concurrently: their common "
                                          "fork-to-join time, divided by the launches in it",
                         "kernel_time_share": share},
            "e2e": {"value": e2e_value, "unit": UNIT, "h2d_bytes_per_step": bytes_step,
                    "d2h_bytes_per_step": bytes_step},
            "forms": {
                "fp32": {"value": pr.ncells * args.steps / t32, "unit": UNIT,
                         "ms_per_step": 1e3 * t32 / args.steps,
                         "description": "WENO-IS, HLLC, HCS and sensor blend in FP32; limiter theta, half-cell "
                                        "states, state, RK combination and relaxation in FP64",
                         "rel_l1_vs_fp64": {"max_over_variables": max(l1_32), "per_variable": l1_32,
                                            "after_steps": args.steps, "dt": dt0,
                                            "definition": "sum|W32 - W64| / sum|W64| per variable; momentum "
                                                          "components over sum |rho u| (vector norm)"},
                         "admissibility_after": adm32,
                         "roofline": {"bound": "alu", "kernel": "k_face32_fast (per-midpoint, FP32 bulk; screen failures deferred to k_face32_fix on a forked stream, outside this timing)",
                                      "achieved": ach32 / 1e12, "unit": "TFLOP/s",
                                      "peak_fp32": fp32_peak / 1e12, "frac_of_fp32_peak": ach32 / fp32_peak,
                                      "peak_fp64": fp64_peak / 1e12,
                                      "avg_launch_ms": 1e3 * tf32 / n32, "kernel_time_share": share32,
                                      "traffic": TRAFFIC_BYTES["k_face32"],
                                      "flops_counted": "the oracle's count over the timed states, as for the "
                                                       "FP64 sweep: the method's arithmetic at non-uniform "
                                                       "midpoints, the node flux at uniform ones (the sweep "
                                                       "takes that flux where its FP32 planes are uniform); "
                                                       "the sweep is bound by the latency of its non-uniform "
                                                       "warps, not by the FP32 pipe (ncu: FMA pipe 13-14 %)",
                                      "uniform_share": uni,
                                      "hbm": {"compulsory_bytes_per_launch": bytes32,
                                              "achieved_gbs": bytes32 / (tf32 / n32) / 1e9,
                                              "peak_gbs": pk.get("hbm_gbs"),
                                              "frac": (bytes32 / (tf32 / n32) / 1e9 / pk["hbm_gbs"]
                                                       if pk.get("hbm_gbs") else None)}}},
            },
            "batched": batched,
            "interface_3d": three_d,
            "decomposed_3d": decomposed,
            "tube_400": tube,
            "final_time": final,
            "learned": learned_block,
            "gpu_launches": int(launches),
            "clocks": clk.summary(),
            "admissibility_after": adm,
            "peaks": {"fp64_fma_tflops": fp64_peak / 1e12, "fp32_fma_tflops": fp32_peak / 1e12,
                      "hbm_gbs": pk.get("hbm_gbs"), "hbm_source": pk_src},
        }
        if learned_runs is not None:
            for name, r in learned_runs.items():
                prec_peak = fp32_peak if name.startswith("fp32") else fp64_peak
                line["forms"][name] = form_summary(hrm, pr, r, Wa, args.steps, faces, faces_g, prec_peak,
                                                   "fp32 fma probe" if name.startswith("fp32") else "fp64 fma probe")
                line["forms"][name]["description"] = (
                    "learned smoothness gate (30-32-32-1 MLP, bf16 tcgen05 inference in a gate kernel before each sweep) "
                    "selects the linear "
                    "WENO weights where it predicts every weight within 0.01 of d_k; limiters always on; "
                    f"fixed dt = {dt0:.6g} s, errors after {args.steps} steps against plain FP64")
    if rank == 0:
        if not args.no_cpu_baseline and ws == 1:
            line["cpu_baseline"] = cpu_baseline(pr)
            line["cpu_baseline"]["serial"] = cpu_serial_rates()
        print(json.dumps(line), flush=True)
    if dist is not None:
        dist.destroy_process_group()


if __name__ == "__main__":
    main()
