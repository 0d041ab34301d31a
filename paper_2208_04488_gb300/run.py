"""Command-line runner: advance one of the built-in workloads on the GPU.

    python -m paper_2208_04488_gb300.run --workload shock_bubble --nx 1024 --ny 512 \
        --steps 10 [--precision fp64|fp32] [--dt 0] [--gate none|all|learned] [--step-path 0|1]
    python -m paper_2208_04488_gb300.run --workload batch --steps 2 [--precision fp64|fp32]

Prints the wall time per step (CUDA events), the simulated time and the
admissibility counters. Used for profiling captures of single kernels.
"""
from __future__ import annotations

import argparse
import json
import os
import sys

sys.path.insert(0, os.path.dirname(os.path.dirname(os.path.abspath(__file__))))

WORKLOADS = ("shock_bubble", "shock_tube", "interface_3d", "water_column", "advection_2d", "mach100_jet",
             "undex", "batch")


def make_problem(name, nx, ny, nz):
    from paper_2208_04488_gb300 import problems as P
    if name == "shock_bubble":
        return P.shock_bubble_2d(nx, ny)
    if name == "shock_tube":
        return P.shock_tube_1d_baseline(nx)
    if name == "interface_3d":
        return P.interface_3d(nx)
    if name == "water_column":
        return P.shock_water_column_2d(nx, ny)
    if name == "advection_2d":
        return P.advection_2d_smooth(nx)
    if name == "mach100_jet":
        return P.mach100_jet_2d(nx, ny)
    if name == "undex":
        return P.undex_2d(nx, ny)
    raise ValueError(name)


def main(argv=None):
    ap = argparse.ArgumentParser()
    ap.add_argument("--workload", default="shock_bubble", choices=WORKLOADS)
    ap.add_argument("--nx", type=int, default=1024)
    ap.add_argument("--ny", type=int, default=512)
    ap.add_argument("--nz", type=int, default=0)
    ap.add_argument("--steps", type=int, default=3)
    ap.add_argument("--precision", default="fp64", choices=["fp64", "fp32"])
    ap.add_argument("--dt", type=float, default=0.0, help="0: CFL step of the workload")
    ap.add_argument("--gate", default="none", choices=["none", "all", "learned"],
                    help="all: every midpoint gated (fixed gate); learned: a detector trained on the small "
                         "training set")
    ap.add_argument("--step-path", type=int, default=0, choices=[0, 1],
                    help="1: the persistent stage kernel where the context allows it (hrm_set_step_path)")
    a = ap.parse_args(argv)
    import torch
    from paper_2208_04488_gb300 import build, hrm
    build.build()
    prec = hrm.FP64 if a.precision == "fp64" else hrm.FP32
    if a.workload == "batch":
        # the 64 seeded uneven 2D instances of the batched form, one persistent launch per stage
        from paper_2208_04488_gb300 import problems as P
        ps = P.batch_instances(64, seed=4242)
        b = hrm.BatchSolver(ps, params=hrm.params_default(cfl=0.4, precision=prec, check=0))
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record()
        b.step(a.steps)
        e1.record()
        e1.synchronize()
        print(json.dumps({"workload": "batch_64", "cells": b.total_cells(),
                          "ms_per_step": e0.elapsed_time(e1) / max(a.steps, 1), "admissibility": b.admissibility()}))
        return
    pr = make_problem(a.workload, a.nx, a.ny, a.nz)
    s = hrm.Solver.from_problem(pr, params=hrm.params_default(cfl=pr.cfl, precision=prec, check=0))
    s.set_step_path(a.step_path)
    if a.gate == "all":
        import numpy as np
        for d in range(pr.D):
            s.set_gate(d, np.ones(s.face_count(d), dtype=np.uint8))
        s.set_params(hrm.params_default(cfl=pr.cfl, precision=prec, check=0, learned=hrm.LEARNED_FIXED))
    elif a.gate == "learned":
        from paper_2208_04488_gb300 import learned
        det, _ = learned.build_detector(scale="small", steps=1000, capacity=1 << 21)
        s.set_detector(det)
        s.set_params(hrm.params_default(cfl=pr.cfl, precision=prec, check=0, learned=hrm.LEARNED_GATE))
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    e0.record()
    s.step(a.dt, a.steps)
    e1.record()
    e1.synchronize()
    t, n = s.time()
    out = {"workload": pr.name, "cells": pr.ncells, "steps": n, "t": t,
           "ms_per_step": e0.elapsed_time(e1) / max(a.steps, 1), "admissibility": s.admissibility()}
    print(json.dumps(out))


if __name__ == "__main__":
    main()
