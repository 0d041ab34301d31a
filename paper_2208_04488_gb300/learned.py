"""Training recipe of the learned smoothness gate.

The detector is trained on stencils the method itself produces: the solver
runs the source problems (a 1D water-air shock tube, a 2D three-species
shock-bubble interaction, a 3D perturbed liquid-gas interface hit by a shock),
and at a few snapshots every midpoint of every direction is labelled by the
WENO-IS weight deviation of the FP64 method and kept with a class-dependent
probability (all rough midpoints, a fraction of the smooth ones, a small
fraction of the uniform ones). The network is then trained with the library's
own forward, back-propagation and Adam kernels. Every computation runs in the
CUDA library; this module only sequences the calls.
"""
from __future__ import annotations

import time
from dataclasses import dataclass, field
from typing import List, Optional

import numpy as np

from . import hrm, problems as P


@dataclass
class Source:
    """A problem the detector learns from: run `steps_between` automatic-dt
    steps before each of `snapshots` collections."""
    problem: P.Problem
    snapshots: int
    steps_between: int
    precision: int = hrm.FP64
    keep_rough: float = 1.0
    keep_smooth: float = 0.1
    keep_flat: float = 0.01


def default_sources(scale: str = "full") -> List[Source]:
    """The training problems: the 400-cell water-air shock tube, the 2D
    shock-bubble interaction (1024 x 512; 256 x 128 when scale="small"), the
    3D perturbed interface (128^3; 32^3 when small) and the periodic smooth
    advection of Sec. 5.2 (256^2; 128^2 when small), whose volume fractions
    vary smoothly at every midpoint (the other problems' smooth stencils are
    mostly interface tails)."""
    small = scale == "small"
    tube = P.shock_tube_1d_baseline(400)
    bubble = P.shock_bubble_2d(256, 128) if small else P.shock_bubble_2d(1024, 512)
    iface = P.interface_3d(32 if small else 128)
    adv = P.advection_2d_smooth(128 if small else 256)
    return [
        Source(adv, snapshots=3, steps_between=10, keep_smooth=0.3 if small else 0.05, keep_flat=0.01),
        Source(tube, snapshots=6, steps_between=60, keep_smooth=1.0, keep_flat=0.2),
        Source(bubble, snapshots=4, steps_between=40 if small else 150, precision=hrm.FP32,
               keep_smooth=0.2 if small else 0.05, keep_flat=0.02 if small else 0.005),
        Source(iface, snapshots=3, steps_between=20 if small else 60, precision=hrm.FP32,
               keep_rough=1.0 if small else 0.25, keep_smooth=0.1 if small else 0.02,
               keep_flat=0.01 if small else 0.001),
    ]


@dataclass
class TrainReport:
    samples: int = 0
    rough: int = 0
    collect_s: float = 0.0
    train_s: float = 0.0
    steps: int = 0
    losses: Optional[np.ndarray] = None
    per_source: list = field(default_factory=list)


def collect(det: "hrm.Detector", sources: List[Source], delta: float = 0.01, stream=None) -> TrainReport:
    rep = TrainReport()
    t0 = time.perf_counter()
    for src in sources:
        prm = hrm.params_default(cfl=src.problem.cfl, precision=src.precision, check=0)
        s = hrm.Solver.from_problem(src.problem, prm, stream=stream)
        got = 0
        for _ in range(src.snapshots):
            s.step(0.0, src.steps_between)
            got += det.collect(s, delta, src.keep_rough, src.keep_smooth, src.keep_flat)
        rep.per_source.append((src.problem.name, got))
        s.close()
    rep.collect_s = time.perf_counter() - t0
    rep.samples = det.size()
    return rep


def train(det: "hrm.Detector", steps: int = 4000, batch: int = 4096, lr: float = 2e-3,
          rep: Optional[TrainReport] = None) -> TrainReport:
    rep = rep or TrainReport()
    t0 = time.perf_counter()
    # two phases: a larger rate, then a tenth of it
    l1 = det.train(steps // 2, batch, lr)
    l2 = det.train(steps - steps // 2, batch, lr * 0.1)
    rep.train_s = time.perf_counter() - t0
    rep.steps = steps
    rep.losses = np.concatenate([l1, l2])
    return rep


def build_detector(scale: str = "full", seed: int = 2208, capacity: int = 1 << 22, steps: int = 4000,
                   delta: float = 0.01, stream=None):
    """Collect from the default sources and train; returns (detector, report)."""
    det = hrm.Detector(capacity=capacity, seed=seed, stream=stream)
    rep = collect(det, default_sources(scale), delta, stream=stream)
    _, y, _ = det.samples()
    rep.rough = int((y < 0.5).sum())
    train(det, steps=steps, rep=rep)
    return det, rep


def validation(det: "hrm.Detector", problem: P.Problem, steps_between: int, snapshots: int, threshold: float,
               delta: float = 0.01, precision: int = hrm.FP32, seed: int = 7, stream=None):
    """Confusion of `det` on midpoints of `problem` (a problem it was not trained
    on): every rough midpoint and a tenth of the others, labelled as in
    training. Positive = gated."""
    val = hrm.Detector(capacity=1 << 22, seed=seed, stream=stream)
    val.set_weights(det.get_weights())
    prm = hrm.params_default(cfl=problem.cfl, precision=precision, check=0)
    s = hrm.Solver.from_problem(problem, prm, stream=stream)
    for _ in range(snapshots):
        s.step(0.0, steps_between)
        val.collect(s, delta, 1.0, 0.1, 0.1)
    s.close()
    out = val.evaluate(threshold, bf16=True)
    out["samples"] = val.size()
    val.close()
    return out
