"""Domain decomposition of one problem over several ranks (one GPU each).

The fractional step shards by space. Rank r owns a slab of consecutive layers
along the slowest direction (y in 2D, z in 3D) and holds it with HALO = 3 ghost
layers on each side that borders another rank: a midpoint's stencil spans
nodes i-2..i+3 and the HCS flux difference of a cell reads node fluxes i-3..i+3
(Sec. 4.3.1), so an owned cell's update reads nothing beyond three layers. On
those inner sides the rank's context uses the transmissive boundary: only ghost
cells see the truncated stencils, and their values are replaced before they
are read again. One step is

    for each RK stage k:  exchange the halo layers of the state stage k reads;
                          at k = 0, take the maxima tau_d over all ranks
                          (Sec. 4.1.2: dt and the directional split sigma_d
                          come from the global maxima) and begin the step;
                          run stage k.

The relaxation is per cell and needs no exchange. Every owned cell then goes
through exactly the arithmetic of a single context over the whole grid, so the
result is the same bit for bit.

This module is host logic only. `local` is the per-rank solver (an
hrm.Solver, or any object with the same stage methods) and `comm` moves
arrays between ranks (TorchComm: torch.distributed with NCCL on GPUs or gloo
on the host). Dirichlet sides are not supported here.
"""
from __future__ import annotations

import dataclasses
from typing import List, Optional

import numpy as np

HALO = 3
TAG_DOWN, TAG_UP = 17, 18  # layers sent to the lower / the upper neighbour


@dataclasses.dataclass
class Slab:
    rank: int
    world: int
    first: int              # first owned layer (global index along the split direction)
    count: int              # owned layers
    ghost_lo: int           # ghost layers held below the owned ones (0 or HALO)
    ghost_hi: int           # ... and above
    lower: Optional[int]    # neighbour rank below (None: a physical side)
    upper: Optional[int]

    @property
    def local_layers(self) -> int:
        return self.ghost_lo + self.count + self.ghost_hi


def partition(n_split: int, world: int, periodic: bool) -> List[Slab]:
    """Slabs of n_split layers over `world` ranks, sizes differing by at most
    one; each rank must own at least HALO layers."""
    base, extra = divmod(n_split, world)
    sizes = [base + (1 if r < extra else 0) for r in range(world)]
    if world > 1 and min(sizes) < HALO:
        raise ValueError(f"{n_split} layers over {world} ranks: each rank needs at least {HALO}")
    slabs, first = [], 0
    for r, cnt in enumerate(sizes):
        lower = r - 1 if r > 0 else (world - 1 if periodic and world > 1 else None)
        upper = r + 1 if r < world - 1 else (0 if periodic and world > 1 else None)
        slabs.append(Slab(r, world, first, cnt, HALO if lower is not None else 0, HALO if upper is not None else 0,
                          lower, upper))
        first += cnt
    return slabs


def local_problem(pr, slab: Slab):
    """The rank's part of problem `pr`: its owned layers with their ghost
    layers (taken across the periodic wrap where the split direction is
    periodic), the same spacing, and transmissive sides where it borders
    another rank."""
    from . import problems
    D = pr.D
    ds = D - 1
    if any(b == 2 for b in pr.bc[:2 * D]):
        raise ValueError("domain decomposition supports transmissive and periodic sides only")
    n_split = pr.n[ds]
    layer = int(np.prod(pr.n[:ds])) if ds > 0 else 1
    rows = (np.arange(slab.first - slab.ghost_lo, slab.first + slab.count + slab.ghost_hi)) % n_split
    prim = pr.prim.reshape(pr.prim.shape[0], n_split, layer)[:, rows, :].reshape(pr.prim.shape[0], -1)
    n = list(pr.n)
    n[ds] = slab.local_layers
    dx = (pr.hi[ds] - pr.lo[ds]) / n_split
    lo, hi = list(pr.lo), list(pr.hi)
    lo[ds] = pr.lo[ds] + (slab.first - slab.ghost_lo) * dx
    hi[ds] = lo[ds] + n[ds] * dx
    bc = list(pr.bc[:2 * D])
    if slab.world > 1:
        bc[2 * ds] = 0 if slab.lower is not None else pr.bc[2 * ds]
        bc[2 * ds + 1] = 0 if slab.upper is not None else pr.bc[2 * ds + 1]
    return problems.Problem(f"{pr.name}_rank{slab.rank}", list(pr.gamma), list(pr.pinf), list(pr.cv), list(pr.q),
                            n, lo, hi, bc, np.ascontiguousarray(prim), cfl=pr.cfl, dt=pr.dt, t_end=pr.t_end,
                            nsteps=pr.nsteps, extra=dict(pr.extra))


class TorchComm:
    """Arrays between ranks with torch.distributed (an initialised default
    process group). NCCL moves CUDA tensors; gloo host tensors."""

    def __init__(self, dist, device: str = "cpu"):
        self.dist = dist
        self.device = device

    def allreduce_max(self, values: np.ndarray) -> np.ndarray:
        import torch
        t = torch.tensor(np.asarray(values, dtype=np.float64), device=self.device)
        self.dist.all_reduce(t, op=self.dist.ReduceOp.MAX)
        return t.cpu().numpy()

    def exchange(self, sends, recvs):
        """sends: [(peer, tag, tensor)]; recvs: [(peer, tag, tensor to fill)],
        posted in this order (NCCL pairs the messages of two ranks by order)."""
        d = self.dist
        ops = [d.P2POp(d.isend, t, peer, tag=tag) for peer, tag, t in sends]
        ops += [d.P2POp(d.irecv, t, peer, tag=tag) for peer, tag, t in recvs]
        if ops:
            for w in d.batch_isend_irecv(ops):
                w.wait()

    def gather_to_root(self, block, root: int = 0):
        """Blocks of every rank (a list on the root, None elsewhere); sizes may differ."""
        import torch
        d = self.dist
        t = torch.as_tensor(np.ascontiguousarray(block, dtype=np.float64)).to(self.device)
        sizes = [torch.zeros(1, dtype=torch.int64, device=self.device) for _ in range(d.get_world_size())]
        d.all_gather(sizes, torch.tensor([t.numel()], dtype=torch.int64, device=self.device))
        big = max(int(s.item()) for s in sizes)
        pad = torch.zeros(big, dtype=torch.float64, device=self.device)
        pad[:t.numel()] = t.reshape(-1)
        out = [torch.zeros(big, dtype=torch.float64, device=self.device) for _ in sizes]
        d.all_gather(out, pad)
        if d.get_rank() != root:
            return None
        return [o[:int(s.item())].cpu().numpy() for o, s in zip(out, sizes)]


class Decomposed:
    """Steps a subdomain in lockstep with the other ranks' (see the module
    docstring). `device_buffers`: exchange through device memory (NCCL);
    otherwise through host arrays."""

    def __init__(self, local, slab: Slab, comm, device_buffers: bool = False):
        self.local, self.slab, self.comm = local, slab, comm
        self.device_buffers = device_buffers
        self.layer = local.layer_cells()
        self.M = local.M
        self.exchanged_bytes = 0

    def _buf(self, count):
        import torch
        if self.device_buffers:
            return torch.empty((self.M, count * self.layer), dtype=torch.float64, device="cuda")
        return torch.empty((self.M, count * self.layer), dtype=torch.float64)

    def _get(self, stage, first, count):
        import torch
        b = self._buf(count)
        if self.device_buffers:
            self.local.get_layers(stage, first, count, out=b)
            return b
        return torch.from_numpy(self.local.get_layers(stage, first, count))

    def exchange(self, stage: int):
        s = self.slab
        own_lo, own_hi = s.ghost_lo, s.ghost_lo + s.count
        sends, recvs = [], []
        if s.lower is not None:
            sends.append((s.lower, TAG_DOWN, self._get(stage, own_lo, HALO)))
        if s.upper is not None:
            sends.append((s.upper, TAG_UP, self._get(stage, own_hi - HALO, HALO)))
        into_hi = self._buf(HALO) if s.upper is not None else None
        into_lo = self._buf(HALO) if s.lower is not None else None
        if s.upper is not None:
            recvs.append((s.upper, TAG_DOWN, into_hi))
        if s.lower is not None:
            recvs.append((s.lower, TAG_UP, into_lo))
        self.comm.exchange(sends, recvs)
        for where, b in ((own_hi, into_hi), (0, into_lo)):
            if b is not None:
                self.local.set_layers(stage, where, HALO, b if self.device_buffers else b.numpy())
        self.exchanged_bytes += sum(int(t.numel()) * 8 for _, _, t in sends)

    def step(self, nsteps: int = 1, dt: float = 0.0):
        for _ in range(nsteps):
            for k in range(self.local.stages()):
                if self.slab.world > 1:
                    self.exchange(k)
                if k == 0:
                    tau = self.comm.allreduce_max(self.local.step_tau()) if self.slab.world > 1 \
                        else self.local.step_tau()
                    self.local.begin_step(tau, dt)
                self.local.stage(k)

    def owned_state(self) -> np.ndarray:
        """W of the owned layers, (M, count x layer)."""
        return np.asarray(self.local.get_layers(0, self.slab.ghost_lo, self.slab.count))

    def gather(self, root: int = 0) -> Optional[np.ndarray]:
        """The whole grid's W on the root rank (None elsewhere)."""
        own = self.owned_state()
        if self.slab.world == 1:
            return own
        parts = self.comm.gather_to_root(own.reshape(-1), root)
        if parts is None:
            return None
        return np.concatenate([p.reshape(self.M, -1) for p in parts], axis=1)
