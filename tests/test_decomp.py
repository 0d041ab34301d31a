"""The domain decomposition's host logic on CPU (paper_2208_04488_gb300.decomp):
the slab partition, the local problems with their ghost layers, and two gloo
ranks stepping subdomains in lockstep -- halo exchange before every RK stage,
the CFL maxima reduced over the ranks (Sec. 4.1.2) -- against one domain over
the whole grid. The per-rank solver here is the CPU oracle taken one SSP-RK3
stage at a time (its right-hand side and relaxation; the Shu-Osher
combination written out below); the GPU tests run the same driver on the
library's contexts.
"""
import os
import sys

import numpy as np
import pytest

from paper_2208_04488_gb300 import decomp
from paper_2208_04488_gb300 import problems as P

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
RK3 = [(0.0, 1.0), (0.75, 0.25), (1.0 / 3.0, 2.0 / 3.0)]


class OracleLocal:
    """A subdomain stepped by the oracle one stage at a time: the same
    interface as hrm.Solver's stage methods."""

    def __init__(self, pr, orc):
        self.orc = orc
        self.f, self.g, W = orc.setup(pr)
        self.p = orc.make_params()
        self.Wn, self.Ws = W.copy(), W.copy()
        self.cfl, self.D, self.M, self.n, self.dx = pr.cfl, pr.D, pr.M, list(pr.n), pr.dx

    def layer_cells(self):
        return int(np.prod(self.n[:-1])) if self.D > 1 else 1

    def stages(self):
        return 3

    def step_tau(self):
        return self.orc.dt(self.f, self.g, self.Wn, self.cfl)[1]

    def begin_step(self, tau, dt=0.0):
        s = float(np.sum(tau))
        self.dt = dt if dt > 0 else self.cfl / s
        self.lam = [self.dt / ((tau[d] / s) * self.dx[d]) for d in range(self.D)]

    def stage(self, k):
        a, b = RK3[k]
        src = self.Wn if k == 0 else self.Ws
        R = self.orc.rhs(self.f, self.p, self.g, src, self.lam)
        W = self.orc.relax(self.f, self.g, a * self.Wn + b * (src + self.dt * R))
        if k == 2:
            self.Wn = W
        else:
            self.Ws = W

    def _state(self, stage):
        return self.Wn if stage == 0 else self.Ws

    def get_layers(self, stage, first, count, out=None):
        L = self.layer_cells()
        return np.ascontiguousarray(self._state(stage)[:, first * L:(first + count) * L])

    def set_layers(self, stage, first, count, buf):
        L = self.layer_cells()
        self._state(stage)[:, first * L:(first + count) * L] = np.asarray(buf).reshape(self.M, count * L)


def test_partition_sizes_neighbours_and_limits():
    s = decomp.partition(10, 3, periodic=False)
    assert [x.count for x in s] == [4, 3, 3] and [x.first for x in s] == [0, 4, 7]
    assert (s[0].lower, s[0].upper, s[2].lower, s[2].upper) == (None, 1, 1, None)
    assert (s[0].ghost_lo, s[0].ghost_hi, s[1].ghost_lo, s[1].ghost_hi) == (0, 3, 3, 3)
    p = decomp.partition(8, 2, periodic=True)
    assert (p[0].lower, p[0].upper, p[1].lower, p[1].upper) == (1, 1, 0, 0)
    assert all(x.ghost_lo == x.ghost_hi == 3 for x in p)
    one = decomp.partition(8, 1, periodic=True)[0]
    assert (one.lower, one.upper, one.ghost_lo, one.ghost_hi) == (None, None, 0, 0)
    with pytest.raises(ValueError):
        decomp.partition(5, 2, periodic=False)


def test_local_problem_takes_ghost_layers_across_the_wrap():
    pr = P.interface_3d(8)
    sl = decomp.partition(8, 2, periodic=True)
    loc = decomp.local_problem(pr, sl[0])
    assert loc.n == [8, 8, 10] and loc.bc[4:6] == [0, 0]
    layer = 64
    full = pr.prim.reshape(pr.prim.shape[0], 8, layer)
    got = loc.prim.reshape(pr.prim.shape[0], 10, layer)
    rows = [5, 6, 7, 0, 1, 2, 3, 4, 5, 6]
    for j, r in enumerate(rows):
        np.testing.assert_array_equal(got[:, j], full[:, r])
    assert loc.lo[2] == pytest.approx(-3 / 8) and loc.hi[2] == pytest.approx(7 / 8)
    tb = decomp.local_problem(P.shock_bubble_2d(16, 12), decomp.partition(12, 2, periodic=False)[1])
    assert tb.n == [16, 9] and tb.bc[2:4] == [0, 0] and tb.lo[1] == pytest.approx(0.25 * (6 - 3) / 3)


def _problem(name):
    if name == "2d":
        return P.shock_bubble_2d(24, 16)
    return P.interface_3d(8)


def _rank_main(rank, world, port, name, nsteps, out_dir):
    import torch.distributed as dist
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    sys.path.insert(0, ROOT)
    import oracle
    from paper_2208_04488_gb300 import decomp as dc
    pr = _problem(name)
    periodic = pr.bc[2 * pr.D - 2] == 1
    slab = dc.partition(pr.n[-1], world, periodic)[rank]
    run = dc.Decomposed(OracleLocal(dc.local_problem(pr, slab), oracle), slab, dc.TorchComm(dist))
    run.step(nsteps)
    W = run.gather()
    if rank == 0:
        np.save(os.path.join(out_dir, "W.npy"), W)
    dist.barrier()
    dist.destroy_process_group()


@pytest.mark.parametrize("name", ["2d", "3d_periodic"])
def test_two_gloo_ranks_equal_one_domain(orc, tmp_path, name):
    import torch.multiprocessing as mp
    nsteps = 3
    port = 29700 + (os.getpid() % 1500) + (0 if name == "2d" else 1)
    mp.start_processes(_rank_main, args=(2, port, name, nsteps, str(tmp_path)), nprocs=2, join=True,
                       start_method="spawn")
    got = np.load(tmp_path / "W.npy")
    pr = _problem(name)
    one = OracleLocal(pr, orc)
    single = decomp.Decomposed(one, decomp.partition(pr.n[-1], 1, False)[0], comm=None)
    single.step(nsteps)
    np.testing.assert_array_equal(got, one.Wn)
    # the steps moved the state (the comparison is not between initial states)
    assert not np.array_equal(one.Wn, orc.setup(pr)[2])
