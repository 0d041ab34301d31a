"""Domain decomposition on the GPU: the stagewise entry points (hrm_step_tau,
hrm_begin_step, hrm_stage, hrm_layers) and two ranks stepping subdomains of
one problem in lockstep (paper_2208_04488_gb300.decomp), against a single
context's hrm_step, bit for bit, in both forms.

The two ranks are two processes sharing one GPU, each with its own context,
exchanging halo layers and CFL maxima through gloo on the host: no kernel of
one rank waits for the other's.
"""
import os
import sys

import numpy as np
import pytest

from paper_2208_04488_gb300 import problems as P

pytestmark = pytest.mark.gpu
ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def hrm():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2208_04488_gb300 import build
    build.build()
    from paper_2208_04488_gb300 import hrm as H
    return H


def _problem(name):
    return {"2d": lambda: P.shock_bubble_2d(128, 64), "3d": lambda: P.interface_3d(24)}[name]()


def _single(H, pr, precision, nsteps):
    s = H.Solver.from_problem(pr, params=H.params_default(cfl=pr.cfl, check=0, precision=precision))
    s.step(0.0, nsteps)
    W = s.get(H.FIELD_W)
    t = s.time()
    s.close()
    return W, t


@pytest.mark.parametrize("precision", ["fp64", "fp32"])
def test_stagewise_steps_equal_hrm_step(hrm, precision):
    prec = hrm.FP64 if precision == "fp64" else hrm.FP32
    pr = P.shock_bubble_2d(96, 48)
    ref, t_ref = _single(hrm, pr, prec, 4)
    s = hrm.Solver.from_problem(pr, params=hrm.params_default(cfl=pr.cfl, check=0, precision=prec))
    assert s.stages() == 3
    for _ in range(4):
        s.begin_step(s.step_tau())
        for k in range(s.stages()):
            s.stage(k)
    np.testing.assert_array_equal(s.get(hrm.FIELD_W), ref)
    assert s.time() == t_ref
    # layers round trip: set what was read, nothing changes
    lay = s.get_layers(0, 5, 3)
    s.set_layers(0, 5, 3, lay)
    np.testing.assert_array_equal(s.get(hrm.FIELD_W), ref)
    np.testing.assert_array_equal(lay, ref[:, 5 * 96:8 * 96])
    with pytest.raises(hrm.HrmError):
        s.get_layers(0, 46, 3)
    with pytest.raises(hrm.HrmError):
        s.begin_step([-1.0, 1.0])
    s.close()


def _rank_main(rank, world, port, name, precision, nsteps, out_dir):
    import torch
    import torch.distributed as dist
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    sys.path.insert(0, ROOT)
    torch.cuda.set_device(0)
    from paper_2208_04488_gb300 import decomp as dc
    from paper_2208_04488_gb300 import hrm as H
    pr = _problem(name)
    slab = dc.partition(pr.n[-1], world, pr.bc[2 * pr.D - 2] == 1)[rank]
    loc = H.Solver.from_problem(dc.local_problem(pr, slab),
                                params=H.params_default(cfl=pr.cfl, check=0, precision=precision))
    run = dc.Decomposed(loc, slab, dc.TorchComm(dist))
    run.step(nsteps)
    W = run.gather()
    if rank == 0:
        np.save(os.path.join(out_dir, "W.npy"), W)
    loc.close()
    dist.barrier()
    dist.destroy_process_group()


@pytest.mark.parametrize("name", ["2d", "3d"])
@pytest.mark.parametrize("precision", ["fp64", "fp32"])
def test_two_ranks_equal_one_context(hrm, tmp_path, name, precision):
    import torch.multiprocessing as mp
    prec = hrm.FP64 if precision == "fp64" else hrm.FP32
    nsteps = 5
    port = 29100 + (os.getpid() % 1000) + 7 * (name == "3d") + 3 * (precision == "fp32")
    mp.start_processes(_rank_main, args=(2, port, name, prec, nsteps, str(tmp_path)), nprocs=2, join=True,
                       start_method="spawn")
    got = np.load(tmp_path / "W.npy")
    ref, _ = _single(hrm, _problem(name), prec, nsteps)
    np.testing.assert_array_equal(got, ref)


class _ThreadComm:
    """Two ranks as threads of one process: CUDA tensors pass through a mailbox
    (the exchange path NCCL takes, device buffers included). Every wait has a
    time limit, so a failing rank cannot leave the other blocked."""

    def __init__(self, rank, world, box):
        self.rank, self.world, self.box = rank, world, box

    def allreduce_max(self, values):
        b = self.box
        b["tau"][self.rank] = np.asarray(values, dtype=np.float64)
        b["bar"].wait()
        out = np.max(np.stack(b["tau"]), axis=0)
        b["bar"].wait()
        return out

    def exchange(self, sends, recvs):
        import torch
        b = self.box
        torch.cuda.current_stream().synchronize()
        with b["cv"]:
            for peer, tag, t in sends:
                b["mail"].setdefault((self.rank, peer, tag), []).append(t.clone())
            b["cv"].notify_all()
        for peer, tag, t in recvs:
            with b["cv"]:
                if not b["cv"].wait_for(lambda: b["mail"].get((peer, self.rank, tag)), timeout=120):
                    raise TimeoutError("halo message did not arrive")
                src = b["mail"][(peer, self.rank, tag)].pop(0)
            t.copy_(src)
        torch.cuda.synchronize()


def test_device_buffer_exchange_two_threads(hrm):
    """The decomposed driver with device-resident halo buffers (as with NCCL):
    two rank threads, each with its own context and stream, equal one context."""
    import threading
    import torch
    from paper_2208_04488_gb300 import decomp as dc
    pr = P.interface_3d(24)
    slabs = dc.partition(pr.n[-1], 2, True)
    box = {"cv": threading.Condition(), "bar": threading.Barrier(2, timeout=120), "tau": [None, None], "mail": {}}
    result, errors = {}, []

    def rank_main(r):
        try:
            torch.cuda.set_device(0)
            stream = torch.cuda.Stream()
            with torch.cuda.stream(stream):
                loc = hrm.Solver.from_problem(dc.local_problem(pr, slabs[r]),
                                              params=hrm.params_default(cfl=pr.cfl, check=0, precision=hrm.FP32),
                                              stream=stream)
                run = dc.Decomposed(loc, slabs[r], _ThreadComm(r, 2, box), device_buffers=True)
                run.step(4)
                result[r] = run.owned_state()
                loc.close()
        except Exception as e:  # reported by the main thread
            errors.append(e)
            box["bar"].abort()

    th = [threading.Thread(target=rank_main, args=(r,)) for r in range(2)]
    for t in th:
        t.start()
    for t in th:
        t.join(timeout=300)
    assert not errors, errors
    got = np.concatenate([result[0], result[1]], axis=1)
    ref, _ = _single(hrm, pr, hrm.FP32, 4)
    np.testing.assert_array_equal(got, ref)
