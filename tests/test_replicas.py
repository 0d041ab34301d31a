"""The multi-rank path of bench.py on CPU: two gloo ranks agree on the whole-job
rate (all ranks' units over the slowest rank's time), and the reference arm
runs on rank 0 only (other ranks exit 0 without output)."""
import os
import subprocess
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _rank_main(rank, world, port, units, seconds, out_dir):
    import torch.distributed as dist
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    sys.path.insert(0, ROOT)
    from paper_2208_04488_gb300.replicas import whole_job_rate
    value, t_max = whole_job_rate(units[rank], seconds[rank], dist)
    with open(os.path.join(out_dir, f"r{rank}.txt"), "w") as f:
        f.write(f"{value!r} {t_max!r}\n")
    dist.barrier()
    dist.destroy_process_group()


def test_whole_job_rate_two_gloo_ranks(tmp_path):
    import torch.multiprocessing as mp
    units, seconds = [1.0e6, 3.0e6], [2.0, 5.0]
    port = 29500 + (os.getpid() % 2000)
    mp.start_processes(_rank_main, args=(2, port, units, seconds, str(tmp_path)), nprocs=2, join=True,
                       start_method="spawn")
    for r in range(2):
        value, t_max = map(float, open(tmp_path / f"r{r}.txt").read().split())
        assert t_max == 5.0
        assert value == pytest.approx(4.0e6 / 5.0, rel=1e-15)


def test_whole_job_rate_single_rank():
    sys.path.insert(0, ROOT)
    from paper_2208_04488_gb300.replicas import whole_job_rate
    assert whole_job_rate(6.0, 3.0) == (2.0, 3.0)


def test_reference_arm_other_ranks_exit_quietly():
    env = dict(os.environ, RANK="1", WORLD_SIZE="2", LOCAL_RANK="1", MASTER_ADDR="127.0.0.1")
    r = subprocess.run([sys.executable, os.path.join(ROOT, "bench.py"), "--impl", "reference", "--gpus", "2",
                        "--steps", "1", "--warmup", "0"], env=env, capture_output=True, text=True, timeout=120)
    assert r.returncode == 0
    assert r.stdout.strip() == ""
