"""The benchmark's multi-rank path on the host (replicas only: one tomography per rank, no data-path
collective): two gloo ranks agree on the max of their timed regions and on the whole-job rate, and
the barrier holds them together.  CPU only (torch.distributed over gloo, 127.0.0.1)."""
import os
import socket
import sys

import pytest

torch = pytest.importorskip("torch")
import torch.distributed as dist  # noqa: E402
import torch.multiprocessing as mp  # noqa: E402

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank(rank, ws, port, out):
    sys.path.insert(0, ROOT)
    import bench
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank), WORLD_SIZE=str(ws),
                      LOCAL_RANK=str(rank))
    dist.init_process_group("gloo", rank=rank, world_size=ws)
    try:
        assert bench.dist_env() == (ws, rank, rank)
        ms_local = [12.5, 20.0, 7.25, 16.0][rank]
        dist.barrier()
        ms_max = bench.max_over_ranks(dist, ws, ms_local)
        dist.barrier()
        out[rank] = (ms_max, bench.job_rate(ws, 20, ms_max))
    finally:
        dist.destroy_process_group()


@pytest.mark.parametrize("ws", [2, 4])
def test_ranks_agree_on_max_time_and_job_rate(ws):
    port = _free_port()
    with mp.Manager() as m:
        out = m.dict()
        mp.start_processes(_rank, args=(ws, port, out), nprocs=ws, start_method="spawn", join=True)
        res = dict(out)
    want = max([12.5, 20.0, 7.25, 16.0][:ws])
    assert sorted(res) == list(range(ws))
    for ms_max, rate in res.values():
        assert ms_max == want
        assert rate == ws * 20 / (want / 1e3)


def test_single_rank_needs_no_process_group():
    sys.path.insert(0, ROOT)
    import bench
    assert bench.max_over_ranks(None, 1, 3.5) == 3.5
    assert bench.job_rate(1, 10, 500.0) == 20.0


def test_reference_arm_other_ranks_exit_without_work():
    """Under torchrun only rank 0 runs the oracle arm; the others exit 0 and print nothing."""
    import subprocess
    env = dict(os.environ, RANK="1", WORLD_SIZE="2", LOCAL_RANK="1")
    r = subprocess.run([sys.executable, os.path.join(ROOT, "bench.py"), "--impl", "reference", "--gpus", "2",
                        "--steps", "1", "--warmup", "0"], env=env, capture_output=True, text=True, timeout=300)
    assert r.returncode == 0, r.stderr
    assert r.stdout.strip() == ""
