"""The benchmark's N > 1 path without GPUs: two ranks over gloo on 127.0.0.1
join the process group, synchronise, take the maximum of their step times
and partition independent units; the reference arm's non-zero ranks exit
without work.  Each rank is a spawned process (no GPU, no fork after CUDA)."""
import os
import socket
import subprocess
import sys

import pytest

torch = pytest.importorskip("torch")

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    port = s.getsockname()[1]
    s.close()
    return port


def _rank_main(rank, world, port, q):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank),
                      WORLD_SIZE=str(world), LOCAL_RANK=str(rank))
    sys.path.insert(0, ROOT)
    import bench
    import torch.distributed as dist
    r, w, _ = bench.dist_setup(backend="gloo")
    bench.barrier(w)
    step_ms = 10.0 + 5.0 * r                     # rank 1 is the slow one
    t_max = bench.all_max(step_ms, w)
    lo, hi = bench.rank_slice(4096, r, w)
    rate = bench.job_rate(1000.0, 3, t_max, w)
    dist.destroy_process_group()
    q.put((r, w, t_max, lo, hi, rate))


def test_two_gloo_ranks_time_and_partition():
    import torch.multiprocessing as mp
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_rank_main, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    out = [q.get(timeout=120) for _ in procs]
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    out.sort()
    assert [o[0] for o in out] == [0, 1] and all(o[1] == 2 for o in out)
    assert all(o[2] == 15.0 for o in out)                 # max over ranks
    assert out[0][3:5] == (0, 2048) and out[1][3:5] == (2048, 4096)
    assert all(o[5] == pytest.approx(2 * 1000.0 * 3 / 15e-3) for o in out)


def test_rank_slice_partitions():
    sys.path.insert(0, ROOT)
    import bench
    for n in (0, 1, 7, 4096, 4099):
        for world in (1, 2, 3, 8):
            parts = [bench.rank_slice(n, r, world) for r in range(world)]
            assert parts[0][0] == 0 and parts[-1][1] == n
            assert all(a[1] == b[0] for a, b in zip(parts, parts[1:]))
            sizes = [h - l for l, h in parts]
            assert max(sizes) - min(sizes) <= 1


def test_reference_arm_other_ranks_exit_without_work():
    env = dict(os.environ, RANK="1", WORLD_SIZE="2", LOCAL_RANK="1", MASTER_ADDR="127.0.0.1",
               MASTER_PORT=str(_free_port()))
    r = subprocess.run([sys.executable, os.path.join(ROOT, "bench.py"), "--impl", "reference",
                        "--gpus", "2", "--steps", "1", "--warmup", "3"],
                       env=env, capture_output=True, text=True, timeout=300)
    assert r.returncode == 0
    assert r.stdout.strip() == ""
