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


def _split_rank_main(rank, world, port, q):
    """One rank of a swarm split over gloo: its slice of a C1 swarm, misfits
    from the oracle (rounded to FP32 nm^2, the library's key precision),
    personal bests, the exchange of split.exchange_dist, the Eq. 8 move of
    its slice by the oracle; plus its share of a sharded image."""
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank),
                      WORLD_SIZE=str(world), LOCAL_RANK=str(rank))
    sys.path.insert(0, ROOT)
    sys.path.insert(0, os.path.join(ROOT, "tests"))
    import bench
    import torch.distributed as dist
    from paper_1109_0334_gb300 import split
    r, w, _ = bench.dist_setup(backend="gloo")
    keys, x_fin = _swarm_run(split, r, w, exchange=True)
    lo, hi = bench.rank_slice(4096 * w, r, w)
    spans = [None] * w
    dist.all_gather_object(spans, (lo, hi))
    dist.destroy_process_group()
    q.put((r, keys, x_fin.tolist(), spans))


def _swarm_run(split, rank, world, exchange):
    """Keys after each generation and the final global-best position."""
    import numpy as np
    import torch
    from oracle import oracle as O
    from paper_1109_0334_gb300 import workloads as W
    from common import oracle_record
    O.build()
    O.set_threads(1)
    spec = W.get("c1", P=64, iters=8)
    c, pm = O.make_case(spec), O.make_pmap(spec)
    _, U_m, _ = oracle_record(O, spec)
    P, D = spec["P"], pm.D
    lo, hi = split.slice_of(P, rank, world) if exchange else (0, P)
    x, v = O.pso_init(hi - lo, D, spec["seed"], 0, p0=lo)
    pb, pbS = x.copy(), np.full(hi - lo, np.inf, dtype=np.float32)
    keys = []
    for it in range(spec["iters"] + 1):
        S32 = (O.misfit_batch(c, pm, x, U_m) / 1e-18).astype(np.float32)
        better = (S32 < pbS) | (it == 0)
        pbS = np.where(better, np.minimum(S32, pbS), pbS).astype(np.float32)
        pb[:, better] = x[:, better]
        loc = [(int(np.float32(s).view(np.uint32)) << 32) | (lo + p) for p, s in enumerate(pbS)]
        key = min(loc)
        if exchange:
            def owner(kmin):
                g = split.key_index(kmin)
                if lo <= g < hi:
                    return True, torch.from_numpy(pb[:, g - lo].astype(np.float32))
                return False, None
            kmin, pos = split.exchange_dist(key, owner, D, torch.device("cpu"))
            gb = pos.numpy().astype(np.float64)
        else:
            kmin = key
            gb = pb[:, split.key_index(kmin)].astype(np.float32).astype(np.float64)
        keys.append(kmin)
        if it < spec["iters"]:
            x, v = O.pso_update(it + 1, spec["seed"], 0, spec["w"], spec["c1"], spec["c2"], x, v,
                                pb, gb, p0=lo)
    return keys, gb


def test_split_swarm_exchange_reproduces_one_rank():
    """Two gloo ranks, each with half of the swarm, reproduce the one-rank
    sequence of global-best keys bit for bit and end on the same position;
    the image shards of the benchmark cover every pixel exactly once."""
    import torch.multiprocessing as mp
    sys.path.insert(0, ROOT)
    sys.path.insert(0, os.path.join(ROOT, "tests"))
    from paper_1109_0334_gb300 import split
    ref_keys, ref_x = _swarm_run(split, 0, 1, exchange=False)
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_split_rank_main, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    out = sorted([q.get(timeout=300) for _ in procs])
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    for r, keys, x_fin, spans in out:
        assert keys == ref_keys
        assert x_fin == ref_x.tolist()
        covered = sorted(i for lo, hi in spans for i in range(lo, hi))
        assert covered == list(range(2 * 4096))
    # the winner moved between the slices at least once (the exchange matters)
    owners = {split.key_index(k) >= 32 for k in ref_keys}
    assert owners == {True, False}
