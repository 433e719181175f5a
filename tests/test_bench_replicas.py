"""The N > 1 bench path on CPU: two gloo ranks run the replica aggregation
bench.py uses (slowest rank's time by all-reduce MAX, whole-job throughput =
all ranks' units over that time), and the reference arm prints from rank 0
only."""
import importlib.util
import json
import os
import socket
import subprocess
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _bench():
    spec = importlib.util.spec_from_file_location("bench_mod", os.path.join(ROOT, "bench.py"))
    mod = importlib.util.module_from_spec(spec)
    spec.loader.exec_module(mod)
    return mod


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _worker(rank, world, port, seconds, q):
    import torch
    import torch.distributed as dist
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    b = _bench()
    t = b.max_over_ranks(seconds[rank], dist, torch.device("cpu"))
    q.put((rank, t, b.replica_throughput(1000, t, world)))
    dist.barrier()
    dist.destroy_process_group()


def test_two_gloo_ranks_take_the_slowest_time():
    import torch.multiprocessing as mp
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    seconds = [0.25, 0.75]
    procs = [ctx.Process(target=_worker, args=(r, 2, port, seconds, q)) for r in range(2)]
    for p in procs:
        p.start()
    for p in procs:
        p.join(timeout=120)
        assert p.exitcode == 0
    res = sorted(q.get(timeout=10) for _ in range(2))
    for rank, t, thr in res:
        assert t == 0.75
        assert thr == pytest.approx(2 * 1000 / 0.75)


def test_single_process_aggregation_is_identity():
    b = _bench()
    assert b.max_over_ranks(0.5, None, None) == 0.5
    assert b.replica_throughput(10, 0.5, 1) == 20


def test_reference_arm_prints_on_rank_zero_only():
    """bench.py --impl reference under WORLD_SIZE=2: rank 1 exits 0 silently,
    rank 0 prints one JSON line (a tiny run of the oracle)."""
    env = dict(os.environ, WORLD_SIZE="2", RANK="1", LOCAL_RANK="1")
    out = subprocess.run([sys.executable, os.path.join(ROOT, "bench.py"), "--impl", "reference", "--steps", "1",
                          "--warmup", "3"], env=env, capture_output=True, text=True, timeout=300)
    assert out.returncode == 0 and out.stdout.strip() == ""


def test_reference_arm_line_on_a_small_headline_mesh():
    """Rank 0 of the reference arm prints the contract's line: the oracle's
    tets/s on the headline workload's recipe (here a 16^3 mesh), with
    cpu_baseline and e2e describing the same run."""
    env = dict(os.environ, WORLD_SIZE="1", RANK="0", LOCAL_RANK="0")
    out = subprocess.run([sys.executable, os.path.join(ROOT, "bench.py"), "--impl", "reference", "--steps", "1",
                          "--warmup", "3", "--n", "16"], env=env, capture_output=True, text=True, timeout=300)
    assert out.returncode == 0, out.stderr
    line = json.loads(out.stdout.strip().splitlines()[-1])
    assert line["impl"] == "reference" and line["unit"] == "tets/s" and line["value"] > 0
    assert line["config"]["n_tets"] == 5 * 16 ** 3
    assert line["cpu_baseline"]["value"] == line["value"] and line["cpu_baseline"]["cores"] == 1
    assert line["e2e"]["h2d_bytes_per_step"] == 0
