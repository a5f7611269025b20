"""The N > 1 host path of bench.py on CPU: two gloo ranks (127.0.0.1) through
the same rank setup, barrier and max-over-ranks timing reduction that the
launcher's torchrun ranks use, and the reference arm's rule that ranks other
than 0 exit without work.  No GPU and no data-path collective: the benchmark
runs independent replicas (weak scaling)."""
import json
import os
import socket
import subprocess
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank_main(rank, world, port, out_dir):
    os.environ.update({"RANK": str(rank), "LOCAL_RANK": str(rank), "WORLD_SIZE": str(world),
                       "MASTER_ADDR": "127.0.0.1", "MASTER_PORT": str(port)})
    sys.path.insert(0, ROOT)
    import bench
    w, r, local, pg = bench.dist_setup(None)
    # each rank "times" a different duration; every rank must see the maximum
    t = bench.max_over_ranks(pg, 10.0 + 5.0 * r)
    bench.barrier(pg)
    with open(os.path.join(out_dir, "rank%d.json" % r), "w") as f:
        json.dump({"world": w, "rank": r, "local": local, "max": t}, f)
    bench.barrier(pg)
    pg.destroy_process_group()


def test_bench_ranks_gloo(tmp_path):
    import torch.multiprocessing as mp
    world = 2
    port = _free_port()
    ctx = mp.get_context("spawn")
    procs = [ctx.Process(target=_rank_main, args=(r, world, port, str(tmp_path))) for r in range(world)]
    for p in procs:
        p.start()
    for p in procs:
        p.join(timeout=120)
    for p in procs:
        if p.is_alive():
            p.kill()
        assert p.exitcode == 0
    for r in range(world):
        d = json.load(open(tmp_path / ("rank%d.json" % r)))
        assert d == {"world": world, "rank": r, "local": r, "max": 15.0}


def test_bench_single_process_needs_no_group():
    sys.path.insert(0, ROOT)
    import bench
    env = {k: os.environ.pop(k) for k in ("WORLD_SIZE", "RANK", "LOCAL_RANK") if k in os.environ}
    try:
        w, r, local, pg = bench.dist_setup(None)
        assert (w, r, local, pg) == (1, 0, 0, None)
        assert bench.max_over_ranks(pg, 3.25) == 3.25
        bench.barrier(pg)
    finally:
        os.environ.update(env)


def test_reference_arm_other_ranks_exit_quietly():
    env = dict(os.environ, RANK="1", LOCAL_RANK="1", WORLD_SIZE="2")
    res = subprocess.run([sys.executable, os.path.join(ROOT, "bench.py"), "--impl", "reference",
                          "--gpus", "2", "--steps", "1", "--warmup", "3"],
                         cwd=ROOT, env=env, capture_output=True, text=True, timeout=120)
    assert res.returncode == 0
    assert res.stdout.strip() == ""
