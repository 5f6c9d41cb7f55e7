"""The N > 1 host logic of the benchmark on CPU with two gloo ranks: every rank optimises its own
replica (own Philox key, no collective on the data path), the timed duration is the slowest
rank's (all-reduce MAX) and the value is the whole job's units over that time; the reference arm
runs on rank 0 only. The oracle shows that the replicas' random streams are independent."""
import json
import os
import socket
import sys

import numpy as np
import pytest
import torch.multiprocessing as mp

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _worker(rank, world, port, out_dir):
    sys.path.insert(0, ROOT)
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank), WORLD_SIZE=str(world))
    import torch.distributed as dist
    import bench
    dist.init_process_group("gloo", rank=rank, world_size=world)
    ms = 10.0 + 5.0 * rank
    ms_max = bench.slowest_rank_ms(ms, dist, "cpu")
    key = bench.replica_scene({"key_id": 77, "width": 4}, rank)["key_id"]
    keys = [None] * world
    dist.all_gather_object(keys, key)
    dist.barrier()
    with open(os.path.join(out_dir, f"rank{rank}.json"), "w") as f:
        json.dump({"ms_max": ms_max, "keys": keys}, f)
    dist.destroy_process_group()


def test_two_gloo_ranks(tmp_path):
    world = 2
    mp.spawn(_worker, args=(world, _free_port(), str(tmp_path)), nprocs=world, join=True)
    res = [json.load(open(tmp_path / f"rank{r}.json")) for r in range(world)]
    for r in res:
        assert r["ms_max"] == 15.0            # the slowest rank's time on every rank
        assert r["keys"] == [0, 1]            # one Philox key per replica
    sys.path.insert(0, ROOT)
    import bench
    assert bench.whole_job_rate(world, 1000, 10, 15.0) == pytest.approx(2 * 1000 * 10 / 0.015)


def test_reference_arm_runs_on_rank_zero_only(monkeypatch):
    sys.path.insert(0, ROOT)
    import bench
    monkeypatch.setenv("RANK", "1")
    monkeypatch.setenv("WORLD_SIZE", "2")
    assert bench.run_reference(bench.parse(["--impl", "reference"])) == 0


def test_replica_streams_independent(oracle_lib):
    """Two ranks' replicas draw different random numbers: same scene, keys 0 and 1."""
    from oracle import orc
    from paper_2309_15676_gb300 import synth
    w = synth.workload_box(8, 8, 8, max_depth=3)
    sys.path.insert(0, ROOT)
    import bench
    a = orc.render_image(orc.Scene(bench.replica_scene(w.scene, 0)), w.init_tex, 1, 0, orc.ST_EVAL)
    b = orc.render_image(orc.Scene(bench.replica_scene(w.scene, 1)), w.init_tex, 1, 0, orc.ST_EVAL)
    assert not np.array_equal(a, b)
