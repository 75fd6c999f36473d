"""The multi-rank host logic of bench.py on CPU (gloo, world size 2): each rank searches its
own curves with no exchange on the data path; the job time is the slowest rank's, the value
counts every rank's curves, and a batch of curves splits into disjoint contiguous shares."""
import json
import os
import socket
import sys

import numpy as np
import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank_main(rank, world, port, out_dir):
    sys.path.insert(0, ROOT)
    import torch.distributed as dist
    import bench
    import synth
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank),
                      WORLD_SIZE=str(world), LOCAL_RANK=str(rank))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    r, w, local = bench.dist_env()
    local_time = 1.5 + rank  # rank 1 is the slow one
    t_max = bench.max_over_ranks(local_time, w)
    value = bench.job_value(10, w, t_max)
    curve = synth.make_workload("tess_2min_27d", seed=1 + r)  # the seed bench.py gives rank r
    share = bench.shard_range(1001, r, w)
    dist.barrier()
    dist.destroy_process_group()
    with open(os.path.join(out_dir, f"rank{rank}.json"), "w") as f:
        json.dump({"rank": r, "world": w, "local": local, "t_max": t_max, "value": value,
                   "flux_head": curve.flux[:8].tolist(), "share": share}, f)


def test_two_gloo_ranks(tmp_path):
    mp = pytest.importorskip("torch.multiprocessing")
    port = _free_port()
    mp.spawn(_rank_main, args=(2, port, str(tmp_path)), nprocs=2, join=True)
    res = [json.load(open(tmp_path / f"rank{r}.json")) for r in range(2)]
    assert [x["rank"] for x in res] == [0, 1] and all(x["world"] == 2 for x in res)
    assert all(x["t_max"] == 2.5 for x in res)          # the slowest rank's time on every rank
    assert all(x["value"] == pytest.approx(20 / 2.5) for x in res)  # both ranks' steps
    assert res[0]["flux_head"] != res[1]["flux_head"]   # each rank its own curve
    (a0, b0), (a1, b1) = res[0]["share"], res[1]["share"]
    assert a0 == 0 and b0 == a1 and b1 == 1001           # disjoint, contiguous, complete


@pytest.mark.parametrize("n,world", [(0, 3), (7, 3), (8192, 8), (5, 8)])
def test_shard_range_covers_every_curve_once(n, world):
    sys.path.insert(0, ROOT)
    import bench
    seen = np.zeros(n, int)
    sizes = []
    for r in range(world):
        a, b = bench.shard_range(n, r, world)
        seen[a:b] += 1
        sizes.append(b - a)
    assert np.all(seen == 1)
    assert max(sizes) - min(sizes) <= 1
    assert bench.max_over_ranks(3.25, 1) == 3.25
