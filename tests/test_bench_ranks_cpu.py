"""Host logic of the benchmark's N > 1 path, on CPU with two gloo ranks (127.0.0.1): the
ranks meet at the barriers around the timed region, the reported time is the slowest
rank's, the value aggregates the units of every rank (independent replicas, weak
scaling), and the reference arm runs on rank 0 only (the other ranks return at once)."""
import json
import os
import socket
import types

import pytest

torch = pytest.importorskip("torch")
import torch.multiprocessing as mp

import bench


def free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def rank_main(rank, world, port, out_dir):
    import torch.distributed as dist

    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank), WORLD_SIZE=str(world),
                      LOCAL_RANK=str(rank))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    r, w, local = bench.dist_env()
    bench.rank_barrier(w)
    ms = 10.0 * (rank + 1)  # rank 1 is the slow one
    ms_max = bench.max_over_ranks(ms, w, "cpu")
    value = bench.whole_job_rate(128 * 5, w, ms_max)
    ref = bench.run_reference(types.SimpleNamespace(steps=1, warmup=0), r, w) if r != 0 else "rank 0 not run"
    bench.rank_barrier(w)
    with open(os.path.join(out_dir, f"rank{rank}.json"), "w") as f:
        json.dump({"env": [r, w, local], "ms_max": ms_max, "value": value, "ref_none": ref is None}, f)
    dist.destroy_process_group()


def test_two_gloo_ranks_take_the_slowest_time(tmp_path):
    mp.spawn(rank_main, args=(2, free_port(), str(tmp_path)), nprocs=2, join=True)
    out = [json.load(open(tmp_path / f"rank{r}.json")) for r in range(2)]
    for r, d in enumerate(out):
        assert d["env"] == [r, 2, r]
        assert d["ms_max"] == 20.0
        # 2 ranks x 640 units in 20 ms
        assert d["value"] == pytest.approx(2 * 640 / 0.020)
    assert out[1]["ref_none"]


def test_single_rank_needs_no_process_group():
    assert bench.max_over_ranks(12.5, 1) == 12.5
    bench.rank_barrier(1)
    assert bench.whole_job_rate(100, 1, 50.0) == pytest.approx(2000.0)
