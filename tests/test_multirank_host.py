"""The N > 1 host path of bench.py on two CPU ranks (gloo, 127.0.0.1): each rank solves its own
survey line (independent noise), and the whole-job figures are the units all ranks processed over
the slowest rank's time.  No GPU, no data-path collective: only the two timing reductions."""

import os
import socket

import pytest


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank_main(rank, world, port, out_dir):
    import json

    import torch.distributed as dist

    import bench

    os.environ.update({"RANK": str(rank), "WORLD_SIZE": str(world), "LOCAL_RANK": str(rank),
                       "MASTER_ADDR": "127.0.0.1", "MASTER_PORT": str(port)})
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        r, w, _ = bench.dist_info()
        units = 1000.0 * (rank + 1)  # ranks finish different numbers of CG iterations
        t_ms = 10.0 + 5.0 * rank
        total, t_max = bench.reduce_over_ranks(units, t_ms, w, "cpu")
        seed = bench.workload("tiny", r).noise_seed
        with open(os.path.join(out_dir, f"rank{rank}.json"), "w") as fh:
            json.dump({"rank": r, "world": w, "total": total, "t_max": t_max, "noise_seed": seed}, fh)
    finally:
        dist.destroy_process_group()


def test_two_rank_totals_and_independent_lines(tmp_path):
    torch = pytest.importorskip("torch")
    import torch.multiprocessing as mp
    if not torch.distributed.is_available() or not torch.distributed.is_gloo_available():
        pytest.skip("gloo backend not available")
    import json
    world, port = 2, _free_port()
    mp.start_processes(_rank_main, args=(world, port, str(tmp_path)), nprocs=world, join=True, start_method="spawn")
    res = [json.load(open(tmp_path / f"rank{r}.json")) for r in range(world)]
    for r, x in enumerate(res):
        assert x["rank"] == r and x["world"] == world
        assert x["total"] == 3000.0  # 1000 + 2000: each rank's own units, not rank 0's times N
        assert x["t_max"] == 15.0    # the slowest rank
    assert res[0]["noise_seed"] != res[1]["noise_seed"]  # independent lines


def test_single_rank_reduction_is_identity():
    import bench
    assert bench.reduce_over_ranks(123.0, 4.5, 1, "cpu") == (123.0, 4.5)
