"""Host side of the frequency-sharded window solve (no GPU): the frequency partition, the
all-reduce callback built on torch.distributed (two gloo ranks on the CPU, host buffers), and the
entry point's argument check."""

import ctypes
import os
import shutil
import socket

import numpy as np
import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def test_frequency_shards_cover_the_axis_once():
    from paper_1801_00819_gb300.sharded import frequency_shard
    for nw in (1, 2, 5, 16, 31, 128):
        for world in range(1, min(nw, 9) + 1):
            parts = [frequency_shard(nw, r, world) for r in range(world)]
            assert parts[0][0] == 0 and parts[-1][1] == nw
            assert all(a[1] == b[0] for a, b in zip(parts, parts[1:]))
            sizes = [b - a for a, b in parts]
            assert max(sizes) - min(sizes) <= 1 and min(sizes) >= 1
    with pytest.raises(ValueError):
        frequency_shard(3, 0, 4)


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank_main(rank, world, port, out_dir):
    import torch.distributed as dist

    from paper_1801_00819_gb300.sharded import torch_allreduce
    dist.init_process_group("gloo", init_method=f"tcp://127.0.0.1:{port}", rank=rank, world_size=world)
    try:
        hook = torch_allreduce(device="cpu")
        img = np.arange(6, dtype=np.float32) * (rank + 1)      # an "image" of float32 values
        qq = np.array([0.5 + rank], dtype=np.float64)          # a float64 scalar
        hook(img.ctypes.data, img.size, 0, 0)
        hook(qq.ctypes.data, 1, 1, 0)
        np.save(os.path.join(out_dir, f"img{rank}.npy"), img)
        np.save(os.path.join(out_dir, f"qq{rank}.npy"), qq)
    finally:
        dist.destroy_process_group()


def test_allreduce_callback_sums_over_two_gloo_ranks(tmp_path):
    import torch.multiprocessing as mp
    mp.spawn(_rank_main, args=(2, _free_port(), str(tmp_path)), nprocs=2, join=True)
    for r in range(2):
        np.testing.assert_array_equal(np.load(tmp_path / f"img{r}.npy"), np.arange(6, dtype=np.float32) * 3)
        assert np.load(tmp_path / f"qq{r}.npy")[0] == 2.0


def test_sharded_entry_point_needs_a_callback():
    if shutil.which("nvcc") is None and not os.path.exists("/usr/local/cuda/bin/nvcc"):
        pytest.skip("nvcc not available")
    from paper_1801_00819_gb300 import build as B
    B.build()
    from paper_1801_00819_gb300 import lsm
    lib = lsm.load_library()
    g = lsm.Grid(64, 8, 10.0, 10.0)
    geo = lsm.Geometry(np.arange(3), None, nx=64)
    f = lsm.Frequencies(np.linspace(5, 30, 4), np.ones(4))
    stats = (lsm.lsm_window_stats * 2)()
    fake = 1 << 20
    before = lsm.lsm_kernel_launches()
    st = lib.rls_window_solve_sharded(ctypes.byref(g.c), fake, ctypes.byref(f.c), ctypes.byref(geo.c), fake, 1.0, 2,
                                      1, 0.0, 3, 0, 0, fake, stats, 2, fake, 1 << 30, 0,
                                      ctypes.cast(None, lsm.ALLREDUCE_FN), None)
    assert st == lsm.LSM_ERR_ARG
    assert lsm.lsm_kernel_launches() == before
