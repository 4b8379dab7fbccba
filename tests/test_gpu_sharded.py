"""The sliding-window solve sharded by frequency over two and three ranks (rls_window_solve_sharded),
run as processes on the one GPU that sum their images and ||q||^2 through gloo on host copies (the
kernels of the processes never wait on each other).  Each rank holds a contiguous block of the
frequencies (uneven blocks with three ranks); the ranks must keep identical images and statistics,
take the single-process solve's iteration counts and return its image and the FP64 oracle's.  The sharded solve adds the ranks' images and ||q||^2 in
another order than the single process does (rank sums, then the ranks), so its iterates differ in
the last bits; over these solves' 21-22 iterations that grows to at most a few 1e-6 (measured 4.3e-6
and 2.1e-6), below the float32 solve's distance from the oracle (up to 1.2e-5): both are bounded
here by 5e-5 and 1e-4."""

import json
import os
import socket

import numpy as np
import pytest

from oracle import lsm_oracle as O
from synth import random_case
from tests._helpers import device_survey, oracle_operator, rel_l2

pytestmark = pytest.mark.gpu

CASE = dict(nx=128, nz=24, ns=8, nw=12, seed=77)
# three ranks on 13 frequencies: shards of 5, 4 and 4
CASE3 = dict(nx=128, nz=24, ns=8, nw=13, seed=78)
K, SLIDE, TOL, ITERS = 4, 2, 1e-2, 40


def _problem(case=CASE):
    sv = random_case(case["nx"], case["nz"], case["ns"], case["nw"], seed=case["seed"])
    op = oracle_operator(sv)
    clean = op.forward(np.asarray(sv.reflectivity, dtype=np.float32).astype(np.float64))
    d = (clean + sv.noise_pct * np.sqrt(np.mean(np.abs(clean) ** 2)) * sv.noise()).astype(np.complex64)
    lam = float(np.float32(O.regularisation_from_adjoint(op, d.astype(np.complex128))))
    return sv, op, d, lam


def _rank_main(rank, world, port, out_dir, d_path, lam, case=CASE):
    import torch
    import torch.distributed as dist

    import paper_1801_00819_gb300 as L
    from paper_1801_00819_gb300 import lsm
    from paper_1801_00819_gb300.device import to_device
    from paper_1801_00819_gb300.sharded import frequency_shard, torch_allreduce

    torch.cuda.set_device(0)
    dist.init_process_group("gloo", init_method=f"tcp://127.0.0.1:{port}", rank=rank, world_size=world)
    try:
        sv = random_case(case["nx"], case["nz"], case["ns"], case["nw"], seed=case["seed"])
        f0, f1 = frequency_shard(sv.nw, rank, world)
        ds = to_device(sv.nx, sv.nz, sv.dx, sv.dz, sv.slowness, sv.src_ix, sv.rec_ix, sv.freqs[f0:f1],
                       sv.wavelet[f0:f1])
        d = torch.as_tensor(np.ascontiguousarray(np.load(d_path)[:, f0:f1, :]), device="cuda")
        ws = torch.empty(L.lsm_workspace_bytes(ds.grid, ds.geom, ds.freqs, K, L.LSM_OP_SOLVE), dtype=torch.uint8,
                         device="cuda")
        m = torch.zeros((sv.nz, sv.nx), dtype=torch.float32, device="cuda")
        _, stats = lsm.rls_window_solve_sharded(ds.grid, ds.slowness, ds.freqs, ds.geom, d, lam, K, SLIDE, TOL, ITERS,
                                                m, ws, torch_allreduce())
        torch.cuda.synchronize()
        np.save(os.path.join(out_dir, f"m{rank}.npy"), m.cpu().numpy())
        with open(os.path.join(out_dir, f"stats{rank}.json"), "w") as fh:
            json.dump(stats, fh)
    finally:
        dist.destroy_process_group()


@pytest.mark.parametrize("world", [2, 3])
def test_frequency_sharded_solve(tmp_path, world):
    """world = 2: 12 frequencies in two shards of 6; world = 3: 13 frequencies in shards of 5, 4, 4."""
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import torch.multiprocessing as mp

    import paper_1801_00819_gb300 as L
    case = CASE if world == 2 else CASE3
    sv, op, d, lam = _problem(case)
    d_path = str(tmp_path / "d.npy")
    np.save(d_path, d)
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        port = s.getsockname()[1]
    mp.spawn(_rank_main, args=(world, port, str(tmp_path), d_path, lam, case), nprocs=world, join=True)

    # the same solve in one process
    ds = device_survey(sv)
    ws = torch.empty(L.lsm_workspace_bytes(ds.grid, ds.geom, ds.freqs, K, L.LSM_OP_SOLVE), dtype=torch.uint8,
                     device="cuda")
    m1 = torch.zeros((sv.nz, sv.nx), dtype=torch.float32, device="cuda")
    _, st1 = L.rls_window_solve(ds.grid, ds.slowness, ds.freqs, ds.geom, torch.as_tensor(d, device="cuda"), lam, K,
                                SLIDE, TOL, ITERS, m1, ws, cuda_graph=False)
    torch.cuda.synchronize()
    single = m1.cpu().numpy().astype(np.float64)
    m_ref, st_ref = O.rls_solve(op, d.astype(np.complex128), lam, K, SLIDE, ITERS, tol=TOL)
    ranks = [np.load(tmp_path / f"m{r}.npy").astype(np.float64) for r in range(world)]
    stats = [json.load(open(tmp_path / f"stats{r}.json")) for r in range(world)]
    print(json.dumps({"iters": [[w["iters"] for w in st] for st in stats], "single": [w["iters"] for w in st1],
                      "oracle": [w.iters for w in st_ref], "vs_single": rel_l2(ranks[0], single),
                      "vs_oracle": rel_l2(ranks[0], m_ref)}))
    for r in range(1, world):
        np.testing.assert_array_equal(ranks[0], ranks[r])  # the ranks keep identical model-space vectors
        assert [{k: v for k, v in w.items() if k != "ms"} for w in stats[r]] == \
            [{k: v for k, v in w.items() if k != "ms"} for w in stats[0]]
    assert [w["iters"] for w in stats[0]] == [w["iters"] for w in st1] == [w.iters for w in st_ref]
    assert rel_l2(ranks[0], single) <= 5e-5
    assert rel_l2(ranks[0], m_ref) <= 1e-4
