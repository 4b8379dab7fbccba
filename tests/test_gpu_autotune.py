"""Launch-shape autotuning (lsm_autotune): the recorded shapes are admissible, launches that use
them still match the FP64 oracle, and A^T stays deterministic under a recorded shape."""

import numpy as np
import pytest

from oracle import lsm_oracle as O
from synth import random_case, config_precision_subsample
from tests._helpers import oracle_operator, rel_l2, device_survey

pytestmark = pytest.mark.gpu


@pytest.fixture()
def torch_cuda():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_1801_00819_gb300 as L
    L.lsm_autotune_reset()
    yield torch
    L.lsm_autotune_reset()  # later tests run the default shapes


def _tune(torch, ds, K, transform="fft"):
    import paper_1801_00819_gb300 as L
    ws = torch.empty(L.lsm_workspace_bytes(ds.grid, ds.geom, ds.freqs, K, L.LSM_OP_SOLVE), dtype=torch.uint8,
                     device="cuda")
    rep = L.lsm_autotune(ds.grid, ds.slowness, ds.freqs, ds.geom, K, ws, transform=transform)
    for sweep in ("source", "adjoint", "forward"):
        e = rep[sweep]
        assert e["candidates"] >= 1 and 1 <= e["warps"] and e["ms"] > 0.0, (sweep, e)
        assert e["ms"] <= e["heuristic_ms"] * 1.0000001 or e["heuristic_ms"] == 0.0, (sweep, e)
    assert rep["adjoint"]["warps"] >= rep["adjoint"]["heuristic_warps"]  # no more partial images
    return rep


def test_tuned_shapes_keep_operator_and_solve_parity(torch_cuda):
    import paper_1801_00819_gb300 as L
    torch = torch_cuda
    sv = random_case(128, 24, 6, 10, seed=7)
    op = oracle_operator(sv)
    ds = device_survey(sv)
    K = 3
    rep = _tune(torch, ds, K)
    print(rep)
    ws = torch.empty(L.lsm_workspace_bytes(ds.grid, ds.geom, ds.freqs, K, L.LSM_OP_ADJOINT), dtype=torch.uint8,
                     device="cuda")
    m = np.asarray(sv.reflectivity, dtype=np.float32)
    rng = np.random.default_rng(3)
    d = (rng.normal(size=(K, sv.nw, sv.nx)) + 1j * rng.normal(size=(K, sv.nw, sv.nx))).astype(np.complex64)
    for shot0 in (0, 2):
        out = torch.empty((K, sv.nw, sv.nx), dtype=torch.complex64, device="cuda")
        L.lsm_forward(ds.grid, ds.slowness, ds.freqs, ds.geom, torch.as_tensor(m, device="cuda"), out, shot0, K, ws)
        imgs = []
        for _ in range(2):
            img = torch.empty((sv.nz, sv.nx), dtype=torch.float32, device="cuda")
            L.lsm_adjoint(ds.grid, ds.slowness, ds.freqs, ds.geom, torch.as_tensor(d, device="cuda"), img, shot0, K,
                          ws)
            imgs.append(img.cpu().numpy())
        torch.cuda.synchronize()
        shots = np.arange(shot0, shot0 + K)
        assert rel_l2(out.cpu().numpy(), op.forward(m.astype(np.float64), shots=shots)) <= 1e-4
        assert rel_l2(imgs[0], op.adjoint(d.astype(np.complex128), shots=shots)) <= 1e-4
        np.testing.assert_array_equal(imgs[0], imgs[1])


def test_tuned_shapes_keep_sliding_solve_parity(torch_cuda):
    """The tiny workload's sliding solve (window 4, slide 2, 10 iterations), whose A and A^T sweeps run
    over K = 4 shots, once on the default and once on the tuned shapes: both match the oracle."""
    import paper_1801_00819_gb300 as L
    from synth import config_tiny
    torch = torch_cuda
    sv = config_tiny()
    op = oracle_operator(sv)
    ds = device_survey(sv)
    m = np.asarray(sv.reflectivity, dtype=np.float32).astype(np.float64)
    clean = op.forward(m)
    dd = (clean + sv.noise_pct * np.sqrt(np.mean(np.abs(clean) ** 2)) * sv.noise()).astype(np.complex64)
    lam = float(np.float32(O.regularisation_from_adjoint(op, dd.astype(np.complex128))))
    m_ref, _ = O.rls_solve(op, dd.astype(np.complex128), lam, sv.window, sv.slide, sv.cg_iters)
    wss = torch.empty(L.lsm_workspace_bytes(ds.grid, ds.geom, ds.freqs, sv.window, L.LSM_OP_SOLVE),
                      dtype=torch.uint8, device="cuda")

    def solve():
        mm = torch.zeros((sv.nz, sv.nx), dtype=torch.float32, device="cuda")
        L.rls_window_solve(ds.grid, ds.slowness, ds.freqs, ds.geom, torch.as_tensor(dd, device="cuda"), lam,
                           sv.window, sv.slide, 0.0, sv.cg_iters, mm, wss)
        torch.cuda.synchronize()
        return mm.cpu().numpy().astype(np.float64)

    m_default = solve()
    _tune(torch, ds, sv.window)
    m_tuned = solve()
    assert rel_l2(m_default, m_ref) <= 1e-4
    assert rel_l2(m_tuned, m_ref) <= 1e-4


def test_tuned_tensor_core_shapes_keep_parity(torch_cuda):
    import paper_1801_00819_gb300 as L
    torch = torch_cuda
    sv = config_precision_subsample(128)
    op = oracle_operator(sv)
    ds = device_survey(sv)
    K = 3
    _tune(torch, ds, K, transform="dft_fp16x3")
    ws = torch.empty(L.lsm_workspace_bytes(ds.grid, ds.geom, ds.freqs, K, L.LSM_OP_ADJOINT), dtype=torch.uint8,
                     device="cuda")
    m = np.asarray(sv.reflectivity, dtype=np.float32)
    out = torch.empty((K, sv.nw, sv.nx), dtype=torch.complex64, device="cuda")
    L.lsm_forward(ds.grid, ds.slowness, ds.freqs, ds.geom, torch.as_tensor(m, device="cuda"), out, 0, K, ws,
                  transform="dft_fp16x3")
    torch.cuda.synchronize()
    assert rel_l2(out.cpu().numpy(), op.forward(m.astype(np.float64), shots=np.arange(K))) <= 1e-4


@pytest.mark.parametrize("shape", [(64, 40, 3, 5), (128, 20, 2, 4)], ids=lambda s: "x".join(map(str, s)))
def test_gradient_stride_tuning_keeps_gradients_bitwise(torch_cuda, shape):
    """lsm_autotune_gradient records one of the candidate (checkpoint stride, warps per block) pairs.
    The modelled data computed afterwards is bitwise the default's, and so are the gradients when the
    warps per block are unchanged (the segments replay the same steps from their checkpoints; another
    block partition changes the last bits of the image sums); all match the FP64 oracle."""
    import paper_1801_00819_gb300 as L
    torch = torch_cuda
    nx, nz, ns, nw = shape
    sv = random_case(nx, nz, ns, nw, seed=nx + 3)
    ds = device_survey(sv)
    op = oracle_operator(sv)
    m = np.asarray(sv.reflectivity, dtype=np.float32)
    rng = np.random.default_rng(nx)
    dobs = (rng.normal(size=(ns, nw, op.nrec)) + 1j * rng.normal(size=(ns, nw, op.nrec))) * 0.05
    g = (op.forward(m.astype(np.float64)) - dobs) * 2.0
    sref = torch.as_tensor(op.sref, device="cuda")
    ws = torch.empty(L.lsm_workspace_bytes(ds.grid, ds.geom, ds.freqs, ns, L.LSM_OP_GRADIENT), dtype=torch.uint8,
                     device="cuda")
    mt = torch.as_tensor(m, device="cuda")
    gt = torch.as_tensor(g.astype(np.complex64), device="cuda")

    def run():
        gm, gs = torch.empty_like(mt), torch.empty_like(mt)
        d = torch.empty((ns, nw, op.nrec), dtype=torch.complex64, device="cuda")
        L.lsm_born_gradient(ds.grid, ds.slowness, sref, ds.freqs, ds.geom, mt, gt, d, gm, gs, 0, ns, ws)
        torch.cuda.synchronize()
        return gm.cpu().numpy(), gs.cpu().numpy(), d.cpu().numpy()

    gm0, gs0, d0 = run()
    rep = L.lsm_autotune_gradient(ds.grid, ds.slowness, ds.freqs, ds.geom, ns, ws)
    print(rep)
    assert rep["default_stride"] == min(L.lsm.LSM_CHECKPOINT_EVERY, nz)
    assert rep["stride"] in {min(c, nz) for c in (8, 16, 32)}
    nstrides = len({min(c, nz) for c in (8, 16, 32, L.lsm.LSM_CHECKPOINT_EVERY)})
    nwarps = rep["default_warps"] - max(1, rep["default_warps"] - 2) + 1
    assert max(1, rep["default_warps"] - 2) <= rep["warps"] <= rep["default_warps"]
    assert rep["candidates"] == nstrides * nwarps
    assert 0.0 < rep["ms"] <= rep["default_ms"]
    gm1, gs1, d1 = run()
    np.testing.assert_array_equal(d1, d0)
    if rep["warps"] == rep["default_warps"]:
        np.testing.assert_array_equal(gm1, gm0)
        np.testing.assert_array_equal(gs1, gs0)
    else:
        assert rel_l2(gm1, gm0) <= 1e-6 and rel_l2(gs1, gs0) <= 1e-6
    gm_ref, gs_ref = O.born_gradients(op, m.astype(np.float64), g)
    assert rel_l2(gm1, gm_ref) <= 1e-4
    assert rel_l2(gs1, gs_ref) <= 1e-4


ALT_TILE_CASES = [(16, 8, 3, 5), (64, 12, 3, 6), (128, 10, 2, 7), (256, 9, 2, 4), (512, 8, 2, 3), (48, 8, 2, 3),
                  (384, 6, 2, 3), (640, 6, 1, 3), (112, 7, 3, 3), (320, 6, 2, 3)]


@pytest.mark.parametrize("case", ALT_TILE_CASES, ids=lambda c: "x".join(map(str, c)))
def test_alternative_fft_tile_matches_oracle(torch_cuda, case):
    """The sweeps with the alternative FFT tile (half the points per thread, a different FFT plan and
    coefficient-table order) against the FP64 oracle: A and A^T within the float32 bar."""
    import paper_1801_00819_gb300 as L
    torch = torch_cuda
    nx, nz, ns, nw = case
    tiles = L.lsm_fft_tiles(nx)
    assert len(tiles) == 2
    L.lsm.lsm_set_fft_tile(nx, ns, nw, tiles[1])
    sv = random_case(nx, nz, ns, nw, seed=500 + nx)
    op = oracle_operator(sv)
    ds = device_survey(sv)
    ws = torch.empty(L.lsm_workspace_bytes(ds.grid, ds.geom, ds.freqs, ns, L.LSM_OP_ADJOINT), dtype=torch.uint8,
                     device="cuda")
    m = np.asarray(sv.reflectivity, dtype=np.float32)
    rng = np.random.default_rng(11)
    d = (rng.normal(size=(ns, nw, nx)) + 1j * rng.normal(size=(ns, nw, nx))).astype(np.complex64)
    out = torch.empty((ns, nw, nx), dtype=torch.complex64, device="cuda")
    L.lsm_forward(ds.grid, ds.slowness, ds.freqs, ds.geom, torch.as_tensor(m, device="cuda"), out, 0, ns, ws)
    img = torch.empty((nz, nx), dtype=torch.float32, device="cuda")
    L.lsm_adjoint(ds.grid, ds.slowness, ds.freqs, ds.geom, torch.as_tensor(d, device="cuda"), img, 0, ns, ws)
    torch.cuda.synchronize()
    assert rel_l2(out.cpu().numpy(), op.forward(m.astype(np.float64))) <= 1e-4
    assert rel_l2(img.cpu().numpy(), op.adjoint(d.astype(np.complex128))) <= 1e-4


def test_pair_tile_partial_receivers_ragged_blocks(torch_cuda):
    """The pair plan (the second tile at nx = 512: one item per warp, the 32-point first stage shared
    by two lanes) with per-shot receiver subsets (a duplicated column included), a shot sub-range,
    accumulation and a ragged last block (5 shots x 31 frequencies = 155 items, one per warp, in
    blocks of 2 warps: the last block holds one item), against the FP64 oracle."""
    import paper_1801_00819_gb300 as L
    torch = torch_cuda
    nx, nz, ns, nw = 512, 9, 6, 31
    tiles = L.lsm_fft_tiles(nx)
    assert tiles[1] == 16
    L.lsm.lsm_set_fft_tile(nx, 5, nw, tiles[1])
    sv = random_case(nx, nz, ns, nw, seed=612)
    rng = np.random.default_rng(8)
    nrec = 300
    rec = np.stack([np.sort(rng.choice(nx, nrec, replace=False)) for _ in range(ns)]).astype(np.int32)
    rec[2, 10] = rec[2, 11]
    op = oracle_operator(sv, rec_ix=rec)
    ds = device_survey(sv, rec_ix=rec)
    ws = torch.empty(L.lsm_workspace_bytes(ds.grid, ds.geom, ds.freqs, 5, L.LSM_OP_ADJOINT), dtype=torch.uint8,
                     device="cuda")
    m = np.asarray(sv.reflectivity, dtype=np.float32)
    out = torch.empty((5, nw, nrec), dtype=torch.complex64, device="cuda")
    L.lsm_forward(ds.grid, ds.slowness, ds.freqs, ds.geom, torch.as_tensor(m, device="cuda"), out, 1, 5, ws)
    d = (rng.normal(size=(5, nw, nrec)) + 1j * rng.normal(size=(5, nw, nrec))).astype(np.complex64)
    base = rng.normal(size=(nz, nx)).astype(np.float32)
    img = torch.as_tensor(base.copy(), device="cuda")
    L.lsm_adjoint(ds.grid, ds.slowness, ds.freqs, ds.geom, torch.as_tensor(d, device="cuda"), img, 1, 5, ws,
                  accumulate=True)
    torch.cuda.synchronize()
    shots = list(range(1, 6))
    assert rel_l2(out.cpu().numpy(), op.forward(m.astype(np.float64), shots=shots)) <= 1e-4
    ref = base.astype(np.float64) + op.adjoint(d.astype(np.complex128), shots=shots)
    assert rel_l2(img.cpu().numpy().astype(np.float64) - base, ref - base) <= 1e-4
    L.lsm.lsm_set_fft_tile(nx, 5, nw, tiles[0])


def test_alternative_fft_tile_sliding_solve(torch_cuda):
    """A sliding solve whose coefficient tables and sweeps all use the alternative tile (window 3,
    slide 2: the refill sweeps over 2 shots run on the window's tables) against the oracle."""
    import paper_1801_00819_gb300 as L
    torch = torch_cuda
    sv = random_case(256, 16, 6, 8, seed=77)
    op = oracle_operator(sv)
    clean = op.forward(np.asarray(sv.reflectivity, dtype=np.float32).astype(np.float64))
    d = (clean + sv.noise_pct * np.sqrt(np.mean(np.abs(clean) ** 2)) * sv.noise()).astype(np.complex64)
    lam = float(np.float32(O.regularisation_from_adjoint(op, d.astype(np.complex128))))
    ds = device_survey(sv)
    L.lsm.lsm_set_fft_tile(256, 3, sv.nw, L.lsm_fft_tiles(256)[1])
    ws = torch.empty(L.lsm_workspace_bytes(ds.grid, ds.geom, ds.freqs, 3, L.LSM_OP_SOLVE), dtype=torch.uint8,
                     device="cuda")
    m = torch.zeros((sv.nz, sv.nx), dtype=torch.float32, device="cuda")
    L.rls_window_solve(ds.grid, ds.slowness, ds.freqs, ds.geom, torch.as_tensor(d, device="cuda"), lam, 3, 2, 0.0,
                       5, m, ws)
    torch.cuda.synchronize()
    m_ref, _ = O.rls_solve(op, d.astype(np.complex128), lam, 3, 2, 5)
    assert rel_l2(m.cpu().numpy().astype(np.float64), m_ref) <= 1e-4
