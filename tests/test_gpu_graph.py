"""CUDA-graph CG (lsm_solve_options.cuda_graph): each window's iterations replayed by a conditional
WHILE node with the stopping test on the device (the default), and the whole solve -- of one line or
of several -- as one graph launch (cuda_graph="solve"), against the host-driven loop
(cuda_graph=False).  The graph runs the host-driven loop's kernels in
the same order, so images must be bitwise identical and iteration counts equal, and both must match
the FP64 oracle's solve."""

import numpy as np
import pytest

from oracle import lsm_oracle as O
from synth import config_tiny, random_case, config_batching_lines
from tests._helpers import oracle_operator, rel_l2, device_survey

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def torch_cuda():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    return torch


def _data(sv, op):
    clean = op.forward(np.asarray(sv.reflectivity, dtype=np.float32).astype(np.float64))
    d = (clean + sv.noise_pct * np.sqrt(np.mean(np.abs(clean) ** 2)) * sv.noise()).astype(np.complex64)
    lam = float(np.float32(O.regularisation_from_adjoint(op, d.astype(np.complex128))))
    return d, lam


def _solve(torch, ds, d, lam, K, slide, tol, iters, **kw):
    import paper_1801_00819_gb300 as L
    ws = torch.empty(L.lsm_workspace_bytes(ds.grid, ds.geom, ds.freqs, K, L.LSM_OP_SOLVE), dtype=torch.uint8,
                     device="cuda")
    m = torch.zeros((ds.nz, ds.nx), dtype=torch.float32, device="cuda")
    status, stats = L.rls_window_solve(ds.grid, ds.slowness, ds.freqs, ds.geom, torch.as_tensor(d, device="cuda"),
                                       lam, K, slide, tol, iters, m, ws, **kw)
    torch.cuda.synchronize()
    return status, m.cpu().numpy(), stats


def _same_stats(a, b):
    assert [w["start"] for w in a] == [w["start"] for w in b]
    assert [w["iters"] for w in a] == [w["iters"] for w in b]
    assert [w["n_forward"] for w in a] == [w["n_forward"] for w in b]
    assert [w["n_adjoint"] for w in a] == [w["n_adjoint"] for w in b]
    for x, y in zip(a, b):
        assert x["rel_res0"] == y["rel_res0"] and x["rel_res"] == y["rel_res"]


def test_graph_fixed_iterations_bitwise_equal_and_oracle(torch_cuda):
    sv = config_tiny()
    op = oracle_operator(sv)
    d, lam = _data(sv, op)
    ds = device_survey(sv)
    _, m_e, st_e = _solve(torch_cuda, ds, d, lam, sv.window, sv.slide, 0.0, sv.cg_iters, cuda_graph=False)
    _, m_g, st_g = _solve(torch_cuda, ds, d, lam, sv.window, sv.slide, 0.0, sv.cg_iters, cuda_graph=True)
    np.testing.assert_array_equal(m_g, m_e)
    _same_stats(st_g, st_e)
    m_ref, _ = O.rls_solve(op, d.astype(np.complex128), lam, sv.window, sv.slide, sv.cg_iters)
    assert rel_l2(m_g.astype(np.float64), m_ref) <= 1e-4


def test_graph_tolerance_stopping_matches_host_loop_and_oracle(torch_cuda):
    sv = random_case(64, 24, 6, 12, seed=71)
    op = oracle_operator(sv)
    d, lam = _data(sv, op)
    ds = device_survey(sv)
    _, m_e, st_e = _solve(torch_cuda, ds, d, lam, 3, 2, 1e-2, 50, cuda_graph=False)
    _, m_g, st_g = _solve(torch_cuda, ds, d, lam, 3, 2, 1e-2, 50, cuda_graph=True)
    np.testing.assert_array_equal(m_g, m_e)
    _same_stats(st_g, st_e)
    _, st_ref = O.rls_solve(op, d.astype(np.complex128), lam, 3, 2, 50, tol=1e-2)
    assert [w["iters"] for w in st_g] == [w.iters for w in st_ref]


def test_graph_zero_iterations_and_converged_start(torch_cuda):
    sv = random_case(32, 8, 4, 5, seed=12)
    op = oracle_operator(sv)
    d, lam = _data(sv, op)
    ds = device_survey(sv)
    _, m0, st0 = _solve(torch_cuda, ds, d, lam, 2, 1, 0.0, 0, cuda_graph=True)
    assert all(w["iters"] == 0 for w in st0) and not np.any(m0)
    _, _, st1 = _solve(torch_cuda, ds, d, lam, 2, 1, 10.0, 5, cuda_graph=True)  # rel_res0 <= tol at once
    assert all(w["iters"] == 0 for w in st1)


def test_graph_preconditioned_and_tensor_core_variants(torch_cuda):
    sv = config_tiny()
    op = oracle_operator(sv)
    d, lam = _data(sv, op)
    ds = device_survey(sv)
    kw = dict(preconditioner="illumination", precond_eps=1e-2)
    _, m_e, st_e = _solve(torch_cuda, ds, d, lam, sv.window, sv.slide, 1e-3, 30, cuda_graph=False, **kw)
    _, m_g, st_g = _solve(torch_cuda, ds, d, lam, sv.window, sv.slide, 1e-3, 30, cuda_graph=True, **kw)
    np.testing.assert_array_equal(m_g, m_e)
    _same_stats(st_g, st_e)
    from synth import config_precision_subsample
    sv2 = config_precision_subsample(128)
    op2 = oracle_operator(sv2)
    d2, lam2 = _data(sv2, op2)
    ds2 = device_survey(sv2)
    _, m_e2, st_e2 = _solve(torch_cuda, ds2, d2, lam2, 3, 2, 0.0, 4, transform="dft_fp16x3", cuda_graph=False)
    _, m_g2, st_g2 = _solve(torch_cuda, ds2, d2, lam2, 3, 2, 0.0, 4, transform="dft_fp16x3", cuda_graph=True)
    np.testing.assert_array_equal(m_g2, m_e2)
    _same_stats(st_g2, st_e2)


def test_graph_breakdown_is_reported(torch_cuda):
    import paper_1801_00819_gb300 as L
    sv = random_case(32, 8, 3, 4, seed=97)
    ds = device_survey(sv)
    d = np.zeros((3, 4, 32), dtype=np.complex64)
    d[1, 2, 5] = np.nan
    status, _, _ = _solve(torch_cuda, ds, d, 1.0, 3, 1, 0.0, 3, cuda_graph=True, raise_on_breakdown=False)
    assert status == L.lsm.LSM_ERR_BREAKDOWN


def test_graph_multi_line_equals_solo_host_loop(torch_cuda):
    import paper_1801_00819_gb300 as L
    from paper_1801_00819_gb300.device import to_device, workspace
    lines = [random_case(nx, 10, 5, 6, seed=300 + nx) for nx in (64, 96, 128)]
    probs, solo = [], []
    for i, sv in enumerate(lines):
        op = oracle_operator(sv)
        d, lam = _data(sv, op)
        ds = to_device(sv.nx, sv.nz, sv.dx, sv.dz, np.asarray(sv.slowness, np.float32), sv.src_ix, sv.rec_ix,
                       sv.freqs, sv.wavelet)
        K, slide = 2 + i, 1
        _, m_solo, st_solo = _solve(torch_cuda, ds, d, lam, K, slide, 1e-2, 20, cuda_graph=False)
        solo.append((m_solo, st_solo))
        ws = workspace(L.lsm_workspace_bytes(ds.grid, ds.geom, ds.freqs, K, L.LSM_OP_SOLVE))
        m = torch_cuda.zeros((sv.nz, sv.nx), dtype=torch_cuda.float32, device="cuda")
        probs.append(L.LineProblem(ds.grid, ds.slowness, ds.freqs, ds.geom, torch_cuda.as_tensor(d, device="cuda"),
                                   lam, K, slide, 1e-2, 20, m, ws, torch_cuda.cuda.Stream()))
    statuses, stats = L.rls_multi_line_solve(probs, cuda_graph=True)
    torch_cuda.cuda.synchronize()
    assert statuses == [0, 0, 0]
    for pr, st, (m_solo, st_solo) in zip(probs, stats, solo):
        np.testing.assert_array_equal(pr.m_inout.cpu().numpy(), m_solo)
        _same_stats(st, st_solo)


def test_default_is_graph_unless_sweeps_are_timed(torch_cuda):
    """The default loop is the graph (its kernels are not event-timed), except while the A / A^T
    sweeps are being timed; both give the same image."""
    import paper_1801_00819_gb300 as L
    sv = config_tiny()
    op = oracle_operator(sv)
    d, lam = _data(sv, op)
    ds = device_survey(sv)
    L.lsm_profile_start(classes=("vector",))
    _, m_a, _ = _solve(torch_cuda, ds, d, lam, sv.window, sv.slide, 0.0, sv.cg_iters)
    prof = L.lsm_profile_stop()
    assert prof["vector"]["launches"] < 3 * 2 * sv.cg_iters  # only the set-up kernels outside the graph
    L.lsm_profile_start(classes=("adjoint", "forward"))
    _, m_b, _ = _solve(torch_cuda, ds, d, lam, sv.window, sv.slide, 0.0, sv.cg_iters)
    prof = L.lsm_profile_stop()
    assert prof["adjoint"]["launches"] == 3 * (2 + sv.cg_iters)  # the host-driven loop, every sweep timed
    np.testing.assert_array_equal(m_a, m_b)


def test_graph_tcgen05_transform_bitwise_equal_to_host_loop(torch_cuda):
    """The tcgen05 transforms (nx = 512) inside the graph-replayed CG iterations: the same images and
    statistics as the host-driven loop, with tolerance stopping."""
    sv = random_case(512, 12, 5, 6, seed=93)
    op = oracle_operator(sv)
    d, lam = _data(sv, op)
    ds = device_survey(sv)
    for transform in ("dft_fp16x3_tcgen05", "dft_bf16x3_tcgen05"):
        s_e, m_e, st_e = _solve(torch_cuda, ds, d, lam, 3, 2, 2e-2, 20, transform=transform, cuda_graph=False)
        s_g, m_g, st_g = _solve(torch_cuda, ds, d, lam, 3, 2, 2e-2, 20, transform=transform, cuda_graph=True)
        assert s_e == s_g == 0
        np.testing.assert_array_equal(m_e, m_g)
        _same_stats(st_e, st_g)
        assert all(0 < w["iters"] < 20 for w in st_g)


# ---------------------------------------------------------------- whole-solve graph (cuda_graph="solve")

@pytest.mark.parametrize("kw", [{}, {"preconditioner": "illumination"}, {"transform": "dft_bf16x3_tcgen05"}],
                         ids=["plain", "illumination", "tcgen05"])
def test_solve_graph_bitwise_equal_to_host_loop(torch_cuda, kw):
    """The whole solve as one graph launch (every window's set-up, WHILE node and outcome record
    chained in one graph): the host-driven loop's images and statistics, with tolerance stopping."""
    sv = random_case(128, 12, 7, 6, seed=95)
    op = oracle_operator(sv)
    d, lam = _data(sv, op)
    ds = device_survey(sv)
    s_e, m_e, st_e = _solve(torch_cuda, ds, d, lam, 3, 2, 2e-2, 20, cuda_graph=False, **kw)
    s_g, m_g, st_g = _solve(torch_cuda, ds, d, lam, 3, 2, 2e-2, 20, cuda_graph="solve", **kw)
    assert s_e == s_g == 0
    np.testing.assert_array_equal(m_g, m_e)
    _same_stats(st_g, st_e)
    assert len(st_g) == 3 and all(0 < w["iters"] < 20 for w in st_g)
    assert all(w["ms"] == 0.0 for w in st_g)


def test_solve_graph_fixed_iterations_and_resume(torch_cuda):
    """Fixed iteration counts (tol 0) on the tiny configuration, the whole call and a call resumed at
    window 1 for two windows, each against the host-driven loop."""
    sv = config_tiny()
    op = oracle_operator(sv)
    d, lam = _data(sv, op)
    ds = device_survey(sv)
    _, m_e, st_e = _solve(torch_cuda, ds, d, lam, sv.window, sv.slide, 0.0, sv.cg_iters, cuda_graph=False)
    _, m_g, st_g = _solve(torch_cuda, ds, d, lam, sv.window, sv.slide, 0.0, sv.cg_iters, cuda_graph="solve")
    np.testing.assert_array_equal(m_g, m_e)
    _same_stats(st_g, st_e)
    _, m_e1, st_e1 = _solve(torch_cuda, ds, d, lam, sv.window, sv.slide, 0.0, sv.cg_iters, cuda_graph=False,
                            first_window=1, n_windows=2)
    _, m_g1, st_g1 = _solve(torch_cuda, ds, d, lam, sv.window, sv.slide, 0.0, sv.cg_iters, cuda_graph="solve",
                            first_window=1, n_windows=2)
    np.testing.assert_array_equal(m_g1, m_e1)
    _same_stats(st_g1[:2], st_e1[:2])


def test_solve_graph_breakdown_halts_later_windows(torch_cuda):
    """A window that breaks down ends the call with LSM_ERR_BREAKDOWN; the windows after it run no
    iterations, so the image is the host-driven loop's (which stops there)."""
    import paper_1801_00819_gb300 as L
    sv = random_case(32, 8, 5, 4, seed=97)
    ds = device_survey(sv)
    rng = np.random.default_rng(1)
    d = (rng.normal(size=(5, 4, 32)) + 1j * rng.normal(size=(5, 4, 32))).astype(np.complex64)
    d[3, 2, 5] = np.nan  # shot 3: windows 1 (shots 1-3) and 2 (shots 2-4)
    s_e, m_e, st_e = _solve(torch_cuda, ds, d, 1.0, 3, 1, 0.0, 3, cuda_graph=False, raise_on_breakdown=False)
    s_g, m_g, st_g = _solve(torch_cuda, ds, d, 1.0, 3, 1, 0.0, 3, cuda_graph="solve", raise_on_breakdown=False)
    assert s_e == s_g == L.lsm.LSM_ERR_BREAKDOWN
    np.testing.assert_array_equal(m_g, m_e)
    assert st_g[0]["iters"] == st_e[0]["iters"] == 3 and st_g[1]["iters"] == st_e[1]["iters"]


def test_solve_graph_multi_line_equals_solo_host_loop(torch_cuda):
    """Three lines of different widths and window lengths, every window of every line in one graph
    launch: each line's image and statistics equal solving it alone with the host-driven loop."""
    import paper_1801_00819_gb300 as L
    from paper_1801_00819_gb300.device import to_device, workspace
    lines = [random_case(nx, 10, 6, 5, seed=310 + nx) for nx in (64, 96, 256)]
    probs, solo = [], []
    for i, sv in enumerate(lines):
        op = oracle_operator(sv)
        d, lam = _data(sv, op)
        ds = to_device(sv.nx, sv.nz, sv.dx, sv.dz, np.asarray(sv.slowness, np.float32), sv.src_ix, sv.rec_ix,
                       sv.freqs, sv.wavelet)
        K, slide = 2 + i, 1 + i % 2
        _, m_solo, st_solo = _solve(torch_cuda, ds, d, lam, K, slide, 1e-2, 20, cuda_graph=False)
        solo.append((m_solo, st_solo))
        ws = workspace(L.lsm_workspace_bytes(ds.grid, ds.geom, ds.freqs, K, L.LSM_OP_SOLVE))
        m = torch_cuda.zeros((sv.nz, sv.nx), dtype=torch_cuda.float32, device="cuda")
        probs.append(L.LineProblem(ds.grid, ds.slowness, ds.freqs, ds.geom, torch_cuda.as_tensor(d, device="cuda"),
                                   lam, K, slide, 1e-2, 20, m, ws, torch_cuda.cuda.Stream()))
    before = L.lsm_kernel_launches()
    statuses, stats = L.rls_multi_line_solve(probs, cuda_graph="solve")
    torch_cuda.cuda.synchronize()
    assert statuses == [0, 0, 0]
    assert L.lsm_kernel_launches() > before
    for pr, st, (m_solo, st_solo) in zip(probs, stats, solo):
        np.testing.assert_array_equal(pr.m_inout.cpu().numpy(), m_solo)
        _same_stats(st, st_solo)


def test_cuda_graph_option_out_of_range_is_rejected(torch_cuda):
    import ctypes

    import paper_1801_00819_gb300 as L
    from paper_1801_00819_gb300 import lsm
    sv = random_case(32, 8, 3, 4, seed=98)
    ds = device_survey(sv)
    ws = torch_cuda.empty(L.lsm_workspace_bytes(ds.grid, ds.geom, ds.freqs, 2, L.LSM_OP_SOLVE),
                          dtype=torch_cuda.uint8, device="cuda")
    m = torch_cuda.zeros((sv.nz, sv.nx), dtype=torch_cuda.float32, device="cuda")
    d = torch_cuda.zeros((3, 4, 32), dtype=torch_cuda.complex64, device="cuda")
    opts = lsm.lsm_solve_options(0, 1e-2, 0, 3)
    stats = (lsm.lsm_window_stats * 4)()
    st = lsm.load_library().rls_window_solve_ex(
        ctypes.byref(ds.grid.c), lsm._ptr(ds.slowness), ctypes.byref(ds.freqs.c), ctypes.byref(ds.geom.c), lsm._ptr(d),
        1.0, 2, 1, 0.0, 2, 0, 0, lsm._ptr(m), stats, 4, lsm._ptr(ws), lsm._nbytes(ws), None, ctypes.byref(opts))
    assert st == lsm.LSM_ERR_ARG


def test_solve_graph_with_no_window_left_launches_nothing(torch_cuda):
    """A call resumed after the last window (first_window = number of windows) returns at once in
    every loop form: no launch, image unchanged."""
    import paper_1801_00819_gb300 as L
    sv = random_case(64, 8, 5, 3, seed=99)
    op = oracle_operator(sv)
    d, lam = _data(sv, op)
    ds = device_survey(sv)
    nwin = L.lsm.load_library().lsm_num_windows(sv.ns, 2, 1)
    ws = torch_cuda.empty(L.lsm_workspace_bytes(ds.grid, ds.geom, ds.freqs, 2, L.LSM_OP_SOLVE),
                          dtype=torch_cuda.uint8, device="cuda")
    m = torch_cuda.full((sv.nz, sv.nx), 0.25, dtype=torch_cuda.float32, device="cuda")
    for mode in (False, True, "solve"):
        before = L.lsm_kernel_launches()
        status, stats = L.rls_window_solve(ds.grid, ds.slowness, ds.freqs, ds.geom,
                                           torch_cuda.as_tensor(d, device="cuda"), lam, 2, 1, 0.0, 3, m, ws,
                                           first_window=nwin, cuda_graph=mode)
        torch_cuda.cuda.synchronize()
        assert status == 0 and stats == [] and L.lsm_kernel_launches() == before
    assert bool((m == 0.25).all())
