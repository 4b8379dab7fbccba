"""Batching row: several survey lines of different widths solved concurrently (rls_multi_line_solve).

Each line's image must equal, bitwise, the image of solving that line alone with rls_window_solve,
and every line of a second concurrent solve is checked against its own FP64 oracle solve."""

import numpy as np
import pytest

from oracle import lsm_oracle as O
from synth import random_case
from tests._helpers import oracle_operator, rel_l2, device_survey

pytestmark = pytest.mark.gpu


def test_multi_line_solve_equals_solo_solves():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_1801_00819_gb300 as L
    from paper_1801_00819_gb300 import lsm

    # nx, nz, ns, nw, K, slide, tol, max_iter; line 0 runs a fixed schedule for the oracle check
    specs = [(64, 20, 7, 9, 3, 2, 0.0, 8), (96, 16, 9, 6, 4, 3, 1e-3, 30), (128, 12, 6, 5, 2, 1, 1e-3, 30)]
    problems, solo, refs = [], [], []
    for i, (nx, nz, ns, nw, K, slide, tol, iters) in enumerate(specs):
        sv = random_case(nx, nz, ns, nw, seed=500 + i)
        op = oracle_operator(sv)
        clean = op.forward(np.asarray(sv.reflectivity, dtype=np.float32).astype(np.float64))
        d = (clean + 0.01 * np.sqrt(np.mean(np.abs(clean) ** 2)) * sv.noise()).astype(np.complex64)
        lam = float(np.float32(O.regularisation_from_adjoint(op, d.astype(np.complex128))))
        ds = device_survey(sv)
        dt = torch.as_tensor(d, device="cuda")
        nbytes = L.lsm_workspace_bytes(ds.grid, ds.geom, ds.freqs, K, L.LSM_OP_SOLVE)
        # solo reference on the default stream
        ws = torch.empty(nbytes, dtype=torch.uint8, device="cuda")
        m_solo = torch.zeros((nz, nx), dtype=torch.float32, device="cuda")
        L.rls_window_solve(ds.grid, ds.slowness, ds.freqs, ds.geom, dt, lam, K, slide, tol, iters, m_solo, ws)
        torch.cuda.synchronize()
        solo.append(m_solo.cpu().numpy())
        if i == 0:
            refs.append(O.rls_solve(op, d.astype(np.complex128), lam, K, slide, iters, tol=tol)[0])
        stream = torch.cuda.Stream()
        problems.append(lsm.LineProblem(ds.grid, ds.slowness, ds.freqs, ds.geom, dt, lam, K, slide, tol, iters,
                                        torch.zeros((nz, nx), dtype=torch.float32, device="cuda"),
                                        torch.empty(nbytes, dtype=torch.uint8, device="cuda"), stream))
    torch.cuda.synchronize()
    statuses, stats = lsm.rls_multi_line_solve(problems)
    torch.cuda.synchronize()
    assert statuses == [0, 0, 0]
    for pr, m_solo, (nx, nz, ns, nw, K, slide, _, _), st in zip(problems, solo, specs, stats):
        np.testing.assert_array_equal(pr.m_inout.cpu().numpy(), m_solo)
        assert len(st) == L.lsm_num_windows(ns, K, slide)
    assert rel_l2(problems[0].m_inout.cpu().numpy().astype(np.float64), refs[0]) <= 1e-4


def test_multi_line_solve_every_line_matches_oracle():
    """Three lines of different widths (mixed radix 48 and 160, power of two 256) and uneven windows
    (K = 3, 4, 2) solved together; every line's image against its own FP64 oracle solve.  lambda is
    1e-1 of each line's top eigenvalue of A^T A (power iteration on the oracle), so that the fixed six
    iterates per window are well conditioned (at 1e-2 the 256-wide line's 18 iterates still amplify the
    float32 operators' 1e-6 errors to 2.9e-4)."""
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_1801_00819_gb300 as L
    from paper_1801_00819_gb300 import lsm

    specs = [(48, 12, 5, 6, 3, 2), (160, 10, 6, 5, 4, 2), (256, 8, 4, 4, 2, 1)]
    problems, refs = [], []
    for i, (nx, nz, ns, nw, K, slide) in enumerate(specs):
        sv = random_case(nx, nz, ns, nw, seed=520 + i)
        op = oracle_operator(sv)
        d = op.forward(np.asarray(sv.reflectivity, dtype=np.float32).astype(np.float64)).astype(np.complex64)
        x = np.random.default_rng(i).normal(size=(nz, nx))
        for _ in range(15):
            y = op.adjoint(op.forward(x))
            top = np.linalg.norm(y) / np.linalg.norm(x)
            x = y / np.linalg.norm(y)
        lam = float(np.float32(1e-1 * top))
        refs.append(O.rls_solve(op, d.astype(np.complex128), lam, K, slide, 6)[0])
        ds = device_survey(sv)
        nbytes = L.lsm_workspace_bytes(ds.grid, ds.geom, ds.freqs, K, L.LSM_OP_SOLVE)
        problems.append(lsm.LineProblem(ds.grid, ds.slowness, ds.freqs, ds.geom, torch.as_tensor(d, device="cuda"),
                                        lam, K, slide, 0.0, 6,
                                        torch.zeros((nz, nx), dtype=torch.float32, device="cuda"),
                                        torch.empty(nbytes, dtype=torch.uint8, device="cuda"), torch.cuda.Stream()))
    torch.cuda.synchronize()
    statuses, _ = lsm.rls_multi_line_solve(problems)
    torch.cuda.synchronize()
    assert statuses == [0, 0, 0]
    for pr, ref in zip(problems, refs):
        assert rel_l2(pr.m_inout.cpu().numpy().astype(np.float64), ref) <= 1e-4
