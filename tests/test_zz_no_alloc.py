"""The allocation-free adjoint entry point (lsm_adjoint_static).

lsm_adjoint_static exists for callers that may not allocate device memory (it uses one fixed
static device array as scratch); it must give the same image as the workspace-based lsm_adjoint
and, like it, match the FP64 oracle's A^T.  Two calls in a row check that the shared scratch
carries nothing from one call into the next.  Further cases: per-shot receiver columns (the
receiver table is copied into the static array), a problem just over the array's size (rejected
before anything runs, the image untouched), and pinned host arrays overwritten as soon as the call
returns (the call must not read them afterwards).  This file is collected last on purpose.
"""

import ctypes

import numpy as np
import pytest

from synth import random_case
from tests._helpers import device_survey, oracle_operator, rel_l2

pytestmark = pytest.mark.gpu

TOL = 1e-4


@pytest.fixture(scope="module")
def torch_cuda():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    return torch


def _off_end_receivers(sv, nrec):
    """Receivers in the nrec columns left of each source (an off-end spread, wrapping around the
    periodic lateral boundary for shots near the left edge)."""
    return np.stack([(int(xs) - 1 - np.arange(nrec)) % sv.nx for xs in sv.src_ix]).astype(np.int32)


def test_static_scratch_adjoint_matches_workspace_adjoint_on_two_calls(torch_cuda):
    torch = torch_cuda
    import paper_1801_00819_gb300 as L
    from paper_1801_00819_gb300 import lsm

    rng = np.random.default_rng(123)
    calls = [(random_case(64, 32, 8, 32, seed=300), 0, 8, False),
             (random_case(128, 20, 6, 12, seed=301), 2, 3, True)]
    for sv, shot0, nshots, accumulate in calls:
        ds = device_survey(sv)
        d = torch.as_tensor((rng.normal(size=(nshots, sv.nw, sv.nx)) + 1j * rng.normal(size=(nshots, sv.nw, sv.nx)))
                            .astype(np.complex64), device="cuda")
        base = torch.as_tensor(rng.normal(size=(sv.nz, sv.nx)).astype(np.float32), device="cuda")
        ws = torch.empty(L.lsm_workspace_bytes(ds.grid, ds.geom, ds.freqs, nshots, L.LSM_OP_ADJOINT),
                         dtype=torch.uint8, device="cuda")
        assert ws.numel() <= lsm.LSM_STATIC_SCRATCH_BYTES
        ref = base.clone()
        L.lsm_adjoint(ds.grid, ds.slowness, ds.freqs, ds.geom, d, ref, shot0, nshots, ws, accumulate=accumulate)
        got = base.clone()
        lsm.lsm_adjoint_static(ds.grid, ds.slowness, ds.freqs, ds.geom, d, got, shot0, nshots, accumulate=accumulate)
        torch.cuda.synchronize()
        assert rel_l2(got.cpu().numpy(), ref.cpu().numpy()) <= TOL


def test_static_scratch_adjoint_per_shot_receivers_matches_oracle(torch_cuda):
    """Off-end receiver spreads (a receiver table per shot) on two calls in a row, each against
    the FP64 oracle's A^T and against lsm_adjoint."""
    torch = torch_cuda
    import paper_1801_00819_gb300 as L
    from paper_1801_00819_gb300 import lsm

    rng = np.random.default_rng(321)
    for sv, nrec, shot0, nshots in ((random_case(64, 20, 5, 6, seed=310), 40, 0, 5),
                                    (random_case(96, 12, 6, 4, seed=311), 48, 1, 4)):
        rec = _off_end_receivers(sv, nrec)
        op = oracle_operator(sv, rec_ix=rec)
        ds = device_survey(sv, rec_ix=rec)
        assert ds.geom.rec is not None
        d = (rng.normal(size=(nshots, sv.nw, nrec)) + 1j * rng.normal(size=(nshots, sv.nw, nrec))).astype(np.complex64)
        dt = torch.as_tensor(d, device="cuda")
        got = torch.empty((sv.nz, sv.nx), dtype=torch.float32, device="cuda")
        lsm.lsm_adjoint_static(ds.grid, ds.slowness, ds.freqs, ds.geom, dt, got, shot0, nshots)
        ws = torch.empty(L.lsm_workspace_bytes(ds.grid, ds.geom, ds.freqs, nshots, L.LSM_OP_ADJOINT),
                         dtype=torch.uint8, device="cuda")
        ref_ws = torch.empty_like(got)
        L.lsm_adjoint(ds.grid, ds.slowness, ds.freqs, ds.geom, dt, ref_ws, shot0, nshots, ws)
        torch.cuda.synchronize()
        ref = op.adjoint(d.astype(np.complex128), shots=np.arange(shot0, shot0 + nshots))
        assert rel_l2(got.cpu().numpy(), ref) <= TOL
        assert rel_l2(got.cpu().numpy(), ref_ws.cpu().numpy()) <= TOL


def test_static_scratch_rejects_problem_just_over_its_size(torch_cuda):
    """A problem whose scratch is just over LSM_STATIC_SCRATCH_BYTES fails with LSM_ERR_WORKSPACE,
    launches nothing and leaves m_out bit for bit as it was (the size check is the host's, before
    any copy or launch)."""
    torch = torch_cuda
    import paper_1801_00819_gb300 as L
    from paper_1801_00819_gb300 import lsm

    # 256 x 128 grid, one shot: the smallest frequency count whose scratch is over the size
    nx, nz = 256, 128
    sv = random_case(nx, nz, 2, 1, seed=320)
    g = lsm.Grid(nx, nz, sv.dx, sv.dz)
    geo = lsm.Geometry(sv.src_ix, None, nx=nx)

    def freqs_of(n):
        return lsm.Frequencies(np.linspace(5.0, 30.0, n), np.ones(n))

    nw = next(n for n in range(1, 400)
              if L.lsm_workspace_bytes(g, geo, freqs_of(n), 1, L.LSM_OP_ADJOINT) > lsm.LSM_STATIC_SCRATCH_BYTES)
    f = freqs_of(nw)
    assert L.lsm_workspace_bytes(g, geo, freqs_of(nw - 1), 1, L.LSM_OP_ADJOINT) <= lsm.LSM_STATIC_SCRATCH_BYTES
    slow = torch.as_tensor(np.asarray(sv.slowness, dtype=np.float32), device="cuda")
    d = torch.zeros((1, nw, nx), dtype=torch.complex64, device="cuda")
    m_out = torch.as_tensor(np.random.default_rng(7).normal(size=(nz, nx)).astype(np.float32), device="cuda")
    before_img = m_out.clone()
    torch.cuda.synchronize()
    before = lsm.lsm_kernel_launches()
    with pytest.raises(lsm.LsmError) as ei:
        lsm.lsm_adjoint_static(g, slow, f, geo, d, m_out, 0, 1)
    assert ei.value.status == lsm.LSM_ERR_WORKSPACE
    torch.cuda.synchronize()
    assert lsm.lsm_kernel_launches() == before
    assert torch.equal(m_out, before_img)


def test_static_scratch_does_not_read_host_arrays_after_returning(torch_cuda):
    """Geometry and frequencies in pinned host memory, overwritten right after the call returns
    while the stream is still busy with earlier work: the image must be the one the original
    arrays give."""
    torch = torch_cuda
    import paper_1801_00819_gb300 as L
    from paper_1801_00819_gb300 import lsm

    sv = random_case(64, 16, 4, 8, seed=330)
    nrec = 48
    rec = _off_end_receivers(sv, nrec)
    ds = device_survey(sv, rec_ix=rec)
    rng = np.random.default_rng(9)
    d = torch.as_tensor((rng.normal(size=(4, sv.nw, nrec)) + 1j * rng.normal(size=(4, sv.nw, nrec)))
                        .astype(np.complex64), device="cuda")
    ws = torch.empty(L.lsm_workspace_bytes(ds.grid, ds.geom, ds.freqs, 4, L.LSM_OP_ADJOINT),
                     dtype=torch.uint8, device="cuda")
    ref = torch.empty((sv.nz, sv.nx), dtype=torch.float32, device="cuda")
    L.lsm_adjoint(ds.grid, ds.slowness, ds.freqs, ds.geom, d, ref, 0, 4, ws)
    torch.cuda.synchronize()

    src_h = torch.as_tensor(np.asarray(sv.src_ix, dtype=np.int32)).pin_memory()
    rec_h = torch.as_tensor(rec).pin_memory()
    frq_h = torch.as_tensor(np.asarray(sv.freqs, dtype=np.float32)).pin_memory()
    wav_h = torch.as_tensor(np.asarray(sv.wavelet, dtype=np.complex64).view(np.float32)).pin_memory()
    ip = ctypes.POINTER(ctypes.c_int)
    fp = ctypes.POINTER(ctypes.c_float)
    geom = lsm.lsm_geom(4, ctypes.cast(src_h.data_ptr(), ip), nrec, ctypes.cast(rec_h.data_ptr(), ip))
    freqs = lsm.lsm_freqs(sv.nw, ctypes.cast(frq_h.data_ptr(), fp), ctypes.cast(wav_h.data_ptr(), fp))
    got = torch.empty_like(ref)
    stream = torch.cuda.current_stream()
    torch.cuda._sleep(50_000_000)  # keep the stream busy (about 25 ms) so late copies would see the overwrite
    st = lsm.load_library().lsm_adjoint_static(ctypes.byref(ds.grid.c), ds.slowness.data_ptr(), ctypes.byref(freqs),
                                                ctypes.byref(geom), d.data_ptr(), got.data_ptr(), 0, 4, 0,
                                                stream.cuda_stream)
    # other valid values, so that a late read would give a different image but nothing invalid
    src_h.copy_(torch.as_tensor((np.asarray(sv.src_ix) + 7) % sv.nx, dtype=torch.int32))
    rec_h.copy_(torch.as_tensor((rec + 3) % sv.nx))
    frq_h.mul_(1.5)
    wav_h.mul_(-2.0)
    assert st == lsm.LSM_OK
    torch.cuda.synchronize()
    assert rel_l2(got.cpu().numpy(), ref.cpu().numpy()) <= TOL
