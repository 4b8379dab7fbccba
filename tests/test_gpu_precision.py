"""Precision row: lateral transforms as tensor-core DFT-matrix products (split BF16 / FP16 three-term
products, FP32 accumulation) against the FP64 oracle, on a subsampled 128 x 64 problem of the
precision workload's construction (6 m grid, layered velocity with anomalies, 3-60 Hz).

The relative L2 error of A and A^T is measured for every precision and checked against a bound per
precision: FP32 FFT 1e-4 (the float32 bar), split FP16 x3 1e-4, split BF16 x3 1e-3, plain BF16 0.2
(one 8-bit-mantissa product per transform, two transforms per depth step, 64 depth steps); the
tcgen05 forms of split FP16 x3 and BF16 x3 are measured beside them at nx = 128, 256, 512, 1024.
The measured errors are printed as JSON, one line per width.
"""

import json
import os

import numpy as np
import pytest

from synth import config_precision_subsample
from oracle import lsm_oracle as O
from tests._helpers import oracle_operator, rel_l2, device_survey

pytestmark = pytest.mark.gpu

BOUNDS = {"fft": 1e-4, "dft_fp16x3": 1e-4, "dft_bf16x3": 1e-3, "dft_bf16x1": 0.2}
# the tcgen05 forms of the split products, at the widths they exist for
TC5_BOUNDS = {"dft_fp16x3_tcgen05": 1e-4, "dft_bf16x3_tcgen05": 1e-3}
TC5_WIDTHS = (128, 256, 512, 1024)


def _subsampled_problem(nx=128):
    return config_precision_subsample(nx)


@pytest.mark.parametrize("nx", [16, 32, 48, 64, 80, 96, 112, 128, 160, 192, 224, 256, 320, 384, 448, 512, 640, 768, 896, 1024])
def test_transform_precisions_against_oracle(nx):
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_1801_00819_gb300 as L
    sv = _subsampled_problem(nx)
    op = oracle_operator(sv)
    ds = device_survey(sv)
    ns = sv.ns
    m = np.asarray(sv.reflectivity, dtype=np.float32)
    rng = np.random.default_rng(0)
    d = (rng.normal(size=(ns, sv.nw, nx)) + 1j * rng.normal(size=(ns, sv.nw, nx))).astype(np.complex64)
    ref_f = op.forward(m.astype(np.float64))
    ref_a = op.adjoint(d.astype(np.complex128))
    ws = torch.empty(L.lsm_workspace_bytes(ds.grid, ds.geom, ds.freqs, ns, L.LSM_OP_ADJOINT), dtype=torch.uint8,
                     device="cuda")
    mt = torch.as_tensor(m, device="cuda")
    dt = torch.as_tensor(d, device="cuda")
    errors = {}
    bounds = dict(BOUNDS, **(TC5_BOUNDS if nx in TC5_WIDTHS else {}))
    for tr, bound in bounds.items():
        out = torch.empty((ns, sv.nw, nx), dtype=torch.complex64, device="cuda")
        L.lsm_forward(ds.grid, ds.slowness, ds.freqs, ds.geom, mt, out, 0, ns, ws, transform=tr)
        img = torch.empty_like(mt)
        L.lsm_adjoint(ds.grid, ds.slowness, ds.freqs, ds.geom, dt, img, 0, ns, ws, transform=tr)
        torch.cuda.synchronize()
        errors[tr] = {"forward": rel_l2(out.cpu().numpy(), ref_f), "adjoint": rel_l2(img.cpu().numpy(), ref_a)}
    print(json.dumps({"nx": nx, "relative_l2_error": errors}))
    out_dir = os.environ.get("LSM_RESULTS_DIR")
    if out_dir:
        with open(os.path.join(out_dir, f"precision_{nx}.json"), "w") as fh:
            json.dump(errors, fh, indent=1)
    for tr, bound in bounds.items():
        assert errors[tr]["forward"] <= bound, (tr, errors[tr])
        assert errors[tr]["adjoint"] <= bound, (tr, errors[tr])


@pytest.mark.parametrize("transform,bound", [("dft_fp16x3", 1e-4), ("dft_bf16x3", 1e-3)])
def test_tensor_core_sliding_solve(transform, bound):
    """The whole sliding-window CG solve with the tensor-core transforms, against the FP64 oracle's
    solve: 128 x 40, 6 shots, window 3 / slide 2, 6 iterations per window."""
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_1801_00819_gb300 as L
    sv = _subsampled_problem(128)
    op = oracle_operator(sv)
    clean = op.forward(np.asarray(sv.reflectivity, dtype=np.float32).astype(np.float64))
    d = (clean + sv.noise_pct * np.sqrt(np.mean(np.abs(clean) ** 2)) * sv.noise()).astype(np.complex64)
    lam = float(np.float32(O.regularisation_from_adjoint(op, d.astype(np.complex128))))
    ds = device_survey(sv)
    ws = torch.empty(L.lsm_workspace_bytes(ds.grid, ds.geom, ds.freqs, 3, L.LSM_OP_SOLVE), dtype=torch.uint8,
                     device="cuda")
    m = torch.zeros((sv.nz, sv.nx), dtype=torch.float32, device="cuda")
    _, stats = L.rls_window_solve(ds.grid, ds.slowness, ds.freqs, ds.geom, torch.as_tensor(d, device="cuda"), lam,
                                  3, 2, 0.0, 6, m, ws, transform=transform)
    torch.cuda.synchronize()
    m_ref, st_ref = O.rls_solve(op, d.astype(np.complex128), lam, 3, 2, 6)
    assert [s["start"] for s in stats] == [s.start for s in st_ref]
    err = rel_l2(m.cpu().numpy().astype(np.float64), m_ref)
    print(json.dumps({"transform": transform, "solve_relative_l2_error": err}))
    assert err <= bound, err


def test_tensor_core_transform_rejects_receiver_subsets():
    """The tensor-core transforms read receivers as the identity map; a receiver table is refused."""
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_1801_00819_gb300 as L
    sv = _subsampled_problem(128)
    rec = np.tile(np.arange(0, 128, 2, dtype=np.int32), (sv.ns, 1))
    ds = device_survey(sv, rec_ix=rec)
    ws = torch.empty(L.lsm_workspace_bytes(ds.grid, ds.geom, ds.freqs, 2, L.LSM_OP_FORWARD), dtype=torch.uint8,
                     device="cuda")
    m = torch.zeros((sv.nz, sv.nx), dtype=torch.float32, device="cuda")
    out = torch.empty((2, sv.nw, 64), dtype=torch.complex64, device="cuda")
    with pytest.raises(L.LsmError):
        L.lsm_forward(ds.grid, ds.slowness, ds.freqs, ds.geom, m, out, 0, 2, ws, transform="dft_fp16x3")


@pytest.mark.parametrize("transform", ["dft_fp16x3", "dft_bf16x3"])
def test_tensor_core_transforms_are_scale_invariant(transform):
    """A is linear: A(c m) = c A(m) for any c.  Wavefields of 1e-6 or 1e4 times the natural size (the
    CG direction vectors take such scales) must keep the precision's relative error; a 16-bit split
    without a block scale loses FP16's narrow exponent range here."""
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_1801_00819_gb300 as L
    sv = _subsampled_problem(128)
    op = oracle_operator(sv)
    ds = device_survey(sv)
    ns = sv.ns
    m = np.asarray(sv.reflectivity, dtype=np.float32)
    ws = torch.empty(L.lsm_workspace_bytes(ds.grid, ds.geom, ds.freqs, ns, L.LSM_OP_ADJOINT), dtype=torch.uint8,
                     device="cuda")
    ref_f = op.forward(m.astype(np.float64))
    rng = np.random.default_rng(1)
    d = (rng.normal(size=(ns, sv.nw, sv.nx)) + 1j * rng.normal(size=(ns, sv.nw, sv.nx))).astype(np.complex64)
    ref_a = op.adjoint(d.astype(np.complex128))
    bound = BOUNDS[transform]
    for c in (1e-6, 1.0, 1e4):
        out = torch.empty((ns, sv.nw, sv.nx), dtype=torch.complex64, device="cuda")
        L.lsm_forward(ds.grid, ds.slowness, ds.freqs, ds.geom, torch.as_tensor(m * np.float32(c), device="cuda"), out,
                      0, ns, ws, transform=transform)
        img = torch.empty((sv.nz, sv.nx), dtype=torch.float32, device="cuda")
        L.lsm_adjoint(ds.grid, ds.slowness, ds.freqs, ds.geom, torch.as_tensor(d * np.complex64(c), device="cuda"),
                      img, 0, ns, ws, transform=transform)
        torch.cuda.synchronize()
        ef = rel_l2(out.cpu().numpy() / c, ref_f)
        ea = rel_l2(img.cpu().numpy() / c, ref_a)
        assert ef <= bound and ea <= bound, (c, ef, ea)
