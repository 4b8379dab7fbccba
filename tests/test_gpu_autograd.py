"""Differentiation row: d = A(s) m as a torch autograd function, against the FP64 oracle gradients
(which are pinned by central differences) and by central differences of the GPU forward itself.

Workload: a 64 x 32 crop with the tiny survey's shape; the slowness perturbation direction is a
Gaussian-smoothed N(0, 1e-5) s/m field; the reference slowness is held at the background's row
means; depth checkpoints every 16 rows.
"""

import numpy as np
import pytest
from scipy.ndimage import gaussian_filter

from oracle import lsm_oracle as O
from synth import random_case
from tests._helpers import oracle_operator, rel_l2, device_survey, f32

pytestmark = pytest.mark.gpu

TOL = 1e-4


@pytest.fixture(scope="module")
def torch_cuda():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    return torch


def _problem(nx=64, nz=32, ns=4, nw=8, seed=11, rec=None):
    sv = random_case(nx, nz, ns, nw, seed=seed)
    ds = device_survey(sv, rec_ix=rec)
    op = oracle_operator(sv, rec_ix=rec)
    rng = np.random.default_rng(seed)
    m = f32(sv.reflectivity)
    nrec = op.nrec
    dobs = (rng.normal(size=(ns, nw, nrec)) + 1j * rng.normal(size=(ns, nw, nrec))).astype(np.complex64) * 0.05
    return sv, ds, op, m, dobs


@pytest.mark.parametrize("shape", [(64, 32, 4, 8), (128, 40, 3, 5), (256, 21, 3, 4), (512, 18, 2, 3), (1024, 20, 2, 3),
                                   (32, 17, 5, 6)],
                         ids=lambda s: "x".join(map(str, s)))
def test_gradients_match_oracle(torch_cuda, shape):
    import paper_1801_00819_gb300 as L
    torch = torch_cuda
    nx, nz, ns, nw = shape
    sv, ds, op, m, dobs = _problem(nx, nz, ns, nw, seed=nx + nz)
    g = (op.forward(m) - dobs.astype(np.complex128)) * 2.0
    gm_ref, gs_ref = O.born_gradients(op, m, g)
    sref = torch.as_tensor(op.sref, device="cuda")
    ws = torch.empty(L.lsm_workspace_bytes(ds.grid, ds.geom, ds.freqs, ns, L.LSM_OP_GRADIENT), dtype=torch.uint8,
                     device="cuda")
    mt = torch.as_tensor(m.astype(np.float32), device="cuda")
    gt = torch.as_tensor(g.astype(np.complex64), device="cuda")
    gm = torch.empty_like(mt)
    gs = torch.empty_like(mt)
    d = torch.empty((ns, nw, op.nrec), dtype=torch.complex64, device="cuda")
    L.lsm_born_gradient(ds.grid, ds.slowness, sref, ds.freqs, ds.geom, mt, gt, d, gm, gs, 0, ns, ws)
    torch.cuda.synchronize()
    assert rel_l2(gm.cpu().numpy(), gm_ref) <= TOL
    assert rel_l2(gs.cpu().numpy(), gs_ref) <= TOL
    assert rel_l2(d.cpu().numpy(), op.forward(m)) <= TOL


def test_partial_spread_gradients(torch_cuda):
    import paper_1801_00819_gb300 as L
    torch = torch_cuda
    rng = np.random.default_rng(2)
    rec = np.stack([np.sort(rng.choice(64, 48, replace=False)) for _ in range(3)]).astype(np.int32)
    sv, ds, op, m, dobs = _problem(64, 20, 3, 6, seed=9, rec=rec)
    g = (op.forward(m) - dobs.astype(np.complex128)) * 2.0
    gm_ref, gs_ref = O.born_gradients(op, m, g)
    ws = torch.empty(L.lsm_workspace_bytes(ds.grid, ds.geom, ds.freqs, 3, L.LSM_OP_GRADIENT), dtype=torch.uint8,
                     device="cuda")
    mt = torch.as_tensor(m.astype(np.float32), device="cuda")
    gm = torch.empty_like(mt)
    gs = torch.empty_like(mt)
    L.lsm_born_gradient(ds.grid, ds.slowness, torch.as_tensor(op.sref, device="cuda"), ds.freqs, ds.geom, mt,
                        torch.as_tensor(g.astype(np.complex64), device="cuda"), None, gm, gs, 0, 3, ws)
    torch.cuda.synchronize()
    assert rel_l2(gm.cpu().numpy(), gm_ref) <= TOL
    assert rel_l2(gs.cpu().numpy(), gs_ref) <= TOL


def test_autograd_function_matches_oracle_and_differences(torch_cuda):
    """loss = ||A(s) m - d||^2 + lam ||m||^2 through torch autograd; m.grad and s.grad against the
    oracle, and the slowness directional derivative against central differences of the GPU forward."""
    torch = torch_cuda
    from paper_1801_00819_gb300.autograd import BornModeling
    sv, ds, op, m, dobs = _problem()
    model = BornModeling(ds)
    lam = 1e-3
    mt = torch.as_tensor(m.astype(np.float32), device="cuda").requires_grad_(True)
    st = ds.slowness.clone().requires_grad_(True)
    dt = torch.as_tensor(dobs, device="cuda")
    loss = (model(mt, st) - dt).abs().pow(2).sum() + lam * mt.pow(2).sum()
    loss.backward()
    sref = model.sref.cpu().numpy()
    op_ref = O.SplitStepOperator(f32(sv.slowness), sv.dx, sv.dz, f32(sv.freqs), op.wavelet, sv.src_ix, sv.rec_ix,
                                 sref=sref)
    r = op_ref.forward(m) - dobs.astype(np.complex128)
    gm_ref, gs_ref = O.born_gradients(op_ref, m, 2.0 * r)
    gm_ref = gm_ref + 2 * lam * m
    assert rel_l2(mt.grad.cpu().numpy(), gm_ref) <= TOL
    assert rel_l2(st.grad.cpu().numpy(), gs_ref) <= TOL
    # central differences of the GPU forward along a smooth slowness direction (s_ref held fixed)
    rng = np.random.default_rng(0)
    ds_dir = gaussian_filter(rng.normal(0.0, 1e-5, size=m.shape), 2.0).astype(np.float32)
    dir_t = torch.as_tensor(ds_dir, device="cuda")
    h = 1.0  # the direction already carries the 1e-5 s/m scale
    with torch.no_grad():
        lp = float((model(mt, ds.slowness + h * dir_t) - dt).abs().pow(2).double().sum())
        lm = float((model(mt, ds.slowness - h * dir_t) - dt).abs().pow(2).double().sum())
    fd = (lp - lm) / (2 * h)
    analytic = float((st.grad.double() * dir_t.double()).sum())
    assert abs(fd - analytic) <= 2e-3 * abs(analytic), (fd, analytic)


def test_modelling_with_fixed_reference_matches_oracle(torch_cuda):
    import paper_1801_00819_gb300 as L
    torch = torch_cuda
    sv, ds, op, m, _ = _problem(256, 24, 3, 5, seed=4)
    # a perturbed slowness modelled with the background's reference slowness
    s_pert = f32(sv.slowness * (1 + 0.02 * np.sin(np.arange(256) / 9.0))[None, :])
    op_p = O.SplitStepOperator(s_pert, sv.dx, sv.dz, f32(sv.freqs), op.wavelet, sv.src_ix, sv.rec_ix, sref=op.sref)
    ws = torch.empty(L.lsm_workspace_bytes(ds.grid, ds.geom, ds.freqs, 3, L.LSM_OP_GRADIENT), dtype=torch.uint8,
                     device="cuda")
    d = torch.empty((3, 5, 256), dtype=torch.complex64, device="cuda")
    L.lsm_born_gradient(ds.grid, torch.as_tensor(s_pert.astype(np.float32), device="cuda"),
                        torch.as_tensor(op.sref, device="cuda"), ds.freqs, ds.geom,
                        torch.as_tensor(m.astype(np.float32), device="cuda"), None, d, None, None, 0, 3, ws)
    torch.cuda.synchronize()
    assert rel_l2(d.cpu().numpy(), op_p.forward(m)) <= TOL


def test_gradients_full_size_properties(torch_cuda):
    """Full size, the 512 x 256 window of 16 shots x 128 frequencies: for L = Re <g, A(s) m> the
    gradient kernel's dL/dm equals A^T g from the separately checked adjoint sweep, and <dL/ds, v>
    matches central differences of L along a smooth slowness direction v, modelled through the
    library (s_ref held at the background's row means).  Property checks: the oracle's gradients are
    out of reach at this size."""
    import paper_1801_00819_gb300 as L
    from synth import config_realistic
    torch = torch_cuda
    sv = config_realistic()
    ds = device_survey(sv)
    K, nw, nz, nx, nrec = sv.window, sv.nw, sv.nz, sv.nx, ds.nrec
    s64 = np.asarray(sv.slowness, dtype=np.float32).astype(np.float64)
    sref = torch.as_tensor(s64.mean(axis=1), device="cuda")
    rng = np.random.default_rng(8)
    g = torch.as_tensor(((rng.normal(size=(K, nw, nrec)) + 1j * rng.normal(size=(K, nw, nrec))) * 0.01)
                        .astype(np.complex64), device="cuda")
    m = torch.as_tensor(np.asarray(sv.reflectivity, dtype=np.float32), device="cuda")
    ws = torch.empty(L.lsm_workspace_bytes(ds.grid, ds.geom, ds.freqs, K, L.LSM_OP_GRADIENT), dtype=torch.uint8,
                     device="cuda")
    gm, gs = torch.empty_like(m), torch.empty_like(m)
    L.lsm_born_gradient(ds.grid, ds.slowness, sref, ds.freqs, ds.geom, m, g, None, gm, gs, 0, K, ws)
    ws_a = torch.empty(L.lsm_workspace_bytes(ds.grid, ds.geom, ds.freqs, K, L.LSM_OP_ADJOINT), dtype=torch.uint8,
                       device="cuda")
    img = torch.empty_like(m)
    L.lsm_adjoint(ds.grid, ds.slowness, ds.freqs, ds.geom, g, img, 0, K, ws_a)
    torch.cuda.synchronize()
    assert rel_l2(gm.cpu().numpy().astype(np.float64), img.cpu().numpy().astype(np.float64)) <= 1e-5

    v = torch.as_tensor(gaussian_filter(rng.normal(0.0, 1e-5, size=(nz, nx)), 2.0).astype(np.float32), device="cuda")
    d = torch.empty((K, nw, nrec), dtype=torch.complex64, device="cuda")

    def loss(s):
        L.lsm_born_gradient(ds.grid, s, sref, ds.freqs, ds.geom, m, None, d, None, None, 0, K, ws)
        torch.cuda.synchronize()
        dd = d.cpu().numpy().astype(np.complex128)
        return float(np.sum(np.real(np.conj(g.cpu().numpy().astype(np.complex128)) * dd)))

    # over 256 depth rows the phase perturbation accumulates, so the central difference converges as
    # O(h^2) from -15 % at h = 4 to 2e-5 at h = 1/8 (measured); h = 1/8 keeps FP32 rounding well below
    h = 0.125
    fd = (loss(ds.slowness + h * v) - loss(ds.slowness - h * v)) / (2.0 * h)
    analytic = float((gs.double() * v.double()).sum())
    assert abs(fd - analytic) <= 1e-3 * abs(analytic), (fd, analytic)


@pytest.mark.parametrize("nx", [384, 896])
def test_gradient_rejects_other_widths_before_launch(torch_cuda, nx):
    """Gradients exist for power-of-two widths only: a mixed-radix width is refused on the host."""
    import paper_1801_00819_gb300 as L
    torch = torch_cuda
    sv, ds, op, m, dobs = _problem(nx, 6, 1, 2, seed=nx)
    ws = torch.empty(max(L.lsm_workspace_bytes(ds.grid, ds.geom, ds.freqs, 1, L.LSM_OP_FORWARD), 256),
                     dtype=torch.uint8, device="cuda")
    mt = torch.as_tensor(m.astype(np.float32), device="cuda")
    gt = torch.zeros((1, 2, op.nrec), dtype=torch.complex64, device="cuda")
    gm = torch.empty_like(mt)
    gs = torch.empty_like(mt)
    before = L.lsm_kernel_launches()
    with pytest.raises(L.LsmError) as ei:
        L.lsm_born_gradient(ds.grid, ds.slowness, torch.as_tensor(op.sref, device="cuda"), ds.freqs, ds.geom, mt, gt,
                            None, gm, gs, 0, 1, ws)
    assert ei.value.status == L.lsm.LSM_ERR_UNSUPPORTED_NX
    assert L.lsm_kernel_launches() == before
