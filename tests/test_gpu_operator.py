"""GPU parity of A (lsm_forward) and A^T (lsm_adjoint) against the FP64 oracle, through the C ABI.

Bar: relative L2 error <= 1e-4 for the float32 path (elementwise comparison on the same seeded,
float32-rounded inputs).  Sizes span several blocks of items and ragged tails; the full-size
realistic workload is checked on sampled (shot, frequency) items the oracle computes one by one.
"""

import numpy as np
import pytest

from oracle import lsm_oracle as O
from synth import random_case, config_tiny, config_realistic, config_precision
from tests._helpers import oracle_operator, rel_l2, device_survey

pytestmark = pytest.mark.gpu

TOL = 1e-4

CASES = [
    (16, 8, 3, 5),
    (32, 9, 2, 7),
    (64, 32, 8, 32),
    (128, 20, 3, 9),
    (256, 12, 2, 6),
    (512, 10, 2, 3),
    (1024, 6, 1, 3),
    (64, 1, 3, 3),
    # degenerate: one frequency; one shot and one frequency with two depths
    (128, 12, 3, 1),
    (256, 2, 1, 1),
    # mixed-radix widths nx = q 2^a, q = 3, 5, 7
    (48, 10, 2, 3),
    (96, 8, 3, 4),
    (112, 9, 3, 5),
    (160, 7, 2, 3),
    (384, 12, 2, 3),
    (640, 8, 1, 2),
    (768, 6, 1, 2),
    (896, 6, 1, 2),
]


@pytest.fixture(scope="module")
def torch_cuda():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    return torch


def _gpu_forward(torch, ds, m, shot0, nshots):
    import paper_1801_00819_gb300 as L
    ws = torch.empty(L.lsm_workspace_bytes(ds.grid, ds.geom, ds.freqs, nshots, L.LSM_OP_FORWARD),
                     dtype=torch.uint8, device="cuda")
    mt = torch.as_tensor(np.asarray(m, dtype=np.float32), device="cuda")
    out = torch.empty((nshots, ds.nw, ds.nrec), dtype=torch.complex64, device="cuda")
    L.lsm_forward(ds.grid, ds.slowness, ds.freqs, ds.geom, mt, out, shot0, nshots, ws)
    torch.cuda.synchronize()
    return out.cpu().numpy().astype(np.complex128)


def _gpu_adjoint(torch, ds, d, shot0, nshots, accumulate=None):
    import paper_1801_00819_gb300 as L
    ws = torch.empty(L.lsm_workspace_bytes(ds.grid, ds.geom, ds.freqs, nshots, L.LSM_OP_ADJOINT),
                     dtype=torch.uint8, device="cuda")
    dt = torch.as_tensor(np.asarray(d, dtype=np.complex64), device="cuda")
    if accumulate is None:
        out = torch.empty((ds.nz, ds.nx), dtype=torch.float32, device="cuda")
        L.lsm_adjoint(ds.grid, ds.slowness, ds.freqs, ds.geom, dt, out, shot0, nshots, ws)
    else:
        out = torch.as_tensor(np.asarray(accumulate, dtype=np.float32), device="cuda")
        L.lsm_adjoint(ds.grid, ds.slowness, ds.freqs, ds.geom, dt, out, shot0, nshots, ws, accumulate=True)
    torch.cuda.synchronize()
    return out.cpu().numpy().astype(np.float64)


@pytest.mark.parametrize("case", CASES, ids=lambda c: "x".join(map(str, c)))
def test_forward_matches_oracle(torch_cuda, case):
    nx, nz, ns, nw = case
    sv = random_case(nx, nz, ns, nw, seed=100 + nx + nz)
    op = oracle_operator(sv)
    ds = device_survey(sv)
    m = np.asarray(sv.reflectivity, dtype=np.float32).astype(np.float64)
    got = _gpu_forward(torch_cuda, ds, m, 0, ns)
    ref = op.forward(m)
    err = rel_l2(got, ref)
    assert err <= TOL, err


@pytest.mark.parametrize("case", CASES, ids=lambda c: "x".join(map(str, c)))
def test_adjoint_matches_oracle(torch_cuda, case):
    nx, nz, ns, nw = case
    sv = random_case(nx, nz, ns, nw, seed=200 + nx + nz)
    op = oracle_operator(sv)
    ds = device_survey(sv)
    rng = np.random.default_rng(7)
    d = (rng.normal(size=(ns, nw, nx)) + 1j * rng.normal(size=(ns, nw, nx))).astype(np.complex64)
    got = _gpu_adjoint(torch_cuda, ds, d, 0, ns)
    ref = op.adjoint(d.astype(np.complex128))
    err = rel_l2(got, ref)
    assert err <= TOL, err


def test_shot_subrange_and_accumulate(torch_cuda):
    sv = random_case(64, 16, 6, 5, seed=31)
    op = oracle_operator(sv)
    ds = device_survey(sv)
    rng = np.random.default_rng(3)
    d = (rng.normal(size=(6, 5, 64)) + 1j * rng.normal(size=(6, 5, 64))).astype(np.complex64)
    base = rng.normal(size=(16, 64)).astype(np.float32)
    got = _gpu_adjoint(torch_cuda, ds, d[2:5], 2, 3, accumulate=base)
    ref = base.astype(np.float64) + op.adjoint(d[2:5].astype(np.complex128), shots=np.arange(2, 5))
    assert rel_l2(got, ref) <= TOL
    m = np.asarray(sv.reflectivity, dtype=np.float32).astype(np.float64)
    gotf = _gpu_forward(torch_cuda, ds, m, 1, 4)
    reff = op.forward(m, shots=np.arange(1, 5))
    assert rel_l2(gotf, reff) <= TOL


def test_partial_receiver_spread(torch_cuda):
    """Per-shot receiver subsets (off-end style spreads), including a duplicated column."""
    sv = random_case(64, 12, 4, 6, seed=41)
    rng = np.random.default_rng(5)
    rec = np.stack([np.sort(rng.choice(64, 40, replace=False)) for _ in range(4)]).astype(np.int32)
    rec[1, 3] = rec[1, 4]
    op = oracle_operator(sv, rec_ix=rec)
    ds = device_survey(sv, rec_ix=rec)
    assert ds.geom.rec is not None
    m = np.asarray(sv.reflectivity, dtype=np.float32).astype(np.float64)
    assert rel_l2(_gpu_forward(torch_cuda, ds, m, 0, 4), op.forward(m)) <= TOL
    d = (rng.normal(size=(4, 6, 40)) + 1j * rng.normal(size=(4, 6, 40))).astype(np.complex64)
    assert rel_l2(_gpu_adjoint(torch_cuda, ds, d, 0, 4), op.adjoint(d.astype(np.complex128))) <= TOL


def test_gpu_dot_product_test(torch_cuda):
    """<A m, d> = <m, A^T d> with both sides from the GPU operator (float32 arithmetic)."""
    sv = random_case(128, 40, 4, 16, seed=51)
    ds = device_survey(sv)
    rng = np.random.default_rng(9)
    m = rng.normal(size=(40, 128)).astype(np.float32)
    d = (rng.normal(size=(4, 16, 128)) + 1j * rng.normal(size=(4, 16, 128))).astype(np.complex64)
    Am = _gpu_forward(torch_cuda, ds, m, 0, 4)
    Atd = _gpu_adjoint(torch_cuda, ds, d, 0, 4)
    lhs = O.real_dot(Am, d.astype(np.complex128))
    rhs = O.real_dot(m.astype(np.float64), Atd)
    assert abs(lhs - rhs) <= 1e-5 * abs(lhs)


def test_adjoint_is_deterministic(torch_cuda):
    sv = random_case(256, 16, 5, 7, seed=61)
    ds = device_survey(sv)
    rng = np.random.default_rng(1)
    d = (rng.normal(size=(5, 7, 256)) + 1j * rng.normal(size=(5, 7, 256))).astype(np.complex64)
    a = _gpu_adjoint(torch_cuda, ds, d, 0, 5)
    b = _gpu_adjoint(torch_cuda, ds, d, 0, 5)
    np.testing.assert_array_equal(a, b)


def test_tiny_config_operator(torch_cuda):
    sv = config_tiny()
    op = oracle_operator(sv)
    ds = device_survey(sv)
    m = np.asarray(sv.reflectivity, dtype=np.float32).astype(np.float64)
    d = _gpu_forward(torch_cuda, ds, m, 0, sv.ns)
    assert rel_l2(d, op.forward(m)) <= TOL
    assert rel_l2(_gpu_adjoint(torch_cuda, ds, d, 0, sv.ns), op.adjoint(d)) <= TOL


@pytest.mark.parametrize("tile", [0, 1], ids=["default_tile", "pair_tile"])
def test_realistic_full_size_sampled_items(torch_cuda, tile):
    """512 x 256, 128 frequencies, one 16-shot window in the solver's launch configuration:
    A is compared on sampled (shot, frequency) rows; A^T on data that is zero except at the
    sampled items, which the oracle migrates one by one.  Both FFT tiles: the default 32 points per
    thread, and the pair plan (16 points, a whole warp per item, 14 warps per block)."""
    import paper_1801_00819_gb300 as L
    sv = config_realistic()
    ds = device_survey(sv)
    K, shot0 = sv.window, 40
    tiles = L.lsm_fft_tiles(sv.nx)
    L.lsm.lsm_set_fft_tile(sv.nx, K, sv.nw, tiles[tile])
    try:
        _realistic_sampled_items(torch_cuda, sv, ds, K, shot0)
    finally:
        L.lsm.lsm_set_fft_tile(sv.nx, K, sv.nw, tiles[0])


def _realistic_sampled_items(torch_cuda, sv, ds, K, shot0):
    m = np.asarray(sv.reflectivity, dtype=np.float32).astype(np.float64)
    got = _gpu_forward(torch_cuda, ds, m, shot0, K)
    samples = [(0, 0), (5, 37), (11, 90), (15, 127)]
    op = oracle_operator(sv)
    for ishot, iw in samples:
        sub = op.with_freqs([iw])
        ref = sub.forward(m, shots=[shot0 + ishot])[0, 0]
        assert rel_l2(got[ishot, iw], ref) <= TOL, (ishot, iw)
    rng = np.random.default_rng(2)
    d = np.zeros((K, sv.nw, sv.nx), dtype=np.complex64)
    ref = np.zeros((sv.nz, sv.nx))
    for ishot, iw in samples[:2]:
        row = (rng.normal(size=sv.nx) + 1j * rng.normal(size=sv.nx)).astype(np.complex64)
        d[ishot, iw] = row
        ref += op.with_freqs([iw]).adjoint(row[None, None, :].astype(np.complex128), shots=[shot0 + ishot])
    img = _gpu_adjoint(torch_cuda, ds, d, shot0, K)
    assert rel_l2(img, ref) <= TOL
    # full-size dot-product property on the whole window
    dd = (rng.normal(size=(K, sv.nw, sv.nx)) + 1j * rng.normal(size=(K, sv.nw, sv.nx))).astype(np.complex64)
    lhs = O.real_dot(got, dd.astype(np.complex128))
    rhs = O.real_dot(m, _gpu_adjoint(torch_cuda, ds, dd, shot0, K))
    assert abs(lhs - rhs) <= 1e-4 * abs(lhs)


def test_largest_workload_full_size_sampled_items(torch_cuda):
    """The largest workload, 1024 x 512 with 256 frequencies, one 16-shot window from shot 96
    (about 21 GB of workspace): A compared on sampled (shot, frequency) rows, A^T on data that is
    zero except at sampled items, which the oracle migrates one by one, and the dot-product
    property on the whole window."""
    sv = config_precision()
    ds = device_survey(sv)
    K, shot0 = sv.window, 96
    m = np.asarray(sv.reflectivity, dtype=np.float32).astype(np.float64)
    got = _gpu_forward(torch_cuda, ds, m, shot0, K)
    samples = [(0, 0), (7, 128), (15, 255)]
    op = oracle_operator(sv)
    for ishot, iw in samples:
        ref = op.with_freqs([iw]).forward(m, shots=[shot0 + ishot])[0, 0]
        assert rel_l2(got[ishot, iw], ref) <= TOL, (ishot, iw)
    rng = np.random.default_rng(5)
    d = np.zeros((K, sv.nw, sv.nx), dtype=np.complex64)
    ref = np.zeros((sv.nz, sv.nx))
    for ishot, iw in samples[1:]:
        row = (rng.normal(size=sv.nx) + 1j * rng.normal(size=sv.nx)).astype(np.complex64)
        d[ishot, iw] = row
        ref += op.with_freqs([iw]).adjoint(row[None, None, :].astype(np.complex128), shots=[shot0 + ishot])
    img = _gpu_adjoint(torch_cuda, ds, d, shot0, K)
    assert rel_l2(img, ref) <= TOL
    dd = (rng.normal(size=(K, sv.nw, sv.nx)) + 1j * rng.normal(size=(K, sv.nw, sv.nx))).astype(np.complex64)
    lhs = O.real_dot(got, dd.astype(np.complex128))
    rhs = O.real_dot(m, _gpu_adjoint(torch_cuda, ds, dd, shot0, K))
    assert abs(lhs - rhs) <= 1e-4 * abs(lhs)


BATCHING_LINES = list(range(8))


@pytest.mark.parametrize("line", BATCHING_LINES, ids=lambda i: f"line{i}")
def test_batching_line_full_size_sampled_items(torch_cuda, line):
    """Every line of the eight-line batching workload (nx 256 ... 1024 including the mixed-radix
    384, 640, 768 and 896, nz = nx/2) at its full size: one window of the line's K shots and all
    its frequencies, in the launch configuration its solve uses.  A is compared with the oracle on
    sampled (shot, frequency) rows, A^T on data that is zero except at sampled items, and the
    dot-product property is checked on the whole window."""
    from synth import config_batching_lines
    sv = config_batching_lines()[line]
    ds = device_survey(sv)
    K = sv.window
    shot0 = sv.slide  # the second window
    m = np.asarray(sv.reflectivity, dtype=np.float32).astype(np.float64)
    got = _gpu_forward(torch_cuda, ds, m, shot0, K)
    samples = [(0, 0), (K // 2, sv.nw // 2), (K - 1, sv.nw - 1)]
    op = oracle_operator(sv)
    for ishot, iw in samples:
        ref = op.with_freqs([iw]).forward(m, shots=[shot0 + ishot])[0, 0]
        assert rel_l2(got[ishot, iw], ref) <= TOL, (ishot, iw)
    rng = np.random.default_rng(40 + line)
    d = np.zeros((K, sv.nw, sv.nx), dtype=np.complex64)
    ref = np.zeros((sv.nz, sv.nx))
    for ishot, iw in samples[1:]:
        row = (rng.normal(size=sv.nx) + 1j * rng.normal(size=sv.nx)).astype(np.complex64)
        d[ishot, iw] = row
        ref += op.with_freqs([iw]).adjoint(row[None, None, :].astype(np.complex128), shots=[shot0 + ishot])
    img = _gpu_adjoint(torch_cuda, ds, d, shot0, K)
    assert rel_l2(img, ref) <= TOL
    dd = (rng.normal(size=(K, sv.nw, sv.nx)) + 1j * rng.normal(size=(K, sv.nw, sv.nx))).astype(np.complex64)
    lhs = O.real_dot(got, dd.astype(np.complex128))
    rhs = O.real_dot(m, _gpu_adjoint(torch_cuda, ds, dd, shot0, K))
    assert abs(lhs - rhs) <= 1e-4 * abs(lhs)
    torch_cuda.cuda.empty_cache()
