"""The allocation-free adjoint entry point (lsm_adjoint_static) against lsm_adjoint.

lsm_adjoint_static exists for callers that may not allocate device memory (it uses one fixed
static device array as scratch); it must give the same image as the workspace-based lsm_adjoint.
Two calls in a row check that the shared scratch carries nothing from one call into the next.
This file is collected last on purpose.
"""

import numpy as np
import pytest

from synth import random_case
from tests._helpers import rel_l2, device_survey

pytestmark = pytest.mark.gpu

TOL = 1e-4


def test_static_scratch_adjoint_matches_workspace_adjoint_on_two_calls():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
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
