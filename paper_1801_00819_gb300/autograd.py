"""Differentiable de-migration d = A(s) m (Eq. 1) for PyTorch.

`BornModeling` wraps one survey line (grid, geometry, frequencies, and a reference slowness held
fixed) and maps a model m [nz][nx] and a slowness s [nz][nx] (float32 CUDA tensors) to the data
d [nshots][nw][nrec] (complex64).  The forward pass is lsm_born_gradient in modelling mode; the
backward pass is lsm_born_gradient in gradient mode, whose model gradient is the A^T kernel and
whose slowness gradient is the adjoint-state recursion with depth-checkpointed recomputation of
the source and adjoint wavefields.  PyTorch's complex gradient convention (dL/dRe + i dL/dIm) is
the one the C ABI takes, so no conversion is needed.
"""

from __future__ import annotations

import torch

from . import lsm as _lsm


class _BornFunction(torch.autograd.Function):
    @staticmethod
    def forward(ctx, m, s, model):
        m = m.contiguous()
        s = s.contiguous()
        d = torch.empty((model.nshots, model.ds.nw, model.ds.nrec), dtype=torch.complex64, device=m.device)
        _lsm.lsm_born_gradient(model.ds.grid, s, model.sref, model.ds.freqs, model.ds.geom, m, None, d, None, None,
                               model.shot0, model.nshots, model.workspace())
        ctx.save_for_backward(m, s)
        ctx.model = model
        return d

    @staticmethod
    def backward(ctx, g):
        m, s = ctx.saved_tensors
        model = ctx.model
        gm = torch.empty_like(m) if ctx.needs_input_grad[0] else None
        gs = torch.empty_like(s) if ctx.needs_input_grad[1] else None
        if gm is None and gs is None:
            return None, None, None
        g = g.contiguous().to(torch.complex64)
        _lsm.lsm_born_gradient(model.ds.grid, s, model.sref, model.ds.freqs, model.ds.geom, m, g, None, gm, gs,
                               model.shot0, model.nshots, model.workspace())
        return gm, gs, None


class BornModeling:
    """d = A(s) m for shots shot0 .. shot0+nshots-1 of a DeviceSurvey, differentiable in m and s.

    sref: the split-step reference slowness held fixed (float64 CUDA tensor [nz]); by default the
    row means of the survey's background slowness.
    """

    def __init__(self, ds, shot0: int = 0, nshots: int | None = None, sref=None):
        self.ds = ds
        self.shot0 = int(shot0)
        self.nshots = int(ds.ns - shot0 if nshots is None else nshots)
        if sref is None:
            sref = ds.slowness.to(torch.float64).mean(dim=1)
        self.sref = sref.to(device=ds.slowness.device, dtype=torch.float64).contiguous()
        self._ws = None

    def workspace(self):
        if self._ws is None:
            n = _lsm.lsm_workspace_bytes(self.ds.grid, self.ds.geom, self.ds.freqs, self.nshots, _lsm.LSM_OP_GRADIENT)
            self._ws = torch.empty(max(n, 16), dtype=torch.uint8, device=self.ds.slowness.device)
        return self._ws

    def __call__(self, m, s=None):
        return _BornFunction.apply(m, self.ds.slowness if s is None else s, self)
