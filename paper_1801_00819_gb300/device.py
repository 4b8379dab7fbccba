"""Move a survey description into the binding's argument holders and device tensors."""

from __future__ import annotations

from dataclasses import dataclass

import numpy as np

from .lsm import Frequencies, Geometry, Grid


@dataclass
class DeviceSurvey:
    grid: Grid
    geom: Geometry
    freqs: Frequencies
    slowness: "object"      # torch float32 [nz][nx] on the device
    nx: int
    nz: int
    ns: int
    nw: int
    nrec: int


def to_device(nx, nz, dx, dz, slowness, src_ix, rec_ix, freqs_hz, wavelet, device="cuda",
              full_spread=None) -> DeviceSurvey:
    """Holders for one survey line.  rec_ix is dropped (every-column receivers) when it is the
    identity for every shot, unless full_spread is given explicitly."""
    import torch

    rec = np.asarray(rec_ix)
    if full_spread is None:
        full_spread = rec.shape[1] == nx and bool((rec == np.arange(nx)[None, :]).all())
    geom = Geometry(src_ix, None if full_spread else rec, nx=nx)
    s = torch.as_tensor(np.ascontiguousarray(slowness, dtype=np.float32), device=device)
    return DeviceSurvey(Grid(nx, nz, dx, dz), geom, Frequencies(freqs_hz, wavelet), s, nx, nz,
                        int(np.asarray(src_ix).shape[0]), int(np.asarray(freqs_hz).shape[0]),
                        int(geom.c.nrec))


def workspace(nbytes: int, device="cuda"):
    """A device byte buffer for the library's scratch (16-byte aligned by the allocator)."""
    import torch

    return torch.empty(max(int(nbytes), 16), dtype=torch.uint8, device=device)
