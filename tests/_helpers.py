"""Shared test helpers: oracle operators on the exact float32-rounded inputs the GPU receives."""

import numpy as np

from oracle import lsm_oracle as O


def f32(a):
    return np.asarray(a, dtype=np.float32).astype(np.float64)


def c64(a):
    return np.asarray(a, dtype=np.complex64).astype(np.complex128)


def oracle_operator(sv, rec_ix=None):
    """FP64 oracle fed the same float32 slowness, frequencies and wavelet as the GPU path."""
    rec = sv.rec_ix if rec_ix is None else rec_ix
    return O.SplitStepOperator(f32(sv.slowness), float(np.float32(sv.dx)), float(np.float32(sv.dz)),
                               f32(sv.freqs), c64(sv.wavelet), sv.src_ix, rec)


def rel_l2(a, b):
    a = np.asarray(a)
    b = np.asarray(b)
    return float(np.linalg.norm((a - b).ravel()) / np.linalg.norm(b.ravel()))


def device_survey(sv, rec_ix=None):
    from paper_1801_00819_gb300.device import to_device

    rec = sv.rec_ix if rec_ix is None else rec_ix
    return to_device(sv.nx, sv.nz, sv.dx, sv.dz, sv.slowness, sv.src_ix, rec, sv.freqs, sv.wavelet)
