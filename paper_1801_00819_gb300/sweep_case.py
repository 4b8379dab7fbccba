"""Run one window of A and A^T on a synthetic survey, for timing and profiling the sweep kernels.

    python -m paper_1801_00819_gb300.sweep_case [--workload realistic|tiny|precision] [--reps N] [--shots K]
        [--freq-stride S] [--transform T] [--tile V] [--gradient [--tune-gradient]]

Prepares the workload's grid, velocity, geometry and frequencies on the device, random data for
one window of K shots, then calls lsm_forward and lsm_adjoint through the C ABI `reps` times each
(each call builds the coefficient tables, computes the window's source wavefields and runs one
sweep).  Prints per-class kernel times from the library's event timing.  --tile records the FFT
tile (points per thread, one of lsm_fft_tiles(nx)) for the window's shape before the calls.  The inputs are random,
so no modelling pass precedes the timed calls.  With --gradient it also calls lsm_born_gradient
(d = A(s) m and the gradients for a random data-space gradient g) on the same window, with the
reference slowness held at the row means of the model.
"""

from __future__ import annotations

import argparse
import json
import os
import sys

import numpy as np

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--workload", default="realistic", choices=("realistic", "tiny", "precision"))
    ap.add_argument("--reps", type=int, default=2)
    ap.add_argument("--shots", type=int, default=0, help="shots per call (default: the window length)")
    ap.add_argument("--freq-stride", type=int, default=1,
                    help="keep every n-th frequency of the workload (smaller captures)")
    ap.add_argument("--transform", default="fft",
                    help="fft, dft_bf16x3, dft_fp16x3, dft_bf16x1, dft_fp16x3_tcgen05 or dft_bf16x3_tcgen05")
    ap.add_argument("--tile", type=int, default=0,
                    help="FFT tile (points per thread) of the register-FFT sweeps; 0: the default")
    ap.add_argument("--gradient", action="store_true", help="also time lsm_born_gradient on the window")
    ap.add_argument("--tune-gradient", action="store_true",
                    help="with --gradient: record the fastest checkpoint stride (lsm_autotune_gradient) first")
    args = ap.parse_args()

    import torch

    import paper_1801_00819_gb300 as L
    from paper_1801_00819_gb300.device import to_device, workspace
    from synth import config_precision, config_realistic, config_tiny

    sv = {"realistic": config_realistic, "tiny": config_tiny, "precision": config_precision}[args.workload]()
    if args.freq_stride > 1:
        sv.freqs = sv.freqs[::args.freq_stride].copy()
        sv.wavelet = sv.wavelet[::args.freq_stride].copy()
    K = args.shots or sv.window
    ds = to_device(sv.nx, sv.nz, sv.dx, sv.dz, sv.slowness, sv.src_ix, sv.rec_ix, sv.freqs, sv.wavelet)
    if args.tile:
        L.lsm.lsm_set_fft_tile(sv.nx, K, sv.nw, args.tile)
    rng = np.random.default_rng(0)
    d = torch.as_tensor((rng.normal(size=(K, sv.nw, sv.nx)) + 1j * rng.normal(size=(K, sv.nw, sv.nx)))
                        .astype(np.complex64), device="cuda")
    m = torch.as_tensor(np.asarray(sv.reflectivity, dtype=np.float32), device="cuda")
    img = torch.empty_like(m)
    out = torch.empty_like(d)
    ws = workspace(L.lsm_workspace_bytes(ds.grid, ds.geom, ds.freqs, K, L.LSM_OP_ADJOINT))
    if args.gradient:
        ws_g = workspace(L.lsm_workspace_bytes(ds.grid, ds.geom, ds.freqs, K, L.LSM_OP_GRADIENT))
        sref = torch.as_tensor(np.asarray(sv.slowness, dtype=np.float64).mean(axis=1), device="cuda")
        grad_m = torch.empty_like(m)
        grad_s = torch.empty_like(m)
    tune = None
    if args.gradient and args.tune_gradient:
        tune = L.lsm_autotune_gradient(ds.grid, ds.slowness, ds.freqs, ds.geom, K, ws_g)
    L.lsm_profile_start()
    for _ in range(args.reps):
        L.lsm_forward(ds.grid, ds.slowness, ds.freqs, ds.geom, m, out, 0, K, ws, transform=args.transform)
        L.lsm_adjoint(ds.grid, ds.slowness, ds.freqs, ds.geom, d, img, 0, K, ws, transform=args.transform)
        if args.gradient:
            L.lsm_born_gradient(ds.grid, ds.slowness, sref, ds.freqs, ds.geom, m, d, out, grad_m, grad_s, 0, K,
                                ws_g)
    torch.cuda.synchronize()
    prof = L.lsm_profile_stop()
    print(json.dumps({"workload": sv.name, "transform": args.transform, "tile": args.tile or L.lsm_fft_tiles(sv.nx)[0],
                      "K": K, "nw": sv.nw, "nz": sv.nz, "nx": sv.nx,
                      "per_launch_ms": {k: (v["ms"] / v["launches"] if v["launches"] else 0.0)
                                        for k, v in prof.items()},
                      "gradient_stride_tune": tune}))


if __name__ == "__main__":
    main()
