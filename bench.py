#!/usr/bin/env python
"""Benchmark of the block-row recursive least-squares migration solve on one GB300.

One step = one complete sliding-window solve of the realistic synthetic survey (512 x 256 grid at
8 m, 96 shots, 128 frequencies 3-40 Hz, window K = 16 shots, slide 8, every window's CG run to a
relative normal-equation residual of 1e-3), warm-started window to window, through the C ABI
(rls_window_solve) with the survey data already resident in HBM.

Metric: shot*omega*depth units per second through A + A^T: each window contributes
(applications of A + applications of A^T) / 2 * K * nw * nz units; value = units of all ranks /
(max over ranks of the timed wall time).  ms_per_step is the time to solve the whole survey to
1e-3 (the time-to-residual half of the metric).

Also reported: the dominant sweep kernel against its roofline (per-launch CUDA-event times taken
live on the library's stream), the end-to-end number with host buffers (pinned host -> device
copies of the data and slowness and the device -> host copy of the image inside the timed
region), SM clocks sampled during the timed region, and the FP64 oracle timed on the host cores
on a bounded sample (cpu_baseline).

`--impl reference` times the FP64 oracle (test infrastructure, pure numpy) on the host cores as
the reference arm: each step is one A + A^T application on one shot and 16 frequencies of
the same workload.

Launch: `python bench.py --gpus 1 --steps K --warmup W`; for N > 1 under torchrun each rank
solves its own independent survey line (weak scaling, no collective on the data path).
"""

from __future__ import annotations

import argparse
import hashlib
import json
import math
import os
import re
import statistics
import subprocess
import sys
import tempfile
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

METRIC = "shot*omega*depth steps/s for A+A^T (window-RLS solve to 1e-3 residual)"
FP32_LANES_PER_SM = 128     # FP32 FMA lanes per Blackwell SM
FALLBACK_HBM_GBS = 6800.0   # profiling recipe's fallback copy bandwidth
PROFILE_SUMMARY = os.path.join(ROOT, "profiles", "sweep_kernels_realistic_512x256.md")


def parse_args():
    ap = argparse.ArgumentParser(description=__doc__, formatter_class=argparse.RawDescriptionHelpFormatter)
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=3)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", choices=("gb300", "reference"), default="gb300")
    ap.add_argument("--workload", choices=("realistic", "tiny", "batching"), default="realistic",
                    help="batching: eight survey lines of mixed widths solved concurrently vs one after another")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--no-variants", action="store_true")
    ap.add_argument("--no-autotune", action="store_true",
                    help="run the default launch shapes instead of tuning them before the untimed warm-up")
    ap.add_argument("--ref-sample-freqs", type=int, default=16,
                    help="frequencies of the oracle sample timed by the reference arm (each step) and by the GPU "
                         "arm's cpu_baseline (repeated for at least 10 s)")
    return ap.parse_args()


def dist_info():
    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return rank, world, local


def reduce_over_ranks(units, t_ms, world, device):
    """Whole-job totals of one timed region: the units every rank processed (each rank solves its
    own survey line, whose CG iteration counts may differ) and the slowest rank's time."""
    if world <= 1:
        return float(units), float(t_ms)
    import torch
    import torch.distributed as dist
    u = torch.tensor([float(units)], dtype=torch.float64, device=device)
    t = torch.tensor([float(t_ms)], dtype=torch.float64, device=device)
    dist.all_reduce(u, op=dist.ReduceOp.SUM)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(u.item()), float(t.item())


def workload(name, rank=0):
    from synth import config_realistic, config_tiny

    sv = config_realistic() if name == "realistic" else config_tiny()
    if name == "tiny":
        sv.cg_tol, sv.cg_iters = 1e-3, 200
    sv.noise_seed = sv.noise_seed + rank  # independent line per rank
    return sv


def workload_config(sv, l2_note=True):
    cfg = {"workload": f"{sv.name} {sv.nx}x{sv.nz} grid, {sv.ns} shots, {sv.nw} freqs "
                       f"{sv.freqs[0]:g}-{sv.freqs[-1]:g} Hz, window {sv.window}, slide {sv.slide}, "
                       f"CG to {sv.cg_tol:g}",
           "nx": sv.nx, "nz": sv.nz, "dx_m": sv.dx, "shots": sv.ns, "freqs": sv.nw, "window_K": sv.window,
           "slide": sv.slide, "cg_tol": sv.cg_tol, "noise_pct": sv.noise_pct * 100}
    if l2_note:
        cfg["l2"] = "inputs larger than L2: each step streams the source-wavefield ring (K*nw*nz*nx c64) " \
                    "and coefficient tables from HBM"
    return cfg


# ------------------------------------------------------------------ clocks


class ClockSampler:
    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index):
        self.gpu = gpu_index
        self.proc = None
        self.path = None

    def start(self):
        fd, self.path = tempfile.mkstemp(prefix="clocks_", suffix=".csv")
        os.close(fd)
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.gpu), f"--query-gpu={self.FIELDS}", "--format=csv,noheader,nounits",
                 "-lms", "200"], stdout=open(self.path, "w"), stderr=subprocess.DEVNULL)
        except OSError:
            self.proc = None

    def stop(self):
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except subprocess.TimeoutExpired:
            self.proc.kill()
        sm, smax, reasons = [], [], set()
        names = ("hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap")
        with open(self.path) as fh:
            for line in fh:
                parts = [p.strip() for p in line.split(",")]
                if len(parts) < 9:
                    continue
                try:
                    sm.append(float(parts[1]))
                    smax.append(float(parts[2]))
                except ValueError:
                    continue
                for n, v in zip(names, parts[5:9]):
                    if v.lower() == "active":
                        reasons.add(n)
        os.unlink(self.path)
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": max(smax) if smax else None,
                "reasons": sorted(reasons), "samples": len(sm)}


# ------------------------------------------------------------------ roofline helpers


def measured_peaks():
    path = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(path):
        with open(path) as fh:
            return json.load(fh), "measured"
    return {"hbm_gbs": FALLBACK_HBM_GBS}, "fallback"


def flops_per_unit(nx):
    """One split-step depth step of one wavefield: forward + inverse nx-point FFT at the nominal
    5 n log2 n each, the phase-shift and split-step complex multiplies (6 nx each), and the imaging
    (adjoint) or scatter-add (forward) term (4 nx)."""
    return 10 * nx * math.log2(nx) + 16 * nx


def bytes_per_unit(nx, nrec, nz, K, cg_adjoint=False):
    """Algorithmic HBM bytes of one unit of an A or A^T sweep: the cached source-wavefield row
    (8 nx), the Phi and D coefficient rows shared by the K shots of the window (16 nx / K), and the
    item's data row read or written once over the depth loop (8 nrec / nz).  The adjoint of a CG
    iteration also reads q and writes the updated residual r back (16 nrec / nz more)."""
    return 8 * nx + 16 * nx / K + (24 if cg_adjoint else 8) * nrec / nz


def kernel_source_hash():
    """Hash of the sources the sweep kernels are compiled from (lsm_fft.cuh, lsm_sweep.cuh,
    lsm_async.cuh, lsm_internal.h, lsm_cg.h and the per-nx instantiation files)."""
    h = hashlib.sha256()
    csrc = os.path.join(ROOT, "paper_1801_00819_gb300", "csrc")
    names = sorted(n for n in os.listdir(csrc)
                   if n in ("lsm_fft.cuh", "lsm_sweep.cuh", "lsm_async.cuh", "lsm_internal.h", "lsm_cg.h")
                   or n.startswith("sweep_n"))
    for name in names:
        with open(os.path.join(csrc, name), "rb") as fh:
            h.update(name.encode())
            h.update(fh.read())
    return h.hexdigest()[:16]


def profiled_traffic(kclass):
    """DRAM bytes per launch recorded in the committed ncu summary, if it was taken on the current
    kernel sources (null otherwise)."""
    if not os.path.exists(PROFILE_SUMMARY):
        return None
    text = open(PROFILE_SUMMARY).read()
    m_hash = re.search(r"kernel_source_hash:\s*([0-9a-f]+)", text)
    m_val = re.search(rf"{kclass}_dram_bytes_per_launch:\s*([0-9.eE+]+)", text)
    if not m_hash or not m_val or m_hash.group(1) != kernel_source_hash():
        return None
    return float(m_val.group(1))


# ------------------------------------------------------------------ GPU arm


def gpu_arm(args):
    import numpy as np
    import torch

    import paper_1801_00819_gb300 as L
    from paper_1801_00819_gb300.device import to_device, workspace

    rank, world, local = dist_info()
    torch.cuda.set_device(local)
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl", device_id=torch.device("cuda", local))
    from paper_1801_00819_gb300 import build as B
    if rank == 0:  # one process brings the in-tree library up to date; the others wait for it
        B.build()
    if world > 1:
        dist.barrier()

    sv = workload(args.workload, rank)
    s32 = np.asarray(sv.slowness, dtype=np.float32)
    ds = to_device(sv.nx, sv.nz, sv.dx, sv.dz, s32, sv.src_ix, sv.rec_ix, sv.freqs, sv.wavelet)
    K, nw, nz, nx, ns = sv.window, sv.nw, sv.nz, sv.nx, sv.ns

    # synthetic data d = A m + noise, modelled with the library itself in chunks of K shots
    m_true = torch.as_tensor(np.asarray(sv.reflectivity, dtype=np.float32), device="cuda")
    d = torch.empty((ns, nw, ds.nrec), dtype=torch.complex64, device="cuda")
    ws_f = workspace(L.lsm_workspace_bytes(ds.grid, ds.geom, ds.freqs, K, L.LSM_OP_ADJOINT))
    for s0 in range(0, ns, K):
        n = min(K, ns - s0)
        L.lsm_forward(ds.grid, ds.slowness, ds.freqs, ds.geom, m_true, d[s0:s0 + n], s0, n, ws_f)
    rms = float(torch.sqrt(torch.mean(torch.abs(d) ** 2)))
    noise = torch.as_tensor(sv.noise().astype(np.complex64), device="cuda")
    d += sv.noise_pct * rms * noise
    del noise
    adj = torch.zeros((nz, nx), dtype=torch.float32, device="cuda")
    for s0 in range(0, ns, K):
        n = min(K, ns - s0)
        L.lsm_adjoint(ds.grid, ds.slowness, ds.freqs, ds.geom, d[s0:s0 + n], adj, s0, n, ws_f, accumulate=True)
    lam = 1e-3 * float(adj.abs().max())
    del ws_f
    torch.cuda.synchronize()

    ws = workspace(L.lsm_workspace_bytes(ds.grid, ds.geom, ds.freqs, K, L.LSM_OP_SOLVE))
    m = torch.zeros((nz, nx), dtype=torch.float32, device="cuda")
    # launch shapes: timed and recorded once, before the warm-up and outside the timed region, for
    # the window's A / A^T / source sweeps (K shots) and the source refills (slide shots)
    tune = None
    if not args.no_autotune:
        tune = {"window_shots": L.lsm_autotune(ds.grid, ds.slowness, ds.freqs, ds.geom, K, ws)}
        if sv.slide != K:
            tune["refill_shots"] = {"source": L.lsm_autotune(ds.grid, ds.slowness, ds.freqs, ds.geom, sv.slide,
                                                             ws)["source"]}
        torch.cuda.synchronize()

    # the FP32 roofline's denominator, measured on this GPU before the warm-up (FMA-chain kernels)
    try:
        fp32_peak = L.lsm_measure_fp32_peak()
    except Exception as exc:  # reported, and the derived figure used instead
        fp32_peak = {"error": str(exc)}
    torch.cuda.synchronize()

    nwin = L.lsm_num_windows(ns, K, sv.slide)
    prof = {}

    def step(timed=False):
        """One solve of every window.  The first window runs the host-driven CG loop; inside the
        timed region its kernels are event-timed (the roofline's launch times: a conditional graph
        node cannot hold event records).  The remaining windows resume from its image with the
        library's default loop, each window's iterations one CUDA graph; the image is bitwise the
        one an uninterrupted solve gives."""
        m.zero_()
        if timed:
            L.lsm_profile_start(classes=("tables", "source", "adjoint", "forward"))
        _, st = L.rls_window_solve(ds.grid, ds.slowness, ds.freqs, ds.geom, d, lam, K, sv.slide, sv.cg_tol,
                                   sv.cg_iters, m, ws, n_windows=1, cuda_graph=False)
        if timed:
            for k, v in L.lsm_profile_stop().items():
                acc = prof.setdefault(k, {"launches": 0, "ms": 0.0})
                acc["launches"] += v["launches"]
                acc["ms"] += v["ms"]
        if nwin > 1:
            _, st_rest = L.rls_window_solve(ds.grid, ds.slowness, ds.freqs, ds.geom, d, lam, K, sv.slide,
                                            sv.cg_tol, sv.cg_iters, m, ws, first_window=1, cuda_graph=True)
            st = st + st_rest
        return st

    def barrier():
        if world > 1:
            import torch.distributed as dist
            dist.barrier()

    for _ in range(args.warmup):
        step()
    torch.cuda.synchronize()

    clocks = ClockSampler(torch.cuda.current_device())
    stream = torch.cuda.current_stream()
    ev0, ev1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    barrier()
    torch.cuda.synchronize()
    clocks.start()
    launches0 = L.lsm_kernel_launches()
    # event timing of the sweep and table kernels of each step's first window only: the roofline
    # needs the sweeps' times, and event records around the two short CG vector launches per
    # iteration would slow the solve
    ev0.record(stream)
    stats = []
    for _ in range(args.steps):
        stats.append(step(timed=True))
    ev1.record(stream)
    torch.cuda.synchronize()
    launches = L.lsm_kernel_launches() - launches0
    barrier()
    clk = clocks.stop()
    m_fp32 = m.clone()  # the plain FP32 solve's image, for the variants' comparisons
    t_ms = ev0.elapsed_time(ev1)
    units_per_pass = K * nw * nz
    units = sum((w["n_forward"] + w["n_adjoint"]) / 2 * units_per_pass for st in stats for w in st)
    units_all, t_max = reduce_over_ranks(units, t_ms, world, "cuda")
    value = units_all / (t_max / 1e3)
    iters = [w["iters"] for w in stats[-1]]
    final_res = [w["rel_res"] for w in stats[-1]]

    # dominant sweep kernel vs its roofline
    dom = max(("adjoint", "forward"), key=lambda k: prof[k]["ms"])
    avg_ms = prof[dom]["ms"] / max(prof[dom]["launches"], 1)
    fl = flops_per_unit(nx) * units_per_pass
    by = bytes_per_unit(nx, ds.nrec, nz, K, cg_adjoint=dom == "adjoint") * units_per_pass
    sm_max = clk.get("sm_max_mhz") or 2070.0
    props = torch.cuda.get_device_properties(torch.cuda.current_device())
    alu_derived = props.multi_processor_count * FP32_LANES_PER_SM * 2 * sm_max * 1e6 / 1e12
    measured_fp32 = [v for k, v in fp32_peak.items() if k in ("ffma", "ffma2")]
    alu_peak = max(measured_fp32) if measured_fp32 else alu_derived
    peaks, peak_src = measured_peaks()
    hbm_peak = float(peaks.get("hbm_gbs", FALLBACK_HBM_GBS))
    alu_ach = fl / (avg_ms / 1e3) / 1e12
    hbm_ach = by / (avg_ms / 1e3) / 1e9
    traffic = profiled_traffic(dom)
    alu = {"bound": "alu", "achieved": round(alu_ach, 3), "peak": round(alu_peak, 2), "unit": "TFLOP/s",
           "frac": round(alu_ach / alu_peak, 4),
           "peak_source": ("measured in this run (of measured): lsm_measure_fp32_peak, FMA-chain kernels on 8 "
                           "blocks of 256 threads per SM, best of 5 CUDA-event-timed launches, the faster of scalar "
                           f"FFMA {fp32_peak['ffma']:.2f} and paired FFMA2 {fp32_peak['ffma2']:.2f} TFLOP/s")
           if measured_fp32 else f"derived (measurement failed: {fp32_peak.get('error')}): "
                                 f"{props.multi_processor_count} SMs x {FP32_LANES_PER_SM} FP32 lanes x 2 x {sm_max:g} MHz",
           "peak_derived": round(alu_derived, 2),
           "peak_derived_source": f"{props.multi_processor_count} SMs x {FP32_LANES_PER_SM} FP32 lanes x 2 x "
                                  f"{sm_max:g} MHz"}
    hbm = {"bound": "hbm", "achieved": round(hbm_ach, 1), "peak": hbm_peak, "unit": "GB/s",
           "frac": round(hbm_ach / hbm_peak, 4), "peak_source": f"{peak_src} (MEASURED_PEAKS.json hbm_gbs)"
           if peak_src == "measured" else "fallback 6.8 TB/s (MEASURED_PEAKS.json absent)"}
    # the sweeps are bound by the FP32 pipe and its dependency latency (ncu: FMA pipe 54-57 % busy,
    # DRAM 35-40 %), so the FP32 roofline is the primary one and HBM the secondary
    primary, secondary = alu, hbm
    roofline = dict(primary)
    roofline["traffic"] = traffic
    roofline["kernel"] = f"{dom} sweep (sweep_kernel MODE_{dom.upper()}, nx={nx})"
    roofline["launch_ms"] = round(avg_ms, 4)
    roofline["algorithmic_per_unit"] = {"flop": flops_per_unit(nx),
                                        "bytes": bytes_per_unit(nx, ds.nrec, nz, K, cg_adjoint=dom == "adjoint")}
    roofline["units_per_launch"] = units_per_pass
    roofline["timed_launches"] = prof[dom]["launches"]  # the first window's, in each timed step
    roofline["secondary"] = secondary

    fwd_ms = prof["forward"]["ms"] / max(prof["forward"]["launches"], 1)
    adj_ms = prof["adjoint"]["ms"] / max(prof["adjoint"]["launches"], 1)
    operator = {"definition": "K*nw*nz / (t_A + t_AT) for one window application, mean event times in the "
                              "timed region",
                "value": round(units_per_pass / ((fwd_ms + adj_ms) / 1e3), 1), "unit": "units/s",
                "t_A_ms": round(fwd_ms, 4), "t_AT_ms": round(adj_ms, 4)}
    out = {"metric": METRIC,
           "value": round(value, 1), "unit": "units/s", "n_gpus": world, "steps": args.steps,
           "warmup": args.warmup, "ms_per_step": round(t_max / args.steps, 3), "higher_is_better": True,
           "scaling": "weak", "vs_baseline": None, "dtype": "f32", "data": "synthetic (seeded)",
           "config": workload_config(sv), "roofline": roofline, "operator": operator, "clocks": clk,
           "gpu_launches": int(launches),
           "autotune": tune,
           "kernel_ms": {k: round(v["ms"], 3) for k, v in prof.items() if k not in ("vector", "gradient")},
           "kernel_launches": {k: v["launches"] for k, v in prof.items() if k not in ("vector", "gradient")},
           "cg": {"windows": len(stats[-1]), "iters_per_window": iters, "total_iters": int(sum(iters)),
                  "max_final_rel_res": max(final_res), "time_to_tol_ms": round(t_max / args.steps, 3),
                  "loop": "first window host-driven, its A / A^T sweeps event-timed for the roofline; the "
                          "other windows resumed from its image with the default loop (CUDA graph per window)"}}

    # end to end through the public API with host buffers; nothing is event-timed here, so the solve
    # runs the library's default loop, each window's CG iterations as one CUDA graph
    if not args.no_e2e:
        d_host = d.cpu().pin_memory()
        s_host = torch.as_tensor(s32).pin_memory()
        img_host = torch.empty((nz, nx), dtype=torch.float32).pin_memory()
        d_dev = torch.empty_like(d)
        s_dev = torch.empty_like(ds.slowness)
        barrier()
        torch.cuda.synchronize()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        stats_e = []
        for _ in range(args.steps):
            d_dev.copy_(d_host, non_blocking=True)
            s_dev.copy_(s_host, non_blocking=True)
            m.zero_()
            _, st = L.rls_window_solve(ds.grid, s_dev, ds.freqs, ds.geom, d_dev, lam, K, sv.slide, sv.cg_tol,
                                       sv.cg_iters, m, ws)
            img_host.copy_(m, non_blocking=True)
            stats_e.append(st)
        e1.record(stream)
        torch.cuda.synchronize()
        te = e0.elapsed_time(e1)
        units_e = sum((w["n_forward"] + w["n_adjoint"]) / 2 * units_per_pass for st in stats_e for w in st)
        units_e_all, te = reduce_over_ranks(units_e, te, world, "cuda")
        out["e2e"] = {"value": round(units_e_all / (te / 1e3), 1), "unit": "units/s",
                      "h2d_bytes_per_step": int(d_host.numel() * 8 + s_host.numel() * 4),
                      "d2h_bytes_per_step": int(img_host.numel() * 4), "ms_per_step": round(te / args.steps, 3),
                      "cg_loop": "CUDA graph (library default)"}

    # the paper's preconditioned variant (illumination preconditioner), one untimed-by-contract solve
    if not args.no_variants:
        torch.cuda.synchronize()
        v0, v1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        tvs = []
        for rep in range(2):  # the first call also pays the first launches of the preconditioner kernels
            m.zero_()
            torch.cuda.synchronize()
            v0.record(stream)
            _, stv = L.rls_window_solve(ds.grid, ds.slowness, ds.freqs, ds.geom, d, lam, K, sv.slide, sv.cg_tol,
                                        sv.cg_iters, m, ws, preconditioner="illumination", precond_eps=1e-2)
            v1.record(stream)
            torch.cuda.synchronize()
            tvs.append(v0.elapsed_time(v1))
        tv = tvs[-1]
        out["variants"] = {"illumination_preconditioned": {
            "time_to_tol_ms": round(tv, 3), "time_to_tol_ms_per_call": [round(x, 3) for x in tvs],
            "total_iters": int(sum(w["iters"] for w in stv)),
            "iters_per_window": [w["iters"] for w in stv],
            "time_to_tol_vs_plain": round((t_max / args.steps) / tv, 3)}}
        # the plain solve with each window's CG iterations replayed as one CUDA graph (conditional
        # WHILE node, stopping test on the device): same kernels, one host wait per window
        tg = []
        for rep in range(2):  # the first call also builds and instantiates its graph; both are timed
            m.zero_()
            torch.cuda.synchronize()
            v0.record(stream)
            _, stg = L.rls_window_solve(ds.grid, ds.slowness, ds.freqs, ds.geom, d, lam, K, sv.slide, sv.cg_tol,
                                        sv.cg_iters, m, ws, cuda_graph=True)
            v1.record(stream)
            torch.cuda.synchronize()
            tg.append(v0.elapsed_time(v1))
        out["variants"]["cuda_graph"] = {
            "time_to_tol_ms": round(tg[-1], 3), "time_to_tol_ms_per_call": [round(x, 3) for x in tg],
            "total_iters": int(sum(w["iters"] for w in stg)),
            "same_iterations_as_plain": [w["iters"] for w in stg] == iters,
            "time_to_tol_vs_plain": round((t_max / args.steps) / tg[-1], 3)}
        # the whole solve (every window's set-up and CG loop) as one graph launch
        ts = []
        for rep in range(2):  # each call captures and instantiates its graph; both are timed
            m.zero_()
            torch.cuda.synchronize()
            v0.record(stream)
            _, sts = L.rls_window_solve(ds.grid, ds.slowness, ds.freqs, ds.geom, d, lam, K, sv.slide, sv.cg_tol,
                                        sv.cg_iters, m, ws, cuda_graph="solve")
            v1.record(stream)
            torch.cuda.synchronize()
            ts.append(v0.elapsed_time(v1))
        out["variants"]["cuda_graph_whole_solve"] = {
            "time_to_tol_ms": round(ts[-1], 3), "time_to_tol_ms_per_call": [round(x, 3) for x in ts],
            "total_iters": int(sum(w["iters"] for w in sts)),
            "same_iterations_as_plain": [w["iters"] for w in sts] == iters,
            "time_to_tol_vs_plain": round((t_max / args.steps) / ts[-1], 3)}
        # the lateral transforms on the tensor cores (split FP16 / BF16 three-term DFT products),
        # every window to the same 1e-3 stopping threshold as the plain FP32 solve
        ref_norm = float(torch.linalg.vector_norm(m_fp32))
        out["variants"]["tensor_core_transforms"] = {}
        kernels = {"dft_fp16x3": "mma.sync four-step DFT products (lsm_tc.cuh)",
                   "dft_bf16x3": "mma.sync four-step DFT products (lsm_tc.cuh)",
                   "dft_fp16x3_tcgen05": "tcgen05.mma four-step DFT products, TMEM accumulators (lsm_tc5.cuh)",
                   "dft_bf16x3_tcgen05": "tcgen05.mma four-step DFT products, TMEM accumulators (lsm_tc5.cuh)"}
        # per-launch times of the window's sweeps with every transform (3 event-timed launches each,
        # after one untimed; the plain FFT sweeps for comparison)
        sweeps = ("source", "adjoint", "forward")
        rep = L.lsm_autotune(ds.grid, ds.slowness, ds.freqs, ds.geom, K, ws)
        sweep_ms = {"fft": {k: round(rep[k]["ms"], 4) for k in sweeps}}
        sweep_ms["fft"]["points_per_thread"] = rep["tile"]["points_per_thread"]
        for transform in kernels:
            rep = L.lsm_autotune(ds.grid, ds.slowness, ds.freqs, ds.geom, K, ws, transform=transform)
            sweep_ms[transform] = {k: round(rep[k]["ms"], 4) for k in sweeps}
        torch.cuda.synchronize()
        out["variants"]["sweep_launch_ms_by_transform"] = sweep_ms
        out["variants"]["sweep_launch_ms_by_transform_precision_1024"] = precision_sweeps_variant(L, torch, kernels)
        for transform in kernels:
            m.zero_()
            torch.cuda.synchronize()
            v0.record(stream)
            _, stt = L.rls_window_solve(ds.grid, ds.slowness, ds.freqs, ds.geom, d, lam, K, sv.slide, sv.cg_tol,
                                        sv.cg_iters, m, ws, transform=transform)
            v1.record(stream)
            torch.cuda.synchronize()
            tt = v0.elapsed_time(v1)
            out["variants"]["tensor_core_transforms"][transform] = {
                "time_to_tol_ms": round(tt, 3), "total_iters": int(sum(w["iters"] for w in stt)),
                "iters_per_window": [w["iters"] for w in stt],
                "max_final_rel_res": max(w["rel_res"] for w in stt),
                "image_rel_l2_vs_fp32_solve": float(torch.linalg.vector_norm(m - m_fp32)) / ref_norm,
                "time_to_tol_vs_plain": round((t_max / args.steps) / tt, 3),
                "kernel": kernels[transform]}
        if world == 1:
            out["variants"]["batching_reduced"] = batching_reduced_variant(L, torch, args)

    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        cb = cpu_baseline(sv, args.ref_sample_freqs)
        # the oracle's time to the same residual, extrapolated from its measured rate over the GPU
        # solve's A + A^T units (every window to 1e-3)
        units_per_solve = out["value"] * out["ms_per_step"] / 1e3
        cb["time_to_tol_extrapolated_s"] = round(units_per_solve / cb["value"], 1)
        cb["time_to_tol_note"] = ("extrapolated, not measured: the GPU solve's A + A^T units at the oracle's "
                                  "measured rate")
        out["cpu_baseline"] = cb
    if world > 1:
        import torch.distributed as dist
        dist.barrier()
        dist.destroy_process_group()
    if rank == 0:
        print(json.dumps(out), flush=True)


# ------------------------------------------------------------------ oracle (CPU) arm


def oracle_sample(sv, n_freqs, n_shots=1):
    """One A + A^T of the FP64 oracle on n_shots shots from shot 40 (or the middle shot) and the
    first n_freqs frequencies, at the workload's full grid; returns (units, seconds)."""
    import numpy as np

    from oracle import lsm_oracle as O

    op = O.SplitStepOperator(sv.slowness, sv.dx, sv.dz, sv.freqs, sv.wavelet, sv.src_ix, sv.rec_ix)
    sub = op.with_freqs(np.arange(min(n_freqs, sv.nw)))
    shot = min(40, sv.ns // 2)
    shots = list(range(shot, min(sv.ns, shot + n_shots)))
    t0 = time.perf_counter()
    dd = sub.forward(sv.reflectivity, shots=shots)
    sub.adjoint(dd, shots=shots)
    dt = time.perf_counter() - t0
    return len(shots) * sub.nw * sv.nz, dt


def host_cores():
    try:
        return len(os.sched_getaffinity(0))
    except AttributeError:  # pragma: no cover
        return os.cpu_count()


def sample_text(sv, n_freqs):
    return (f"one A + A^T of the FP64 oracle (numpy, naive DFT matrices) on 1 shot x {min(n_freqs, sv.nw)} "
            f"frequencies x {sv.nz} depths at {sv.nx} columns of the workload = {min(n_freqs, sv.nw) * sv.nz} units")


def cpu_baseline(sv, n_freqs, min_seconds=10.0):
    """The oracle on the same bounded sample as the reference arm's steps, repeated until at least
    min_seconds of host time (after one untimed repetition)."""
    oracle_sample(sv, n_freqs)
    units, secs, reps = 0, 0.0, 0
    while secs < min_seconds or reps < 3:
        u, dt = oracle_sample(sv, n_freqs)
        units += u
        secs += dt
        reps += 1
    return {"value": round(units / secs, 2), "unit": "units/s", "cores": host_cores(), "kind": "oracle",
            "sample": f"{sample_text(sv, n_freqs)}, repeated {reps} times ({secs:.1f} s)"}


def reference_arm(args):
    rank, world, _ = dist_info()
    if rank != 0:
        return
    sv = workload(args.workload, 0)
    for _ in range(args.warmup):
        oracle_sample(sv, args.ref_sample_freqs)
    units_total, t_total = 0, 0.0
    for _ in range(args.steps):
        u, dt = oracle_sample(sv, args.ref_sample_freqs)
        units_total += u
        t_total += dt
    value = units_total / t_total
    base = {"value": round(value, 2), "unit": "units/s", "cores": host_cores(), "kind": "oracle",
            "sample": f"each step: {sample_text(sv, args.ref_sample_freqs)}"}
    out = {"impl": "reference", "metric": METRIC,
           "value": round(value, 2), "unit": "units/s", "n_gpus": world, "steps": args.steps,
           "warmup": args.warmup, "ms_per_step": round(1e3 * t_total / args.steps, 3), "higher_is_better": True,
           "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic (seeded)",
           "config": workload_config(sv), "cpu_baseline": base,
           "e2e": {"value": round(value, 2), "unit": "units/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(out), flush=True)


def build_line(L, lsm, torch, sv):
    """One survey line on the device: data d = A m + noise modelled with the library, lambda =
    1e-3 max|A^T d|, a solve workspace, a zero image and a stream of its own."""
    import numpy as np

    from paper_1801_00819_gb300.device import to_device, workspace

    ds = to_device(sv.nx, sv.nz, sv.dx, sv.dz, sv.slowness, sv.src_ix, sv.rec_ix, sv.freqs, sv.wavelet)
    K = sv.window
    m_true = torch.as_tensor(np.asarray(sv.reflectivity, dtype=np.float32), device="cuda")
    d = torch.empty((sv.ns, sv.nw, ds.nrec), dtype=torch.complex64, device="cuda")
    ws_f = workspace(L.lsm_workspace_bytes(ds.grid, ds.geom, ds.freqs, K, L.LSM_OP_ADJOINT))
    for s0 in range(0, sv.ns, K):
        n = min(K, sv.ns - s0)
        L.lsm_forward(ds.grid, ds.slowness, ds.freqs, ds.geom, m_true, d[s0:s0 + n], s0, n, ws_f)
    rms = float(torch.sqrt(torch.mean(torch.abs(d) ** 2)))
    d += sv.noise_pct * rms * torch.as_tensor(sv.noise().astype(np.complex64), device="cuda")
    adj = torch.zeros((sv.nz, sv.nx), dtype=torch.float32, device="cuda")
    for s0 in range(0, sv.ns, K):
        n = min(K, sv.ns - s0)
        L.lsm_adjoint(ds.grid, ds.slowness, ds.freqs, ds.geom, d[s0:s0 + n], adj, s0, n, ws_f, accumulate=True)
    lam = 1e-3 * float(adj.abs().max())
    del ws_f
    ws = workspace(L.lsm_workspace_bytes(ds.grid, ds.geom, ds.freqs, K, L.LSM_OP_SOLVE))
    m = torch.zeros((sv.nz, sv.nx), dtype=torch.float32, device="cuda")
    return lsm.LineProblem(ds.grid, ds.slowness, ds.freqs, ds.geom, d, lam, K, sv.slide, sv.cg_tol, sv.cg_iters, m,
                           ws, torch.cuda.Stream())


def tune_lines(lsm, lines):
    """Launch shapes of every line's window (K shots) and refill (slide shots) sweeps."""
    tuned = []
    for pr in lines:
        rep = lsm.lsm_autotune(pr.grid, pr.slowness, pr.freqs, pr.geom, pr.K, pr.workspace)
        sweeps = ("source", "adjoint", "forward")
        entry = {"nx": pr.grid.c.nx, "K": pr.K, "warps": {k: rep[k]["warps"] for k in sweeps},
                 "heuristic_warps": {k: rep[k]["heuristic_warps"] for k in sweeps},
                 "points_per_thread": rep["tile"]["points_per_thread"],
                 "default_points_per_thread": rep["tile"]["default_points_per_thread"]}
        if pr.slide != pr.K:
            entry["refill_source_warps"] = lsm.lsm_autotune(pr.grid, pr.slowness, pr.freqs, pr.geom, pr.slide,
                                                            pr.workspace)["source"]["warps"]
        tuned.append(entry)
    return tuned


def line_units(lines, stats_per_line):
    total = 0
    for pr, st in zip(lines, stats_per_line):
        per_pass = pr.K * pr.freqs.c.nw * pr.grid.c.nz
        total += sum((w["n_forward"] + w["n_adjoint"]) / 2 * per_pass for w in st)
    return total


def precision_sweeps_variant(L, torch, transforms):
    """Per-launch times of the sweeps of one window of the precision workload (1024 x 512, 256
    frequencies 3-60 Hz, 4 shots: 1,024 items) with the FP32 FFT and every tensor-core transform
    (lsm_autotune's report: 3 event-timed launches each after one untimed)."""
    from paper_1801_00819_gb300.device import to_device, workspace
    from synth import config_precision

    sv = config_precision()
    K = 4
    ds = to_device(sv.nx, sv.nz, sv.dx, sv.dz, sv.slowness, sv.src_ix, sv.rec_ix, sv.freqs, sv.wavelet)
    ws = workspace(L.lsm_workspace_bytes(ds.grid, ds.geom, ds.freqs, K, L.LSM_OP_SOLVE))
    out = {"workload": f"{sv.nx} x {sv.nz}, {K} shots x {sv.nw} frequencies"}
    for transform in ["fft"] + list(transforms):
        rep = L.lsm_autotune(ds.grid, ds.slowness, ds.freqs, ds.geom, K, ws, transform=transform)
        out[transform] = {k: round(rep[k]["ms"], 4) for k in ("source", "adjoint", "forward")}
    torch.cuda.synchronize()
    del ws
    return out


def batching_reduced_variant(L, torch, args):
    """The eight-line batching workload cut to each line's first three windows and every other
    frequency: every window of every line to 1e-3, solved line after line with the plain FP32 solve
    (the library's default loop) and all lines together (rls_multi_line_solve: one host worker and
    stream per line).  Host wall clock around each whole solve, the GPU synchronised on both sides;
    best of two runs each."""
    from paper_1801_00819_gb300 import lsm
    from synth import config_batching_lines_reduced

    lines = [build_line(L, lsm, torch, sv) for sv in config_batching_lines_reduced()]
    torch.cuda.synchronize()
    tuned = tune_lines(lsm, lines) if not args.no_autotune else None
    torch.cuda.synchronize()

    def looped():
        out = []
        for pr in lines:
            pr.m_inout.zero_()
            _, st = L.rls_window_solve(pr.grid, pr.slowness, pr.freqs, pr.geom, pr.d, pr.lam, pr.K, pr.slide,
                                       pr.cg_tol, pr.max_iter, pr.m_inout, pr.workspace)
            out.append(st)
        return out

    def together():
        for pr in lines:
            pr.m_inout.zero_()
        torch.cuda.synchronize()
        return lsm.rls_multi_line_solve(lines)[1]

    def one_graph():
        for pr in lines:
            pr.m_inout.zero_()
        torch.cuda.synchronize()
        return lsm.rls_multi_line_solve(lines, cuda_graph="solve")[1]

    def timed(fn):
        best, stats = None, None
        for _ in range(2):
            torch.cuda.synchronize()
            t0 = time.perf_counter()
            st = fn()
            torch.cuda.synchronize()
            dt = time.perf_counter() - t0
            if best is None or dt < best:
                best, stats = dt, st
        return best, stats

    together()  # first launches and graph instantiations outside the timing
    t_loop, st_loop = timed(looped)
    imgs_loop = [pr.m_inout.clone() for pr in lines]
    t_tog, st_tog = timed(together)
    same = all(torch.equal(a, pr.m_inout) for a, pr in zip(imgs_loop, lines))
    one_graph()
    t_one, st_one = timed(one_graph)
    same_one = all(torch.equal(a, pr.m_inout) for a, pr in zip(imgs_loop, lines))
    out = {"workload": "batching (reduced): the 8 lines nx 256-1024 (incl. 384, 640, 768, 896), nz = nx/2, "
                       "each line's first 3 windows of K 4-32 shots, every other frequency (52-91), CG to 1e-3",
           "lines": [{"nx": pr.grid.c.nx, "shots": pr.geom.c.ns, "freqs": pr.freqs.c.nw, "K": pr.K,
                      "slide": pr.slide, "iters": int(sum(w["iters"] for w in st))}
                     for pr, st in zip(lines, st_tog)],
           "looped_ms": round(1e3 * t_loop, 1), "together_ms": round(1e3 * t_tog, 1),
           "speedup_together_vs_looped": round(t_loop / t_tog, 3),
           "units_per_s_together": round(line_units(lines, st_tog) / t_tog, 1),
           "units_per_s_looped": round(line_units(lines, st_loop) / t_loop, 1),
           "max_final_rel_res": max(w["rel_res"] for st in st_tog for w in st),
           "images_bitwise_equal": bool(same),
           "one_graph_ms": round(1e3 * t_one, 1),
           "speedup_one_graph_vs_looped": round(t_loop / t_one, 3),
           "one_graph_images_bitwise_equal": bool(same_one),
           "one_graph": "every window of every line in one CUDA graph launch (cuda_graph=\"solve\"): the "
                        "lines as independent branches, each window's CG iterations a conditional WHILE node; "
                        "graph capture and instantiation inside the timed call",
           "timing": "host wall clock around each whole solve, GPU synchronised on both sides, best of 2",
           "autotune": tuned}
    del lines
    torch.cuda.empty_cache()
    return out


def batching_arm(args):
    """Eight independent survey lines (nx 256..1024 incl. 384, 640, 768, 896; K 4..32), every window
    to 1e-3: one step solves all lines concurrently (rls_multi_line_solve, a stream per line); the
    comparison loops the plain per-line solve over the same lines.  Both run the host-driven CG loop;
    a third arm runs the concurrent solve with graph-replayed CG iterations, a fourth every window of
    every line as one graph launch."""
    import torch

    import paper_1801_00819_gb300 as L
    from paper_1801_00819_gb300 import build as B
    from paper_1801_00819_gb300 import lsm
    from synth import config_batching_lines

    torch.cuda.set_device(0)
    B.build()
    lines = [build_line(L, lsm, torch, sv) for sv in config_batching_lines()]
    torch.cuda.synchronize()
    tuned = []
    if not args.no_autotune:  # launch shapes per line, before any timed solve
        tuned = tune_lines(lsm, lines)
        torch.cuda.synchronize()

    def units_of(stats_per_line):
        return line_units(lines, stats_per_line)

    def sequential():
        out = []
        for pr in lines:
            pr.m_inout.zero_()
            _, st = L.rls_window_solve(pr.grid, pr.slowness, pr.freqs, pr.geom, pr.d, pr.lam, pr.K, pr.slide,
                                       pr.cg_tol, pr.max_iter, pr.m_inout, pr.workspace, cuda_graph=False)
            out.append(st)
        return out

    def concurrent(graph=False):
        for pr in lines:
            pr.m_inout.zero_()
        torch.cuda.synchronize()
        _, st = lsm.rls_multi_line_solve(lines, cuda_graph=graph)
        return st

    for _ in range(max(args.warmup, 1)):
        concurrent()
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    st_conc = [concurrent() for _ in range(args.steps)][-1]
    torch.cuda.synchronize()
    t_conc = (time.perf_counter() - t0) / args.steps
    # the same concurrent solve with each window's CG iterations replayed as a CUDA graph
    concurrent(graph=True)
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    st_graph = [concurrent(graph=True) for _ in range(args.steps)][-1]
    torch.cuda.synchronize()
    t_graph = (time.perf_counter() - t0) / args.steps
    # every window of every line as one graph launch (no host worker threads)
    concurrent(graph="solve")
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    st_one = [concurrent(graph="solve") for _ in range(args.steps)][-1]
    torch.cuda.synchronize()
    t_one = (time.perf_counter() - t0) / args.steps
    t0 = time.perf_counter()
    st_seq = sequential()
    torch.cuda.synchronize()
    t_seq = time.perf_counter() - t0
    units = units_of(st_conc)
    out = {"metric": "shot*omega*depth steps/s for A+A^T (eight-line batched window-RLS solve to 1e-3)",
           "value": round(units / t_conc, 1), "unit": "units/s", "n_gpus": 1, "steps": args.steps,
           "warmup": args.warmup, "ms_per_step": round(1e3 * t_conc, 1), "higher_is_better": True,
           "scaling": "weak", "vs_baseline": None, "dtype": "f32", "data": "synthetic (seeded)",
           "config": {"workload": "batching: 8 lines nx 256-1024 (incl. 384, 640, 768, 896), nz = nx/2, shots 64-200, "
                                  "freqs 96-192, K 4-32, slide ceil(K/2), CG to 1e-3",
                      "lines": [{"nx": pr.grid.c.nx, "shots": pr.geom.c.ns, "freqs": pr.freqs.c.nw, "K": pr.K,
                                 "slide": pr.slide,
                                 "iters": int(sum(w["iters"] for w in st))} for pr, st in zip(lines, st_conc)]},
           "timing": "host wall clock around each whole solve, GPU synchronised on both sides",
           "sequential_ms": round(1e3 * t_seq, 1), "concurrent_ms": round(1e3 * t_conc, 1),
           "speedup_concurrent_vs_sequential": round(t_seq / t_conc, 3),
           "sequential_units_per_s": round(units_of(st_seq) / t_seq, 1),
           "concurrent_cuda_graph_ms": round(1e3 * t_graph, 1),
           "concurrent_cuda_graph_units_per_s": round(units_of(st_graph) / t_graph, 1),
           "speedup_concurrent_cuda_graph_vs_sequential": round(t_seq / t_graph, 3),
           "cuda_graph_same_iterations": [[w["iters"] for w in st] for st in st_graph] ==
                                         [[w["iters"] for w in st] for st in st_conc],
           "one_graph_ms": round(1e3 * t_one, 1),
           "one_graph_units_per_s": round(units_of(st_one) / t_one, 1),
           "speedup_one_graph_vs_sequential": round(t_seq / t_one, 3),
           "one_graph_same_iterations": [[w["iters"] for w in st] for st in st_one] ==
                                        [[w["iters"] for w in st] for st in st_conc],
           "autotune": tuned or None}
    print(json.dumps(out), flush=True)


def main():
    args = parse_args()
    if args.impl == "reference":
        reference_arm(args)
    elif args.workload == "batching":
        batching_arm(args)
    else:
        gpu_arm(args)


if __name__ == "__main__":
    main()
