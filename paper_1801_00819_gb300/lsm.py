"""Python binding of the C ABI in include/lsm.h (argument marshalling only).

Every entry point has the C name and forwards to liblsm_gb300.so through ctypes; all arithmetic
runs in that library's CUDA kernels.  Device arrays are torch CUDA tensors (or raw integer
device addresses); host geometry and frequency arrays are numpy arrays.  There is no CPU
fallback: if the library has not been built, loading it raises.
"""

from __future__ import annotations

import ctypes
import os

import numpy as np

_PKG = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_PKG, "liblsm_gb300.so")

LSM_OK = 0
LSM_ERR_ARG = -1
LSM_ERR_CUDA = -2
LSM_ERR_WORKSPACE = -3
LSM_ERR_BREAKDOWN = -4
LSM_ERR_TIMEOUT = -5
LSM_ERR_UNSUPPORTED_NX = -6

LSM_OP_FORWARD = 0
LSM_OP_ADJOINT = 1
LSM_OP_SOLVE = 2
LSM_OP_GRADIENT = 3
LSM_CHECKPOINT_EVERY = 16

EXPORTED = ("lsm_workspace_bytes", "lsm_forward", "lsm_adjoint", "lsm_num_windows", "rls_window_solve",
            "lsm_status_string", "lsm_kernel_launches", "lsm_profile_start", "lsm_profile_stop",
            "lsm_adjoint_static", "lsm_born_gradient", "rls_window_solve_ex", "rls_multi_line_solve",
            "lsm_forward_ex", "lsm_adjoint_ex", "lsm_profile_start_classes", "lsm_autotune",
            "lsm_autotune_reset", "lsm_autotune_gradient", "lsm_measure_fp32_peak",
            "lsm_check_bounded_wait", "rls_window_solve_sharded", "lsm_fft_tiles", "lsm_set_fft_tile", "lsm_tcgen05_shape")

TRANSFORMS = {"fft": 0, "dft_bf16x3": 1, "dft_fp16x3": 2, "dft_bf16x1": 3, "dft_fp16x3_tcgen05": 4,
              "dft_bf16x3_tcgen05": 5}

LSM_PRECOND_NONE = 0
LSM_PRECOND_ILLUMINATION = 1
LSM_CUDA_GRAPH_WINDOW = 1
LSM_CUDA_GRAPH_SOLVE = 2

LSM_STATIC_SCRATCH_BYTES = 64 << 20

KERNEL_CLASSES = ("tables", "source", "adjoint", "forward", "vector", "gradient")


class LsmError(RuntimeError):
    def __init__(self, status: int, where: str):
        self.status = status
        super().__init__(f"{where}: {lsm_status_string(status)} ({status})")


class lsm_grid(ctypes.Structure):
    _fields_ = [("nx", ctypes.c_int), ("nz", ctypes.c_int), ("dx", ctypes.c_float), ("dz", ctypes.c_float)]


class lsm_geom(ctypes.Structure):
    _fields_ = [("ns", ctypes.c_int), ("src_ix", ctypes.POINTER(ctypes.c_int)), ("nrec", ctypes.c_int),
                ("rec_ix", ctypes.POINTER(ctypes.c_int))]


class lsm_freqs(ctypes.Structure):
    _fields_ = [("nw", ctypes.c_int), ("freq_hz", ctypes.POINTER(ctypes.c_float)),
                ("wavelet", ctypes.POINTER(ctypes.c_float))]


class lsm_solve_options(ctypes.Structure):
    _fields_ = [("preconditioner", ctypes.c_int), ("precond_eps", ctypes.c_double), ("transform", ctypes.c_int),
                ("cuda_graph", ctypes.c_int)]


def _options(preconditioner=None, precond_eps=1e-2, transform="fft", cuda_graph=None):
    if transform not in TRANSFORMS:
        raise ValueError(f"unknown transform {transform!r}")
    if preconditioner is None:
        pc = LSM_PRECOND_NONE
    elif preconditioner == "illumination":
        pc = LSM_PRECOND_ILLUMINATION
    else:
        raise ValueError(f"unknown preconditioner {preconditioner!r}")
    # None: the library's default; True: one graph per window's CG iterations; "solve": the whole
    # call as one graph launch; False: the host-driven loop
    if cuda_graph is None:
        graph = 0
    elif cuda_graph == "solve":
        graph = LSM_CUDA_GRAPH_SOLVE
    elif cuda_graph is True or cuda_graph == "window":
        graph = LSM_CUDA_GRAPH_WINDOW
    elif cuda_graph is False:
        graph = -1
    else:
        raise ValueError(f"unknown cuda_graph {cuda_graph!r}")
    return lsm_solve_options(pc, float(precond_eps), TRANSFORMS[transform], graph)


class lsm_line(ctypes.Structure):
    pass  # fields assigned after lsm_window_stats


class lsm_window_stats(ctypes.Structure):
    _fields_ = [("start", ctypes.c_int), ("iters", ctypes.c_int), ("rel_res0", ctypes.c_double),
                ("rel_res", ctypes.c_double), ("n_forward", ctypes.c_int), ("n_adjoint", ctypes.c_int),
                ("ms", ctypes.c_float)]

    def as_dict(self):
        return {k: getattr(self, k) for k, _ in self._fields_}


lsm_line._fields_ = [("grid", lsm_grid), ("slowness", ctypes.c_void_p), ("freqs", lsm_freqs), ("geom", lsm_geom),
                     ("d", ctypes.c_void_p), ("lambda_", ctypes.c_double), ("K", ctypes.c_int),
                     ("slide", ctypes.c_int), ("cg_tol", ctypes.c_double), ("max_iter", ctypes.c_int),
                     ("m_inout", ctypes.c_void_p), ("stats", ctypes.POINTER(lsm_window_stats)),
                     ("stats_cap", ctypes.c_int), ("workspace", ctypes.c_void_p), ("workspace_bytes", ctypes.c_size_t),
                     ("stream", ctypes.c_void_p), ("status", ctypes.c_int)]


class lsm_profile(ctypes.Structure):
    _fields_ = [("launches", ctypes.c_ulonglong * 6), ("ms", ctypes.c_double * 6)]


class lsm_tune_entry(ctypes.Structure):
    _fields_ = [("warps", ctypes.c_int), ("heuristic_warps", ctypes.c_int), ("candidates", ctypes.c_int),
                ("ms", ctypes.c_double), ("heuristic_ms", ctypes.c_double)]

    def as_dict(self):
        return {"warps": int(self.warps), "heuristic_warps": int(self.heuristic_warps),
                "candidates": int(self.candidates), "ms": float(self.ms), "heuristic_ms": float(self.heuristic_ms)}


class lsm_tune_report(ctypes.Structure):
    _fields_ = [("source", lsm_tune_entry), ("adjoint", lsm_tune_entry), ("forward", lsm_tune_entry),
                ("points_per_thread", ctypes.c_int), ("default_points_per_thread", ctypes.c_int),
                ("tiles", ctypes.c_int), ("tile_ms", ctypes.c_double), ("default_tile_ms", ctypes.c_double)]


class lsm_ckpt_tune_report(ctypes.Structure):
    _fields_ = [("stride", ctypes.c_int), ("default_stride", ctypes.c_int), ("warps", ctypes.c_int),
                ("default_warps", ctypes.c_int), ("candidates", ctypes.c_int), ("ms", ctypes.c_double),
                ("default_ms", ctypes.c_double)]


# int allreduce(void* ctx, void* buf, size_t count, int is_double, void* stream)
ALLREDUCE_FN = ctypes.CFUNCTYPE(ctypes.c_int, ctypes.c_void_p, ctypes.c_void_p, ctypes.c_size_t, ctypes.c_int,
                                ctypes.c_void_p)

_lib_handle = None


def load_library(path: str = LIB_PATH) -> ctypes.CDLL:
    """Load liblsm_gb300.so (built by paper_1801_00819_gb300.build); raises if it is missing."""
    global _lib_handle
    if _lib_handle is not None:
        return _lib_handle
    if not os.path.exists(path):
        raise RuntimeError(f"{path} is missing: build it with `python -m paper_1801_00819_gb300.build` "
                           "(there is no CPU fallback)")
    try:  # share the CUDA runtime that torch has already loaded, if any
        import torch  # noqa: F401
    except Exception:  # pragma: no cover
        pass
    lib = ctypes.CDLL(path)
    P = ctypes.c_void_p
    lib.lsm_workspace_bytes.restype = ctypes.c_size_t
    lib.lsm_workspace_bytes.argtypes = [ctypes.POINTER(lsm_grid), ctypes.POINTER(lsm_geom),
                                        ctypes.POINTER(lsm_freqs), ctypes.c_int, ctypes.c_int]
    lib.lsm_forward.restype = ctypes.c_int
    lib.lsm_forward.argtypes = [ctypes.POINTER(lsm_grid), P, ctypes.POINTER(lsm_freqs), ctypes.POINTER(lsm_geom),
                                P, P, ctypes.c_int, ctypes.c_int, P, ctypes.c_size_t, P]
    lib.lsm_adjoint.restype = ctypes.c_int
    lib.lsm_adjoint.argtypes = [ctypes.POINTER(lsm_grid), P, ctypes.POINTER(lsm_freqs), ctypes.POINTER(lsm_geom),
                                P, P, ctypes.c_int, ctypes.c_int, ctypes.c_int, P, ctypes.c_size_t, P]
    lib.lsm_adjoint_static.restype = ctypes.c_int
    lib.lsm_adjoint_static.argtypes = [ctypes.POINTER(lsm_grid), P, ctypes.POINTER(lsm_freqs),
                                       ctypes.POINTER(lsm_geom), P, P, ctypes.c_int, ctypes.c_int, ctypes.c_int, P]
    lib.lsm_born_gradient.restype = ctypes.c_int
    lib.lsm_born_gradient.argtypes = [ctypes.POINTER(lsm_grid), P, P, ctypes.POINTER(lsm_freqs),
                                      ctypes.POINTER(lsm_geom), P, P, P, P, P, ctypes.c_int, ctypes.c_int, P,
                                      ctypes.c_size_t, P]
    lib.lsm_forward_ex.restype = ctypes.c_int
    lib.lsm_forward_ex.argtypes = list(lib.lsm_forward.argtypes) + [ctypes.POINTER(lsm_solve_options)]
    lib.lsm_adjoint_ex.restype = ctypes.c_int
    lib.lsm_adjoint_ex.argtypes = list(lib.lsm_adjoint.argtypes) + [ctypes.POINTER(lsm_solve_options)]
    lib.lsm_num_windows.restype = ctypes.c_int
    lib.lsm_num_windows.argtypes = [ctypes.c_int, ctypes.c_int, ctypes.c_int]
    lib.rls_window_solve.restype = ctypes.c_int
    lib.rls_window_solve.argtypes = [ctypes.POINTER(lsm_grid), P, ctypes.POINTER(lsm_freqs),
                                     ctypes.POINTER(lsm_geom), P, ctypes.c_double, ctypes.c_int, ctypes.c_int,
                                     ctypes.c_double, ctypes.c_int, ctypes.c_int, ctypes.c_int, P,
                                     ctypes.POINTER(lsm_window_stats), ctypes.c_int, P, ctypes.c_size_t, P]
    lib.rls_window_solve_ex.restype = ctypes.c_int
    lib.rls_window_solve_ex.argtypes = list(lib.rls_window_solve.argtypes) + [ctypes.POINTER(lsm_solve_options)]
    lib.rls_window_solve_sharded.restype = ctypes.c_int
    lib.rls_window_solve_sharded.argtypes = list(lib.rls_window_solve.argtypes) + [ALLREDUCE_FN, ctypes.c_void_p]
    lib.rls_multi_line_solve.restype = ctypes.c_int
    lib.rls_multi_line_solve.argtypes = [ctypes.POINTER(lsm_line), ctypes.c_int, ctypes.POINTER(lsm_solve_options)]
    lib.lsm_autotune.restype = ctypes.c_int
    lib.lsm_autotune.argtypes = [ctypes.POINTER(lsm_grid), ctypes.c_void_p, ctypes.POINTER(lsm_freqs),
                                 ctypes.POINTER(lsm_geom), ctypes.c_int, ctypes.POINTER(lsm_solve_options),
                                 ctypes.c_void_p, ctypes.c_size_t, ctypes.c_void_p, ctypes.POINTER(lsm_tune_report)]
    lib.lsm_autotune_gradient.restype = ctypes.c_int
    lib.lsm_autotune_gradient.argtypes = [ctypes.POINTER(lsm_grid), ctypes.c_void_p, ctypes.POINTER(lsm_freqs),
                                          ctypes.POINTER(lsm_geom), ctypes.c_int, ctypes.c_void_p, ctypes.c_size_t,
                                          ctypes.c_void_p, ctypes.POINTER(lsm_ckpt_tune_report)]
    lib.lsm_fft_tiles.restype = ctypes.c_int
    lib.lsm_fft_tiles.argtypes = [ctypes.c_int, ctypes.POINTER(ctypes.c_int), ctypes.c_int]
    lib.lsm_set_fft_tile.restype = ctypes.c_int
    lib.lsm_set_fft_tile.argtypes = [ctypes.c_int, ctypes.c_int, ctypes.c_int, ctypes.c_int]
    lib.lsm_tcgen05_shape.restype = ctypes.c_int
    lib.lsm_tcgen05_shape.argtypes = [ctypes.c_int, ctypes.c_int, ctypes.c_int] + \
        [ctypes.POINTER(ctypes.c_int)] * 4 + [ctypes.POINTER(ctypes.c_size_t)]
    lib.lsm_autotune_reset.restype = None
    lib.lsm_autotune_reset.argtypes = []
    lib.lsm_status_string.restype = ctypes.c_char_p
    lib.lsm_status_string.argtypes = [ctypes.c_int]
    lib.lsm_kernel_launches.restype = ctypes.c_ulonglong
    lib.lsm_kernel_launches.argtypes = []
    lib.lsm_profile_start.restype = None
    lib.lsm_profile_start.argtypes = []
    lib.lsm_profile_start_classes.restype = None
    lib.lsm_profile_start_classes.argtypes = [ctypes.c_uint]
    lib.lsm_profile_stop.restype = ctypes.c_int
    lib.lsm_profile_stop.argtypes = [ctypes.POINTER(lsm_profile)]
    lib.lsm_check_bounded_wait.restype = ctypes.c_int
    lib.lsm_check_bounded_wait.argtypes = [ctypes.c_void_p]
    lib.lsm_measure_fp32_peak.restype = ctypes.c_int
    lib.lsm_measure_fp32_peak.argtypes = [ctypes.POINTER(ctypes.c_double), ctypes.POINTER(ctypes.c_double),
                                          ctypes.c_void_p]
    _lib_handle = lib
    return lib


# ------------------------------------------------------------------ argument holders


class Grid:
    def __init__(self, nx: int, nz: int, dx: float, dz: float):
        self.c = lsm_grid(int(nx), int(nz), float(dx), float(dz))


class Geometry:
    """Host geometry: src_ix [ns] and rec_ix [ns][nrec] (None: receivers at every column)."""

    def __init__(self, src_ix, rec_ix=None, nx: int | None = None):
        self.src = np.ascontiguousarray(src_ix, dtype=np.int32)
        ns = int(self.src.shape[0])
        if rec_ix is None:
            if nx is None:
                raise ValueError("nx is needed when rec_ix is None")
            self.rec = None
            nrec = int(nx)
            rec_ptr = ctypes.POINTER(ctypes.c_int)()
        else:
            self.rec = np.ascontiguousarray(rec_ix, dtype=np.int32)
            nrec = int(self.rec.shape[1])
            rec_ptr = self.rec.ctypes.data_as(ctypes.POINTER(ctypes.c_int))
        self.c = lsm_geom(ns, self.src.ctypes.data_as(ctypes.POINTER(ctypes.c_int)), nrec, rec_ptr)


class Frequencies:
    """Host frequency axis (Hz) and complex source spectrum."""

    def __init__(self, freq_hz, wavelet):
        self.f = np.ascontiguousarray(freq_hz, dtype=np.float32)
        self.w = np.ascontiguousarray(np.asarray(wavelet, dtype=np.complex64).view(np.float32))
        self.c = lsm_freqs(int(self.f.shape[0]), self.f.ctypes.data_as(ctypes.POINTER(ctypes.c_float)),
                           self.w.ctypes.data_as(ctypes.POINTER(ctypes.c_float)))


def _ptr(x) -> int:
    if x is None:
        return 0
    if isinstance(x, int):
        return x
    return int(x.data_ptr())


def _stream(stream) -> int:
    if stream is None:
        import torch
        return int(torch.cuda.current_stream().cuda_stream)
    if isinstance(stream, int):
        return stream
    return int(stream.cuda_stream)


def _nbytes(ws) -> int:
    if ws is None:
        return 0
    return int(ws.numel() * ws.element_size())


def _check(status: int, where: str):
    if status != LSM_OK:
        raise LsmError(status, where)


# ------------------------------------------------------------------ entry points (C names)


def lsm_status_string(status: int) -> str:
    return load_library().lsm_status_string(int(status)).decode()


def lsm_kernel_launches() -> int:
    return int(load_library().lsm_kernel_launches())


def lsm_profile_start(classes=None) -> None:
    """Start per-launch CUDA-event timing of the kernels the library launches: every class, or
    only the named ones (names from KERNEL_CLASSES), leaving the others without event records."""
    if classes is None:
        load_library().lsm_profile_start()
    else:
        mask = 0
        for name in classes:
            mask |= 1 << KERNEL_CLASSES.index(name)
        load_library().lsm_profile_start_classes(ctypes.c_uint(mask))


def lsm_profile_stop() -> dict:
    """Stop timing; returns {class: {"launches": n, "ms": total}} for each kernel class."""
    prof = lsm_profile()
    _check(load_library().lsm_profile_stop(ctypes.byref(prof)), "lsm_profile_stop")
    return {name: {"launches": int(prof.launches[i]), "ms": float(prof.ms[i])}
            for i, name in enumerate(KERNEL_CLASSES)}


def lsm_measure_fp32_peak(stream=None) -> dict:
    """Measured FP32 FMA throughput of the current device in TFLOP/s: {"ffma": scalar FMA
    instructions, "ffma2": paired FP32 FMA instructions} (see include/lsm.h)."""
    a, b = ctypes.c_double(), ctypes.c_double()
    _check(load_library().lsm_measure_fp32_peak(ctypes.byref(a), ctypes.byref(b), _stream(stream)),
           "lsm_measure_fp32_peak")
    return {"ffma": float(a.value), "ffma2": float(b.value)}


def lsm_check_bounded_wait(stream=None) -> int:
    """Run the bounded-wait self-check (see include/lsm.h); returns its status code, LSM_ERR_TIMEOUT
    being the expected one."""
    return int(load_library().lsm_check_bounded_wait(_stream(stream)))


def lsm_num_windows(ns: int, K: int, slide: int) -> int:
    return int(load_library().lsm_num_windows(int(ns), int(K), int(slide)))


def lsm_workspace_bytes(grid: Grid, geom: Geometry, freqs: Frequencies, nshots: int, op: int) -> int:
    return int(load_library().lsm_workspace_bytes(ctypes.byref(grid.c), ctypes.byref(geom.c),
                                                  ctypes.byref(freqs.c), int(nshots), int(op)))


def lsm_forward(grid, slowness, freqs, geom, m, d_out, shot0, nshots, workspace, stream=None, transform="fft"):
    """d_out[nshots][nw][nrec] (complex64) = A m for shots shot0 .. shot0+nshots-1.

    transform: "fft" (FP32 register FFTs) or a tensor-core precision variant ("dft_bf16x3",
    "dft_fp16x3", "dft_bf16x1"; every supported nx, receivers at every column)."""
    lib = load_library()
    args = (ctypes.byref(grid.c), _ptr(slowness), ctypes.byref(freqs.c), ctypes.byref(geom.c), _ptr(m), _ptr(d_out),
            int(shot0), int(nshots), _ptr(workspace), _nbytes(workspace), _stream(stream))
    if transform == "fft":
        st = lib.lsm_forward(*args)
    else:
        st = lib.lsm_forward_ex(*args, ctypes.byref(_options(transform=transform)))
    _check(st, "lsm_forward")


def lsm_adjoint(grid, slowness, freqs, geom, d, m_out, shot0, nshots, workspace, accumulate=False,
                stream=None, transform="fft"):
    """m_out[nz][nx] (=, or += when accumulate) A^T d for shots shot0 .. shot0+nshots-1."""
    lib = load_library()
    args = (ctypes.byref(grid.c), _ptr(slowness), ctypes.byref(freqs.c), ctypes.byref(geom.c), _ptr(d), _ptr(m_out),
            int(shot0), int(nshots), 1 if accumulate else 0, _ptr(workspace), _nbytes(workspace), _stream(stream))
    if transform == "fft":
        st = lib.lsm_adjoint(*args)
    else:
        st = lib.lsm_adjoint_ex(*args, ctypes.byref(_options(transform=transform)))
    _check(st, "lsm_adjoint")


def lsm_adjoint_static(grid, slowness, freqs, geom, d, m_out, shot0, nshots, accumulate=False, stream=None):
    """A^T d like lsm_adjoint, but with the library's fixed static device scratch instead of a
    workspace, for callers that cannot allocate device memory (see include/lsm.h)."""
    st = load_library().lsm_adjoint_static(ctypes.byref(grid.c), _ptr(slowness), ctypes.byref(freqs.c),
                                           ctypes.byref(geom.c), _ptr(d), _ptr(m_out), int(shot0), int(nshots),
                                           1 if accumulate else 0, _stream(stream))
    _check(st, "lsm_adjoint_static")


def lsm_born_gradient(grid, slowness, sref, freqs, geom, m, g, d_out, grad_m, grad_s, shot0, nshots, workspace,
                      stream=None):
    """Model d = A(s) m (g None) or the gradients dL/dm, dL/ds with s_ref held fixed (see include/lsm.h)."""
    st = load_library().lsm_born_gradient(ctypes.byref(grid.c), _ptr(slowness), _ptr(sref), ctypes.byref(freqs.c),
                                          ctypes.byref(geom.c), _ptr(m), _ptr(g), _ptr(d_out), _ptr(grad_m),
                                          _ptr(grad_s), int(shot0), int(nshots), _ptr(workspace), _nbytes(workspace),
                                          _stream(stream))
    _check(st, "lsm_born_gradient")


def rls_window_solve(grid, slowness, freqs, geom, d, lam, K, slide, cg_tol, max_iter, m_inout, workspace,
                     first_window=0, n_windows=0, stream=None, raise_on_breakdown=True, preconditioner=None,
                     precond_eps=1e-2, transform="fft", cuda_graph=None):
    """Sliding-window CG solve; returns (status, [stats dicts]).  m_inout is updated in place.

    With the defaults this calls rls_window_solve; otherwise rls_window_solve_ex with the options:
    preconditioner="illumination" (diagonal source-illumination preconditioner, stabiliser
    precond_eps times its maximum), a tensor-core `transform`, or cuda_graph=True / "solve" / False
    (each window's CG iterations replayed as one CUDA graph with a device-side stopping test, the
    whole solve as one graph launch, or the host-driven loop; None: the per-window graph unless the
    A / A^T sweeps are being event-timed).
    """
    lib = load_library()
    nwin = lib.lsm_num_windows(int(geom.c.ns), int(K), int(slide))
    cap = max(nwin, 1)
    stats = (lsm_window_stats * cap)()
    args = (ctypes.byref(grid.c), _ptr(slowness), ctypes.byref(freqs.c), ctypes.byref(geom.c), _ptr(d), float(lam),
            int(K), int(slide), float(cg_tol), int(max_iter), int(first_window), int(n_windows), _ptr(m_inout), stats,
            cap, _ptr(workspace), _nbytes(workspace), _stream(stream))
    if preconditioner is None and transform == "fft" and cuda_graph is None:
        st = lib.rls_window_solve(*args)
    else:
        opts = _options(preconditioner, precond_eps, transform, cuda_graph)
        st = lib.rls_window_solve_ex(*args, ctypes.byref(opts))
    last = nwin if n_windows <= 0 else min(nwin, first_window + n_windows)
    out = [stats[i].as_dict() for i in range(max(0, last - first_window))]
    if st != LSM_OK and (st != LSM_ERR_BREAKDOWN or raise_on_breakdown):
        raise LsmError(st, "rls_window_solve")
    return st, out


def rls_window_solve_sharded(grid, slowness, freqs, geom, d, lam, K, slide, cg_tol, max_iter, m_inout, workspace,
                             allreduce, first_window=0, n_windows=0, stream=None, raise_on_breakdown=True):
    """This rank's share of a sliding-window solve sharded by frequency (see include/lsm.h): `freqs`
    and `d` hold this rank's frequencies.  `allreduce(buf, count, is_double, stream)` must replace the
    `count` float32 / float64 values at device address `buf` by their sum over the ranks, ordered on
    the CUDA stream `stream` (integer handles).  Returns (status, [stats dicts])."""
    lib = load_library()
    nwin = lib.lsm_num_windows(int(geom.c.ns), int(K), int(slide))
    cap = max(nwin, 1)
    stats = (lsm_window_stats * cap)()
    failures = []

    def hook(_ctx, buf, count, is_double, st):
        try:
            allreduce(int(buf or 0), int(count), int(is_double), int(st or 0))
            return 0
        except Exception as exc:  # reported after the call; the library stops the solve
            failures.append(exc)
            return 1

    cb = ALLREDUCE_FN(hook)
    st = lib.rls_window_solve_sharded(ctypes.byref(grid.c), _ptr(slowness), ctypes.byref(freqs.c),
                                      ctypes.byref(geom.c), _ptr(d), float(lam), int(K), int(slide), float(cg_tol),
                                      int(max_iter), int(first_window), int(n_windows), _ptr(m_inout), stats, cap,
                                      _ptr(workspace), _nbytes(workspace), _stream(stream), cb, None)
    if failures:
        raise RuntimeError("allreduce callback failed") from failures[0]
    last = nwin if n_windows <= 0 else min(nwin, first_window + n_windows)
    out = [stats[i].as_dict() for i in range(max(0, last - first_window))]
    if st != LSM_OK and (st != LSM_ERR_BREAKDOWN or raise_on_breakdown):
        raise LsmError(st, "rls_window_solve_sharded")
    return st, out


class LineProblem:
    """One survey line for rls_multi_line_solve: argument holders, device tensors and a stream."""

    def __init__(self, grid, slowness, freqs, geom, d, lam, K, slide, cg_tol, max_iter, m_inout, workspace, stream):
        self.grid, self.slowness, self.freqs, self.geom = grid, slowness, freqs, geom
        self.d, self.lam, self.K, self.slide = d, lam, K, slide
        self.cg_tol, self.max_iter, self.m_inout, self.workspace, self.stream = cg_tol, max_iter, m_inout, workspace, stream


def rls_multi_line_solve(problems, preconditioner=None, precond_eps=1e-2, raise_on_error=True, transform="fft",
                         cuda_graph=None):
    """Solve several LineProblems concurrently; returns ([status], [[stats dicts]]).  cuda_graph="solve"
    runs every window of every line as one graph launch instead of one host worker per line."""
    lib = load_library()
    n = len(problems)
    arr = (lsm_line * n)()
    keep = []
    for i, pr in enumerate(problems):
        nwin = max(lib.lsm_num_windows(int(pr.geom.c.ns), int(pr.K), int(pr.slide)), 1)
        stats = (lsm_window_stats * nwin)()
        keep.append((stats, nwin))
        arr[i] = lsm_line(pr.grid.c, _ptr(pr.slowness), pr.freqs.c, pr.geom.c, _ptr(pr.d), float(pr.lam), int(pr.K),
                          int(pr.slide), float(pr.cg_tol), int(pr.max_iter), _ptr(pr.m_inout),
                          ctypes.cast(stats, ctypes.POINTER(lsm_window_stats)), nwin, _ptr(pr.workspace),
                          _nbytes(pr.workspace), _stream(pr.stream), 0)
    opts = ctypes.byref(_options(preconditioner, precond_eps, transform, cuda_graph))
    st = lib.rls_multi_line_solve(arr, n, opts)
    statuses = [int(arr[i].status) for i in range(n)]
    out = [[keep[i][0][k].as_dict() for k in range(keep[i][1])] for i in range(n)]
    if st != LSM_OK and raise_on_error:
        raise LsmError(st, "rls_multi_line_solve")
    return statuses, out


def lsm_autotune(grid, slowness, freqs, geom, nshots, workspace, stream=None, transform="fft") -> dict:
    """Time every admissible FFT tile and launch shape of the source, A^T and A sweeps for launches over
    `nshots` shots and record the fastest for later calls (see include/lsm.h).  `workspace` must hold
    lsm_workspace_bytes(..., nshots, LSM_OP_SOLVE).  Returns {sweep: {warps, heuristic_warps,
    candidates, ms, heuristic_ms}} for the chosen tile, and "tile": {points_per_thread,
    default_points_per_thread, tiles, a_plus_at_ms, default_a_plus_at_ms}."""
    rep = lsm_tune_report()
    st = load_library().lsm_autotune(ctypes.byref(grid.c), _ptr(slowness), ctypes.byref(freqs.c),
                                      ctypes.byref(geom.c), int(nshots), ctypes.byref(_options(transform=transform)),
                                      _ptr(workspace), _nbytes(workspace), _stream(stream), ctypes.byref(rep))
    _check(st, "lsm_autotune")
    return {"source": rep.source.as_dict(), "adjoint": rep.adjoint.as_dict(), "forward": rep.forward.as_dict(),
            "tile": {"points_per_thread": int(rep.points_per_thread),
                     "default_points_per_thread": int(rep.default_points_per_thread), "tiles": int(rep.tiles),
                     "a_plus_at_ms": float(rep.tile_ms), "default_a_plus_at_ms": float(rep.default_tile_ms)}}


def lsm_autotune_gradient(grid, slowness, freqs, geom, nshots, workspace, stream=None) -> dict:
    """Time lsm_born_gradient's kernel at each candidate checkpoint stride and warps per block for
    launches over `nshots` shots and record the fastest pair for later calls (see include/lsm.h).
    `workspace` must hold lsm_workspace_bytes(..., nshots, LSM_OP_GRADIENT).  Returns {stride,
    default_stride, warps, default_warps, candidates, ms, default_ms}."""
    rep = lsm_ckpt_tune_report()
    st = load_library().lsm_autotune_gradient(ctypes.byref(grid.c), _ptr(slowness), ctypes.byref(freqs.c),
                                               ctypes.byref(geom.c), int(nshots), _ptr(workspace),
                                               _nbytes(workspace), _stream(stream), ctypes.byref(rep))
    _check(st, "lsm_autotune_gradient")
    return {"stride": int(rep.stride), "default_stride": int(rep.default_stride), "warps": int(rep.warps),
            "default_warps": int(rep.default_warps), "candidates": int(rep.candidates), "ms": float(rep.ms),
            "default_ms": float(rep.default_ms)}


def lsm_fft_tiles(nx: int) -> list:
    """The FFT tiles (points per thread) compiled for width nx, the default first."""
    buf = (ctypes.c_int * 2)()
    n = load_library().lsm_fft_tiles(int(nx), buf, 2)
    return [int(buf[i]) for i in range(min(n, 2))]


def lsm_tcgen05_shape(nx: int, nshots: int, nw: int) -> dict:
    """Launch shape of the tcgen05 transform variants for nshots x nw items of width nx (host only)."""
    v = [ctypes.c_int() for _ in range(4)]
    smem = ctypes.c_size_t()
    _check(load_library().lsm_tcgen05_shape(int(nx), int(nshots), int(nw), *[ctypes.byref(x) for x in v],
                                            ctypes.byref(smem)), "lsm_tcgen05_shape")
    return {"items": v[0].value, "threads": v[1].value, "blocks": v[2].value, "wslots": v[3].value,
            "smem_bytes": int(smem.value)}


def lsm_set_fft_tile(nx: int, nshots: int, nw: int, points_per_thread: int) -> None:
    """Record the FFT tile of calls over `nshots` shots of nx columns and nw frequencies (see
    include/lsm.h), as lsm_autotune would."""
    _check(load_library().lsm_set_fft_tile(int(nx), int(nshots), int(nw), int(points_per_thread)),
           "lsm_set_fft_tile")


def lsm_autotune_reset() -> None:
    """Forget every launch shape recorded by lsm_autotune and every stride recorded by
    lsm_autotune_gradient."""
    load_library().lsm_autotune_reset()
