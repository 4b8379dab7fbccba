"""Helpers for the frequency-sharded window solve (rls_window_solve_sharded).

A window's (shot, frequency) items are independent inside A and A^T, so N ranks can each take a
contiguous block of the frequency axis; the only exchanges are the sums over the ranks of the A^T
images and of ||q||^2, which the library asks for through a callback.  `torch_allreduce` builds that
callback on torch.distributed: NCCL reduces the device buffer in place on the library's stream;
a backend without CUDA reductions (gloo) goes through a host copy.
"""

from __future__ import annotations

import ctypes


def frequency_shard(nw: int, rank: int, world: int) -> tuple[int, int]:
    """[start, stop) of this rank's frequencies: contiguous blocks whose sizes differ by at most one,
    the larger ones first."""
    if world < 1 or not 0 <= rank < world or nw < world:
        raise ValueError("need 0 <= rank < world <= nw")
    base, extra = divmod(nw, world)
    start = rank * base + min(rank, extra)
    return start, start + base + (1 if rank < extra else 0)


class _CudaBuffer:
    """A device address seen as a 1-D CUDA array (zero copy) through __cuda_array_interface__."""

    def __init__(self, ptr: int, count: int, typestr: str):
        self.__cuda_array_interface__ = {"shape": (count,), "typestr": typestr, "data": (ptr, False),
                                         "version": 2}


def buffer_tensor(ptr: int, count: int, is_double: int, device: str = "cuda"):
    """A torch tensor viewing `count` float32 / float64 values at `ptr` (device memory, or host memory
    when device is "cpu"), without copying."""
    import numpy as np
    import torch

    if device == "cpu":
        ctype = ctypes.c_double if is_double else ctypes.c_float
        arr = np.ctypeslib.as_array((ctype * count).from_address(ptr))
        return torch.from_numpy(arr)
    return torch.as_tensor(_CudaBuffer(ptr, count, "<f8" if is_double else "<f4"), device=device)


def torch_allreduce(group=None, device: str = "cuda"):
    """The callback rls_window_solve_sharded needs, on the default (or given) torch.distributed group:
    sum the buffer over the ranks in place, ordered on the library's CUDA stream."""
    import torch
    import torch.distributed as dist

    backend = dist.get_backend(group)

    def allreduce(ptr: int, count: int, is_double: int, stream: int) -> None:
        t = buffer_tensor(ptr, count, is_double, device)
        if device == "cpu":
            dist.all_reduce(t, op=dist.ReduceOp.SUM, group=group)
            return
        # the library's stream: 0 is the legacy default stream, which is torch's default stream
        lib_stream = torch.cuda.default_stream() if stream == 0 else torch.cuda.ExternalStream(stream)
        with torch.cuda.stream(lib_stream):
            if backend == "nccl":
                dist.all_reduce(t, op=dist.ReduceOp.SUM, group=group)
            else:
                host = t.cpu()  # waits for the library's work on the stream
                dist.all_reduce(host, op=dist.ReduceOp.SUM, group=group)
                t.copy_(host)

    return allreduce
