"""The sharded form of the detection increment over torch.distributed ranks.

One usFFT instance on P GPUs (one process per GPU): usfft_increment_sharded splits each coupled
step's lattice nodes by residue (rank p solves the nodes i = p + P i2), runs the rank's
length-M/P lattice FFT with the phase factor of its residue class, and exchanges through a
collective hook -- a sum all-reduce of the G x |J| coefficients and a maximum all-reduce of one
flag byte per candidate (see include/usfft.h).  This module supplies that hook over a
torch.distributed process group (NCCL on GPUs) and a plan wrapper.  Argument marshalling only:
the numeric steps run in the library's kernels, the exchange in torch.distributed.
"""
from __future__ import annotations

import ctypes

import numpy as np

from . import binding

_TYPESTR = {binding.RED_F64: "<f8", binding.RED_U8: "|u1"}
_CTYPE = {binding.RED_F64: ctypes.c_double, binding.RED_U8: ctypes.c_uint8}


class _DeviceBuffer:
    """A device pointer as an object with __cuda_array_interface__ (torch.as_tensor wraps it
    without copying)."""

    def __init__(self, ptr: int, count: int, typestr: str):
        self.__cuda_array_interface__ = {"shape": (int(count),), "typestr": typestr, "data": (int(ptr), False),
                                         "version": 2}


class TorchAllreduce:
    """The collective hook of usfft_increment_sharded over a torch.distributed group.

    on_device=True (the library's calls): buf is a device pointer and the all-reduce is issued
    on the plan's stream.  on_device=False: buf is a host pointer (gloo groups on the CPU).
    `fn` is the ctypes function pointer to hand to the library; keep this object alive while the
    plan may call it (increments and replays)."""

    def __init__(self, group=None, on_device: bool = True):
        self.group = group
        self.on_device = on_device
        self.failures = 0
        self.fn = binding.ALLREDUCE_FN(self._call)

    def _call(self, buf, count, dtype, op, stream, ctx):
        try:
            import torch
            import torch.distributed as dist
            rop = dist.ReduceOp.SUM if op == binding.RED_SUM else dist.ReduceOp.MAX
            if self.on_device:
                t = torch.as_tensor(_DeviceBuffer(buf, count, _TYPESTR[dtype]), device="cuda")
                s = torch.cuda.ExternalStream(stream) if stream else torch.cuda.default_stream()
                with torch.cuda.stream(s):
                    dist.all_reduce(t, op=rop, group=self.group)
            else:
                arr = np.ctypeslib.as_array((_CTYPE[dtype] * int(count)).from_address(int(buf)))
                dist.all_reduce(torch.from_numpy(arr), op=rop, group=self.group)
            return 0
        except Exception:                     # reported to the library as a failed collective
            self.failures += 1
            return 1


class ShardedPlan(binding.Plan):
    """A plan whose increments run as rank `rank` of `nranks` of the sharded form."""

    def __init__(self, problem, params, rank: int, nranks: int, group=None, stream=None):
        super().__init__(problem, params, stream=stream)
        self.rank = int(rank)
        self.nranks = int(nranks)
        self.reducer = TorchAllreduce(group)

    def increment(self) -> dict:
        return binding.usfft_increment_sharded(self, self.rank, self.nranks, self.reducer.fn)
