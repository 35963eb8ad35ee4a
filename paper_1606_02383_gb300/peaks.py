"""Measured compute peaks of this GPU (roofline denominators).

``measure("fp32")`` times packed f32x2 FMA chains and ``measure("tf32")``
back-to-back tcgen05 TF32 MMAs with resident operands, both through the
library's ``bem_peak_probe``.  The 3xTF32 translations run three products per
algorithmic flop, so their algorithmic ceiling is a third of the TF32 rate.
"""
from __future__ import annotations

import ctypes

import torch

from . import _lib

_WHICH = {"fp32": 0, "tf32": 1}
_ITERS = {"fp32": 2000, "tf32": 4000}


def measure(kind: str, iters: int | None = None) -> float:
    """TFLOP/s of the pipe (an FMA counts 2 flops) on the current device and stream."""
    if kind not in _WHICH:
        raise ValueError("kind must be 'fp32' or 'tf32'")
    lib = _lib.load()
    out = ctypes.c_double(0.0)
    n = _ITERS[kind] if iters is None else int(iters)
    rc = lib.bem_peak_probe(_WHICH[kind], n, ctypes.byref(out),
                            ctypes.c_void_p(torch.cuda.current_stream().cuda_stream))
    _lib.check(rc)
    return float(out.value)
