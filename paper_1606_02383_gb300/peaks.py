"""Measured compute peaks of this GPU (roofline denominators).

``measure("fp32")`` times packed f32x2 FMA chains, ``measure("tf32")`` and
``measure("fp16")`` back-to-back tcgen05 TF32 and FP16 MMAs with resident
operands, all through the library's ``bem_peak_probe``.  The translations run
three products per algorithmic flop (3xTF32 or the FP16 split), so their
algorithmic ceiling is a third of the rate of the form in use.
"""
from __future__ import annotations

import ctypes

import torch

from . import _lib

_WHICH = {"fp32": 0, "tf32": 1, "fp16": 2}
_ITERS = {"fp32": 2000, "tf32": 4000, "fp16": 4000}


def measure(kind: str, iters: int | None = None) -> float:
    """TFLOP/s of the pipe (an FMA counts 2 flops) on the current device and stream."""
    if kind not in _WHICH:
        raise ValueError("kind must be 'fp32', 'tf32' or 'fp16'")
    lib = _lib.load()
    out = ctypes.c_double(0.0)
    n = _ITERS[kind] if iters is None else int(iters)
    rc = lib.bem_peak_probe(_WHICH[kind], n, ctypes.byref(out),
                            ctypes.c_void_p(torch.cuda.current_stream().cuda_stream))
    _lib.check(rc)
    return float(out.value)
