"""Measured compute peaks of the GPU pipes that bound the render (libgsrf_peaks.so).

The render's roofline needs the rate of plain FP32 arithmetic and of the special-
function unit (MUFU: ex2, rcp, rsqrt, sqrt, sin, cos), which the copy-bandwidth and
cuBLAS figures of the GPU do not give.  `measure()` times each microbenchmark with CUDA
events on the current stream after one warm-up launch, on a grid that fills every SM
(8 CTAs of 256 threads each), sized to run for a few milliseconds, and returns operations
per second: FP32 and FP64 fused multiply-adds (one operation each; the packed FP32x2
instruction counts its two), special-function results, and TF32 FLOP of the warp-level
mma.sync form (2 per multiply-add).

  python -m paper_2502_01826_gb300.peaks      # prints the figures as JSON
"""
from __future__ import annotations

import ctypes as C
import json
import os

from . import _build

KINDS = ["fma32", "ex2", "rcp", "rsqrt", "sqrt", "sin", "cos", "fma64", "mma_tf32", "fma32x2"]
# issue slots per SM and clock that each kind has on this architecture's SM (4 sub-
# partitions): 128 FP32 lanes; 16 special-function results; used only to express a
# measured rate per SM and clock beside the nominal figure
NOMINAL_PER_SM_CLK = {"fma32": 128, "ex2": 16, "rcp": 16, "rsqrt": 16, "sqrt": 16, "sin": 16, "cos": 16}

_lib = None


def load():
    global _lib
    if _lib is None:
        if not os.path.exists(_build.PEAKS_SO):
            raise RuntimeError("libgsrf_peaks.so not built (%s); call __graft_entry__.build()" % _build.PEAKS_SO)
        L = C.CDLL(_build.PEAKS_SO)
        L.gsrf_peak_launch.argtypes = [C.c_int, C.c_int, C.c_int, C.c_void_p, C.c_void_p]
        L.gsrf_peak_launch.restype = C.c_int
        L.gsrf_peak_ops.argtypes = [C.c_int, C.c_int, C.c_int]
        L.gsrf_peak_ops.restype = C.c_double
        _lib = L
    return _lib


def measure(target_ms: float = 4.0, kinds=None) -> dict:
    """Operations per second of each kind on the current device, with the SM count."""
    import torch

    L = load()
    dev = torch.cuda.current_device()
    sms = torch.cuda.get_device_properties(dev).multi_processor_count
    blocks = sms * 8
    out = torch.empty(blocks * 256, dtype=torch.float32, device="cuda")
    stream = torch.cuda.current_stream()
    sp = C.c_void_p(stream.cuda_stream)
    res = {"sms": sms, "blocks": blocks, "threads_per_block": 256}

    def run(k, iters):
        code = L.gsrf_peak_launch(k, blocks, iters, C.c_void_p(out.data_ptr()), sp)
        if code != 0:
            raise RuntimeError("gsrf_peak_launch(%s) returned %d" % (KINDS[k], code))

    def timed(k, iters, reps=3):
        best = None
        for _ in range(reps):
            a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            a.record(stream)
            run(k, iters)
            b.record(stream)
            b.synchronize()
            ms = a.elapsed_time(b)
            best = ms if best is None else min(best, ms)
        return best

    for name in kinds or KINDS:
        k = KINDS.index(name)
        iters = 4
        run(k, iters)
        ms = timed(k, iters, reps=1)
        while ms < 0.25 * target_ms and iters < (1 << 20):
            iters *= 4
            ms = timed(k, iters, reps=1)
        if ms < 0.25 * target_ms:  # a kind whose work did not run is reported, not used
            res[name] = {"error": "%d rounds ran in %.3g ms" % (iters, ms)}
            continue
        iters = max(1, min(1 << 24, int(iters * target_ms / ms)))
        ms = timed(k, iters)
        ops = L.gsrf_peak_ops(k, blocks, iters)
        res[name] = {"ops_per_s": ops / (ms * 1e-3), "ms": ms, "iters": iters, "ops": ops}
    return res


if __name__ == "__main__":
    print(json.dumps(measure(), indent=1))
